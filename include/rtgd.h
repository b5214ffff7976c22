/*
 * rtgd.h -- C ABI of the GB300 (sm_103a) RTM-GD ray-fan tracer.
 *
 * RTM-GD (arXiv 2506.18579) traces HF rays through a gridded ionosphere: the
 * Haselgrove ray equations in spherical coordinates (Sec. II-A, Eq. 1a-1f)
 * with the cold-plasma Hamiltonian (Eq. 2) and the Appleton-Hartree
 * refractive index without collisions (Eq. 3), where electron density and its
 * gradient come from the C1 Galerkin-Difference p=3 interpolant of the grid
 * samples (Sec. II-B, Eq. 13, Appendix A), integrated by Runge-Kutta until the
 * ray returns to the ground or leaves the ionosphere (Sec. II-C).  Inputs of
 * the paper's problem statement (Sec. II-C): a gridded Ne field plus a
 * geomagnetic field model (preprocessing module), and transmitter position,
 * azimuth, elevation and frequency per ray (main module); outputs: group path,
 * ground distance, azimuth deviation and reflection height.
 *
 * Conventions for every call:
 *   - The return value carries the call status (rt_err).  On any error the
 *     message is available from rt_last_error() on the calling thread.
 *   - Per-ray failures are not call errors; they are reported in
 *     rt_ray_result.status.
 *   - Units: degrees, km, MHz, electrons per m^3, tesla.
 *   - A CUDA GPU is required.  There is no CPU fallback: without a usable
 *     device every call returns RT_EUNSUPPORTED or RT_ECUDA.
 *   - "stream" arguments are cudaStream_t values passed as void*; NULL means
 *     the legacy default stream.
 *   - Grid handles are immutable after creation and may be used from several
 *     threads and streams at once; rt_grid_destroy must not race with them.
 */
#ifndef RTGD_H
#define RTGD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTGD_API_VERSION 2

typedef enum rt_err {
    RT_OK = 0,
    RT_EINVAL = 1,       /* bad argument: null pointer, bad size, bad descriptor field */
    RT_ENOMEM = 2,       /* device or host allocation failed */
    RT_ECUDA = 3,        /* a CUDA runtime call failed */
    RT_ETIMEOUT = 4,     /* a bounded wait expired */
    RT_EUNSUPPORTED = 5  /* no usable CUDA device, or a feature this build lacks */
} rt_err;

/* Sample type of the Ne array handed to rt_grid_create. */
enum { RT_F32 = 0, RT_F64 = 1 };

/* rt_grid_desc.flags */
enum {
    RT_GRID_TABLE = 1u,       /* also build the per-cell stencil table (64 FP32 values per
                                 cell, Sec. II-C "weights computed once per grid cell") */
    RT_GRID_CATMULL_ROM = 2u  /* interpolate with the Catmull-Rom spline of Sec. II-B-1
                                 (Eq. 6-9), the paper's comparison scheme, instead of GD */
};

/* Centred tilted dipole standing in for the geomagnetic model (Sec. II-C):
 * B = -B0 (R_E/r)^3 [3 (m.p) p - m], m = unit vector to the geomagnetic north
 * pole at (pole_lat_deg, pole_lon_deg).  b0_tesla = 0 gives an isotropic
 * medium (no field; O and X modes coincide). */
typedef struct rt_dipole {
    double b0_tesla;
    double pole_lat_deg;
    double pole_lon_deg;
} rt_dipole;

/* Uniform geographic grid (Sec. II-B, Eq. 12-13).  Sample (i, j, k) sits at
 * lat0 + i*dlat, lon0 + j*dlon, alt0 + k*dalt; the host array is laid out
 * [lat][lon][alt] with alt fastest.  Each dimension needs >= 4 nodes. */
typedef struct rt_grid_desc {
    int32_t n_lat, n_lon, n_alt;
    int32_t dtype;              /* RT_F32 or RT_F64 */
    double lat0_deg, lon0_deg, alt0_km;
    double dlat_deg, dlon_deg, dalt_km;
    double earth_radius_km;     /* e.g. 6371 */
    rt_dipole field;
    uint32_t flags;             /* RT_GRID_* */
    uint32_t reserved;          /* must be 0 */
} rt_grid_desc;

typedef struct rt_grid rt_grid;  /* opaque; owned by the library until rt_grid_destroy */

/* Create a device-resident grid (Sec. II-C preprocessing module).  ne_host
 * points to n_lat*n_lon*n_alt samples of the given dtype in host memory; they
 * are copied (the caller keeps ownership).  The library pads the grid with one
 * ghost layer per face (quadratic extrapolation, so quadratics stay exact up
 * to the faces), converts it to the layouts the kernels read and, with
 * RT_GRID_TABLE, builds the per-cell stencil table.  Blocks until done.
 * Errors: RT_EINVAL (null pointer, dims < 4, non-positive spacing or radius,
 * unknown dtype/flags), RT_ENOMEM, RT_ECUDA, RT_EUNSUPPORTED (no device). */
rt_err rt_grid_create(const rt_grid_desc *desc, const void *ne_host, rt_grid **out);

/* Release a grid and its device memory.  NULL is accepted.  Must not be called
 * while work that uses the grid is still queued on any stream. */
rt_err rt_grid_destroy(rt_grid *grid);

/* Bytes of device memory the grid holds. */
size_t rt_grid_device_bytes(const rt_grid *grid);

/* Ray modes (bit mask), integrators, precisions. */
enum { RT_MODE_O = 1u, RT_MODE_X = 2u };
enum { RT_RK4 = 0, RT_RKF45 = 1 };
enum {
    RT_FP64 = 0,  /* every step of the path in double precision */
    RT_MIXED = 1  /* interpolation, Appleton-Hartree and derivatives in FP32; the ray's
                     position and its RK accumulation, the group path and the landing /
                     exit solve in FP64; the wave vector as a compensated pair of floats */
};

/* A fan of rays (Sec. II-C main module): every combination of frequency,
 * mode, elevation and azimuth from one transmitter.  Ray results are ordered
 * canonically as [freq][mode][el][az] (ordinary before extraordinary when
 * both modes are set).  The three arrays are host memory, read during the
 * call only.
 *   integrator RT_RK4: fixed step h_km in group path P' (Sec. II-C).
 *   integrator RT_RKF45: Fehlberg 4(5) with initial step h_km; the step is
 *     accepted when err <= 1 with err = max(pos_err / (atol_km + rtol * r),
 *     k_err / (rtol * max(|k|, 1e-3))), pos_err = max(|dr|, r|dtheta|,
 *     r sin(theta)|dphi|) and k_err = max|dk_i| (k in units of omega/c),
 *     the error estimate being h * sum((b5_i - b4_i) k_i).  The nominal
 *     step h changes only by its quantised factor q = 2^(floor(4 log2(f))/4),
 *     f = min(5, max(0.2, 0.9 err^-0.2)): h *= q after a rejection or an
 *     accepted step, clamped to [h_min_km, h_max_km]; a rejected step below
 *     h_min_km stops the ray.  An attempt whose step would cross a cell face
 *     of the interpolant (where its second derivatives jump), predicted
 *     linearly from dy/dP' at the step start, is shortened to end 1e-4 of
 *     its length past that face; such a step never enlarges h (q <= 1).
 *     Both rules keep the step sequence a function of discrete decisions,
 *     so round-off cannot steer it.
 *   max_steps bounds the RK step attempts of one ray (rejected steps and
 *     landing-solve trial steps included).
 *   max_group_path_km > 0 stops the ray at exactly that group path. */
typedef struct rt_fan_desc {
    double tx_lat_deg, tx_lon_deg, tx_alt_km;
    const double *freq_mhz;     /* n_freq values > 0 */
    const double *el_deg;       /* n_el values, elevation above the local horizontal */
    const double *az_deg;       /* n_az values, clockwise from geographic north */
    int32_t n_freq, n_el, n_az;
    uint32_t modes;             /* RT_MODE_O | RT_MODE_X */
    int32_t integrator;         /* RT_RK4 or RT_RKF45 */
    int32_t precision;          /* RT_FP64 or RT_MIXED */
    double h_km, rtol, atol_km, h_min_km, h_max_km;
    int32_t max_steps;
    int32_t reserved;           /* must be 0 */
    double max_group_path_km;   /* <= 0: unlimited */
} rt_fan_desc;

/* Per-ray status. */
enum {
    RT_RAY_NOT_RUN = 0,
    RT_RAY_LANDED = 1,         /* returned to r = R_E (landing point solved to |r - R_E| < 1e-9 km
                                  on the FP64 path, 1e-5 km on the mixed path) */
    RT_RAY_ESCAPED = 2,        /* left through the top of the grid (exit point solved like landing) */
    RT_RAY_LEFT_GRID = 3,      /* left the grid sideways inside its altitude span */
    RT_RAY_MAX_STEPS = 4,      /* max_steps attempts used */
    RT_RAY_STEP_UNDERFLOW = 5, /* RKF45 needed a step below h_min_km */
    RT_RAY_NONFINITE = 6,      /* non-finite state, or mu^2 <= 0 at the transmitter */
    RT_RAY_MAX_PATH = 7        /* reached max_group_path_km */
};

/* Per-ray result (64 bytes).  Quantities refer to the final state: the
 * landing point for LANDED rays, the exit point on the grid top for ESCAPED
 * rays (both solved on the last step), the last accepted state otherwise.
 * ground_range_km = R_E times the central angle from the transmitter;
 * az_dev_deg = bearing of the final point from the transmitter minus the
 * launch azimuth, in [-180, 180); apogee_km = the reflection height (maximum
 * altitude, refined by a cubic Hermite fit where dr/dP' changes sign). */
typedef struct rt_ray_result {
    double group_path_km;
    double ground_range_km;
    double az_dev_deg;
    double apogee_km;
    double land_lat_deg;
    double land_lon_deg;        /* in [-180, 180) */
    int32_t status;             /* RT_RAY_* */
    int32_t n_steps;            /* accepted steps (the final landing step included) */
    int32_t n_attempts;         /* all RK step attempts: accepted + rejected + landing trials */
    int32_t n_evals;            /* right-hand-side (stage) evaluations, the launch one included */
} rt_ray_result;

/* Number of rays a fan expands to (0 on an invalid descriptor). */
size_t rt_fan_size(const rt_fan_desc *fan);

/* Kernel choices.  Zero-initialise for the library's defaults. */
enum { RT_KERNEL_AUTO = 0, RT_KERNEL_PLAIN = 1, RT_KERNEL_PERSISTENT = 2 };
enum { RT_STENCIL_AUTO = 0, RT_STENCIL_GATHER = 1, RT_STENCIL_QUAD = 2, RT_STENCIL_TABLE = 3 };
enum { RT_ORDER_CANONICAL = 0, RT_ORDER_ELEVATION_FASTEST = 1 };
typedef struct rt_launch_config {
    int32_t kernel;        /* RT_KERNEL_*: PLAIN = one lane group per ray, one launch-wide grid of
                              groups (the default); PERSISTENT = one resident grid whose lane
                              groups claim rays from an atomic counter (mixed only) */
    int32_t stencil;       /* RT_STENCIL_*: where the mixed path reads the 4x4x4 samples:
                              GATHER = padded FP32 grid, QUAD = 4 consecutive altitude samples
                              per float4, TABLE = per-cell table (needs RT_GRID_TABLE) */
    int32_t block_threads; /* 0 = default (128); a multiple of 32 in [32, 128] */
    int32_t order;         /* RT_ORDER_*: order in which rays are handed to lane groups (both
                              kernels); ELEVATION_FASTEST keeps neighbouring elevations of one
                              azimuth in one warp (similar paths, nearby cells) */
    int32_t blocks_per_sm; /* persistent kernel: resident blocks per SM (0 = occupancy limit) */
    int32_t lanes_per_ray; /* mixed path: 1, 2 or 4 lanes share one ray (they split the 16 sample
                              rows of every stage; 32 / lanes rays per warp); 0 = chosen from the
                              fan size (more lanes per ray when the fan cannot fill the GPU) */
    int32_t reserved[2];
} rt_launch_config;

/* Trace a fan; blocking.  out_host receives rt_fan_size(fan) results in
 * canonical order (out_len must be at least that).  The call copies the fan
 * arrays to the device, runs the kernels on `stream`, copies the results back
 * and synchronises the stream.  cfg may be NULL (defaults).  Device scratch
 * (fan tables, result staging, the persistent kernel's ray counter) is
 * allocated stream-ordered and released stream-ordered.
 * The wait for the trace is bounded: RTGD_SYNC_TIMEOUT_S seconds (environment
 * variable, read at every call; default 900).  When it expires the call
 * returns RT_ETIMEOUT with the trace still queued or running on `stream`
 * (and its scratch released after it, stream-ordered); out_host is left
 * untouched and is not written later, because the copy of the records is
 * queued only after the trace has finished (that copy is then waited for
 * without a deadline).  On every return the caller owns out_host again.
 * Errors: RT_EINVAL (null pointers, empty or invalid fan, out_len too small,
 * bad cfg), RT_ENOMEM, RT_ECUDA, RT_ETIMEOUT, RT_EUNSUPPORTED. */
rt_err rt_trace(const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_host,
                size_t out_len, const rt_launch_config *cfg, void *stream);

/* Same as rt_trace but asynchronous: out_dev is device memory (e.g. a PyTorch
 * CUDA tensor) of at least rt_fan_size(fan) records; the call returns once the
 * work is queued on `stream`.  The fan arrays are copied into library memory
 * before return (pinned or pageable), so the caller may reuse them at once. */
rt_err rt_trace_device(const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_dev,
                       size_t out_len, const rt_launch_config *cfg, void *stream);

/* Several fans on one grid in one launch (e.g. the fans of several
 * transmitters, or many small requests): fans[0..n_fans-1] (1 <= n_fans <=
 * 4096), all RT_MIXED and with one integrator.  out_dev (device memory) receives
 * their records fan after fan: fan k's rt_fan_size(fans[k]) records start
 * after those of fans 0..k-1, each fan in its own canonical order; out_len
 * must cover them all.  The launch runs four lanes per ray with cfg's
 * stencil, block size and ray order (cfg->kernel must be AUTO or PLAIN and
 * cfg->lanes_per_ray 0 or 4; cfg may be NULL).  A fan's records do not
 * depend on the other fans of the launch.  They equal those of
 * rt_trace_device with four lanes per ray on the plain kernel up to float
 * rounding, because the two kernels are compiled apart.  This is the
 * kernel a request server with fuse_max_rays > 0 runs for small requests.
 * Worth it for fans that each leave the GPU mostly idle (up to a quarter of
 * its resident lanes).  Asynchronous like rt_trace_device: the fan arrays
 * are read before return; scratch is allocated and released stream-ordered.
 * Errors: RT_EINVAL (null pointers, n_fans out of range, an invalid or FP64
 * fan, mixed integrators, out_len too small, a grid on another device, bad
 * cfg), RT_ENOMEM, RT_ECUDA, RT_EUNSUPPORTED. */
rt_err rt_trace_fans_device(const rt_grid *grid, const rt_fan_desc *const *fans, int32_t n_fans,
                            rt_ray_result *out_dev, size_t out_len, const rt_launch_config *cfg,
                            void *stream);

/* Same as rt_trace_device, for callers that cannot allocate device memory
 * while they trace (an allocator that must not be re-entered, a fixed device
 * memory budget, device memory owned by another runtime).  This call makes no
 * cudaMalloc/cudaFree (or other allocating) call: its scratch -- the ray
 * counter and the fan tables -- is a fixed array inside the library (16 bytes
 * + 3 x 4096 doubles, about 96 KiB, held on every GPU that loads the library
 * until the process exits), filled from a fixed host staging array of the
 * same size.
 * The paper has no counterpart; it is an interface variant of
 * rt_trace_device.  Limits and rules:
 *   - n_freq + n_el + n_az must not exceed 4096 (RT_EINVAL otherwise).
 *   - All calls share the scratch: work queued by one call must be finished
 *     on the GPU before another call's work starts (calls that overlap on the
 *     GPU, e.g. on two streams, race and give wrong results).  Every call
 *     resets the ray counter and rewrites the tables it uses.
 *   - The first call on a device looks up the scratch's device address (a
 *     runtime query, once per device); make that first call before any stream
 *     capture begins on the device.
 *   - The fan arrays are copied before return, as in rt_trace_device.
 * Results, errors and stream semantics are those of rt_trace_device. */
rt_err rt_trace_device_noalloc(const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_dev,
                               size_t out_len, const rt_launch_config *cfg, void *stream);

/* Autotuner: times the candidate launch configurations (kernel x stencil x
 * claim order x lanes per ray x 32, 64, 96 or 128 threads per block) for this grid
 * and fan shape on `stream`, each candidate on a strided sub-fan of at most
 * max_rays rays (0 = 65536; one warm-up and three timed launches each,
 * every timed launch after a 256 MiB fill that evicts L2), then the four
 * with the lowest median again in seven interleaved rounds, and returns the
 * one with the lowest median of those seven in *best and that time in
 * *best_ms.  A fan of at least two waves of
 * resident lanes at one lane per ray is issue-bound: it tries one lane per
 * ray only, on a sub-fan of at least four such waves (a smaller sub-fan would
 * reward the latency of its slowest rays instead).  Blocking.  Uses
 * stream-ordered scratch: the sub-fan's records and the fill buffer
 * (RT_ENOMEM without them).  Results are also cached inside the library,
 * keyed by grid, integrator and fan size, and used by later calls whose
 * kernel and stencil are both AUTO; rt_grid_destroy drops them. */
rt_err rt_tune(const rt_grid *grid, const rt_fan_desc *fan, size_t max_rays, void *stream,
               rt_launch_config *best, float *best_ms);

/* ------------------------------------------------------------------ plans */
/* A plan binds a grid, a fan and a launch configuration once: the fan tables
 * and the ray counter live in device memory owned by the plan (allocated by
 * rt_plan_create), so rt_plan_execute only resets the counter and launches
 * the trace kernel -- two stream operations that can be captured into a CUDA
 * graph and replayed.  The grid must outlive the plan.
 * Errors: as rt_trace_device; rt_plan_execute also RT_EINVAL on NULL. */
typedef struct rt_plan rt_plan;
rt_err rt_plan_create(const rt_grid *grid, const rt_fan_desc *fan, const rt_launch_config *cfg,
                      rt_plan **out);
size_t rt_plan_rays(const rt_plan *plan);
rt_err rt_plan_execute(const rt_plan *plan, rt_ray_result *out_dev, size_t out_len, void *stream);
rt_err rt_plan_destroy(rt_plan *plan);

/* Longest-first order for a plan (batched uneven fans; the paper has no
 * counterpart: it traces one scan at a time on a CPU).  A batch of uneven
 * rays lasts as long as its most expensive rays take one after the other; this
 * call lets a plan start those first and give them more lanes.
 *   cost_dev: device records of an earlier trace of a fan of the same shape
 *     (rt_plan_rays(plan) records, canonical order): the plan's previous
 *     execution, or the same scan on the previous ionosphere snapshot.  A
 *     ray's expected cost is the largest n_evals within `spread` (0..64)
 *     elevation and frequency steps of it (same mode and azimuth) in those
 *     records, so that a boundary that moved a few steps between snapshots
 *     keeps its rays marked expensive.  NULL: back to the plan's own order.
 *   long_factor > 0 (mixed-precision plans): rays whose expected cost is at
 *     least long_factor times the median (at most a sixteenth of the rays)
 *     are traced at four lanes per ray by a plain launch of their own, on a
 *     second, high-priority stream forked from and joined back to the
 *     execute call's stream, in the plan's own claim order (neighbouring
 *     rays of a trace share a warp); *n_long (may be NULL) receives their
 *     number.
 *   flags: by default the other rays are handed out in descending order of
 *     expected cost as well (rays of costs within 2^(1/8) of each other keep
 *     their canonical order); RT_PLAN_REST_IN_PLAN_ORDER keeps the plan's own
 *     claim order for them.  RT_PLAN_LONG_EXCLUSIVE makes the four-lane
 *     launch's blocks two warps wide and gives each an SM of its own (the
 *     block reserves the SM's whole shared memory, so no other block is
 *     resident beside it): its rays then run at the latency of a lone warp
 *     instead of sharing issue slots with the rest of the scan, and the other
 *     rays have that many SMs fewer.  The share is then cut to at most an
 *     eighth of the SM count in blocks (its most expensive rays), and the
 *     other rays' launch waits until all of its blocks have begun (a
 *     launch-completion event; the runtime documents it as best effort).
 *     RT_PLAN_LONG_ALONE gives each ray of the four-lane launch a warp of its
 *     own (by default a warp holds eight of them, which then wait for one
 *     another's branches and gathers at every attempt).
 * rt_plan_execute traces the other rays with the plan's launch
 * configuration.  A ray's record does
 * not depend on the order; rays in the four-lane launch give the records of
 * a four-lane plain trace (their contraction sums in another order).  The
 * execute step stays graph-capturable (the fork and join are stream events).
 * A graph captured from rt_plan_execute holds the launch sizes of the order
 * in effect at capture but reads the claim list from the plan's memory, which
 * the next rt_plan_order call rewrites: after ordering again (or back to
 * NULL), discard such graphs and capture anew (an old graph could then trace
 * some rays twice and skip others).
 * Blocking: gathers the costs on the device (into an array the plan then
 * keeps), copies them to the host, sorts and uploads the order (about 4-5 ms
 * of host time for 495,122 rays).  Not concurrent with an execution of the
 * same plan.  Errors: RT_EINVAL,
 * RT_ENOMEM, RT_ECUDA, RT_ETIMEOUT. */
enum { RT_PLAN_REST_IN_PLAN_ORDER = 1u, RT_PLAN_LONG_EXCLUSIVE = 2u, RT_PLAN_LONG_ALONE = 4u };
rt_err rt_plan_order(rt_plan *plan, const rt_ray_result *cost_dev, int32_t spread, double long_factor,
                     uint32_t flags, size_t *n_long, void *stream);

/* The claim list rt_plan_order builds, from host costs; host arithmetic only
 * (no GPU call, usable without a device).
 *   cost: n = n_freq * n_modes * n_el * n_az costs (stage evaluations) of an
 *     earlier trace, canonical order [freq][mode][el][az], caller-owned.
 *   claim_order: the plan's claim order (RT_ORDER_CANONICAL or
 *     RT_ORDER_ELEVATION_FASTEST); spread, long_factor, flags: as in
 *     rt_plan_order; mixed: nonzero for a mixed-precision plan (only those
 *     take a four-lane share); sm_count: the device's SM count (used with
 *     RT_PLAN_LONG_EXCLUSIVE).
 *   claims (out, caller-owned, claims_cap entries): canonical ray indices in
 *     claim order, -1 for a hole; the first entries, *n_long rays (each with
 *     seven holes after it with RT_PLAN_LONG_ALONE), are the four-lane share,
 *     the rest one entry per other ray.  *n_claims receives the number of
 *     entries written: n, plus 7 * *n_long with RT_PLAN_LONG_ALONE (at most
 *     n + 7 * (n / 16)).
 * Errors: RT_EINVAL (NULL cost or claims, bad dimensions or order, spread,
 * flags, factor, sm_count, or claims_cap below the entries needed). */
rt_err rt_order_claims(const int32_t *cost, int32_t n_freq, int32_t n_modes, int32_t n_el, int32_t n_az,
                       int32_t claim_order, int32_t spread, double long_factor, int32_t mixed, uint32_t flags,
                       int32_t sm_count, int32_t *claims, size_t claims_cap, size_t *n_long, size_t *n_claims);

/* --------------------------------------------------------------- ionogram */
/* Oblique-ionogram synthesis (Sec. IV-B-4: joint frequency-elevation scan,
 * group path against frequency at the receiver).  The fan is launched from
 * the transmitter towards the receiver (azimuth = initial bearing of the
 * great circle), every frequency x mode x elevation.  For each frequency and
 * mode, every pair of neighbouring elevations whose LANDED rays bracket the
 * transmitter-receiver ground distance D_rx gives one ionogram point, by
 * linear interpolation in D of group path and elevation.  Points are returned
 * sorted by (frequency, mode, elevation); branch numbers the crossings of
 * one trace from the lowest elevation (0: the low ray, 1: the high ray, ...).
 * Elevations must be ascending.  At most cap points are written; *n_points
 * receives the total found.  Blocking. */
typedef struct rt_ionogram_desc {
    double tx_lat_deg, tx_lon_deg, tx_alt_km;
    double rx_lat_deg, rx_lon_deg;
    const double *freq_mhz;     /* n_freq values */
    const double *el_deg;       /* n_el ascending values */
    int32_t n_freq, n_el;
    uint32_t modes;             /* RT_MODE_O | RT_MODE_X */
    int32_t integrator, precision;
    int32_t max_steps;
    double h_km, rtol, atol_km, h_min_km, h_max_km;
} rt_ionogram_desc;

typedef struct rt_ionogram_point {
    double freq_mhz;
    double group_path_km;       /* P' at the receiver distance */
    double el_deg;              /* launch elevation reaching the receiver distance */
    double ground_range_km;     /* D_rx */
    int32_t mode;               /* +1 ordinary, -1 extraordinary */
    int32_t branch;
} rt_ionogram_point;           /* 40 bytes */

rt_err rt_ionogram(const rt_grid *grid, const rt_ionogram_desc *desc, rt_ionogram_point *out_host, size_t cap,
                   size_t *n_points, const rt_launch_config *cfg, void *stream);

/* ---------------------------------------------------------------- serving */
/* A request server for fans of uneven size against resident grids
 * (continuous batching).  Submitted requests wait in a FIFO; a dispatcher
 * thread admits them as soon as one of max_inflight stream slots is free and
 * the free device memory (cudaMemGetInfo, or the caller's free_bytes
 * function) stays at least mem_reserve_bytes above the request's own needs
 * (twice its records plus 4 KiB of fan tables per request; the grids are
 * resident and already in use), so requests that arrive while others run are
 * traced concurrently with them on the GPU.  A request that does not fit
 * waits for running requests to finish; when none runs, it is admitted if its
 * own needs fit in the free memory (the reserve is then waived, so a lone
 * request always makes progress) and otherwise finishes at once with status
 * RT_ENOMEM, without touching the GPU, while the requests behind it proceed.  A
 * completion thread copies each result to the caller's host buffer (through
 * pinned staging) and wakes rt_server_wait.  Every request uses the launch
 * configuration given at creation, so its records equal those of rt_trace
 * with that configuration whatever else is in flight.  Optionally, small
 * requests queued at the same time are fused into one launch (fuse_max_rays)
 * so that they fill the GPU together.  The paper has no
 * counterpart (it traces one scan at a time on a CPU). */
typedef struct rt_server rt_server;

typedef struct rt_server_config {
    int32_t max_inflight;        /* stream slots, 1..64 (0 = 8) */
    int32_t fuse_max_rays;       /* 0 = one launch per request.  > 0: fusion.  Small requests are the
                                    mixed ones that the automatic lane choice would trace at four lanes
                                    per ray on their own (at most a quarter of the resident lanes:
                                    14,592 rays on 152 SMs with the default block) and of at most
                                    fuse_max_rays rays.  The dispatcher admits a small head request
                                    together with the queued small requests on the same grid with the
                                    same integrator, in queue order, up to fuse_max_rays rays in total
                                    and 256 requests, and traces them as one launch in one slot.  Every
                                    small request, alone or not, runs the fused kernel: four lanes per
                                    ray, the stencil, block size and ray order of `launch` (whose kernel
                                    must be AUTO or PLAIN and lanes_per_ray 0 or 4).  Its records
                                    therefore do not depend on what shares its launch; they equal those
                                    of rt_trace on the plain kernel at four lanes per ray up to float
                                    rounding (the two kernels are compiled apart).  Other requests run
                                    as without fusion. */
    size_t mem_reserve_bytes;    /* device memory kept free by admission */
    rt_launch_config launch;     /* kernel choice for every request (zero = library defaults) */
    /* Optional: the device memory admission may use, asked before every
     * admission decision (from the dispatcher thread) instead of
     * cudaMemGetInfo's free bytes -- e.g. a budget shared with another
     * runtime on the same GPU.  NULL: cudaMemGetInfo. */
    size_t (*free_bytes)(void *user);
    void *free_bytes_user;
} rt_server_config;

typedef struct rt_request_stats {
    double queue_s;              /* submit -> admitted */
    double run_s;                /* admitted -> result in the caller's buffer */
    double total_s;              /* submit -> result in the caller's buffer */
    int64_t n_rays;
    int32_t status;              /* rt_err of the request */
    int32_t batch_size;          /* requests traced by the launch that traced this one (1 = alone) */
} rt_request_stats;

/* Creates a server on the current device (threads start immediately). */
rt_err rt_server_create(const rt_server_config *cfg, rt_server **out);
/* Queues a request; the fan arrays are copied, out_host (rt_fan_size(fan)
 * records) must stay valid until rt_server_wait returns for the ticket. */
rt_err rt_server_submit(rt_server *srv, const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_host,
                        size_t out_len, uint64_t *ticket);
/* Waits for a request (timeout_s <= 0: no limit); RT_ETIMEOUT if it has not
 * finished in time (the request stays queued or running).  A waited ticket
 * is released.  stats may be NULL. */
rt_err rt_server_wait(rt_server *srv, uint64_t ticket, double timeout_s, rt_request_stats *stats);
/* Finishes every queued and running request, then stops the threads. */
rt_err rt_server_destroy(rt_server *srv);

/* ------------------------------------------------------------ measurement */
/* Ceilings of the current GPU measured with kernels of this library: FP32 and
 * FP64 fused multiply-add throughput (independent FMA chains on every lane of
 * every SM; an FMA counts 2 flop) and L2 read bandwidth (a 48 MiB buffer read
 * repeatedly through L2, bypassing L1).  Takes about a second.  The paper has
 * no counterpart: the benchmark uses these as the roofline ceilings of the
 * tracer (FP32 issue for the mixed path, FP64 for the all-FP64 path, L2 for
 * the sample gathers). */
typedef struct rt_peaks {
    double fp32_fma_flops;       /* flop/s */
    double fp64_fma_flops;       /* flop/s */
    double l2_read_bytes_per_s;  /* bytes/s */
    int32_t sm_count;
    int32_t reserved;
    double max_sm_mhz;           /* the device's maximum SM clock */
} rt_peaks;

rt_err rt_measure_peaks(rt_peaks *out);

/* Diagnostic: the right-hand side dy/dP' of the ray equations (Eq. 1a-1f)
 * at n given states, exactly as one stage of the tracer evaluates it.
 * y_host: n x 6 doubles (r km, theta rad colatitude, phi rad longitude,
 * k_r, k_theta, k_phi in units of omega/c); dy_host: n x 6 doubles out;
 * mu2_host: n doubles out (mu^2 of Eq. 3 at the state).  mode: +1 ordinary,
 * -1 extraordinary.  precision RT_FP64 or RT_MIXED; stencil as in
 * rt_launch_config (mixed only; AUTO = QUAD).  Blocking; allocates device
 * scratch with cudaMalloc.  Errors: RT_EINVAL, RT_ENOMEM, RT_ECUDA. */
rt_err rt_eval_rhs(const rt_grid *grid, double freq_mhz, int32_t mode, int32_t precision, int32_t stencil,
                   const double *y_host, double *dy_host, double *mu2_host, size_t n);

/* Message of the last failed call on this thread ("" if none). */
const char *rt_last_error(void);

/* RTGD_API_VERSION of the library. */
int32_t rt_version(void);

#ifdef __cplusplus
}
#endif
#endif
