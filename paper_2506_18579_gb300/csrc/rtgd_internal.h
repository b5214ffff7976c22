// rtgd_internal.h -- structures shared by the host API and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "rtgd.h"
#include "rtgd_device.cuh"

namespace rtgd {

struct GridSizes {
    int n_lat, n_lon, n_alt;
};

// Per-fan tables the host prepares (fan_tables_into): per frequency the
// frequency and the float factors of the mixed path, per elevation and
// azimuth the sines and cosines of the launch direction -- computed once per
// fan instead of once per ray (a double division or sincos costs a warp many
// cycles of GB300's 1/64-rate FP64 pipe, and a persistent kernel's refills run
// it for one lane at a time).
struct FanFreq {
    double f_hz;      // frequency (Hz)
    float xfac;       // 80.6 / f^2 (X = xfac Ne), rounded from double
    float ab0;        // f_H / f per tesla times the dipole's B0, rounded from double
};
struct FanEl {
    double s, c;      // sin, cos of the elevation
};
struct FanAz {
    double s, c;      // sin, cos of the azimuth
    double rad;       // azimuth (rad)
};
// Doubles a fan's tables take: 2 per frequency, 2 per elevation, 3 per azimuth.
inline size_t fan_table_doubles(int n_freq, int n_el, int n_az) {
    return 2 * (size_t)n_freq + 2 * (size_t)n_el + 3 * (size_t)n_az;
}

// Device view of a fan (arrays in device memory) plus the integrator settings.
struct FanDev {
    const FanFreq *freq;
    const FanEl *el;
    const FanAz *az;
    int n_freq, n_el, n_az, n_modes;
    int mode0, mode1;    // mode sign of mode index 0 / 1 (+1 ordinary, -1 extraordinary)
    int integrator, precision, max_steps, order;
    long long n_rays;
    double tx_r, tx_th, tx_ph;  // launch position (km, rad, rad)
    double h0, rtol, atol, hmin, hmax, max_path;
    double land_tol;            // |r - R_E| accepted by the landing solve (km)
    float rtol_f, atol_f, h0_f, hmin_f, hmax_f;
    int has_max_path;           // max_path > 0
    // Optional claim order (an ordered plan): claim c of this launch traces
    // canonical ray perm[perm_off + c]; n_rays then counts this launch's
    // claims.  A negative entry is a hole (no ray); holes occur only in the
    // claims of an ordered plan's four-lane launch (plain kernel).
    const int *perm;
    long long perm_off;
};

struct LaunchPlan {
    int kernel;   // RT_KERNEL_PLAIN / RT_KERNEL_PERSISTENT
    int stencil;  // RT_STENCIL_GATHER / QUAD / TABLE
    int threads;
    int blocks;   // persistent grid size
    int lanes;    // lanes per ray (1, 2, 4)
    int smem = 0; // plain kernel: dynamic shared memory per block (bytes); see plain_exclusive_smem
    // plain kernel: an event (timing disabled) that the launch records once
    // all of its blocks have begun (a launch-completion event), or null
    cudaEvent_t started = nullptr;
};

cudaError_t launch_grid_prep(const void *raw, int dtype, const GridSizes &sz, double *pad64, float *pad32,
                             float4 *quad, float4 *table, cudaStream_t st);
cudaError_t upload_tableaus();
// Trace launch then (mixed path) the pass that turns the raw final states
// into the records' outputs.
cudaError_t launch_trace(const GridDev &g, const FanDev &f, rt_ray_result *out, unsigned long long *counter,
                         const LaunchPlan &lp, cudaStream_t st);
// The two steps separately (an ordered plan finishes once after its two launches).
cudaError_t launch_trace_only(const GridDev &g, const FanDev &f, rt_ray_result *out, unsigned long long *counter,
                              const LaunchPlan &lp, cudaStream_t st);
cudaError_t launch_finish(const GridDev &g, const FanDev &f, rt_ray_result *out, long long n, cudaStream_t st);
cudaError_t persistent_occupancy(int stencil, int lanes, int threads, int *blocks_per_sm);
// ev[i] = rec[i].n_evals for i < n (the cost field of n records, packed).
cudaError_t launch_gather_evals(const rt_ray_result *rec, int32_t *ev, long long n, cudaStream_t st);
// Dynamic shared memory that makes a block of the plain kernel of lp (with
// interpolant interp) fill a whole SM's shared memory, so that no other block
// of any kernel is resident beside it; also raises the kernel's limit to it.
cudaError_t plain_exclusive_smem(const LaunchPlan &lp, int interp, int *bytes);
// Mixed path, four lanes per ray: n_fans fans (device array fans) in one
// launch; first (device, n_fans + 1 entries) holds each fan's first ray in
// the launch and the total; out receives the records fan after fan.
cudaError_t launch_trace_fans(const GridDev &g, const FanDev *fans, const long long *first, int n_fans,
                              long long n_total, int integrator, rt_ray_result *out, const LaunchPlan &lp,
                              cudaStream_t st);
}  // namespace rtgd

// Entry points shared between the translation units of the host library
// (defined in rtgd_api.cu).
rt_err rtgd_queue_trace(const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_dev, size_t out_len,
                        const rt_launch_config *cfg, cudaStream_t st);
// Queues n_fans mixed-precision fans with one integrator on one grid as one
// launch (four lanes per ray; stencil, block size and ray order from cfg);
// out_dev receives the records fan after fan.  A fan's records do not
// depend on the other fans of the launch.
rt_err rtgd_queue_trace_fans(const rt_grid *grid, const rt_fan_desc *const *fans, int n_fans, rt_ray_result *out_dev,
                             size_t out_len, const rt_launch_config *cfg, cudaStream_t st);
rt_err rtgd_set_error(rt_err code, const char *msg);
// Largest fan that the automatic lane choice traces at four lanes per ray
// on this device with cfg's stencil and block size.
rt_err rtgd_four_lane_limit(int device, const rt_launch_config *cfg, size_t *limit);

namespace rtgd {

cudaError_t launch_ionogram(const rt_ray_result *res, const double *freq, const double *el, int n_freq, int n_modes,
                            int mode0, int n_el, double d_rx, rt_ionogram_point *out, unsigned long long cap,
                            unsigned long long *count, cudaStream_t st);

// Scratch of rt_trace_device_noalloc (rtgd_noalloc.cu): ray counter + the
// tables of a fan with n_freq + n_el + n_az <= kNoallocMaxTable (at most 3
// doubles per entry).
constexpr int kNoallocMaxTable = 4096;
constexpr size_t kNoallocScratchBytes = 16 + 3 * (size_t)kNoallocMaxTable * sizeof(double);
cudaError_t noalloc_scratch(int device, void **ptr, size_t *bytes);

cudaError_t launch_eval_rhs(const GridDev &g, const double *ys, double *dys, double *mu2s, double freq_mhz, int mode,
                            int precision, int stencil, long long n, cudaStream_t st);

}  // namespace rtgd
