// rtgd_api.cu -- host side of the C ABI declared in include/rtgd.h.
//
// Grid handles own their device memory (cudaMalloc).  Trace calls take their
// scratch (fan tables, the persistent kernel's ray counter, staged results)
// from the stream-ordered allocator and release it stream-ordered, so they
// are safe to issue from several threads on several streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "rtgd.h"
#include "rtgd_internal.h"

namespace rtgd {
// The cost field of n records, packed (rt_plan_order reads it back in one piece).
__global__ void gather_evals_kernel(const rt_ray_result *__restrict__ rec, int32_t *__restrict__ ev, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) ev[i] = rec[i].n_evals;
}

cudaError_t launch_gather_evals(const rt_ray_result *rec, int32_t *ev, long long n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    gather_evals_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(rec, ev, n);
    return cudaGetLastError();
}
}  // namespace rtgd

using namespace rtgd;

struct rt_grid {
    rt_grid_desc desc;
    int device;
    GridDev g;
    double *pad64 = nullptr;
    float *pad32 = nullptr;
    float4 *quad = nullptr;
    float4 *table = nullptr;
    size_t bytes = 0;
};

namespace {

thread_local std::string g_err;

rt_err fail(rt_err code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

rt_err cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) return fail(RT_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        return fail(RT_EUNSUPPORTED, "%s: %s", what, cudaGetErrorString(e));
    return fail(RT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(call)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

std::mutex g_dev_mu;
std::map<int, bool> g_dev_ready;

// Checks for a usable device and uploads the Butcher tables once per device.
rt_err ensure_device(int *dev_out) {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return fail(RT_EUNSUPPORTED, "no CUDA device available (%s)", cudaGetErrorString(e));
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_dev_ready[dev]) {
        CUDA_TRY(upload_tableaus());
        g_dev_ready[dev] = true;
    }
    if (dev_out) *dev_out = dev;
    return RT_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

rt_err validate_grid_desc(const rt_grid_desc *d) {
    if (!d) return fail(RT_EINVAL, "grid descriptor is NULL");
    if (d->n_lat < 4 || d->n_lon < 4 || d->n_alt < 4)
        return fail(RT_EINVAL, "grid needs at least 4 nodes per dimension (got %d x %d x %d)", d->n_lat, d->n_lon,
                    d->n_alt);
    if ((long long)d->n_lat * d->n_lon * d->n_alt > (1LL << 34)) return fail(RT_EINVAL, "grid too large");
    if (d->dtype != RT_F32 && d->dtype != RT_F64) return fail(RT_EINVAL, "unknown dtype %d", d->dtype);
    if (!finite_pos(d->dlat_deg) || !finite_pos(d->dlon_deg) || !finite_pos(d->dalt_km))
        return fail(RT_EINVAL, "grid spacings must be finite and > 0");
    if (!finite_pos(d->earth_radius_km)) return fail(RT_EINVAL, "earth_radius_km must be finite and > 0");
    if (!std::isfinite(d->lat0_deg) || !std::isfinite(d->lon0_deg) || !std::isfinite(d->alt0_km))
        return fail(RT_EINVAL, "grid origin must be finite");
    if (d->lat0_deg < -90.0 || d->lat0_deg + (d->n_lat - 1) * d->dlat_deg > 90.0)
        return fail(RT_EINVAL, "grid latitudes must lie in [-90, 90]");
    if (!std::isfinite(d->field.b0_tesla) || d->field.b0_tesla < 0.0 || !std::isfinite(d->field.pole_lat_deg) ||
        !std::isfinite(d->field.pole_lon_deg))
        return fail(RT_EINVAL, "dipole parameters must be finite, b0 >= 0");
    if (d->flags & ~(uint32_t)(RT_GRID_TABLE | RT_GRID_CATMULL_ROM))
        return fail(RT_EINVAL, "unknown grid flags 0x%x", d->flags);
    if (d->reserved != 0) return fail(RT_EINVAL, "reserved field must be 0");
    return RT_OK;
}

size_t fan_rays(const rt_fan_desc *f) {
    const int nm = ((f->modes & RT_MODE_O) ? 1 : 0) + ((f->modes & RT_MODE_X) ? 1 : 0);
    return (size_t)f->n_freq * (size_t)nm * (size_t)f->n_el * (size_t)f->n_az;
}

rt_err validate_fan(const rt_fan_desc *f) {
    if (!f) return fail(RT_EINVAL, "fan descriptor is NULL");
    if (f->n_freq < 1 || f->n_el < 1 || f->n_az < 1)
        return fail(RT_EINVAL, "fan needs n_freq, n_el, n_az >= 1 (got %d, %d, %d)", f->n_freq, f->n_el, f->n_az);
    if (!f->freq_mhz || !f->el_deg || !f->az_deg) return fail(RT_EINVAL, "fan arrays must not be NULL");
    if (f->modes == 0 || (f->modes & ~3u)) return fail(RT_EINVAL, "modes must be a non-empty subset of O|X");
    if (f->integrator != RT_RK4 && f->integrator != RT_RKF45) return fail(RT_EINVAL, "unknown integrator %d", f->integrator);
    if (f->precision != RT_FP64 && f->precision != RT_MIXED) return fail(RT_EINVAL, "unknown precision %d", f->precision);
    if (!finite_pos(f->h_km)) return fail(RT_EINVAL, "h_km must be finite and > 0");
    if (f->integrator == RT_RKF45) {
        if (!finite_pos(f->rtol) || !std::isfinite(f->atol_km) || f->atol_km < 0.0)
            return fail(RT_EINVAL, "RKF45 needs rtol > 0 and atol_km >= 0");
        if (!finite_pos(f->h_min_km) || !finite_pos(f->h_max_km) || f->h_max_km < f->h_min_km)
            return fail(RT_EINVAL, "RKF45 needs 0 < h_min_km <= h_max_km");
    }
    if (f->max_steps < 1) return fail(RT_EINVAL, "max_steps must be >= 1");
    if (f->reserved != 0) return fail(RT_EINVAL, "reserved field must be 0");
    if (!std::isfinite(f->tx_lat_deg) || !std::isfinite(f->tx_lon_deg) || !std::isfinite(f->tx_alt_km) ||
        f->tx_lat_deg <= -90.0 || f->tx_lat_deg >= 90.0)
        return fail(RT_EINVAL, "transmitter position must be finite with |lat| < 90");
    if (!std::isfinite(f->max_group_path_km)) return fail(RT_EINVAL, "max_group_path_km must be finite");
    for (int i = 0; i < f->n_freq; ++i)
        if (!finite_pos(f->freq_mhz[i])) return fail(RT_EINVAL, "freq_mhz[%d] must be finite and > 0", i);
    for (int i = 0; i < f->n_el; ++i)
        if (!std::isfinite(f->el_deg[i])) return fail(RT_EINVAL, "el_deg[%d] is not finite", i);
    for (int i = 0; i < f->n_az; ++i)
        if (!std::isfinite(f->az_deg[i])) return fail(RT_EINVAL, "az_deg[%d] is not finite", i);
    return RT_OK;
}

struct DevProps {
    int sms = 0;
};
std::mutex g_props_mu;
std::map<int, DevProps> g_props;

DevProps props(int dev) {
    std::lock_guard<std::mutex> lk(g_props_mu);
    auto it = g_props.find(dev);
    if (it != g_props.end()) return it->second;
    DevProps p;
    cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev);
    g_props[dev] = p;
    return p;
}

// Autotuner cache: (grid, integrator, ray-count bucket) -> launch config.
std::mutex g_tune_mu;
std::map<std::tuple<const rt_grid *, int, int>, rt_launch_config> g_tuned;

int ray_bucket(size_t n) {
    int b = 0;
    while (n > 1) {
        n >>= 1;
        ++b;
    }
    return b;
}

rt_err make_plan(const rt_grid *grid, const rt_fan_desc *fan, size_t n_rays, const rt_launch_config *cfg,
                 LaunchPlan *lp, int *order) {
    rt_launch_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    if (c.kernel < 0 || c.kernel > RT_KERNEL_PERSISTENT) return fail(RT_EINVAL, "unknown kernel %d", c.kernel);
    if (c.stencil < 0 || c.stencil > RT_STENCIL_TABLE) return fail(RT_EINVAL, "unknown stencil %d", c.stencil);
    if (c.block_threads != 0 && (c.block_threads < 32 || c.block_threads > 128 || c.block_threads % 32))
        return fail(RT_EINVAL, "block_threads must be 0 or a multiple of 32 in [32, 128]");
    if (c.order != RT_ORDER_CANONICAL && c.order != RT_ORDER_ELEVATION_FASTEST)
        return fail(RT_EINVAL, "unknown order %d", c.order);
    if (c.blocks_per_sm < 0) return fail(RT_EINVAL, "blocks_per_sm must be >= 0");
    if (c.lanes_per_ray != 0 && c.lanes_per_ray != 1 && c.lanes_per_ray != 2 && c.lanes_per_ray != 4)
        return fail(RT_EINVAL, "lanes_per_ray must be 0, 1, 2 or 4");
    if (c.reserved[0] != 0 || c.reserved[1] != 0) return fail(RT_EINVAL, "reserved fields must be 0");
    if (fan->precision == RT_MIXED && c.kernel == RT_KERNEL_AUTO && c.stencil == RT_STENCIL_AUTO) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(std::make_tuple(grid, fan->integrator, ray_bucket(n_rays)));
        if (it != g_tuned.end()) c = it->second;
    }
    if (c.kernel == RT_KERNEL_AUTO) c.kernel = RT_KERNEL_PLAIN;  // measured faster on GB300 for small and large fans
    if (fan->precision == RT_FP64 && c.kernel != RT_KERNEL_PLAIN)
        return fail(RT_EINVAL, "the FP64 path runs the plain one-thread-per-ray kernel only");
    if (c.stencil == RT_STENCIL_AUTO) c.stencil = RT_STENCIL_QUAD;
    if (c.stencil == RT_STENCIL_TABLE && !grid->table)
        return fail(RT_EINVAL, "stencil TABLE needs a grid created with RT_GRID_TABLE");
    if (c.order == RT_ORDER_CANONICAL && cfg == nullptr) c.order = RT_ORDER_ELEVATION_FASTEST;
    if (fan->precision == RT_FP64 && c.lanes_per_ray > 1)
        return fail(RT_EINVAL, "the FP64 path runs one lane per ray");
    lp->kernel = c.kernel;
    lp->stencil = c.stencil;
    lp->threads = c.block_threads ? c.block_threads : 128;
    lp->blocks = 0;
    lp->lanes = 1;
    if (fan->precision == RT_MIXED) {
        int lanes = c.lanes_per_ray;
        if (lanes == 0) {
            // as many lanes per ray as keep the fan within the resident lanes
            int occ = 0;
            CUDA_TRY(persistent_occupancy(c.stencil, 1, lp->threads, &occ));
            const long long resident = (long long)props(grid->device).sms * std::max(occ, 1) * lp->threads;
            lanes = 1;
            while (lanes < 4 && (long long)n_rays * lanes * 2 <= resident) lanes *= 2;
        }
        lp->lanes = lanes;
    }
    if (fan->precision == RT_MIXED && c.kernel == RT_KERNEL_PERSISTENT) {
        int occ = 0;
        CUDA_TRY(persistent_occupancy(c.stencil, lp->lanes, lp->threads, &occ));
        if (occ < 1) return fail(RT_ECUDA, "persistent kernel does not fit on an SM with %d threads", lp->threads);
        if (c.blocks_per_sm > 0) occ = std::min(occ, c.blocks_per_sm);
        const long long want = (long long)props(grid->device).sms * occ;
        const long long need = (long long)((n_rays * lp->lanes + lp->threads - 1) / lp->threads);
        lp->blocks = (int)std::max(1LL, std::min(want, need));
    }
    *order = c.order;
    return RT_OK;
}

double sync_timeout_s() {
    const char *s = std::getenv("RTGD_SYNC_TIMEOUT_S");
    if (s) {
        const double v = std::atof(s);
        if (v > 0) return v;
    }
    return 900.0;
}

// Waits for the stream with a deadline instead of blocking indefinitely.
rt_err sync_with_timeout(cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    const double limit = sync_timeout_s();
    // polls every <= 100 us for the first second (a fan finishing between
    // two polls costs the caller at most that), then every <= 2 ms
    int sleep_us = 10;
    for (;;) {
        const cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return RT_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "kernel execution");
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt > limit) return fail(RT_ETIMEOUT, "stream did not finish within %.0f s", limit);
        std::this_thread::sleep_for(std::chrono::microseconds(sleep_us));
        sleep_us = std::min(sleep_us * 2, dt < 1.0 ? 100 : 2000);
    }
}

// Device view of a fan whose tables (fan_tables_into) start at tab.
FanDev fill_fandev(const rt_grid *grid, const rt_fan_desc *fan, size_t n, int order, const double *tab) {
    FanDev f;
    std::memset(&f, 0, sizeof(f));
    f.freq = (const FanFreq *)tab;
    f.el = (const FanEl *)(tab + 2 * (size_t)fan->n_freq);
    f.az = (const FanAz *)(tab + 2 * (size_t)fan->n_freq + 2 * (size_t)fan->n_el);
    f.n_freq = fan->n_freq;
    f.n_el = fan->n_el;
    f.n_az = fan->n_az;
    f.n_modes = ((fan->modes & RT_MODE_O) ? 1 : 0) + ((fan->modes & RT_MODE_X) ? 1 : 0);
    f.mode0 = (fan->modes & RT_MODE_O) ? 1 : -1;
    f.mode1 = -1;
    f.integrator = fan->integrator;
    f.precision = fan->precision;
    f.max_steps = fan->max_steps;
    f.order = order;
    f.n_rays = (long long)n;
    f.tx_r = grid->desc.earth_radius_km + fan->tx_alt_km;
    f.tx_th = (90.0 - fan->tx_lat_deg) * kDeg2Rad;
    f.tx_ph = fan->tx_lon_deg * kDeg2Rad;
    f.h0 = fan->h_km;
    f.rtol = fan->rtol;
    f.atol = fan->atol_km;
    f.hmin = fan->integrator == RT_RKF45 ? fan->h_min_km : 0.0;
    f.hmax = fan->integrator == RT_RKF45 ? fan->h_max_km : fan->h_km;
    f.max_path = fan->max_group_path_km;
    // FP64: 1e-9 km; mixed: the float increment resolves ~1e-6 km, so 1e-5 km
    f.land_tol = fan->precision == RT_FP64 ? 1e-9 : 1e-5;
    f.rtol_f = (float)fan->rtol;
    f.atol_f = (float)fan->atol_km;
    f.h0_f = (float)f.h0;
    f.hmin_f = (float)f.hmin;
    f.hmax_f = (float)f.hmax;
    f.has_max_path = f.max_path > 0.0 ? 1 : 0;
    return f;
}

// The tables of a fan (layout FanFreq[n_freq], FanEl[n_el], FanAz[n_az], all
// in doubles: fan_table_doubles) written to dst.  The float factors are the
// double expressions rounded once; the sines and cosines are the host's.
void fan_tables_into(const rt_grid *grid, const rt_fan_desc *fan, double *dst) {
    FanFreq *fq = (FanFreq *)dst;
    FanEl *fe = (FanEl *)(dst + 2 * (size_t)fan->n_freq);
    FanAz *fa = (FanAz *)(dst + 2 * (size_t)fan->n_freq + 2 * (size_t)fan->n_el);
    for (int i = 0; i < fan->n_freq; ++i) {
        const double f_hz = fan->freq_mhz[i] * 1e6;
        fq[i].f_hz = f_hz;
        fq[i].xfac = (float)(kPlasmaHz2PerM3 / (f_hz * f_hz));
        fq[i].ab0 = (float)(kGyroHzPerTesla / f_hz * grid->desc.field.b0_tesla);
    }
    for (int i = 0; i < fan->n_el; ++i) {
        const double el = fan->el_deg[i] * kDeg2Rad;
        fe[i].s = std::sin(el);
        fe[i].c = std::cos(el);
    }
    for (int i = 0; i < fan->n_az; ++i) {
        const double az = fan->az_deg[i] * kDeg2Rad;
        fa[i].s = std::sin(az);
        fa[i].c = std::cos(az);
        fa[i].rad = az;
    }
}

// The device scratch image of a fan: a zeroed 16-byte ray counter followed
// by the fan's tables, built in library-owned pageable host memory
// (fan_image_bytes(fan) bytes at img).  Uploading this image (one
// cudaMemcpyAsync) instead of the caller's arrays means the caller may change
// or free its arrays as soon as the call returns, whether they are pinned or
// not: a copy from pageable memory has read its source when cudaMemcpyAsync
// returns.
size_t fan_image_bytes(const rt_fan_desc *fan) {
    return 16 + fan_table_doubles(fan->n_freq, fan->n_el, fan->n_az) * sizeof(double);
}

void fan_image_into(const rt_grid *grid, const rt_fan_desc *fan, char *img) {
    std::memset(img, 0, 16);
    fan_tables_into(grid, fan, (double *)(img + 16));
}

std::vector<char> fan_image(const rt_grid *grid, const rt_fan_desc *fan) {
    std::vector<char> img(fan_image_bytes(fan));
    fan_image_into(grid, fan, img.data());
    return img;
}

// Queues one trace: scratch allocation, fan upload, kernel, scratch release.
rt_err queue_trace(const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_dev, size_t out_len,
                   const rt_launch_config *cfg, cudaStream_t st) {
    rt_err r = validate_fan(fan);
    if (r != RT_OK) return r;
    if (!grid) return fail(RT_EINVAL, "grid is NULL");
    if (!out_dev) return fail(RT_EINVAL, "output pointer is NULL");
    int dev = 0;
    if ((r = ensure_device(&dev)) != RT_OK) return r;
    if (dev != grid->device) return fail(RT_EINVAL, "grid lives on device %d, current device is %d", grid->device, dev);
    const size_t n = fan_rays(fan);
    if (out_len < n) return fail(RT_EINVAL, "out_len %zu < %zu rays", out_len, n);
    if (n >= ((size_t)1 << 31)) return fail(RT_EINVAL, "fan too large (at most 2^31 - 1 rays)");
    LaunchPlan lp;
    int order = 0;
    if ((r = make_plan(grid, fan, n, cfg, &lp, &order)) != RT_OK) return r;

    const std::vector<char> img = fan_image(grid, fan);
    char *ws = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&ws, img.size(), st));
    unsigned long long *counter = (unsigned long long *)ws;
    double *tab = (double *)(ws + 16);
    cudaError_t e = cudaMemcpyAsync(ws, img.data(), img.size(), cudaMemcpyHostToDevice, st);
    const FanDev f = fill_fandev(grid, fan, n, order, tab);
    if (e == cudaSuccess) e = launch_trace(grid->g, f, out_dev, counter, lp, st);
    const cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "trace launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return RT_OK;
}

}  // namespace

rt_err rtgd_queue_trace(const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_dev, size_t out_len,
                        const rt_launch_config *cfg, cudaStream_t st) {
    return queue_trace(grid, fan, out_dev, out_len, cfg, st);
}

rt_err rtgd_queue_trace_fans(const rt_grid *grid, const rt_fan_desc *const *fans, int n_fans, rt_ray_result *out_dev,
                             size_t out_len, const rt_launch_config *cfg, cudaStream_t st) {
    if (!grid || !fans || n_fans < 1 || !out_dev) return fail(RT_EINVAL, "fused trace: NULL argument or no fans");
    int dev = 0;
    rt_err r = ensure_device(&dev);
    if (r != RT_OK) return r;
    if (dev != grid->device) return fail(RT_EINVAL, "grid lives on device %d, current device is %d", grid->device, dev);
    size_t n_total = 0, n_tab = 0;
    for (int k = 0; k < n_fans; ++k) {
        if ((r = validate_fan(fans[k])) != RT_OK) return r;
        if (fans[k]->precision != RT_MIXED) return fail(RT_EINVAL, "fused trace: mixed-precision fans only");
        if (fans[k]->integrator != fans[0]->integrator) return fail(RT_EINVAL, "fused trace: fans differ in integrator");
        n_total += fan_rays(fans[k]);
        n_tab += fan_table_doubles(fans[k]->n_freq, fans[k]->n_el, fans[k]->n_az);
    }
    if (out_len < n_total) return fail(RT_EINVAL, "out_len %zu < %zu rays", out_len, n_total);
    if (n_total >= ((size_t)1 << 31)) return fail(RT_EINVAL, "fused trace too large (at most 2^31 - 1 rays)");
    rt_launch_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    c.kernel = RT_KERNEL_PLAIN;
    c.lanes_per_ray = 4;
    LaunchPlan lp;
    int order = 0;
    if ((r = make_plan(grid, fans[0], n_total, &c, &lp, &order)) != RT_OK) return r;
    // scratch: the fans' device views, the n_fans + 1 ray offsets, the fan tables
    const size_t off_first = (size_t)n_fans * sizeof(FanDev);
    const size_t off_tab = off_first + (size_t)(n_fans + 1) * sizeof(long long);
    const size_t bytes = off_tab + n_tab * sizeof(double);
    std::vector<char> blob(bytes);
    char *ws = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&ws, bytes, st));
    FanDev *fd = (FanDev *)blob.data();
    long long *first = (long long *)(blob.data() + off_first);
    double *tab_h = (double *)(blob.data() + off_tab);
    const double *tab_d = (const double *)(ws + off_tab);
    size_t t = 0;
    long long acc = 0;
    for (int k = 0; k < n_fans; ++k) {
        const rt_fan_desc *fk = fans[k];
        const size_t nk = fan_rays(fk);
        fan_tables_into(grid, fk, tab_h + t);
        fd[k] = fill_fandev(grid, fk, nk, order, tab_d + t);
        first[k] = acc;
        acc += (long long)nk;
        t += fan_table_doubles(fk->n_freq, fk->n_el, fk->n_az);
    }
    first[n_fans] = acc;
    cudaError_t e = cudaMemcpyAsync(ws, blob.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_trace_fans(grid->g, (const FanDev *)ws, (const long long *)(ws + off_first), n_fans, acc,
                              fans[0]->integrator, out_dev, lp, st);
    const cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "fused trace launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return RT_OK;
}

rt_err rtgd_four_lane_limit(int device, const rt_launch_config *cfg, size_t *limit) {
    const int stencil = cfg && cfg->stencil != RT_STENCIL_AUTO ? cfg->stencil : RT_STENCIL_QUAD;
    const int threads = cfg && cfg->block_threads ? cfg->block_threads : 128;
    int occ = 0;
    CUDA_TRY(persistent_occupancy(stencil, 1, threads, &occ));
    // the automatic lane choice gives four lanes to fans of at most a quarter of the resident lanes
    *limit = (size_t)props(device).sms * (size_t)std::max(occ, 1) * (size_t)threads / 4;
    return RT_OK;
}

rt_err rtgd_set_error(rt_err code, const char *msg) { return fail(code, "%s", msg); }

extern "C" {

int32_t rt_version(void) { return RTGD_API_VERSION; }

const char *rt_last_error(void) { return g_err.c_str(); }

size_t rt_fan_size(const rt_fan_desc *fan) {
    if (!fan || fan->n_freq < 1 || fan->n_el < 1 || fan->n_az < 1 || fan->modes == 0 || (fan->modes & ~3u)) return 0;
    return fan_rays(fan);
}

rt_err rt_grid_create(const rt_grid_desc *desc, const void *ne_host, rt_grid **out) {
    if (!out) return fail(RT_EINVAL, "out is NULL");
    *out = nullptr;
    rt_err r = validate_grid_desc(desc);
    if (r != RT_OK) return r;
    if (!ne_host) return fail(RT_EINVAL, "ne_host is NULL");
    int dev = 0;
    if ((r = ensure_device(&dev)) != RT_OK) return r;
    rt_grid *g = new rt_grid();
    g->desc = *desc;
    g->device = dev;
    const long long nl = desc->n_lat, nn = desc->n_lon, na = desc->n_alt;
    const size_t n_raw = (size_t)(nl * nn * na);
    const size_t n_pad = (size_t)((nl + 2) * (nn + 2) * (na + 2));
    const size_t n_quad = (size_t)((nl + 2) * (nn + 2) * (na - 1));
    const size_t n_tab = (desc->flags & RT_GRID_TABLE) ? (size_t)((nl - 1) * (nn - 1) * (na - 1) * 16) : 0;
    const size_t esz = desc->dtype == RT_F64 ? 8 : 4;
    void *raw = nullptr;
    cudaStream_t st = nullptr;
    auto cleanup = [&](rt_err code) {
        if (st) cudaStreamDestroy(st);
        if (raw) cudaFree(raw);
        if (code != RT_OK) {
            cudaFree(g->pad64);
            cudaFree(g->pad32);
            cudaFree(g->quad);
            cudaFree(g->table);
            delete g;
        }
        return code;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&raw, n_raw * esz);
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->pad64, n_pad * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->pad32, n_pad * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->quad, n_quad * sizeof(float4));
    if (e == cudaSuccess && n_tab) e = cudaMalloc((void **)&g->table, n_tab * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemcpyAsync(raw, ne_host, n_raw * esz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        GridSizes sz{desc->n_lat, desc->n_lon, desc->n_alt};
        e = launch_grid_prep(raw, desc->dtype, sz, g->pad64, g->pad32, g->quad, g->table, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "rt_grid_create"));
    g->bytes = n_pad * (sizeof(double) + sizeof(float)) + n_quad * sizeof(float4) + n_tab * sizeof(float4);
    GridDev &d = g->g;
    d.n_lat = desc->n_lat;
    d.n_lon = desc->n_lon;
    d.n_alt = desc->n_alt;
    d.p_lon = desc->n_lon + 2;
    d.p_alt = desc->n_alt + 2;
    d.q_alt = desc->n_alt - 1;
    d.lat0 = desc->lat0_deg;
    d.lon0 = desc->lon0_deg;
    d.alt0 = desc->alt0_km;
    d.inv_dlat = 1.0 / desc->dlat_deg;
    d.inv_dlon = 1.0 / desc->dlon_deg;
    d.inv_dalt = 1.0 / desc->dalt_km;
    d.R_E = desc->earth_radius_km;
    d.top = desc->alt0_km + (desc->n_alt - 1) * desc->dalt_km;
    d.b0 = desc->field.b0_tesla;
    const double plat = desc->field.pole_lat_deg * kDeg2Rad, plon = desc->field.pole_lon_deg * kDeg2Rad;
    d.m[0] = std::cos(plat) * std::cos(plon);
    d.m[1] = std::cos(plat) * std::sin(plon);
    d.m[2] = std::sin(plat);
    d.sa = (float)(-kRad2Deg / desc->dlat_deg);
    d.sb = (float)(kRad2Deg / desc->dlon_deg);
    d.sc = (float)(1.0 / desc->dalt_km);
    d.R_Ef = (float)d.R_E;
    d.mf[0] = (float)d.m[0];
    d.mf[1] = (float)d.m[1];
    d.mf[2] = (float)d.m[2];
    d.top_f = (float)d.top;
    d.iso = d.b0 == 0.0 ? 1 : 0;
    d.interp = (desc->flags & RT_GRID_CATMULL_ROM) ? 1 : 0;
    d.pad64 = g->pad64;
    d.pad32 = g->pad32;
    d.quad = g->quad;
    d.table = g->table;
    *out = g;
    return cleanup(RT_OK);
}

rt_err rt_grid_destroy(rt_grid *grid) {
    if (!grid) return RT_OK;
    cudaError_t e = cudaSuccess;
    for (void *p : {(void *)grid->pad64, (void *)grid->pad32, (void *)grid->quad, (void *)grid->table}) {
        if (!p) continue;
        const cudaError_t ei = cudaFree(p);
        if (ei != cudaSuccess && e == cudaSuccess) e = ei;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto it = g_tuned.begin(); it != g_tuned.end();) {
            if (std::get<0>(it->first) == grid) it = g_tuned.erase(it);
            else ++it;
        }
    }
    delete grid;
    if (e != cudaSuccess) return cuda_fail(e, "rt_grid_destroy");
    return RT_OK;
}

size_t rt_grid_device_bytes(const rt_grid *grid) { return grid ? grid->bytes : 0; }

rt_err rt_trace_device(const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_dev, size_t out_len,
                       const rt_launch_config *cfg, void *stream) {
    return queue_trace(grid, fan, out_dev, out_len, cfg, (cudaStream_t)stream);
}

rt_err rt_trace_fans_device(const rt_grid *grid, const rt_fan_desc *const *fans, int32_t n_fans,
                            rt_ray_result *out_dev, size_t out_len, const rt_launch_config *cfg, void *stream) {
    if (n_fans < 1 || n_fans > 4096) return fail(RT_EINVAL, "n_fans must be in 1..4096 (got %d)", n_fans);
    if (!fans) return fail(RT_EINVAL, "fans is NULL");
    for (int k = 0; k < n_fans; ++k)
        if (!fans[k]) return fail(RT_EINVAL, "fans[%d] is NULL", k);
    if (cfg && cfg->kernel != RT_KERNEL_AUTO && cfg->kernel != RT_KERNEL_PLAIN)
        return fail(RT_EINVAL, "rt_trace_fans_device runs a plain kernel (cfg->kernel AUTO or PLAIN)");
    if (cfg && cfg->lanes_per_ray != 0 && cfg->lanes_per_ray != 4)
        return fail(RT_EINVAL, "rt_trace_fans_device runs four lanes per ray (cfg->lanes_per_ray 0 or 4)");
    return rtgd_queue_trace_fans(grid, fans, n_fans, out_dev, out_len, cfg, (cudaStream_t)stream);
}

rt_err rt_trace(const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_host, size_t out_len,
                const rt_launch_config *cfg, void *stream) {
    if (!out_host) return fail(RT_EINVAL, "out_host is NULL");
    rt_err r = validate_fan(fan);
    if (r != RT_OK) return r;
    if ((r = ensure_device(nullptr)) != RT_OK) return r;
    const size_t n = fan_rays(fan);
    if (out_len < n) return fail(RT_EINVAL, "out_len %zu < %zu rays", out_len, n);
    cudaStream_t st = (cudaStream_t)stream;
    rt_ray_result *dev = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&dev, n * sizeof(rt_ray_result), st));
    r = queue_trace(grid, fan, dev, n, cfg, st);
    // The bounded wait covers the trace.  The copy into out_host is queued
    // only once the trace has finished, and waited for without a deadline (a
    // copy of finished records), so that a call returning RT_ETIMEOUT has
    // queued no write into out_host: the caller's buffer is free on return
    // whatever the status.
    if (r == RT_OK) r = sync_with_timeout(st);
    if (r == RT_OK) {
        cudaError_t e = cudaMemcpyAsync(out_host, dev, n * sizeof(rt_ray_result), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = cuda_fail(e, "result copy");
    }
    const cudaError_t e2 = cudaFreeAsync(dev, st);
    if (r == RT_OK && e2 != cudaSuccess) r = cuda_fail(e2, "cudaFreeAsync");
    return r;
}

rt_err rt_tune(const rt_grid *grid, const rt_fan_desc *fan, size_t max_rays, void *stream, rt_launch_config *best,
               float *best_ms) {
    if (!grid || !best) return fail(RT_EINVAL, "NULL argument");
    rt_err r = validate_fan(fan);
    if (r != RT_OK) return r;
    if ((r = ensure_device(nullptr)) != RT_OK) return r;
    if (max_rays == 0) max_rays = 65536;
    cudaStream_t st = (cudaStream_t)stream;
    // A fan of at least two waves of resident lanes at one lane per ray is
    // bound by issue throughput, where splitting a ray over lanes only
    // duplicates work, and a sub-fan of about one wave would instead reward
    // the latency of its slowest rays.  Such fans are timed on a sub-fan of at
    // least four waves, with one lane per ray.
    int occ = 0;
    CUDA_TRY(persistent_occupancy(RT_STENCIL_QUAD, 1, 128, &occ));
    const long long resident = (long long)props(grid->device).sms * std::max(occ, 1) * 128;
    const bool throughput = fan->precision == RT_MIXED && (long long)fan_rays(fan) >= 2 * resident;
    if (throughput) max_rays = std::max(max_rays, (size_t)(4 * resident));
    // strided sub-fan with at most max_rays rays (every k-th elevation, azimuth, frequency)
    std::vector<double> fr(fan->freq_mhz, fan->freq_mhz + fan->n_freq), el(fan->el_deg, fan->el_deg + fan->n_el),
        az(fan->az_deg, fan->az_deg + fan->n_az);
    auto thin = [](std::vector<double> &v) {
        std::vector<double> o;
        for (size_t i = 0; i < v.size(); i += 2) o.push_back(v[i]);
        v.swap(o);
    };
    rt_fan_desc sub = *fan;
    for (int guard = 0; guard < 64; ++guard) {
        sub.freq_mhz = fr.data();
        sub.el_deg = el.data();
        sub.az_deg = az.data();
        sub.n_freq = (int)fr.size();
        sub.n_el = (int)el.size();
        sub.n_az = (int)az.size();
        if (fan_rays(&sub) <= max_rays) break;
        if (el.size() >= az.size() && el.size() > 1) thin(el);
        else if (az.size() > 1) thin(az);
        else if (fr.size() > 1) thin(fr);
        else break;
    }
    const size_t n = fan_rays(&sub);
    std::vector<rt_launch_config> cands;
    rt_launch_config c;
    std::memset(&c, 0, sizeof(c));
    if (fan->precision == RT_FP64) {
        c.kernel = RT_KERNEL_PLAIN;
        cands.push_back(c);
    } else {
        for (int kernel : {RT_KERNEL_PLAIN, RT_KERNEL_PERSISTENT})
            for (int stencil : {RT_STENCIL_GATHER, RT_STENCIL_QUAD, RT_STENCIL_TABLE})
                for (int order : {RT_ORDER_CANONICAL, RT_ORDER_ELEVATION_FASTEST})
                    for (int lanes : {1, 2, 4})
                        for (int threads : {32, 64, 96, 128}) {
                        if (throughput && lanes > 1) continue;
                        if (stencil == RT_STENCIL_TABLE && !grid->table) continue;
                        c.kernel = kernel;
                        c.stencil = stencil;
                        c.order = order;
                        c.block_threads = threads;
                        c.lanes_per_ray = lanes;
                        cands.push_back(c);
                    }
    }
    rt_ray_result *out = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&out, n * sizeof(rt_ray_result), st));
    // Each timed launch starts from a cold L2 (a 256 MiB fill evicts the
    // ~126 MB L2), as a fan does when its grid was not just traced: with a warm
    // L2 the kernels rank differently.
    const size_t flush_bytes = (size_t)256 << 20;
    void *flush = nullptr;
    if (cudaMallocAsync(&flush, flush_bytes, st) != cudaSuccess) {
        cudaFreeAsync(out, st);
        return fail(RT_ENOMEM, "rt_tune: no device memory for the L2 flush buffer");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // one timed launch of candidate cc from a cold L2 (ms; < 0 on failure)
    auto time_once = [&](const rt_launch_config &cc, int rep) -> float {
        cudaMemsetAsync(flush, rep & 0xff, flush_bytes, st);
        cudaEventRecord(e0, st);
        r = queue_trace(grid, &sub, out, n, &cc, st);
        cudaEventRecord(e1, st);
        if (r == RT_OK) r = sync_with_timeout(st);
        float ms = 0.0f;
        if (r != RT_OK || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0f;
        return ms;
    };
    auto median = [](std::vector<float> ts) {
        std::sort(ts.begin(), ts.end());
        return ts[ts.size() / 2];
    };
    std::vector<std::pair<float, size_t>> timed;  // (median ms, candidate index)
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        const auto &cc = cands[ci];
        if ((r = queue_trace(grid, &sub, out, n, &cc, st)) != RT_OK) break;  // warm-up
        // median of three timed launches: a launch whose slowest ray happened to
        // share its SM with little other work must not decide the choice
        std::vector<float> ts;
        for (int rep = 0; rep < 3 && r == RT_OK; ++rep) {
            const float ms = time_once(cc, rep);
            if (ms >= 0.0f) ts.push_back(ms);
        }
        if (r != RT_OK) break;
        if (!ts.empty()) timed.emplace_back(median(ts), ci);
    }
    // the best few again, in interleaved rounds (clock and neighbour drift
    // then touch them alike), seven launches each: candidates within a few
    // per cent of each other are otherwise ranked by noise
    float best_t = 1e30f;
    rt_launch_config best_c = cands[0];
    if (r == RT_OK && !timed.empty()) {
        std::sort(timed.begin(), timed.end());
        const size_t k = std::min<size_t>(timed.size(), 4);
        std::vector<std::vector<float>> ts(k);
        for (int round = 0; round < 7 && r == RT_OK; ++round)
            for (size_t j = 0; j < k && r == RT_OK; ++j) {
                const float ms = time_once(cands[timed[j].second], round);
                if (ms >= 0.0f) ts[j].push_back(ms);
            }
        for (size_t j = 0; j < k && r == RT_OK; ++j) {
            const float t = ts[j].empty() ? timed[j].first : median(ts[j]);
            if (t < best_t) {
                best_t = t;
                best_c = cands[timed[j].second];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    cudaFreeAsync(flush, st);
    if (r != RT_OK) return r;
    if (fan->precision == RT_MIXED) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[std::make_tuple(grid, fan->integrator, ray_bucket(fan_rays(fan)))] = best_c;
    }
    *best = best_c;
    if (best_ms) *best_ms = best_t;
    return RT_OK;
}

struct rt_plan {
    const rt_grid *grid = nullptr;
    FanDev f;
    LaunchPlan lp;
    size_t n = 0;
    char *ws = nullptr;  // ray counter (16 B) + fan tables
    // longest-first order (rt_plan_order): claim order over all rays, the
    // first n_long_claims of which (n_long rays, and holes when each has a
    // warp of its own) run in a four-lane launch on the side stream
    int *perm = nullptr;
    int32_t *evals = nullptr;  // the costs of the last rt_plan_order, gathered on the device
    size_t n_long = 0, n_long_claims = 0;
    LaunchPlan lp_long;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t started = nullptr;  // all blocks of the four-lane launch have begun
};

rt_err rt_plan_create(const rt_grid *grid, const rt_fan_desc *fan, const rt_launch_config *cfg, rt_plan **out) {
    if (!out) return fail(RT_EINVAL, "out is NULL");
    *out = nullptr;
    rt_err r = validate_fan(fan);
    if (r != RT_OK) return r;
    if (!grid) return fail(RT_EINVAL, "grid is NULL");
    int dev = 0;
    if ((r = ensure_device(&dev)) != RT_OK) return r;
    if (dev != grid->device) return fail(RT_EINVAL, "grid lives on device %d, current device is %d", grid->device, dev);
    const size_t n = fan_rays(fan);
    if (n >= ((size_t)1 << 31)) return fail(RT_EINVAL, "fan too large (at most 2^31 - 1 rays)");
    rt_plan *p = new rt_plan();
    int order = 0;
    if ((r = make_plan(grid, fan, n, cfg, &p->lp, &order)) != RT_OK) {
        delete p;
        return r;
    }
    const std::vector<char> img = fan_image(grid, fan);
    cudaError_t e = cudaMalloc((void **)&p->ws, img.size());
    double *tab = (double *)(p->ws + 16);
    if (e == cudaSuccess) e = cudaMemcpy(p->ws, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->ws);
        delete p;
        return cuda_fail(e, "rt_plan_create");
    }
    p->grid = grid;
    p->n = n;
    p->f = fill_fandev(grid, fan, n, order, tab);
    *out = p;
    return RT_OK;
}

size_t rt_plan_rays(const rt_plan *plan) { return plan ? plan->n : 0; }

rt_err rt_plan_execute(const rt_plan *plan, rt_ray_result *out_dev, size_t out_len, void *stream) {
    if (!plan || !out_dev) return fail(RT_EINVAL, "NULL argument");
    if (out_len < plan->n) return fail(RT_EINVAL, "out_len %zu < %zu rays", out_len, plan->n);
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(plan->ws, 0, 16, st));
    if (!plan->perm) {
        CUDA_TRY(launch_trace(plan->grid->g, plan->f, out_dev, (unsigned long long *)plan->ws, plan->lp, st));
        return RT_OK;
    }
    // ordered: the n_long most expensive rays at four lanes each on the side
    // stream (forked from and joined back to `stream`, so the two launches
    // run concurrently and a capture of `stream` records both), the rest in
    // descending cost order on `stream`
    FanDev fl = plan->f, fb = plan->f;
    fl.perm = fb.perm = plan->perm;
    fl.perm_off = 0;
    fl.n_rays = (long long)plan->n_long_claims;
    fb.perm_off = (long long)plan->n_long_claims;
    fb.n_rays = (long long)(plan->n - plan->n_long);
    if (plan->n_long > 0) {
        CUDA_TRY(cudaEventRecord(plan->fork, st));
        CUDA_TRY(cudaStreamWaitEvent(plan->side, plan->fork, 0));
        CUDA_TRY(launch_trace_only(plan->grid->g, fl, out_dev, nullptr, plan->lp_long, plan->side));
        CUDA_TRY(cudaEventRecord(plan->join, plan->side));
        // SMs of their own for the four-lane blocks: the other rays' blocks
        // wait until all of those have begun (else they could take every SM
        // first and the four-lane blocks would wait for whole SMs to drain)
        if (plan->lp_long.started) CUDA_TRY(cudaStreamWaitEvent(st, plan->lp_long.started, 0));
    }
    CUDA_TRY(launch_trace_only(plan->grid->g, fb, out_dev, (unsigned long long *)plan->ws, plan->lp, st));
    if (plan->n_long > 0) CUDA_TRY(cudaStreamWaitEvent(st, plan->join, 0));
    CUDA_TRY(launch_finish(plan->grid->g, plan->f, out_dev, (long long)plan->n, st));
    return RT_OK;
}

// Warps per block of an exclusive four-lane share (RT_PLAN_LONG_EXCLUSIVE):
// two warps on an SM of their own run as fast as one (C2 fan: 11.10 against
// 11.07 ms) and take half the SMs.
constexpr int kExclusiveWarps = 2;

// The claim list of a longest-first order (rt_order_claims, which
// rt_plan_order calls): host arithmetic only.
static void order_claims(std::vector<int32_t> ev, size_t n, long long n_f, long long n_m, long long n_e,
                         long long n_a, int claim_order, int32_t spread, double long_factor, bool mixed,
                         uint32_t flags, int sm_count, std::vector<int> &perm, size_t &nl, size_t &nc) {
    // expected cost: the largest cost within `spread` elevation and frequency
    // steps of the same mode and azimuth (canonical order [freq][mode][el][az])
    std::vector<int32_t> cost;
    if (spread == 0) {
        cost.swap(ev);
    } else {
        std::vector<int32_t> tmp(n);
        cost.resize(n);
        // elevation, then frequency: the maximum over a window of each line
        // of the canonical array, whose elements lie `stride` apart (whole
        // rows at once where the lines are far apart)
        auto dilate = [&](const std::vector<int32_t> &in, std::vector<int32_t> &out, long long len,
                          long long stride, long long outer) {
            for (long long o = 0; o < outer; ++o) {
                const int32_t *src = in.data() + o * len * stride;
                int32_t *dst = out.data() + o * len * stride;
                for (long long x = 0; x < len; ++x) {
                    const long long lo = std::max(0LL, x - spread), hi = std::min(len - 1, x + (long long)spread);
                    int32_t *row = dst + x * stride;
                    if (stride == 1) {
                        int32_t v = src[lo];
                        for (long long d = lo + 1; d <= hi; ++d) v = std::max(v, src[d]);
                        *row = v;
                        continue;
                    }
                    std::copy(src + lo * stride, src + (lo + 1) * stride, row);
                    for (long long d = lo + 1; d <= hi; ++d) {
                        const int32_t *sr = src + d * stride;
                        for (long long k = 0; k < stride; ++k) row[k] = std::max(row[k], sr[k]);
                    }
                }
            }
        };
        dilate(ev, tmp, n_e, n_a, n_f * n_m);
        dilate(tmp, cost, n_f, n_m * n_e * n_a, 1);
    }
    // descending cost, eight buckets per octave (rays of one bucket keep
    // their canonical order, so neighbours stay together): a counting sort on
    // the key floor(8 log2 cost), found with integer comparisons against
    // ceil(2^(e + j/8)) for the cost's octave e
    static const std::vector<uint64_t> kThr = [] {
        std::vector<uint64_t> t(32 * 8);
        for (int e = 0; e < 32; ++e)
            for (int j = 0; j < 8; ++j) t[e * 8 + j] = (uint64_t)std::ceil(std::exp2((double)e + j / 8.0));
        return t;
    }();
    auto key = [](int32_t c) {
        const uint32_t u = (uint32_t)std::max(c, 1);
        const int e = 31 - __builtin_clz(u);  // floor(log2 u)
        int k = 8 * e;
        for (int j = 1; j < 8; ++j) k += (uint64_t)u >= kThr[e * 8 + j];
        return k;
    };
    constexpr int kKeys = 8 * 32;
    std::vector<uint8_t> keys(n);
    std::vector<size_t> start(kKeys + 1, 0);
    for (size_t i = 0; i < n; ++i) {
        keys[i] = (uint8_t)key(cost[i]);
        ++start[kKeys - 1 - keys[i] + 1];
    }
    for (int k = 0; k < kKeys; ++k) start[k + 1] += start[k];
    perm.assign(n, 0);
    for (size_t i = 0; i < n; ++i) perm[start[kKeys - 1 - keys[i]]++] = (int)i;
    // the four-lane share: rays whose expected cost is at least long_factor
    // times the median (mixed path only), at most a sixteenth of the rays
    nl = 0;
    if (long_factor > 0.0 && mixed) {
        // the median cost (the element of rank n/2): a radix select over the
        // upper, then the lower 16 bits of the (non-negative) costs
        std::vector<size_t> hist(1 << 16);
        for (size_t i = 0; i < n; ++i) ++hist[(uint32_t)std::max(cost[i], 0) >> 16];
        size_t rank = n / 2, hi = 0;
        while (rank >= hist[hi]) rank -= hist[hi++];
        std::fill(hist.begin(), hist.end(), 0);
        for (size_t i = 0; i < n; ++i) {
            const uint32_t u = (uint32_t)std::max(cost[i], 0);
            if ((u >> 16) == hi) ++hist[u & 0xFFFFu];
        }
        size_t lo = 0;
        while (rank >= hist[lo]) rank -= hist[lo++];
        const double median = (double)((hi << 16) | lo);
        const double thr = long_factor * median;
        while (nl < n / 16 && (double)cost[perm[nl]] >= thr) ++nl;
    }
    if ((flags & RT_PLAN_LONG_EXCLUSIVE) && nl > 0) {
        // blocks of kExclusiveWarps warps on SMs of their own: at most an
        // eighth of the SMs, so that a cost estimate that marks too many
        // rays does not take the GPU from the rest of the scan
        const size_t per_block = ((flags & RT_PLAN_LONG_ALONE) ? 1 : 32 / 4) * (size_t)kExclusiveWarps;
        nl = std::min(nl, (size_t)std::max(sm_count / 8, 1) * per_block);
    }
    if (nl > 1) {
        // the four-lane share in the plan's claim order: neighbouring rays of
        // one trace share a warp (rays of similar cost from all over the scan
        // would wait for one another's branches and gathers at every attempt)
        auto claim_of = [&](long long ray) {
            if (claim_order != RT_ORDER_ELEVATION_FASTEST) return ray;
            const long long a = ray % n_a, e = (ray / n_a) % n_e, fm = ray / (n_a * n_e);
            return (fm * n_a + a) * n_e + e;
        };
        std::sort(perm.begin(), perm.begin() + (long long)nl,
                  [&](int x, int y) { return claim_of(x) < claim_of(y); });
    }
    if (flags & RT_PLAN_REST_IN_PLAN_ORDER) {
        // the other rays in the plan's own claim order
        std::vector<char> is_long(n, 0);
        for (size_t i = 0; i < nl; ++i) is_long[perm[i]] = 1;
        const char *in_share = is_long.data();
        int *out = perm.data() + nl;
        if (claim_order == RT_ORDER_ELEVATION_FASTEST) {  // as the kernels' claim_to_ray
            for (long long fm = 0; fm < n_f * n_m; ++fm)
                for (long long a = 0; a < n_a; ++a)
                    for (long long e = 0; e < n_e; ++e) {
                        const long long ray = (fm * n_e + e) * n_a + a;
                        if (!in_share[ray]) *out++ = (int)ray;
                    }
        } else {
            for (long long ray = 0; ray < (long long)n; ++ray)
                if (!in_share[ray]) *out++ = (int)ray;
        }
    }
    nc = nl;
    if ((flags & RT_PLAN_LONG_ALONE) && nl > 0) {
        // a warp per ray in the four-lane launch: each ray's group of four
        // lanes is followed by seven holes
        constexpr size_t kGroups = 32 / 4;
        std::vector<int> claims(nl * kGroups + (n - nl), -1);
        for (size_t i = 0; i < nl; ++i) claims[i * kGroups] = perm[i];
        std::copy(perm.begin() + (long long)nl, perm.end(), claims.begin() + (long long)(nl * kGroups));
        nc = nl * kGroups;
        perm.swap(claims);
    }
}


rt_err rt_plan_order(rt_plan *plan, const rt_ray_result *cost_dev, int32_t spread, double long_factor,
                     uint32_t flags, size_t *n_long, void *stream) {
    if (!plan) return fail(RT_EINVAL, "plan is NULL");
    if (spread < 0 || spread > 64) return fail(RT_EINVAL, "spread must be in 0..64");
    if (flags & ~(uint32_t)(RT_PLAN_REST_IN_PLAN_ORDER | RT_PLAN_LONG_EXCLUSIVE | RT_PLAN_LONG_ALONE))
        return fail(RT_EINVAL, "unknown flags 0x%x", flags);
    if (!std::isfinite(long_factor)) return fail(RT_EINVAL, "long_factor must be finite");
    if (n_long) *n_long = 0;
    if (!cost_dev) {  // back to the plan's own order
        if (plan->perm) cudaFree(plan->perm);
        plan->perm = nullptr;
        plan->n_long = plan->n_long_claims = 0;
        return RT_OK;
    }
    const size_t n = plan->n;
    cudaStream_t st = (cudaStream_t)stream;
    // the n_evals field of every record, gathered on the device into the
    // plan's cost array and copied back in one piece
    if (!plan->evals) CUDA_TRY(cudaMalloc((void **)&plan->evals, n * sizeof(int32_t)));
    CUDA_TRY(launch_gather_evals(cost_dev, plan->evals, (long long)n, st));
    std::vector<int32_t> ev(n);
    CUDA_TRY(cudaMemcpyAsync(ev.data(), plan->evals, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    rt_err r = sync_with_timeout(st);
    if (r != RT_OK) return r;
    std::vector<int> perm;
    size_t nl = 0, nc = 0;
    int sms = 0;
    if (flags & RT_PLAN_LONG_EXCLUSIVE)
        CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->grid->device));
    const FanDev &f = plan->f;
    order_claims(std::move(ev), n, f.n_freq, f.n_modes, f.n_el, f.n_az, f.order, spread, long_factor,
                 f.precision == RT_MIXED, flags, sms, perm, nl, nc);
    // capacity for the largest claim list: n rays plus 7 holes for each of at
    // most n / 16 four-lane rays
    if (!plan->perm) CUDA_TRY(cudaMalloc((void **)&plan->perm, (n + 7 * (n / 16)) * sizeof(int)));
    CUDA_TRY(cudaMemcpy(plan->perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!plan->side) {
        int lo = 0, hi = 0;
        CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        // the four-lane launch gets the highest priority: when both launches
        // have blocks waiting, an SM that frees up takes one of its blocks
        CUDA_TRY(cudaStreamCreateWithPriority(&plan->side, cudaStreamNonBlocking, hi));
        CUDA_TRY(cudaEventCreateWithFlags(&plan->fork, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&plan->join, cudaEventDisableTiming));
    }
    LaunchPlan ll = plan->lp;
    ll.kernel = RT_KERNEL_PLAIN;
    ll.lanes = 4;
    ll.blocks = 0;
    ll.smem = 0;
    if ((flags & RT_PLAN_LONG_EXCLUSIVE) && nl > 0) {
        // blocks of kExclusiveWarps warps, each block alone on its SM
        ll.threads = 32 * kExclusiveWarps;
        CUDA_TRY(plain_exclusive_smem(ll, plan->grid->g.interp, &ll.smem));
        if (!plan->started) CUDA_TRY(cudaEventCreateWithFlags(&plan->started, cudaEventDisableTiming));
        ll.started = plan->started;
    }
    plan->n_long = nl;
    plan->n_long_claims = nc;
    plan->lp_long = ll;
    if (n_long) *n_long = nl;
    return RT_OK;
}

rt_err rt_order_claims(const int32_t *cost, int32_t n_freq, int32_t n_modes, int32_t n_el, int32_t n_az,
                       int32_t claim_order, int32_t spread, double long_factor, int32_t mixed, uint32_t flags,
                       int32_t sm_count, int32_t *claims, size_t claims_cap, size_t *n_long, size_t *n_claims) {
    if (!cost || !claims) return fail(RT_EINVAL, "NULL argument");
    if (n_freq < 1 || n_modes < 1 || n_modes > 2 || n_el < 1 || n_az < 1)
        return fail(RT_EINVAL, "bad fan dimensions %d x %d x %d x %d", n_freq, n_modes, n_el, n_az);
    const size_t n = (size_t)n_freq * (size_t)n_modes * (size_t)n_el * (size_t)n_az;
    if (n >= ((size_t)1 << 31)) return fail(RT_EINVAL, "too many rays (at most 2^31 - 1)");
    if (claim_order != RT_ORDER_CANONICAL && claim_order != RT_ORDER_ELEVATION_FASTEST)
        return fail(RT_EINVAL, "unknown claim order %d", claim_order);
    if (spread < 0 || spread > 64) return fail(RT_EINVAL, "spread must be in 0..64");
    if (flags & ~(uint32_t)(RT_PLAN_REST_IN_PLAN_ORDER | RT_PLAN_LONG_EXCLUSIVE | RT_PLAN_LONG_ALONE))
        return fail(RT_EINVAL, "unknown flags 0x%x", flags);
    if (!std::isfinite(long_factor)) return fail(RT_EINVAL, "long_factor must be finite");
    if ((flags & RT_PLAN_LONG_EXCLUSIVE) && sm_count < 1) return fail(RT_EINVAL, "sm_count must be positive");
    std::vector<int> perm;
    size_t nl = 0, nc = 0;
    order_claims(std::vector<int32_t>(cost, cost + n), n, n_freq, n_modes, n_el, n_az, claim_order, spread,
                 long_factor, mixed != 0, flags, sm_count, perm, nl, nc);
    if (claims_cap < perm.size()) return fail(RT_EINVAL, "claims_cap %zu < %zu claims", claims_cap, perm.size());
    std::copy(perm.begin(), perm.end(), claims);
    if (n_long) *n_long = nl;
    if (n_claims) *n_claims = perm.size();
    return RT_OK;
}

rt_err rt_plan_destroy(rt_plan *plan) {
    if (!plan) return RT_OK;
    cudaError_t e = cudaFree(plan->ws);
    if (plan->perm) cudaFree(plan->perm);
    if (plan->evals) cudaFree(plan->evals);
    if (plan->side) cudaStreamDestroy(plan->side);
    if (plan->fork) cudaEventDestroy(plan->fork);
    if (plan->join) cudaEventDestroy(plan->join);
    if (plan->started) cudaEventDestroy(plan->started);
    delete plan;
    if (e != cudaSuccess) return cuda_fail(e, "rt_plan_destroy");
    return RT_OK;
}

rt_err rt_ionogram(const rt_grid *grid, const rt_ionogram_desc *d, rt_ionogram_point *out_host, size_t cap,
                   size_t *n_points, const rt_launch_config *cfg, void *stream) {
    if (!grid || !d || !n_points || (cap > 0 && !out_host)) return fail(RT_EINVAL, "NULL argument");
    *n_points = 0;
    if (!std::isfinite(d->rx_lat_deg) || !std::isfinite(d->rx_lon_deg) || d->rx_lat_deg <= -90.0 ||
        d->rx_lat_deg >= 90.0)
        return fail(RT_EINVAL, "receiver position must be finite with |lat| < 90");
    for (int i = 1; i < d->n_el && d->el_deg; ++i)
        if (!(d->el_deg[i] > d->el_deg[i - 1])) return fail(RT_EINVAL, "el_deg must be ascending");
    // great-circle distance and initial bearing transmitter -> receiver
    const double p1 = d->tx_lat_deg * kDeg2Rad, p2 = d->rx_lat_deg * kDeg2Rad;
    const double dl = (d->rx_lon_deg - d->tx_lon_deg) * kDeg2Rad;
    const double x = std::cos(p1) * std::sin(p2) - std::sin(p1) * std::cos(p2) * std::cos(dl);
    const double yv = std::sin(dl) * std::cos(p2);
    const double c = std::sin(p1) * std::sin(p2) + std::cos(p1) * std::cos(p2) * std::cos(dl);
    const double ang = std::atan2(std::sqrt(x * x + yv * yv), c);
    if (!(ang > 0.0)) return fail(RT_EINVAL, "receiver coincides with the transmitter");
    const double d_rx = grid->desc.earth_radius_km * ang;
    const double az = std::atan2(yv, x) * kRad2Deg;
    rt_fan_desc fan;
    std::memset(&fan, 0, sizeof(fan));
    fan.tx_lat_deg = d->tx_lat_deg;
    fan.tx_lon_deg = d->tx_lon_deg;
    fan.tx_alt_km = d->tx_alt_km;
    fan.freq_mhz = d->freq_mhz;
    fan.el_deg = d->el_deg;
    fan.az_deg = &az;
    fan.n_freq = d->n_freq;
    fan.n_el = d->n_el;
    fan.n_az = 1;
    fan.modes = d->modes;
    fan.integrator = d->integrator;
    fan.precision = d->precision;
    fan.h_km = d->h_km;
    fan.rtol = d->rtol;
    fan.atol_km = d->atol_km;
    fan.h_min_km = d->h_min_km;
    fan.h_max_km = d->h_max_km;
    fan.max_steps = d->max_steps;
    rt_err r = validate_fan(&fan);
    if (r != RT_OK) return r;
    if ((r = ensure_device(nullptr)) != RT_OK) return r;
    const size_t n = fan_rays(&fan);
    const int n_modes = ((d->modes & RT_MODE_O) ? 1 : 0) + ((d->modes & RT_MODE_X) ? 1 : 0);
    // the reduction can emit at most (n_el - 1) points per trace
    const size_t max_pts = (size_t)d->n_freq * n_modes * (size_t)(d->n_el > 1 ? d->n_el - 1 : 0);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t tab = (size_t)d->n_freq + d->n_el;
    const size_t bytes = 16 + tab * sizeof(double) + n * sizeof(rt_ray_result) + max_pts * sizeof(rt_ionogram_point);
    char *ws = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&ws, bytes, st));
    unsigned long long *count = (unsigned long long *)ws;
    double *tf = (double *)(ws + 16);
    rt_ray_result *res = (rt_ray_result *)(tf + tab);
    rt_ionogram_point *pts = (rt_ionogram_point *)(res + n);
    cudaError_t e = cudaMemsetAsync(count, 0, 16, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tf, d->freq_mhz, d->n_freq * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tf + d->n_freq, d->el_deg, d->n_el * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(ws, st);
        return cuda_fail(e, "rt_ionogram");
    }
    r = queue_trace(grid, &fan, res, n, cfg, st);
    if (r == RT_OK) {
        e = launch_ionogram(res, tf, tf + d->n_freq, d->n_freq, n_modes, (d->modes & RT_MODE_O) ? 1 : -1, d->n_el,
                            d_rx, pts, max_pts, count, st);
        if (e != cudaSuccess) r = cuda_fail(e, "ionogram kernel");
    }
    unsigned long long total = 0;
    std::vector<rt_ionogram_point> hp;
    if (r == RT_OK) r = sync_with_timeout(st);
    if (r == RT_OK) {
        e = cudaMemcpy(&total, count, sizeof(total), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && total > 0) {
            hp.resize((size_t)std::min<unsigned long long>(total, max_pts));
            e = cudaMemcpy(hp.data(), pts, hp.size() * sizeof(rt_ionogram_point), cudaMemcpyDeviceToHost);
        }
        if (e != cudaSuccess) r = cuda_fail(e, "ionogram copy");
    }
    cudaFreeAsync(ws, st);
    if (r != RT_OK) return r;
    // deterministic order and branch numbers: (frequency, mode O first, elevation)
    std::sort(hp.begin(), hp.end(), [](const rt_ionogram_point &a, const rt_ionogram_point &b) {
        if (a.freq_mhz != b.freq_mhz) return a.freq_mhz < b.freq_mhz;
        if (a.mode != b.mode) return a.mode > b.mode;
        return a.el_deg < b.el_deg;
    });
    for (size_t i = 0; i < hp.size(); ++i) {
        const bool same = i > 0 && hp[i].freq_mhz == hp[i - 1].freq_mhz && hp[i].mode == hp[i - 1].mode;
        hp[i].branch = same ? hp[i - 1].branch + 1 : 0;
    }
    const size_t w = std::min(cap, hp.size());
    if (w) std::memcpy(out_host, hp.data(), w * sizeof(rt_ionogram_point));
    *n_points = hp.size();
    return RT_OK;
}

}  // extern "C"

namespace {
// Host staging of rt_trace_device_noalloc's fan image (fixed size, no allocation).
std::mutex g_noalloc_img_mu;
char g_noalloc_img[kNoallocScratchBytes];
}  // namespace

extern "C" {

rt_err rt_trace_device_noalloc(const rt_grid *grid, const rt_fan_desc *fan, rt_ray_result *out_dev,
                               size_t out_len, const rt_launch_config *cfg, void *stream) {
    rt_err r = validate_fan(fan);
    if (r != RT_OK) return r;
    if (!grid) return fail(RT_EINVAL, "grid is NULL");
    if (!out_dev) return fail(RT_EINVAL, "output pointer is NULL");
    int dev = 0;
    if ((r = ensure_device(&dev)) != RT_OK) return r;
    if (dev != grid->device) return fail(RT_EINVAL, "grid lives on device %d, current device is %d", grid->device, dev);
    const size_t n = fan_rays(fan);
    if (out_len < n) return fail(RT_EINVAL, "out_len %zu < %zu rays", out_len, n);
    if (n >= ((size_t)1 << 31)) return fail(RT_EINVAL, "fan too large (at most 2^31 - 1 rays)");
    const size_t n_tab = (size_t)fan->n_freq + fan->n_el + fan->n_az;
    if (n_tab > (size_t)kNoallocMaxTable)
        return fail(RT_EINVAL, "rt_trace_device_noalloc: n_freq + n_el + n_az = %zu exceeds the fixed scratch of %d entries",
                    n_tab, kNoallocMaxTable);
    LaunchPlan lp;
    int order = 0;
    if ((r = make_plan(grid, fan, n, cfg, &lp, &order)) != RT_OK) return r;
    void *scratch = nullptr;
    size_t cap = 0;
    CUDA_TRY(noalloc_scratch(dev, &scratch, &cap));
    if (fan_image_bytes(fan) > cap) return fail(RT_EINVAL, "fan tables exceed the fixed scratch");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *counter = (unsigned long long *)scratch;
    double *tab = (double *)((char *)scratch + 16);
    // one copy of the fan image: its leading 16 zero bytes reset the ray
    // counter (the array keeps the last call's contents), the tables follow.
    // The image is staged in a fixed host array (no allocation) that the
    // lock keeps to one call at a time until cudaMemcpyAsync has read it.
    {
        std::lock_guard<std::mutex> lk(g_noalloc_img_mu);
        fan_image_into(grid, fan, g_noalloc_img);
        CUDA_TRY(cudaMemcpyAsync(scratch, g_noalloc_img, fan_image_bytes(fan), cudaMemcpyHostToDevice, st));
    }
    const FanDev f = fill_fandev(grid, fan, n, order, tab);
    CUDA_TRY(launch_trace(grid->g, f, out_dev, counter, lp, st));
    return RT_OK;
}

rt_err rt_eval_rhs(const rt_grid *grid, double freq_mhz, int32_t mode, int32_t precision, int32_t stencil,
                   const double *y_host, double *dy_host, double *mu2_host, size_t n) {
    if (!grid || !y_host || !dy_host || !mu2_host) return fail(RT_EINVAL, "NULL argument");
    if (!finite_pos(freq_mhz)) return fail(RT_EINVAL, "freq_mhz must be finite and > 0");
    if (mode != 1 && mode != -1) return fail(RT_EINVAL, "mode must be +1 (O) or -1 (X)");
    if (precision != RT_FP64 && precision != RT_MIXED) return fail(RT_EINVAL, "unknown precision");
    if (stencil < 0 || stencil > RT_STENCIL_TABLE) return fail(RT_EINVAL, "unknown stencil");
    if (stencil == RT_STENCIL_TABLE && !grid->table) return fail(RT_EINVAL, "grid has no table");
    rt_err r = ensure_device(nullptr);
    if (r != RT_OK) return r;
    if (n == 0) return RT_OK;
    double *buf = nullptr;
    CUDA_TRY(cudaMalloc((void **)&buf, n * 13 * sizeof(double)));
    cudaError_t e = cudaMemcpy(buf, y_host, n * 6 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_eval_rhs(grid->g, buf, buf + n * 6, buf + n * 12, freq_mhz, mode, precision, stencil,
                            (long long)n, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(dy_host, buf + n * 6, n * 6 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(mu2_host, buf + n * 12, n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "rt_eval_rhs");
    return RT_OK;
}

}  // extern "C"
