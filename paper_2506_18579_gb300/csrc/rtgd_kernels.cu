// rtgd_kernels.cu -- CUDA kernels of the RTM-GD tracer (sm_103a).
//
//   grid preparation  : ghost padding (FP64 + FP32 copies), the "quad" layout
//                       (4 consecutive altitude samples per float4) and the
//                       optional per-cell 64-sample table (Sec. II-C: the
//                       interpolation data are prepared once per grid cell).
//   trace_fp64        : all-FP64 tracer, one thread per ray.
//   trace_mixed_*     : mixed-precision tracer.  A group of 1, 2 or 4 lanes
//                       carries one ray; every loop iteration runs one whole
//                       RK attempt for all lanes of a warp (the stage index
//                       is warp-uniform), so the lanes stay converged.  The
//                       plain kernel gives each group one ray; the persistent
//                       kernel keeps a resident grid whose warps claim their
//                       next rays from an atomic counter once their current
//                       rays have ended.
//   eval_rhs          : diagnostic evaluation of dy/dP' at given states.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <stdint.h>

#include "rtgd.h"
#include "rtgd_device.cuh"
#include "rtgd_internal.h"

namespace rtgd {

// ===================================================================== grid
// Padded value at padded index (pi, pj, pk): interior nodes are copied; a
// ghost index maps to quadratic extrapolation u_{-1} = 3u_0 - 3u_1 + u_2
// (and its mirror at the far face), applied along every ghost axis (tensor
// product, so corners combine up to 27 nodes).
__device__ __forceinline__ int ghost_taps(int p, int n, int idx[3], double w[3]) {
    if (p == 0) {
        idx[0] = 0; idx[1] = 1; idx[2] = 2;
        w[0] = 3.0; w[1] = -3.0; w[2] = 1.0;
        return 3;
    }
    if (p == n + 1) {
        idx[0] = n - 1; idx[1] = n - 2; idx[2] = n - 3;
        w[0] = 3.0; w[1] = -3.0; w[2] = 1.0;
        return 3;
    }
    idx[0] = p - 1;
    w[0] = 1.0;
    return 1;
}

template <typename T>
__global__ void pad_kernel(const T *__restrict__ raw, double *__restrict__ pad64, float *__restrict__ pad32,
                           int n_lat, int n_lon, int n_alt) {
    const long long P_lon = n_lon + 2, P_alt = n_alt + 2;
    const long long total = (long long)(n_lat + 2) * P_lon * P_alt;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int pk = (int)(e % P_alt);
        const int pj = (int)((e / P_alt) % P_lon);
        const int pi = (int)(e / (P_alt * P_lon));
        int ia[3], ja[3], ka[3];
        double wa[3], wb[3], wc[3];
        const int na = ghost_taps(pi, n_lat, ia, wa);
        const int nb = ghost_taps(pj, n_lon, ja, wb);
        const int nc = ghost_taps(pk, n_alt, ka, wc);
        double v = 0.0;
        for (int a = 0; a < na; ++a)
            for (int b = 0; b < nb; ++b)
                for (int c = 0; c < nc; ++c)
                    v += wa[a] * wb[b] * wc[c] *
                         (double)raw[((long long)ia[a] * n_lon + ja[b]) * n_alt + ka[c]];
        pad64[e] = v;
        pad32[e] = (float)v;
    }
}

// quad[(pi, pj, k)] = padded samples k..k+3 (nodes k-1..k+2) of cell k.
__global__ void quad_kernel(const float *__restrict__ pad32, float4 *__restrict__ quad, int n_lat, int n_lon,
                            int n_alt) {
    const long long P_lon = n_lon + 2, P_alt = n_alt + 2, Q = n_alt - 1;
    const long long total = (long long)(n_lat + 2) * P_lon * Q;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long k = e % Q;
        const long long row = e / Q;  // pi * P_lon + pj
        const float *p = pad32 + row * P_alt + k;
        quad[e] = make_float4(p[0], p[1], p[2], p[3]);
    }
}

// table[cell * 16 + a * 4 + b] = the 4 altitude samples of row (a, b) of the
// 4x4x4 stencil of cell (i, j, k), each minus the cell's reference node
// (i, j, k) (padded (i+1, j+1, k+1)); cells are ordered [i][j][k].  The stage
// evaluation contracts samples relative to that node, so storing them that
// way saves the subtraction (the same float operation, done once per grid).
__global__ void table_kernel(const float4 *__restrict__ quad, float4 *__restrict__ table, int n_lat, int n_lon,
                             int n_alt) {
    const long long C_lon = n_lon - 1, C_alt = n_alt - 1, P_lon = n_lon + 2;
    const long long total = (long long)(n_lat - 1) * C_lon * C_alt * 16;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ab = (int)(e & 15);
        const long long cell = e >> 4;
        const long long k = cell % C_alt;
        const long long j = (cell / C_alt) % C_lon;
        const long long i = cell / (C_alt * C_lon);
        const int a = ab >> 2, b = ab & 3;
        const float4 u = quad[((i + a) * P_lon + (j + b)) * C_alt + k];
        const float ref = quad[((i + 1) * P_lon + (j + 1)) * C_alt + k].y;
        table[e] = make_float4(u.x - ref, u.y - ref, u.z - ref, u.w - ref);
    }
}

static int blocks_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_grid_prep(const void *raw, int dtype, const GridSizes &sz, double *pad64, float *pad32,
                             float4 *quad, float4 *table, cudaStream_t st) {
    const long long n_pad = (long long)(sz.n_lat + 2) * (sz.n_lon + 2) * (sz.n_alt + 2);
    if (dtype == RT_F64)
        pad_kernel<double><<<blocks_for(n_pad, 256), 256, 0, st>>>((const double *)raw, pad64, pad32, sz.n_lat,
                                                                    sz.n_lon, sz.n_alt);
    else
        pad_kernel<float><<<blocks_for(n_pad, 256), 256, 0, st>>>((const float *)raw, pad64, pad32, sz.n_lat,
                                                                   sz.n_lon, sz.n_alt);
    const long long n_quad = (long long)(sz.n_lat + 2) * (sz.n_lon + 2) * (sz.n_alt - 1);
    quad_kernel<<<blocks_for(n_quad, 256), 256, 0, st>>>(pad32, quad, sz.n_lat, sz.n_lon, sz.n_alt);
    if (table) {
        const long long n_tab = (long long)(sz.n_lat - 1) * (sz.n_lon - 1) * (sz.n_alt - 1) * 16;
        table_kernel<<<blocks_for(n_tab, 256), 256, 0, st>>>(quad, table, sz.n_lat, sz.n_lon, sz.n_alt);
    }
    return cudaGetLastError();
}

// ====================================================================== fan
// Canonical ray index -> (frequency, mode, elevation, azimuth) of the fan,
// order [freq][mode][el][az], with the per-fan table entries of each.
struct RayParams {
    double f_hz;
    float xfac, ab0;        // the mixed path's per-frequency factors
    double se, ce, sa, ca;  // sin, cos of elevation and azimuth
    double az;              // azimuth (rad)
    int mode;
};

// Fans hold fewer than 2^31 rays (checked on the host), so 32-bit index
// arithmetic suffices (64-bit divisions are long instruction sequences).
__device__ __forceinline__ RayParams ray_params(const FanDev &f, long long id64) {
    const unsigned id = (unsigned)id64;
    const unsigned a = id % (unsigned)f.n_az;
    const unsigned rest = id / (unsigned)f.n_az;
    const unsigned e = rest % (unsigned)f.n_el;
    const unsigned rest2 = rest / (unsigned)f.n_el;
    const unsigned m = rest2 % (unsigned)f.n_modes;
    const unsigned q = rest2 / (unsigned)f.n_modes;
    RayParams p;
    p.f_hz = f.freq[q].f_hz;
    p.xfac = f.freq[q].xfac;
    p.ab0 = f.freq[q].ab0;
    p.se = f.el[e].s;
    p.ce = f.el[e].c;
    p.sa = f.az[a].s;
    p.ca = f.az[a].c;
    p.az = f.az[a].rad;
    p.mode = (m == 0) ? f.mode0 : f.mode1;
    return p;
}

// Claim index -> canonical index.  ORDER_ELEVATION_FASTEST hands out
// neighbouring elevations of one azimuth together (similar paths, so the
// lanes of a warp gather from nearby cells).
__device__ __forceinline__ long long claim_to_ray(const FanDev &f, long long c64) {
    if (f.perm) return f.perm[f.perm_off + c64];
    if (f.order != RT_ORDER_ELEVATION_FASTEST) return c64;
    const unsigned c = (unsigned)c64;
    const unsigned e = c % (unsigned)f.n_el;
    const unsigned rest = c / (unsigned)f.n_el;
    const unsigned a = rest % (unsigned)f.n_az;
    const unsigned fm = rest / (unsigned)f.n_az;  // freq * n_modes + mode
    return ((long long)fm * f.n_el + e) * f.n_az + a;
}

// ================================================================ utilities
__device__ __forceinline__ double wrap180(double x) { return x - 360.0 * floor((x + 180.0) / 360.0); }

// Peak of the cubic Hermite fit of r(s), s in [0,1], through (r0, h d0) and
// (r1, h d1) with d0 > 0 >= d1 (zero of p'(s) by bisection).
__device__ double hermite_peak(double r0, double r1, double d0, double d1, double h) {
    const double m0 = h * d0, m1 = h * d1;
    const double A = 2.0 * (r0 - r1) + m0 + m1;
    const double B = 3.0 * (r1 - r0) - 2.0 * m0 - m1;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double dp = m0 + 2.0 * B * mid + 3.0 * A * mid * mid;
        if (dp > 0.0) lo = mid;
        else hi = mid;
    }
    const double s = 0.5 * (lo + hi);
    return r0 + m0 * s + B * s * s + A * s * s * s;
}

// Output quantities of a final state (Sec. II-C: group path, ground distance,
// azimuth deviation, reflection height): central angle and initial bearing
// on the sphere from the transmitter (tx_th, tx_ph) to (th, ph).  Out of line
// (it runs once per ray) with scalar arguments, so that neither the caller's
// state nor the kernel parameters need an address.
__device__ __noinline__ void finish_result(double tx_th, double tx_ph, double az_launch, double th, double ph,
                                           double P, double apo, int status, int n_steps, int n_att, int n_evals,
                                           double R_E, rt_ray_result *out) {
    double s0, c0, s1, c1, sd, cd;
    sincos(tx_th, &s0, &c0);
    sincos(th, &s1, &c1);
    sincos(ph - tx_ph, &sd, &cd);
    const double east = s1 * sd;                 // components of the final point in the
    const double north = s0 * c1 - c0 * s1 * cd;  // tangent plane at the transmitter
    const double dot = s0 * s1 * cd + c0 * c1;
    const double ang = atan2(sqrt(east * east + north * north), dot);
    rt_ray_result r;
    r.group_path_km = P;
    r.ground_range_km = R_E * ang;
    r.az_dev_deg = ang > 1e-15 ? wrap180(atan2(east, north) * kRad2Deg - az_launch * kRad2Deg) : 0.0;
    r.apogee_km = apo;
    r.land_lat_deg = 90.0 - th * kRad2Deg;
    r.land_lon_deg = wrap180(ph * kRad2Deg);
    r.status = status;
    r.n_steps = n_steps;
    r.n_attempts = n_att;
    r.n_evals = n_evals;
    *out = r;
}

__device__ __forceinline__ bool finite6(const double y[6]) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) ok = ok && isfinite(y[i]);
    return ok;
}

// Lateral position inside the grid's lat/lon span?
__device__ __forceinline__ bool inside_latlon(const GridDev &g, double th, double ph) {
    const double lat = 90.0 - th * kRad2Deg;
    double lonrel = ph * kRad2Deg - g.lon0;
    lonrel -= 360.0 * floor(lonrel / 360.0);
    const double xa = (lat - g.lat0) * g.inv_dlat;
    const double xb = lonrel * g.inv_dlon;
    return xa >= 0.0 && xa <= (double)(g.n_lat - 1) && xb >= 0.0 && xb <= (double)(g.n_lon - 1);
}

// ================================================================ FP64 path
// dy/dP' at state y, all in double: Ne and its gradient from the FP64 padded
// grid (Eq. 13), then the dipole, Appleton-Hartree and Eq. 1.
__device__ void rhs64(const GridDev &g, const RayPhys<double> &rp, const double y[6], double dy[6],
                      double *mu2) {
    StageIn<double> s;
    s.r = y[0];
    sincos(y[1], &s.sth, &s.cth);
    sincos(y[2], &s.sph, &s.cph);
    s.k[0] = y[3];
    s.k[1] = y[4];
    s.k[2] = y[5];
    const double alt = y[0] - g.R_E;
    const double lat = 90.0 - y[1] * kRad2Deg;
    double lonrel = y[2] * kRad2Deg - g.lon0;
    lonrel -= 360.0 * floor(lonrel / 360.0);
    const double xa = (lat - g.lat0) * g.inv_dlat;
    const double xb = lonrel * g.inv_dlon;
    const double xc = (alt - g.alt0) * g.inv_dalt;
    int ia, ib, ic;
    double ta, tb, tc;
    s.X = 0.0;
    s.dX[0] = s.dX[1] = s.dX[2] = 0.0;
    if (cell_coord<double>(xa, g.n_lat, ia, ta) && cell_coord<double>(xb, g.n_lon, ib, tb) &&
        cell_coord<double>(xc, g.n_alt, ic, tc)) {
        double wa[4], da[4], wb[4], db[4], wc[4], dc[4], out[4];
        interp_weights<double>(ta, wa, da, g.interp);
        interp_weights<double>(tb, wb, db, g.interp);
        interp_weights<double>(tc, wc, dc, g.interp);
        const long long sj = g.p_alt, si = (long long)g.p_lon * g.p_alt;
        // padded index of node (ia-1, ib-1, ic-1) is (ia, ib, ic)
        const double *base = g.pad64 + (long long)ia * si + (long long)ib * sj + ic;
#define RTGD_ROW64(a, b, u0, u1, u2, u3)              \
    {                                                 \
        const double *p_ = base + (a) * si + (b) * sj; \
        u0 = __ldg(p_);                               \
        u1 = __ldg(p_ + 1);                           \
        u2 = __ldg(p_ + 2);                           \
        u3 = __ldg(p_ + 3);                           \
    }
        RTGD_CONTRACT(double, false, RTGD_ROW64, 0.0, 0, 4, wa, da, wb, db, wc, dc, out);
#undef RTGD_ROW64
        s.X = rp.xfac * out[0];
        s.dX[0] = rp.xfac * out[3] * g.inv_dalt;
        s.dX[1] = -rp.xfac * out[1] * g.inv_dlat * kRad2Deg;
        s.dX[2] = rp.xfac * out[2] * g.inv_dlon * kRad2Deg;
    }
    const FieldTerms<double> F = field_terms<double>(rp, s);
    ray_rhs<double>(rp, s, F, dy, mu2);
}

__device__ void rk4_step64(const GridDev &g, const RayPhys<double> &rp, const double y[6], const double k1[6],
                           double h, double yn[6]) {
    double k2[6], k3[6], k4[6], t[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    rhs64(g, rp, t, k2, nullptr);
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    rhs64(g, rp, t, k3, nullptr);
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = y[i] + h * k3[i];
    rhs64(g, rp, t, k4, nullptr);
#pragma unroll
    for (int i = 0; i < 6; ++i) yn[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

// Runge-Kutta-Fehlberg 4(5): fourth-order solution in yn, local error
// estimate (5th - 4th order) in e, formed as h sum((b5_i - b4_i) k_i) so it
// keeps full relative precision (y5 - y4 would cancel against r ~ 6371 km).
__device__ void rkf45_step64(const GridDev &g, const RayPhys<double> &rp, const double y[6], const double k1[6],
                             double h, double yn[6], double e[6]) {
    double k2[6], k3[6], k4[6], k5[6], k6[6], t[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = y[i] + h * (k1[i] / 4.0);
    rhs64(g, rp, t, k2, nullptr);
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = y[i] + h * (3.0 / 32.0 * k1[i] + 9.0 / 32.0 * k2[i]);
    rhs64(g, rp, t, k3, nullptr);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        t[i] = y[i] + h * (1932.0 / 2197.0 * k1[i] - 7200.0 / 2197.0 * k2[i] + 7296.0 / 2197.0 * k3[i]);
    rhs64(g, rp, t, k4, nullptr);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        t[i] = y[i] + h * (439.0 / 216.0 * k1[i] - 8.0 * k2[i] + 3680.0 / 513.0 * k3[i] - 845.0 / 4104.0 * k4[i]);
    rhs64(g, rp, t, k5, nullptr);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        t[i] = y[i] + h * (-8.0 / 27.0 * k1[i] + 2.0 * k2[i] - 3544.0 / 2565.0 * k3[i] + 1859.0 / 4104.0 * k4[i] -
                           11.0 / 40.0 * k5[i]);
    rhs64(g, rp, t, k6, nullptr);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        yn[i] = y[i] + h * (25.0 / 216.0 * k1[i] + 1408.0 / 2565.0 * k3[i] + 2197.0 / 4104.0 * k4[i] - k5[i] / 5.0);
        e[i] = h * ((16.0 / 135.0 - 25.0 / 216.0) * k1[i] + (6656.0 / 12825.0 - 1408.0 / 2565.0) * k3[i] +
                    (28561.0 / 56430.0 - 2197.0 / 4104.0) * k4[i] + (1.0 / 5.0 - 9.0 / 50.0) * k5[i] +
                    2.0 / 55.0 * k6[i]);
    }
}

// RKF45 error norm (<= 1 accepts) and step factor, as documented in rtgd.h.
template <typename R>
__device__ __forceinline__ R rkf45_err(R r, R sth, R kmag, const R e[6], R rtol, R atol) {
    const R pos = fmax(fabs(e[0]), fmax(r * fabs(e[1]), r * sth * fabs(e[2])));
    const R kerr = fmax(fabs(e[3]), fmax(fabs(e[4]), fabs(e[5])));
    return fmax(fdiv(pos, atol + rtol * r), fdiv(kerr, rtol * fmax(kmag, R(1e-3))));
}

// Step-size factor: 0.9 err^(-1/5) limited to [0.2, 5], rounded down to a
// power of 2^(1/4), so step sizes change through discrete decisions only and
// round-off in err cannot feed back into the step sequence.
template <typename R>
__device__ __forceinline__ double step_factor(R err) {
    const R fac = (err == R(0)) ? R(5) : fmin(R(5), fmax(R(0.2), R(0.9) * pow(err, R(-0.2))));
    return exp2(floor(4.0 * log2((double)fac)) * 0.25);
}

// Launch direction (elevation above the horizontal, azimuth clockwise from
// north; the theta unit vector points south) and position of a ray, from the
// fan's sine and cosine tables.
__device__ __forceinline__ void launch_dir(const FanDev &f, const RayParams &p, double y[6]) {
    y[0] = f.tx_r;
    y[1] = f.tx_th;
    y[2] = f.tx_ph;
    y[3] = p.se;
    y[4] = -p.ce * p.ca;
    y[5] = p.ce * p.sa;
}

// Group path to the next cell face the ray reaches, predicted linearly from
// dy/dP' = k1.  Faces are where the C1 interpolant's second derivatives jump
// (the right-hand side is only C0 there), the grid's outer faces included;
// lateral faces count only inside the altitude span.  Adaptive steps end just
// past such a face instead of straddling it.
__device__ double face_distance64(const GridDev &g, const double y[6], const double k1[6]) {
    const double lat = 90.0 - y[1] * kRad2Deg;
    double lonrel = y[2] * kRad2Deg - g.lon0;
    lonrel -= 360.0 * floor(lonrel * (1.0 / 360.0));
    const double x[3] = {(lat - g.lat0) * g.inv_dlat, lonrel * g.inv_dlon, (y[0] - g.R_E - g.alt0) * g.inv_dalt};
    const double v[3] = {-k1[1] * kRad2Deg * g.inv_dlat, k1[2] * kRad2Deg * g.inv_dlon, k1[0] * g.inv_dalt};
    const int n[3] = {g.n_lat, g.n_lon, g.n_alt};
    const bool in_alt = x[2] >= 0.0 && x[2] <= (double)(g.n_alt - 1);
    double best = HUGE_VAL;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < 2 && !in_alt) continue;
        if (v[a] > 0.0) {
            double F = floor(x[a]) + 1.0;
            if (F < 0.0) F = 0.0;
            if (F <= (double)(n[a] - 1)) best = fmin(best, (F - x[a]) / v[a]);
        } else if (v[a] < 0.0) {
            double F = ceil(x[a]) - 1.0;
            if (F > (double)(n[a] - 1)) F = (double)(n[a] - 1);
            if (F >= 0.0) best = fmin(best, (F - x[a]) / v[a]);
        }
    }
    return best;
}

__device__ void trace_ray_fp64(const GridDev &g, const FanDev &f, long long id, rt_ray_result *out) {
    const RayParams p = ray_params(f, id);
    const RayPhys<double> rp = make_phys<double>(g, p.f_hz, p.mode);
    const double RE = g.R_E;
    double y[6], dummy[6], mu2 = 0.0;
    launch_dir(f, p, y);
    rhs64(g, rp, y, dummy, &mu2);  // mu^2 at the transmitter for this direction
    if (!(mu2 > 0.0)) {
        finish_result(f.tx_th, f.tx_ph, p.az, y[1], y[2], 0.0, f.tx_r - RE, RT_RAY_NONFINITE, 0, 0, 1, RE, out);
        return;
    }
    const double mu = sqrt(mu2);
    y[3] *= mu;
    y[4] *= mu;
    y[5] *= mu;
    const bool adaptive = f.integrator == RT_RKF45;
    double P = 0.0, h = f.h0, apo = y[0] - RE;
    int n_steps = 0, n_att = 0, n_ev = 1, status = RT_RAY_NOT_RUN;
    const int ev_per_step = adaptive ? 5 : 3;  // stage evaluations besides k1
    bool have_prev = false, k1_valid = false;
    double r_prev = 0.0, dr_prev = 0.0, h_prev = 0.0;
    double k1[6];
    while (status == RT_RAY_NOT_RUN) {
        if (n_att >= f.max_steps) {
            status = RT_RAY_MAX_STEPS;
            break;
        }
        double hs = h;
        if (!k1_valid) {
            rhs64(g, rp, y, k1, nullptr);
            k1_valid = true;
            ++n_ev;
        }
        bool at_face = false;
        if (adaptive) {
            const double hf = face_distance64(g, y, k1);
            if (hf > 1e-3 * hs && hf < hs) {
                hs = hf * (1.0 + 1e-4);
                at_face = true;
            }
        }
        if (f.max_path > 0.0 && P + hs > f.max_path) hs = f.max_path - P;
        if (have_prev && dr_prev > 0.0 && k1[0] <= 0.0)
            apo = fmax(apo, hermite_peak(r_prev, y[0], dr_prev, k1[0], h_prev) - RE);
        have_prev = false;
        double yn[6], e[6];
        if (adaptive) rkf45_step64(g, rp, y, k1, hs, yn, e);
        else rk4_step64(g, rp, y, k1, hs, yn);
        ++n_att;
        n_ev += ev_per_step;
        double h_next = h;
        if (adaptive) {
            const double err = rkf45_err<double>(y[0], sin(y[1]), sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]), e,
                                                 f.rtol, f.atol);
            const double fac = step_factor<double>(err);
            // the nominal step changes only by quantised factors of itself
            if (!(err <= 1.0)) {
                h = h * fac;
                if (h < f.hmin) status = RT_RAY_STEP_UNDERFLOW;
                continue;
            }
            h_next = fmin(fmax(h * (at_face ? fmin(1.0, fac) : fac), f.hmin), f.hmax);
        }
        if (!finite6(yn)) {
            status = RT_RAY_NONFINITE;
            break;
        }
        const bool lands = yn[0] < RE;
        const bool exits = !lands && yn[0] - RE > g.top;
        if (lands || exits) {
            // ground return or exit through the grid top inside this step:
            // r(step(h*)) = R_E (or R_E + top) for h* in (0, hs], Illinois regula
            // falsi; sg makes the bracket function positive at the step start
            const double rt = lands ? RE : RE + g.top, sg = lands ? 1.0 : -1.0;
            double a = 0.0, fa = sg * (y[0] - rt), b = hs, fb = sg * (yn[0] - rt), c = b;
            double yc[6], ec[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) yc[i] = yn[i];
            int side = 0;
            for (int it = 0; it < 60; ++it) {
                c = b - fb * (b - a) / (fb - fa);
                if (adaptive) rkf45_step64(g, rp, y, k1, c, yc, ec);
                else rk4_step64(g, rp, y, k1, c, yc);
                ++n_att;
                n_ev += ev_per_step;
                const double fc = sg * (yc[0] - rt);
                if (fabs(fc) < 1e-9) break;
                if (fc < 0.0) {
                    b = c;
                    fb = fc;
                    if (side == -1) fa *= 0.5;
                    side = -1;
                } else {
                    a = c;
                    fa = fc;
                    if (side == 1) fb *= 0.5;
                    side = 1;
                }
            }
            P += c;
            ++n_steps;
#pragma unroll
            for (int i = 0; i < 6; ++i) y[i] = yc[i];
            if (exits) apo = fmax(apo, y[0] - RE);
            status = lands ? RT_RAY_LANDED : RT_RAY_ESCAPED;
            break;
        }
        P += hs;
        ++n_steps;
        apo = fmax(apo, yn[0] - RE);
        have_prev = true;
        r_prev = y[0];
        dr_prev = k1[0];
        h_prev = hs;
#pragma unroll
        for (int i = 0; i < 6; ++i) y[i] = yn[i];
        k1_valid = false;
        const double alt = y[0] - RE;
        if (alt >= g.alt0 && !inside_latlon(g, y[1], y[2])) {
            status = RT_RAY_LEFT_GRID;
            break;
        }
        if (f.max_path > 0.0 && P >= f.max_path - 1e-12) {
            status = RT_RAY_MAX_PATH;
            break;
        }
        h = h_next;
    }
    finish_result(f.tx_th, f.tx_ph, p.az, y[1], y[2], P, apo, status, n_steps, n_att, n_ev, RE, out);
}

__global__ void __launch_bounds__(128) trace_fp64_kernel(GridDev g, FanDev f, rt_ray_result *__restrict__ out) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= f.n_rays) return;
    const long long ray = claim_to_ray(f, id);
    rt_ray_result r;
    trace_ray_fp64(g, f, ray, &r);
    out[ray] = r;
}

// =============================================================== mixed path
// The ray state (r, theta, phi, k) and the group path stay in double.  Each
// step attempt starts from a "base": the grid cell and in-cell coordinates of
// the state plus float copies of r, k and of the sines and cosines of theta
// and phi.  A stage works on float offsets delta from the base: its grid
// coordinates are base + delta * (d coord / d state) (the coordinates are
// linear in r, theta, phi), and sin/cos of theta + delta by angle addition,
// so everything after (weights, contraction, dipole, Appleton-Hartree, Eq. 1)
// runs in float without losing the base's resolution.  An accepted step adds
// the float increment to the double position (r, theta, phi) and the double
// group path -- the only FP64 arithmetic of a step; the wave vector, a
// quantity of order 1, accumulates as a compensated float pair (hi + lo).
// The base (cells, altitude, radius, sines and cosines) follows by the same
// increment in float and is recomputed from the double state every
// kResyncSteps accepted steps.  GB300 issues FP64 at 1/64 of the FP32 rate,
// so the step bookkeeping must stay out of double precision.
constexpr int kResyncSteps = 16;

struct Base32 {
    int ia, ib, ic;            // cell of the base (may lie outside the grid)
    float ta, tb, tc;          // in-cell coordinates
    float r, alt;              // radius and altitude (km)
    float sth, cth, sph, cph;  // sin/cos of colatitude and longitude
    float k[3];
};

// 2^(k/4) for k = -10..9: the quantised step factors (see step_factor).
__constant__ float c_pow2q[20];

__device__ __forceinline__ int clamp_cell(double f) { return (int)fmin(fmax(f, -1e6), 1e6); }

// Base of a double state (double arithmetic; used at launch and to resync).
// Out of line with scalar arguments (it runs at launch and every kResyncSteps
// accepted steps), returning the base by value.
__device__ __noinline__ Base32 base_of(double lat0, double lon0, double inv_dlat, double inv_dlon, double R_E,
                                       double alt0, double inv_dalt, double r, double th, double ph, double k0,
                                       double k1, double k2) {
    Base32 b;
    const double lat = 90.0 - th * kRad2Deg;
    double lonrel = ph * kRad2Deg - lon0;
    lonrel -= 360.0 * floor(lonrel * (1.0 / 360.0));
    const double xa = (lat - lat0) * inv_dlat;
    const double xb = lonrel * inv_dlon;
    const double xc = (r - R_E - alt0) * inv_dalt;
    const double fa = floor(xa), fb = floor(xb), fc = floor(xc);
    // positions far outside the grid are clamped so the integer stays small; they
    // remain outside (and non-finite positions give NaN fractions, also outside)
    b.ia = clamp_cell(fa);
    b.ib = clamp_cell(fb);
    b.ic = clamp_cell(fc);
    b.ta = (float)(xa - fa);
    b.tb = (float)(xb - fb);
    b.tc = (float)(xc - fc);
    b.r = (float)r;
    b.alt = (float)(r - R_E);
    sincosf((float)th, &b.sth, &b.cth);
    sincosf((float)ph, &b.sph, &b.cph);
    b.k[0] = (float)k0;
    b.k[1] = (float)k1;
    b.k[2] = (float)k2;
    return b;
}

__device__ __forceinline__ void base_from_state(const GridDev &g, const double y[6], Base32 &b) {
    b = base_of(g.lat0, g.lon0, g.inv_dlat, g.inv_dlon, g.R_E, g.alt0, g.inv_dalt, y[0], y[1], y[2], y[3], y[4], y[5]);
}

__device__ __forceinline__ void shift_axis(int &i, float &t, float dt) {
    const float u = t + dt;
    const float fl = fminf(fmaxf(floorf(u), -1e6f), 1e6f);
    i += (int)fl;
    t = u - fl;
}

// sin/cos of (x0 + d) from sin/cos of x0, for |d| well below 0.1 rad (series
// error < d^7/5040).
__device__ __forceinline__ void angle_add(float s0, float c0, float d, float &s, float &c) {
    const float d2 = d * d;
    const float sd = d * (1.0f - d2 * (1.0f / 6.0f) * (1.0f - d2 * 0.05f));
    const float cd = 1.0f - 0.5f * d2 * (1.0f - d2 * (1.0f / 12.0f));
    s = s0 * cd + c0 * sd;
    c = c0 * cd - s0 * sd;
}

// Moves the base by the accepted increment d in float; k_hi is the new wave
// vector (high parts).
__device__ __forceinline__ void advance_base(const GridDev &g, Base32 &b, const float d[6], const float k_hi[3]) {
    shift_axis(b.ia, b.ta, g.sa * d[1]);
    shift_axis(b.ib, b.tb, g.sb * d[2]);
    shift_axis(b.ic, b.tc, g.sc * d[0]);
    b.r += d[0];
    b.alt += d[0];
    float s, c;
    angle_add(b.sth, b.cth, d[1], s, c);
    b.sth = s;
    b.cth = c;
    angle_add(b.sph, b.cph, d[2], s, c);
    b.sph = s;
    b.cph = c;
    b.k[0] = k_hi[0];
    b.k[1] = k_hi[1];
    b.k[2] = k_hi[2];
}

// hi + lo += d with the rounding error of hi + d kept in lo (Knuth's TwoSum).
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float d) {
    const float s = hi + d;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (d - bp);
    hi = s;
    lo += err;
}

// Stage cell along one axis from base cell i0 and offset coordinate t = t0 +
// delta * scale; false outside [0, n-1], and then cell 0 at t = 0, so that the
// caller can gather from an in-bounds cell without branching.
__device__ __forceinline__ bool stage_cell(int i0, float t, int n, int &i, float &tt) {
    // floor of t clamped to +-1e6 (keeps the int sum far from overflow) without
    // conversion instructions: adding 1.5 * 2^23 rounds to the nearest integer,
    // which sits in the low mantissa bits; one less if that rounded up.  A NaN
    // t clamps to -1e6 and then fails the cell index test below.
    const float magic = 12582912.0f;
    const float tc = fminf(fmaxf(t, -1e6f), 1e6f);
    const float big = tc + magic;
    const float near = big - magic;
    const bool up = near > tc;
    const float fl = up ? near - 1.0f : near;
    int ii = i0 + (__float_as_int(big) - __float_as_int(magic)) - (up ? 1 : 0);
    float tr = t - fl;
    const bool last = (ii == n - 1) & (tr == 0.0f);  // the last node: cell n-2 at t = 1
    ii = last ? n - 2 : ii;
    tr = last ? 1.0f : tr;
    // tr = t - floor(t) lies in [0, 1] by construction, so the cell index alone
    // decides; a NaN or an offset beyond the clamp puts it ~1e6 cells out
    const bool ok = (unsigned)ii < (unsigned)(n - 1);
    i = ok ? ii : 0;
    tt = ok ? tr : 0.0f;
    return ok;
}

// Lat-weights of the rows a = q*4/G .. (q+1)*4/G - 1 handled by lane q of a
// group of G lanes (G = 1: all four).
template <int G, int IP>
__device__ __forceinline__ void own_lat_weights(float ta, int q, float wa[4], float da[4]) {
    if (G == 1) {
        axis_weights<float, IP>(ta, wa, da);
    } else if (G == 2) {
        const bool hi = q != 0;  // rows 2, 3: nodes j+1, j+2
        float wm1, w0, dm1, d0;
        half_weights<float, IP>(hi ? 1.0f - ta : ta, wm1, w0, dm1, d0);
        wa[0] = hi ? w0 : wm1;
        wa[1] = hi ? wm1 : w0;
        da[0] = hi ? -d0 : dm1;
        da[1] = hi ? -dm1 : d0;
    } else {
        const bool hi = q >= 2;
        float wm1, w0, dm1, d0;
        half_weights<float, IP>(hi ? 1.0f - ta : ta, wm1, w0, dm1, d0);
        const bool outer = q == 0 || q == 3;  // nodes j-1, j+2
        wa[0] = outer ? wm1 : w0;
        da[0] = (outer ? dm1 : d0) * (hi ? -1.0f : 1.0f);
    }
}

// dy/dP' (float) at base + delta.  STENCIL selects where the 64 samples come
// from and IP the interpolant (0 GD, 1 Catmull-Rom); with G > 1 the G lanes
// of a group (lane q, shuffle mask gmask) split the 16 sample rows and combine
// their partial sums with a butterfly, whose every addition is commutative,
// so all lanes hold bitwise equal results.  The body has no branch: the field
// terms (which do not need Ne) come first and can overlap the sample gathers,
// and a stage outside the grid gathers from cell 0 and discards the result.
template <int STENCIL, int G, int IP>
__device__ __forceinline__ void rhs_mixed(const GridDev &g, const RayPhys<float> &rp, const Base32 &b,
                                          const float d[6], float dy[6], float *mu2, int q, unsigned gmask) {
    StageIn<float> s;
    s.r = b.r + d[0];
    angle_add(b.sth, b.cth, d[1], s.sth, s.cth);
    angle_add(b.sph, b.cph, d[2], s.sph, s.cph);
    s.k[0] = b.k[0] + d[3];
    s.k[1] = b.k[1] + d[4];
    s.k[2] = b.k[2] + d[5];
    const FieldTerms<float> F = field_terms<float>(rp, s);
    int ia, ib, ic;
    float ta, tb, tc;
    const bool in_a = stage_cell(b.ia, b.ta + g.sa * d[1], g.n_lat, ia, ta);
    const bool in_b = stage_cell(b.ib, b.tb + g.sb * d[2], g.n_lon, ib, tb);
    const bool in_c = stage_cell(b.ic, b.tc + g.sc * d[0], g.n_alt, ic, tc);
    const bool inside = in_a & in_b & in_c;
    ia = inside ? ia : 0;
    ib = inside ? ib : 0;
    ic = inside ? ic : 0;
    float wa[4], da[4], wb[4], db[4], wc[4], dc[4], out[4], ref;
    constexpr int NA = 4 / G;
    const int a0 = q * NA;
    own_lat_weights<G, IP>(ta, q, wa, da);
    axis_weights<float, IP>(tb, wb, db);
    axis_weights<float, IP>(tc, wc, dc);
    if (STENCIL == RT_STENCIL_QUAD) {
        // quad (pi, pj, k): 4 samples of cell k in padded row (pi, pj); node i-1 -> padded i
        const long long sj = g.q_alt, si = (long long)(g.n_lon + 2) * g.q_alt;
        const float4 *qp = g.quad + (long long)ia * si + (long long)ib * sj + ic;
        ref = __ldg(qp + si + sj).y;  // node (ia, ib, ic)
#define RTGD_ROWQ(a, b, u0, u1, u2, u3)                    \
    {                                                      \
        const float4 v_ = __ldg(qp + (a) * si + (b) * sj); \
        u0 = v_.x;                                        \
        u1 = v_.y;                                        \
        u2 = v_.z;                                        \
        u3 = v_.w;                                        \
    }
        RTGD_CONTRACT(float, (G > 1), RTGD_ROWQ, ref, a0, NA, wa, da, wb, db, wc, dc, out);
#undef RTGD_ROWQ
    } else if (STENCIL == RT_STENCIL_TABLE) {
        const long long cell = ((long long)ia * (g.n_lon - 1) + ib) * (g.n_alt - 1) + ic;
        const float4 *qp = g.table + cell * 16;  // samples minus the node (ia, ib, ic)
        ref = __ldg(g.pad32 + (long long)(ia + 1) * g.p_lon * g.p_alt + (long long)(ib + 1) * g.p_alt + ic + 1);
#define RTGD_ROWT(a, b, u0, u1, u2, u3)              \
    {                                                \
        const float4 v_ = __ldg(qp + (a) * 4 + (b)); \
        u0 = v_.x;                                  \
        u1 = v_.y;                                  \
        u2 = v_.z;                                  \
        u3 = v_.w;                                  \
    }
        RTGD_CONTRACT(float, (G > 1), RTGD_ROWT, 0.0f, a0, NA, wa, da, wb, db, wc, dc, out);
#undef RTGD_ROWT
    } else {
        const long long sj = g.p_alt, si = (long long)g.p_lon * g.p_alt;
        const float *p = g.pad32 + (long long)ia * si + (long long)ib * sj + ic;
        ref = __ldg(p + si + sj + 1);  // node (ia, ib, ic)
#define RTGD_ROWG(a, b, u0, u1, u2, u3)            \
    {                                              \
        const float *p_ = p + (a) * si + (b) * sj; \
        u0 = __ldg(p_);                            \
        u1 = __ldg(p_ + 1);                        \
        u2 = __ldg(p_ + 2);                        \
        u3 = __ldg(p_ + 3);                        \
    }
        RTGD_CONTRACT(float, (G > 1), RTGD_ROWG, ref, a0, NA, wa, da, wb, db, wc, dc, out);
#undef RTGD_ROWG
    }
    if (G > 1) {
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i) out[i] += __shfl_xor_sync(gmask, out[i], o);
        }
    }
    out[0] += ref;
    // Ne = 0 outside the grid box (selects, so that samples gathered there,
    // whatever they hold, never reach the result)
    s.X = inside ? rp.xfac * out[0] : 0.0f;
    s.dX[0] = inside ? rp.xfac * out[3] * g.sc : 0.0f;
    s.dX[1] = inside ? rp.xfac * out[1] * g.sa : 0.0f;
    s.dX[2] = inside ? rp.xfac * out[2] * g.sb : 0.0f;
    ray_rhs<float>(rp, s, F, dy, mu2);
}

// Butcher tables in "shifted accumulator" form.  After stage s produced k_s,
// acc[t] <- acc[t+1] + A[s][t] k_s (t = 0..4, acc[5] = 0), so acc[0] always
// holds sum_j a[s+1][j] k_j, the offset (over h) of the next stage; y4 and the
// error estimate accumulate B4[s] k_s and E[s] k_s.
struct Tableau {
    // row s: {A[s][0..3]} and {A[s][4], B4[s], E[s], 0}, two 16-byte loads per stage
    float4 lo[6];
    float4 hi[6];
    int ns;
};

__constant__ Tableau c_tab[2];  // [RT_RK4], [RT_RKF45]

// Quantised step factor in float (the mixed path's counterpart of step_factor).
__device__ __forceinline__ float step_factor_f(float err) {
    const float fac = (err == 0.0f) ? 5.0f : fminf(5.0f, fmaxf(0.2f, 0.9f * __powf(err, -0.2f)));
    int k = (int)floorf(4.0f * __log2f(fac));
    k = k < -10 ? -10 : (k > 9 ? 9 : k);
    return c_pow2q[k + 10];
}

// Peak rise of the cubic Hermite fit over one step, relative to its start:
// p(s) = m0 s + B s^2 + A s^3 with p(1) = dr, p'(0) = m0 > 0 >= p'(1) = m1.
__device__ __noinline__ float hermite_rise_f(float dr, float m0, float m1) {  // once per ray: out of line
    const float A = m0 + m1 - 2.0f * dr, B = 3.0f * dr - 2.0f * m0 - m1;
    float lo = 0.0f, hi = 1.0f;
    for (int it = 0; it < 24; ++it) {
        const float mid = 0.5f * (lo + hi);
        if (m0 + 2.0f * B * mid + 3.0f * A * mid * mid > 0.0f) lo = mid;
        else hi = mid;
    }
    const float s = 0.5f * (lo + hi);
    return s * (m0 + s * (B + s * A));
}

// Float counterpart of face_distance64 on the base's (cell, fraction) grid
// coordinates: the distance to the next face is (integer - fraction) / rate.
__device__ __forceinline__ float face_axis_f(int i, float t, int n, float v) {
    if (v > 0.0f) {
        int F = i + 1;
        if (F < 0) F = 0;
        return F <= n - 1 ? fdiv((float)(F - i) - t, v) : INFINITY;
    }
    if (v < 0.0f) {
        int F = t > 0.0f ? i : i - 1;
        if (F > n - 1) F = n - 1;
        return F >= 0 ? fdiv((float)(F - i) - t, v) : INFINITY;
    }
    return INFINITY;
}

__device__ __forceinline__ float face_distance_f(const GridDev &g, const Base32 &b, const float k1[6]) {
    float best = face_axis_f(b.ic, b.tc, g.n_alt, g.sc * k1[0]);
    const bool in_alt = b.ic >= 0 && (b.ic < g.n_alt - 1 || (b.ic == g.n_alt - 1 && b.tc == 0.0f));
    if (in_alt) {
        best = fminf(best, face_axis_f(b.ia, b.ta, g.n_lat, g.sa * k1[1]));
        best = fminf(best, face_axis_f(b.ib, b.tb, g.n_lon, g.sb * k1[2]));
    }
    return best;
}

// Per-lane state of the mixed tracer.
struct Lane {
    double y[3];              // r (km), theta, phi (rad): the FP64 position
    double P;                 // group path (km)
    float inc_hi[4], inc_lo[4];  // increments of (r, theta, phi, P') not yet added to y and P,
                                 // as compensated float pairs (see lane_fold)
    float k_hi[3], k_lo[3];   // wave vector as a compensated float pair
    float r_prev;             // radius at the start of the last accepted step
    float h, hs;              // next step / step of the current attempt (km)
    float h_prev, dr_prev;    // last accepted step and its dr/dP' at the start
    float apo;                // reflection height so far (km)
    float acc[5][6];
    float y4[6], e[6];
    float k1[6];
    float xfac, ab0;
    Base32 b;
    int out_id, mode;
    int n_steps, n_att, n_ev, status, since_sync;
    bool active, launch, landing, exiting, have_prev, k1_valid, at_face;
};

// State of the landing / exit solve of one lane (Illinois regula falsi on the
// step size: bracket [la, lb] with signed distances lfa, lfb from the target
// radius).  Used only on a ray's last step: the persistent kernel keeps it in
// a per-thread shared-memory slot (its refill code leaves fewer registers for
// the ray state; measured 8 % faster on the 495k-ray batch), the plain
// kernels in registers.
struct LandState {
    double la, lfa, lb, lfb;
    int side, it;
};

__device__ __forceinline__ RayPhys<float> lane_phys(const GridDev &g, const Lane &L) {
    RayPhys<float> p;
    p.xfac = L.xfac;
    p.ab0 = L.ab0;
    p.R_E = g.R_Ef;
    p.m[0] = g.mf[0];
    p.m[1] = g.mf[1];
    p.m[2] = g.mf[2];
    p.iso = g.iso != 0;
    p.mode = L.mode;
    return p;
}

// Stage 0 of an attempt: acc/y4/e start from k1.
__device__ __forceinline__ void accumulate_first(Lane &L, const Tableau &T, const float k1[6]) {
    const float4 lo = T.lo[0], hi = T.hi[0];
    const float A[5] = {lo.x, lo.y, lo.z, lo.w, hi.x};
    const float b4 = hi.y, e = hi.z;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
#pragma unroll
        for (int t = 0; t < 5; ++t) L.acc[t][c] = A[t] * k1[c];
        L.y4[c] = b4 * k1[c];
        L.e[c] = e * k1[c];
    }
}

// Stage s >= 1: shift the accumulators and add stage s's output ks.
__device__ __forceinline__ void accumulate_next(Lane &L, const Tableau &T, int s, const float ks[6]) {
    const float4 lo = T.lo[s], hi = T.hi[s];
    const float A[5] = {lo.x, lo.y, lo.z, lo.w, hi.x};
    const float b4 = hi.y, e = hi.z;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
#pragma unroll
        for (int t = 0; t < 4; ++t) L.acc[t][c] = L.acc[t + 1][c] + A[t] * ks[c];
        L.acc[4][c] = A[4] * ks[c];
        L.y4[c] += b4 * ks[c];
        L.e[c] += e * ks[c];
    }
}

// Base of the transmitter position (the launch state of every ray of the
// fan; the wave vector part is set per ray).
__device__ __forceinline__ Base32 tx_base(const GridDev &g, const FanDev &f) {
    return base_of(g.lat0, g.lon0, g.inv_dlat, g.inv_dlon, g.R_E, g.alt0, g.inv_dalt, f.tx_r, f.tx_th, f.tx_ph, 0.0,
                   0.0, 0.0);
}

// Starts ray `id`: per-ray constants from the fan's tables, FP64 launch
// state, and the float base: the transmitter's (btx, shared by the fan) with
// this ray's wave vector.
__device__ void lane_begin_ray(Lane &L, const GridDev &g, const FanDev &f, long long id, const Base32 &btx) {
    const RayParams p = ray_params(f, id);
    L.out_id = (int)id;
    L.xfac = p.xfac;
    L.ab0 = p.ab0;
    L.mode = p.mode;
    double y[6];
    launch_dir(f, p, y);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        L.y[i] = y[i];
        L.k_hi[i] = (float)y[3 + i];
        L.k_lo[i] = 0.0f;
    }
    L.P = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) L.inc_hi[i] = L.inc_lo[i] = 0.0f;
    L.h = f.h0_f;
    L.apo = (float)(f.tx_r - g.R_E);
    L.n_steps = L.n_att = L.n_ev = 0;
    L.since_sync = 0;
    L.status = RT_RAY_NOT_RUN;
    L.have_prev = L.k1_valid = L.landing = L.exiting = false;
    L.launch = true;
    L.b = btx;
#pragma unroll
    for (int i = 0; i < 3; ++i) L.b.k[i] = (float)y[3 + i];
}

// Adds the pending increments to the FP64 position and group path.  An
// accepted step adds its float increments of r, theta, phi and P' to
// compensated float pairs (TwoSum: hi + lo carries their sum to ~2^-48
// relative), and the pairs reach the double state only here: at the base
// resync every kResyncSteps steps, before a landing / exit solve and when the
// ray ends.  So the FP64 pipe (1/64 of the FP32 rate on GB300) sees four
// conversions and additions per component every kResyncSteps steps instead of
// two per component every step; the position agrees with step-by-step double
// accumulation to ~1e-12 km.
__device__ __forceinline__ void lane_fold(Lane &L) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        L.y[i] += (double)L.inc_hi[i] + (double)L.inc_lo[i];
        L.inc_hi[i] = L.inc_lo[i] = 0.0f;
    }
    L.P += (double)L.inc_hi[3] + (double)L.inc_lo[3];
    L.inc_hi[3] = L.inc_lo[3] = 0.0f;
}

// Double copy of the full state (position, wave vector hi + lo); the pending
// increments must have been folded in.
__device__ __forceinline__ void lane_state(const Lane &L, double y[6]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        y[i] = L.y[i];
        y[3 + i] = (double)L.k_hi[i] + (double)L.k_lo[i];
    }
}

// Writes a ray's raw final state into its record: colatitude and longitude
// (rad) stand in the ground-range and azimuth-deviation fields until
// finish_records_kernel turns them into the outputs.  The outputs' double
// trigonometry would otherwise run here, in a branch taken by the lanes of
// one ray while the rest of the warp waits on the 1/64-rate FP64 pipe.
__device__ __forceinline__ void lane_finish(Lane &L, const GridDev &g, const FanDev &f, rt_ray_result *out,
                                            bool writer = true) {
    L.active = false;
    if (!writer) return;
    lane_fold(L);
    rt_ray_result r;
    r.group_path_km = L.P;
    r.ground_range_km = L.y[1];
    r.az_dev_deg = L.y[2];
    r.apogee_km = (double)L.apo;
    r.land_lat_deg = 0.0;
    r.land_lon_deg = 0.0;
    r.status = L.status;
    r.n_steps = L.n_steps;
    r.n_attempts = L.n_att;
    r.n_evals = L.n_ev;
    out[L.out_id] = r;
}

// Final outputs of the mixed path's records, one thread per record (a
// converged pass after the trace): record k of a fan holds the raw final
// state lane_finish wrote; k is its canonical index, which gives the launch
// azimuth.
__global__ void finish_records_kernel(double R_E, FanDev f, rt_ray_result *__restrict__ out, long long n) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const rt_ray_result r = out[k];
    const double az = f.az[(unsigned)k % (unsigned)f.n_az].rad;
    finish_result(f.tx_th, f.tx_ph, az, r.ground_range_km, r.az_dev_deg, r.group_path_km, r.apogee_km, r.status,
                  r.n_steps, r.n_attempts, r.n_evals, R_E, out + k);
}

// The same for the records of several fans traced in one launch: record i
// belongs to fan k with first[k] <= i < first[k + 1].
__global__ void finish_fans_records_kernel(double R_E, const FanDev *__restrict__ fans,
                                           const long long *__restrict__ first, int n_fans,
                                           rt_ray_result *__restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= first[n_fans]) return;
    int lo = 0, hi = n_fans - 1;
    while (lo < hi) {  // largest k with first[k] <= i
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const FanDev &f = fans[lo];
    const long long k = i - first[lo];
    const rt_ray_result r = out[i];
    const double az = f.az[(unsigned)k % (unsigned)f.n_az].rad;
    finish_result(f.tx_th, f.tx_ph, az, r.ground_range_km, r.az_dev_deg, r.group_path_km, r.apogee_km, r.status,
                  r.n_steps, r.n_attempts, r.n_evals, R_E, out + i);
}

// Once k1 is known: end an adaptive step just past the next cell face, and
// clip it at the group-path limit.
__device__ __forceinline__ void lane_limit_step(Lane &L, const GridDev &g, const FanDev &f) {
    if (L.landing) return;
    if (f.integrator == RT_RKF45) {
        const float hf = face_distance_f(g, L.b, L.k1);
        if (hf > 1e-3f * L.hs && hf < L.hs) {
            L.hs = hf * (1.0f + 1e-4f);
            L.at_face = true;
        }
    }
    if (f.has_max_path) {
        const double P = L.P + ((double)L.inc_hi[3] + (double)L.inc_lo[3]);
        if (P + (double)L.hs > f.max_path) L.hs = (float)(f.max_path - P);
    }
}

// Sets up the next step attempt from the current state; returns false when
// the ray stops (step budget).
__device__ __forceinline__ bool lane_next_attempt(Lane &L, const FanDev &f) {
    if (L.n_att >= f.max_steps) {
        L.status = RT_RAY_MAX_STEPS;
        return false;
    }
    if (!L.landing) {
        L.hs = L.h;
        L.at_face = false;
    }
    return true;
}

// The launch evaluation: mu^2 at the transmitter for the launch direction,
// then |k| = mu.  Returns true when the ray has finished (status set).
template <int STENCIL, int G, int IP>
__device__ bool lane_launch(Lane &L, const GridDev &g, const FanDev &f, int q, unsigned gmask) {
    const RayPhys<float> rp = lane_phys(g, L);
    float d[6], ks[6], mu2;
#pragma unroll
    for (int c = 0; c < 6; ++c) d[c] = 0.0f;
    rhs_mixed<STENCIL, G, IP>(g, rp, L.b, d, ks, &mu2, q, gmask);
    ++L.n_ev;
    L.launch = false;
    if (!(mu2 > 0.0f)) {
        L.status = RT_RAY_NONFINITE;
        return true;
    }
    // |k| = mu: rescale the launch direction (double), split into hi + lo
    const double mu = sqrt((double)mu2);
    double y[6];
    lane_state(L, y);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double k = y[3 + i] * mu;
        L.k_hi[i] = (float)k;
        L.k_lo[i] = (float)(k - (double)L.k_hi[i]);
        L.b.k[i] = L.k_hi[i];
    }
    return !lane_next_attempt(L, f);
}

// Stage 0 bookkeeping once k1 is known: apogee check, face-limited step,
// accumulators.
__device__ __forceinline__ void lane_stage0_done(Lane &L, const GridDev &g, const FanDev &f, const Tableau &T,
                                                 bool fresh) {
    if (fresh) {
        L.k1_valid = true;
        if (L.have_prev && L.dr_prev > 0.0f && L.k1[0] <= 0.0f) {
            const float rise = hermite_rise_f(L.b.r - L.r_prev, L.h_prev * L.dr_prev, L.h_prev * L.k1[0]);
            L.apo = fmaxf(L.apo, L.b.alt - (L.b.r - L.r_prev) + rise);
        }
        L.have_prev = false;
    }
    lane_limit_step(L, g, f);
    accumulate_first(L, T, L.k1);
}

// The stages of one step attempt.  Every lane of a warp runs its attempt in
// the same loop, so the stage index is warp-uniform: the lanes stay converged
// and the Butcher coefficients are broadcast reads.  Stage 0 is evaluated
// only when k1 at the current state is not yet known (after a rejected
// attempt or during the landing solve it is): such lanes sit out that one
// evaluation.  With one lane per ray (throughput-bound fans) one copy of the
// stage evaluation serves all stages, which keeps the loop inside the
// instruction cache; with 2 or 4 lanes per ray (latency-bound fans) stage 0
// is a separate copy, which schedules better.
template <int STENCIL, int G, int IP>
__device__ __forceinline__ void lane_attempt(Lane &L, const GridDev &g, const FanDev &f, const Tableau &T, int q,
                                             unsigned gmask) {
    const RayPhys<float> rp = lane_phys(g, L);
    float d[6], ks[6];
    if (G == 1) {
#pragma unroll 1
        for (int s = 0; s < T.ns; ++s) {
            const bool fresh = s == 0 && !L.k1_valid;
            if (s > 0 || fresh) {
#pragma unroll
                for (int c = 0; c < 6; ++c) d[c] = s == 0 ? 0.0f : L.hs * L.acc[0][c];
                rhs_mixed<STENCIL, G, IP>(g, rp, L.b, d, ks, nullptr, q, gmask);
                ++L.n_ev;
            }
            if (s == 0) {
                if (fresh) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) L.k1[c] = ks[c];
                }
                lane_stage0_done(L, g, f, T, fresh);
            } else {
                accumulate_next(L, T, s, ks);
            }
        }
    } else {
        const bool fresh = !L.k1_valid;
        if (fresh) {
#pragma unroll
            for (int c = 0; c < 6; ++c) d[c] = 0.0f;
            rhs_mixed<STENCIL, G, IP>(g, rp, L.b, d, L.k1, nullptr, q, gmask);
            ++L.n_ev;
        }
        lane_stage0_done(L, g, f, T, fresh);
#pragma unroll 1
        for (int s = 1; s < T.ns; ++s) {
#pragma unroll
            for (int c = 0; c < 6; ++c) d[c] = L.hs * L.acc[0][c];
            rhs_mixed<STENCIL, G, IP>(g, rp, L.b, d, ks, nullptr, q, gmask);
            ++L.n_ev;
            accumulate_next(L, T, s, ks);
        }
    }
}

// Bracket of the landing / exit solve (Illinois regula falsi on the step size).
struct Bracket {
    double la, lfa, lb, lfb;
    int side;
};

// One regula falsi update with the new point (c, fc); returns the next step
// size.  Out of line: it runs only on the last step of a ray.
__device__ __noinline__ double bracket_update(Bracket &B, double c, double fc) {
    if (fc < 0.0) {
        B.lb = c;
        B.lfb = fc;
        if (B.side == -1) B.lfa *= 0.5;
        B.side = -1;
    } else {
        B.la = c;
        B.lfa = fc;
        if (B.side == 1) B.lfb *= 0.5;
        B.side = 1;
    }
    return B.lb - B.lfb * (B.lb - B.la) / (B.lfb - B.lfa);
}

__device__ __noinline__ double bracket_first(double lb, double lfa, double lfb) {
    return lb - lfb * lb / (lfb - lfa);  // la = 0
}

// Bookkeeping after an attempt: landing/exit solve, accept or reject, state
// update in double.  Returns true when the ray has finished (status set).
__device__ bool lane_end_attempt(Lane &L, const GridDev &g, const FanDev &f, LandState &ls) {
    const double RE = g.R_E;
    const float hf = L.hs;
    ++L.n_att;
    float dy4[6], ef[6];
    bool fin = true;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        dy4[c] = hf * L.y4[c];
        ef[c] = hf * L.e[c];
        fin = fin && isfinite(dy4[c]);
    }
    if (L.landing) {
        // Illinois regula falsi on the step size: f(h*) = +-(r(step(h*)) - target)
        const double sg = L.exiting ? -1.0 : 1.0;
        const double r_target = L.exiting ? RE + g.top : RE;
        const double fc = sg * ((L.y[0] - r_target) + (double)dy4[0]);
        ++ls.it;
        const double c = (double)L.hs;
        const bool done = fabs(fc) < f.land_tol || ls.it >= 60 || fabs(ls.lb - ls.la) < 1e-9 || !fin;
        if (!done) {
            Bracket B{ls.la, ls.lfa, ls.lb, ls.lfb, ls.side};
            L.hs = (float)bracket_update(B, c, fc);
            ls.la = B.la;
            ls.lfa = B.lfa;
            ls.lb = B.lb;
            ls.lfb = B.lfb;
            ls.side = B.side;
            return !lane_next_attempt(L, f);
        }
        if (!fin) {
            L.status = RT_RAY_NONFINITE;
            return true;
        }
        L.P += c;
        ++L.n_steps;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            L.y[i] += (double)dy4[i];
            two_sum_add(L.k_hi[i], L.k_lo[i], dy4[3 + i]);
        }
        if (L.exiting) L.apo = fmaxf(L.apo, (float)(L.y[0] - RE));
        L.status = L.exiting ? RT_RAY_ESCAPED : RT_RAY_LANDED;
        return true;
    }
    float h_next = L.h;
    if (f.integrator == RT_RKF45) {
        const float kmag = fsqrt(L.b.k[0] * L.b.k[0] + L.b.k[1] * L.b.k[1] + L.b.k[2] * L.b.k[2]);
        const float err = rkf45_err<float>(L.b.r, L.b.sth, kmag, ef, f.rtol_f, f.atol_f);
        const float fac = step_factor_f(err);
        // the nominal step changes only by quantised factors of itself
        if (!(err <= 1.0f)) {
            L.h = L.h * fac;
            if (L.h < f.hmin_f) {
                L.status = RT_RAY_STEP_UNDERFLOW;
                return true;
            }
            return !lane_next_attempt(L, f);
        }
        h_next = fminf(fmaxf(L.h * (L.at_face ? fminf(1.0f, fac) : fac), f.hmin_f), f.hmax_f);
    }
    if (!fin) {
        L.status = RT_RAY_NONFINITE;
        return true;
    }
    const float alt_new = L.b.alt + dy4[0];
    const bool lands = alt_new < 0.0f;
    if (lands || alt_new > g.top_f) {
        // ground return or exit through the grid top inside this step
        lane_fold(L);
        const double r_new = L.y[0] + (double)dy4[0];
        L.landing = true;
        L.exiting = !lands;
        const double r_target = lands ? RE : RE + g.top;
        const double sg = lands ? 1.0 : -1.0;
        ls.la = 0.0;
        ls.lfa = sg * (L.y[0] - r_target);
        ls.lb = (double)L.hs;
        ls.lfb = sg * (r_new - r_target);
        ls.side = 0;
        ls.it = 0;
        L.hs = (float)bracket_first(ls.lb, ls.lfa, ls.lfb);
        return !lane_next_attempt(L, f);
    }
    L.r_prev = L.b.r;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        two_sum_add(L.inc_hi[i], L.inc_lo[i], dy4[i]);
        two_sum_add(L.k_hi[i], L.k_lo[i], dy4[3 + i]);
    }
    two_sum_add(L.inc_hi[3], L.inc_lo[3], L.hs);
    ++L.n_steps;
    L.apo = fmaxf(L.apo, alt_new);
    L.have_prev = true;
    L.dr_prev = L.k1[0];
    L.h_prev = L.hs;
    L.k1_valid = false;
    if (++L.since_sync >= kResyncSteps) {
        L.since_sync = 0;
        lane_fold(L);
        double y[6];
        lane_state(L, y);
        base_from_state(g, y, L.b);
    } else {
        advance_base(g, L.b, dy4, L.k_hi);
    }
    if (L.b.alt >= (float)g.alt0) {
        const bool in_lat = L.b.ia >= 0 && (L.b.ia < g.n_lat - 1 || (L.b.ia == g.n_lat - 1 && L.b.ta == 0.0f));
        const bool in_lon = L.b.ib >= 0 && (L.b.ib < g.n_lon - 1 || (L.b.ib == g.n_lon - 1 && L.b.tb == 0.0f));
        if (!(in_lat && in_lon)) {
            L.status = RT_RAY_LEFT_GRID;
            return true;
        }
    }
    if (f.has_max_path) {
        lane_fold(L);
        if (L.P >= f.max_path - 1e-6) {
            L.status = RT_RAY_MAX_PATH;
            return true;
        }
    }
    L.h = h_next;
    return !lane_next_attempt(L, f);
}

// Loads the Butcher table of the fan's integrator into shared memory; the
// stage loop reads it at a warp-uniform stage index (broadcast reads).  With
// btx, also the transmitter's base of fan f (computed once per block: it is
// double arithmetic, and the persistent kernel would otherwise redo it for
// every lane it refills).
__device__ __forceinline__ void load_tableau(Tableau &T, int integrator, Base32 *btx = nullptr,
                                             const GridDev *g = nullptr, const FanDev *f = nullptr) {
    const Tableau &src = c_tab[integrator == RT_RKF45 ? 1 : 0];
    const float *s = (const float *)&src;
    float *d = (float *)&T;
    for (int i = threadIdx.x; i < (int)(sizeof(Tableau) / sizeof(float)); i += blockDim.x) d[i] = s[i];
    if (btx && threadIdx.x == 0) *btx = tx_base(*g, *f);
    __syncthreads();
}

// Shuffle mask of the G-lane group of this lane.
template <int G>
__device__ __forceinline__ unsigned group_mask(int lane) {
    return G == 1 ? (1u << lane) : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

// One ray per thread group of G lanes; each group loops attempt by attempt
// until its ray ends.  Launch bounds: one lane per ray is throughput-bound
// (three blocks of 128 per SM, <= 168 registers); 2 or 4 lanes per ray serve
// fans whose time is the latency of their slowest ray, and there the
// compiler's own register choice (~200, two blocks per SM) schedules a lone
// warp's stage evaluation faster.
template <int STENCIL, int G, int IP>
__global__ void __launch_bounds__(128, G == 1 ? 3 : 2) trace_mixed_plain_kernel(GridDev g, FanDev f, rt_ray_result *__restrict__ out) {
    __shared__ Tableau T;
    __shared__ Base32 btx;
    load_tableau(T, f.integrator, &btx, &g, &f);
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long id = tid / G;
    if (id >= f.n_rays) return;  // whole groups leave together
    const int lane = threadIdx.x & 31, q = lane % G;
    const unsigned gmask = group_mask<G>(lane);
    const long long ray = claim_to_ray(f, id);
    if (ray < 0) return;  // a hole in an ordered plan's claim order: no ray for this group
    Lane L;
    L.active = true;
    lane_begin_ray(L, g, f, ray, btx);
    bool done = lane_launch<STENCIL, G, IP>(L, g, f, q, gmask);
    // the landing state stays in registers here (a shared-memory slot per
    // thread would take L1 that the sample gathers use; measured 3 % slower on
    // the 495k-ray batch), unlike in the persistent kernel
    LandState land;
    // bounded: every attempt counts against max_steps, so max_steps + 1 attempts end every ray
    const long long max_att = (long long)f.max_steps + 2;
    for (long long it = 0; it < max_att && !done; ++it) {
        lane_attempt<STENCIL, G, IP>(L, g, f, T, q, gmask);
        done = lane_end_attempt(L, g, f, land);
    }
    if (!done) L.status = RT_RAY_MAX_STEPS;
    lane_finish(L, g, f, out, q == 0);
}

// Persistent kernel: resident blocks whose warps claim rays from an atomic
// counter (one atomicAdd per warp), between attempts, where all lanes of the
// warp meet; a warp takes its next rays once all of its current ones ended.
template <int STENCIL, int G, int IP>
__global__ void __launch_bounds__(128, G == 1 ? 3 : 2) trace_mixed_persistent_kernel(GridDev g, FanDev f,
                                                                     rt_ray_result *__restrict__ out,
                                                                     unsigned long long *__restrict__ counter) {
    __shared__ Tableau T;
    __shared__ Base32 btx;
    __shared__ LandState land[128];
    load_tableau(T, f.integrator, &btx, &g, &f);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, q = lane % G;
    const unsigned gmask = group_mask<G>(lane);
    Lane L;
    L.active = false;
    bool exhausted = false;  // warp-uniform
    long long iters = 0;
    const long long n = f.n_rays;
    // bound on the warp's loop iterations: every ray ends within max_steps + 1
    // attempts (+ its launch), and a warp runs at most all n rays
    const long long max_iter = ((long long)f.max_steps + 4) * (n + 32) + 64;
    for (;;) {
        // The warp refills once all its rays have ended, with the next 32 / G
        // consecutive claims: rays launched together from neighbouring
        // elevations cross the same cells at the same time, so their stencil
        // gathers coalesce in L1.  Refilling each lane as soon as its ray ends
        // keeps the lanes busier but puts rays of different ages side by side;
        // on the 495,122-ray batch that took 96 ms against 69 ms for warp-wide
        // refills (a refill at 8 / 16 / 24 idle lanes: 84 / 77 / 78 ms).
        const bool idle_warp = !__any_sync(FULL, L.active);
        if (idle_warp && !exhausted) {
            const int n_take = 32 / G;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(counter, (unsigned long long)n_take);
            base = __shfl_sync(FULL, base, 0);
            if (base + (unsigned long long)n_take >= (unsigned long long)n) exhausted = true;
            const unsigned long long c = base + (unsigned long long)(lane / G);
            if (c < (unsigned long long)n) {
                L.active = true;
                lane_begin_ray(L, g, f, claim_to_ray(f, (long long)c), btx);
                if (lane_launch<STENCIL, G, IP>(L, g, f, q, gmask)) lane_finish(L, g, f, out, q == 0);
            }
        }
        if (!__any_sync(FULL, L.active)) break;
        // the warp's rays to their end; the refill above stays out of this
        // hot loop (with it inside, the loop ran 1-2 % slower on the batch)
        bool over = false;
        do {
            if (++iters > max_iter) {  // defensive bound; never reached for valid inputs
                if (L.active) {
                    L.status = RT_RAY_MAX_STEPS;
                    lane_finish(L, g, f, out, q == 0);
                    L.active = false;
                }
                over = true;
                break;
            }
            if (L.active) {
                lane_attempt<STENCIL, G, IP>(L, g, f, T, q, gmask);
                if (lane_end_attempt(L, g, f, land[threadIdx.x])) lane_finish(L, g, f, out, q == 0);
            }
        } while (__any_sync(FULL, L.active));
        if (over) break;
    }
}

// ================================================================ fused fans
// Several small fans on one grid in one launch (the request server's fused
// batches).  Ray i of the launch belongs to fan k with first[k] <= i <
// first[k + 1] (binary search over the n_fans + 1 offsets); its record goes
// to out + first[k] + its index within fan k.  The fans share one integrator
// (the block's Butcher table).  Four lanes per ray, as for any fan too small
// to fill the GPU: the per-ray code is that of the four-lane plain kernel,
// with the fan read from global memory.
template <int STENCIL, int IP>
__global__ void __launch_bounds__(128, 2) trace_mixed_fans_kernel(GridDev g, const FanDev *__restrict__ fans,
                                                                  const long long *__restrict__ first, int n_fans,
                                                                  int integrator, rt_ray_result *__restrict__ out) {
    constexpr int G = 4;
    __shared__ Tableau T;
    load_tableau(T, integrator);
    const long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
    if (i >= first[n_fans]) return;  // whole groups leave together
    int lo = 0, hi = n_fans - 1;
    while (lo < hi) {  // largest k with first[k] <= i
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const FanDev &f = fans[lo];
    const int lane = threadIdx.x & 31, q = lane % G;
    const unsigned gmask = group_mask<G>(lane);
    Lane L;
    L.active = true;
    lane_begin_ray(L, g, f, claim_to_ray(f, i - first[lo]), tx_base(g, f));
    bool done = lane_launch<STENCIL, G, IP>(L, g, f, q, gmask);
    LandState land;
    const long long max_att = (long long)f.max_steps + 2;
    for (long long it = 0; it < max_att && !done; ++it) {
        lane_attempt<STENCIL, G, IP>(L, g, f, T, q, gmask);
        done = lane_end_attempt(L, g, f, land);
    }
    if (!done) L.status = RT_RAY_MAX_STEPS;
    lane_finish(L, g, f, out + first[lo], q == 0);
}

// ================================================================ ionogram
// One warp per (frequency, mode) trace: lanes scan neighbouring elevation
// pairs; the pairs whose landed rays bracket the receiver distance d_rx emit
// an ionogram point, appended through one atomicAdd per warp (ballot +
// popc rank: warp-level compaction).  Branch numbers are assigned after the
// host sorts the points.
__global__ void ionogram_kernel(const rt_ray_result *__restrict__ res, const double *__restrict__ freq,
                                const double *__restrict__ el, int n_freq, int n_modes, int mode0, int n_el,
                                double d_rx, rt_ionogram_point *__restrict__ out, unsigned long long cap,
                                unsigned long long *__restrict__ count) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long trace = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
    if (trace >= (long long)n_freq * n_modes) return;  // whole warps leave together
    const int fi = (int)(trace / n_modes), mi = (int)(trace % n_modes);
    const rt_ray_result *row = res + trace * n_el;  // the fan has one azimuth
    for (int j0 = 0; j0 < n_el - 1; j0 += 32) {
        const int j = j0 + lane;
        bool hit = false;
        rt_ionogram_point p;
        if (j < n_el - 1) {
            const rt_ray_result a = row[j], b = row[j + 1];
            if (a.status == RT_RAY_LANDED && b.status == RT_RAY_LANDED) {
                const double fa = a.ground_range_km - d_rx, fb = b.ground_range_km - d_rx;
                if ((fa < 0.0 && fb >= 0.0) || (fa >= 0.0 && fb < 0.0)) {
                    const double t = fa / (fa - fb);
                    p.freq_mhz = freq[fi];
                    p.group_path_km = a.group_path_km + t * (b.group_path_km - a.group_path_km);
                    p.el_deg = el[j] + t * (el[j + 1] - el[j]);
                    p.ground_range_km = d_rx;
                    p.mode = (mi == 0) ? mode0 : -1;
                    p.branch = 0;
                    hit = true;
                }
            }
        }
        const unsigned m = __ballot_sync(FULL, hit);
        if (m) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(m));
            base = __shfl_sync(FULL, base, 0);
            if (hit) {
                const unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
                if (idx < cap) out[idx] = p;
            }
        }
    }
}

cudaError_t launch_ionogram(const rt_ray_result *res, const double *freq, const double *el, int n_freq, int n_modes,
                            int mode0, int n_el, double d_rx, rt_ionogram_point *out, unsigned long long cap,
                            unsigned long long *count, cudaStream_t st) {
    const long long threads = (long long)n_freq * n_modes * 32;
    if (threads == 0) return cudaSuccess;
    ionogram_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(res, freq, el, n_freq, n_modes, mode0, n_el,
                                                                      d_rx, out, cap, count);
    return cudaGetLastError();
}

// ============================================================== diagnostics
__global__ void eval_rhs_kernel(GridDev g, const double *__restrict__ ys, double *__restrict__ dys,
                                double *__restrict__ mu2s, double freq_mhz, int mode, int precision, int stencil,
                                long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double y[6], dy[6], mu2 = 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) y[c] = ys[i * 6 + c];
    if (precision == RT_FP64) {
        const RayPhys<double> rp = make_phys<double>(g, freq_mhz * 1e6, mode);
        rhs64(g, rp, y, dy, &mu2);
    } else {
        const RayPhys<float> rp = make_phys<float>(g, freq_mhz * 1e6, mode);
        Base32 b;
        base_from_state(g, y, b);
        float d[6] = {0, 0, 0, 0, 0, 0}, dyf[6], m2;
        if (g.interp == 1) {
            if (stencil == RT_STENCIL_TABLE) rhs_mixed<RT_STENCIL_TABLE, 1, 1>(g, rp, b, d, dyf, &m2, 0, 0u);
            else if (stencil == RT_STENCIL_GATHER) rhs_mixed<RT_STENCIL_GATHER, 1, 1>(g, rp, b, d, dyf, &m2, 0, 0u);
            else rhs_mixed<RT_STENCIL_QUAD, 1, 1>(g, rp, b, d, dyf, &m2, 0, 0u);
        } else {
            if (stencil == RT_STENCIL_TABLE) rhs_mixed<RT_STENCIL_TABLE, 1, 0>(g, rp, b, d, dyf, &m2, 0, 0u);
            else if (stencil == RT_STENCIL_GATHER) rhs_mixed<RT_STENCIL_GATHER, 1, 0>(g, rp, b, d, dyf, &m2, 0, 0u);
            else rhs_mixed<RT_STENCIL_QUAD, 1, 0>(g, rp, b, d, dyf, &m2, 0, 0u);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) dy[c] = dyf[c];
        mu2 = m2;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) dys[i * 6 + c] = dy[c];
    mu2s[i] = mu2;
}

// ================================================================ launchers
// Packs Butcher coefficients A[s][t], B4[s], E[s] (s = 0..5) into the
// two-float4-per-stage layout of Tableau.
static void pack_tableau(Tableau &T, const float A[6][5], const float B4[6], const float E[6], int ns) {
    for (int s = 0; s < 6; ++s) {
        T.lo[s] = make_float4(A[s][0], A[s][1], A[s][2], A[s][3]);
        T.hi[s] = make_float4(A[s][4], B4[s], E[s], 0.0f);
    }
    T.ns = ns;
}

static void fill_tableaus(Tableau tab[2]) {
    float A[6][5], B4[6], E[6];
    auto clear = [&]() {
        for (int s = 0; s < 6; ++s) {
            for (int u = 0; u < 5; ++u) A[s][u] = 0.0f;
            B4[s] = E[s] = 0.0f;
        }
    };
    // classic RK4: a21 = a32 = 1/2, a43 = 1; b = (1, 2, 2, 1)/6; A[s][t] = a[s+1+t][s]
    clear();
    double a4[4][4] = {{0}};
    a4[1][0] = 0.5;
    a4[2][1] = 0.5;
    a4[3][2] = 1.0;
    const double b4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    for (int s = 0; s < 4; ++s) {
        for (int u = 0; u < 5; ++u) A[s][u] = (s + 1 + u < 4) ? (float)a4[s + 1 + u][s] : 0.0f;
        B4[s] = (float)b4[s];
    }
    pack_tableau(tab[0], A, B4, E, 4);
    // Fehlberg 4(5)
    clear();
    double a[6][6] = {{0}};
    a[1][0] = 1.0 / 4.0;
    a[2][0] = 3.0 / 32.0;
    a[2][1] = 9.0 / 32.0;
    a[3][0] = 1932.0 / 2197.0;
    a[3][1] = -7200.0 / 2197.0;
    a[3][2] = 7296.0 / 2197.0;
    a[4][0] = 439.0 / 216.0;
    a[4][1] = -8.0;
    a[4][2] = 3680.0 / 513.0;
    a[4][3] = -845.0 / 4104.0;
    a[5][0] = -8.0 / 27.0;
    a[5][1] = 2.0;
    a[5][2] = -3544.0 / 2565.0;
    a[5][3] = 1859.0 / 4104.0;
    a[5][4] = -11.0 / 40.0;
    const double b4f[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
    const double b5f[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
    for (int s = 0; s < 6; ++s) {
        for (int u = 0; u < 5; ++u) A[s][u] = (s + 1 + u < 6) ? (float)a[s + 1 + u][s] : 0.0f;
        B4[s] = (float)b4f[s];
        E[s] = (float)(b5f[s] - b4f[s]);
    }
    pack_tableau(tab[1], A, B4, E, 6);
}

cudaError_t upload_tableaus() {
    Tableau tab[2];
    fill_tableaus(tab);
    cudaError_t e = cudaMemcpyToSymbol(c_tab, tab, sizeof(tab));
    if (e != cudaSuccess) return e;
    float q[20];
    for (int k = -10; k <= 9; ++k) q[k + 10] = (float)std::exp2(k * 0.25);
    return cudaMemcpyToSymbol(c_pow2q, q, sizeof(q));
}

template <int STENCIL, int G, int IP>
static cudaError_t launch_mixed_gi(const GridDev &g, const FanDev &f, rt_ray_result *out,
                                   unsigned long long *counter, const LaunchPlan &lp, cudaStream_t st) {
    if (lp.kernel == RT_KERNEL_PERSISTENT) {
        trace_mixed_persistent_kernel<STENCIL, G, IP><<<lp.blocks, lp.threads, 0, st>>>(g, f, out, counter);
    } else {
        const long long blocks = (f.n_rays * G + lp.threads - 1) / lp.threads;
        if (lp.started) {
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3((unsigned)blocks);
            lc.blockDim = dim3((unsigned)lp.threads);
            lc.dynamicSmemBytes = (size_t)lp.smem;
            lc.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeLaunchCompletionEvent;
            at[0].val.launchCompletionEvent.event = lp.started;
            at[0].val.launchCompletionEvent.flags = 0;
            lc.attrs = at;
            lc.numAttrs = 1;
            return cudaLaunchKernelEx(&lc, trace_mixed_plain_kernel<STENCIL, G, IP>, g, f, out);
        }
        trace_mixed_plain_kernel<STENCIL, G, IP><<<(unsigned)blocks, lp.threads, (size_t)lp.smem, st>>>(g, f, out);
    }
    return cudaGetLastError();
}

template <int STENCIL, int G, int IP>
static cudaError_t exclusive_smem_gi(int *bytes) {
    int dev = 0, per_sm = 0, per_block = 0, reserved = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, trace_mixed_plain_kernel<STENCIL, G, IP>);
    if (e != cudaSuccess) return e;
    // the block's static + dynamic shared memory plus the per-block
    // reservation take the SM's whole capacity
    const int dyn = std::min(per_block, per_sm - reserved) - (int)fa.sharedSizeBytes;
    if (dyn <= 0) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(trace_mixed_plain_kernel<STENCIL, G, IP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             dyn);
    if (e == cudaSuccess) *bytes = dyn;
    return e;
}

template <int STENCIL, int G>
static cudaError_t exclusive_smem_g(int interp, int *bytes) {
    return interp == 1 ? exclusive_smem_gi<STENCIL, G, 1>(bytes) : exclusive_smem_gi<STENCIL, G, 0>(bytes);
}

template <int STENCIL>
static cudaError_t exclusive_smem_s(int lanes, int interp, int *bytes) {
    switch (lanes) {
        case 2: return exclusive_smem_g<STENCIL, 2>(interp, bytes);
        case 4: return exclusive_smem_g<STENCIL, 4>(interp, bytes);
        default: return exclusive_smem_g<STENCIL, 1>(interp, bytes);
    }
}

cudaError_t plain_exclusive_smem(const LaunchPlan &lp, int interp, int *bytes) {
    switch (lp.stencil) {
        case RT_STENCIL_GATHER: return exclusive_smem_s<RT_STENCIL_GATHER>(lp.lanes, interp, bytes);
        case RT_STENCIL_TABLE: return exclusive_smem_s<RT_STENCIL_TABLE>(lp.lanes, interp, bytes);
        default: return exclusive_smem_s<RT_STENCIL_QUAD>(lp.lanes, interp, bytes);
    }
}

template <int STENCIL, int G>
static cudaError_t launch_mixed_g(const GridDev &g, const FanDev &f, rt_ray_result *out,
                                  unsigned long long *counter, const LaunchPlan &lp, cudaStream_t st) {
    return g.interp == 1 ? launch_mixed_gi<STENCIL, G, 1>(g, f, out, counter, lp, st)
                         : launch_mixed_gi<STENCIL, G, 0>(g, f, out, counter, lp, st);
}

template <int STENCIL>
static cudaError_t launch_mixed(const GridDev &g, const FanDev &f, rt_ray_result *out,
                                unsigned long long *counter, const LaunchPlan &lp, cudaStream_t st) {
    switch (lp.lanes) {
        case 2: return launch_mixed_g<STENCIL, 2>(g, f, out, counter, lp, st);
        case 4: return launch_mixed_g<STENCIL, 4>(g, f, out, counter, lp, st);
        default: return launch_mixed_g<STENCIL, 1>(g, f, out, counter, lp, st);
    }
}

cudaError_t launch_trace_only(const GridDev &g, const FanDev &f, rt_ray_result *out, unsigned long long *counter,
                              const LaunchPlan &lp, cudaStream_t st) {
    if (f.n_rays == 0) return cudaSuccess;
    if (f.precision == RT_FP64) {
        const int threads = 128;
        const long long blocks = (f.n_rays + threads - 1) / threads;
        trace_fp64_kernel<<<(unsigned)blocks, threads, 0, st>>>(g, f, out);
        return cudaGetLastError();
    }
    switch (lp.stencil) {
        case RT_STENCIL_GATHER: return launch_mixed<RT_STENCIL_GATHER>(g, f, out, counter, lp, st);
        case RT_STENCIL_TABLE: return launch_mixed<RT_STENCIL_TABLE>(g, f, out, counter, lp, st);
        default: return launch_mixed<RT_STENCIL_QUAD>(g, f, out, counter, lp, st);
    }
}

cudaError_t launch_finish(const GridDev &g, const FanDev &f, rt_ray_result *out, long long n, cudaStream_t st) {
    if (f.precision == RT_FP64 || n == 0) return cudaSuccess;  // the FP64 kernel writes final records itself
    const int threads = 128;
    finish_records_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(g.R_E, f, out, n);
    return cudaGetLastError();
}

cudaError_t launch_trace(const GridDev &g, const FanDev &f, rt_ray_result *out, unsigned long long *counter,
                         const LaunchPlan &lp, cudaStream_t st) {
    const cudaError_t e = launch_trace_only(g, f, out, counter, lp, st);
    if (e != cudaSuccess) return e;
    return launch_finish(g, f, out, f.n_rays, st);
}

template <int STENCIL>
static cudaError_t launch_fans_s(const GridDev &g, const FanDev *fans, const long long *first, int n_fans,
                                 long long n_total, int integrator, rt_ray_result *out, int threads, cudaStream_t st) {
    const unsigned blocks = (unsigned)((n_total * 4 + threads - 1) / threads);  // four lanes per ray
    if (g.interp == 1)
        trace_mixed_fans_kernel<STENCIL, 1><<<blocks, threads, 0, st>>>(g, fans, first, n_fans, integrator, out);
    else
        trace_mixed_fans_kernel<STENCIL, 0><<<blocks, threads, 0, st>>>(g, fans, first, n_fans, integrator, out);
    return cudaGetLastError();
}

cudaError_t launch_trace_fans(const GridDev &g, const FanDev *fans, const long long *first, int n_fans,
                              long long n_total, int integrator, rt_ray_result *out, const LaunchPlan &lp,
                              cudaStream_t st) {
    if (n_total == 0) return cudaSuccess;
    cudaError_t e;
    switch (lp.stencil) {
        case RT_STENCIL_GATHER:
            e = launch_fans_s<RT_STENCIL_GATHER>(g, fans, first, n_fans, n_total, integrator, out, lp.threads, st);
            break;
        case RT_STENCIL_TABLE:
            e = launch_fans_s<RT_STENCIL_TABLE>(g, fans, first, n_fans, n_total, integrator, out, lp.threads, st);
            break;
        default:
            e = launch_fans_s<RT_STENCIL_QUAD>(g, fans, first, n_fans, n_total, integrator, out, lp.threads, st);
    }
    if (e != cudaSuccess) return e;
    const int threads = 128;
    finish_fans_records_kernel<<<(unsigned)((n_total + threads - 1) / threads), threads, 0, st>>>(g.R_E, fans, first,
                                                                                                 n_fans, out);
    return cudaGetLastError();
}

template <int STENCIL>
static cudaError_t occupancy_s(int lanes, int threads, int *blocks_per_sm) {
    switch (lanes) {
        case 2:
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                blocks_per_sm, trace_mixed_persistent_kernel<STENCIL, 2, 0>, threads, 0);
        case 4:
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                blocks_per_sm, trace_mixed_persistent_kernel<STENCIL, 4, 0>, threads, 0);
        default:
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                blocks_per_sm, trace_mixed_persistent_kernel<STENCIL, 1, 0>, threads, 0);
    }
}

cudaError_t persistent_occupancy(int stencil, int lanes, int threads, int *blocks_per_sm) {
    switch (stencil) {
        case RT_STENCIL_GATHER: return occupancy_s<RT_STENCIL_GATHER>(lanes, threads, blocks_per_sm);
        case RT_STENCIL_TABLE: return occupancy_s<RT_STENCIL_TABLE>(lanes, threads, blocks_per_sm);
        default: return occupancy_s<RT_STENCIL_QUAD>(lanes, threads, blocks_per_sm);
    }
}

cudaError_t launch_eval_rhs(const GridDev &g, const double *ys, double *dys, double *mu2s, double freq_mhz, int mode,
                            int precision, int stencil, long long n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int threads = 128;
    eval_rhs_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(g, ys, dys, mu2s, freq_mhz, mode,
                                                                               precision, stencil, n);
    return cudaGetLastError();
}

}  // namespace rtgd
