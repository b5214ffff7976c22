// rtgd_device.cuh -- device-side building blocks of the RTM-GD tracer.
//
// Everything the stage evaluation needs, written once and instantiated for
// double (the all-FP64 path) and float (the mixed path):
//   - p = 3 Galerkin-Difference weights and their derivatives (Appendix A),
//   - the 4x4x4 tensor contraction of Eq. 13 giving Ne and its gradient,
//   - the centred dipole field and its Jacobian in local spherical components,
//   - Appleton-Hartree (Eq. 3) with hand-derived partial derivatives,
//   - the Hamiltonian partials (Eq. 2) and the ray equations (Eq. 1a-1f).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rtgd.h"

namespace rtgd {

constexpr double kPi = 3.14159265358979323846;
constexpr double kRad2Deg = 180.0 / kPi;
constexpr double kDeg2Rad = kPi / 180.0;
// f_N^2 = 80.6 Ne (Hz^2, Ne in m^-3), so X = f_N^2 / f^2 (Sec. II-A).
constexpr double kPlasmaHz2PerM3 = 80.6;
// f_H = e B / (2 pi m_e) in Hz per tesla, so Y = f_H / f (Sec. II-A).
constexpr double kGyroHzPerTesla = 2.7992489872e10;

// Device view of a grid.  Node (i, j, k), i in [0, n_lat), sits at padded
// index (i+1, j+1, k+1) of the ghost-padded arrays.
struct GridDev {
    int n_lat, n_lon, n_alt;
    int p_lon, p_alt;                // padded sizes n_lon + 2, n_alt + 2
    int q_alt;                       // n_alt - 1 cells per (lat, lon) row of the quad layout
    double lat0, lon0, alt0;
    double inv_dlat, inv_dlon, inv_dalt;
    double R_E, top;                 // earth radius; top = alt0 + (n_alt - 1) dalt
    double b0;                       // dipole strength (0: isotropic)
    double m[3];                     // unit vector to the geomagnetic north pole
    float sa, sb, sc;                // d(grid coord)/d(theta, phi, r): -rad2deg/dlat, rad2deg/dlon, 1/dalt
    float R_Ef, mf[3];               // float copies of R_E and m
    float top_f;                     // top as float
    int iso;                         // no field (b0 == 0)
    int interp;                      // 0: Galerkin-Difference p=3, 1: Catmull-Rom (comparison)
    const double *pad64;             // (n_lat+2)(n_lon+2)(n_alt+2) doubles
    const float *pad32;              // same, rounded to float
    const float4 *quad;              // (n_lat+2)(n_lon+2)(n_alt-1): samples k-1..k+2 of cell k
    const float4 *table;             // (n_lat-1)(n_lon-1)(n_alt-1) cells x 16 float4 (64 samples)
};

// --------------------------------------------------------------------------
// GD p = 3 weights (Appendix A).  For a point at local coordinate t in [0, 1]
// of the cell [x_j, x_{j+1}], the weight of node j-1 is the printed piece
// psi_1 (in powers of t), of node j the piece psi_0, of node j+1 psi_{-1} and
// of node j+2 psi_{-2}.  The global basis function is even, so the last two
// are the first two mirrored: w_{j+1}(t) = w_j(1-t), w_{j+2}(t) = w_{j-1}(1-t).
// w[a] / d[a] hold the weight of node j-1+a and its t-derivative.
template <typename R>
__device__ __forceinline__ void gd_weights(R t, R w[4], R d[4]) {
    const R s = R(1) - t;
    w[0] = t * (R(-0.5) + t * (R(11.0 / 12.0) + t * (R(-1.0 / 6.0) + t * (R(-5.0 / 12.0) + t * R(1.0 / 6.0)))));
    w[1] = R(1) + t * t * (R(-2.25) + t * (R(0.5) + t * (R(1.25) - t * R(0.5))));
    w[2] = R(1) + s * s * (R(-2.25) + s * (R(0.5) + s * (R(1.25) - s * R(0.5))));
    w[3] = s * (R(-0.5) + s * (R(11.0 / 12.0) + s * (R(-1.0 / 6.0) + s * (R(-5.0 / 12.0) + s * R(1.0 / 6.0)))));
    d[0] = R(-0.5) + t * (R(11.0 / 6.0) + t * (R(-0.5) + t * (R(-5.0 / 3.0) + t * R(5.0 / 6.0))));
    d[1] = t * (R(-4.5) + t * (R(1.5) + t * (R(5.0) - t * R(2.5))));
    d[2] = -(s * (R(-4.5) + s * (R(1.5) + s * (R(5.0) - s * R(2.5)))));
    d[3] = -(R(-0.5) + s * (R(11.0 / 6.0) + s * (R(-0.5) + s * (R(-5.0 / 3.0) + s * R(5.0 / 6.0)))));
}

// The weights of nodes j-1 and j (and their t-derivatives) at local
// coordinate s; mirrored (s = 1 - t, derivatives negated) they are the
// weights of nodes j+2 and j+1.  interp 0: GD p = 3 (Appendix A); interp 1:
// Catmull-Rom (Eq. 7), w_{-1} = (-s^3 + 2s^2 - s)/2, w_0 = (3s^3 - 5s^2 + 2)/2,
// whose mirror images are w_2 and w_1.
template <typename R>
__device__ __forceinline__ void gd_half(R s, R &wm1, R &w0, R &dm1, R &d0, int interp = 0) {
    if (interp == 1) {
        wm1 = s * (R(-0.5) + s * (R(1) - s * R(0.5)));
        w0 = R(1) + s * s * (R(-2.5) + s * R(1.5));
        dm1 = R(-0.5) + s * (R(2) - s * R(1.5));
        d0 = s * (R(-5) + s * R(4.5));
        return;
    }
    wm1 = s * (R(-0.5) + s * (R(11.0 / 12.0) + s * (R(-1.0 / 6.0) + s * (R(-5.0 / 12.0) + s * R(1.0 / 6.0)))));
    w0 = R(1) + s * s * (R(-2.25) + s * (R(0.5) + s * (R(1.25) - s * R(0.5))));
    dm1 = R(-0.5) + s * (R(11.0 / 6.0) + s * (R(-0.5) + s * (R(-5.0 / 3.0) + s * R(5.0 / 6.0))));
    d0 = s * (R(-4.5) + s * (R(1.5) + s * (R(5.0) - s * R(2.5))));
}

// gd_half with the interpolant fixed at compile time (IP = 0 GD, 1 CR).
template <typename R, int IP>
__device__ __forceinline__ void half_weights(R s, R &wm1, R &w0, R &dm1, R &d0) {
    if (IP == 1) {
        wm1 = s * (R(-0.5) + s * (R(1) - s * R(0.5)));
        w0 = R(1) + s * s * (R(-2.5) + s * R(1.5));
        dm1 = R(-0.5) + s * (R(2) - s * R(1.5));
        d0 = s * (R(-5) + s * R(4.5));
    } else {
        wm1 = s * (R(-0.5) + s * (R(11.0 / 12.0) + s * (R(-1.0 / 6.0) + s * (R(-5.0 / 12.0) + s * R(1.0 / 6.0)))));
        w0 = R(1) + s * s * (R(-2.25) + s * (R(0.5) + s * (R(1.25) - s * R(0.5))));
        dm1 = R(-0.5) + s * (R(11.0 / 6.0) + s * (R(-0.5) + s * (R(-5.0 / 3.0) + s * R(5.0 / 6.0))));
        d0 = s * (R(-4.5) + s * (R(1.5) + s * (R(5.0) - s * R(2.5))));
    }
}

// All four weights of one axis, interpolant fixed at compile time: nodes j-1,
// j from half_weights(t), nodes j+2, j+1 from its mirror half_weights(1 - t).
template <typename R, int IP>
__device__ __forceinline__ void axis_weights(R t, R w[4], R d[4]) {
    R wp2, wp1, dp2, dp1;
    half_weights<R, IP>(t, w[0], w[1], d[0], d[1]);
    half_weights<R, IP>(R(1) - t, wp2, wp1, dp2, dp1);
    w[2] = wp1;
    w[3] = wp2;
    d[2] = -dp1;
    d[3] = -dp2;
}

// All four weights of one axis (w[a], d[a] for node j-1+a), GD or CR.
template <typename R>
__device__ __forceinline__ void interp_weights(R t, R w[4], R d[4], int interp) {
    if (interp == 1) {
        R wm1, w0, dm1, d0, wp2, wp1, dp2, dp1;
        gd_half<R>(t, wm1, w0, dm1, d0, 1);
        gd_half<R>(R(1) - t, wp2, wp1, dp2, dp1, 1);
        w[0] = wm1;
        w[1] = w0;
        w[2] = wp1;
        w[3] = wp2;
        d[0] = dm1;
        d[1] = d0;
        d[2] = -dp1;
        d[3] = -dp2;
        return;
    }
    gd_weights<R>(t, w, d);
}

// Eq. 13 contraction of one row of 4 altitude samples.  PACK (float only):
// packed FMAs on the sample pairs (u0, u1) and (u2, u3) against the weight
// pairs, then one addition per sum -- four instructions fewer per two sums
// and a shorter chain; the sum is formed in another order (pairs first).
template <typename R, bool PACK = false>
__device__ __forceinline__ void row4(R u0, R u1, R u2, R u3, const R wc[4], const R dc[4], R &v, R &dv) {
    v = u0 * wc[0] + u1 * wc[1] + u2 * wc[2] + u3 * wc[3];
    dv = u0 * dc[0] + u1 * dc[1] + u2 * dc[2] + u3 * dc[3];
}

template <>
__device__ __forceinline__ void row4<float, true>(float u0, float u1, float u2, float u3, const float wc[4],
                                                  const float dc[4], float &v, float &dv) {
    const float2 a = make_float2(u0, u1), b = make_float2(u2, u3);
    const float2 p = __ffma2_rn(b, make_float2(wc[2], wc[3]), __fmul2_rn(a, make_float2(wc[0], wc[1])));
    const float2 q = __ffma2_rn(b, make_float2(dc[2], dc[3]), __fmul2_rn(a, make_float2(dc[0], dc[1])));
    v = p.x + p.y;
    dv = q.x + q.y;
}

// Accumulates the (a, b) row into the lon/lat partial sums.
template <typename R>
__device__ __forceinline__ void acc_row(R v, R dv, R wb, R db, R &s, R &sb, R &sc) {
    s += v * wb;
    sb += v * db;
    sc += dv * wb;
}

// Partial sums {Ne - REF, dNe/dxa, dNe/dxb, dNe/dxc} (per-cell units) over
// the rows a = A0 .. A0+NA-1 (all b) of the 16 rows of 4 altitude samples;
// wa/da hold the NA lat-weights of those rows.  ROW(a, b, u0..u3) loads row
// (a, b).  The samples are contracted relative to REF (Ne = REF + sum (u -
// REF) w, the weights summing to 1 and their derivatives to 0), so that in
// float the sums do not cancel against the magnitude of Ne; the caller adds
// REF back (after combining partial sums, when the rows are split).  PACK
// selects the packed altitude rows (row4).
#define RTGD_CONTRACT(R, PACK, ROW, REF, A0, NA, wa, da, wb, db, wc, dc, out)     \
    do {                                                                          \
        R n_ = R(0), na_ = R(0), nb_ = R(0), nc_ = R(0);                          \
        _Pragma("unroll") for (int a_ = 0; a_ < (NA); ++a_) {                     \
            R s_ = R(0), sb_ = R(0), sc_ = R(0);                                  \
            _Pragma("unroll") for (int b_ = 0; b_ < 4; ++b_) {                    \
                R u0_, u1_, u2_, u3_, v_, dv_;                                    \
                ROW((A0) + a_, b_, u0_, u1_, u2_, u3_);                           \
                u0_ -= (REF);                                                     \
                u1_ -= (REF);                                                     \
                u2_ -= (REF);                                                     \
                u3_ -= (REF);                                                     \
                row4<R, (PACK)>(u0_, u1_, u2_, u3_, wc, dc, v_, dv_);             \
                acc_row<R>(v_, dv_, wb[b_], db[b_], s_, sb_, sc_);                \
            }                                                                     \
            n_ += s_ * wa[a_];                                                    \
            na_ += s_ * da[a_];                                                   \
            nb_ += sb_ * wa[a_];                                                  \
            nc_ += sc_ * wa[a_];                                                  \
        }                                                                         \
        out[0] = n_;                                                              \
        out[1] = na_;                                                             \
        out[2] = nb_;                                                             \
        out[3] = nc_;                                                             \
    } while (0)

// 1/x: correctly rounded in double; in float the fast reciprocal (MUFU.RCP,
// within 2 ulp), which is ample for the mixed path's tolerance.
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }

// sqrt: correctly rounded in double; in float x * rsqrt(x) (MUFU.RSQ, a few
// ulp, no special-case branch), 0 for x <= 0.
__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float fsqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// a / b: correctly rounded in double; in float the fast division (MUFU.RCP
// based, 2 ulp, no special-case branch) for the step-control arithmetic.
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }

// Cell index and local coordinate along one axis; false outside [0, n-1].
template <typename R>
__device__ __forceinline__ bool cell_coord(R x, int n, int &i, R &t) {
    if (!(x >= R(0) && x <= R(n - 1))) return false;
    R f = floor(x);
    int fi = (int)f;
    if (fi > n - 2) fi = n - 2;
    i = fi;
    t = x - R(fi);
    return true;
}

// --------------------------------------------------------------------------
// Physics at one stage: everything after the interpolation.
template <typename R>
struct StageIn {
    R r, sth, cth, sph, cph;  // position (km, sin/cos of colatitude and longitude)
    R k[3];                   // wave vector (r, theta, phi components), units of omega/c
    R X;                      // f_N^2 / f^2
    R dX[3];                  // dX/dr, dX/dtheta, dX/dphi
};

// Per-ray physics constants in the precision of the stage arithmetic.
template <typename R>
struct RayPhys {
    R xfac;   // 80.6 / f^2: X = xfac * Ne
    R ab0;    // (kGyroHzPerTesla / f) * B0: |Y| at the magnetic equator on the ground
    R R_E;
    R m[3];   // unit vector to the geomagnetic north pole
    bool iso; // no field
    int mode; // +1 ordinary, -1 extraordinary
};

template <typename R>
__device__ __forceinline__ RayPhys<R> make_phys(const GridDev &g, double f_hz, int mode) {
    RayPhys<R> p;
    p.xfac = R(kPlasmaHz2PerM3 / (f_hz * f_hz));
    p.ab0 = R(kGyroHzPerTesla / f_hz * g.b0);
    p.R_E = R(g.R_E);
    p.m[0] = R(g.m[0]);
    p.m[1] = R(g.m[1]);
    p.m[2] = R(g.m[2]);
    p.iso = g.iso != 0;
    p.mode = mode;
    return p;
}

// Appleton-Hartree mu^2(X, L = Y_L^2, T = Y_T^2) (Eq. 3) and its partials.
// Ordinary wave (upper sign): the printed denominator 2u - T + S (u = 1 - X,
// S = sqrt(T^2 + 4 L u^2)) is rewritten with S - T = 4 L u^2 / (S + T), which
// gives mu^2 = 1 - X / (1 + g), g = 2 L u / (S + T): the same function, free
// of the 0/0 at X = 1.  Extraordinary wave: the printed form.
template <typename R>
__device__ __forceinline__ void appleton_hartree(R X, R L, R T, int mode, R &mu2, R &FX, R &FL, R &FT) {
    const R u = R(1) - X;
    const R S = fsqrt(T * T + R(4) * L * u * u);
    if (mode > 0) {
        // one reciprocal gives 1/S, 1/W and 1/(1 + g) = W/V with V = W + 2 L u
        const R W = S + T;
        const R V = W + R(2) * L * u;
        const R SW = S * W;
        const R m = recip(SW * V);
        const R iS = W * V * m;
        const R iW = S * V * m;
        const R g = R(2) * L * u * iW;
        const R opg = R(1) + g;
        const R iopg = SW * W * m;
        const R gX = R(2) * L * (R(4) * L * u * u * iS - W) * iW * iW;
        const R gL = R(2) * u * iW - R(4) * L * u * u * u * iS * iW * iW;
        const R gT = -g * iS;
        mu2 = R(1) - X * iopg;
        const R i2 = iopg * iopg;
        FX = (X * gX - opg) * i2;
        FL = X * gL * i2;
        FT = X * gT * i2;
    } else {
        const R D = R(2) * u - T - S;
        const R m = recip(S * D);  // 1/S and 1/D from one reciprocal
        const R iS = D * m;
        const R iD = S * m;
        const R N = R(2) * X * u;
        const R SX = R(-4) * L * u * iS;
        const R SL = R(2) * u * u * iS;
        const R ST = T * iS;
        const R iD2 = iD * iD;
        mu2 = R(1) - N * iD;
        FX = (N * (R(-2) - SX) - (R(2) - R(4) * X) * D) * iD2;
        FL = N * (-SL) * iD2;
        FT = N * (R(-1) - ST) * iD2;
    }
}

// Field terms of one stage that do not depend on the electron density: the
// centred dipole Y = A (-2 m_r, m_th, m_ph) with A = ab0 (R_E / r)^3, |Y|^2,
// k . Y, and the partials of |Y|^2 and of k . Y along (r, theta, phi).  From
// dm_r/dth = m_th, dm_th/dth = -m_r, dm_ph/dth = 0, dm_r/dph = sin m_ph,
// dm_th/dph = cos m_ph, dm_ph/dph = -(sin m_r + cos m_th):
//   dY/dr = -3 Y / r,  dY/dth = A (-2 m_th, -m_r, 0),
//   dY/dph = A (-2 sin m_ph, cos m_ph, -(sin m_r + cos m_th)),
// so d|Y|^2/dx = 2 Y . dY/dx = (-6 |Y|^2 / r, 6 A^2 m_r m_th, 6 A^2 m_r sin m_ph).
template <typename R>
struct FieldTerms {
    R Y[3];     // Y (units of the wave frequency)
    R YY, kY;   // |Y|^2, k . Y
    R gYY[3];   // d|Y|^2 / d(r, theta, phi)
    R gkY[3];   // d(k . Y) / d(r, theta, phi) at fixed k
    R ir;       // 1 / r
};

template <typename R>
__device__ __forceinline__ FieldTerms<R> field_terms(const RayPhys<R> &rp, const StageIn<R> &s) {
    FieldTerms<R> F;
    const R kr = s.k[0], kt = s.k[1], kp = s.k[2];
    const R mx = rp.m[0], my = rp.m[1], mz = rp.m[2];
    const R mr = mx * s.sth * s.cph + my * s.sth * s.sph + mz * s.cth;
    const R mt = mx * s.cth * s.cph + my * s.cth * s.sph - mz * s.sth;
    const R mp = -mx * s.sph + my * s.cph;
    F.ir = recip(s.r);
    const R q = rp.R_E * F.ir;
    const R A = rp.ab0 * q * q * q;
    F.Y[0] = R(-2) * A * mr;
    F.Y[1] = A * mt;
    F.Y[2] = A * mp;
    const R A2 = A * A;
    F.YY = A2 * (R(1) + R(3) * mr * mr);  // m is a unit vector
    F.kY = kr * F.Y[0] + kt * F.Y[1] + kp * F.Y[2];
    const R smp = s.sth * mp;
    const R A6mr = R(6) * A2 * mr;
    F.gYY[0] = R(-6) * F.YY * F.ir;
    F.gYY[1] = A6mr * mt;
    F.gYY[2] = A6mr * smp;
    F.gkY[0] = R(-3) * F.kY * F.ir;
    F.gkY[1] = A * (R(-2) * kr * mt - kt * mr);
    F.gkY[2] = A * (R(-2) * kr * smp + kt * s.cth * mp - kp * (s.sth * mr + s.cth * mt));
    return F;
}

// Hamiltonian H = (|k|^2 - mu^2)/2 (Eq. 2, k in units of omega/c) and the ray
// equations (Eq. 1a-1f, with k_phi sin(theta) dphi/dP' in the k_r equation as
// the canonical momentum p_phi = r sin(theta) k_phi requires).  With G =
// omega dH/domega at fixed k:
//   dr/dP' = -H_kr/G, dtheta/dP' = -H_kth/(r G), dphi/dP' = -H_kph/(r sin G),
//   dk_r/dP'   = H_r/G + k_th dtheta + k_ph sin dphi,
//   dk_th/dP'  = (H_th/G - k_th dr + k_ph r cos dphi) / r,
//   dk_ph/dP'  = (H_ph/G - k_ph sin dr - k_ph r cos dtheta) / (r sin).
// F holds the field terms of the same stage; mu2_out receives mu^2.
template <typename R>
__device__ __forceinline__ void ray_rhs(const RayPhys<R> &rp, const StageIn<R> &s, const FieldTerms<R> &F, R dy[6],
                                        R *mu2_out) {
    const R kr = s.k[0], kt = s.k[1], kp = s.k[2];
    const R kk = kr * kr + kt * kt + kp * kp;
    R Hr, Ht, Hp, Hk0, Hk1, Hk2, G, mu2;
    if (rp.iso) {
        // no field: mu^2 = 1 - X, so H_x = grad(X)/2, H_k = k, G = -|k|^2 - X
        mu2 = R(1) - s.X;
        Hr = R(0.5) * s.dX[0];
        Ht = R(0.5) * s.dX[1];
        Hp = R(0.5) * s.dX[2];
        Hk0 = kr;
        Hk1 = kt;
        Hk2 = kp;
        G = -kk - s.X;
    } else {
        const R ikk = recip(kk);
        const R L = F.kY * F.kY * ikk;
        R T = F.YY - L;
        if (T < R(0)) T = R(0);
        R Fm, FX, FL, FT;
        appleton_hartree<R>(s.X, L, T, rp.mode, Fm, FX, FL, FT);
        mu2 = Fm;
        // mu^2 = F(X, L, T) with T = Y^2 - L: d/dY^2 = F_T, d/dL|_{Y^2} = F_L - F_T;
        // dL/dx at fixed k = c2 d(k . Y)/dx with c2 = 2 kY / |k|^2
        const R FYL = FL - FT;
        const R c2 = R(2) * F.kY * ikk;
        const R cL = FYL * c2;
        Hr = R(-0.5) * (FX * s.dX[0] + FT * F.gYY[0] + cL * F.gkY[0]);
        Ht = R(-0.5) * (FX * s.dX[1] + FT * F.gYY[1] + cL * F.gkY[1]);
        Hp = R(-0.5) * (FX * s.dX[2] + FT * F.gYY[2] + cL * F.gkY[2]);
        // dL/dk_i = (2 kY / |k|^2) (Y_i - (kY / |k|^2) k_i)
        const R kYn = F.kY * ikk;
        const R hf = R(0.5) * cL;
        Hk0 = kr - hf * (F.Y[0] - kYn * kr);
        Hk1 = kt - hf * (F.Y[1] - kYn * kt);
        Hk2 = kp - hf * (F.Y[2] - kYn * kp);
        // omega dH/domega: X, L and T all scale as omega^-2, |k|^2 as omega^-2
        G = -kk + s.X * FX + L * FL + T * FT;
    }
    const R iG = recip(G);
    const R ir = F.ir;
    const R irs = ir * recip(s.sth);
    const R dr = -Hk0 * iG;
    const R dt = -Hk1 * iG * ir;
    const R dp = -Hk2 * iG * irs;
    dy[0] = dr;
    dy[1] = dt;
    dy[2] = dp;
    dy[3] = Hr * iG + kt * dt + kp * s.sth * dp;
    dy[4] = (Ht * iG - kt * dr + kp * s.r * s.cth * dp) * ir;
    dy[5] = (Hp * iG - kp * s.sth * dr - kp * s.r * s.cth * dt) * irs;
    if (mu2_out) *mu2_out = mu2;
}

}  // namespace rtgd
