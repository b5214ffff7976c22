/*
 * rtgd_oracle.cpp -- plain, slow, FP64 CPU restatement of the RTM-GD ray tracer.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, by the smoke check and by the
 * CPU-baseline leg of bench.py.  The CUDA library never links or calls it, and
 * it shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, in the paper's order (arXiv 2506.18579):
 *   - Sec. II-A, Eq. 1a-1f: Haselgrove ray equations in spherical coordinates
 *     (r, theta = colatitude, phi = longitude), independent variable P' (group
 *     path).  The k_r equation is used with k_phi*sin(theta)*dphi/dP' (the
 *     printed Eq. 1d drops the sin(theta); the canonical-momentum derivation
 *     p_phi = r sin(theta) k_phi requires it).
 *   - Eq. 2: H = 1/2 [c^2 k^2 / omega^2 - mu^2]; Eq. 3: Appleton-Hartree
 *     without collisions, upper sign = ordinary mode.
 *   - Sec. II-B, Eq. 13 and Appendix A: p = 3 Galerkin-Difference tensor
 *     interpolant of Ne over 4x4x4 nodes, built from the four printed quintic
 *     pieces psi_{-2}, psi_{-1}, psi_0, psi_1 of the global basis function.
 *   - Sec. II-C: RK4 integration (fixed step) until the ray returns to the
 *     ground or leaves the ionospheric region; outputs group path, ground
 *     distance, azimuth deviation and reflection height.
 * Every partial derivative of H (position, wave vector, omega) comes from
 * forward-mode dual numbers propagated through the whole evaluation, so no
 * hand-derived derivative formula appears here.
 *
 * Readings of points the paper leaves open (each one stated where used):
 * wave vector in units of omega/c; f_N^2 = 80.6 Ne; f_H = 2.7992489872e10 B;
 * centred tilted dipole instead of IGRF; ghost nodes by quadratic
 * extrapolation; Ne = 0 outside the grid box; RKF45 (Fehlberg 4(5)) as the
 * adaptive option with the error norm and controller documented at rkf45_err;
 * landing (and exit through the grid top) by regula falsi (Illinois) on the
 * size of the last step; reflection
 * height from a cubic Hermite fit on the step where dr/dP' changes sign.
 */
#include "rtgd_oracle.h"

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double DEG = PI / 180.0;
constexpr double PLASMA_HZ2_PER_M3 = 80.6;       /* f_N^2 = 80.6 Ne  (Sec. II-A, X = f_N^2/f^2) */
constexpr double GYRO_HZ_PER_T = 2.7992489872e10; /* f_H = e B / (2 pi m_e)   (Y = f_H/f)       */

/* ---------------------------------------------------------------- duals -- */
/* Variables: r, theta, phi, k_r, k_theta, k_phi, s = ln(omega/omega_0). */
constexpr int NV = 7;
enum { VR = 0, VTH = 1, VPH = 2, VKR = 3, VKTH = 4, VKPH = 5, VS = 6 };

struct Dual {
    double v;
    double d[NV];
};

Dual cst(double x) {
    Dual a;
    a.v = x;
    for (int i = 0; i < NV; ++i) a.d[i] = 0.0;
    return a;
}
Dual var(double x, int i) {
    Dual a = cst(x);
    a.d[i] = 1.0;
    return a;
}
Dual operator+(const Dual &a, const Dual &b) {
    Dual c;
    c.v = a.v + b.v;
    for (int i = 0; i < NV; ++i) c.d[i] = a.d[i] + b.d[i];
    return c;
}
Dual operator-(const Dual &a, const Dual &b) {
    Dual c;
    c.v = a.v - b.v;
    for (int i = 0; i < NV; ++i) c.d[i] = a.d[i] - b.d[i];
    return c;
}
Dual operator-(const Dual &a) {
    Dual c;
    c.v = -a.v;
    for (int i = 0; i < NV; ++i) c.d[i] = -a.d[i];
    return c;
}
Dual operator*(const Dual &a, const Dual &b) {
    Dual c;
    c.v = a.v * b.v;
    for (int i = 0; i < NV; ++i) c.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return c;
}
Dual operator/(const Dual &a, const Dual &b) {
    Dual c;
    c.v = a.v / b.v;
    for (int i = 0; i < NV; ++i) c.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
    return c;
}
Dual operator+(const Dual &a, double b) { return a + cst(b); }
Dual operator-(const Dual &a, double b) { return a - cst(b); }
Dual operator-(double a, const Dual &b) { return cst(a) - b; }
Dual operator*(const Dual &a, double b) { return a * cst(b); }
Dual operator*(double a, const Dual &b) { return cst(a) * b; }
Dual operator/(const Dual &a, double b) { return a / cst(b); }
Dual operator/(double a, const Dual &b) { return cst(a) / b; }

Dual dsqrt(const Dual &a) {
    Dual c;
    c.v = std::sqrt(a.v);
    for (int i = 0; i < NV; ++i) c.d[i] = a.d[i] / (2.0 * c.v);
    return c;
}
Dual dsin(const Dual &a) {
    Dual c;
    c.v = std::sin(a.v);
    const double cs = std::cos(a.v);
    for (int i = 0; i < NV; ++i) c.d[i] = cs * a.d[i];
    return c;
}
Dual dcos(const Dual &a) {
    Dual c;
    c.v = std::cos(a.v);
    const double sn = std::sin(a.v);
    for (int i = 0; i < NV; ++i) c.d[i] = -sn * a.d[i];
    return c;
}
Dual pw(const Dual &a, int n) { /* a^n by repeated products, n >= 1 */
    Dual c = a;
    for (int i = 1; i < n; ++i) c = c * a;
    return c;
}

/* ------------------------------------------------ GD basis, Appendix A -- */
/* Global 1-D basis function psi of the node at offset 0, evaluated at offset
 * xi (in cells).  Its four quintic pieces are the ones printed in Appendix A:
 * psi_{-2} on [-2,-1] in powers of (xi+2), psi_{-1} on [-1,0] in powers of
 * (xi+1), psi_0 on [0,1] in powers of xi, psi_1 on [1,2] in powers of (xi-1);
 * psi vanishes outside [-2, 2]. */
Dual gd_psi(const Dual &xi) {
    const double x = xi.v;
    if (x <= -2.0 || x >= 2.0) return cst(0.0);
    if (x < -1.0) {
        const Dual s = xi + 2.0;
        return -pw(s, 5) / 6.0 + 5.0 * pw(s, 4) / 12.0 + pw(s, 3) / 6.0 - 5.0 * pw(s, 2) / 12.0;
    }
    if (x < 0.0) {
        const Dual s = xi + 1.0;
        return pw(s, 5) / 2.0 - 5.0 * pw(s, 4) / 4.0 - pw(s, 3) / 2.0 + 7.0 * pw(s, 2) / 4.0 + s / 2.0;
    }
    if (x < 1.0) {
        const Dual s = xi;
        return -pw(s, 5) / 2.0 + 5.0 * pw(s, 4) / 4.0 + pw(s, 3) / 2.0 - 9.0 * pw(s, 2) / 4.0 + 1.0;
    }
    const Dual s = xi - 1.0;
    return pw(s, 5) / 6.0 - 5.0 * pw(s, 4) / 12.0 - pw(s, 3) / 6.0 + 11.0 * pw(s, 2) / 12.0 - s / 2.0;
}

/* Catmull-Rom global basis (Eq. 7): the weight w_k(t) of node j+k for t in
 * the cell [j, j+1], rewritten as a function of the offset xi = t - k. */
Dual cr_basis(const Dual &xi) {
    const double x = xi.v;
    if (x <= -2.0 || x >= 2.0) return cst(0.0);
    if (x < -1.0) { /* node j+2, t = xi + 2: w_2 = (t^3 - t^2)/2 */
        const Dual t = xi + 2.0;
        return (pw(t, 3) - pw(t, 2)) / 2.0;
    }
    if (x < 0.0) { /* node j+1, t = xi + 1: w_1 = (-3t^3 + 4t^2 + t)/2 */
        const Dual t = xi + 1.0;
        return (-3.0 * pw(t, 3) + 4.0 * pw(t, 2) + t) / 2.0;
    }
    if (x < 1.0) { /* node j, t = xi: w_0 = (3t^3 - 5t^2 + 2)/2 */
        const Dual t = xi;
        return (3.0 * pw(t, 3) - 5.0 * pw(t, 2) + 2.0) / 2.0;
    }
    const Dual t = xi - 1.0; /* node j-1, t = xi - 1: w_{-1} = (-t^3 + 2t^2 - t)/2 */
    return (-pw(t, 3) + 2.0 * pw(t, 2) - t) / 2.0;
}

/* --------------------------------------------------------------- grid -- */
size_t flat_index(const or_grid &g, int i, int j, int k) {
    return ((size_t)i * (size_t)g.n_lon + (size_t)j) * (size_t)g.n_alt + (size_t)k;
}

/* Nodal value, with one ghost layer on every face obtained by quadratic
 * extrapolation from the three nearest nodes (u_{-1} = 3u_0 - 3u_1 + u_2),
 * applied axis by axis.  This keeps the interpolant exact for tensor
 * polynomials of degree <= 2 up to the grid faces (the paper is silent). */
double node(const or_grid &g, int i, int j, int k) {
    if (i < 0) return 3.0 * node(g, 0, j, k) - 3.0 * node(g, 1, j, k) + node(g, 2, j, k);
    if (i >= g.n_lat) {
        const int n = g.n_lat;
        return 3.0 * node(g, n - 1, j, k) - 3.0 * node(g, n - 2, j, k) + node(g, n - 3, j, k);
    }
    if (j < 0) return 3.0 * node(g, i, 0, k) - 3.0 * node(g, i, 1, k) + node(g, i, 2, k);
    if (j >= g.n_lon) {
        const int n = g.n_lon;
        return 3.0 * node(g, i, n - 1, k) - 3.0 * node(g, i, n - 2, k) + node(g, i, n - 3, k);
    }
    if (k < 0) return 3.0 * node(g, i, j, 0) - 3.0 * node(g, i, j, 1) + node(g, i, j, 2);
    if (k >= g.n_alt) {
        const int n = g.n_alt;
        return 3.0 * node(g, i, j, n - 1) - 3.0 * node(g, i, j, n - 2) + node(g, i, j, n - 3);
    }
    return g.ne[flat_index(g, i, j, k)];
}

int cell_of(double x, int n) { /* cell index in [0, n-2] for x in [0, n-1] */
    int i = (int)std::floor(x);
    if (i > n - 2) i = n - 2;
    if (i < 0) i = 0;
    return i;
}

/* Eq. 13 (q = 2): Ne at fractional grid coordinates (xa, xb, xc) measured in
 * cells from the first node along lat, lon, alt.  Outside the grid box the
 * medium is free space: Ne = 0 with zero gradient. */
Dual ne_index(const or_grid &g, const Dual &xa, const Dual &xb, const Dual &xc, bool *inside) {
    const bool in = xa.v >= 0.0 && xa.v <= g.n_lat - 1 && xb.v >= 0.0 && xb.v <= g.n_lon - 1 &&
                    xc.v >= 0.0 && xc.v <= g.n_alt - 1;
    if (inside) *inside = in;
    if (!in) return cst(0.0);
    const int i = cell_of(xa.v, g.n_lat), j = cell_of(xb.v, g.n_lon), k = cell_of(xc.v, g.n_alt);
    Dual pa[4], pb[4], pc[4];
    for (int a = 0; a < 4; ++a) {
        const int off = a - 1; /* nodes i-1 .. i+2 */
        if (g.interp == 1) {
            pa[a] = cr_basis(xa - (double)(i + off));
            pb[a] = cr_basis(xb - (double)(j + off));
            pc[a] = cr_basis(xc - (double)(k + off));
        } else {
            pa[a] = gd_psi(xa - (double)(i + off));
            pb[a] = gd_psi(xb - (double)(j + off));
            pc[a] = gd_psi(xc - (double)(k + off));
        }
    }
    Dual sum = cst(0.0);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c) {
                const double u = node(g, i + a - 1, j + b - 1, k + c - 1);
                sum = sum + u * (pa[a] * pb[b] * pc[c]);
            }
    return sum;
}

/* Geographic position -> fractional grid coordinates.  lat = 90 deg - theta,
 * lon = phi (taken modulo 360 deg relative to the first grid longitude),
 * alt = r - R_E. */
void grid_coords(const or_grid &g, const Dual &r, const Dual &th, const Dual &ph, Dual *xa,
                 Dual *xb, Dual *xc) {
    const Dual lat = 90.0 - th / DEG;
    Dual lonrel = ph / DEG - g.lon0_deg;
    lonrel.v -= 360.0 * std::floor(lonrel.v / 360.0);
    const Dual alt = r - g.earth_radius_km;
    *xa = (lat - g.lat0_deg) / g.dlat_deg;
    *xb = lonrel / g.dlon_deg;
    *xc = (alt - g.alt0_km) / g.dalt_km;
}

/* ------------------------------------------------------------- dipole -- */
/* Centred tilted dipole standing in for the geomagnetic model of Sec. II-C:
 * B = -B0 (R_E/r)^3 [3 (m.p) p - m], with p the unit position vector and m
 * the unit vector towards the geomagnetic north pole; |B| = B0 on the
 * magnetic equator at r = R_E.  Returned as spherical components. */
void dipole(const or_grid &g, const Dual &r, const Dual &th, const Dual &ph, Dual B[3]) {
    const Dual st = dsin(th), ct = dcos(th), sp = dsin(ph), cp = dcos(ph);
    const Dual p[3] = {st * cp, st * sp, ct};
    const Dual eth[3] = {ct * cp, ct * sp, -st};
    const Dual eph[3] = {-sp, cp, cst(0.0)};
    const double plat = g.pole_lat_deg * DEG, plon = g.pole_lon_deg * DEG;
    const double m[3] = {std::cos(plat) * std::cos(plon), std::cos(plat) * std::sin(plon),
                         std::sin(plat)};
    const Dual mp = m[0] * p[0] + m[1] * p[1] + m[2] * p[2];
    const Dual q = pw(g.earth_radius_km / r, 3) * (-g.b0_tesla);
    Dual bc[3];
    for (int i = 0; i < 3; ++i) bc[i] = q * (3.0 * mp * p[i] - m[i]);
    B[0] = bc[0] * p[0] + bc[1] * p[1] + bc[2] * p[2];
    B[1] = bc[0] * eth[0] + bc[1] * eth[1] + bc[2] * eth[2];
    B[2] = bc[0] * eph[0] + bc[1] * eph[1] + bc[2] * eph[2];
}

/* ----------------------------------------------- Appleton-Hartree, Eq. 3 -- */
/* mu^2 = 1 - 2X(1-X) / (2(1-X) - Y_T^2 +/- sqrt(Y_T^4 + 4 Y_L^2 (1-X)^2)),
 * mode = +1 takes the upper sign (ordinary wave), -1 the lower (extraordinary).
 * With no field the two modes coincide at mu^2 = 1 - X. */
Dual ah_mu2(const Dual &X, const Dual &YL2, const Dual &YT2, int mode) {
    if (YL2.v == 0.0 && YT2.v == 0.0) return 1.0 - X;
    const Dual u = 1.0 - X;
    const Dual S = dsqrt(YT2 * YT2 + 4.0 * YL2 * u * u);
    const Dual den = 2.0 * u - YT2 + (double)mode * S;
    return 1.0 - 2.0 * X * u / den;
}

/* ---------------------------------------------------- Hamiltonian, Eq. 2 -- */
struct Ctx {
    const or_grid *g;
    double f_hz;
    int mode;
};

/* H(y) = 1/2 (|k|^2 - mu^2) with k in units of omega/c.  The derivative along
 * s = ln(omega) is taken at fixed physical k, so the scaled wave vector, X and
 * Y carry the factors e^{-s}, e^{-2s}, e^{-s}; H.d[VS] is omega dH/domega. */
Dual hamiltonian(const Ctx &c, const double y[6]) {
    const or_grid &g = *c.g;
    const Dual r = var(y[0], VR), th = var(y[1], VTH), ph = var(y[2], VPH);
    Dual es = cst(1.0); /* e^{-s} at s = 0 */
    es.d[VS] = -1.0;
    const Dual k[3] = {var(y[3], VKR) * es, var(y[4], VKTH) * es, var(y[5], VKPH) * es};
    Dual xa, xb, xc;
    grid_coords(g, r, th, ph, &xa, &xb, &xc);
    const Dual ne = ne_index(g, xa, xb, xc, nullptr);
    const Dual X = ne * (PLASMA_HZ2_PER_M3 / (c.f_hz * c.f_hz)) * es * es;
    const Dual kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    Dual mu2;
    if (g.b0_tesla == 0.0) {
        mu2 = 1.0 - X;
    } else {
        Dual B[3];
        dipole(g, r, th, ph, B);
        Dual Y[3];
        for (int i = 0; i < 3; ++i) Y[i] = B[i] * (GYRO_HZ_PER_T / c.f_hz) * es;
        const Dual Y2 = Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2];
        const Dual kY = k[0] * Y[0] + k[1] * Y[1] + k[2] * Y[2];
        const Dual YL2 = kY * kY / kk;
        const Dual YT2 = Y2 - YL2;
        mu2 = ah_mu2(X, YL2, YT2, c.mode);
    }
    return 0.5 * (kk - mu2);
}

/* ------------------------------------------------ ray equations, Eq. 1 -- */
/* With k scaled by omega/c, Eq. 1a-1f read (G = omega dH/domega):
 *   dr/dP'     = -H_kr / G
 *   dtheta/dP' = -H_kth / (r G)
 *   dphi/dP'   = -H_kph / (r sin(theta) G)
 *   dkr/dP'    =  H_r / G + k_th dtheta/dP' + k_ph sin(theta) dphi/dP'
 *   dkth/dP'   = (H_th / G - k_th dr/dP' + k_ph r cos(theta) dphi/dP') / r
 *   dkph/dP'   = (H_ph / G - k_ph sin(theta) dr/dP' - k_ph r cos(theta) dtheta/dP') / (r sin(theta)) */
void rhs(const Ctx &c, const double y[6], double dy[6], double *h_out) {
    const Dual H = hamiltonian(c, y);
    if (h_out) *h_out = H.v;
    const double G = H.d[VS];
    const double r = y[0], st = std::sin(y[1]), ct = std::cos(y[1]);
    const double kth = y[4], kph = y[5];
    dy[0] = -H.d[VKR] / G;
    dy[1] = -H.d[VKTH] / (r * G);
    dy[2] = -H.d[VKPH] / (r * st * G);
    dy[3] = H.d[VR] / G + kth * dy[1] + kph * st * dy[2];
    dy[4] = (H.d[VTH] / G - kth * dy[0] + kph * r * ct * dy[2]) / r;
    dy[5] = (H.d[VPH] / G - kph * st * dy[0] - kph * r * ct * dy[1]) / (r * st);
}

/* ---------------------------------------------------------- integrators -- */
void rk4_step(const Ctx &c, const double y[6], const double k1[6], double h, double yn[6]) {
    double k2[6], k3[6], k4[6], t[6];
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    rhs(c, t, k2, nullptr);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    rhs(c, t, k3, nullptr);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + h * k3[i];
    rhs(c, t, k4, nullptr);
    for (int i = 0; i < 6; ++i) yn[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Runge-Kutta-Fehlberg 4(5) (Fehlberg 1969).  Returns the fourth-order
 * solution in yn and the local error estimate (fifth minus fourth order) in
 * e, formed directly as h * sum((b5_i - b4_i) k_i): the difference of the two
 * solutions would cancel against r ~ 6371 km and keep only a few digits. */
void rkf45_step(const Ctx &c, const double y[6], const double k1[6], double h, double yn[6],
                double e[6]) {
    double k2[6], k3[6], k4[6], k5[6], k6[6], t[6];
    for (int i = 0; i < 6; ++i) t[i] = y[i] + h * (k1[i] / 4.0);
    rhs(c, t, k2, nullptr);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + h * (3.0 / 32.0 * k1[i] + 9.0 / 32.0 * k2[i]);
    rhs(c, t, k3, nullptr);
    for (int i = 0; i < 6; ++i)
        t[i] = y[i] + h * (1932.0 / 2197.0 * k1[i] - 7200.0 / 2197.0 * k2[i] + 7296.0 / 2197.0 * k3[i]);
    rhs(c, t, k4, nullptr);
    for (int i = 0; i < 6; ++i)
        t[i] = y[i] + h * (439.0 / 216.0 * k1[i] - 8.0 * k2[i] + 3680.0 / 513.0 * k3[i] -
                           845.0 / 4104.0 * k4[i]);
    rhs(c, t, k5, nullptr);
    for (int i = 0; i < 6; ++i)
        t[i] = y[i] + h * (-8.0 / 27.0 * k1[i] + 2.0 * k2[i] - 3544.0 / 2565.0 * k3[i] +
                           1859.0 / 4104.0 * k4[i] - 11.0 / 40.0 * k5[i]);
    rhs(c, t, k6, nullptr);
    for (int i = 0; i < 6; ++i) {
        yn[i] = y[i] + h * (25.0 / 216.0 * k1[i] + 1408.0 / 2565.0 * k3[i] +
                            2197.0 / 4104.0 * k4[i] - k5[i] / 5.0);
        e[i] = h * ((16.0 / 135.0 - 25.0 / 216.0) * k1[i] +
                    (6656.0 / 12825.0 - 1408.0 / 2565.0) * k3[i] +
                    (28561.0 / 56430.0 - 2197.0 / 4104.0) * k4[i] +
                    (-9.0 / 50.0 + 1.0 / 5.0) * k5[i] + 2.0 / 55.0 * k6[i]);
    }
}

/* Error norm of an RKF45 step (accepted when <= 1): position error in km,
 * max(|dr|, r|dtheta|, r sin(theta)|dphi|), against atol + rtol*r, and
 * wave-vector error max|dk_i| against rtol*max(|k|, 1e-3). */
double rkf45_err(const double y[6], const double e[6], double rtol, double atol) {
    const double r = y[0], st = std::sin(y[1]);
    const double pos = std::max(std::fabs(e[0]), std::max(r * std::fabs(e[1]), r * st * std::fabs(e[2])));
    const double kmag = std::sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
    const double kerr = std::max(std::fabs(e[3]), std::max(std::fabs(e[4]), std::fabs(e[5])));
    return std::max(pos / (atol + rtol * r), kerr / (rtol * std::max(kmag, 1e-3)));
}

/* Step-size factor: the classical 0.9 err^(-1/5) limited to [0.2, 5], then
 * rounded down to a power of 2^(1/4).  Step sizes thus change only through
 * discrete decisions; a continuous factor lets round-off in err feed back
 * into the step sequence, which then diverges chaotically because the error
 * estimate of a step that crosses a cell face of the C1 interpolant depends
 * sharply on where the face falls inside the step. */
double step_factor(double err) {
    const double fac = (err == 0.0) ? 5.0 : std::min(5.0, std::max(0.2, 0.9 * std::pow(err, -0.2)));
    return std::exp2(std::floor(4.0 * std::log2(fac)) * 0.25);
}

/* Peak of the cubic Hermite fit of r(s), s in [0,1], through (r0, h*d0) and
 * (r1, h*d1) where d0 > 0 >= d1: the zero of p'(s) by bisection. */
double hermite_peak(double r0, double r1, double d0, double d1, double h) {
    const double m0 = h * d0, m1 = h * d1;
    const double A = 2.0 * (r0 - r1) + m0 + m1;
    const double B = 3.0 * (r1 - r0) - 2.0 * m0 - m1;
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double dp = m0 + 2.0 * B * mid + 3.0 * A * mid * mid;
        if (dp > 0.0) lo = mid; else hi = mid;
    }
    const double s = 0.5 * (lo + hi);
    return r0 + m0 * s + B * s * s + A * s * s * s;
}

double wrap180(double x) { return x - 360.0 * std::floor((x + 180.0) / 360.0); }

bool finite6(const double y[6]) {
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(y[i])) return false;
    return true;
}

/* Launch state: transmitter position and direction (elevation above the local
 * horizontal, azimuth clockwise from north; the theta unit vector points
 * south) with |k| = mu at the transmitter for that direction. */
bool launch(const Ctx &c, const or_ray &ray, double y0[6]) {
    const or_grid &g = *c.g;
    const double el = ray.el_deg * DEG, az = ray.az_deg * DEG;
    y0[0] = g.earth_radius_km + ray.tx_alt_km;
    y0[1] = (90.0 - ray.tx_lat_deg) * DEG;
    y0[2] = ray.tx_lon_deg * DEG;
    y0[3] = std::sin(el);
    y0[4] = -std::cos(el) * std::cos(az);
    y0[5] = std::cos(el) * std::sin(az);
    const double mu2 = 1.0 - 2.0 * hamiltonian(c, y0).v; /* H = (1 - mu^2)/2 for |k| = 1 */
    if (!(mu2 > 0.0)) return false;
    const double mu = std::sqrt(mu2);
    for (int i = 3; i < 6; ++i) y0[i] *= mu;
    return true;
}

void unit_vec(double th, double ph, double p[3]) {
    p[0] = std::sin(th) * std::cos(ph);
    p[1] = std::sin(th) * std::sin(ph);
    p[2] = std::cos(th);
}

void finish(const or_grid &g, const or_ray &ray, const double y0[6], const double y[6], double P,
            double apogee, or_result *res) {
    const double lat = 90.0 - y[1] / DEG;
    res->group_path_km = P;
    res->apogee_km = apogee;
    res->land_lat_deg = lat;
    res->land_lon_deg = wrap180(y[2] / DEG);
    double p0[3], p1[3];
    unit_vec(y0[1], y0[2], p0);
    unit_vec(y[1], y[2], p1);
    const double cx = p0[1] * p1[2] - p0[2] * p1[1];
    const double cy = p0[2] * p1[0] - p0[0] * p1[2];
    const double cz = p0[0] * p1[1] - p0[1] * p1[0];
    const double dot = p0[0] * p1[0] + p0[1] * p1[1] + p0[2] * p1[2];
    const double ang = std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz), dot);
    res->ground_range_km = g.earth_radius_km * ang;
    /* bearing of the landing point seen from the transmitter */
    const double north[3] = {-std::cos(y0[1]) * std::cos(y0[2]), -std::cos(y0[1]) * std::sin(y0[2]),
                             std::sin(y0[1])};
    const double east[3] = {-std::sin(y0[2]), std::cos(y0[2]), 0.0};
    const double pn = p1[0] * north[0] + p1[1] * north[1] + p1[2] * north[2];
    const double pe = p1[0] * east[0] + p1[1] * east[1] + p1[2] * east[2];
    res->az_dev_deg = (ang > 1e-15) ? wrap180(std::atan2(pe, pn) / DEG - ray.az_deg) : 0.0;
}

void push_traj(double *traj, int32_t cap, int32_t *len, double P, const double y[6], double H) {
    if (!traj || *len >= cap) return;
    double *row = traj + (size_t)(*len) * 8;
    row[0] = P;
    for (int i = 0; i < 6; ++i) row[1 + i] = y[i];
    row[7] = H;
    ++*len;
}

/* Group path to the next cell face of the interpolant that the ray reaches,
 * predicted linearly from dy/dP' = k1 at y.  Faces are where the C1
 * interpolant's second derivatives jump (the right-hand side is only C0
 * there); the grid's outer faces count too.  Lateral faces count only while
 * the ray is inside the altitude span (below it Ne = 0).  Infinite if none. */
double face_distance(const or_grid &g, const double y[6], const double k1[6]) {
    Dual xa, xb, xc;
    grid_coords(g, cst(y[0]), cst(y[1]), cst(y[2]), &xa, &xb, &xc);
    const double x[3] = {xa.v, xb.v, xc.v};
    const double v[3] = {-k1[1] / DEG / g.dlat_deg, k1[2] / DEG / g.dlon_deg, k1[0] / g.dalt_km};
    const int n[3] = {g.n_lat, g.n_lon, g.n_alt};
    const bool in_alt = x[2] >= 0.0 && x[2] <= g.n_alt - 1;
    double best = HUGE_VAL;
    for (int a = 0; a < 3; ++a) {
        if (a < 2 && !in_alt) continue;
        if (v[a] > 0.0) {
            double F = std::floor(x[a]) + 1.0;
            if (F < 0.0) F = 0.0;
            if (F <= n[a] - 1) best = std::min(best, (F - x[a]) / v[a]);
        } else if (v[a] < 0.0) {
            double F = std::ceil(x[a]) - 1.0;
            if (F > n[a] - 1) F = n[a] - 1;
            if (F >= 0.0) best = std::min(best, (F - x[a]) / v[a]);
        }
    }
    return best;
}

void trace(const or_grid &g, const or_ray &ray, or_result *res, double *traj, int32_t cap,
           int32_t *tlen) {
    *res = or_result{};
    int32_t dummy = 0;
    if (!tlen) tlen = &dummy;
    *tlen = 0;
    const Ctx c{&g, ray.freq_mhz * 1e6, ray.mode};
    const double RE = g.earth_radius_km;
    const double top = g.alt0_km + (g.n_alt - 1) * g.dalt_km;
    double y0[6], y[6];
    if (!launch(c, ray, y0)) {
        for (int i = 0; i < 6; ++i) y[i] = y0[i];
        finish(g, ray, y0, y, 0.0, ray.tx_alt_km, res);
        res->status = OR_NONFINITE;
        return;
    }
    for (int i = 0; i < 6; ++i) y[i] = y0[i];
    const bool adaptive = ray.integrator == 1;
    double P = 0.0, h = ray.h_km, apogee = y[0] - RE;
    int n_steps = 0, n_att = 0, status = OR_RUNNING;
    bool have_prev = false;
    double r_prev = 0.0, dr_prev = 0.0, h_prev = 0.0;
    {
        double k[6], H;
        rhs(c, y, k, &H);
        push_traj(traj, cap, tlen, P, y, H);
    }
    while (status == OR_RUNNING) {
        if (n_att >= ray.max_steps) {
            status = OR_MAX_STEPS;
            break;
        }
        double hs = h;
        double k1[6];
        rhs(c, y, k1, nullptr);
        /* adaptive steps end just past the next cell face instead of straddling it */
        bool at_face = false;
        if (adaptive) {
            const double hf = face_distance(g, y, k1);
            if (hf > 1e-3 * hs && hf < hs) {
                hs = hf * (1.0 + 1e-4);
                at_face = true;
            }
        }
        if (ray.max_group_path_km > 0.0 && P + hs > ray.max_group_path_km) hs = ray.max_group_path_km - P;
        if (have_prev && dr_prev > 0.0 && k1[0] <= 0.0)
            apogee = std::max(apogee, hermite_peak(r_prev, y[0], dr_prev, k1[0], h_prev) - RE);
        have_prev = false;
        double yn[6], e[6];
        if (adaptive) rkf45_step(c, y, k1, hs, yn, e);
        else rk4_step(c, y, k1, hs, yn);
        ++n_att;
        double h_next = h;
        if (adaptive) {
            const double err = rkf45_err(y, e, ray.rtol, ray.atol_km);
            const double fac = step_factor(err);
            /* the nominal step h changes only by quantised factors of itself, never
             * through the length of a face-shortened step, so rounding in where a
             * step ends cannot feed back into later step sizes */
            if (!(err <= 1.0)) {
                h = h * fac;
                if (h < ray.h_min_km) status = OR_STEP_UNDERFLOW;
                continue;
            }
            h_next = std::min(std::max(h * (at_face ? std::min(1.0, fac) : fac), ray.h_min_km), ray.h_max_km);
        }
        if (!finite6(yn)) {
            status = OR_NONFINITE;
            break;
        }
        const bool lands = yn[0] < RE;
        const bool exits = !lands && yn[0] - RE > top;
        if (lands || exits) {
            /* ground return or exit through the grid top inside this step: solve
             * r(step(h*)) = R_E (or R_E + top) for h* in (0, hs]; sg makes the
             * bracket function positive at the start of the step */
            const double rt = lands ? RE : RE + top, sg = lands ? 1.0 : -1.0;
            double a = 0.0, fa = sg * (y[0] - rt), b = hs, fb = sg * (yn[0] - rt), cc = b;
            double yc[6], ec[6];
            for (int i = 0; i < 6; ++i) yc[i] = yn[i];
            int side = 0;
            for (int it = 0; it < 60; ++it) {
                cc = b - fb * (b - a) / (fb - fa);
                if (adaptive) rkf45_step(c, y, k1, cc, yc, ec);
                else rk4_step(c, y, k1, cc, yc);
                ++n_att;
                const double fc = sg * (yc[0] - rt);
                if (std::fabs(fc) < 1e-9) break;
                if (fc < 0.0) {
                    b = cc;
                    fb = fc;
                    if (side == -1) fa *= 0.5;
                    side = -1;
                } else {
                    a = cc;
                    fa = fc;
                    if (side == 1) fb *= 0.5;
                    side = 1;
                }
            }
            P += cc;
            ++n_steps;
            for (int i = 0; i < 6; ++i) y[i] = yc[i];
            if (exits) apogee = std::max(apogee, y[0] - RE);
            double kk[6], H;
            rhs(c, y, kk, &H);
            push_traj(traj, cap, tlen, P, y, H);
            status = lands ? OR_LANDED : OR_ESCAPED;
            break;
        }
        P += hs;
        ++n_steps;
        apogee = std::max(apogee, yn[0] - RE);
        have_prev = true;
        r_prev = y[0];
        dr_prev = k1[0];
        h_prev = hs;
        for (int i = 0; i < 6; ++i) y[i] = yn[i];
        if (traj) {
            double kk[6], H;
            rhs(c, y, kk, &H);
            push_traj(traj, cap, tlen, P, y, H);
        }
        /* leaving the ionospheric region sideways (Sec. II-C) */
        const double alt = y[0] - RE;
        if (alt >= g.alt0_km) {
            Dual xa, xb, xc;
            grid_coords(g, cst(y[0]), cst(y[1]), cst(y[2]), &xa, &xb, &xc);
            if (xa.v < 0.0 || xa.v > g.n_lat - 1 || xb.v < 0.0 || xb.v > g.n_lon - 1) {
                status = OR_LEFT_GRID;
                break;
            }
        }
        if (ray.max_group_path_km > 0.0 && P >= ray.max_group_path_km - 1e-12) {
            status = OR_MAX_PATH;
            break;
        }
        h = h_next;
    }
    finish(g, ray, y0, y, P, apogee, res);
    res->status = status;
    res->n_steps = n_steps;
    res->n_attempts = n_att;
}

} // namespace

extern "C" {

void or_gd_psi(double xi, double *val, double *dval) {
    const Dual p = gd_psi(var(xi, 0));
    *val = p.v;
    *dval = p.d[0];
}

void or_cr_weights(double t, double w[4]) {
    for (int a = 0; a < 4; ++a) w[a] = cr_basis(cst(t - (double)(a - 1))).v;
}

void or_ne(const or_grid *g, double lat_deg, double lon_deg, double alt_km, double out[5]) {
    double lonrel = lon_deg - g->lon0_deg;
    lonrel -= 360.0 * std::floor(lonrel / 360.0);
    const Dual xa = var((lat_deg - g->lat0_deg) / g->dlat_deg, 0);
    const Dual xb = var(lonrel / g->dlon_deg, 1);
    const Dual xc = var((alt_km - g->alt0_km) / g->dalt_km, 2);
    bool inside = false;
    const Dual n = ne_index(*g, xa, xb, xc, &inside);
    out[0] = n.v;
    out[1] = n.d[0] / g->dlat_deg;
    out[2] = n.d[1] / g->dlon_deg;
    out[3] = n.d[2] / g->dalt_km;
    out[4] = inside ? 1.0 : 0.0;
}

void or_ah(double X, double YL2, double YT2, int32_t mode, double out[4]) {
    const Dual m = ah_mu2(var(X, 0), var(YL2, 1), var(YT2, 2), mode);
    out[0] = m.v;
    out[1] = m.d[0];
    out[2] = m.d[1];
    out[3] = m.d[2];
}

void or_dipole(const or_grid *g, double r_km, double theta, double phi, double out[3]) {
    Dual B[3];
    dipole(*g, cst(r_km), cst(theta), cst(phi), B);
    for (int i = 0; i < 3; ++i) out[i] = B[i].v;
}

void or_hamiltonian(const or_grid *g, double freq_mhz, int32_t mode, const double y[6],
                    double out[8]) {
    const Ctx c{g, freq_mhz * 1e6, mode};
    const Dual H = hamiltonian(c, y);
    out[0] = H.v;
    for (int i = 0; i < NV; ++i) out[1 + i] = H.d[i];
}

void or_rhs(const or_grid *g, double freq_mhz, int32_t mode, const double y[6], double dy[6]) {
    const Ctx c{g, freq_mhz * 1e6, mode};
    rhs(c, y, dy, nullptr);
}

int32_t or_launch(const or_grid *g, const or_ray *ray, double y0[6]) {
    const Ctx c{g, ray->freq_mhz * 1e6, ray->mode};
    return launch(c, *ray, y0) ? 1 : 0;
}

void or_trace_ray(const or_grid *g, const or_ray *ray, or_result *res, double *traj,
                  int32_t traj_cap, int32_t *traj_len) {
    trace(*g, *ray, res, traj, traj_cap, traj_len);
}

void or_trace_many(const or_grid *g, const or_ray *rays, int32_t n, or_result *res,
                   int32_t n_threads) {
    if (n_threads <= 0) n_threads = (int32_t)std::max(1u, std::thread::hardware_concurrency());
    n_threads = std::max(1, std::min(n_threads, n));
    std::vector<std::thread> pool;
    for (int t = 0; t < n_threads; ++t)
        pool.emplace_back([=]() {
            for (int i = t; i < n; i += n_threads) trace(*g, rays[i], &res[i], nullptr, 0, nullptr);
        });
    for (auto &th : pool) th.join();
}

} // extern "C"
