/*
 * rtgd_oracle.h -- C interface of the plain FP64 CPU reference tracer.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists so that the tests, the smoke
 * check and the CPU-baseline leg of the benchmark can compare the CUDA path
 * against an obviously-correct restatement of the RTM-GD method.  The product
 * path (the CUDA library and its Python binding) never includes, links or
 * calls anything declared here, and this file includes nothing from it.
 *
 * Everything is double precision.  Units: km, degrees at the interface,
 * radians inside, frequency in MHz, electron density in m^-3, field in tesla.
 */
#ifndef RTGD_ORACLE_H
#define RTGD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Uniform lat/lon/alt grid of Ne samples, layout [lat][lon][alt] (alt fastest). */
typedef struct or_grid {
    int32_t n_lat, n_lon, n_alt;
    int32_t interp;           /* 0: Galerkin-Difference p=3, 1: Catmull-Rom */
    double lat0_deg, lon0_deg, alt0_km;
    double dlat_deg, dlon_deg, dalt_km;
    double earth_radius_km;
    double b0_tesla;          /* 0 => isotropic medium (no field) */
    double pole_lat_deg, pole_lon_deg;
    const double *ne;         /* n_lat*n_lon*n_alt samples, caller-owned */
} or_grid;

/* One ray.  mode: +1 ordinary, -1 extraordinary.  integrator: 0 RK4, 1 RKF45. */
typedef struct or_ray {
    double tx_lat_deg, tx_lon_deg, tx_alt_km;
    double freq_mhz, el_deg, az_deg;
    int32_t mode, integrator;
    double h_km, rtol, atol_km, h_min_km, h_max_km;
    int32_t max_steps, pad0;
    double max_group_path_km;  /* <= 0: no limit */
} or_ray;

/* Per-ray result; status codes below. */
typedef struct or_result {
    double group_path_km, ground_range_km, az_dev_deg, apogee_km;
    double land_lat_deg, land_lon_deg;
    int32_t status, n_steps, n_attempts, pad0;
} or_result;

enum {
    OR_RUNNING = 0, OR_LANDED = 1, OR_ESCAPED = 2, OR_LEFT_GRID = 3,
    OR_MAX_STEPS = 4, OR_STEP_UNDERFLOW = 5, OR_NONFINITE = 6, OR_MAX_PATH = 7
};

/* 1-D global GD basis function (p=3) at offset xi from its node: value and d/dxi. */
void or_gd_psi(double xi, double *val, double *dval);

/* Catmull-Rom 1-D weights at t in [0,1] for nodes j-1..j+2 (comparison interpolant). */
void or_cr_weights(double t, double w[4]);

/* GD interpolant at a geographic point.  out = {Ne, dNe/dlat_deg, dNe/dlon_deg,
 * dNe/dalt_km, inside}.  Outside the grid box Ne and its gradient are 0. */
void or_ne(const or_grid *g, double lat_deg, double lon_deg, double alt_km, double out[5]);

/* Appleton-Hartree mu^2 (no collisions) and its partials with respect to
 * (X, Y_L^2, Y_T^2): out = {mu2, d/dX, d/dYL2, d/dYT2}. */
void or_ah(double X, double YL2, double YT2, int32_t mode, double out[4]);

/* Dipole flux density, spherical components (B_r, B_theta, B_phi) in tesla. */
void or_dipole(const or_grid *g, double r_km, double theta, double phi, double out[3]);

/* Hamiltonian at state y = (r, theta, phi, kr, ktheta, kphi) (k in units of
 * omega/c): out = {H, dH/dr, dH/dtheta, dH/dphi, dH/dkr, dH/dkth, dH/dkph,
 * omega dH/domega}. */
void or_hamiltonian(const or_grid *g, double freq_mhz, int32_t mode,
                    const double y[6], double out[8]);

/* Right-hand side dy/dP' of the ray equations. */
void or_rhs(const or_grid *g, double freq_mhz, int32_t mode, const double y[6], double dy[6]);

/* Launch state of a ray: y0[6]; returns 0 if mu^2 <= 0 at the transmitter. */
int32_t or_launch(const or_grid *g, const or_ray *ray, double y0[6]);

/* Trace one ray.  If traj != NULL, each accepted state (P', y[6], H) -- 8
 * doubles -- is appended (the launch state first) up to traj_cap rows; the
 * number of rows written is stored in *traj_len. */
void or_trace_ray(const or_grid *g, const or_ray *ray, or_result *res,
                  double *traj, int32_t traj_cap, int32_t *traj_len);

/* Trace n rays on n_threads host threads (static cyclic split). */
void or_trace_many(const or_grid *g, const or_ray *rays, int32_t n, or_result *res,
                   int32_t n_threads);

#ifdef __cplusplus
}
#endif
#endif
