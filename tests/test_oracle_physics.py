"""Pins of the oracle's refractive index, field and Hamiltonian partials.

Paper: Eq. 2 (Hamiltonian), Eq. 3 (Appleton-Hartree without collisions, upper
sign ordinary), Sec. II-C (geomagnetic field; a centred dipole stands in for
IGRF).  Checks: textbook special cases of Eq. 3, dual-number partials against
finite differences of the oracle's own values, dipole values fixed by
magnetostatics, and the magnetoionic ray direction / group index.
"""
import numpy as np
import pytest

from paper_2506_18579_gb300 import workloads as wl


@pytest.mark.parametrize("X", [0.0, 0.3, 0.7, 0.95])
def test_ah_no_field(orc, X):
    for mode in (1, -1):
        assert orc.ah(X, 0.0, 0.0, mode)[0] == pytest.approx(1.0 - X, abs=1e-15)


@pytest.mark.parametrize("YL2,YT2", [(0.01, 0.02), (0.04, 0.0001), (1e-4, 0.09), (0.2, 0.3)])
def test_ah_reflection_points(orc, YL2, YT2):
    # ordinary wave: mu^2 -> 0 as X -> 1 for every propagation angle (Eq. 3 as
    # printed is 0/0 at X = 1 exactly; the oracle keeps the printed form)
    # (the printed form loses relative accuracy in mu^2 as X -> 1: 1 - N/D with N/D -> 1)
    m5, m7 = orc.ah(1.0 - 1e-5, YL2, YT2, 1)[0], orc.ah(1.0 - 1e-7, YL2, YT2, 1)[0]
    assert m5 > 0 and m7 > 0
    assert m5 / m7 == pytest.approx(100.0, rel=1e-2)  # vanishes linearly in 1 - X
    # extraordinary wave: mu^2 = 0 at X = 1 - Y
    Y = np.sqrt(YL2 + YT2)
    assert orc.ah(1.0 - Y, YL2, YT2, -1)[0] == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("X", [0.1, 0.5, 0.8])
def test_ah_longitudinal_and_transverse_limits(orc, X):
    YL = 0.3
    # quasi-longitudinal limit (Y_T = 0): mu^2 = 1 - X / (1 +/- |Y_L|)
    assert orc.ah(X, YL * YL, 0.0, 1)[0] == pytest.approx(1 - X / (1 + YL), rel=1e-13)
    assert orc.ah(X, YL * YL, 0.0, -1)[0] == pytest.approx(1 - X / (1 - YL), rel=1e-13)
    # transverse propagation (Y_L = 0): ordinary 1 - X, extraordinary 1 - X(1-X)/(1-X-Y^2)
    YT2 = 0.09
    assert orc.ah(X, 0.0, YT2, 1)[0] == pytest.approx(1 - X, rel=1e-13)
    assert orc.ah(X, 0.0, YT2, -1)[0] == pytest.approx(1 - X * (1 - X) / (1 - X - YT2), rel=1e-12)


def test_ah_partials_vs_finite_differences(orc):
    rng = np.random.default_rng(5)
    for _ in range(40):
        X, YL2, YT2 = rng.uniform(0.05, 0.9), rng.uniform(0.001, 0.1), rng.uniform(0.001, 0.1)
        for mode in (1, -1):
            out = orc.ah(X, YL2, YT2, mode)
            if mode == -1 and abs(1 - X - np.sqrt(YL2 + YT2)) < 0.05:
                continue
            for i, base in enumerate((X, YL2, YT2)):
                e = 1e-6 * max(abs(base), 1e-3)
                args_p = [X, YL2, YT2]
                args_m = [X, YL2, YT2]
                args_p[i] += e
                args_m[i] -= e
                fd = (orc.ah(*args_p, mode)[0] - orc.ah(*args_m, mode)[0]) / (2 * e)
                assert out[1 + i] == pytest.approx(fd, rel=2e-5, abs=1e-8)


def _dipole_grid(b0=3.1e-5, pole_lat=79.0, pole_lon=-68.0):
    spec = wl.GridSpec(n_lat=4, n_lon=4, n_alt=4, lat0_deg=0.0, lon0_deg=0.0, alt0_km=100.0,
                       dlat_deg=1.0, dlon_deg=1.0, dalt_km=10.0, b0_tesla=b0,
                       pole_lat_deg=pole_lat, pole_lon_deg=pole_lon)
    return spec, np.zeros(spec.shape)


def test_dipole_magnetostatics(orc):
    spec, ne = _dipole_grid(pole_lat=90.0, pole_lon=0.0)
    g = orc.Grid(spec, ne)
    RE = spec.earth_radius_km
    # magnetic equator at the surface: |B| = B0, horizontal, pointing north (-theta)
    B = orc.dipole(g, RE, np.pi / 2, 0.3)
    np.testing.assert_allclose(B, [0.0, -3.1e-5, 0.0], atol=1e-18)
    # magnetic north pole: |B| = 2 B0, pointing down
    B = orc.dipole(g, RE, 0.0, 0.0)
    np.testing.assert_allclose(B, [-6.2e-5, 0.0, 0.0], atol=1e-18)
    # |B| ~ r^-3 and |B| = B0 sqrt(1 + 3 cos^2 theta_m)
    for th in (0.3, 1.0, 2.0):
        B1 = np.linalg.norm(orc.dipole(g, RE, th, 1.0))
        B2 = np.linalg.norm(orc.dipole(g, 2 * RE, th, 1.0))
        assert B1 == pytest.approx(3.1e-5 * np.sqrt(1 + 3 * np.cos(th) ** 2), rel=1e-13)
        assert B2 == pytest.approx(B1 / 8, rel=1e-13)
    # tilted pole: the field points straight down at the pole position
    spec, ne = _dipole_grid()
    g = orc.Grid(spec, ne)
    B = orc.dipole(g, RE, np.radians(11.0), np.radians(-68.0))
    np.testing.assert_allclose(B, [-6.2e-5, 0, 0], atol=1e-17)


def _chapman_dipole_grid():
    w = wl.config2(elev_step=10.0, az_step=90.0, freqs=(12.0,))
    return w


def test_hamiltonian_partials_vs_finite_differences(orc):
    w = _chapman_dipole_grid()
    g = orc.Grid(w.grid, w.ne)
    RE = w.grid.earth_radius_km
    rng = np.random.default_rng(9)
    for _ in range(12):
        y = np.array([RE + rng.uniform(150, 320), np.radians(90 - rng.uniform(20, 40)),
                      np.radians(rng.uniform(100, 125)), *rng.normal(size=3) * 0.5])
        f = 12.0
        for mode in (1, -1):
            out = orc.hamiltonian(g, f, mode, y)
            steps = [1e-4, 1e-7, 1e-7, 1e-6, 1e-6, 1e-6]
            for i in range(6):
                yp, ym = y.copy(), y.copy()
                yp[i] += steps[i]
                ym[i] -= steps[i]
                fd = (orc.hamiltonian(g, f, mode, yp)[0] - orc.hamiltonian(g, f, mode, ym)[0]) / (2 * steps[i])
                assert out[1 + i] == pytest.approx(fd, rel=1e-5, abs=1e-9), (i, mode)
            # omega dH/domega at fixed physical k: k/omega scales as 1/f
            e = 1e-6
            hp = orc.hamiltonian(g, f * (1 + e), mode, np.r_[y[:3], y[3:] / (1 + e)])[0]
            hm = orc.hamiltonian(g, f * (1 - e), mode, np.r_[y[:3], y[3:] / (1 - e)])[0]
            assert out[7] == pytest.approx((hp - hm) / (2 * e), rel=1e-5, abs=1e-9)


def test_isotropic_rhs_is_k(orc):
    """No field: dx/dP' = k (|dx/dP'| = mu, Sec. II-A) and dk/dP' = grad(X)/2."""
    w = wl.config1()
    g = orc.Grid(w.grid, w.ne)
    RE = w.grid.earth_radius_km
    y = np.array([RE + 250.0, np.radians(60.0), np.radians(112.0), 0.3, -0.5, 0.2])
    r, th = y[0], y[1]
    ne = orc.ne(g, 90 - np.degrees(th), np.degrees(y[2]), r - RE)
    X = 80.6 * ne[0] / (10e6) ** 2
    dXdr = 80.6 * ne[3] / (10e6) ** 2
    y[3:] *= np.sqrt(1 - X) / np.linalg.norm(y[3:])  # on the dispersion surface H = 0
    d = orc.rhs(g, 10.0, 1, y)
    assert d[0] == pytest.approx(y[3], rel=1e-12)
    assert r * d[1] == pytest.approx(y[4], rel=1e-12)
    assert r * np.sin(th) * d[2] == pytest.approx(y[5], rel=1e-12)
    # radial wave-vector equation: dk_r/dP' = -dX/dr / 2 + (k_th^2 + k_ph^2)/r
    assert d[3] == pytest.approx(-0.5 * dXdr + (y[4] ** 2 + y[5] ** 2) / r, rel=1e-10)


def test_magnetoionic_ray_direction_and_group_index(orc):
    """In a magnetised plasma the ray leaves the wave normal at the angle
    tan(alpha) = -(1/mu) dmu/dTheta and its group path grows as
    dP'/ds = mu' cos(alpha) with mu' = d(f mu)/df (Budden, Radio Waves in the
    Ionosphere, Sec. 5.9 and 13.2).  Checked at points of a uniform-Ne grid."""
    spec, _ = _dipole_grid()
    spec = wl.GridSpec(**{**spec.__dict__, "lat0_deg": 25.0, "lon0_deg": 105.0, "dlat_deg": 5.0,
                          "dlon_deg": 5.0, "alt0_km": 100.0, "dalt_km": 100.0})
    for X0 in (0.3, 0.6):
        f = 8.0
        ne = np.full(spec.shape, X0 * (f * 1e6) ** 2 / 80.6)
        g = orc.Grid(spec, ne)
        RE = spec.earth_radius_km
        pos = np.array([RE + 230.0, np.radians(90 - 31.0), np.radians(112.0)])
        Bs = orc.dipole(g, *pos)
        b = Bs / np.linalg.norm(Bs)
        rng = np.random.default_rng(int(X0 * 10))
        for _ in range(4):
            kh = rng.normal(size=3)
            kh /= np.linalg.norm(kh)
            e_perp = b - (b @ kh) * kh
            e_perp /= np.linalg.norm(e_perp)
            for mode in (1, -1):
                def mu(k_dir, freq=f):
                    return np.sqrt(1 - 2 * orc.hamiltonian(g, freq, mode, np.r_[pos, k_dir])[0])
                m0 = mu(kh)
                if not np.isfinite(m0) or m0 < 0.2:
                    continue
                d = 1e-5
                dmu_ddelta = (mu(np.cos(d) * kh + np.sin(d) * e_perp) -
                              mu(np.cos(-d) * kh + np.sin(-d) * e_perp)) / (2 * d)
                ef = 1e-6
                mu_group = m0 + f * (mu(kh, f * (1 + ef)) - mu(kh, f * (1 - ef))) / (2 * f * ef)
                dy = orc.rhs(g, f, mode, np.r_[pos, m0 * kh])
                v = np.array([dy[0], pos[0] * dy[1], pos[0] * np.sin(pos[1]) * dy[2]])
                assert v @ kh == pytest.approx(1.0 / mu_group, rel=1e-6)
                assert (v @ e_perp) / (v @ kh) == pytest.approx(-dmu_ddelta / m0, rel=1e-5, abs=1e-9)
                # the ray stays in the plane of k and B
                n = np.cross(kh, e_perp)
                assert abs(v @ n) < 1e-9
