"""Whole-ray pins of the oracle tracer.

Paper: Eq. 1a-1f (ray equations), Sec. II-C (RK4, termination, outputs:
group path, ground distance, azimuth deviation, reflection height).  Checks:
straight rays in free space (group path = chord length), the closed-form ray
in a flat-Earth linear layer (Breit-Tuve), the Bouguer invariant in a
spherically symmetric medium, H = 0 along rays, fourth-order step convergence
of RK4, and the termination statuses.
"""
import numpy as np
import pytest

from paper_2506_18579_gb300 import workloads as wl

RE = wl.EARTH_RADIUS_KM


def _empty_grid(**kw):
    spec = wl.GridSpec(n_lat=21, n_lon=21, n_alt=61, lat0_deg=10.0, lon0_deg=92.0, alt0_km=60.0,
                       dlat_deg=2.0, dlon_deg=2.0, dalt_km=10.0, **kw)
    return spec, np.zeros(spec.shape)


def _fan(**kw):
    base = dict(tx_lat_deg=30.0, tx_lon_deg=112.0, tx_alt_km=0.0, freq_mhz=[10.0], el_deg=[20.0],
                az_deg=[90.0], modes=wl.MODE_O, integrator=wl.RK4, h_km=1.0, max_steps=20000)
    base.update(kw)
    return wl.FanSpec(**base)


def _cart(traj):
    r, th, ph = traj[:, 1], traj[:, 2], traj[:, 3]
    p = np.stack([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)], 1)
    er = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    et = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1)
    ep = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], 1)
    k = traj[:, 4:5] * er + traj[:, 5:6] * et + traj[:, 6:7] * ep
    return p, k


@pytest.mark.parametrize("el,az", [(20.0, 90.0), (5.0, 37.0), (60.0, 250.0)])
def test_free_space_ray_is_straight(orc, el, az):
    """Ne = 0, no field: the ray is a straight line with constant k, P' is
    the chord length from the launch point, Delta-az is zero.  An eastward ray
    off the equator also fails without the sin(theta) in the k_r equation."""
    spec, ne = _empty_grid()
    g = orc.Grid(spec, ne)
    fan = _fan(el_deg=[el], az_deg=[az])
    ray = orc.fan_rays(fan)[0]
    res, traj = orc.trajectory(g, ray)
    assert res["status"] == orc.ESCAPED
    p, k = _cart(traj)
    d = p - p[0]
    u = k[0] / np.linalg.norm(k[0])
    assert np.max(np.linalg.norm(d - np.outer(d @ u, u), axis=1)) < 1e-8  # collinear
    assert np.max(np.abs(k - k[0])) < 1e-12                                 # constant k
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), traj[:, 0], rtol=1e-12, atol=1e-8)
    r = traj[-1, 1]
    assert r == pytest.approx(RE + 660.0, abs=1e-9)  # exit point solved on the grid top
    e = np.radians(el)
    L = np.sqrt(r * r - RE * RE * np.cos(e) ** 2) - RE * np.sin(e)
    assert res["group_path_km"] == pytest.approx(L, abs=1e-8)
    gamma = np.arcsin(L * np.cos(e) / r)
    assert res["ground_range_km"] == pytest.approx(RE * gamma, abs=1e-7)
    assert abs(res["az_dev_deg"]) < 1e-9


def test_flat_earth_linear_layer_closed_form(orc):
    """Earth radius 1e6 x 6371 km (flat to within metres over the path),
    isotropic linear layer X = (z - z0)/L above z0: D = 2 z0 tan i + 2 L sin 2i,
    P' = 2 z0 / cos i + 4 L cos i (= D / sin i, Breit-Tuve), apex z0 + L cos^2 i,
    with i = 90 deg - elevation.  The interpolant reproduces the linear
    profile exactly, so this runs the full grid path."""
    big = RE * 1e6
    z0, L, f = 100.0, 200.0, 10.0
    deg_per_km = 180.0 / (np.pi * big)
    spec = wl.GridSpec(n_lat=9, n_lon=9, n_alt=21, lat0_deg=-4 * 800 * deg_per_km,
                       lon0_deg=-4 * 800 * deg_per_km, alt0_km=z0, dlat_deg=800 * deg_per_km,
                       dlon_deg=800 * deg_per_km, dalt_km=20.0, earth_radius_km=big)
    _, _, alt = spec.axes()
    ne = np.broadcast_to((alt - z0) / L * (f * 1e6) ** 2 / 80.6, spec.shape).copy()
    g = orc.Grid(spec, ne)
    for el in (20.0, 35.0, 50.0, 65.0):
        fan = _fan(tx_lat_deg=0.0, tx_lon_deg=0.0, el_deg=[el], az_deg=[0.0], integrator=wl.RKF45,
                   rtol=1e-10, atol_km=1e-9, h_km=1.0, h_max_km=20.0, h_min_km=1e-9,
                   max_steps=200000)
        res = orc.trace_fan(g, fan)[0]
        i = np.radians(90.0 - el)
        D = 2 * z0 * np.tan(i) + 2 * L * np.sin(2 * i)
        P = 2 * z0 / np.cos(i) + 4 * L * np.cos(i)
        assert res["status"] == orc.LANDED
        assert res["ground_range_km"] == pytest.approx(D, abs=5e-5)
        assert res["group_path_km"] == pytest.approx(P, abs=5e-5)
        assert res["apogee_km"] == pytest.approx(z0 + L * np.cos(i) ** 2, abs=5e-5)
        assert abs(res["az_dev_deg"]) < 1e-6


def _chapman_sym():
    w = wl.config1()
    return w.grid, w.ne


def test_bouguer_invariant_spherical_symmetry(orc):
    """In a spherically symmetric isotropic medium r mu sin(psi) =
    r sqrt(k_th^2 + k_ph^2) is conserved along the ray and the ray stays in
    its great-circle plane (Delta-az = 0)."""
    spec, ne = _chapman_sym()
    g = orc.Grid(spec, ne)
    for el, az in ((10.0, 30.0), (35.0, 100.0), (48.0, 200.0)):
        fan = _fan(el_deg=[el], az_deg=[az], integrator=wl.RKF45, rtol=1e-10, atol_km=1e-8,
                   h_max_km=5.0)
        res, traj = orc.trajectory(g, orc.fan_rays(fan)[0])
        assert res["status"] == orc.LANDED
        inv = traj[:, 1] * np.hypot(traj[:, 5], traj[:, 6])
        assert np.max(np.abs(inv / inv[0] - 1)) < 1e-8
        assert inv[0] == pytest.approx(RE * np.cos(np.radians(el)), rel=1e-14)
        assert abs(res["az_dev_deg"]) < 1e-7


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_hamiltonian_stays_zero(orc, cfg):
    if cfg == "c1":
        w = wl.config1()
        idx = [0, 7, 15]
        tol = 1e-6  # fixed-step RK4, h = 1 km
    else:
        w = wl.config2(elev_step=7.0, az_step=60.0)
        idx = [3, 40, 77, 101, 150]
        tol = 1e-5  # RKF45: per-step wave-vector tolerance 1e-8, a few hundred steps
    g = orc.Grid(w.grid, w.ne)
    rays = orc.fan_rays(w.fan, idx)
    for ray in rays:
        res, traj = orc.trajectory(g, ray)
        assert res["status"] in (orc.LANDED, orc.ESCAPED)
        # an escaped ray ends one step above the grid top, where Ne = 0 (free
        # space outside the grid box), so its last point is off the surface
        rows = traj if res["status"] == orc.LANDED else traj[:-1]
        assert np.max(np.abs(rows[:, 7])) < tol
        # the landing solve puts the end point on the ground
        if res["status"] == orc.LANDED:
            assert abs(traj[-1, 1] - w.grid.earth_radius_km) < 1e-9
            assert res["apogee_km"] >= np.max(traj[:, 1] - w.grid.earth_radius_km) - 1e-12


def test_rk4_fourth_order_convergence(orc):
    """A density quadratic in altitude and linear in latitude is reproduced
    exactly by the interpolant (smooth RHS), so RK4 errors at fixed group path
    shrink by 2^4 per halving of h."""
    spec = wl.GridSpec(n_lat=21, n_lon=21, n_alt=61, lat0_deg=10.0, lon0_deg=92.0, alt0_km=60.0,
                       dlat_deg=2.0, dlon_deg=2.0, dalt_km=10.0)
    lat, lon, alt = spec.axes()
    LAT, _, ALT = np.meshgrid(lat, lon, alt, indexing="ij")
    X = 0.05 + 0.6 * ((ALT - 60) / 400) ** 2 * (1 + 0.01 * (LAT - 30))
    ne = X * (10e6) ** 2 / 80.6
    g = orc.Grid(spec, ne)
    outs = []
    for h in (16.0, 8.0, 4.0, 2.0):
        fan = _fan(tx_alt_km=120.0, el_deg=[30.0], az_deg=[20.0], h_km=h, max_group_path_km=400.0)
        res, traj = orc.trajectory(g, orc.fan_rays(fan)[0])
        assert res["status"] == orc.MAX_PATH
        assert traj[-1, 0] == pytest.approx(400.0, abs=1e-9)
        outs.append(traj[-1, 1:7])
    outs = np.array(outs)
    scale = np.array([1.0, RE, RE, 1.0, 1.0, 1.0])
    d = np.abs(np.diff(outs, axis=0)) * scale
    ratio = d[:-1].max(axis=1) / d[1:].max(axis=1)
    assert np.all(ratio > 14.0) and np.all(ratio < 18.5), ratio


def test_rkf45_agrees_with_fine_rk4(orc):
    spec, ne = _chapman_sym()
    g = orc.Grid(spec, ne)
    a = orc.trace_fan(g, _fan(el_deg=[12.0, 40.0], integrator=wl.RKF45, rtol=1e-10, atol_km=1e-8))
    b = orc.trace_fan(g, _fan(el_deg=[12.0, 40.0], h_km=0.125))
    np.testing.assert_allclose(a["group_path_km"], b["group_path_km"], atol=5e-4)
    np.testing.assert_allclose(a["ground_range_km"], b["ground_range_km"], atol=5e-4)


def test_statuses(orc):
    spec, ne = _chapman_sym()
    g = orc.Grid(spec, ne)
    # above the critical frequency at steep elevation: escapes through the top
    assert orc.trace_fan(g, _fan(freq_mhz=[30.0], el_deg=[70.0]))[0]["status"] == orc.ESCAPED
    # a step budget that is too small
    r = orc.trace_fan(g, _fan(max_steps=10))[0]
    assert r["status"] == orc.MAX_STEPS and r["n_attempts"] == 10
    # a narrow grid: the ray leaves it sideways inside the altitude span
    narrow = wl.GridSpec(**{**spec.__dict__, "n_lat": 5, "n_lon": 5, "lat0_deg": 26.0,
                            "lon0_deg": 108.0})
    gn = orc.Grid(narrow, ne[8:13, 8:13, :])
    assert orc.trace_fan(gn, _fan(el_deg=[10.0]))[0]["status"] == orc.LEFT_GRID
    # non-finite density stops the ray with a status, not a hang
    bad = ne.copy()
    bad[:, :, 10:] = np.nan
    assert orc.trace_fan(orc.Grid(spec, bad), _fan())[0]["status"] == orc.NONFINITE
    # a step-size floor above what the tolerance needs
    r = orc.trace_fan(g, _fan(integrator=wl.RKF45, rtol=1e-14, atol_km=1e-14, h_min_km=0.5))[0]
    assert r["status"] == orc.STEP_UNDERFLOW


def test_rkf45_step_sequence_is_well_conditioned(orc):
    """With the step factor quantised to powers of 2^(1/4), perturbing the
    launch elevations by 1 part in 1e13 leaves every step sequence unchanged
    and moves group paths by round-off only (a continuous factor makes the
    sequence chaotic at C1 cell faces: km-level changes)."""
    w = wl.config2(elev_step=12.0, az_step=90.0)
    g = orc.Grid(w.grid, w.ne)
    a = orc.trace_fan(g, w.fan)
    b = orc.trace_fan(g, w.fan.replace(el_deg=w.fan.el_deg * (1 + 1e-13)))
    assert np.array_equal(a["n_attempts"], b["n_attempts"])
    assert np.abs(a["group_path_km"] - b["group_path_km"]).max() < 1e-7


def test_rkf45_converges_with_rtol(orc):
    """Face-aligned RKF45: the group-path error against a tight run shrinks
    roughly in proportion to rtol."""
    w = wl.config2(elev_step=9.0, az_step=90.0, freqs=(8.0, 12.0))
    g = orc.Grid(w.grid, w.ne)
    ref = orc.trace_fan(g, w.fan.replace(rtol=1e-12, atol_km=1e-10))
    errs = []
    for rtol in (1e-8, 1e-10):
        a = orc.trace_fan(g, w.fan.replace(rtol=rtol))
        ok = a["status"] == ref["status"]
        errs.append(np.quantile(np.abs(a["group_path_km"] - ref["group_path_km"])[ok], 0.9))
    assert errs[1] < errs[0] / 20.0, errs
    assert errs[1] < 2e-3, errs


def test_ionogram_points_hand_computed(orc):
    """The ionogram reduction on hand-made records: crossings of the receiver
    distance between neighbouring landed elevations, P' and elevation linear
    in D, branches counted per (frequency, mode), no crossing across a ray
    that did not land."""
    fan = wl.FanSpec(tx_lat_deg=0.0, tx_lon_deg=0.0, tx_alt_km=0.0, freq_mhz=[5.0, 7.0],
                     el_deg=[10.0, 20.0, 30.0, 40.0], az_deg=[45.0], modes=wl.MODE_O | wl.MODE_X)
    res = np.zeros(fan.n_rays, dtype=orc.RESULT_DTYPE).reshape(2, 2, 4)
    res["status"] = orc.LANDED
    res["ground_range_km"] = 900.0  # frequency 7 MHz: never reaches 1,500 km
    # 5 MHz, O: D rises through 1,500 km and falls back through it
    res[0, 0]["ground_range_km"] = [1000.0, 1400.0, 1600.0, 1200.0]
    res[0, 0]["group_path_km"] = [1100.0, 1500.0, 1700.0, 1300.0]
    # 5 MHz, X: the second elevation escapes, so only the last pair counts
    res[0, 1]["ground_range_km"] = [1000.0, 1600.0, 1700.0, 1300.0]
    res[0, 1]["group_path_km"] = [1000.0, 1700.0, 1800.0, 1400.0]
    res[0, 1, 1]["status"] = orc.ESCAPED
    pts = orc.ionogram_points(res.reshape(-1), fan, 1500.0)
    want = [(5.0, 1600.0, 25.0, 1, 0), (5.0, 1600.0, 32.5, 1, 1), (5.0, 1600.0, 35.0, -1, 0)]
    assert len(pts) == len(want)
    for p, q in zip(pts, want):
        assert p[0] == q[0] and p[3] == q[3] and p[4] == q[4]
        assert abs(p[1] - q[1]) < 1e-9 and abs(p[2] - q[2]) < 1e-12
