"""Host-side helpers of bench.py (no GPU): the one-ray fan used for the
critical-path measurement must be the canonical ray it names, the boundary
filter must flag both neighbours of a jump, and the Richardson extrapolation
must recover a known limit and order."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2506_18579_gb300 import workloads as wl  # noqa: E402


def test_one_ray_spec_is_the_canonical_ray():
    spec = wl.config2(elev_step=3.0, az_step=30.0).fan
    rng = np.random.default_rng(3)
    for i in list(rng.integers(0, spec.n_rays, 200)) + [0, spec.n_rays - 1]:
        one = bench.one_ray_spec(wl, spec, int(i))
        assert one.n_rays == 1
        f, m, el, az = spec.ray_params(int(i))
        assert one.freq_mhz[0] == f and one.el_deg[0] == el and one.az_deg[0] == az
        assert one.mode_list == [m]


def test_near_boundary_flags_both_neighbours_of_a_jump():
    spec = wl.FanSpec(30.0, 112.0, 0.0, freq_mhz=[10.0], el_deg=np.arange(5.0, 10.01, 0.5), az_deg=[0.0, 90.0])
    n_el, n_az = len(spec.el_deg), 2
    res = np.zeros(spec.n_rays, dtype=[("status", "i4"), ("ground_range_km", "f8"), ("group_path_km", "f8")])
    res["status"] = 1
    r = res.reshape(n_el, n_az)
    r["ground_range_km"][:, 0] = 1000.0 - 10.0 * np.arange(n_el)  # smooth
    r["ground_range_km"][:, 1] = 1000.0 - 10.0 * np.arange(n_el)
    r["ground_range_km"][6:, 1] += 200.0  # a jump between elevations 5 and 6 at azimuth 90
    r["group_path_km"] = r["ground_range_km"]
    flag = bench.near_boundary(res, spec).reshape(n_el, n_az)
    assert not flag[:, 0].any()
    assert flag[5, 1] and flag[6, 1] and flag[:, 1].sum() == 2


def test_richardson_extrapolation_recovers_the_limit_and_the_order():
    """y(h) = y* + c h^p: three steps h, h/2, h/4 give back p and y* (to
    rounding), for the fourth order and for the order ~2 that fixed-step RK4
    shows where the field's gradient is only continuous."""
    rng = np.random.default_rng(3)
    y_star = rng.uniform(100.0, 3000.0, 50)
    c = rng.uniform(0.5, 2.0, 50)
    for p_true in (4.0, 2.25):
        ys = [y_star + c * h ** p_true for h in (1.0, 0.5, 0.25)]
        ref, p = bench.richardson_extrapolate(*ys)
        assert abs(p - p_true) < 1e-9
        assert np.max(np.abs(ref - y_star)) < 1e-9 * np.max(y_star)
    # differences below the floor are rounding: left out, order 4 by default
    flat = [np.full(5, 7.0)] * 3
    ref, p = bench.richardson_extrapolate(*flat)
    assert p == 4.0 and np.all(ref == 7.0)
