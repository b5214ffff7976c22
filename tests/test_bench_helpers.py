"""Host-side helpers of bench.py (no GPU): the one-ray fan used for the
critical-path measurement must be the canonical ray it names, the accuracy
block must count statuses, shares within the bar and the compared rays as
stated, and the Richardson extrapolation must recover a known limit and
order."""
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


def test_gate_errors_counts_statuses_shares_and_the_rays_it_compares():
    """The accuracy block: statuses over all rays, errors and shares within
    the bar over the well-conditioned rays whose statuses agree."""
    dt = np.dtype([(f, "f8") for f in bench.ERROR_FIELDS] + [("status", "i4")])
    ref = np.zeros(10, dt)
    ref["status"] = 1
    r = ref.copy()
    r["group_path_km"] = [0.0, 0.01, 0.04, 0.06, 0.2, 0.0, 0.0, 0.0, 9.0, 5.0]
    r["az_dev_deg"] = [0.0, 2e-4, 0, 0, 0, 0, 0, 0, 0, 0]
    r["status"][9] = 2  # another status: counted, not compared
    well = np.ones(10, bool)
    well[8] = False  # near a boundary: not compared
    e = bench.gate_errors(r, ref, well)
    assert e["status_mismatch"] == 1 and e["rays_compared"] == 8
    assert e["group_path_km"]["max"] == 0.2
    assert e["group_path_km"]["within_bar"] == 6 / 8
    assert e["p_and_d_beyond_bar_rays"] == 2
    assert e["az_dev_deg"]["within_bar"] == 7 / 8
    idx = np.array([0, 4, 9])  # the same with an index into the records
    e2 = bench.gate_errors(r, ref[idx], np.ones(3, bool), idx)
    assert e2["status_mismatch"] == 1 and e2["rays_compared"] == 2 and e2["group_path_km"]["max"] == 0.2


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
