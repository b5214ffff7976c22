"""The boundary locator of the accuracy gate (oracle/boundaries.py), on
hand-made traces whose boundaries are known exactly (no GPU, no ray tracing):
it must find a jump in ground range, a change of status and the end of a
singular (Pedersen-like) branch to below 0.01 deg, must not call a smooth
but steep stretch of D(el) a boundary, and must exclude exactly the rays
within 0.05 deg of what it found -- for whole fans and for sampled rays, with
each trace's own (frequency, mode, azimuth) passed to the tracer."""
import numpy as np

from oracle import boundaries as bd
from oracle import oracle
from paper_2506_18579_gb300 import workloads as wl

REC = np.dtype([("status", "i4"), ("ground_range_km", "f8"), ("group_path_km", "f8")])


def _records(el, shift=0.0):
    """A made-up trace: D rises smoothly and steeply (600 km/deg), jumps by
    200 km at 17.3137 + shift, runs off to infinity like a Pedersen ray as el
    approaches 33.4 + shift (status LANDED below, LEFT_GRID above), then
    lands again, and escapes from 41.0712 + shift on."""
    el = np.asarray(el, dtype=np.float64)
    r = np.zeros(len(el), REC)
    d = 1000.0 + 600.0 * el
    d += np.where(el > 17.3137 + shift, 200.0, 0.0)
    below = el < 33.4 + shift
    d += np.where(below, 20.0 / np.maximum(33.4 + shift - el, 1e-9), 0.0)
    r["status"] = np.where(el >= 41.0712 + shift, 2, np.where(below | (el >= 34.0 + shift), 1, 3))
    r["ground_range_km"] = d
    r["group_path_km"] = 1.1 * d
    return r


TRUE = (17.3137, 33.4, 34.0, 41.0712)


def test_locate_finds_jumps_status_changes_and_singular_ends_only():
    els = np.arange(5.0, 50.0 + 1e-9, 0.5)
    calls = []

    def trace(t_idx, el):
        calls.append(len(el))
        return _records(el)

    found = bd.locate([els], [_records(els)], trace)[0]
    assert len(found) == len(TRUE), found
    for (lo, hi), x in zip(found, TRUE):
        assert lo <= x <= hi
        # the approach to the singular end at 33.4 (D ~ 20 km / (33.4 - el)) is
        # steeper than JUMP_KM per RESOLUTION_DEG from ~0.08 deg below it
        assert hi - lo <= (0.1 if x == 33.4 else bd.RESOLUTION_DEG), (x, lo, hi)
    assert sum(calls) < len(els) * 2 ** 6  # bisection: far fewer traces than a 0.01-deg scan
    # a smooth stretch steeper than JUMP_KM per fan spacing is no boundary
    steep = np.arange(5.0, 15.0, 0.5)
    assert bd.locate([steep], [_records(steep)], trace)[0] == []


def test_near_excludes_within_the_radius_only():
    found = [[(17.31, 17.318)]]
    els = np.array([17.0, 17.25, 17.26, 17.3, 17.368, 17.369, 17.5])
    flag = bd.near([els], found)[0]
    assert flag.tolist() == [False, False, True, True, True, False, False]


class _FakeOracle:
    """fan_rays of the oracle; trace_rays answers from _records, its
    boundaries shifted by the ray's frequency and azimuth so that a trace
    handed the wrong (frequency, azimuth) finds them in the wrong place."""

    fan_rays = staticmethod(oracle.fan_rays)

    @staticmethod
    def trace_rays(grid, rays, n_threads=0):
        out = np.zeros(len(rays), REC)
        for k, ray in enumerate(rays):
            out[k] = _records([ray["el_deg"]], shift=_shift(ray["freq_mhz"], ray["az_deg"], ray["mode"]))[0]
        return out


def _shift(f, az, mode):
    return 0.1 * (f - 8.0) + 0.002 * az + (0.05 if mode < 0 else 0.0)


def _fan():
    return wl.FanSpec(30.0, 112.0, 0.0, freq_mhz=[8.0, 12.0], el_deg=np.round(np.arange(5.0, 50.0 + 1e-9, 0.5), 10),
                      az_deg=[0.0, 90.0], modes=wl.MODE_O | wl.MODE_X)


def _all_records(fan):
    res = np.zeros(fan.n_rays, REC)
    for i in range(fan.n_rays):
        f, m, el, az = fan.ray_params(i)
        res[i] = _records([el], _shift(f, az, m))[0]
    return res


def test_fan_exclusion_uses_each_traces_own_parameters():
    fan = _fan()
    res = _all_records(fan)
    mask, n_b = bd.fan_exclusion(_FakeOracle, None, fan, res)
    assert n_b == len(TRUE) * 2 * 2 * 2
    for i in range(fan.n_rays):
        f, m, el, az = fan.ray_params(i)
        s = _shift(f, az, m)
        dist = min(abs(el - (x + s)) for x in TRUE)
        # the singular end's boundary region reaches ~0.08 deg below it
        far = min(abs(el - (x + s)) if x != 33.4 else max(0.0, (x + s - 0.1) - el, el - (x + s))
                  for x in TRUE)
        if far > bd.EXCLUSION_DEG + bd.RESOLUTION_DEG:
            assert not mask[i], (f, m, el, az)
        elif dist <= bd.EXCLUSION_DEG:
            assert mask[i], (f, m, el, az)
    assert 0 < mask.sum() < 0.1 * fan.n_rays


def test_sample_exclusion_agrees_with_the_whole_fan():
    fan = _fan()
    res = _all_records(fan)
    whole, _ = bd.fan_exclusion(_FakeOracle, None, fan, res)
    idx = np.arange(fan.n_rays)
    part, _ = bd.sample_exclusion(_FakeOracle, None, fan, idx, res[idx])
    assert np.array_equal(part, whole)
