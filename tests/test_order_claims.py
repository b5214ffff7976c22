"""The longest-first claim list (rt_order_claims, the host arithmetic that
rt_plan_order uploads), checked on the CPU against a plain numpy statement
of the rule, element for element:

  1. expected cost = the largest cost within `spread` elevation steps, then
     within `spread` frequency steps (same mode and azimuth);
  2. rays in descending key floor(8 log2 cost), canonical order within a key;
  3. the four-lane share (mixed plans, long_factor > 0): the leading rays of
     that order whose expected cost is at least long_factor times the median
     (the element of rank n/2), at most n/16 of them; with SMs of their own,
     at most sm_count/8 two-warp blocks of them;
  4. the share in the plan's claim order; the other rays in the order of
     step 2, or in the plan's claim order;
  5. with a warp per share ray, seven holes (-1) after each share ray.
No GPU is used: the call is host arithmetic only."""
import ctypes
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2506_18579_gb300 import rtgd as rt  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2506_18579_gb300 import build as rtbuild
    rtbuild.build()
    return rt.load()


def _window_max(a, axis, spread):
    out = a.copy()
    length = a.shape[axis]
    for d in range(1, spread + 1):
        if d >= length:
            break
        lo = [slice(None)] * a.ndim
        hi = [slice(None)] * a.ndim
        lo[axis] = slice(0, length - d)
        hi[axis] = slice(d, length)
        out[tuple(lo)] = np.maximum(out[tuple(lo)], a[tuple(hi)])
        out[tuple(hi)] = np.maximum(out[tuple(hi)], a[tuple(lo)])
    return out


def _claim_sequence(dims, claim_order):
    """Canonical ray index of each claim of the plan's own order."""
    n_f, n_m, n_e, n_a = dims
    n = n_f * n_m * n_e * n_a
    c = np.arange(n)
    if claim_order != rt.RT_ORDER_ELEVATION_FASTEST:
        return c
    e, rest = c % n_e, c // n_e
    a, fm = rest % n_a, rest // n_a
    return (fm * n_e + e) * n_a + a


def reference(cost, dims, claim_order, spread, long_factor, mixed, rest, exclusive, alone, sm_count):
    n_f, n_m, n_e, n_a = dims
    n = n_f * n_m * n_e * n_a
    c = np.asarray(cost, dtype=np.int64).reshape(n_f, n_m, n_e, n_a)
    if spread:
        c = _window_max(_window_max(c, 2, spread), 0, spread)
    c = c.reshape(-1)
    key = np.floor(8.0 * np.log2(np.maximum(c, 1))).astype(np.int64)
    perm = np.argsort(-key, kind="stable")
    nl = 0
    if mixed and long_factor > 0:
        median = np.sort(c)[n // 2]
        while nl < n // 16 and c[perm[nl]] >= long_factor * median:
            nl += 1
    if exclusive and nl > 0:
        nl = min(nl, max(sm_count // 8, 1) * (1 if alone else 8) * 2)
    position = np.empty(n, np.int64)
    position[_claim_sequence(dims, claim_order)] = np.arange(n)  # claim index of each ray
    share = list(perm[:nl])
    if nl > 1:
        share.sort(key=lambda r: position[r])
    if rest:
        in_share = set(share)
        others = [r for r in _claim_sequence(dims, claim_order) if r not in in_share]
    else:
        others = list(perm[nl:])
    head = [x for r in share for x in ([r] + [-1] * 7)] if alone else share
    return np.array(head + others, dtype=np.int64), nl


def _costs(rng, dims):
    """Lognormal costs with a few long ridges along elevation (the shape of
    near-critical rays) and some exact ties."""
    n_f, n_m, n_e, n_a = dims
    c = rng.lognormal(7.5, 0.4, size=dims)
    for _ in range(3):
        f, m, a = rng.integers(n_f), rng.integers(n_m), rng.integers(n_a)
        e0 = rng.integers(n_e)
        c[f, m, e0:e0 + 3, a] *= rng.uniform(4.0, 12.0)
    c = np.round(c).astype(np.int32)
    c.reshape(-1)[rng.integers(0, c.size, 5)] = 2048  # powers of two sit on key boundaries
    return c.reshape(-1)


CASES = [
    # dims, claim order, spread, long factor, mixed, rest, exclusive, alone, SMs
    ((3, 2, 40, 4), 1, 0, 3.0, True, False, False, False, 152),
    ((3, 2, 40, 4), 1, 1, 2.0, True, False, False, True, 152),
    ((3, 2, 40, 4), 0, 2, 2.0, True, True, False, False, 152),
    ((5, 1, 33, 1), 1, 1, 1.5, True, True, True, True, 152),
    ((5, 1, 33, 1), 1, 0, 1.2, True, False, True, False, 16),
    ((4, 2, 17, 3), 0, 3, 0.0, True, True, False, False, 152),
    ((4, 2, 17, 3), 1, 1, 2.0, False, False, True, True, 152),  # FP64 plan: no share
    ((2, 2, 9, 1), 1, 64, 1.0, True, False, False, True, 152),   # spread past the edges
    ((1, 1, 1, 1), 1, 2, 2.0, True, True, True, True, 152),     # a one-ray fan
    ((7, 2, 50, 2), 1, 1, 1.05, True, False, True, True, 8),    # a tiny GPU: one exclusive block
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_claims_follow_the_rule(case):
    dims, order, spread, lf, mixed, rest, excl, alone, sms = CASES[case]
    rng = np.random.default_rng(100 + case)
    cost = _costs(rng, dims)
    got, nl = rt.rt_order_claims(cost, dims, claim_order=order, spread=spread, long_factor=lf, mixed=mixed,
                                 rest_in_plan_order=rest, long_exclusive=excl, long_alone=alone, sm_count=sms)
    want, nl_want = reference(cost, dims, order, spread, lf, mixed, rest, excl, alone, sms)
    assert nl == nl_want
    np.testing.assert_array_equal(got, want)
    # every ray is claimed exactly once; holes only behind share rays
    n = cost.size
    rays = got[got >= 0]
    assert np.array_equal(np.sort(rays), np.arange(n))
    assert (got < 0).sum() == (7 * nl if alone else 0)


def test_the_share_is_what_the_factor_selects():
    """A fan whose costs are known exactly: 4 rays cost 10x the rest; with
    factor 5 the share is those 4 rays, in claim order, at the front."""
    dims = (2, 1, 20, 2)
    cost = np.full(80, 1000, np.int32)
    long_rays = [5, 22, 41, 70]
    cost[long_rays] = 10000
    claims, nl = rt.rt_order_claims(cost, dims, spread=0, long_factor=5.0)
    assert nl == 4
    # claim order is elevation fastest: ray ((f*n_m+m)*n_e+e)*n_a+a has claim ((f*n_m+m)*n_a+a)*n_e+e
    assert list(claims[:4]) == [22, 5, 70, 41]
    assert sorted(claims[4:]) == sorted(set(range(80)) - set(long_rays))
    # no share with factor 0, and none for an FP64 plan
    assert rt.rt_order_claims(cost, dims, spread=0, long_factor=0.0)[1] == 0
    assert rt.rt_order_claims(cost, dims, spread=0, long_factor=5.0, mixed=False)[1] == 0


def test_the_median_is_the_element_of_rank_n_over_2():
    """64 rays: 32 cost 1000, 28 cost 1001, 4 cost 2001.  The element of rank
    32 is 1001, so a factor of 2 (threshold 2002) takes no ray and 1.999
    (2000.999) takes the four; a median of 1000 would take them at 2."""
    rng = np.random.default_rng(7)
    cost = np.array([1000] * 32 + [1001] * 28 + [2001] * 4, np.int32)[rng.permutation(64)]
    dims = (1, 1, 64, 1)
    assert rt.rt_order_claims(cost, dims, spread=0, long_factor=2.0)[1] == 0
    claims, nl = rt.rt_order_claims(cost, dims, spread=0, long_factor=1.999)
    assert nl == 4 and np.all(cost[claims[:4]] == 2001)


def test_bad_arguments_are_refused():
    lib = rt.load()
    cost = np.full(40, 100, np.int32)
    out = np.empty(100, np.int32)
    nl, nc = ctypes.c_size_t(), ctypes.c_size_t()

    def call(dims=(2, 1, 10, 2), order=1, spread=0, lf=2.0, flags=0, sms=152, cap=100):
        return lib.rt_order_claims(cost.ctypes.data, *dims, order, spread, ctypes.c_double(lf), 1, flags, sms,
                                   out.ctypes.data, cap, ctypes.byref(nl), ctypes.byref(nc))

    assert call() == rt.RT_OK and nc.value == 40
    for kw in (dict(dims=(0, 1, 10, 2)), dict(dims=(2, 3, 10, 2)), dict(order=2), dict(spread=65),
               dict(spread=-1), dict(lf=float("inf")), dict(flags=8), dict(flags=2, sms=0), dict(cap=39)):
        assert call(**kw) == rt.RT_EINVAL, kw
