"""Skip / Pedersen boundaries of ray fans, located with the FP64 oracle.

TEST INFRASTRUCTURE ONLY: used by tests/ and by the CPU-baseline leg of
bench.py to decide which rays the mixed-precision accuracy bar applies to.
The product path never imports it.

Near-critical rays (Sec. IV-B-3) are ill-conditioned: close to the
elevation where a trace (one frequency, mode and azimuth) changes outcome --
a ray that lands next to one that escapes or leaves the grid, the far end of
a Pedersen ray, the hand-over from E-layer to F-layer reflection -- ground
range and group path change without bound for a vanishing change of
elevation.  The accuracy bar for the mixed path applies to rays more than
0.05 deg of elevation away from such a boundary.  This module finds the
boundaries, from oracle records only:

  1. A pair of neighbouring elevations of a trace is a candidate when the two
     rays' statuses differ or their ground ranges or group paths differ by
     more than JUMP_KM.
  2. A candidate pair is bisected in elevation with the oracle: the midpoint
     is traced and each half that is still a candidate (same test, same
     JUMP_KM) is kept, until the halves are narrower than RESOLUTION_DEG.  A
     discontinuity keeps its jump however narrow the interval; a smooth but
     steep stretch of D(el) stops being a candidate once the interval is
     narrow enough (its difference shrinks with the width) and is not a
     boundary.  Near a singular end (D -> infinity) D(el) stays steeper than
     that over a short stretch; the touching intervals found there merge
     into one boundary region.
  3. A ray is excluded when its elevation lies within EXCLUSION_DEG of a
     located boundary interval (the boundary itself lies somewhere inside
     the interval, so this excludes at most RESOLUTION_DEG more than needed).
"""
from __future__ import annotations

import numpy as np

JUMP_KM = 30.0
RESOLUTION_DEG = 0.01
EXCLUSION_DEG = 0.05


def is_candidate(ra, rb, jump_km=JUMP_KM):
    """Elementwise: do records ra and rb (same trace, neighbouring
    elevations) straddle a possible boundary?"""
    return ((ra["status"] != rb["status"]) |
            (np.abs(ra["ground_range_km"] - rb["ground_range_km"]) > jump_km) |
            (np.abs(ra["group_path_km"] - rb["group_path_km"]) > jump_km))


def locate(els, recs, trace_fn, jump_km=JUMP_KM, resolution_deg=RESOLUTION_DEG):
    """Boundary intervals of several traces.

    els[t]: ascending elevations (deg) of trace t; recs[t]: its records
    (fields status, ground_range_km, group_path_km) at those elevations.
    trace_fn(t_idx, el) traces rays of traces t_idx (int array) at elevations
    el (float array) and returns their records.  Returns, per trace, a list of
    (lo, hi) elevation intervals, each narrower than resolution_deg and
    holding one boundary; touching intervals are merged, so the approach to a
    singular end, where D(el) stays steeper than jump_km per resolution_deg
    for a while, comes back as one wider interval."""
    found = [[] for _ in els]
    act_t, act_a, act_b, act_ra, act_rb = [], [], [], [], []
    for t, (e, r) in enumerate(zip(els, recs)):
        e = np.asarray(e, dtype=np.float64)
        if len(e) < 2:
            continue
        c = np.nonzero(is_candidate(r[:-1], r[1:], jump_km))[0]
        act_t.append(np.full(len(c), t))
        act_a.append(e[c])
        act_b.append(e[c + 1])
        act_ra.append(r[c])
        act_rb.append(r[c + 1])
    if not act_t:
        return found
    t_i = np.concatenate(act_t)
    a = np.concatenate(act_a)
    b = np.concatenate(act_b)
    ra = np.concatenate(act_ra)
    rb = np.concatenate(act_rb)
    for _ in range(64):  # each pass halves every interval: 64 passes resolve any double range
        narrow = (b - a) <= resolution_deg
        for t, lo, hi in zip(t_i[narrow], a[narrow], b[narrow]):
            found[int(t)].append((float(lo), float(hi)))
        keep = ~narrow
        t_i, a, b, ra, rb = t_i[keep], a[keep], b[keep], ra[keep], rb[keep]
        if len(t_i) == 0:
            break
        m = 0.5 * (a + b)
        rm = trace_fn(t_i, m)
        left = is_candidate(ra, rm, jump_km)
        right = is_candidate(rm, rb, jump_km)
        t_i = np.concatenate([t_i[left], t_i[right]])
        a, b = np.concatenate([a[left], m[right]]), np.concatenate([m[left], b[right]])
        ra, rb = np.concatenate([ra[left], rm[right]]), np.concatenate([rm[left], rb[right]])
    for k, f in enumerate(found):  # touching intervals: one boundary region
        f.sort()
        merged = []
        for lo, hi in f:
            if merged and lo <= merged[-1][1]:
                merged[-1] = (merged[-1][0], max(hi, merged[-1][1]))
            else:
                merged.append((lo, hi))
        found[k] = merged
    return found


def near(els, found, radius_deg=EXCLUSION_DEG):
    """Per trace, a boolean array over els[t]: elevation within radius_deg of
    one of the trace's boundary intervals."""
    out = []
    for e, intervals in zip(els, found):
        e = np.asarray(e, dtype=np.float64)
        flag = np.zeros(len(e), bool)
        for lo, hi in intervals:
            flag |= (e >= lo - radius_deg) & (e <= hi + radius_deg)
        out.append(flag)
    return out


def fan_traces(fan):
    """(freq_mhz, mode sign, az_deg) of every trace of a fan, in the order
    [freq][mode][az] that fan_records_by_trace uses."""
    return [(f, m, az) for f in fan.freq_mhz for m in fan.mode_list for az in fan.az_deg]


def fan_records_by_trace(res, fan):
    """Records of a whole fan (canonical order [freq][mode][el][az]) split into
    traces: an array [n_trace, n_el]."""
    n_f, n_m, n_e, n_a = len(fan.freq_mhz), len(fan.mode_list), len(fan.el_deg), len(fan.az_deg)
    r = np.asarray(res).reshape(n_f, n_m, n_e, n_a)
    return np.ascontiguousarray(r.transpose(0, 1, 3, 2)).reshape(n_f * n_m * n_a, n_e)


def oracle_trace_fn(oracle, grid, fan, traces, n_threads=0):
    """trace_fn for locate(): rays of `fan`'s settings with (frequency, mode,
    azimuth) of traces[t] at the given elevations, traced by the oracle."""
    tr = np.array(traces, dtype=np.float64).reshape(-1, 3)

    def fn(t_idx, el):
        t_idx = np.asarray(t_idx, dtype=np.int64)
        rays = np.repeat(oracle.fan_rays(fan, [0]), len(t_idx))
        rays["freq_mhz"] = tr[t_idx, 0]
        rays["mode"] = tr[t_idx, 1].astype(np.int32)
        rays["az_deg"] = tr[t_idx, 2]
        rays["el_deg"] = np.asarray(el, dtype=np.float64)
        return oracle.trace_rays(grid, rays, n_threads)
    return fn


def fan_exclusion(oracle, grid, fan, res, n_threads=0, radius_deg=EXCLUSION_DEG):
    """Rays of a whole fan (canonical order) within radius_deg of a skip or
    Pedersen boundary, located with the oracle from its records res of the
    same fan.  Returns (mask over the fan's rays, number of boundaries)."""
    traces = fan_traces(fan)
    by_trace = fan_records_by_trace(res, fan)
    els = [fan.el_deg] * len(traces)
    found = locate(els, list(by_trace), oracle_trace_fn(oracle, grid, fan, traces, n_threads))
    flags = np.array(near(els, found, radius_deg))  # [n_trace, n_el]
    n_f, n_m, n_e, n_a = len(fan.freq_mhz), len(fan.mode_list), len(fan.el_deg), len(fan.az_deg)
    mask = flags.reshape(n_f, n_m, n_a, n_e).transpose(0, 1, 3, 2).reshape(-1)
    return mask, sum(len(f) for f in found)


def sample_exclusion(oracle, grid, fan, idx, res_idx, n_threads=0, radius_deg=EXCLUSION_DEG):
    """For sampled rays idx of a fan (with oracle records res_idx): which lie
    within radius_deg of a boundary.  Each sampled ray's neighbouring fan
    elevations (one below, one above) are traced by the oracle and the two
    pairs they form with it are searched as in locate().  Returns (mask over
    idx, number of boundaries)."""
    idx = np.asarray(idx)
    n_a, n_e = len(fan.az_deg), len(fan.el_deg)
    modes = fan.mode_list
    a = idx % n_a
    e = (idx // n_a) % n_e
    m = (idx // (n_a * n_e)) % len(modes)
    f = idx // (n_a * n_e * len(modes))
    traces = [(fan.freq_mhz[fi], modes[mi], fan.az_deg[ai]) for fi, mi, ai in zip(f, m, a)]
    lo = np.maximum(e - 1, 0)
    hi = np.minimum(e + 1, n_e - 1)
    fn = oracle_trace_fn(oracle, grid, fan, traces, n_threads)
    t_all = np.arange(len(idx))
    r_lo = fn(t_all, fan.el_deg[lo])
    r_hi = fn(t_all, fan.el_deg[hi])
    els, recs = [], []
    for k in range(len(idx)):
        ek, rk = [], []
        if lo[k] < e[k]:
            ek.append(fan.el_deg[lo[k]])
            rk.append(r_lo[k])
        ek.append(fan.el_deg[e[k]])
        rk.append(res_idx[k])
        if hi[k] > e[k]:
            ek.append(fan.el_deg[hi[k]])
            rk.append(r_hi[k])
        els.append(np.array(ek))
        recs.append(np.array(rk, dtype=np.asarray(res_idx).dtype))
    found = locate(els, recs, fn)
    mask = np.zeros(len(idx), bool)
    for k, intervals in enumerate(found):
        el = fan.el_deg[e[k]]
        mask[k] = any(lo_ - radius_deg <= el <= hi_ + radius_deg for lo_, hi_ in intervals)
    return mask, sum(len(x) for x in found)
