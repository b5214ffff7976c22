"""Parity of the CUDA tracer with the FP64 CPU oracle, through the C ABI.

Tolerances: the all-FP64 path agrees within 1e-6 km in group path, ground
range and apogee and 1e-7 deg in azimuth deviation; the mixed path within
0.05 km and 1e-4 deg over rays that are not within 0.05 deg of elevation of
a skip or Pedersen boundary.  The boundaries are located with the oracle
alone (oracle/boundaries.py: a status change or a jump of ground range or
group path between neighbouring elevations, bisected in elevation with the
oracle to below 0.01 deg; a smooth steep stretch is not a boundary), never
from the records under test.

Sizes: whole fans where the oracle finishes in seconds, the whole 24,840-ray
anisotropic fan at the tolerance the benchmark times (rtol 1e-8), a seeded
5,000-ray sample of the 495,122-ray ionogram batch at its timed rtol, plus
ragged and degenerate cases.

At rtol 1e-8 the integrator's own truncation error on grazing rays (low
elevation: a vertical error shows up ~1/sin(el) times larger in the landing
point) reaches 0.1-0.2 km -- in the oracle too, against a run converged at
rtol 1e-11.  A mixed-path ray whose float error estimate tips one discrete
step decision (accept/reject, the quantised step factor, a face-aligned
step) the other way than the oracle's takes a different step sequence, and
on such rays the two then differ by that truncation error.  The whole-fan
checks therefore bound the share of well-conditioned rays outside the bar
(and how far out they may be), and the bar holds for every well-conditioned
ray at ten times tighter rtol.  Azimuth deviation is the bearing of the end
point: for rays ending a few km from the transmitter (near-vertical rays)
1e-4 deg is millimetres, below the mixed path's position resolution, so it
too is checked as a share.
"""
import numpy as np
import pytest

from oracle import boundaries as bd
from paper_2506_18579_gb300 import build as rtbuild
from paper_2506_18579_gb300 import rtgd as rt
from paper_2506_18579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_KM, FP64_DEG = 1e-6, 1e-7
MIX_KM, MIX_DEG = 0.05, 1e-4
# whole-fan bounds of the mixed path at the timed tolerance (see the docstring)
MIX_SHARE_KM, MIX_CAP_KM = 0.9995, 0.5  # share of well-conditioned rays within MIX_KM; cap for the rest
MIX_SHARE_DEG, MIX_CAP_DEG = 0.995, 1e-3
MIX_STATUS_SHARE = 0.001  # at most 0.1 % of rays may end with another status than the oracle's


@pytest.fixture(scope="module", autouse=True)
def lib():
    rtbuild.build()
    return rt.load()


def _close64(gpu, ref, idx=None, km=FP64_KM, deg=FP64_DEG):
    g = gpu if idx is None else gpu[idx]
    assert np.array_equal(g["status"], ref["status"]), (g["status"], ref["status"])
    # landing latitude / longitude: the position tolerance in km, as degrees on
    # the sphere (1 deg of latitude = 111.19 km; longitude degrees up to 60 N)
    pos_deg = max(deg, km / 55.0)
    for f, tol in (("group_path_km", km), ("ground_range_km", km), ("apogee_km", km),
                   ("az_dev_deg", deg), ("land_lat_deg", pos_deg), ("land_lon_deg", pos_deg)):
        d = np.abs(g[f] - ref[f])
        assert np.all(d <= tol), (f, d.max(), int(np.argmax(d)))


def _mixed_vs_oracle(gpu, ref, well, what=""):
    """Whole-fan bounds of mixed records against oracle records: statuses,
    then P' and D (the accuracy gate) and the azimuth deviation over the
    well-conditioned rays with the oracle's status.  Returns the share of
    well-conditioned rays within the bar."""
    n = len(ref)
    mism = gpu["status"] != ref["status"]
    assert mism.sum() <= MIX_STATUS_SHARE * n, (what, int(mism.sum()))
    m = well & ~mism
    assert m.sum() >= 0.9 * well.sum(), what
    inside = np.ones(n, bool)
    for f in ("group_path_km", "ground_range_km"):
        d = np.abs(gpu[f] - ref[f])[m]
        assert np.mean(d <= MIX_KM) >= MIX_SHARE_KM, (what, f, int((d > MIX_KM).sum()), d.max())
        assert d.max() <= MIX_CAP_KM, (what, f, d.max())
        inside[m] &= np.abs(gpu[f] - ref[f])[m] <= MIX_KM
    d = np.abs(gpu["az_dev_deg"] - ref["az_dev_deg"])[m]
    assert np.mean(d <= MIX_DEG) >= MIX_SHARE_DEG, (what, int((d > MIX_DEG).sum()), d.max())
    assert d.max() <= MIX_CAP_DEG, (what, d.max())
    return float(inside[m].mean())


def _well(orc, og, spec, ref):
    """Rays not within 0.05 deg of a boundary located with the oracle."""
    mask, _ = bd.fan_exclusion(orc, og, spec, ref)
    return ~mask


# ------------------------------------------------------------------ RHS
def _states(w, n, seed):
    rng = np.random.default_rng(seed)
    RE = w.grid.earth_radius_km
    lat = rng.uniform(w.grid.lat0_deg + 1, w.grid.lat0_deg + (w.grid.n_lat - 2) * w.grid.dlat_deg, n)
    lon = rng.uniform(w.grid.lon0_deg + 1, w.grid.lon0_deg + (w.grid.n_lon - 2) * w.grid.dlon_deg, n)
    alt = rng.uniform(w.grid.alt0_km - 20, w.grid.alt0_km + (w.grid.n_alt - 1) * w.grid.dalt_km + 20, n)
    k = rng.normal(size=(n, 3))
    k *= (rng.uniform(0.3, 1.0, n) / np.linalg.norm(k, axis=1))[:, None]
    return np.column_stack([RE + alt, np.radians(90 - lat), np.radians(lon), k])


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_rhs_matches_oracle(orc, cfg):
    w = wl.config1() if cfg == "c1" else wl.config2()
    g = rt.Grid(w.grid, w.ne, table=True)
    og = orc.Grid(w.grid, w.ne)
    ys = _states(w, 400, 5)
    for f, mode in ((10.0, 1), (12.0, -1), (8.0, 1)):
        ref = np.array([orc.rhs(og, f, mode, y) for y in ys])
        scale = np.abs(ref).max(axis=0) + 1e-300
        dy64, _ = rt.rt_eval_rhs(g, f, mode, ys, rt.RT_FP64)
        assert np.max(np.abs(dy64 - ref) / scale) < 1e-10
        prev = None
        for st in (rt.RT_STENCIL_GATHER, rt.RT_STENCIL_QUAD, rt.RT_STENCIL_TABLE):
            dym, _ = rt.rt_eval_rhs(g, f, mode, ys, rt.RT_MIXED, st)
            assert np.max(np.abs(dym - ref) / scale) < 2e-4
            if prev is not None:  # the three sample layouts hold the same values
                assert np.array_equal(prev, dym)
            prev = dym


# ------------------------------------------------------------- FP64 path
def test_fp64_config1_all_rays(orc):
    w = wl.config1()
    g = rt.Grid(w.grid, w.ne)
    gpu = rt.rt_trace(g, rt.Fan(w.fan, rt.RT_FP64))
    ref = orc.trace_fan(orc.Grid(w.grid, w.ne), w.fan)
    assert np.all(ref["status"] == orc.LANDED)
    _close64(gpu, ref)
    assert np.array_equal(gpu["n_steps"], ref["n_steps"])
    assert np.array_equal(gpu["n_attempts"], ref["n_attempts"])


def _c2_small():
    return wl.config2(elev_step=6.0, az_step=60.0)  # 3 x 2 x 10 x 6 = 360 rays


def test_fp64_rkf45_small_fan(orc):
    w = _c2_small()
    g = rt.Grid(w.grid, w.ne)
    gpu = rt.rt_trace(g, rt.Fan(w.fan, rt.RT_FP64))
    ref = orc.trace_fan(orc.Grid(w.grid, w.ne), w.fan)
    _close64(gpu, ref)
    assert np.mean(gpu["n_attempts"] == ref["n_attempts"]) > 0.98


@pytest.fixture(scope="module")
def c2_oracle(orc):
    """The whole 24,840-ray anisotropic fan at the benchmark's rtol 1e-8:
    oracle records (all host cores, ~10 s) and the rays away from the
    boundaries the oracle locates."""
    w = wl.config2()
    assert w.fan.n_rays == 24840 and w.fan.rtol == 1e-8
    og = orc.Grid(w.grid, w.ne)
    ref = orc.trace_fan(og, w.fan)
    return w, og, ref, _well(orc, og, w.fan, ref)


def test_fp64_config2_whole_fan_against_the_oracle(c2_oracle):
    """Every ray of the fan, no exclusion: identical statuses, and the FP64
    tolerance on all but at most 0.02 % of the rays (a step decision within
    round-off of its threshold, e.g. a fused multiply-add on the GPU against
    the oracle's separate rounding, may go the other way), those within 1e-3 km."""
    w, _, ref, _ = c2_oracle
    g = rt.Grid(w.grid, w.ne)
    gpu = rt.rt_trace(g, rt.Fan(w.fan, rt.RT_FP64))
    assert np.array_equal(gpu["status"], ref["status"])
    off = np.zeros(len(ref), bool)
    for f, tol in (("group_path_km", FP64_KM), ("ground_range_km", FP64_KM), ("apogee_km", FP64_KM),
                   ("az_dev_deg", FP64_DEG)):
        d = np.abs(gpu[f] - ref[f])
        off |= d > tol
        assert d.max() <= (1e-3 if f != "az_dev_deg" else 1e-5), (f, d.max())
    assert off.sum() <= 0.0002 * len(ref), np.nonzero(off)[0]


# ------------------------------------------------------------ mixed path
@pytest.mark.parametrize("kernel", [rt.RT_KERNEL_PLAIN, rt.RT_KERNEL_PERSISTENT])
def test_mixed_config1_all_rays(orc, kernel):
    w = wl.config1()
    g = rt.Grid(w.grid, w.ne)
    gpu = rt.rt_trace(g, rt.Fan(w.fan, rt.RT_MIXED), cfg=rt.launch_config(kernel=kernel))
    ref = orc.trace_fan(orc.Grid(w.grid, w.ne), w.fan)
    _close64(gpu, ref, km=MIX_KM, deg=MIX_DEG)


def _variants():
    """Every launch configuration the autotuner may choose for the fan (kernel
    x stencil, the library's lane choice) and a few explicit lane counts."""
    keys = [(st, kern, 0) for st in (rt.RT_STENCIL_GATHER, rt.RT_STENCIL_QUAD, rt.RT_STENCIL_TABLE)
            for kern in (rt.RT_KERNEL_PLAIN, rt.RT_KERNEL_PERSISTENT)]
    return keys + [(rt.RT_STENCIL_QUAD, rt.RT_KERNEL_PERSISTENT, 1), (rt.RT_STENCIL_TABLE, rt.RT_KERNEL_PLAIN, 1),
                   (rt.RT_STENCIL_TABLE, rt.RT_KERNEL_PLAIN, 2), (rt.RT_STENCIL_GATHER, rt.RT_KERNEL_PLAIN, 4)]


def test_mixed_config2_whole_fan_against_the_oracle(c2_oracle):
    """The benchmark's workload itself (24,840 rays, rtol 1e-8), every launch
    configuration the tuner may time, against the oracle's records of the
    whole fan, over the rays away from oracle-located boundaries."""
    w, _, ref, well = c2_oracle
    assert well.mean() > 0.98  # boundaries exclude a few rays, not a band
    g = rt.Grid(w.grid, w.ne, table=True)
    fan = rt.Fan(w.fan, rt.RT_MIXED)
    for key in _variants():
        st, kern, lanes = key
        res = rt.rt_trace(g, fan, cfg=rt.launch_config(kernel=kern, stencil=st, lanes_per_ray=lanes))
        assert np.all(res["status"] != rt.RT_RAY_NOT_RUN), key
        _mixed_vs_oracle(res, ref, well, key)


def test_config2_fan_ordered_on_sms_of_its_own_keeps_every_record():
    """The benchmark's fan as a four-lane plan ordered by its own previous
    costs, its longest rays a warp each on SMs of their own (the bench's
    `fan_ordered`): the same records, byte for byte, as the plan's canonical
    execution -- eager and replayed from a captured graph."""
    torch = pytest.importorskip("torch")
    w = wl.config2()
    g = rt.Grid(w.grid, w.ne, table=True)
    fan = rt.Fan(w.fan, rt.RT_MIXED)
    n = fan.n_rays
    s = torch.cuda.current_stream()
    plan = rt.Plan(g, fan, rt.launch_config(kernel=rt.RT_KERNEL_PLAIN, stencil=rt.RT_STENCIL_TABLE,
                                            lanes_per_ray=4, block_threads=96,
                                            order=rt.RT_ORDER_ELEVATION_FASTEST))
    ref = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    plan.execute(ref.data_ptr(), n, stream=s.cuda_stream)
    s.synchronize()
    want = ref.cpu().numpy().tobytes()
    n_long = plan.order(ref.data_ptr(), spread=0, long_factor=2.0, rest_in_plan_order=True, long_exclusive=True,
                        long_alone=True, stream=s.cuda_stream)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 0 < n_long <= 2 * (sms // 8)
    out = torch.full((n * 64,), 0xAB, dtype=torch.uint8, device="cuda")
    plan.execute(out.data_ptr(), n, stream=s.cuda_stream)
    s.synchronize()
    assert out.cpu().numpy().tobytes() == want
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.execute(out.data_ptr(), n, stream=side.cuda_stream)
    for _ in range(2):
        out.fill_(0xAB)
        graph.replay()
        torch.cuda.synchronize()
        assert out.cpu().numpy().tobytes() == want
    del graph
    plan.close()


def test_mixed_config2_tighter_rtol_meets_the_bar_on_every_ray(orc):
    """At rtol 1e-9 the truncation error of a diverged step sequence is well
    inside 0.05 km: every well-conditioned ray of the fan (every second
    azimuth, 12,420 rays) meets the mixed bar in P', D and the apogee."""
    w = wl.config2()
    spec = w.fan.replace(rtol=1e-9, az_deg=w.fan.az_deg[::2])
    og = orc.Grid(w.grid, w.ne)
    ref = orc.trace_fan(og, spec)
    well = _well(orc, og, spec, ref)
    g = rt.Grid(w.grid, w.ne, table=True)
    for st, lanes in ((rt.RT_STENCIL_TABLE, 4), (rt.RT_STENCIL_QUAD, 1)):
        res = rt.rt_trace(g, rt.Fan(spec, rt.RT_MIXED), cfg=rt.launch_config(stencil=st, lanes_per_ray=lanes))
        m = well & (res["status"] == ref["status"])
        assert (~(res["status"] == ref["status"])).sum() <= MIX_STATUS_SHARE * len(ref)
        for f in ("group_path_km", "ground_range_km", "apogee_km"):
            d = np.abs(res[f] - ref[f])[m]
            assert d.max() <= MIX_KM, (st, lanes, f, d.max(), int((d > MIX_KM).sum()))


# --------------------------------------------------------- edge cases
def test_ragged_and_tiny_fans(orc):
    w = _c2_small()
    g = rt.Grid(w.grid, w.ne)
    og = orc.Grid(w.grid, w.ne)
    for n_el in (1, 3, 33):
        spec = w.fan.replace(el_deg=np.linspace(5.0, 55.0, n_el), az_deg=[17.0], freq_mhz=[9.0])
        ref = orc.trace_fan(og, spec)
        _close64(rt.rt_trace(g, rt.Fan(spec, rt.RT_FP64)), ref)
        spec9 = spec.replace(rtol=1e-9)
        ref9 = orc.trace_fan(og, spec9)
        ok = _well(orc, og, spec9, ref9)
        for kern in (rt.RT_KERNEL_PLAIN, rt.RT_KERNEL_PERSISTENT):
            for lanes in (1, 2, 4):
                gm = rt.rt_trace(g, rt.Fan(spec9, rt.RT_MIXED),
                                 cfg=rt.launch_config(kernel=kern, lanes_per_ray=lanes))
                _close64(gm[ok], ref9[ok], km=MIX_KM, deg=MIX_DEG)


@pytest.mark.parametrize("interp,stencil,integrator", [("gd", rt.RT_STENCIL_QUAD, wl.RKF45),
                                                       ("gd", rt.RT_STENCIL_TABLE, wl.RKF45),
                                                       ("cr", rt.RT_STENCIL_GATHER, wl.RKF45),
                                                       ("gd", rt.RT_STENCIL_QUAD, wl.RK4)])
def test_fused_requests_match_oracle(orc, interp, stencil, integrator):
    """The request server's fused kernel: the small C2-shaped fan split into
    one request per (frequency, azimuth), submitted at once to a fusing
    server (so that requests share launches), stitched back into fan order
    and compared with the oracle (GD and the Catmull-Rom option)."""
    w = _c2_small()
    # elevations 1.25 deg apart, so that neighbours show where a ray is near a boundary
    spec = w.fan.replace(rtol=1e-9, freq_mhz=[8.0, 12.0], el_deg=np.linspace(5.0, 55.0, 41),
                         integrator=integrator, h_km=1.0 if integrator == wl.RKF45 else 2.0)
    g = rt.Grid(w.grid, w.ne, table=stencil == rt.RT_STENCIL_TABLE, interp=interp)
    n_f, n_el, n_az = len(spec.freq_mhz), len(spec.el_deg), len(spec.az_deg)
    n_m = spec.n_rays // (n_f * n_el * n_az)
    parts = [(i, a, spec.replace(freq_mhz=[spec.freq_mhz[i]], az_deg=[spec.az_deg[a]]))
             for i in range(n_f) for a in range(n_az)]
    srv = rt.Server(max_inflight=1, cfg=rt.launch_config(stencil=stencil), fuse_max_rays=100000)
    fans = [rt.Fan(p, rt.RT_MIXED) for _, _, p in parts]
    tickets = [srv.submit(g, f) for f in fans]
    full = np.zeros(spec.n_rays, dtype=rt.RESULT_DTYPE)
    view = full.reshape(n_f, n_m, n_el, n_az)  # canonical order: frequency, mode, elevation, azimuth
    sizes = []
    for (i, a, _), (t, out) in zip(parts, tickets):
        st = srv.wait(t, timeout_s=300.0)
        assert st.status == rt.RT_OK
        sizes.append(st.batch_size)
        view[i, :, :, a] = out.reshape(n_m, n_el)
    srv.close()
    assert max(sizes) > 1
    og = orc.Grid(w.grid, w.ne, interp=interp)
    ref = orc.trace_fan(og, spec)
    ok = _well(orc, og, spec, ref)
    assert ok.sum() >= 200  # of 984 rays; the rest neighbour a status change or a range jump
    _close64(full[ok], ref[ok], km=MIX_KM, deg=MIX_DEG)


def test_trace_fans_device_matches_oracle_and_each_fan_alone(orc):
    """rt_trace_fans_device: fans of two transmitters 400 km apart and of
    several frequencies in one launch.  The records come fan after fan.
    Each fan's records equal, bit for bit, those of the same fan traced
    alone by the same call, and match the oracle."""
    torch = pytest.importorskip("torch")
    w = _c2_small()
    g = rt.Grid(w.grid, w.ne)
    og = orc.Grid(w.grid, w.ne)
    base = w.fan.replace(rtol=1e-9, el_deg=np.linspace(5.0, 55.0, 41), az_deg=[0.0, 120.0, 240.0])
    specs = [base.replace(freq_mhz=[8.0]), base.replace(freq_mhz=[12.0], tx_lat_deg=base.tx_lat_deg + 2.0),
             base.replace(freq_mhz=[10.0], modes=wl.MODE_O), base.replace(freq_mhz=[14.0], el_deg=[30.0], az_deg=[45.0])]
    fans = [rt.Fan(sp, rt.RT_MIXED) for sp in specs]
    sizes = [f.n_rays for f in fans]
    n = sum(sizes)
    cfg = rt.launch_config(stencil=rt.RT_STENCIL_QUAD)
    out = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    rt.rt_trace_fans_device(g, fans, out.data_ptr(), n, cfg=cfg, stream=s.cuda_stream)
    s.synchronize()
    res = rt.results_view(out.cpu().numpy(), n)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for k, (sp, f) in enumerate(zip(specs, fans)):
        part = res[off[k]:off[k + 1]]
        one = torch.zeros(f.n_rays * 64, dtype=torch.uint8, device="cuda")
        rt.rt_trace_fans_device(g, [f], one.data_ptr(), f.n_rays, cfg=cfg, stream=s.cuda_stream)
        s.synchronize()
        assert part.tobytes() == rt.results_view(one.cpu().numpy(), f.n_rays).tobytes(), k
        ref = orc.trace_fan(og, sp)
        ok = _well(orc, og, sp, ref)
        assert ok.sum() >= min(f.n_rays, 30)
        _close64(part[ok], ref[ok], km=MIX_KM, deg=MIX_DEG)


def test_trace_fans_device_with_hundreds_of_one_ray_fans():
    """300 one-ray fans in one call (the binary search over the fans' first
    rays, the record offsets) give the records of one 300-elevation fan."""
    torch = pytest.importorskip("torch")
    w = _c2_small()
    g = rt.Grid(w.grid, w.ne)
    els = np.linspace(3.0, 60.0, 300)
    whole = rt.Fan(w.fan.replace(freq_mhz=[10.0], modes=wl.MODE_X, el_deg=els, az_deg=[30.0]), rt.RT_MIXED)
    ones = [rt.Fan(w.fan.replace(freq_mhz=[10.0], modes=wl.MODE_X, el_deg=[e], az_deg=[30.0]), rt.RT_MIXED)
            for e in els]
    a = torch.zeros(300 * 64, dtype=torch.uint8, device="cuda")
    b = torch.zeros(300 * 64, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    rt.rt_trace_fans_device(g, [whole], a.data_ptr(), 300, stream=s.cuda_stream)
    rt.rt_trace_fans_device(g, ones, b.data_ptr(), 300, stream=s.cuda_stream)
    s.synchronize()
    ra = rt.results_view(a.cpu().numpy(), 300)
    assert np.all(ra["status"] != rt.RT_RAY_NOT_RUN)
    assert ra.tobytes() == rt.results_view(b.cpu().numpy(), 300).tobytes()


def test_trace_fans_device_refuses_what_it_cannot_fuse():
    torch = pytest.importorskip("torch")
    w = _c2_small()
    g = rt.Grid(w.grid, w.ne)
    mixed = rt.Fan(w.fan, rt.RT_MIXED)
    out = torch.zeros(mixed.n_rays * 2 * 64, dtype=torch.uint8, device="cuda")
    bad = [([], None), ([rt.Fan(w.fan, rt.RT_FP64)], None),
           ([mixed, rt.Fan(w.fan.replace(integrator=wl.RK4), rt.RT_MIXED)], None),
           ([mixed], rt.launch_config(kernel=rt.RT_KERNEL_PERSISTENT)),
           ([mixed], rt.launch_config(lanes_per_ray=1))]
    for fans, cfg in bad:
        with pytest.raises(rt.RtError) as ei:
            rt.rt_trace_fans_device(g, fans, out.data_ptr(), mixed.n_rays * 2, cfg=cfg)
        assert ei.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RtError) as ei:  # out_len below the rays of both fans
        rt.rt_trace_fans_device(g, [mixed, mixed], out.data_ptr(), mixed.n_rays * 2 - 1)
    assert ei.value.code == rt.RT_EINVAL


def test_statuses_match_oracle(orc):
    w = wl.config1()
    g = rt.Grid(w.grid, w.ne)
    og = orc.Grid(w.grid, w.ne)
    cases = [w.fan.replace(freq_mhz=[30.0], el_deg=[70.0]),        # escapes
             w.fan.replace(max_steps=10),                            # step budget
             w.fan.replace(tx_alt_km=150.0, max_group_path_km=123.4), # group-path limit
             w.fan.replace(integrator=wl.RKF45, rtol=1e-14, atol_km=1e-14, h_min_km=0.5)]  # underflow
    for spec in cases:
        ref = orc.trace_fan(og, spec)
        for prec in (rt.RT_FP64, rt.RT_MIXED):
            gpu = rt.rt_trace(g, rt.Fan(spec, prec))
            assert np.array_equal(gpu["status"], ref["status"]), (spec, prec)
    bad = w.ne.copy()
    bad[:, :, 10:] = np.nan
    gb = rt.Grid(w.grid, bad)
    for prec in (rt.RT_FP64, rt.RT_MIXED):
        assert np.all(rt.rt_trace(gb, rt.Fan(w.fan, prec))["status"] == rt.RT_RAY_NONFINITE)


def test_invalid_calls_are_errors():
    w = wl.config1()
    g = rt.Grid(w.grid, w.ne)
    fan = rt.Fan(w.fan)
    fan.desc.n_el = 0
    with pytest.raises(rt.RtError) as ei:
        rt.rt_trace(g, fan, out=np.zeros(16, dtype=rt.RESULT_DTYPE))
    assert ei.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RtError):
        rt.rt_trace(g, rt.Fan(w.fan), out=np.zeros(3, dtype=rt.RESULT_DTYPE))
    with pytest.raises(rt.RtError):  # table stencil on a grid without a table
        rt.rt_trace(g, rt.Fan(w.fan, rt.RT_MIXED), cfg=rt.launch_config(stencil=rt.RT_STENCIL_TABLE))
    with pytest.raises(rt.RtError):  # 3 lanes per ray
        rt.rt_trace(g, rt.Fan(w.fan, rt.RT_MIXED), cfg=rt.launch_config(lanes_per_ray=3))
    with pytest.raises(rt.RtError):  # the FP64 path is one lane per ray
        rt.rt_trace(g, rt.Fan(w.fan, rt.RT_FP64), cfg=rt.launch_config(lanes_per_ray=2))
    spec = w.grid
    with pytest.raises(rt.RtError):
        rt.Grid(wl.GridSpec(**{**spec.__dict__, "n_alt": 3}), w.ne[:, :, :3])


def test_fans_of_two_to_the_31_rays_are_refused():
    """The largest fan is 2^31 - 1 rays (32-bit ray indices on the device): a
    2^32-ray descriptor is refused before anything is queued, on every entry
    point that takes a fan (the output buffer here is deliberately tiny; the
    size check comes before any use of it)."""
    torch = pytest.importorskip("torch")
    w = wl.config1()
    g = rt.Grid(w.grid, w.ne)
    huge = rt.Fan(w.fan.replace(freq_mhz=np.full(65536, 10.0), el_deg=np.linspace(5.0, 50.0, 32768),
                                az_deg=[0.0], modes=wl.MODE_O | wl.MODE_X), rt.RT_MIXED)
    assert huge.n_rays == 1 << 32
    out = torch.empty(64, dtype=torch.uint8, device="cuda")
    for fn in (rt.rt_trace_device, rt.rt_trace_device_noalloc):
        with pytest.raises(rt.RtError) as ei:
            fn(g, huge, out.data_ptr(), huge.n_rays)
        assert ei.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RtError) as ei:
        rt.Plan(g, huge)
    assert ei.value.code == rt.RT_EINVAL
    torch.cuda.synchronize()


def test_device_output_and_tuner():
    torch = pytest.importorskip("torch")
    w = _c2_small()
    g = rt.Grid(w.grid, w.ne, table=True)
    fan = rt.Fan(w.fan, rt.RT_MIXED)
    n = fan.n_rays
    out = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    rt.rt_trace_device(g, fan, out.data_ptr(), n, stream=s.cuda_stream)
    s.synchronize()
    dev = rt.results_view(out.cpu().numpy(), n)
    host = rt.rt_trace(g, fan)
    assert dev.tobytes() == host.tobytes()
    best, ms = rt.rt_tune(g, fan, max_rays=512)
    assert ms > 0 and best.kernel in (rt.RT_KERNEL_PLAIN, rt.RT_KERNEL_PERSISTENT)
    tuned = rt.rt_trace(g, fan)  # picks the cached configuration
    assert np.array_equal(tuned["status"], host["status"])
    # the tuner releases its scratch (results and the 256 MiB L2-flush buffer):
    # repeated calls leave the device's free memory where it was
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rt.rt_tune(g, fan, max_rays=512)
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < (128 << 20)


def test_tuner_keeps_one_lane_per_ray_for_large_fans():
    """A fan of many waves of resident lanes is issue-bound: the tuner must
    not split rays over lanes there (it tries one lane per ray only); a fan
    smaller than the GPU may get more lanes."""
    w = wl.config1()
    g = rt.Grid(w.grid, w.ne)
    # 256,000 rays: above two waves of resident lanes (152 SMs x 3 or 4 blocks x 128)
    big = w.fan.replace(freq_mhz=np.linspace(6.0, 14.0, 16), el_deg=np.linspace(5.0, 50.0, 200),
                        az_deg=np.linspace(0.0, 351.0, 40), modes=wl.MODE_O | wl.MODE_X, h_km=2.0)
    fan = rt.Fan(big, rt.RT_MIXED)
    assert fan.n_rays == 256000
    best, ms = rt.rt_tune(g, fan, max_rays=16384)
    assert ms > 0 and best.lanes_per_ray == 1
    small = rt.Fan(w.fan.replace(h_km=2.0), rt.RT_MIXED)  # 16 rays
    best_s, _ = rt.rt_tune(g, small)
    assert best_s.lanes_per_ray in (1, 2, 4)
    res = rt.rt_trace(g, fan)  # the cached choice traces the whole fan
    assert np.all(res["status"] != rt.RT_RAY_NOT_RUN)


def test_catmull_rom_option_matches_oracle(orc):
    """The comparison interpolant (Eq. 6-9) as a grid option: RHS and whole
    rays against the oracle's Catmull-Rom, FP64 (1e-6 km) and mixed."""
    w = wl.config2(elev_step=6.0, az_step=60.0)
    g = rt.Grid(w.grid, w.ne, interp="cr")
    og = orc.Grid(w.grid, w.ne, interp="cr")
    ys = _states(w, 200, 8)
    ref = np.array([orc.rhs(og, 12.0, -1, y) for y in ys])
    scale = np.abs(ref).max(axis=0)
    dy64, _ = rt.rt_eval_rhs(g, 12.0, -1, ys, rt.RT_FP64)
    assert np.max(np.abs(dy64 - ref) / scale) < 1e-10
    dym, _ = rt.rt_eval_rhs(g, 12.0, -1, ys, rt.RT_MIXED)
    assert np.max(np.abs(dym - ref) / scale) < 2e-4
    spec = w.fan.replace(integrator=wl.RK4, h_km=1.0, el_deg=[8.0, 20.0, 32.0, 44.0], az_deg=[0.0, 120.0])
    ref_r = orc.trace_fan(og, spec)
    _close64(rt.rt_trace(g, rt.Fan(spec, rt.RT_FP64)), ref_r)
    ok = _well(orc, og, spec, ref_r)
    for lanes in (1, 2, 4):
        gm = rt.rt_trace(g, rt.Fan(spec, rt.RT_MIXED), cfg=rt.launch_config(lanes_per_ray=lanes))
        _close64(gm[ok], ref_r[ok], km=MIX_KM, deg=MIX_DEG)


def test_plan_execute_and_graph_replay():
    """A plan's execute step is a counter reset plus one launch: it gives the
    same records as rt_trace_device and can be captured into a CUDA graph."""
    torch = pytest.importorskip("torch")
    w = _c2_small()
    g = rt.Grid(w.grid, w.ne)
    for prec in (rt.RT_MIXED, rt.RT_FP64):
        fan = rt.Fan(w.fan, prec)
        n = fan.n_rays
        cfg = rt.launch_config(kernel=rt.RT_KERNEL_PERSISTENT if prec == rt.RT_MIXED else rt.RT_KERNEL_PLAIN,
                               stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=1)
        ref = rt.rt_trace(g, fan, cfg=cfg)
        plan = rt.Plan(g, fan, cfg)
        assert plan.n_rays == n
        out = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
        s = torch.cuda.current_stream()
        plan.execute(out.data_ptr(), n, stream=s.cuda_stream)
        s.synchronize()
        assert rt.results_view(out.cpu().numpy(), n).tobytes() == ref.tobytes()
        graph = torch.cuda.CUDAGraph()
        cap_out = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                plan.execute(cap_out.data_ptr(), n, stream=side.cuda_stream)
        for _ in range(2):
            cap_out.zero_()
            graph.replay()
            torch.cuda.synchronize()
            assert rt.results_view(cap_out.cpu().numpy(), n).tobytes() == ref.tobytes()
        plan.close()


def _rows(a):
    return np.ascontiguousarray(a).view(np.dtype((np.void, a.dtype.itemsize)))


@pytest.mark.parametrize("kernel", [rt.RT_KERNEL_PLAIN, rt.RT_KERNEL_PERSISTENT])
def test_ordered_plan_keeps_every_record(kernel):
    """rt_plan_order: longest-first claims give each ray the record it has in
    the plan's own order; with a four-lane share, every ray's record is either
    its one-lane record or (the rays of that share, the most expensive among
    them) its record from a four-lane plain trace.  Captured in a graph, the
    ordered plan replays deterministically; the four-lane share on SMs of its
    own or with a warp per ray gives the same records; ordering back to NULL
    restores the plan's own launch."""
    torch = pytest.importorskip("torch")
    w = wl.config2(elev_step=1.0, az_step=30.0)  # 3 x 2 x 58 x 12 = 4,176 rays
    g = rt.Grid(w.grid, w.ne)
    fan = rt.Fan(w.fan, rt.RT_MIXED)
    n = fan.n_rays
    s = torch.cuda.current_stream()

    def run(plan):
        out = torch.full((n * 64,), 0xAB, dtype=torch.uint8, device="cuda")
        plan.execute(out.data_ptr(), n, stream=s.cuda_stream)
        s.synchronize()
        return out, rt.results_view(out.cpu().numpy(), n).copy()

    plan = rt.Plan(g, fan, rt.launch_config(kernel=kernel, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=1))
    cost, ref = run(plan)
    assert np.all(ref["status"] != rt.RT_RAY_NOT_RUN)
    assert plan.order(cost.data_ptr(), spread=1, long_factor=0.0, stream=s.cuda_stream) == 0
    assert run(plan)[1].tobytes() == ref.tobytes()
    n_long = plan.order(cost.data_ptr(), spread=1, long_factor=3.0, stream=s.cuda_stream)
    assert 0 < n_long <= n // 16
    four = rt.rt_trace(g, fan, cfg=rt.launch_config(kernel=rt.RT_KERNEL_PLAIN, stencil=rt.RT_STENCIL_QUAD,
                                                    lanes_per_ray=4))
    got = run(plan)[1]
    is1, is4 = _rows(got) == _rows(ref), _rows(got) == _rows(four)
    assert np.all(is1 | is4)
    assert (~is1).sum() <= n_long
    top = int(np.argmax(ref["n_evals"]))
    assert is4[top]
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    cap = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.execute(cap.data_ptr(), n, stream=side.cuda_stream)
    for _ in range(2):
        cap.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert rt.results_view(cap.cpu().numpy(), n).tobytes() == got.tobytes()
    del graph
    # the four-lane share with a warp per ray (holes in the claim list), on SMs
    # of its own (cut to half the SM count in blocks), and both: four-lane
    # records for the share, the plan's own for the rest; captured and
    # replayed as well
    for excl, alone in ((True, False), (False, True), (True, True)):
        nl = plan.order(cost.data_ptr(), spread=1, long_factor=3.0, long_exclusive=excl, long_alone=alone,
                        stream=s.cuda_stream)
        assert 0 < nl <= n_long
        if not (excl and alone):
            assert nl == n_long
        got_x = run(plan)[1]
        is1, is4 = _rows(got_x) == _rows(ref), _rows(got_x) == _rows(four)
        assert np.all(is1 | is4) and (~is1).sum() <= nl and is4[top]
        if nl == n_long:
            assert got_x.tobytes() == got.tobytes()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                plan.execute(cap.data_ptr(), n, stream=side.cuda_stream)
        cap.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert rt.results_view(cap.cpu().numpy(), n).tobytes() == got_x.tobytes()
        del graph
    assert plan.order(None) == 0
    assert run(plan)[1].tobytes() == ref.tobytes()
    plan.close()


def test_plan_order_arguments_and_the_exclusive_cap():
    """rt_plan_order refuses unknown flags, a spread outside 0..64 and a
    non-finite factor (RT_EINVAL); with SMs of their own
    the four-lane share is cut to an eighth of the SM count in two-warp
    blocks (one ray per warp with a warp per ray), its most expensive rays
    first; an FP64 plan is ordered without a four-lane share and keeps its
    records."""
    import ctypes
    torch = pytest.importorskip("torch")
    w = wl.config2(elev_step=1.0, az_step=30.0)  # 4,176 rays
    g = rt.Grid(w.grid, w.ne)
    fan = rt.Fan(w.fan, rt.RT_MIXED)
    n = fan.n_rays
    s = torch.cuda.current_stream()
    plan = rt.Plan(g, fan, rt.launch_config(kernel=rt.RT_KERNEL_PLAIN, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=4))
    cost = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    plan.execute(cost.data_ptr(), n, stream=s.cuda_stream)
    s.synchronize()
    ref = rt.results_view(cost.cpu().numpy(), n).copy()
    lib = rt.load()
    nl = ctypes.c_size_t(7)
    for spread, factor, flags in ((0, 2.0, 8), (65, 2.0, 0), (-1, 2.0, 0), (0, float("nan"), 0)):
        r = lib.rt_plan_order(plan.handle, ctypes.c_void_p(cost.data_ptr()), spread, ctypes.c_double(factor),
                              flags, ctypes.byref(nl), ctypes.c_void_p(s.cuda_stream))
        assert r == rt.RT_EINVAL, (spread, factor, flags)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert plan.order(cost.data_ptr(), spread=0, long_factor=1e-3, stream=s.cuda_stream) == n // 16
    n_alone = plan.order(cost.data_ptr(), spread=0, long_factor=1e-3, long_exclusive=True, long_alone=True,
                         stream=s.cuda_stream)
    assert n_alone == min(n // 16, 2 * (sms // 8))
    n_excl = plan.order(cost.data_ptr(), spread=0, long_factor=1e-3, long_exclusive=True, stream=s.cuda_stream)
    assert n_excl == min(n // 16, 16 * (sms // 8))
    out = torch.full((n * 64,), 0xAB, dtype=torch.uint8, device="cuda")
    plan.execute(out.data_ptr(), n, stream=s.cuda_stream)
    s.synchronize()
    # every ray traced; with four lanes throughout, the order changes no record
    assert rt.results_view(out.cpu().numpy(), n).tobytes() == ref.tobytes()
    plan.close()
    # an FP64 plan takes the longest-first order (one thread per ray, no
    # four-lane share whatever the factor and flags) and keeps every record
    plan64 = rt.Plan(g, rt.Fan(w.fan, rt.RT_FP64))
    c64 = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    plan64.execute(c64.data_ptr(), n, stream=s.cuda_stream)
    s.synchronize()
    ref64 = rt.results_view(c64.cpu().numpy(), n).copy()
    assert plan64.order(c64.data_ptr(), spread=1, long_factor=3.0, long_exclusive=True, long_alone=True,
                        stream=s.cuda_stream) == 0
    out.fill_(0xAB)
    plan64.execute(out.data_ptr(), n, stream=s.cuda_stream)
    s.synchronize()
    assert rt.results_view(out.cpu().numpy(), n).tobytes() == ref64.tobytes()
    plan64.close()


@pytest.mark.parametrize("prec", [rt.RT_FP64, rt.RT_MIXED])
def test_ionogram_matches_oracle(orc, prec):
    w = wl.config2()
    g = rt.Grid(w.grid, w.ne)
    tx, rx = (30.0, 112.0, 0.0), (36.0, 119.0)
    freqs = np.arange(5.0, 17.0, 2.0)
    els = np.arange(2.0, 61.0, 1.0)
    pts, n = rt.rt_ionogram(g, tx, rx, freqs, els, precision=prec)
    assert n == len(pts) and n > 10
    # the same fan through the oracle (azimuth = initial bearing to the receiver)
    p1, p2, dl = np.radians(tx[0]), np.radians(rx[0]), np.radians(rx[1] - tx[1])
    x = np.cos(p1) * np.sin(p2) - np.sin(p1) * np.cos(p2) * np.cos(dl)
    y = np.sin(dl) * np.cos(p2)
    c = np.sin(p1) * np.sin(p2) + np.cos(p1) * np.cos(p2) * np.cos(dl)
    d_rx = w.grid.earth_radius_km * np.arctan2(np.hypot(x, y), c)
    spec = w.fan.replace(freq_mhz=freqs, el_deg=els, az_deg=[np.degrees(np.arctan2(y, x))])
    ref = orc.ionogram_points(orc.trace_fan(orc.Grid(w.grid, w.ne), spec), spec, d_rx)
    assert len(ref) == n
    km = FP64_KM if prec == rt.RT_FP64 else MIX_KM
    for p, q in zip(pts, ref):
        assert p["freq_mhz"] == q[0] and p["mode"] == q[3] and p["branch"] == q[4]
        assert abs(p["group_path_km"] - q[1]) <= (km if prec == rt.RT_FP64 else 0.5)
        assert p["ground_range_km"] == pytest.approx(d_rx, abs=1e-9)
    if prec == rt.RT_FP64:
        np.testing.assert_allclose([p["el_deg"] for p in pts], [q[2] for q in ref], atol=1e-6)


@pytest.fixture(scope="module")
def c4_sample(orc):
    """The ionogram-synthesis batch at its timed rtol: a seeded 5,000-ray
    sample traced by the oracle, and which of those rays lie away from the
    boundaries the oracle locates around them."""
    w = wl.config4()
    assert w.fan.n_rays == 495122 and w.fan.rtol == 1e-8
    og = orc.Grid(w.grid, w.ne)
    idx = wl.sample_indices(w.fan.n_rays, 5000, seed=1234)
    ref = orc.trace_fan(og, w.fan, indices=idx)
    near, _ = bd.sample_exclusion(orc, og, w.fan, idx, ref)
    return w, idx, ref, ~near


def test_config4_batched_fan_in_captured_graph(c4_sample):
    """The ionogram-synthesis batch at full size and its timed rtol 1e-8:
    181x361x301 grid, 281 frequencies x 881 elevations x O/X = 495,122 rays of
    50-5000 steps, run as one plan captured in a CUDA graph (mixed; plain and
    persistent kernel) and by the FP64 kernel; 5,000 seeded rays of each
    against the oracle."""
    torch = pytest.importorskip("torch")
    w, idx, ref, well = c4_sample
    g = rt.Grid(w.grid, w.ne)
    n = w.fan.n_rays
    plan = rt.Plan(g, rt.Fan(w.fan, rt.RT_MIXED))
    out = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.execute(out.data_ptr(), n, stream=side.cuda_stream)
    graph.replay()
    torch.cuda.synchronize()
    mixed = rt.results_view(out.cpu().numpy(), n).copy()
    assert np.all(mixed["status"] != rt.RT_RAY_NOT_RUN)
    st = np.bincount(mixed["status"], minlength=8)
    assert st[rt.RT_RAY_LANDED] > 0.1 * n and st[rt.RT_RAY_ESCAPED] > 0.1 * n  # mixed outcomes
    steps = mixed["n_steps"]
    assert steps.min() < 150 and steps.max() > 5000  # uneven ray lengths (~100 to ~7,600 steps)
    assert well.mean() > 0.98
    _mixed_vs_oracle(mixed[idx], ref, well, "plain graph")
    plan.close()
    fp64 = rt.rt_trace(g, rt.Fan(w.fan, rt.RT_FP64))[idx]  # every sampled ray, no exclusion
    assert np.array_equal(fp64["status"], ref["status"])
    off = np.zeros(len(idx), bool)
    for f, tol in (("group_path_km", FP64_KM), ("ground_range_km", FP64_KM), ("apogee_km", FP64_KM),
                   ("az_dev_deg", FP64_DEG)):
        d = np.abs(fp64[f] - ref[f])
        off |= d > tol
        assert d.max() <= (1e-3 if f != "az_dev_deg" else 1e-5), (f, d.max())
    assert off.sum() <= 2, np.nonzero(off)[0]
    # the same batch as one persistent launch (lane groups claim rays from an
    # atomic counter), also captured in a graph and replayed twice
    cfg = rt.launch_config(kernel=rt.RT_KERNEL_PERSISTENT, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=1,
                           order=rt.RT_ORDER_ELEVATION_FASTEST)
    pplan = rt.Plan(g, rt.Fan(w.fan, rt.RT_MIXED), cfg=cfg)
    outp = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    pgraph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(pgraph, stream=side):
            pplan.execute(outp.data_ptr(), n, stream=side.cuda_stream)
    pgraph.replay()
    torch.cuda.synchronize()
    first = outp.cpu().numpy().copy()
    pgraph.replay()
    torch.cuda.synchronize()
    pers = rt.results_view(outp.cpu().numpy(), n).copy()
    assert pers.tobytes() == first.tobytes()  # replays are deterministic
    assert np.all(pers["status"] != rt.RT_RAY_NOT_RUN)
    _mixed_vs_oracle(pers[idx], ref, well, "persistent graph")
    # longest-first, with the costs of the same scan on a later snapshot of
    # the ionosphere (the TID advanced by 5 % of its period) and the most
    # expensive rays at four lanes: the records still meet the bars
    w5 = wl.config4(tid_phase_shift=0.05)
    g5 = rt.Grid(w5.grid, w5.ne)
    prev = torch.zeros(n * 64, dtype=torch.uint8, device="cuda")
    rt.rt_trace_device(g5, rt.Fan(w5.fan, rt.RT_MIXED), prev.data_ptr(), n, cfg=cfg, stream=side.cuda_stream)
    torch.cuda.synchronize()
    n_long = pplan.order(prev.data_ptr(), spread=2, long_factor=6.0, stream=side.cuda_stream)
    assert 0 < n_long < 0.01 * n
    assert pplan.order(prev.data_ptr(), spread=2, long_factor=6.0, rest_in_plan_order=True,
                       stream=side.cuda_stream) == n_long
    outp.zero_()
    pplan.execute(outp.data_ptr(), n, stream=side.cuda_stream)
    torch.cuda.synchronize()
    ordered = rt.results_view(outp.cpu().numpy(), n).copy()
    assert np.all(ordered["status"] != rt.RT_RAY_NOT_RUN)
    _mixed_vs_oracle(ordered[idx], ref, well, "ordered persistent")
    # the four-lane share on SMs of its own (cut to an eighth of the SMs)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n_excl = pplan.order(prev.data_ptr(), spread=2, long_factor=6.0, long_exclusive=True, stream=side.cuda_stream)
    assert 0 < n_excl <= min(n_long, 16 * (sms // 8))
    outp.zero_()
    pplan.execute(outp.data_ptr(), n, stream=side.cuda_stream)
    torch.cuda.synchronize()
    excl = rt.results_view(outp.cpu().numpy(), n).copy()
    assert np.all(excl["status"] != rt.RT_RAY_NOT_RUN)
    _mixed_vs_oracle(excl[idx], ref, well, "ordered persistent, exclusive share")
    pplan.close()
    g5.close()
