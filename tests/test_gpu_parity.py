"""Parity of the CUDA tracer with the FP64 CPU oracle, through the C ABI.

Tolerances: the all-FP64 path agrees within 1e-6 km in group path and ground
range and 1e-7 deg in azimuth deviation; the mixed path within 0.05 km and
1e-4 deg, over rays that are not next to a skip or Pedersen boundary (a
status change or a range jump between neighbouring elevations).  Sizes: full
fans where the oracle finishes in seconds, seeded samples of the full-size
fans otherwise, plus ragged and degenerate cases.
"""
import numpy as np
import pytest

from paper_2506_18579_gb300 import build as rtbuild
from paper_2506_18579_gb300 import rtgd as rt
from paper_2506_18579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_KM, FP64_DEG = 1e-6, 1e-7
MIX_KM, MIX_DEG = 0.05, 1e-4


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


def near_boundary(res, fan):
    """Rays adjacent (in elevation) to a status change or a jump of ground
    range or group path larger than 30 km between neighbouring elevations."""
    n_az, n_el = len(fan.az_deg), len(fan.el_deg)
    r = res.reshape(-1, n_el, n_az)
    flag = np.zeros(r.shape, bool)
    jump = ((r["status"][:, 1:] != r["status"][:, :-1]) |
            (np.abs(np.diff(r["ground_range_km"], axis=1)) > 30.0) |
            (np.abs(np.diff(r["group_path_km"], axis=1)) > 30.0))
    flag[:, 1:] |= jump
    flag[:, :-1] |= jump
    return flag.reshape(-1)


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


def test_fp64_config2_full_size_sampled(orc):
    w = wl.config2()
    assert w.fan.n_rays == 24840
    g = rt.Grid(w.grid, w.ne)
    gpu = rt.rt_trace(g, rt.Fan(w.fan, rt.RT_FP64))
    idx = wl.sample_indices(w.fan.n_rays, 48, seed=21)
    ref = orc.trace_fan(orc.Grid(w.grid, w.ne), w.fan, indices=idx)
    _close64(gpu[idx], ref)
    assert np.all(gpu["status"] != rt.RT_RAY_NOT_RUN)


# ------------------------------------------------------------ mixed path
@pytest.mark.parametrize("kernel", [rt.RT_KERNEL_PLAIN, rt.RT_KERNEL_PERSISTENT])
def test_mixed_config1_all_rays(orc, kernel):
    w = wl.config1()
    g = rt.Grid(w.grid, w.ne)
    gpu = rt.rt_trace(g, rt.Fan(w.fan, rt.RT_MIXED), cfg=rt.launch_config(kernel=kernel))
    ref = orc.trace_fan(orc.Grid(w.grid, w.ne), w.fan)
    _close64(gpu, ref, km=MIX_KM, deg=MIX_DEG)


def test_mixed_config2_full_size(orc):
    """C2 at full size, every kernel and stencil variant.  Accuracy is judged
    at rtol 1e-9, for each variant: at the C2 setting of
    1e-8 the integrator's own error reaches ~0.1 km on long-range rays (in FP64
    too), so two runs whose step sequences differ (the mixed path's FP32 error
    estimate sees round-off at the 1e-8 level) cannot agree to 0.05 km there."""
    w = wl.config2()
    g = rt.Grid(w.grid, w.ne, table=True)
    fan = rt.Fan(w.fan, rt.RT_MIXED)
    outs = {}
    for st in (rt.RT_STENCIL_GATHER, rt.RT_STENCIL_QUAD, rt.RT_STENCIL_TABLE):
        for kern in (rt.RT_KERNEL_PLAIN, rt.RT_KERNEL_PERSISTENT):
            outs[(st, kern)] = rt.rt_trace(g, fan, cfg=rt.launch_config(kernel=kern, stencil=st))
    for v in outs.values():
        assert np.all(v["status"] != rt.RT_RAY_NOT_RUN)

    spec = w.fan.replace(rtol=1e-9)
    fp64 = rt.rt_trace(g, rt.Fan(spec, rt.RT_FP64))
    conv = rt.rt_trace(g, rt.Fan(w.fan.replace(rtol=1e-11, atol_km=1e-9), rt.RT_FP64))
    ok = ~near_boundary(fp64, spec)
    assert ok.mean() > 0.6
    keys = [(st, kern, 0) for st, kern in outs] + [
        (rt.RT_STENCIL_QUAD, rt.RT_KERNEL_PERSISTENT, 1), (rt.RT_STENCIL_QUAD, rt.RT_KERNEL_PERSISTENT, 4),
        (rt.RT_STENCIL_TABLE, rt.RT_KERNEL_PLAIN, 2), (rt.RT_STENCIL_GATHER, rt.RT_KERNEL_PLAIN, 4)]
    variants = {k: rt.rt_trace(g, rt.Fan(spec, rt.RT_MIXED),
                               cfg=rt.launch_config(kernel=k[1], stencil=k[0], lanes_per_ray=k[2]))
                for k in keys}
    mixed = variants[(rt.RT_STENCIL_QUAD, rt.RT_KERNEL_PERSISTENT, 0)]
    for key, mv in variants.items():
        same = (mv["status"] == fp64["status"]) & (conv["status"] == fp64["status"])
        assert same[ok].mean() > 0.999, key
        m = ok & same
        for ref in (fp64, conv):
            for f, tol in (("group_path_km", MIX_KM), ("ground_range_km", MIX_KM), ("az_dev_deg", MIX_DEG)):
                d = np.abs(mv[f] - ref[f])[m]
                assert np.all(d <= tol), (key, f, d.max())
    m = ok & (mixed["status"] == fp64["status"])
    idx = wl.sample_indices(w.fan.n_rays, 48, seed=22)
    idx = idx[m[idx]]
    ref = orc.trace_fan(orc.Grid(w.grid, w.ne), spec, indices=idx)
    _close64(mixed[idx], ref, km=MIX_KM, deg=MIX_DEG)
    _close64(fp64[idx], ref)


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
        ok = ~near_boundary(ref9, spec9)
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
    ref = orc.trace_fan(orc.Grid(w.grid, w.ne, interp=interp), spec)
    ok = ~near_boundary(ref, spec)
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
        ok = ~near_boundary(ref, sp) if len(sp.el_deg) > 1 else np.ones(f.n_rays, bool)
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
    ok = ~near_boundary(ref_r, spec)
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


def test_config4_batched_fan_in_captured_graph(orc):
    """The ionogram-synthesis batch at full size: 181x361x301 grid, 281
    frequencies x 881 elevations x O/X = 495,122 rays of 50-5000 steps, run as
    one plan captured in a CUDA graph (mixed; plain and persistent kernel) and
    by the FP64 kernel; sampled rays against the oracle."""
    torch = pytest.importorskip("torch")
    w = wl.config4()
    assert w.fan.n_rays == 495122
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
    assert steps.min() < 100 and steps.max() > 1000  # uneven ray lengths
    fp64 = rt.rt_trace(g, rt.Fan(w.fan, rt.RT_FP64))
    idx = wl.sample_indices(n, 24, seed=44)
    ref = orc.trace_fan(orc.Grid(w.grid, w.ne), w.fan, indices=idx)
    _close64(fp64[idx], ref)
    ok = ~near_boundary(fp64, w.fan)[idx] & (mixed["status"][idx] == ref["status"])
    _close64(mixed[idx][ok], ref[ok], km=MIX_KM, deg=MIX_DEG)
    plan.close()
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
    # The two kernels run the same per-ray arithmetic, but their instantiations
    # may contract a few multiply-adds differently; at this batch's rtol 1e-7 a
    # handful of sensitive rays turn such last-bit differences into different
    # step sequences.  Nearly every ray must agree within the mixed tolerance.
    well = ~near_boundary(mixed, w.fan) & (pers["status"] == mixed["status"])
    assert well.sum() > 0.9 * n and (pers["status"] != mixed["status"]).sum() < 0.001 * n
    close = np.ones(n, bool)
    for f, tol in (("group_path_km", MIX_KM), ("ground_range_km", MIX_KM), ("az_dev_deg", MIX_DEG)):
        close &= np.abs(pers[f] - mixed[f]) <= tol
    assert close[well].mean() > 0.999, (close[well].mean(), int((~close[well]).sum()))
    pplan.close()


def test_config4_inputs_at_the_precision_forms_tolerance(orc):
    """The batch's inputs (181x361x301 grid, day/night gradient) traced at
    rtol 1e-8, the tolerance of the precision form: the mixed path meets its
    bar (0.05 km, 1e-4 deg) against the oracle on sampled rays away from skip
    and Pedersen boundaries.  (At the batch's own rtol 1e-7 the two differ by
    the integrator's truncation error instead.)"""
    w = wl.config4(rtol=1e-8)
    g = rt.Grid(w.grid, w.ne)
    mixed = rt.rt_trace(g, rt.Fan(w.fan, rt.RT_MIXED))
    idx = wl.sample_indices(w.fan.n_rays, 300, seed=48)
    ref = orc.trace_fan(orc.Grid(w.grid, w.ne), w.fan, indices=idx)
    ok = ~near_boundary(mixed, w.fan)[idx] & (mixed["status"][idx] == ref["status"])
    assert ok.sum() > 250
    _close64(mixed[idx][ok], ref[ok], km=MIX_KM, deg=MIX_DEG)
