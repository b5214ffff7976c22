"""The request server (continuous batching over resident grids).

Requests of uneven size against four resident grids are submitted together
and staggered; each result must equal the same request traced alone with the
same launch configuration (identical per-ray arithmetic, so byte-identical
records), and the latency statistics must be consistent.
"""
import time

import numpy as np
import pytest

from paper_2506_18579_gb300 import build as rtbuild
from paper_2506_18579_gb300 import rtgd as rt
from paper_2506_18579_gb300 import workloads as wl


def test_server_needs_a_gpu_or_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rtbuild.build()
    with pytest.raises(rt.RtError) as ei:
        rt.Server()
    assert ei.value.code == rt.RT_EUNSUPPORTED


def _requests(seed):
    rng = np.random.default_rng(seed)
    grids = wl.serving_grids()[:3]  # the largest (181x361x301) is exercised by the C4 test
    reqs = []
    for i in range(14):
        gi = int(rng.integers(len(grids)))
        n_el = int(np.exp(rng.uniform(np.log(1), np.log(120))))
        n_az = int(rng.integers(1, 8))
        f0 = rng.uniform(3.0, 20.0)
        spec = wl.FanSpec(tx_lat_deg=30.0 + rng.uniform(-3, 3), tx_lon_deg=112.0 + rng.uniform(-3, 3), tx_alt_km=0.0,
                          freq_mhz=[f0, f0 + 2.0], el_deg=np.linspace(3.0, 60.0, n_el),
                          az_deg=np.linspace(0.0, 300.0, n_az), modes=wl.MODE_O if i % 2 else wl.MODE_X,
                          integrator=wl.RKF45, rtol=1e-8, precision=wl.MIXED)
        reqs.append((gi, spec))
    return grids, reqs


@pytest.mark.gpu
def test_results_in_the_mix_equal_solo_results():
    rtbuild.build()
    grids, reqs = _requests(5)
    handles = [rt.Grid(g, ne) for g, ne in grids]
    cfg = rt.launch_config(kernel=rt.RT_KERNEL_PERSISTENT, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=1)
    solo = [rt.rt_trace(handles[gi], rt.Fan(spec), cfg=cfg) for gi, spec in reqs]
    srv = rt.Server(max_inflight=4, cfg=cfg)
    fans = [rt.Fan(spec) for _, spec in reqs]
    tickets = []
    for k, (gi, spec) in enumerate(reqs):  # half at once, half staggered while others run
        tickets.append(srv.submit(handles[gi], fans[k]))
        if k >= len(reqs) // 2:
            time.sleep(0.002)
    for k, (t, out) in enumerate(tickets):
        st = srv.wait(t, timeout_s=300.0)
        assert st.status == rt.RT_OK and st.n_rays == fans[k].n_rays
        assert st.total_s >= st.run_s > 0 and st.queue_s >= 0
        assert out.tobytes() == solo[k].tobytes(), k
    srv.close()


@pytest.mark.gpu
def test_unknown_ticket_and_invalid_fan():
    rtbuild.build()
    w = wl.config1()
    g = rt.Grid(w.grid, w.ne)
    srv = rt.Server(max_inflight=2)
    with pytest.raises(rt.RtError):
        srv.wait(12345)
    bad = rt.Fan(w.fan)
    bad.desc.n_el = 0
    with pytest.raises(rt.RtError):
        srv.submit(g, bad, out=np.zeros(16, dtype=rt.RESULT_DTYPE))
    t, out = srv.submit(g, rt.Fan(w.fan))
    assert srv.wait(t).status == rt.RT_OK
    assert np.all(out["status"] == rt.RT_RAY_LANDED)
    srv.close()


def test_request_stream_is_seeded_and_shaped():
    specs = [g for g, _ in (
        (wl.centred_grid(*wl.TX[:2], 21, 21, 61, 2.0, 2.0, 10.0), None),
        (wl.centred_grid(*wl.TX[:2], 181, 361, 301, 0.5, 0.5, 2.0), None))]
    a = wl.serving_requests(400, 9, specs)
    b = wl.serving_requests(400, 9, specs)
    assert [(g, f.n_rays, f.tx_lat_deg) for g, f in a] == [(g, f.n_rays, f.tx_lat_deg) for g, f in b]
    n = np.array([f.n_rays for _, f in a])
    assert n.min() >= 1 and n.max() <= wl.SERVING_MAX_RAYS
    assert np.median(n) < 2000 < n.mean()  # log-uniform: heavy tail of large requests
    assert {g for g, _ in a} == {0, 1}
    for g, f in a:
        assert f.mode_list in ([1], [-1]) and f.integrator == wl.RKF45 and f.precision == wl.MIXED
        assert 3.0 <= min(f.freq_mhz) and max(f.freq_mhz) <= 30.0
        assert 1.0 <= f.el_deg[0] <= f.el_deg[-1] <= 89.0
        gs = specs[g]
        assert abs(f.tx_lat_deg - (gs.lat0_deg + 0.5 * gs.dlat_deg * (gs.n_lat - 1))) <= 5.0
    shapes = {(len(f.az_deg) == 1) for _, f in a}
    assert shapes == {True, False}  # both ionogram-synthesis and OTHR-registration requests


@pytest.mark.gpu
@pytest.mark.parametrize("fuse", [0, 4096])
def test_many_small_requests_through_few_slots(fuse):
    """Hundreds of 1-3 ray requests through 3 slots: slots are reused while
    others run, so a request must never be reported finished before its own
    work is queued (each record must equal its solo trace).  With fusion the
    queued requests share launches: the records of each must still land in
    its own buffer, equal to the same request served alone."""
    rtbuild.build()
    w = wl.config1()
    g = rt.Grid(w.grid, w.ne)
    rng = np.random.default_rng(11)
    specs = []
    for i in range(240):
        k = int(rng.integers(1, 4))
        specs.append(w.fan.replace(el_deg=np.sort(rng.uniform(5.0, 50.0, k)), az_deg=[rng.uniform(0.0, 360.0)],
                                   integrator=wl.RKF45, rtol=1e-8, precision=wl.MIXED))
    cfg = rt.launch_config(kernel=rt.RT_KERNEL_PLAIN, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=0 if fuse else 1)
    fans = [rt.Fan(s) for s in specs]
    if fuse:
        solo = _served_one_at_a_time(rt.Server(max_inflight=3, cfg=cfg, fuse_max_rays=fuse), [(g, f) for f in fans])
    else:
        solo = [rt.rt_trace(g, rt.Fan(s), cfg=cfg) for s in specs]
    srv = rt.Server(max_inflight=3, cfg=cfg, fuse_max_rays=fuse)
    tickets = [srv.submit(g, f) for f in fans]
    batch = []
    for k, (t, out) in enumerate(tickets):
        st = srv.wait(t, timeout_s=300.0)
        assert st.status == rt.RT_OK
        assert out.tobytes() == solo[k].tobytes(), k
        batch.append(st.batch_size)
    srv.close()
    if fuse:
        assert max(batch) > 1  # submitted together, so most wait and share launches
    else:
        assert set(batch) == {1}


def _served_one_at_a_time(srv, items):
    """Records of each (grid, fan) served alone: submit, wait, next."""
    outs = []
    for h, fan in items:
        t, out = srv.submit(h, fan)
        st = srv.wait(t, timeout_s=300.0)
        assert st.status == rt.RT_OK and st.batch_size == 1
        outs.append(out.copy())
    srv.close()
    return outs


def _close_up_to_rounding(a, b):
    """Mixed-path records of two separately compiled kernels: float rounding
    moves a few sensitive rays, so most rays must agree to 0.05 km."""
    same = a["status"] == b["status"]
    assert same.mean() >= 0.97
    for f in ("group_path_km", "ground_range_km"):
        d = np.abs(a[f] - b[f])[same]
        assert np.mean(d <= 0.05) >= 0.97, (f, d.max())


@pytest.mark.gpu
def test_fused_launches_mix_grids_integrators_and_precisions():
    """A fusing server fed requests on three grids, RKF45 and RK4, mixed and
    FP64, submitted at once: launches fuse only requests of one grid, one
    integrator and the mixed path; every request's records equal those of the
    same request served alone (FP64: of rt_trace), and the mixed ones agree
    with rt_trace on the plain four-lane kernel up to float rounding."""
    rtbuild.build()
    grids, reqs = _requests(7)
    rng = np.random.default_rng(8)
    more = []
    for gi, spec in reqs:
        more.append((gi, spec))
        if rng.uniform() < 0.5:
            more.append((gi, spec.replace(integrator=wl.RK4, h_km=5.0)))
        if rng.uniform() < 0.2:
            more.append((gi, spec.replace(precision=wl.FP64)))
    handles = [rt.Grid(g, ne) for g, ne in grids]
    cfg = rt.launch_config(kernel=rt.RT_KERNEL_PLAIN, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=4)
    mixed = [k for k in range(len(more)) if more[k][1].precision == wl.MIXED]
    plain = {k: rt.rt_trace(handles[more[k][0]], rt.Fan(more[k][1]), cfg=cfg) for k in mixed}
    fans = [rt.Fan(spec) for _, spec in more]
    scfg = rt.launch_config(stencil=rt.RT_STENCIL_QUAD)
    alone = _served_one_at_a_time(rt.Server(max_inflight=2, cfg=scfg, fuse_max_rays=20000),
                                  [(handles[gi], fans[k]) for k, (gi, _) in enumerate(more)])
    srv = rt.Server(max_inflight=2, cfg=scfg, fuse_max_rays=20000)
    tickets = [srv.submit(handles[gi], fans[k]) for k, (gi, _) in enumerate(more)]
    sizes = []
    for k, (t, out) in enumerate(tickets):
        st = srv.wait(t, timeout_s=300.0)
        assert st.status == rt.RT_OK and st.n_rays == fans[k].n_rays
        assert out.tobytes() == alone[k].tobytes(), k
        sizes.append(st.batch_size)
        if more[k][1].precision == wl.FP64:  # never fused; the plain kernel as configured
            assert st.batch_size == 1
            assert out.tobytes() == rt.rt_trace(handles[more[k][0]], fans[k], cfg=scfg).tobytes(), k
    srv.close()
    assert max(sizes) > 1
    _close_up_to_rounding(np.concatenate([alone[k] for k in mixed]), np.concatenate([plain[k] for k in mixed]))


@pytest.mark.gpu
def test_fusion_needs_the_plain_one_lane_kernel():
    rtbuild.build()
    for cfg in (rt.launch_config(kernel=rt.RT_KERNEL_PERSISTENT), rt.launch_config(lanes_per_ray=1),
                rt.launch_config(lanes_per_ray=2)):
        with pytest.raises(rt.RtError) as ei:
            rt.Server(cfg=cfg, fuse_max_rays=1000)
        assert ei.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RtError):
        rt.Server(fuse_max_rays=-1)
