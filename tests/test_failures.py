"""Host-side failure paths, none of which faults, traps or hangs a GPU.

- A blocking trace whose bounded wait expires returns RT_ETIMEOUT, leaves the
  caller's host buffer untouched (and unwritten afterwards), and the library
  stays usable: the work it queued finishes on the stream.
- The request server admits by device memory: with a reserve as large as the
  device only one request runs at a time (each still equal to its solo
  trace); a request that does not fit even on an idle device (a budget
  function reporting little free memory stands in for a full device) is
  refused with RT_ENOMEM while the requests behind it are served.
"""
import os
import time

import numpy as np
import pytest

from paper_2506_18579_gb300 import build as rtbuild
from paper_2506_18579_gb300 import rtgd as rt
from paper_2506_18579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    rtbuild.build()
    return rt.load()


def test_timeout_returns_etimeout_and_leaves_the_host_buffer_alone(monkeypatch):
    torch = pytest.importorskip("torch")
    w = wl.config2()  # 24,840 rays: well over 10 ms on the GPU
    g = rt.Grid(w.grid, w.ne)
    fan = rt.Fan(w.fan, rt.RT_MIXED)
    n = fan.n_rays
    out = np.full(n, 0, dtype=rt.RESULT_DTYPE)
    out["status"] = -7  # sentinel: no record has this status
    out["group_path_km"] = -1.0
    monkeypatch.setenv("RTGD_SYNC_TIMEOUT_S", "1e-4")
    with pytest.raises(rt.RtError) as ei:
        rt.rt_trace(g, fan, out=out)
    assert ei.value.code == rt.RT_ETIMEOUT
    assert "did not finish" in rt.rt_last_error()
    torch.cuda.synchronize()  # the queued trace runs to its end on the stream ...
    time.sleep(0.05)
    assert np.all(out["status"] == -7) and np.all(out["group_path_km"] == -1.0)  # ... without writing out_host
    monkeypatch.delenv("RTGD_SYNC_TIMEOUT_S")
    res = rt.rt_trace(g, fan, out=out)  # the library and the stream are still usable
    assert np.all(res["status"] != rt.RT_RAY_NOT_RUN)
    g.close()


def _requests():
    w = wl.config2(elev_step=6.0, az_step=60.0)
    specs = [w.fan.replace(freq_mhz=[f], el_deg=np.linspace(5.0, 55.0, 7 + k), az_deg=[15.0 * k],
                           precision=wl.MIXED)
             for k, f in enumerate((8.0, 9.5, 11.0, 12.5, 14.0, 15.5))]
    return w, specs


def test_memory_reserve_serialises_requests_with_solo_results():
    w, specs = _requests()
    g = rt.Grid(w.grid, w.ne)
    cfg = rt.launch_config(kernel=rt.RT_KERNEL_PLAIN, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=4)
    solo = [rt.rt_trace(g, rt.Fan(s), cfg=cfg) for s in specs]
    torch = pytest.importorskip("torch")
    total = torch.cuda.mem_get_info()[1]
    # a reserve of the whole device: no request fits beside another one, so
    # the server admits the next only once nothing runs
    srv = rt.Server(max_inflight=4, cfg=cfg, mem_reserve_bytes=total)
    fans = [rt.Fan(s) for s in specs]
    t_sub, tickets = [], []
    for f in fans:
        t_sub.append(time.perf_counter())
        tickets.append(srv.submit(g, f))
    spans = []
    for k, (t, out) in enumerate(tickets):
        st = srv.wait(t, timeout_s=300.0)
        assert st.status == rt.RT_OK and st.batch_size == 1
        assert out.tobytes() == solo[k].tobytes(), k
        spans.append((t_sub[k] + st.queue_s, t_sub[k] + st.queue_s + st.run_s))
    srv.close()
    spans.sort()
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1 - 1e-4, (a0, a1, b0, b1)  # one request on the device at a time
    g.close()


def test_request_beyond_free_memory_is_refused_with_enomem():
    w, specs = _requests()
    g = rt.Grid(w.grid, w.ne)
    cfg = rt.launch_config(kernel=rt.RT_KERNEL_PLAIN, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=4)
    small = specs[:3]
    big = w.fan.replace(freq_mhz=[10.0], el_deg=np.linspace(5.0, 55.0, 400), az_deg=np.arange(0.0, 360.0, 10.0),
                        precision=wl.MIXED)  # 28,800 rays: 3.7 MB of records, twice counted
    asked = []

    def budget():  # a device with 1 MiB free: enough for the small requests only
        asked.append(1)
        return 1 << 20

    solo = [rt.rt_trace(g, rt.Fan(s), cfg=cfg) for s in small]
    srv = rt.Server(max_inflight=2, cfg=cfg, free_bytes=budget)
    order = [small[0], big, small[1], small[2]]
    tickets = [srv.submit(g, rt.Fan(s)) for s in order]
    with pytest.raises(rt.RtError) as ei:
        srv.wait(tickets[1][0], timeout_s=300.0)
    assert ei.value.code == rt.RT_ENOMEM
    assert "device memory" in rt.rt_last_error()
    assert np.all(tickets[1][1]["status"] == rt.RT_RAY_NOT_RUN)  # never traced
    for k, s_i in ((0, 0), (2, 1), (3, 2)):
        st = srv.wait(tickets[k][0], timeout_s=300.0)
        assert st.status == rt.RT_OK
        assert tickets[k][1].tobytes() == solo[s_i].tobytes(), k
    srv.close()
    assert len(asked) >= 4  # admission asked the budget function, not cudaMemGetInfo
    g.close()
