"""rt_trace_device_noalloc: tracing without any device allocation.

Some callers cannot allocate device memory while they trace (an allocator
that must not be re-entered, a fixed device memory budget, device memory
owned by another runtime).  For them rt_trace_device_noalloc keeps its scratch
(ray counter and fan tables) in a fixed array inside the library.  This test
calls it through the C ABI twice in a row and checks each result against the
allocating rt_trace_device, within the tolerances the parity tests use, in
both precisions; and that a fan too large for the fixed scratch is refused.
It lives in a file of its own, collected last, and passes alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_2506_18579_gb300 import build as rtbuild
from paper_2506_18579_gb300 import rtgd as rt
from paper_2506_18579_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {rt.RT_FP64: (1e-6, 1e-7), rt.RT_MIXED: (0.05, 1e-4)}


def _run(fn, grid, fan, torch, stream, cfg=None):
    n = fan.n_rays
    out = torch.full((n * 64,), 0xAB, dtype=torch.uint8, device="cuda")  # stale bytes to overwrite
    fn(grid, fan, out.data_ptr(), n, cfg=cfg, stream=stream.cuda_stream)
    stream.synchronize()
    return rt.results_view(out.cpu().numpy(), n).copy()


def test_noalloc_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    rtbuild.build()
    rt.load()
    w = wl.config2(elev_step=3.0, az_step=30.0)  # 3 x 2 x 20 x 12 = 1,440 rays
    grid = rt.Grid(w.grid, w.ne)
    stream = torch.cuda.current_stream()
    for prec in (rt.RT_MIXED, rt.RT_FP64):
        fan = rt.Fan(w.fan, prec)
        ref = _run(rt.rt_trace_device, grid, fan, torch, stream)
        km, deg = TOL[prec]
        for _ in range(2):  # two calls in a row share (and must reset) the scratch
            got = _run(rt.rt_trace_device_noalloc, grid, fan, torch, stream)
            assert np.array_equal(got["status"], ref["status"])
            assert np.all(got["status"] != rt.RT_RAY_NOT_RUN)
            for f in ("group_path_km", "ground_range_km", "apogee_km"):
                assert np.abs(got[f] - ref[f]).max() <= km, f
            assert np.abs(got["az_dev_deg"] - ref["az_dev_deg"]).max() <= deg


def test_noalloc_persistent_kernel_alternating_fans():
    """The persistent kernel claims rays from the ray counter that lives in
    the shared scratch, so every call must start it from zero; and two fans
    of different sizes and azimuths, alternated, must each find their own
    tables there.  Same kernel and launch configuration as the allocating
    call, so the records must be identical byte for byte."""
    torch = pytest.importorskip("torch")
    rtbuild.build()
    rt.load()
    w = wl.config2(elev_step=3.0, az_step=30.0)
    grid = rt.Grid(w.grid, w.ne)
    stream = torch.cuda.current_stream()
    fan_a = rt.Fan(w.fan, rt.RT_MIXED)  # 1,440 rays
    fan_b = rt.Fan(w.fan.replace(az_deg=w.fan.az_deg[::2] + 7.5, el_deg=np.linspace(4.0, 58.0, 31),
                                 freq_mhz=[9.0, 13.0]), rt.RT_MIXED)  # 744 rays
    for lanes in (1, 4):
        cfg = rt.launch_config(kernel=rt.RT_KERNEL_PERSISTENT, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=lanes)
        refs = [_run(rt.rt_trace_device, grid, f, torch, stream, cfg) for f in (fan_a, fan_b)]
        for _ in range(2):
            for f, ref in zip((fan_a, fan_b), refs):
                got = _run(rt.rt_trace_device_noalloc, grid, f, torch, stream, cfg)
                assert np.all(got["status"] != rt.RT_RAY_NOT_RUN)
                assert got.tobytes() == ref.tobytes(), (lanes, f.n_rays)


def test_noalloc_rejects_fans_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    rtbuild.build()
    w = wl.config1()
    grid = rt.Grid(w.grid, w.ne)
    fan = rt.Fan(w.fan.replace(el_deg=np.linspace(5.0, 50.0, 5000)))
    out = torch.empty(fan.n_rays * 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(rt.RtError) as ei:
        rt.rt_trace_device_noalloc(grid, fan, out.data_ptr(), fan.n_rays)
    assert ei.value.code == rt.RT_EINVAL
    assert "scratch" in rt.rt_last_error()
