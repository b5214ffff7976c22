"""Thin ctypes binding of librtgd.so (the C ABI in include/rtgd.h).

Argument marshalling only: every step of the ray tracing runs in the CUDA
library.  Functions keep the C names; a few helpers convert the dataclasses
of ``workloads`` into the C descriptors and wrap results as numpy records.
There is no CPU fallback: if the library cannot be loaded, or no GPU is
present, calls raise ``RtError``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librtgd.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ETIMEOUT, RT_EUNSUPPORTED = range(6)
RT_F32, RT_F64 = 0, 1
RT_GRID_TABLE, RT_GRID_CATMULL_ROM = 1, 2
RT_MODE_O, RT_MODE_X = 1, 2
RT_RK4, RT_RKF45 = 0, 1
RT_FP64, RT_MIXED = 0, 1
(RT_RAY_NOT_RUN, RT_RAY_LANDED, RT_RAY_ESCAPED, RT_RAY_LEFT_GRID, RT_RAY_MAX_STEPS,
 RT_RAY_STEP_UNDERFLOW, RT_RAY_NONFINITE, RT_RAY_MAX_PATH) = range(8)
RT_KERNEL_AUTO, RT_KERNEL_PLAIN, RT_KERNEL_PERSISTENT = 0, 1, 2
RT_STENCIL_AUTO, RT_STENCIL_GATHER, RT_STENCIL_QUAD, RT_STENCIL_TABLE = 0, 1, 2, 3
RT_ORDER_CANONICAL, RT_ORDER_ELEVATION_FASTEST = 0, 1
RT_PLAN_REST_IN_PLAN_ORDER = 1
RT_PLAN_LONG_EXCLUSIVE = 2
RT_PLAN_LONG_ALONE = 4

EXPORTED = ["rt_grid_create", "rt_grid_destroy", "rt_grid_device_bytes", "rt_fan_size",
            "rt_trace", "rt_trace_device", "rt_trace_fans_device", "rt_tune", "rt_eval_rhs", "rt_last_error",
            "rt_version", "rt_plan_create", "rt_plan_rays", "rt_plan_execute", "rt_plan_destroy", "rt_plan_order",
            "rt_ionogram", "rt_trace_device_noalloc", "rt_server_create", "rt_server_submit",
            "rt_server_wait", "rt_server_destroy", "rt_measure_peaks", "rt_order_claims"]


class RtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("rtgd error %d: %s" % (code, msg))
        self.code = code


class rt_dipole(ctypes.Structure):
    _fields_ = [("b0_tesla", ctypes.c_double), ("pole_lat_deg", ctypes.c_double),
                ("pole_lon_deg", ctypes.c_double)]


class rt_grid_desc(ctypes.Structure):
    _fields_ = [("n_lat", ctypes.c_int32), ("n_lon", ctypes.c_int32), ("n_alt", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("lat0_deg", ctypes.c_double),
                ("lon0_deg", ctypes.c_double), ("alt0_km", ctypes.c_double),
                ("dlat_deg", ctypes.c_double), ("dlon_deg", ctypes.c_double),
                ("dalt_km", ctypes.c_double), ("earth_radius_km", ctypes.c_double),
                ("field", rt_dipole), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


_DP = ctypes.POINTER(ctypes.c_double)


class rt_fan_desc(ctypes.Structure):
    _fields_ = [("tx_lat_deg", ctypes.c_double), ("tx_lon_deg", ctypes.c_double),
                ("tx_alt_km", ctypes.c_double), ("freq_mhz", _DP), ("el_deg", _DP),
                ("az_deg", _DP), ("n_freq", ctypes.c_int32), ("n_el", ctypes.c_int32),
                ("n_az", ctypes.c_int32), ("modes", ctypes.c_uint32),
                ("integrator", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("h_km", ctypes.c_double), ("rtol", ctypes.c_double), ("atol_km", ctypes.c_double),
                ("h_min_km", ctypes.c_double), ("h_max_km", ctypes.c_double),
                ("max_steps", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_group_path_km", ctypes.c_double)]


class rt_launch_config(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("stencil", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("order", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("lanes_per_ray", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class rt_ionogram_desc(ctypes.Structure):
    _fields_ = [("tx_lat_deg", ctypes.c_double), ("tx_lon_deg", ctypes.c_double),
                ("tx_alt_km", ctypes.c_double), ("rx_lat_deg", ctypes.c_double),
                ("rx_lon_deg", ctypes.c_double), ("freq_mhz", ctypes.POINTER(ctypes.c_double)),
                ("el_deg", ctypes.POINTER(ctypes.c_double)), ("n_freq", ctypes.c_int32),
                ("n_el", ctypes.c_int32), ("modes", ctypes.c_uint32), ("integrator", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_steps", ctypes.c_int32), ("h_km", ctypes.c_double),
                ("rtol", ctypes.c_double), ("atol_km", ctypes.c_double), ("h_min_km", ctypes.c_double),
                ("h_max_km", ctypes.c_double)]


FREE_BYTES_FN = ctypes.CFUNCTYPE(ctypes.c_size_t, ctypes.c_void_p)


class rt_server_config(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int32), ("fuse_max_rays", ctypes.c_int32),
                ("mem_reserve_bytes", ctypes.c_size_t), ("launch", rt_launch_config),
                ("free_bytes", FREE_BYTES_FN), ("free_bytes_user", ctypes.c_void_p)]


class rt_request_stats(ctypes.Structure):
    _fields_ = [("queue_s", ctypes.c_double), ("run_s", ctypes.c_double), ("total_s", ctypes.c_double),
                ("n_rays", ctypes.c_int64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_int32)]


class rt_peaks(ctypes.Structure):
    _fields_ = [("fp32_fma_flops", ctypes.c_double), ("fp64_fma_flops", ctypes.c_double),
                ("l2_read_bytes_per_s", ctypes.c_double), ("sm_count", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("max_sm_mhz", ctypes.c_double)]


IONOGRAM_DTYPE = np.dtype([("freq_mhz", "f8"), ("group_path_km", "f8"), ("el_deg", "f8"),
                           ("ground_range_km", "f8"), ("mode", "i4"), ("branch", "i4")])
assert IONOGRAM_DTYPE.itemsize == 40

RESULT_DTYPE = np.dtype([("group_path_km", "f8"), ("ground_range_km", "f8"),
                         ("az_dev_deg", "f8"), ("apogee_km", "f8"), ("land_lat_deg", "f8"),
                         ("land_lon_deg", "f8"), ("status", "i4"), ("n_steps", "i4"),
                         ("n_attempts", "i4"), ("n_evals", "i4")])
assert RESULT_DTYPE.itemsize == 64

_lib = None


def load(path=None):
    """Load librtgd.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RtError(RT_EUNSUPPORTED, "CUDA library %s is not built (run build.build())" % path)
    L = ctypes.CDLL(path)
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    L.rt_grid_create.argtypes = [ctypes.POINTER(rt_grid_desc), vp, ctypes.POINTER(vp)]
    L.rt_grid_create.restype = ctypes.c_int
    L.rt_grid_destroy.argtypes = [vp]
    L.rt_grid_destroy.restype = ctypes.c_int
    L.rt_grid_device_bytes.argtypes = [vp]
    L.rt_grid_device_bytes.restype = sz
    L.rt_fan_size.argtypes = [ctypes.POINTER(rt_fan_desc)]
    L.rt_fan_size.restype = sz
    L.rt_trace.argtypes = [vp, ctypes.POINTER(rt_fan_desc), vp, sz, ctypes.POINTER(rt_launch_config), vp]
    L.rt_trace.restype = ctypes.c_int
    L.rt_trace_device.argtypes = [vp, ctypes.POINTER(rt_fan_desc), vp, sz,
                                  ctypes.POINTER(rt_launch_config), vp]
    L.rt_trace_device.restype = ctypes.c_int
    L.rt_trace_fans_device.argtypes = [vp, ctypes.POINTER(ctypes.POINTER(rt_fan_desc)), ctypes.c_int32, vp, sz,
                                       ctypes.POINTER(rt_launch_config), vp]
    L.rt_trace_fans_device.restype = ctypes.c_int
    L.rt_trace_device_noalloc.argtypes = [vp, ctypes.POINTER(rt_fan_desc), vp, sz,
                                          ctypes.POINTER(rt_launch_config), vp]
    L.rt_trace_device_noalloc.restype = ctypes.c_int
    L.rt_tune.argtypes = [vp, ctypes.POINTER(rt_fan_desc), sz, vp, ctypes.POINTER(rt_launch_config),
                          ctypes.POINTER(ctypes.c_float)]
    L.rt_tune.restype = ctypes.c_int
    L.rt_eval_rhs.argtypes = [vp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                              _DP, _DP, _DP, sz]
    L.rt_eval_rhs.restype = ctypes.c_int
    L.rt_plan_create.argtypes = [vp, ctypes.POINTER(rt_fan_desc), ctypes.POINTER(rt_launch_config),
                                 ctypes.POINTER(vp)]
    L.rt_plan_create.restype = ctypes.c_int
    L.rt_plan_rays.argtypes = [vp]
    L.rt_plan_rays.restype = sz
    L.rt_plan_execute.argtypes = [vp, vp, sz, vp]
    L.rt_plan_execute.restype = ctypes.c_int
    L.rt_plan_destroy.argtypes = [vp]
    L.rt_plan_destroy.restype = ctypes.c_int
    L.rt_plan_order.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_double, ctypes.c_uint32, ctypes.POINTER(sz), vp]
    L.rt_plan_order.restype = ctypes.c_int
    i32 = ctypes.c_int32
    L.rt_order_claims.argtypes = [vp, i32, i32, i32, i32, i32, i32, ctypes.c_double, i32, ctypes.c_uint32, i32,
                                  vp, sz, ctypes.POINTER(sz), ctypes.POINTER(sz)]
    L.rt_order_claims.restype = ctypes.c_int
    L.rt_ionogram.argtypes = [vp, ctypes.POINTER(rt_ionogram_desc), vp, sz, ctypes.POINTER(sz),
                              ctypes.POINTER(rt_launch_config), vp]
    L.rt_ionogram.restype = ctypes.c_int
    L.rt_server_create.argtypes = [ctypes.POINTER(rt_server_config), ctypes.POINTER(vp)]
    L.rt_server_create.restype = ctypes.c_int
    L.rt_server_submit.argtypes = [vp, vp, ctypes.POINTER(rt_fan_desc), vp, sz, ctypes.POINTER(ctypes.c_uint64)]
    L.rt_server_submit.restype = ctypes.c_int
    L.rt_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(rt_request_stats)]
    L.rt_server_wait.restype = ctypes.c_int
    L.rt_server_destroy.argtypes = [vp]
    L.rt_server_destroy.restype = ctypes.c_int
    L.rt_measure_peaks.argtypes = [ctypes.POINTER(rt_peaks)]
    L.rt_measure_peaks.restype = ctypes.c_int
    L.rt_last_error.argtypes = []
    L.rt_last_error.restype = ctypes.c_char_p
    L.rt_version.argtypes = []
    L.rt_version.restype = ctypes.c_int32
    _lib = L
    return L


def _check(code):
    if code != RT_OK:
        raise RtError(code, load().rt_last_error().decode())


def rt_last_error():
    return load().rt_last_error().decode()


def rt_version():
    return load().rt_version()


# ------------------------------------------------------------------ grids
def grid_desc(spec, dtype=RT_F32, table=False, interp="gd"):
    flags = (RT_GRID_TABLE if table else 0) | (RT_GRID_CATMULL_ROM if interp == "cr" else 0)
    return rt_grid_desc(spec.n_lat, spec.n_lon, spec.n_alt, dtype, spec.lat0_deg, spec.lon0_deg,
                        spec.alt0_km, spec.dlat_deg, spec.dlon_deg, spec.dalt_km,
                        spec.earth_radius_km,
                        rt_dipole(spec.b0_tesla, spec.pole_lat_deg, spec.pole_lon_deg), flags, 0)


class Grid:
    """Device-resident grid handle (rt_grid_create / rt_grid_destroy)."""

    def __init__(self, spec, ne, table=False, interp="gd"):
        ne = np.ascontiguousarray(ne)
        if ne.dtype not in (np.float32, np.float64):
            ne = ne.astype(np.float32)
        assert ne.shape == (spec.n_lat, spec.n_lon, spec.n_alt)
        self.spec = spec
        self.desc = grid_desc(spec, RT_F64 if ne.dtype == np.float64 else RT_F32, table, interp)
        self.handle = rt_grid_create(self.desc, ne)

    @property
    def device_bytes(self):
        return load().rt_grid_device_bytes(self.handle)

    def close(self):
        if self.handle:
            rt_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rt_grid_create(desc, ne_host):
    h = ctypes.c_void_p()
    _check(load().rt_grid_create(ctypes.byref(desc), ne_host.ctypes.data, ctypes.byref(h)))
    return h


def rt_grid_destroy(handle):
    _check(load().rt_grid_destroy(handle))


# ------------------------------------------------------------------- fans
class Fan:
    """rt_fan_desc plus the arrays it points to (kept alive)."""

    def __init__(self, spec, precision=None):
        self.spec = spec
        self.freq = np.ascontiguousarray(spec.freq_mhz, dtype=np.float64)
        self.el = np.ascontiguousarray(spec.el_deg, dtype=np.float64)
        self.az = np.ascontiguousarray(spec.az_deg, dtype=np.float64)
        prec = spec.precision if precision is None else precision
        self.desc = rt_fan_desc(
            spec.tx_lat_deg, spec.tx_lon_deg, spec.tx_alt_km, self.freq.ctypes.data_as(_DP),
            self.el.ctypes.data_as(_DP), self.az.ctypes.data_as(_DP), len(self.freq), len(self.el),
            len(self.az), spec.modes, spec.integrator, prec, spec.h_km, spec.rtol, spec.atol_km,
            spec.h_min_km, spec.h_max_km, spec.max_steps, 0, spec.max_group_path_km)

    @property
    def n_rays(self):
        return rt_fan_size(self.desc)

    @property
    def host_bytes(self):
        return self.freq.nbytes + self.el.nbytes + self.az.nbytes


def rt_fan_size(desc):
    return load().rt_fan_size(ctypes.byref(desc))


def launch_config(kernel=0, stencil=0, block_threads=0, order=0, blocks_per_sm=0, lanes_per_ray=0):
    return rt_launch_config(kernel, stencil, block_threads, order, blocks_per_sm, lanes_per_ray)


def _cfg_ptr(cfg):
    return ctypes.byref(cfg) if cfg is not None else None


def rt_trace(grid, fan, out=None, cfg=None, stream=None):
    """Blocking trace into a host numpy record array (allocated if out is None)."""
    n = fan.n_rays
    if out is None:
        out = np.zeros(n, dtype=RESULT_DTYPE)
    assert out.dtype == RESULT_DTYPE and out.flags.c_contiguous
    _check(load().rt_trace(grid.handle, ctypes.byref(fan.desc), out.ctypes.data, len(out),
                           _cfg_ptr(cfg), stream))
    return out


def rt_trace_device(grid, fan, out_ptr, out_len, cfg=None, stream=None):
    """Asynchronous trace into device memory (e.g. torch tensor .data_ptr())."""
    _check(load().rt_trace_device(grid.handle, ctypes.byref(fan.desc), ctypes.c_void_p(out_ptr),
                                  out_len, _cfg_ptr(cfg), stream))


def rt_trace_fans_device(grid, fans, out_ptr, out_len, cfg=None, stream=None):
    """Several fans (Fan objects) on one grid in one launch into device memory;
    records fan after fan."""
    arr = (ctypes.POINTER(rt_fan_desc) * max(len(fans), 1))(*[ctypes.pointer(f.desc) for f in fans])
    _check(load().rt_trace_fans_device(grid.handle, arr, len(fans), ctypes.c_void_p(out_ptr), out_len,
                                       _cfg_ptr(cfg), stream))


class Plan:
    """rt_plan: grid + fan + launch configuration bound once; execute() queues a
    counter reset and one kernel launch (capturable into a CUDA graph)."""

    def __init__(self, grid, fan, cfg=None):
        self.grid, self.fan = grid, fan  # keep both alive
        h = ctypes.c_void_p()
        _check(load().rt_plan_create(grid.handle, ctypes.byref(fan.desc), _cfg_ptr(cfg), ctypes.byref(h)))
        self.handle = h

    @property
    def n_rays(self):
        return load().rt_plan_rays(self.handle)

    def execute(self, out_ptr, out_len, stream=None):
        _check(load().rt_plan_execute(self.handle, ctypes.c_void_p(out_ptr), out_len, stream))

    def order(self, cost_ptr, spread=2, long_factor=0.0, rest_in_plan_order=False, long_exclusive=False,
              long_alone=False, stream=None):
        """rt_plan_order: longest-first order from device records at cost_ptr
        (None: back to the plan's own order); returns the number of rays
        traced at four lanes each.  long_exclusive: each block of those rays
        gets an SM of its own; long_alone: each of those rays a warp of its
        own."""
        n_long = ctypes.c_size_t()
        flags = ((RT_PLAN_REST_IN_PLAN_ORDER if rest_in_plan_order else 0) |
                 (RT_PLAN_LONG_EXCLUSIVE if long_exclusive else 0) |
                 (RT_PLAN_LONG_ALONE if long_alone else 0))
        _check(load().rt_plan_order(self.handle, None if cost_ptr is None else ctypes.c_void_p(cost_ptr),
                                    int(spread), float(long_factor), flags, ctypes.byref(n_long), stream))
        return n_long.value

    def close(self):
        if self.handle:
            _check(load().rt_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rt_order_claims(cost, dims, claim_order=RT_ORDER_ELEVATION_FASTEST, spread=2, long_factor=0.0, mixed=True,
                    rest_in_plan_order=False, long_exclusive=False, long_alone=False, sm_count=0):
    """rt_order_claims: the claim list of a longest-first order from host
    costs (canonical order, dims = (n_freq, n_modes, n_el, n_az)); returns
    (claims int32 array, -1 for holes; number of four-lane rays)."""
    cost = np.ascontiguousarray(cost, dtype=np.int32)
    n_f, n_m, n_e, n_a = (int(x) for x in dims)
    cap = cost.size + 7 * (cost.size // 16)
    claims = np.empty(max(cap, 1), dtype=np.int32)
    n_long, n_claims = ctypes.c_size_t(), ctypes.c_size_t()
    flags = ((RT_PLAN_REST_IN_PLAN_ORDER if rest_in_plan_order else 0) |
             (RT_PLAN_LONG_EXCLUSIVE if long_exclusive else 0) | (RT_PLAN_LONG_ALONE if long_alone else 0))
    _check(load().rt_order_claims(cost.ctypes.data, n_f, n_m, n_e, n_a, int(claim_order), int(spread),
                                  float(long_factor), int(bool(mixed)), flags, int(sm_count), claims.ctypes.data,
                                  claims.size, ctypes.byref(n_long), ctypes.byref(n_claims)))
    return claims[:n_claims.value].copy(), n_long.value


def rt_ionogram(grid, tx, rx, freq_mhz, el_deg, modes=RT_MODE_O | RT_MODE_X, integrator=RT_RKF45,
                precision=RT_MIXED, h_km=1.0, rtol=1e-8, atol_km=1e-6, h_min_km=1e-6, h_max_km=20.0,
                max_steps=200000, cap=None, cfg=None, stream=None):
    """Oblique ionogram points (IONOGRAM_DTYPE records) for a transmitter
    tx = (lat, lon, alt_km) and receiver rx = (lat, lon)."""
    freq = np.ascontiguousarray(freq_mhz, dtype=np.float64)
    el = np.ascontiguousarray(el_deg, dtype=np.float64)
    d = rt_ionogram_desc(tx[0], tx[1], tx[2], rx[0], rx[1], freq.ctypes.data_as(_DP), el.ctypes.data_as(_DP),
                         len(freq), len(el), modes, integrator, precision, max_steps, h_km, rtol, atol_km,
                         h_min_km, h_max_km)
    n_modes = (1 if modes & RT_MODE_O else 0) + (1 if modes & RT_MODE_X else 0)
    cap = cap if cap is not None else max(1, len(freq) * n_modes * max(len(el) - 1, 0))
    out = np.zeros(cap, dtype=IONOGRAM_DTYPE)
    n = ctypes.c_size_t()
    _check(load().rt_ionogram(grid.handle, ctypes.byref(d), out.ctypes.data, cap, ctypes.byref(n),
                              _cfg_ptr(cfg), stream))
    return out[: min(n.value, cap)], n.value


def rt_trace_device_noalloc(grid, fan, out_ptr, out_len, cfg=None, stream=None):
    """rt_trace_device without any device allocation (fixed in-library scratch)."""
    _check(load().rt_trace_device_noalloc(grid.handle, ctypes.byref(fan.desc), ctypes.c_void_p(out_ptr),
                                          out_len, _cfg_ptr(cfg), stream))


class Server:
    """rt_server: continuous-batching request server on the current device."""

    def __init__(self, max_inflight=8, mem_reserve_bytes=0, cfg=None, fuse_max_rays=0, free_bytes=None):
        """free_bytes: optional Python callable returning the device memory
        (bytes) admission may use, asked from the server's dispatcher thread
        instead of cudaMemGetInfo."""
        self._free_fn = FREE_BYTES_FN(lambda _user: int(free_bytes())) if free_bytes is not None \
            else FREE_BYTES_FN()
        c = rt_server_config(max_inflight, fuse_max_rays, mem_reserve_bytes,
                             cfg if cfg is not None else rt_launch_config(), self._free_fn, None)
        h = ctypes.c_void_p()
        _check(load().rt_server_create(ctypes.byref(c), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, grid, fan, out=None):
        """Queue a fan; returns (ticket, out) where out receives the records."""
        n = fan.n_rays
        out = np.zeros(n, dtype=RESULT_DTYPE) if out is None else out
        t = ctypes.c_uint64()
        _check(load().rt_server_submit(self.handle, grid.handle, ctypes.byref(fan.desc), out.ctypes.data, len(out),
                                       ctypes.byref(t)))
        self._keep[t.value] = (grid, fan, out)
        return t.value, out

    def wait(self, ticket, timeout_s=0.0):
        st = rt_request_stats()
        code = load().rt_server_wait(self.handle, ticket, timeout_s, ctypes.byref(st))
        if code != RT_ETIMEOUT:
            self._keep.pop(ticket, None)
        _check(code)
        return st

    def close(self):
        if self.handle:
            _check(load().rt_server_destroy(self.handle))
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rt_measure_peaks():
    """This GPU's FP32/FP64 FMA flop/s and L2 read bytes/s (rt_peaks)."""
    p = rt_peaks()
    _check(load().rt_measure_peaks(ctypes.byref(p)))
    return {"fp32_fma_tflops": p.fp32_fma_flops / 1e12, "fp64_fma_tflops": p.fp64_fma_flops / 1e12,
            "l2_read_gbs": p.l2_read_bytes_per_s / 1e9, "sm_count": p.sm_count, "max_sm_mhz": p.max_sm_mhz}


def rt_tune(grid, fan, max_rays=0, stream=None):
    best = rt_launch_config()
    ms = ctypes.c_float()
    _check(load().rt_tune(grid.handle, ctypes.byref(fan.desc), max_rays, stream, ctypes.byref(best),
                          ctypes.byref(ms)))
    return best, ms.value


def rt_eval_rhs(grid, freq_mhz, mode, y, precision=RT_FP64, stencil=RT_STENCIL_AUTO):
    y = np.ascontiguousarray(np.atleast_2d(y), dtype=np.float64)
    n = len(y)
    dy = np.zeros((n, 6))
    mu2 = np.zeros(n)
    _check(load().rt_eval_rhs(grid.handle, float(freq_mhz), int(mode), int(precision), int(stencil),
                              y.ctypes.data_as(_DP), dy.ctypes.data_as(_DP), mu2.ctypes.data_as(_DP),
                              n))
    return dy, mu2


def results_view(tensor_or_array, n):
    """Record view of n results held in a uint8/int64 host buffer."""
    a = np.asarray(tensor_or_array).view(np.uint8)[: n * 64]
    return a.view(RESULT_DTYPE)
