"""ctypes wrapper of the FP64 CPU oracle (oracle/rtgd_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py.  The product path never imports this module.

Objects passed in are duck-typed: a grid spec with the fields of
``or_grid`` (n_lat, ..., pole_lon_deg), an Ne array of shape
(n_lat, n_lon, n_alt), and a fan spec with tx/freq/el/az/modes/integrator
fields.  Nothing here depends on the CUDA package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rtgd_oracle.cpp")
HDR = os.path.join(HERE, "rtgd_oracle.h")
LIB = os.path.join(HERE, "librtgd_oracle.so")

# Status codes (same meaning as the CUDA library's, numbered independently).
LANDED, ESCAPED, LEFT_GRID, MAX_STEPS, STEP_UNDERFLOW, NONFINITE, MAX_PATH = 1, 2, 3, 4, 5, 6, 7

COMPILE = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
           "-o", LIB, SRC]

_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle shared library if missing or older than its sources."""
    stale = (not os.path.exists(LIB) or
             os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
    if force or stale:
        subprocess.run(COMPILE, check=True)
    return LIB


class OrGrid(ctypes.Structure):
    _fields_ = [("n_lat", ctypes.c_int32), ("n_lon", ctypes.c_int32), ("n_alt", ctypes.c_int32),
                ("interp", ctypes.c_int32),
                ("lat0_deg", ctypes.c_double), ("lon0_deg", ctypes.c_double),
                ("alt0_km", ctypes.c_double), ("dlat_deg", ctypes.c_double),
                ("dlon_deg", ctypes.c_double), ("dalt_km", ctypes.c_double),
                ("earth_radius_km", ctypes.c_double), ("b0_tesla", ctypes.c_double),
                ("pole_lat_deg", ctypes.c_double), ("pole_lon_deg", ctypes.c_double),
                ("ne", ctypes.POINTER(ctypes.c_double))]


RAY_DTYPE = np.dtype([("tx_lat_deg", "f8"), ("tx_lon_deg", "f8"), ("tx_alt_km", "f8"),
                      ("freq_mhz", "f8"), ("el_deg", "f8"), ("az_deg", "f8"),
                      ("mode", "i4"), ("integrator", "i4"),
                      ("h_km", "f8"), ("rtol", "f8"), ("atol_km", "f8"), ("h_min_km", "f8"),
                      ("h_max_km", "f8"), ("max_steps", "i4"), ("pad0", "i4"),
                      ("max_group_path_km", "f8")])
assert RAY_DTYPE.itemsize == 112

RESULT_DTYPE = np.dtype([("group_path_km", "f8"), ("ground_range_km", "f8"),
                         ("az_dev_deg", "f8"), ("apogee_km", "f8"), ("land_lat_deg", "f8"),
                         ("land_lon_deg", "f8"), ("status", "i4"), ("n_steps", "i4"),
                         ("n_attempts", "i4"), ("pad0", "i4")])
assert RESULT_DTYPE.itemsize == 64

_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            G = ctypes.POINTER(OrGrid)
            vp = ctypes.c_void_p
            L.or_gd_psi.argtypes = [ctypes.c_double, _D, _D]
            L.or_cr_weights.argtypes = [ctypes.c_double, _D]
            L.or_ne.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
            L.or_ah.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32, _D]
            L.or_dipole.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
            L.or_hamiltonian.argtypes = [G, ctypes.c_double, ctypes.c_int32, _D, _D]
            L.or_rhs.argtypes = [G, ctypes.c_double, ctypes.c_int32, _D, _D]
            L.or_launch.argtypes = [G, vp, _D]
            L.or_launch.restype = ctypes.c_int32
            L.or_trace_ray.argtypes = [G, vp, vp, _D, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
            L.or_trace_many.argtypes = [G, vp, ctypes.c_int32, vp, ctypes.c_int32]
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(_D)


class Grid:
    """Holds an or_grid and keeps its FP64 sample array alive."""

    def __init__(self, spec, ne, interp="gd"):
        self.ne = np.ascontiguousarray(ne, dtype=np.float64)
        assert self.ne.shape == (spec.n_lat, spec.n_lon, spec.n_alt)
        self.spec = spec
        self.c = OrGrid(spec.n_lat, spec.n_lon, spec.n_alt, 1 if interp == "cr" else 0,
                        spec.lat0_deg, spec.lon0_deg, spec.alt0_km, spec.dlat_deg,
                        spec.dlon_deg, spec.dalt_km, spec.earth_radius_km, spec.b0_tesla,
                        spec.pole_lat_deg, spec.pole_lon_deg, _dptr(self.ne))

    @property
    def ref(self):
        return ctypes.byref(self.c)


def gd_psi(xi):
    v, d = ctypes.c_double(), ctypes.c_double()
    lib().or_gd_psi(float(xi), ctypes.byref(v), ctypes.byref(d))
    return v.value, d.value


def cr_weights(t):
    w = np.zeros(4)
    lib().or_cr_weights(float(t), _dptr(w))
    return w


def ne(grid: Grid, lat, lon, alt):
    """(Ne, dNe/dlat, dNe/dlon, dNe/dalt, inside) at one point."""
    out = np.zeros(5)
    lib().or_ne(grid.ref, float(lat), float(lon), float(alt), _dptr(out))
    return out


def ah(X, YL2, YT2, mode):
    """(mu^2, d/dX, d/dYL2, d/dYT2); mode +1 ordinary, -1 extraordinary."""
    out = np.zeros(4)
    lib().or_ah(float(X), float(YL2), float(YT2), int(mode), _dptr(out))
    return out


def dipole(grid: Grid, r, theta, phi):
    out = np.zeros(3)
    lib().or_dipole(grid.ref, float(r), float(theta), float(phi), _dptr(out))
    return out


def hamiltonian(grid: Grid, freq_mhz, mode, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(8)
    lib().or_hamiltonian(grid.ref, float(freq_mhz), int(mode), _dptr(y), _dptr(out))
    return out


def rhs(grid: Grid, freq_mhz, mode, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(6)
    lib().or_rhs(grid.ref, float(freq_mhz), int(mode), _dptr(y), _dptr(out))
    return out


def make_ray(fan, freq, mode, el, az):
    r = np.zeros(1, dtype=RAY_DTYPE)
    r["tx_lat_deg"], r["tx_lon_deg"], r["tx_alt_km"] = fan.tx_lat_deg, fan.tx_lon_deg, fan.tx_alt_km
    r["freq_mhz"], r["el_deg"], r["az_deg"], r["mode"] = freq, el, az, mode
    r["integrator"], r["h_km"], r["rtol"], r["atol_km"] = fan.integrator, fan.h_km, fan.rtol, fan.atol_km
    r["h_min_km"], r["h_max_km"], r["max_steps"] = fan.h_min_km, fan.h_max_km, fan.max_steps
    r["max_group_path_km"] = fan.max_group_path_km
    return r


def fan_rays(fan, indices=None):
    """Oracle ray records for a fan, in canonical order [freq][mode][el][az]
    (or only the given canonical indices)."""
    n_az, n_el, modes = len(fan.az_deg), len(fan.el_deg), fan.mode_list
    n = len(fan.freq_mhz) * len(modes) * n_el * n_az
    idx = np.arange(n) if indices is None else np.asarray(indices)
    a = idx % n_az
    e = (idx // n_az) % n_el
    m = (idx // (n_az * n_el)) % len(modes)
    f = idx // (n_az * n_el * len(modes))
    rays = np.zeros(len(idx), dtype=RAY_DTYPE)
    rays["tx_lat_deg"], rays["tx_lon_deg"], rays["tx_alt_km"] = fan.tx_lat_deg, fan.tx_lon_deg, fan.tx_alt_km
    rays["freq_mhz"] = fan.freq_mhz[f]
    rays["mode"] = np.asarray(modes, dtype=np.int32)[m]
    rays["el_deg"] = fan.el_deg[e]
    rays["az_deg"] = fan.az_deg[a]
    rays["integrator"], rays["h_km"], rays["rtol"], rays["atol_km"] = fan.integrator, fan.h_km, fan.rtol, fan.atol_km
    rays["h_min_km"], rays["h_max_km"], rays["max_steps"] = fan.h_min_km, fan.h_max_km, fan.max_steps
    rays["max_group_path_km"] = fan.max_group_path_km
    return rays


def trace_rays(grid: Grid, rays, n_threads=0):
    rays = np.ascontiguousarray(rays, dtype=RAY_DTYPE)
    res = np.zeros(len(rays), dtype=RESULT_DTYPE)
    if len(rays):
        lib().or_trace_many(grid.ref, rays.ctypes.data, len(rays), res.ctypes.data, int(n_threads))
    return res


def trace_fan(grid: Grid, fan, indices=None, n_threads=0):
    return trace_rays(grid, fan_rays(fan, indices), n_threads)


def ionogram_points(res, fan, d_rx):
    """Oblique-ionogram points (Sec. IV-B-4, read as in the C ABI's
    rt_ionogram): for each frequency and mode of a one-azimuth fan, wherever
    the ground ranges D of two neighbouring elevations that both landed lie
    on either side of the receiver distance d_rx, one point with P' and the
    elevation interpolated linearly in D; branches numbered 0, 1, ... by
    elevation within each trace.  res holds per-ray records in canonical
    order.  Returns (freq_mhz, group_path_km, el_deg, mode, branch) tuples."""
    pts = []
    n_el = len(fan.el_deg)
    modes = fan.mode_list
    r = np.asarray(res).reshape(len(fan.freq_mhz), len(modes), n_el)
    for fi, f in enumerate(fan.freq_mhz):
        for mi, m in enumerate(modes):
            row = r[fi, mi]
            br = 0
            for j in range(n_el - 1):
                a, b = row[j], row[j + 1]
                if a["status"] != LANDED or b["status"] != LANDED:
                    continue
                fa, fb = a["ground_range_km"] - d_rx, b["ground_range_km"] - d_rx
                if (fa < 0) != (fb < 0):
                    t = fa / (fa - fb)
                    pts.append((f, a["group_path_km"] + t * (b["group_path_km"] - a["group_path_km"]),
                                fan.el_deg[j] + t * (fan.el_deg[j + 1] - fan.el_deg[j]), m, br))
                    br += 1
    return pts


def trajectory(grid: Grid, ray, cap=200000):
    """(result, traj) for one ray; traj rows are (P', r, theta, phi, kr, kth, kph, H)."""
    ray = np.ascontiguousarray(ray, dtype=RAY_DTYPE).reshape(1)
    res = np.zeros(1, dtype=RESULT_DTYPE)
    traj = np.zeros((cap, 8))
    n = ctypes.c_int32(0)
    lib().or_trace_ray(grid.ref, ray.ctypes.data, res.ctypes.data, _dptr(traj), cap, ctypes.byref(n))
    return res[0], traj[: n.value]


def launch(grid: Grid, ray):
    ray = np.ascontiguousarray(ray, dtype=RAY_DTYPE).reshape(1)
    y0 = np.zeros(6)
    ok = lib().or_launch(grid.ref, ray.ctypes.data, _dptr(y0))
    return bool(ok), y0
