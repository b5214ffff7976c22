"""The C-ABI library: builds, loads, exports every symbol include/rtgd.h
declares, and its ctypes mirror has the header's struct layouts.  No compute
call is made here (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2506_18579_gb300 import build as rtbuild
from paper_2506_18579_gb300 import rtgd as rt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtgd.h")


@pytest.fixture(scope="module")
def lib():
    rtbuild.build()
    return rt.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:rt_err|size_t|int32_t|const char \*)\s*(rt_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(lib):
    decl = _declared_functions()
    assert len(decl) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", rt.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rt_\w+)$", out, re.M))
    missing = [d for d in decl if d not in exported]
    assert not missing, missing
    assert set(decl) == set(rt.EXPORTED)
    for name in decl:
        assert hasattr(lib, name)


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "probe.c"
    src.write_text('''
#include <stdio.h>
#include <stddef.h>
#include "rtgd.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(rt_grid_desc), sizeof(rt_fan_desc), sizeof(rt_ray_result),
         sizeof(rt_launch_config), sizeof(rt_dipole));
  printf("%zu %zu %zu %zu\\n", offsetof(rt_grid_desc, field), offsetof(rt_grid_desc, flags),
         offsetof(rt_fan_desc, n_freq), offsetof(rt_fan_desc, max_group_path_km));
  printf("%zu %zu\\n", offsetof(rt_ray_result, status), offsetof(rt_ray_result, n_attempts));
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[:5] == [ctypes.sizeof(rt.rt_grid_desc), ctypes.sizeof(rt.rt_fan_desc), rt.RESULT_DTYPE.itemsize,
                        ctypes.sizeof(rt.rt_launch_config), ctypes.sizeof(rt.rt_dipole)]
    assert vals[5:9] == [rt.rt_grid_desc.field.offset, rt.rt_grid_desc.flags.offset,
                         rt.rt_fan_desc.n_freq.offset, rt.rt_fan_desc.max_group_path_km.offset]
    assert vals[9:] == [rt.RESULT_DTYPE.fields["status"][1], rt.RESULT_DTYPE.fields["n_attempts"][1]]
    assert vals[2] == 64


def test_every_struct_size_and_field_offset_matches(tmp_path):
    """Every ctypes mirror of a header struct: size and each field's offset."""
    mirrors = {"rt_dipole": rt.rt_dipole, "rt_grid_desc": rt.rt_grid_desc, "rt_fan_desc": rt.rt_fan_desc,
               "rt_launch_config": rt.rt_launch_config, "rt_ionogram_desc": rt.rt_ionogram_desc,
               "rt_server_config": rt.rt_server_config, "rt_request_stats": rt.rt_request_stats,
               "rt_peaks": rt.rt_peaks}
    lines = []
    for name, cls in mirrors.items():
        lines.append('  printf("%%zu\\n", sizeof(%s));' % name)
        for fname, _ in cls._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (name, fname))
    for dt_name, dt, cname in (("RESULT", rt.RESULT_DTYPE, "rt_ray_result"),
                               ("IONO", rt.IONOGRAM_DTYPE, "rt_ionogram_point")):
        lines.append('  printf("%%zu\\n", sizeof(%s));' % cname)
        for fname in dt.names:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cname, fname))
    src = tmp_path / "probe_all.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"rtgd.h\"\nint main(void) {\n" +
                   "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "probe_all"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    vals = iter(int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split())
    for name, cls in mirrors.items():
        assert next(vals) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert next(vals) == getattr(cls, fname).offset, (name, fname)
    for dt in (rt.RESULT_DTYPE, rt.IONOGRAM_DTYPE):
        assert next(vals) == dt.itemsize
        for fname in dt.names:
            assert next(vals) == dt.fields[fname][1], fname


def test_version_and_fan_size(lib):
    from paper_2506_18579_gb300 import workloads as wl
    assert rt.rt_version() == 2
    w = wl.config2(elev_step=1.0, az_step=30.0)
    fan = rt.Fan(w.fan)
    assert fan.n_rays == w.fan.n_rays == 3 * 2 * 58 * 12
    bad = rt.Fan(w.fan)
    bad.desc.n_el = 0
    assert rt.rt_fan_size(bad.desc) == 0
    bad = rt.Fan(w.fan)
    bad.desc.modes = 4
    assert rt.rt_fan_size(bad.desc) == 0


def test_no_gpu_means_unsupported_not_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_18579_gb300 import workloads as wl
    w = wl.config1()
    with pytest.raises(rt.RtError) as ei:
        rt.Grid(w.grid, w.ne)
    assert ei.value.code == rt.RT_EUNSUPPORTED


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(rt, "_lib", None)
    with pytest.raises(rt.RtError):
        rt.load(str(tmp_path / "nope.so"))
