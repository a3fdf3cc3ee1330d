"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/dem.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "dem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(dem_[a-z_]+)\s*\(", src))


def test_library_builds_and_exports_header_symbols():
    from paper_2501_05300_gb300 import buildlib, dem
    path = buildlib.build()
    assert os.path.exists(path)
    names = declared()
    assert {"dem_create_bed", "dem_step", "dem_apply_plate_velocity", "dem_read_forces",
            "dem_read_state", "dem_destroy_bed"} <= names
    lib = ctypes.CDLL(path)
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(dem.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dem_[a-z_]+)", out))
    assert names <= exported


def test_binding_loads_without_gpu():
    from paper_2501_05300_gb300 import dem
    lib = dem.load()
    assert lib.dem_last_error() == b""
    # a NULL descriptor is rejected on the host, before any CUDA call
    h = ctypes.c_void_p()
    st = lib.dem_create_bed(None, None, ctypes.byref(h))
    assert st == dem.DEM_ERR_ARG
    assert b"desc" in lib.dem_last_error()
    assert lib.dem_step(None, 1) == dem.DEM_ERR_ARG
    assert lib.dem_destroy_bed(None) == dem.DEM_OK


@pytest.mark.parametrize("name", ["dem_geom", "dem_bed_desc", "dem_info"])
def test_struct_layouts_match_the_binding(name, tmp_path):
    """Every field of the header's structs sits at the offset the ctypes
    binding uses, and the sizes agree (a C program compiled against
    include/dem.h prints them)."""
    from paper_2501_05300_gb300 import dem
    cls = getattr(dem, name)
    fields = [f[0] for f in cls._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dem.h"', "int main(void) {",
             f'  printf("size %zu\\n", sizeof({name}));']
    lines += [f'  printf("{f} %zu\\n", offsetof({name}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(cls), name
    for f in fields:
        assert int(out[f]) == getattr(cls, f).offset, (name, f)
