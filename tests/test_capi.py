"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point (CPU only)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(dem_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
@pytest.mark.parametrize("checks", [False, True])
def test_library_builds_loads_and_exports_every_declared_symbol(checks):
    # the plain library and its bounds-checked build export the same entry points
    from paper_1705_03850_gb300 import build
    path = build.build(checks=checks)
    assert path == (build.LIB_CHECKED if checks else build.LIB)
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert "dem_create" in declared and "dem_step" in declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_checked_library_is_selected_by_the_environment(monkeypatch):
    from paper_1705_03850_gb300 import build, dem
    monkeypatch.setenv("CGDEM_CHECKED", "1")
    assert dem.lib_path() == build.LIB_CHECKED
    monkeypatch.setenv("CGDEM_CHECKED", "0")
    assert dem.lib_path() == build.LIB
    monkeypatch.delenv("CGDEM_CHECKED")
    assert dem.lib_path() == build.LIB


def test_every_status_code_has_a_name():
    # each dem_status enumerator in the header is named in the binding's table
    from paper_1705_03850_gb300 import dem
    src = open(os.path.join(ROOT, "include", "dem.h")).read()
    codes = {int(v): k for k, v in re.findall(r"\b(DEM_(?:OK|ERR_\w+))\s*=\s*(\d+)", src)}
    assert codes and codes == dem.STATUS


def test_binding_lists_every_declared_symbol():
    from paper_1705_03850_gb300 import dem
    assert _declared() <= set(dem.exported_symbols())


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layout_matches_header(tmp_path):
    # the ctypes mirrors must agree with the C compiler's layout of include/dem.h
    import subprocess
    from paper_1705_03850_gb300 import dem
    structs = {"dem_instance_desc": dem.InstanceDesc, "dem_config": dem.Config,
               "dem_instance_info": dem.InstanceInfo, "dem_stats_t": dem.Stats, "dem_coupling": dem.CouplingSpec}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dem.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_header_compiles_as_cpp_with_c_linkage(tmp_path):
    # the boundary is usable from C++ callers: the header compiles there and its entry points
    # keep C linkage (unmangled names)
    import subprocess
    src = tmp_path / "use.cpp"
    src.write_text('#include "dem.h"\ndem_status (*volatile p)(dem_ctx*, int64_t) = &dem_step;\n'
                   'int main() { return p == nullptr; }\n')
    obj = tmp_path / "use.o"
    subprocess.check_call(["g++", "-std=c++17", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c",
                           str(src), "-o", str(obj)])
    syms = subprocess.check_output(["nm", str(obj)]).decode()
    assert " U dem_step" in syms
