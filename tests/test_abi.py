"""The C-ABI library builds, loads and exports every symbol include/*.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(pm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1610_05258_gb300 import build
    try:
        return build.build()
    except (RuntimeError, FileNotFoundError) as e:  # no nvcc in this environment
        pytest.skip(f"cannot build: {e}")


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ["pm_ctx_create", "pm_interpolate", "pm_assign_delta", "pm_assign_flip", "pm_assign_mass",
              "pm_mass_solve"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_are_c_linkage(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    for n in declared_symbols():
        assert n in exported


def test_binding_names_match_header():
    import paper_1610_05258_gb300 as pm
    assert set(pm.EXPORTS) <= declared_symbols()


def test_header_compiles_as_c_and_cpp(tmp_path):
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "use.c"
    src.write_text('#include "pmt.h"\nint main(void) { pm_solve_opts o; o.solver = PM_SOLVER_CHEBYSHEV; return o.solver - 1; }\n')
    for comp, lang in (("gcc", "c"), ("g++", "c++")):
        r = subprocess.run([comp, "-x", lang, "-std=" + ("c99" if lang == "c" else "c++17"), "-Wall", "-Werror",
                            "-fsyntax-only", "-I", inc, str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_binding_struct_layouts_match_c(tmp_path):
    """The ctypes mirrors of pm_solve_opts and pm_solve_info have the C sizes
    and field offsets (as the C compiler lays them out)."""
    import paper_1610_05258_gb300 as pm
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pmt.h"', 'int main(void) {']
    for st, cls in (("pm_solve_opts", pm._Opts), ("pm_solve_info", pm._Info)):
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for name, _ in cls._fields_:
            lines.append(f'printf("{st}.{name} %zu\\n", offsetof({st}, {name}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for st, cls in (("pm_solve_opts", pm._Opts), ("pm_solve_info", pm._Info)):
        assert int(got[st]) == ctypes.sizeof(cls), st
        for name, _ in cls._fields_:
            assert int(got[f"{st}.{name}"]) == getattr(cls, name).offset, (st, name)
