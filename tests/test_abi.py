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
