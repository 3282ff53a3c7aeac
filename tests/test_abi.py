"""The C-ABI library builds for sm_103a and exports every entry point of include/sc.h.

Runs without a GPU: nvcc cross-compiles, and loading the library calls no CUDA API.
"""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_pipeline():
    names = declared_functions()
    for f in ("sc_create", "sc_set_mesh", "sc_set_state", "sc_set_timestep", "sc_assemble",
              "sc_condense", "sc_solve", "sc_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol():
    from paper_1911_02366_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(sc_[a-z0-9_]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_without_gpu_and_binding_matches():
    from paper_1911_02366_gb300 import sc
    L = sc.lib()
    for f in declared_functions():
        assert hasattr(L, f)
    assert set(sc.EXPORTS) <= set(declared_functions())
