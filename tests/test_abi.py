"""The C-ABI library builds for sm_103a and exports every entry point of include/sc.h.

Runs without a GPU: nvcc cross-compiles, and loading the library calls no CUDA API.
"""
import os
import re
import subprocess

import pytest

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


def test_default_config_values():
    from paper_1911_02366_gb300 import sc
    cfg = sc.default_config()
    assert (cfg.gmres_restart, cfg.gmres_max_iters, cfg.rel_tol, cfg.inner_tol) == (30, 4000, 1e-8, 1e-4)
    assert (cfg.precision, cfg.precond, cfg.tensor_cores) == (sc.SC_PREC_FP64, sc.SC_PC_BLOCK_JACOBI, 1)
    assert (cfg.outer_krylov, cfg.inner_iters, cfg.factor_fp16, cfg.explicit_schur) == (0, 0, 0, 0)
    assert cfg.interior_fp64 == 0 and cfg.adv_flux == sc.SC_FLUX_ROE
    assert (cfg.visc_flux, cfg.ip_penalty) == (sc.SC_VISC_BR1, 1.0)
    assert (cfg.gamma, cfg.Pr, cfg.Re, cfg.Ma) == (1.4, 0.72, 1600.0, 0.1)


def test_create_rejects_invalid_configs_before_any_cuda_call():
    # argument checks come first, so they answer SC_ERR_ARG without a GPU
    import ctypes
    from paper_1911_02366_gb300 import sc
    bad = [dict(gmres_restart=0), dict(gmres_restart=401), dict(gmres_max_iters=0), dict(rel_tol=0.0),
           dict(Re=0.0), dict(Ma=-1.0), dict(gamma=1.0), dict(Pr=0.0), dict(precision=7),
           dict(outer_krylov=31), dict(outer_krylov=-1), dict(inner_iters=-1), dict(precond=-1), dict(precond=5),
           dict(interior_fp64=2), dict(adv_flux=2), dict(visc_flux=2), dict(visc_flux=-1),
           dict(visc_flux=1, ip_penalty=0.0), dict(visc_flux=1, ip_penalty=-1.0),
           dict(visc_flux=1, ip_penalty=float("nan")), dict(ip_penalty=float("inf"))]
    L = sc.lib()
    for kw in bad:
        cfg = sc.default_config(**kw)
        h = ctypes.c_void_p()
        assert L.sc_create(ctypes.byref(cfg), None, ctypes.byref(h)) == sc.SC_ERR_ARG, kw
        assert not h.value


def test_hessenberg_eigenvalues_match_numpy():
    """Host QR step of the spectrum estimate (sc_hessenberg_eigvals), no GPU needed."""
    import numpy as np
    from paper_1911_02366_gb300 import sc
    rng = np.random.default_rng(5)
    for m in (1, 2, 7, 30, 60):
        H = np.triu(rng.standard_normal((m, m)), -1)
        got = sc.sc_hessenberg_eigvals(H)
        ref = np.linalg.eigvals(H)
        # each computed eigenvalue next to a reference one and vice versa (multisets match)
        d = np.abs(got[:, None] - ref[None, :])
        tol = 1e-9 * max(1.0, np.max(np.abs(ref)))
        assert np.max(d.min(axis=1)) <= tol and np.max(d.min(axis=0)) <= tol, m
    # a matrix with a known real spectrum and one with an exact zero subdiagonal
    H = np.diag([5.0, -3.0, 1e-3, 2.0]) + np.diag([1.0, 0.0, 1.0], -1)
    assert np.allclose(np.sort_complex(sc.sc_hessenberg_eigvals(H)), np.sort_complex(np.linalg.eigvals(H)))


def test_mixed_mesh_create_rejects_invalid_arguments_before_any_cuda_call():
    import ctypes
    import numpy as np
    from paper_1911_02366_gb300 import sc
    L = sc.lib()
    good = np.full(8, 3, np.int32)
    cases = [(dict(), 2, np.full(8, 7, np.int32)), (dict(), 2, np.full(8, 1, np.int32)),
             (dict(), 1, np.full(1, 3, np.int32)), (dict(precision=sc.SC_PREC_FP64), 2, good),
             (dict(visc_flux=sc.SC_VISC_SIPG), 2, good), (dict(precond=sc.SC_PC_RED_BLACK), 2, good),
             (dict(gmres_restart=0), 2, good)]
    for kw, n, orders in cases:
        cfg = sc.default_config(**{"precision": sc.SC_PREC_MIXED, **kw})
        h = ctypes.c_void_p()
        st = L.sc_mixed_create(ctypes.byref(cfg), None, n, 6.28, orders.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               0, ctypes.byref(h))
        assert st == sc.SC_ERR_ARG and not h.value, (kw, n)


def test_mixed_context_binding_checks_its_arguments_without_a_gpu():
    import numpy as np
    from paper_1911_02366_gb300 import sc
    with pytest.raises(ValueError):
        sc.MixedContext(2, np.full(7, 3))          # one order per element
    with pytest.raises(sc.SCError) as ei:
        sc.MixedContext(2, np.full(8, 9))          # orders outside 2..6
    assert ei.value.status == sc.SC_ERR_ARG
    with pytest.raises(sc.SCError):
        sc.MixedContext(2, np.full(8, 3), visc_flux=sc.SC_VISC_SIPG)
