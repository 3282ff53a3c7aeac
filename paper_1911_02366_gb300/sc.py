"""ctypes binding of the C ABI in include/sc.h (argument marshalling only).

Every function here forwards to the CUDA library of the same name; all arithmetic of
the Newton solve runs in the library's kernels.  Arrays are numpy (host) or torch CUDA
tensors (device); device tensors are passed by their data pointer.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SC_OK, SC_ERR_ARG, SC_ERR_CUDA, SC_ERR_OOM, SC_ERR_STATE = 0, 1, 2, 3, 4
SC_ERR_SINGULAR_BLOCK, SC_ERR_NONFINITE, SC_ERR_NOT_CONVERGED = 5, 6, 7
SC_PREC_FP64, SC_PREC_MIXED = 0, 1
SC_PC_BLOCK_JACOBI, SC_PC_NONE, SC_PC_LEARNED, SC_PC_RED_BLACK, SC_PC_RB_SCHUR = 0, 1, 2, 3, 4
SC_FLUX_ROE, SC_FLUX_LF = 0, 1
SC_VISC_BR1, SC_VISC_SIPG = 0, 1
SC_DIRECT_GLOBAL, SC_DIRECT_CONDENSED = 0, 1

_lib = None


class SCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sc status {status}: {msg}")
        self.status = status


class sc_config(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Re", ctypes.c_double),
                ("Ma", ctypes.c_double), ("Ts", ctypes.c_double), ("sutherland", ctypes.c_int),
                ("roe_delta", ctypes.c_double), ("precision", ctypes.c_int), ("precond", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("gmres_max_iters", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("rel_tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("tensor_cores", ctypes.c_int), ("learned_min_reduction", ctypes.c_double),
                ("factor_fp16", ctypes.c_int), ("explicit_schur", ctypes.c_int),
                ("outer_krylov", ctypes.c_int), ("inner_iters", ctypes.c_int), ("interior_fp64", ctypes.c_int),
                ("adv_flux", ctypes.c_int), ("visc_flux", ctypes.c_int), ("ip_penalty", ctypes.c_double)]


class sc_solve_stats(ctypes.Structure):
    _fields_ = [("gmres_iters", ctypes.c_int), ("refinements", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("cond_rel_residual", ctypes.c_double),
                ("ms_rhs", ctypes.c_double), ("ms_gmres", ctypes.c_double),
                ("ms_backsub", ctypes.c_double), ("ms_refine", ctypes.c_double),
                ("first_bad_element", ctypes.c_int), ("learned_fallbacks", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTS = ["sc_default_config", "sc_create", "sc_destroy", "sc_last_error", "sc_set_mesh", "sc_node_coords",
           "sc_set_state", "sc_set_timestep", "sc_assemble", "sc_condense", "sc_solve", "sc_get_rhs",
           "sc_apply_jacobian", "sc_get_jacobian_block", "sc_condensed_matvec", "sc_sizes",
           "sc_launch_count", "sc_profile_kernel", "sc_profile_read", "sc_kernel_work",
           "sc_condensed_matvec_static", "sc_gemm_tf32", "sc_mlp_forward", "sc_mlp_backward", "sc_mlp_loss",
           "sc_mlp_adam", "sc_learned_features", "sc_learned_targets", "sc_set_learned_weights", "sc_set_learned_correction",
           "sc_get_state", "sc_condensed_rhs", "sc_backsubstitute", "sc_newton_step", "sc_batch_create",
           "sc_batch_condense", "sc_batch_tiles", "sc_batch_destroy", "sc_spectrum_estimate",
           "sc_hessenberg_eigvals", "sc_steady_residual", "sc_explicit_march", "sc_implicit_march",
           "sc_precond_apply", "sc_profile_elements", "sc_mlp_bf16", "sc_mlp_train", "sc_mlp_save", "sc_mlp_load", "sc_load_mlp",
           "sc_direct_factor", "sc_direct_solve", "sc_partition_slabs", "sc_partition_halo",
           "sc_mixed_create", "sc_mixed_destroy", "sc_mixed_last_error", "sc_mixed_sizes", "sc_mixed_set_state",
           "sc_mixed_residual", "sc_mixed_jvp", "sc_mixed_own_block", "sc_mixed_condense", "sc_mixed_solve",
           "sc_mixed_launch_count", "sc_mixed_profile", "sc_mixed_profile_read"]

SC_KERNEL_COND_INTERIOR, SC_KERNEL_COND_BOUNDARY, SC_KERNEL_LU_SOLVE, SC_KERNEL_LU = 0, 1, 2, 3
SC_KERNEL_SCHUR_GEMM, SC_KERNEL_GJ_INV, SC_KERNEL_ASSEMBLE_OWN, SC_KERNEL_GLOBAL_APPLY = 4, 5, 6, 7
SC_KERNEL_EXPLICIT_GEMM, SC_KERNEL_EXPLICIT_APPLY = 8, 9


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libsc.so (building it first if it is missing).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)
    L.sc_default_config.argtypes = [ctypes.POINTER(sc_config)]
    L.sc_mixed_create.argtypes = [ctypes.POINTER(sc_config), vp, ctypes.c_int, ctypes.c_double, ip, ctypes.c_int,
                                  ctypes.POINTER(vp)]
    L.sc_mixed_destroy.argtypes = [vp]; L.sc_mixed_destroy.restype = None
    L.sc_mixed_last_error.argtypes = [vp]; L.sc_mixed_last_error.restype = ctypes.c_char_p
    L.sc_mixed_sizes.argtypes = [vp] + [ctypes.POINTER(ctypes.c_longlong)] * 3
    L.sc_mixed_set_state.argtypes = [vp, dp, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    L.sc_mixed_residual.argtypes = [vp, dp, ctypes.c_int]
    L.sc_mixed_jvp.argtypes = [vp, dp, dp, ctypes.c_int]
    L.sc_mixed_own_block.argtypes = [vp, ctypes.c_int, dp]
    L.sc_mixed_condense.argtypes = [vp]
    L.sc_mixed_solve.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(sc_solve_stats)]
    L.sc_mixed_launch_count.argtypes = [vp]; L.sc_mixed_launch_count.restype = ctypes.c_longlong
    L.sc_mixed_profile.argtypes = [vp, ctypes.c_int]
    L.sc_mixed_profile_read.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.sc_create.argtypes = [ctypes.POINTER(sc_config), vp, ctypes.POINTER(vp)]
    L.sc_destroy.argtypes = [vp]; L.sc_destroy.restype = None
    L.sc_last_error.argtypes = [vp]; L.sc_last_error.restype = ctypes.c_char_p
    L.sc_set_mesh.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    L.sc_node_coords.argtypes = [vp, dp]
    L.sc_set_state.argtypes = [vp, dp, dp, dp, ctypes.c_int]
    L.sc_set_timestep.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.sc_assemble.argtypes = [vp]
    L.sc_condense.argtypes = [vp]
    L.sc_solve.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(sc_solve_stats)]
    L.sc_get_rhs.argtypes = [vp, dp, ctypes.c_int]
    L.sc_apply_jacobian.argtypes = [vp, dp, dp, ctypes.c_int]
    L.sc_get_jacobian_block.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp]
    L.sc_condensed_matvec.argtypes = [vp, dp, dp]
    L.sc_condensed_matvec_static.argtypes = [vp, dp, dp]
    ll, fl, ci = ctypes.c_longlong, ctypes.c_float, ctypes.c_int
    L.sc_gemm_tf32.argtypes = [ci, ci, ci, ci, fl, vp, ll, ci, ci, vp, ll, ci, ci, fl, vp, ll, ci, vp]
    L.sc_mlp_forward.argtypes = [vp, vp, vp, ci, vp, vp, vp]
    L.sc_mlp_backward.argtypes = [vp, vp, vp, vp, ci, vp, vp, vp, vp]
    L.sc_mlp_loss.argtypes = [vp, vp, ci, vp, vp, vp]
    L.sc_mlp_adam.argtypes = [vp, vp, vp, vp, vp, vp, vp, ci, fl, vp]
    L.sc_learned_features.argtypes = [vp, vp, vp]
    L.sc_learned_targets.argtypes = [vp, vp]
    L.sc_set_learned_weights.argtypes = [vp, vp, vp]
    L.sc_set_learned_correction.argtypes = [vp, vp, ctypes.c_float]
    L.sc_get_state.argtypes = [vp, dp, ctypes.c_int]
    L.sc_condensed_rhs.argtypes = [vp, dp, ctypes.c_int]
    L.sc_backsubstitute.argtypes = [vp, dp, dp, ctypes.c_int]
    L.sc_newton_step.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(sc_solve_stats),
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.sc_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
    L.sc_batch_condense.argtypes = [vp, ctypes.c_int]
    L.sc_batch_tiles.argtypes = [vp, ctypes.c_int, ip, ip, ip, ip]
    L.sc_batch_destroy.argtypes = [vp]; L.sc_batch_destroy.restype = None
    L.sc_sizes.argtypes = [vp, ip, ip, ip, ip]
    L.sc_spectrum_estimate.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
    L.sc_hessenberg_eigvals.argtypes = [ctypes.c_int, dp, dp, dp]
    L.sc_steady_residual.argtypes = [vp, dp]
    L.sc_precond_apply.argtypes = [vp, dp, dp]
    L.sc_profile_elements.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.sc_mlp_bf16.argtypes = [vp, vp, ctypes.c_int, vp]
    L.sc_mlp_train.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int), vp, vp, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_float, ctypes.c_uint64, vp, vp]
    L.sc_mlp_save.argtypes = [ctypes.c_char_p, vp, vp]
    L.sc_mlp_load.argtypes = [ctypes.c_char_p, vp, vp, vp]
    L.sc_load_mlp.argtypes = [vp, ctypes.c_char_p]
    L.sc_direct_factor.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.sc_direct_solve.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(sc_solve_stats)]
    L.sc_partition_slabs.argtypes = [ctypes.c_int, ctypes.c_int, vp]
    L.sc_partition_halo.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, vp]
    L.sc_explicit_march.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, dp]
    L.sc_implicit_march.argtypes = [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    dp, dp, dp, ctypes.POINTER(ctypes.c_int)]
    L.sc_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.sc_profile_kernel.argtypes = [vp, ctypes.c_int]
    L.sc_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double)]
    L.sc_kernel_work.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    for f in EXPORTS:
        if f not in ("sc_destroy", "sc_last_error", "sc_batch_destroy"):
            getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a):
    """(pointer, on_device) for a numpy array or a torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if a.dtype.__str__() != "torch.float64" or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(type(a))


def default_config(**kw) -> sc_config:
    cfg = sc_config()
    lib().sc_default_config(ctypes.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


class MixedContext:
    """One periodic mesh of mixed polynomial order (wraps sc_mixed_create / sc_mixed_destroy).
    States are flat ragged arrays [sum_e (N_e+1)^3 * 5] (numpy on the host or torch on the
    device)."""

    def __init__(self, n: int, orders, L: float = 2 * np.pi, force_mortar: bool = False,
                 cfg: sc_config | None = None, stream: int | None = None, **kw):
        self._L = lib()
        kw.setdefault("precision", SC_PREC_MIXED)
        self.cfg = cfg if cfg is not None else default_config(**kw)
        self.orders = np.ascontiguousarray(orders, dtype=np.int32)
        if self.orders.shape != (n ** 3,):
            raise ValueError("one order per element")
        h = ctypes.c_void_p()
        st = self._L.sc_mixed_create(ctypes.byref(self.cfg), ctypes.c_void_p(stream or 0), int(n), float(L),
                                     self.orders.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(force_mortar),
                                     ctypes.byref(h))
        if st != SC_OK:
            raise SCError(st, "sc_mixed_create rejected the arguments")
        self.h = h

    def _check(self, status):
        if status != SC_OK:
            raise SCError(status, self._L.sc_mixed_last_error(self.h).decode() if self.h else "")

    def close(self):
        if getattr(self, "h", None):
            self._L.sc_mixed_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sizes(self):
        v = [ctypes.c_longlong() for _ in range(3)]
        self._check(self._L.sc_mixed_sizes(self.h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_state(self, Q, Qs=None, Qsm1=None, dt: float = 1.0, bdf: int = 1):
        Qs = Q if Qs is None else Qs
        (pq, dq), (ps, ds), (pm, dm) = _ptr(Q), _ptr(Qs), _ptr(Qsm1)
        if ds != dq or (Qsm1 is not None and dm != dq):
            raise ValueError("all state arrays must live on the same side")
        self._check(self._L.sc_mixed_set_state(self.h, pq, ps, pm, float(dt), int(bdf), dq))

    def residual(self, R):
        p, dev = _ptr(R)
        self._check(self._L.sc_mixed_residual(self.h, p, dev))
        return R

    def jvp(self, x, y):
        (px, dx), (py, dy) = _ptr(x), _ptr(y)
        if dx != dy:
            raise ValueError("x and y must live on the same side")
        self._check(self._L.sc_mixed_jvp(self.h, px, py, dx))
        return y

    def own_block(self, e: int) -> np.ndarray:
        ne = 5 * (int(self.orders[e]) + 1) ** 3
        out = np.zeros((ne, ne))
        self._check(self._L.sc_mixed_own_block(self.h, int(e), out.ctypes.data))
        return out

    def condense(self):
        self._check(self._L.sc_mixed_condense(self.h))

    def solve(self, dQ, raise_on_not_converged: bool = True):
        st = sc_solve_stats()
        p, dev = _ptr(dQ)
        s = self._L.sc_mixed_solve(self.h, p, dev, ctypes.byref(st))
        if s != SC_OK and not (s == SC_ERR_NOT_CONVERGED and not raise_on_not_converged):
            self._check(s)
        return st.as_dict() | {"status": s}

    def launch_count(self) -> int:
        return int(self._L.sc_mixed_launch_count(self.h))

    def profile(self, on: bool):
        self._check(self._L.sc_mixed_profile(self.h, int(on)))

    def profile_read(self):
        """(block-Jacobi applications, their total device ms, algorithmic bytes of one)."""
        n, ms, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        self._check(self._L.sc_mixed_profile_read(self.h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b)))
        return n.value, ms.value, b.value


class Context:
    """One solver context (wraps sc_create / sc_destroy)."""

    def __init__(self, cfg: sc_config | None = None, stream: int | None = None, **kw):
        self._L = lib()
        self.cfg = cfg if cfg is not None else default_config(**kw)
        h = ctypes.c_void_p()
        self._check(self._L.sc_create(ctypes.byref(self.cfg), ctypes.c_void_p(stream or 0), ctypes.byref(h)), None)
        self.h = h

    def _check(self, status, h=...):
        if status != SC_OK:
            hh = self.h if h is ... else h
            msg = self._L.sc_last_error(hh).decode() if hh else ""
            raise SCError(status, msg)

    def close(self):
        if getattr(self, "h", None):
            self._L.sc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sc_set_mesh(self, n: int, L: float, N: int):
        self._check(self._L.sc_set_mesh(self.h, n, L, N))

    def sc_sizes(self):
        v = [ctypes.c_int() for _ in range(4)]
        self._check(self._L.sc_sizes(self.h, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def sc_node_coords(self) -> np.ndarray:
        K, ne, _, _ = self.sc_sizes()
        out = np.zeros((K, ne // 5, 3))
        self._check(self._L.sc_node_coords(self.h, out.ctypes.data))
        return out

    def sc_set_timestep(self, dt: float, bdf: int = 1):
        self._check(self._L.sc_set_timestep(self.h, dt, bdf))

    def sc_set_state(self, Q, Qs=None, Qsm1=None):
        Qs = Q if Qs is None else Qs
        (pq, dq), (ps, ds), (pm, dm) = _ptr(Q), _ptr(Qs), _ptr(Qsm1)
        if Qsm1 is not None and dm != dq:
            raise ValueError("all state arrays must live on the same side")
        if ds != dq:
            raise ValueError("all state arrays must live on the same side")
        self._check(self._L.sc_set_state(self.h, pq, ps, pm, dq))

    def sc_assemble(self):
        self._check(self._L.sc_assemble(self.h))

    def sc_condense(self):
        self._check(self._L.sc_condense(self.h))

    def sc_solve(self, dQ, raise_on_not_converged: bool = True):
        st = sc_solve_stats()
        p, dev = _ptr(dQ)
        s = self._L.sc_solve(self.h, p, dev, ctypes.byref(st))
        if s != SC_OK and not (s == SC_ERR_NOT_CONVERGED and not raise_on_not_converged):
            self._check(s)
        return st.as_dict() | {"status": s}

    def sc_get_rhs(self, B):
        p, dev = _ptr(B)
        self._check(self._L.sc_get_rhs(self.h, p, dev))
        return B

    def sc_get_state(self, Q):
        p, dev = _ptr(Q)
        self._check(self._L.sc_get_state(self.h, p, dev))
        return Q

    def sc_condensed_rhs(self, g):
        p, dev = _ptr(g)
        self._check(self._L.sc_condensed_rhs(self.h, p, dev))
        return g

    def sc_backsubstitute(self, xb, dQ):
        (px, dx), (pq, dq) = _ptr(xb), _ptr(dQ)
        if dx != dq:
            raise ValueError("xb and dQ must live on the same side")
        self._check(self._L.sc_backsubstitute(self.h, px, pq, dq))
        return dQ

    def sc_newton_step(self, max_newton=10, newton_tol=1e-8):
        """Newton iterations on the current step; returns (updates, ||R||/||R0||, last solve stats)."""
        st = sc_solve_stats()
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        self._check(self._L.sc_newton_step(self.h, max_newton, newton_tol, ctypes.byref(st), ctypes.byref(it),
                                           ctypes.byref(rel)))
        return it.value, rel.value, st.as_dict()

    def sc_apply_jacobian(self, x, y):
        (px, dx), (py, dy) = _ptr(x), _ptr(y)
        if dx != dy:
            raise ValueError("x and y must live on the same side")
        self._check(self._L.sc_apply_jacobian(self.h, px, py, dx))
        return y

    def sc_get_jacobian_block(self, e: int, c: int) -> np.ndarray:
        _, ne, _, _ = self.sc_sizes()
        out = np.zeros((ne, ne))
        self._check(self._L.sc_get_jacobian_block(self.h, e, c, out.ctypes.data))
        return out

    def sc_condensed_matvec(self, xb, yb):
        (px, dx), (py, dy) = _ptr(xb), _ptr(yb)
        if not (dx and dy):
            raise ValueError("condensed_matvec takes device tensors")
        self._check(self._L.sc_condensed_matvec(self.h, px, py))
        return yb

    def sc_launch_count(self) -> int:
        v = ctypes.c_longlong()
        self._check(self._L.sc_launch_count(self.h, ctypes.byref(v)))
        return v.value

    def sc_profile_kernel(self, kernel_id: int):
        self._check(self._L.sc_profile_kernel(self.h, kernel_id))

    def sc_profile_read(self):
        n = ctypes.c_longlong(); ms = ctypes.c_double()
        self._check(self._L.sc_profile_read(self.h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def sc_profile_elements(self) -> int:
        n = ctypes.c_longlong()
        self._check(self._L.sc_profile_elements(self.h, ctypes.byref(n)))
        return n.value

    def sc_kernel_work(self, kernel_id: int):
        f = ctypes.c_double(); b = ctypes.c_double()
        self._check(self._L.sc_kernel_work(self.h, kernel_id, ctypes.byref(f), ctypes.byref(b)))
        return f.value, b.value

    def sc_learned_features(self, F, snorm):
        """Features [K*nbn, 128] and ||[S_ee]_kk||_F [K*nbn] (float32 device tensors)."""
        self._check(self._L.sc_learned_features(self.h, F.data_ptr(), snorm.data_ptr()))
        return F, snorm

    def sc_learned_targets(self, T):
        """Training targets [K*nbn, 25] (float32 device tensor); small meshes only."""
        self._check(self._L.sc_learned_targets(self.h, T.data_ptr()))
        return T

    def sc_set_learned_weights(self, net):
        """Copy the parameters of an MLP (its BF16 weights and biases) into the context."""
        self._check(self._L.sc_set_learned_weights(self.h, net.Wh.data_ptr(), net.b.data_ptr()))

    def sc_set_learned_correction(self, Ck, scale=1.0):
        """Replace the per-node corrections by scale * Ck ([K*nbn, 25] float32 device)."""
        self._check(self._L.sc_set_learned_correction(self.h, Ck.data_ptr(), ctypes.c_float(scale)))

    def sc_spectrum_estimate(self, which: str = "S", m_max: int = 30, m_min: int = 30, inv_tol: float = 1e-12):
        """Largest and smallest eigenvalues of A ('A') or S ('S') and their modulus ratio."""
        out = np.zeros(6)
        self._check(self._L.sc_spectrum_estimate(self.h, {"A": 0, "S": 1}[which], m_max, m_min, inv_tol,
                                                 out.ctypes.data))
        return {"lam_max": complex(out[0], out[1]), "lam_min": complex(out[2], out[3]), "cond": out[4],
                "inner_iters": int(out[5])}

    def sc_direct_factor(self, which: str = "S"):
        """Dense LU of the global A ('A') or the condensed S ('S'); returns (ms_form, ms_factor)."""
        f, g = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.sc_direct_factor(self.h, {"A": SC_DIRECT_GLOBAL, "S": SC_DIRECT_CONDENSED}[which],
                                             ctypes.byref(f), ctypes.byref(g)))
        return f.value, g.value

    def sc_direct_solve(self, dQ, raise_on_not_converged: bool = True):
        st = sc_solve_stats()
        p, dev = _ptr(dQ)
        s = self._L.sc_direct_solve(self.h, p, dev, ctypes.byref(st))
        if s != SC_OK and not (s == SC_ERR_NOT_CONVERGED and not raise_on_not_converged):
            self._check(s)
        return st.as_dict() | {"status": s}

    def sc_load_mlp(self, path: str):
        """Load a saved network (sc_mlp_save format) as the context's learned weights."""
        self._check(self._L.sc_load_mlp(self.h, path.encode()))

    def sc_precond_apply(self, v, z):
        """z = P v with the context's condensed preconditioner (device float64 tensors)."""
        (pv, dv), (pz, dz) = _ptr(v), _ptr(z)
        if not (dv and dz):
            raise ValueError("precond_apply takes device tensors")
        self._check(self._L.sc_precond_apply(self.h, pv, pz))
        return z

    def sc_steady_residual(self) -> float:
        """||M^-1 H(Q)||_inf of the current state."""
        r = np.zeros(1)
        self._check(self._L.sc_steady_residual(self.h, r.ctypes.data))
        return float(r[0])

    def sc_explicit_march(self, cfl: float, nsteps: int, dfl: float = 0.0):
        """Low-storage RK3 steps; returns (residual history, dt history, device ms)."""
        res, dts, ms = np.zeros(nsteps + 1), np.zeros(max(nsteps, 1)), np.zeros(1)
        self._check(self._L.sc_explicit_march(self.h, cfl, dfl, nsteps, res.ctypes.data, dts.ctypes.data,
                                              ms.ctypes.data))
        return res, dts[:nsteps], float(ms[0])

    def sc_implicit_march(self, dt: float, nsteps: int, jacobian_every: int = 0, direct: str | None = None,
                          steady_tol: float = 0.0):
        """Linearised BDF1 steps with a reused Jacobian, solved by condensed GMRES (direct=None)
        or dense LU of A ('A') or S ('S'); stops early at steady_tol > 0.  Returns (residual
        history, cumulative device ms, GMRES iterations per step), cut to the steps taken."""
        res, ms = np.zeros(nsteps + 1), np.zeros(nsteps + 1)
        its = np.zeros(max(nsteps, 1), dtype=np.int32)
        taken = ctypes.c_int()
        d = {None: -1, "A": SC_DIRECT_GLOBAL, "S": SC_DIRECT_CONDENSED}[direct]
        self._check(self._L.sc_implicit_march(self.h, dt, nsteps, jacobian_every, d, steady_tol, res.ctypes.data,
                                              ms.ctypes.data, its.ctypes.data, ctypes.byref(taken)))
        k = taken.value
        return res[:k + 1], ms[:k + 1], its[:k]

    def sc_condensed_matvec_static(self, xb, yb):
        """S x_b without any allocation in the call (fixed 8 MiB device scratch); enqueues only."""
        (px, dx), (py, dy) = _ptr(xb), _ptr(yb)
        if not (dx and dy):
            raise ValueError("condensed_matvec_static takes device tensors")
        self._check(self._L.sc_condensed_matvec_static(self.h, px, py))
        return yb


def sc_hessenberg_eigvals(H: np.ndarray) -> np.ndarray:
    """Eigenvalues of an upper Hessenberg matrix (host routine of the spectrum estimate)."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    m = H.shape[0]
    re, im = np.zeros(m), np.zeros(m)
    s = lib().sc_hessenberg_eigvals(m, H.ctypes.data, re.ctypes.data, im.ctypes.data)
    if s != SC_OK:
        raise SCError(s, "Hessenberg QR failed")
    return re + 1j * im


def sc_partition_slabs(n: int, nparts: int) -> np.ndarray:
    """Rank of every element of the n^3 mesh: slabs of whole z-planes (host only)."""
    part = np.zeros(n ** 3, dtype=np.int32)
    s = lib().sc_partition_slabs(n, nparts, part.ctypes.data)
    if s != SC_OK:
        raise SCError(s, "partition: need 1 <= nparts <= n <= 32")
    return part


def sc_partition_halo(n: int, part: np.ndarray, rank: int):
    """(owned, halo_b, halo_u) element indices of one rank (host only): the owned elements,
    the elements whose boundary values and whose interior values the owned rows need."""
    part = np.ascontiguousarray(part, dtype=np.int32)
    K = n ** 3
    counts = np.zeros(3, dtype=np.int32)
    owned, hb, hu = (np.zeros(K, dtype=np.int32) for _ in range(3))
    s = lib().sc_partition_halo(n, part.ctypes.data, rank, counts.ctypes.data, owned.ctypes.data, hb.ctypes.data,
                                hu.ctypes.data)
    if s != SC_OK:
        raise SCError(s, "partition halo: bad arguments")
    return owned[:counts[0]].copy(), hb[:counts[1]].copy(), hu[:counts[2]].copy()


def sc_gemm_tf32(A, B, C, alpha=1.0, beta=0.0, stream=None, trans_a=False, trans_b=False):
    """C[b] = alpha op(A[b]) @ op(B[b]) + beta C[b] on the TF32 tensor cores.

    float32 contiguous CUDA tensors: A is [batch, M, K] ([batch, K, M] with trans_a),
    B is [batch, K, N] ([batch, N, K] with trans_b), C is [batch, M, N]."""
    L = lib()
    for t in (A, B, C):
        if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"):
            raise ValueError("contiguous float32 CUDA tensors required")
    bt, M, N = C.shape
    K = A.shape[1] if trans_a else A.shape[2]
    s = L.sc_gemm_tf32(bt, M, N, K, alpha, A.data_ptr(), A.shape[1] * A.shape[2], A.shape[2], int(trans_a),
                       B.data_ptr(), B.shape[1] * B.shape[2], B.shape[2], int(trans_b), beta, C.data_ptr(), M * N, N,
                       ctypes.c_void_p(stream or 0))
    if s != SC_OK:
        raise SCError(s, "sc_gemm_tf32 failed")
    return C


# ---- learned correction of the red-black sweep: the network ---------------------
MLP_IN, MLP_H, MLP_OUT = 128, 256, 25
MLP_NW = MLP_H * MLP_IN + MLP_H * MLP_H + MLP_OUT * MLP_H
MLP_NB = 2 * MLP_H + MLP_OUT


class MLP:
    """Device parameters of the correction network and the C-ABI calls on them.

    W: [W1 | W2 | W3] FP32 masters and their BF16 copy, b: [b1 | b2 | b3]; gradients and
    Adam moments alongside.  Every computation runs in the library's kernels."""

    def __init__(self, W, b, stream=None):
        import numpy as np
        import torch
        self._L = lib()
        self.stream = stream or 0
        W = np.asarray(W, dtype=np.float32).reshape(-1)
        b = np.asarray(b, dtype=np.float32).reshape(-1)
        if W.size != MLP_NW or b.size != MLP_NB:
            raise ValueError("wrong parameter sizes")
        dev = "cuda"
        self.W = torch.tensor(W, device=dev)
        self.Wh = torch.empty(MLP_NW, dtype=torch.int16, device=dev)
        self._ck(self._L.sc_mlp_bf16(self.W.data_ptr(), self.Wh.data_ptr(), MLP_NW, ctypes.c_void_p(self.stream)),
                 "sc_mlp_bf16")
        self.b = torch.tensor(b, device=dev)
        self.gW = torch.zeros(MLP_NW, device=dev)
        self.gb = torch.zeros(MLP_NB, device=dev)
        self.m = torch.zeros(MLP_NW + MLP_NB, device=dev)
        self.v = torch.zeros(MLP_NW + MLP_NB, device=dev)
        self.step = 0

    def _ck(self, s, what):
        if s != SC_OK:
            raise SCError(s, what)

    def forward(self, X, Y, cache=None):
        self._ck(self._L.sc_mlp_forward(self.Wh.data_ptr(), self.b.data_ptr(), X.data_ptr(), X.shape[0], Y.data_ptr(),
                                        cache.data_ptr() if cache is not None else None,
                                        ctypes.c_void_p(self.stream)), "sc_mlp_forward")
        return Y

    def backward(self, X, cache, dY, work):
        self._ck(self._L.sc_mlp_backward(self.Wh.data_ptr(), X.data_ptr(), cache.data_ptr(), dY.data_ptr(),
                                         X.shape[0], self.gW.data_ptr(), self.gb.data_ptr(), work.data_ptr(),
                                         ctypes.c_void_p(self.stream)), "sc_mlp_backward")

    def loss(self, Y, T, dY=None, loss_sum=None):
        self._ck(self._L.sc_mlp_loss(Y.data_ptr(), T.data_ptr(), Y.shape[0],
                                     dY.data_ptr() if dY is not None else None,
                                     loss_sum.data_ptr() if loss_sum is not None else None,
                                     ctypes.c_void_p(self.stream)), "sc_mlp_loss")

    def adam(self, lr):
        self.step += 1
        self._ck(self._L.sc_mlp_adam(self.W.data_ptr(), self.Wh.data_ptr(), self.b.data_ptr(), self.gW.data_ptr(),
                                     self.gb.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.step,
                                     ctypes.c_float(lr), ctypes.c_void_p(self.stream)), "sc_mlp_adam")

    def train(self, X, T, epochs, batch, lr, seed=0):
        """Shuffled mini-batch Adam on device features X [n, 64] and targets T [n, 25]
        (sc_mlp_train); returns the per-epoch mean loss."""
        import numpy as np
        hist = np.zeros(max(epochs, 1), dtype=np.float32)
        step = ctypes.c_int(self.step)
        self._ck(self._L.sc_mlp_train(self.W.data_ptr(), self.Wh.data_ptr(), self.b.data_ptr(), self.m.data_ptr(),
                                      self.v.data_ptr(), ctypes.byref(step), X.data_ptr(), T.data_ptr(), X.shape[0],
                                      epochs, batch, ctypes.c_float(lr), ctypes.c_uint64(seed), hist.ctypes.data,
                                      ctypes.c_void_p(self.stream)), "sc_mlp_train")
        self.step = step.value
        return [float(x) for x in hist[:epochs]]

    def save(self, path: str):
        self._ck(self._L.sc_mlp_save(path.encode(), self.W.data_ptr(), self.b.data_ptr()), "sc_mlp_save")

    @classmethod
    def load(cls, path: str, stream=None):
        import numpy as np
        net = cls(np.zeros(MLP_NW), np.zeros(MLP_NB), stream=stream)
        net._ck(net._L.sc_mlp_load(path.encode(), net.W.data_ptr(), net.Wh.data_ptr(), net.b.data_ptr()),
                "sc_mlp_load")
        return net


SC_BATCH_GRAPH, SC_BATCH_AUTOTUNE = 1, 2


class Batch:
    """Batched condensation of several assembled systems of (possibly) different orders."""

    def __init__(self, contexts):
        self._L = lib()
        self.h = None
        self.contexts = list(contexts)  # kept alive with the batch
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.h for c in self.contexts])
        h = ctypes.c_void_p()
        s = self._L.sc_batch_create(arr, len(self.contexts), ctypes.byref(h))
        if s != SC_OK:
            raise SCError(s, "sc_batch_create failed")
        self.h = h

    def condense(self, graph=True, autotune=True):
        flags = (SC_BATCH_GRAPH if graph else 0) | (SC_BATCH_AUTOTUNE if autotune else 0)
        s = self._L.sc_batch_condense(self.h, flags)
        if s != SC_OK:
            msg = self._L.sc_last_error(self.contexts[0].h).decode()
            raise SCError(s, msg or "sc_batch_condense failed")

    def tiles(self, c):
        v = [ctypes.c_int() for _ in range(4)]
        s = self._L.sc_batch_tiles(self.h, c, *[ctypes.byref(x) for x in v])
        if s != SC_OK:
            raise SCError(s, "sc_batch_tiles failed")
        return tuple(x.value for x in v)

    def close(self):
        if self.h:
            self._L.sc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
