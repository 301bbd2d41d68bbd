"""Thin Python binding of libmw (ctypes): argument marshalling only, same names as the C ABI.

Every step of the method runs in libmw's CUDA kernels.  Device buffers are torch tensors (torch
provides device memory and the stream); host buffers are numpy arrays.  The library must be
built (``paper_2311_05322_gb300.build.build()``); there is no fallback when it is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmw.so")

MW_OK, MW_EINVAL, MW_ECUDA, MW_ENOMEM, MW_ENOCONV, MW_ETIMEOUT, MW_ESTATE, MW_ESINGULAR = range(8)
MW_PREC_FP64, MW_PREC_FP32, MW_PREC_BF16, MW_PREC_FP64_FROM_FP32, MW_PREC_SPARSE, MW_PREC_SPARSE_BF16 = 0, 1, 2, 3, 4, 5
MW_MODE_FP64, MW_MODE_MIXED = 0, 1
STATUS_NAMES = {0: "MW_OK", 1: "MW_EINVAL", 2: "MW_ECUDA", 3: "MW_ENOMEM", 4: "MW_ENOCONV", 5: "MW_ETIMEOUT",
                6: "MW_ESTATE", 7: "MW_ESINGULAR"}


class MWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mw_mesh_info(C.Structure):
    _fields_ = [("n_vert", C.c_int64), ("n_tet", C.c_int64), ("n_edge", C.c_int64), ("n_face", C.c_int64),
                ("n_bface", C.c_int64), ("nnz", C.c_int64)]


class mw_port(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("u", C.c_double * 3), ("v", C.c_double * 3), ("a", C.c_double),
                ("eps_fill", C.c_double * 2)]


class mw_solve_opts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("restart", C.c_int32), ("batch", C.c_int32), ("max_it", C.c_int32),
                ("tol", C.c_double), ("inner_tol", C.c_double), ("max_outer", C.c_int32),
                ("use_precond", C.c_int32)]


class mw_solve_stats(C.Structure):
    _fields_ = [("n_cols", C.c_int32), ("n_converged", C.c_int32), ("outer_steps", C.c_int32),
                ("arnoldi_steps", C.c_int32), ("max_relres", C.c_double), ("solve_ms", C.c_double),
                ("iters", C.POINTER(C.c_int32)), ("relres", C.POINTER(C.c_double))]


class mw_launch_shapes(C.Structure):
    _fields_ = [("tc_stages", C.c_int32), ("dots_stages", C.c_int32), ("update_stages", C.c_int32),
                ("spmm_threads", C.c_int32)]


TUNE_KERNELS = ("tc", "dots", "update", "spmm")   # MW_TUNE_* order


class mw_tune_report(C.Structure):
    _fields_ = [("n_cols", C.c_int32), ("mode", C.c_int32), ("restart", C.c_int32), ("chosen", mw_launch_shapes),
                ("n_cand", C.c_int32 * 4), ("cand", (C.c_int32 * 8) * 4), ("ms", (C.c_double * 8) * 4)]


class mw_nn_opts(C.Structure):
    _fields_ = [("batch", C.c_int32), ("epochs", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64)]


class mw_nn_stats(C.Structure):
    _fields_ = [("epochs_run", C.c_int32), ("epoch_loss", C.POINTER(C.c_double)), ("seconds", C.c_double)]


class mw_inv_opts(C.Structure):
    _fields_ = [("m", C.c_int32), ("max_it", C.c_int32), ("c1", C.c_double), ("max_ls", C.c_int32),
                ("first_step", C.c_double), ("alpha", C.c_double), ("target_J", C.c_double)]


class mw_inv_history(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("evaluations", C.c_int32), ("J", C.POINTER(C.c_double)),
                ("seconds", C.POINTER(C.c_double))]


_P = C.c_void_p
_SIGS = {
    "mw_create": (C.c_int32, [C.POINTER(_P), C.c_int, _P]),
    "mw_destroy": (None, [_P]),
    "mw_last_error": (C.c_char_p, [_P]),
    "mw_set_memory_cap": (C.c_int32, [_P, C.c_int64]),
    "mw_set_graphs": (C.c_int32, [_P, C.c_int32]),
    "mw_set_autotune": (C.c_int32, [_P, C.c_int32]),
    "mw_set_launch_shapes": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(mw_launch_shapes)]),
    "mw_autotune": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, C.POINTER(mw_tune_report)]),
    "mw_set_mesh": (C.c_int32, [_P, C.c_int64, _P, C.c_int64, _P, C.POINTER(mw_mesh_info)]),
    "mw_get_topology": (C.c_int32, [_P, _P, _P, _P, _P, _P]),
    "mw_get_element_matrices": (C.c_int32, [_P, _P, _P, _P]),
    "mw_assemble": (C.c_int32, [_P, C.c_int32, _P, _P, _P]),
    "mw_get_matrix": (C.c_int32, [_P, C.c_int32, _P]),
    "mw_apply_matrix": (C.c_int32, [_P, C.c_int32, C.c_int32, _P, _P, C.c_int32]),
    "mw_set_sources": (C.c_int32, [_P, C.c_int32, _P, _P, _P, _P]),
    "mw_set_ports": (C.c_int32, [_P, C.c_int32, C.POINTER(mw_port), C.c_int64, _P, _P]),
    "mw_get_port_vectors": (C.c_int32, [_P, _P, _P]),
    "mw_setup_preconditioner": (C.c_int32, [_P, C.c_int32, _P, C.c_int32, C.c_int32]),
    "mw_apply_preconditioner": (C.c_int32, [_P, C.c_int32, _P, _P, C.c_int32]),
    "mw_get_partition": (C.c_int32, [_P, _P, _P]),
    "mw_solve": (C.c_int32, [_P, C.POINTER(mw_solve_opts), _P, _P, C.POINTER(mw_solve_stats)]),
    "mw_solve_rhs": (C.c_int32, [_P, C.POINTER(mw_solve_opts), C.c_int32, _P, _P, C.POINTER(mw_solve_stats)]),
    "mw_gradient": (C.c_int32, [_P, C.POINTER(mw_solve_opts), _P, _P, C.c_double, C.POINTER(C.c_double), _P, _P]),
    "mw_tikhonov": (C.c_int32, [_P, _P, C.POINTER(C.c_double), _P]),
    "mw_lbfgs_create": (C.c_int32, [C.POINTER(_P), C.c_int64, C.POINTER(mw_inv_opts)]),
    "mw_lbfgs_step": (C.c_int32, [_P, _P, C.c_double, _P, C.POINTER(C.c_int32)]),
    "mw_lbfgs_destroy": (None, [_P]),
    "mw_invert": (C.c_int32, [_P, C.POINTER(mw_inv_opts), C.POINTER(mw_solve_opts), _P, _P, _P,
                              C.POINTER(mw_inv_history)]),
    "mw_set_adjoint_mode": (C.c_int32, [_P, C.c_int32]),
    "mw_set_z_storage": (C.c_int32, [_P, C.c_int32]),
    "mw_set_sweep_schedule": (C.c_int32, [_P, C.c_int32]),
    "mw_forward_cols": (C.c_int32, [_P, C.POINTER(mw_solve_opts), C.c_int32, C.c_int32, _P]),
    "mw_gradient_cols": (C.c_int32, [_P, C.POINTER(mw_solve_opts), _P, _P, _P, C.POINTER(C.c_double), _P]),
    "mw_assemble_dev": (C.c_int32, [_P, C.c_int32, _P, _P, _P]),
    "mw_gradient_dev": (C.c_int32, [_P, C.POINTER(mw_solve_opts), _P, _P, C.c_double, C.POINTER(C.c_double), _P]),
    "mw_kernel_launches": (C.c_int64, []),
    "mw_profile_enable": (C.c_int32, [_P, C.c_uint32]),
    "mw_profile_read": (C.c_int32, [_P, _P, _P, _P, _P]),
    "mw_apply_preconditioner_noalloc": (C.c_int32, [_P, C.c_int32, _P, _P, C.c_int32]),
    "mw_krylov_dots": (C.c_int32, [_P, C.c_int32, _P, C.c_int64, _P, C.c_int64, C.c_int32, _P]),
    "mw_selftest_bounded_wait": (C.c_int32, [_P, C.c_int64, C.POINTER(C.c_int32)]),
    "mw_nn_param_count": (C.c_int64, [C.c_int32]),
    "mw_sparse_plan_stats": (C.c_int32, [C.c_int64, _P, C.c_int64, _P, C.c_int32, _P, C.c_int32, C.c_int32, _P]),
    "mw_spmm_plan_stats": (C.c_int32, [C.c_int64, _P, C.c_int64, _P, C.c_int32, _P]),
    "mw_nn_init": (C.c_int32, [_P, C.c_int32, _P]),
    "mw_nn_get_params": (C.c_int32, [_P, _P]),
    "mw_nn_loss_grad": (C.c_int32, [_P, C.c_int64, _P, _P, C.POINTER(C.c_double), _P]),
    "mw_nn_train": (C.c_int32, [_P, C.POINTER(mw_nn_opts), C.c_int64, _P, _P, C.POINTER(mw_nn_stats)]),
    "mw_nn_infer": (C.c_int32, [_P, C.c_int64, _P, _P]),
    "mw_nn_grid_to_tets": (C.c_int32, [_P, _P, C.c_int32, _P, _P]),
}

MW_ADJOINT_SOLVE, MW_ADJOINT_RECIPROCAL = 0, 1
(MW_K_SPMM, MW_K_ORAS, MW_K_CGS_DOTS, MW_K_CGS_UPDATE, MW_K_RESIDUAL, MW_K_REASSEMBLE, MW_K_GRADIENT, MW_K_FACTOR,
 MW_K_NN_GEMM, MW_K_NN_CONV, MW_K_NN_OTHER, MW_K_NCLASS) = range(12)
K_CLASS_NAMES = ("spmm", "oras_apply", "cgs_dots", "cgs_update", "residual_fp64", "reassemble", "gradient",
                 "factor", "nn_gemm", "nn_conv", "nn_other")

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmw.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmw.so not built at {path}; run paper_2311_05322_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _ptr(a) -> int | None:
    """Host numpy array or device torch tensor -> raw pointer (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous, "host arrays must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "device tensors must be contiguous"
        return a.data_ptr()
    raise TypeError(type(a))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def solve_opts(mode=MW_MODE_FP64, restart=50, batch=0, max_it=5000, tol=1e-8, inner_tol=1e-2, max_outer=20,
               use_precond=1) -> mw_solve_opts:
    return mw_solve_opts(mode, restart, batch, max_it, tol, inner_tol, max_outer, use_precond)


class Context:
    """One libmw context on one device and stream."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.lib = load_library()
        self.h = _P()
        self._check(self.lib.mw_create(C.byref(self.h), device, stream))
        self.info = None
        self.n_freq = 0
        self.n_src = 0

    def close(self):
        if self.h:
            self.lib.mw_destroy(self.h)
            self.h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, allow=()):
        if st != MW_OK and st not in allow:
            msg = self.lib.mw_last_error(self.h).decode() if self.h else "mw_create failed"
            raise MWError(st, msg)
        return st

    # -- mesh -----------------------------------------------------------------------------
    def set_mesh(self, xyz: np.ndarray, tets: np.ndarray) -> mw_mesh_info:
        xyz = _c(xyz, np.float64)
        tets = _c(tets, np.int32)
        info = mw_mesh_info()
        self._check(self.lib.mw_set_mesh(self.h, xyz.shape[0], _ptr(xyz), tets.shape[0], _ptr(tets), C.byref(info)))
        self.info = info
        return info

    def set_memory_cap(self, nbytes: int):
        self._check(self.lib.mw_set_memory_cap(self.h, int(nbytes)))

    def set_autotune(self, enable: bool):
        """Tune launch shapes at the first solve of each block shape (default) or use defaults."""
        self._check(self.lib.mw_set_autotune(self.h, 1 if enable else 0))

    def autotune(self, n_cols: int, mode: int = MW_MODE_MIXED, restart: int = 50) -> dict:
        """Tune the launch shapes of one block shape now; returns the choices and, per kernel, the
        mean device time per launch of every candidate."""
        r = mw_tune_report()
        self._check(self.lib.mw_autotune(self.h, n_cols, mode, restart, C.byref(r)))
        out = {k: getattr(r.chosen, k) for k, _ in mw_launch_shapes._fields_}
        for k, name in enumerate(TUNE_KERNELS):
            out[name + "_ms"] = {int(r.cand[k][i]): float(r.ms[k][i]) for i in range(r.n_cand[k])}
        return out

    def set_launch_shapes(self, n_cols: int, mode: int, restart: int, tc_stages: int = 0, dots_stages: int = 0,
                          update_stages: int = 0, spmm_threads: int = 0):
        """Pin the launch shapes of one block shape (0 = the kernel's default)."""
        sh = mw_launch_shapes(tc_stages, dots_stages, update_stages, spmm_threads)
        self._check(self.lib.mw_set_launch_shapes(self.h, n_cols, mode, restart, C.byref(sh)))

    def set_graphs(self, enable: bool):
        """Replay restart cycles from captured CUDA graphs, or run them eagerly (the default)."""
        self._check(self.lib.mw_set_graphs(self.h, 1 if enable else 0))

    def get_topology(self):
        i = self.info
        ev = np.empty((i.n_edge, 2), np.int32)
        te = np.empty((i.n_tet, 6), np.int32)
        ts = np.empty((i.n_tet, 6), np.int8)
        rp = np.empty(i.n_edge + 1, np.int64)
        ci = np.empty(i.nnz, np.int32)
        self._check(self.lib.mw_get_topology(self.h, _ptr(ev), _ptr(te), _ptr(ts), _ptr(rp), _ptr(ci)))
        return ev, te, ts, rp, ci

    def get_element_matrices(self):
        T = self.info.n_tet
        K = np.empty((T, 6, 6))
        M = np.empty((T, 6, 6))
        vol = np.empty(T)
        self._check(self.lib.mw_get_element_matrices(self.h, _ptr(K), _ptr(M), _ptr(vol)))
        return K, M, vol

    # -- assembly -------------------------------------------------------------------------
    def assemble(self, freqs, eps_r: np.ndarray, eps_bg: complex):
        fr = _c(np.atleast_1d(freqs), np.float64)
        e = _c(eps_r, np.float64)
        bg = np.array([complex(eps_bg).real, complex(eps_bg).imag])
        self._check(self.lib.mw_assemble(self.h, fr.size, _ptr(fr), _ptr(e), _ptr(bg)))
        self.n_freq = fr.size

    def get_matrix(self, f: int = 0) -> np.ndarray:
        v = np.empty(self.info.nnz, np.complex128)
        self._check(self.lib.mw_get_matrix(self.h, f, _ptr(v)))
        return v

    def apply_matrix(self, f: int, prec: int, x, y, n_cols: int):
        self._check(self.lib.mw_apply_matrix(self.h, f, prec, _ptr(x), _ptr(y), n_cols))

    # -- sources --------------------------------------------------------------------------
    def set_sources(self, pos: np.ndarray, direc: np.ndarray):
        pos = _c(pos, np.float64)
        direc = _c(direc, np.float64)
        n = pos.shape[0]
        e = np.empty(n, np.int32)
        s = np.empty(n, np.int8)
        self._check(self.lib.mw_set_sources(self.h, n, _ptr(pos), _ptr(direc), _ptr(e), _ptr(s)))
        self.n_src = n
        self.src_edges, self.src_signs = e, s
        return e, s

    def set_ports(self, origin, u, v, a, eps_fill, face_vert, face_label):
        """Waveguide ports and metal faces (mw_set_ports): per-port origin/u/v [P, 3], width a [P],
        filling eps_fill [P] complex; faces [n, 3] with labels -1 (metal) or the port index."""
        a = np.atleast_1d(np.asarray(a, dtype=np.float64))
        P = a.shape[0]
        arr = (mw_port * max(P, 1))()
        for p in range(P):
            e = complex(np.atleast_1d(eps_fill)[p])
            arr[p] = mw_port((C.c_double * 3)(*np.asarray(origin[p], float)), (C.c_double * 3)(*np.asarray(u[p], float)),
                             (C.c_double * 3)(*np.asarray(v[p], float)), float(a[p]), (C.c_double * 2)(e.real, e.imag))
        fv = _c(np.asarray(face_vert).reshape(-1, 3), np.int32)
        lab = _c(face_label, np.int32)
        assert lab.shape[0] == fv.shape[0]
        self._check(self.lib.mw_set_ports(self.h, P, arr, fv.shape[0], _ptr(fv), _ptr(lab)))
        if P:
            self.n_src = P
        self.n_freq = 0

    def get_port_vectors(self):
        W = np.empty((self.info.n_edge, self.n_src))
        n = np.empty(self.n_src)
        self._check(self.lib.mw_get_port_vectors(self.h, _ptr(W), _ptr(n)))
        return W, n

    # -- preconditioner -------------------------------------------------------------------
    def setup_preconditioner(self, n_sub: int, tet_part: np.ndarray, overlap: int, inv_prec: int):
        p = _c(tet_part, np.int32)
        self._check(self.lib.mw_setup_preconditioner(self.h, n_sub, _ptr(p), overlap, inv_prec))
        self.n_sub = n_sub

    def apply_preconditioner(self, f: int, r, z, n_cols: int):
        self._check(self.lib.mw_apply_preconditioner(self.h, f, _ptr(r), _ptr(z), n_cols))

    def apply_preconditioner_noalloc(self, f: int, r, z, n_cols: int):
        """Allocation-free apply (complex64 device in/out, BF16 preconditioner only)."""
        self._check(self.lib.mw_apply_preconditioner_noalloc(self.h, f, _ptr(r), _ptr(z), n_cols))

    def krylov_dots(self, V, w, nvec: int, vstride: int, n_rows: int, n_cols: int) -> np.ndarray:
        """h[i][c] = V_i[:, c]^H w[:, c] for i < nvec (complex64 device inputs, the solver's
        streaming dots kernel); returns complex128 [nvec][n_cols]."""
        h = np.empty((nvec, n_cols), np.complex128)
        self._check(self.lib.mw_krylov_dots(self.h, nvec, _ptr(V), vstride, _ptr(w), n_rows, n_cols, _ptr(h)))
        return h

    def get_partition(self):
        owner = np.empty(self.info.n_edge, np.int32)
        sizes = np.empty(self.n_sub, np.int32)
        self._check(self.lib.mw_get_partition(self.h, _ptr(owner), _ptr(sizes)))
        return owner, sizes

    # -- solves ---------------------------------------------------------------------------
    def _stats(self, n):
        st = mw_solve_stats()
        its = np.zeros(n, np.int32)
        rel = np.zeros(n)
        st.iters = its.ctypes.data_as(C.POINTER(C.c_int32))
        st.relres = rel.ctypes.data_as(C.POINTER(C.c_double))
        return st, its, rel

    def solve(self, opts: mw_solve_opts | None = None, fields=None, want_S: bool = True, allow_noconv=False):
        o = opts or solve_opts()
        n = self.n_freq * self.n_src
        st, its, rel = self._stats(n)
        S = np.empty((self.n_freq, self.n_src, self.n_src), np.complex128) if want_S else None
        code = self._check(self.lib.mw_solve(self.h, C.byref(o), _ptr(fields), _ptr(S), C.byref(st)),
                           allow=(MW_ENOCONV,) if allow_noconv else ())
        return S, {"n_cols": st.n_cols, "n_converged": st.n_converged, "outer_steps": st.outer_steps,
                   "arnoldi_steps": st.arnoldi_steps, "max_relres": st.max_relres, "solve_ms": st.solve_ms,
                   "iters": its, "relres": rel, "status": code}

    def solve_rhs(self, n_cols: int, b, x, opts: mw_solve_opts | None = None, allow_noconv=False):
        o = opts or solve_opts()
        st, its, rel = self._stats(self.n_freq * n_cols)
        code = self._check(self.lib.mw_solve_rhs(self.h, C.byref(o), n_cols, _ptr(b), _ptr(x), C.byref(st)),
                           allow=(MW_ENOCONV,) if allow_noconv else ())
        return {"n_converged": st.n_converged, "max_relres": st.max_relres, "solve_ms": st.solve_ms,
                "arnoldi_steps": st.arnoldi_steps, "iters": its, "relres": rel, "status": code}

    # -- cost, gradient, inversion -----------------------------------------------------------
    def gradient(self, S_obs, S_empty, alpha: float = 0.0, opts: mw_solve_opts | None = None, want_S=False,
                 out: np.ndarray | None = None):
        """J and dJ/d(Re eps, Im eps) [T, 2]; `out` (float64 [T, 2], C order, e.g. pinned host
        memory) receives the gradient instead of a new array."""
        o = opts or solve_opts()
        So = _c(S_obs, np.complex128)
        Se = _c(S_empty, np.complex128)
        J = C.c_double()
        if out is not None:
            if out.dtype != np.float64 or out.shape != (self.info.n_tet, 2) or not out.flags.c_contiguous:
                raise ValueError("out must be a C-contiguous float64 array of shape [n_tet, 2]")
            g = out
        else:
            g = np.empty((self.info.n_tet, 2))
        S = np.empty_like(So) if want_S else None
        self._check(self.lib.mw_gradient(self.h, C.byref(o), _ptr(So), _ptr(Se), alpha, C.byref(J), _ptr(g), _ptr(S)))
        return (J.value, g, S) if want_S else (J.value, g)

    def set_adjoint_mode(self, reciprocal: bool):
        """Adjoint fields by explicit solves (default) or by reciprocity from the forward fields."""
        self._check(self.lib.mw_set_adjoint_mode(self.h, MW_ADJOINT_RECIPROCAL if reciprocal else MW_ADJOINT_SOLVE))

    def set_sweep_schedule(self, persistent: bool):
        """Tensor-core sweeps of the sparse preconditioner: persistent CTAs (default) or one CTA
        per output tile (bit-identical)."""
        self._check(self.lib.mw_set_sweep_schedule(self.h, 1 if persistent else 0))

    def set_z_storage(self, bf16: bool):
        """Preconditioned Krylov vectors of the tensor-core path stored in BF16 (default) or FP32."""
        self._check(self.lib.mw_set_z_storage(self.h, 1 if bf16 else 0))

    def forward_cols(self, j0: int, n_cols: int, opts: mw_solve_opts | None = None) -> np.ndarray:
        """Forward solves of transmitters j0 .. j0+n_cols-1; returns their S columns
        [n_freq][n_src][n_cols]."""
        o = opts or solve_opts()
        S = np.empty((self.n_freq, self.n_src, n_cols), np.complex128)
        self._check(self.lib.mw_forward_cols(self.h, C.byref(o), j0, n_cols, _ptr(S)))
        return S

    def gradient_cols(self, S_full, S_obs, S_empty, opts: mw_solve_opts | None = None):
        """Cost of the whole S and the last window's share of the data gradient [n_tet][2]."""
        o = opts or solve_opts()
        J = C.c_double()
        g = np.empty((self.info.n_tet, 2))
        self._check(self.lib.mw_gradient_cols(self.h, C.byref(o), _ptr(_c(S_full, np.complex128)),
                                              _ptr(_c(S_obs, np.complex128)), _ptr(_c(S_empty, np.complex128)),
                                              C.byref(J), _ptr(g)))
        return J.value, g

    def tikhonov(self, eps_r):
        e = _c(eps_r, np.float64)
        R = C.c_double()
        g = np.empty_like(e)
        self._check(self.lib.mw_tikhonov(self.h, _ptr(e), C.byref(R), _ptr(g)))
        return R.value, g

    def selftest_bounded_wait(self, spins: int) -> int:
        code = C.c_int32()
        self._check(self.lib.mw_selftest_bounded_wait(self.h, spins, C.byref(code)))
        return code.value

    # -- learned initialiser -----------------------------------------------------------------
    def nn_init(self, n_in: int, theta: np.ndarray):
        th = _c(theta, np.float32)
        assert th.size == self.lib.mw_nn_param_count(n_in)
        self._check(self.lib.mw_nn_init(self.h, n_in, _ptr(th)))
        self.nn_in = n_in

    def nn_get_params(self) -> np.ndarray:
        th = np.empty(self.lib.mw_nn_param_count(self.nn_in), np.float32)
        self._check(self.lib.mw_nn_get_params(self.h, _ptr(th)))
        return th

    def nn_loss_grad(self, x, t):
        x = _c(x, np.float32)
        t = _c(t, np.float32)
        L = C.c_double()
        g = np.empty(self.lib.mw_nn_param_count(self.nn_in), np.float32)
        self._check(self.lib.mw_nn_loss_grad(self.h, x.shape[0], _ptr(x), _ptr(t), C.byref(L), _ptr(g)))
        return L.value, g

    def nn_train(self, x, t, batch=64, epochs=10, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=1):
        x = _c(x, np.float32)
        t = _c(t, np.float32)
        losses = np.zeros(max(epochs, 1))
        st = mw_nn_stats(0, losses.ctypes.data_as(C.POINTER(C.c_double)), 0.0)
        o = mw_nn_opts(batch, epochs, lr, beta1, beta2, eps, seed)
        self._check(self.lib.mw_nn_train(self.h, C.byref(o), x.shape[0], _ptr(x), _ptr(t), C.byref(st)))
        return losses[:epochs].copy(), st.seconds

    def nn_infer(self, x) -> np.ndarray:
        x = _c(x, np.float32)
        y = np.empty((x.shape[0], 2, 32, 32, 32), np.float32)
        self._check(self.lib.mw_nn_infer(self.h, x.shape[0], _ptr(x), _ptr(y)))
        return y

    def nn_grid_to_tets(self, grid, box) -> np.ndarray:
        g = _c(grid, np.float32)
        b = _c(box, np.float64)
        out = np.empty((self.info.n_tet, 2))
        self._check(self.lib.mw_nn_grid_to_tets(self.h, _ptr(g), g.shape[-1], _ptr(b), _ptr(out)))
        return out

    # -- device-resident variants -----------------------------------------------------------
    def assemble_dev(self, freqs, eps_dev, eps_bg: complex):
        fr = _c(np.atleast_1d(freqs), np.float64)
        bg = np.array([complex(eps_bg).real, complex(eps_bg).imag])
        self._check(self.lib.mw_assemble_dev(self.h, fr.size, _ptr(fr), _ptr(eps_dev), _ptr(bg)))

    def gradient_dev(self, S_obs_dev, S_empty_dev, grad_dev, alpha: float = 0.0, opts: mw_solve_opts | None = None):
        o = opts or solve_opts()
        J = C.c_double()
        self._check(self.lib.mw_gradient_dev(self.h, C.byref(o), _ptr(S_obs_dev), _ptr(S_empty_dev), alpha,
                                             C.byref(J), _ptr(grad_dev)))
        return J.value

    # -- event profiler -----------------------------------------------------------------------
    def profile_enable(self, mask: int):
        self._check(self.lib.mw_profile_enable(self.h, mask))

    def profile_read(self):
        ms = np.zeros(MW_K_NCLASS)
        n = np.zeros(MW_K_NCLASS, np.int64)
        b = np.zeros(MW_K_NCLASS)
        fl = np.zeros(MW_K_NCLASS)
        self._check(self.lib.mw_profile_read(self.h, _ptr(ms), _ptr(n), _ptr(b), _ptr(fl)))
        return {K_CLASS_NAMES[k]: {"ms": float(ms[k]), "launches": int(n[k]), "bytes": float(b[k]),
                                   "flops": float(fl[k])}
                for k in range(MW_K_NCLASS)}

    def invert(self, S_obs, S_empty, eps0, inv: mw_inv_opts, opts: mw_solve_opts | None = None):
        o = opts or solve_opts()
        So = _c(S_obs, np.complex128)
        Se = _c(S_empty, np.complex128)
        eps = _c(eps0, np.float64).copy()
        Jh = np.zeros(inv.max_it + 1)
        th = np.zeros(inv.max_it + 1)
        hist = mw_inv_history(0, 0, Jh.ctypes.data_as(C.POINTER(C.c_double)), th.ctypes.data_as(C.POINTER(C.c_double)))
        self._check(self.lib.mw_invert(self.h, C.byref(inv), C.byref(o), _ptr(So), _ptr(Se), _ptr(eps), C.byref(hist)))
        k = hist.iterations
        return eps, {"iterations": k, "evaluations": hist.evaluations, "J": Jh[:k + 1].copy(),
                     "seconds": th[:k + 1].copy()}


def spmm_plan_stats(xyz, tets, halo_max: int = 480) -> dict:
    """Host-only check and statistics of the halo-tiled SpMM plan (mw_spmm_plan_stats)."""
    lib = load_library()
    xyz = _c(xyz, np.float64)
    tets = _c(tets, np.int32)
    out = np.zeros(4, np.int64)
    st = lib.mw_spmm_plan_stats(xyz.shape[0], _ptr(xyz), tets.shape[0], _ptr(tets), halo_max, _ptr(out))
    if st != MW_OK:
        raise MWError(st, "SpMM plan check failed")
    return dict(zip(("blocks", "halo_total", "halo_max", "nnz"), (int(v) for v in out)))


def sparse_plan_stats(xyz, tets, n_sub: int, tet_part, overlap: int, leaf: int = 256) -> dict:
    """Host-only check and statistics of the sparse subdomain plan (mw_sparse_plan_stats)."""
    lib = load_library()
    xyz = _c(xyz, np.float64)
    tets = _c(tets, np.int32)
    part = _c(tet_part, np.int32)
    out = np.zeros(6, np.int64)
    st = lib.mw_sparse_plan_stats(xyz.shape[0], _ptr(xyz), tets.shape[0], _ptr(tets), n_sub, _ptr(part), overlap,
                                  leaf, _ptr(out))
    if st != MW_OK:
        raise MWError(st, "sparse plan check failed")
    return dict(zip(("nodes", "height", "max_front", "factor_entries", "max_workspace", "dense_entries"),
                    (int(v) for v in out)))


def kernel_launches() -> int:
    return int(load_library().mw_kernel_launches())


class LBFGS:
    """Reverse-communication L-BFGS of libmw (host FP64)."""

    def __init__(self, n: int, opts: mw_inv_opts):
        self.lib = load_library()
        self.h = _P()
        st = self.lib.mw_lbfgs_create(C.byref(self.h), n, C.byref(opts))
        if st != MW_OK:
            raise MWError(st, "mw_lbfgs_create")

    def step(self, x: np.ndarray, f: float, g: np.ndarray) -> bool:
        req = C.c_int32()
        gg = _c(g, np.float64)
        st = self.lib.mw_lbfgs_step(self.h, _ptr(x), float(f), _ptr(gg), C.byref(req))
        if st != MW_OK:
            raise MWError(st, "mw_lbfgs_step")
        return bool(req.value)

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.mw_lbfgs_destroy(self.h)
            self.h = _P()


def inv_opts(m=8, max_it=20, c1=1e-4, max_ls=10, first_step=1.0, alpha=0.0, target_J=0.0) -> mw_inv_opts:
    return mw_inv_opts(m, max_it, c1, max_ls, first_step, alpha, target_J)
