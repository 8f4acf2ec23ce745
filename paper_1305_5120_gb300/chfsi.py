"""ctypes binding of libchfsi.so (include/chfsi.h): argument marshalling only.

Device memory and streams come from PyTorch; every step of the computation runs in the
library's CUDA kernels.  The library must be built (``paper_1305_5120_gb300.build``); there
is no CPU fallback: on a machine without the library or without a GPU every call raises.

Matrices cross the boundary as complex128, column-major.  A torch tensor of shape
(cols, rows) in row-major memory is exactly that layout, so ``colmajor(A)`` uploads the
mathematical matrix A (rows x cols) as ``A.T`` and ``to_numpy`` undoes it.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CHFSI_PREC_FP64 = 0
CHFSI_PREC_MIXED = 1

STATUS = {0: "ok", 1: "invalid argument", 2: "S not HPD", 3: "not converged", 4: "out of memory",
          5: "CUDA error", 6: "device wait timed out", 7: "call out of order", 8: "non-finite value",
          9: "completeness check failed"}


class ChfsiError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int), ("degree_min", ctypes.c_int), ("degree_max", ctypes.c_int),
                ("per_vector_degree", ctypes.c_int), ("max_iter", ctypes.c_int), ("lanczos_steps", ctypes.c_int),
                ("precision", ctypes.c_int), ("mixed_switch", ctypes.c_double), ("seed", ctypes.c_ulonglong),
                ("check_inertia", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("locked", ctypes.c_int), ("filter_col_steps", ctypes.c_longlong),
                ("filter_col_steps_lowp", ctypes.c_longlong), ("max_resid", ctypes.c_double),
                ("kappa_L", ctypes.c_double), ("bounds", ctypes.c_double * 3), ("ms_stage", ctypes.c_double * 8),
                ("ms_filter_lowp", ctypes.c_double), ("ms_gemm_tc", ctypes.c_double),
                ("gemm_tc_flop", ctypes.c_double), ("ms_eig", ctypes.c_double), ("eig_sweeps", ctypes.c_int),
                ("eig_rounds", ctypes.c_longlong), ("eig_flop", ctypes.c_double), ("n_floor", ctypes.c_int),
                ("completeness", ctypes.c_int), ("ms_filter_steps", ctypes.c_double),
                ("filter_step_cols", ctypes.c_longlong), ("eig_refined", ctypes.c_int),
                ("eig_refine_iters", ctypes.c_int), ("eig_f32_sweeps", ctypes.c_int), ("eig_fallbacks", ctypes.c_int),
                ("ms_chol", ctypes.c_double),
                ("chol_flop", ctypes.c_double)]

    def as_dict(self):
        return {"iterations": self.iterations, "locked": self.locked, "filter_col_steps": self.filter_col_steps,
                "filter_col_steps_lowp": self.filter_col_steps_lowp, "max_resid": self.max_resid,
                "kappa_L": self.kappa_L, "bounds": list(self.bounds), "ms_stage": list(self.ms_stage),
                "ms_filter_lowp": self.ms_filter_lowp, "ms_gemm_tc": self.ms_gemm_tc,
                "gemm_tc_flop": self.gemm_tc_flop, "ms_eig": self.ms_eig, "eig_sweeps": self.eig_sweeps,
                "eig_rounds": self.eig_rounds, "eig_flop": self.eig_flop, "n_floor": self.n_floor,
                "completeness": self.completeness, "ms_filter_steps": self.ms_filter_steps,
                "filter_step_cols": self.filter_step_cols, "eig_refined": self.eig_refined,
                "eig_refine_iters": self.eig_refine_iters, "eig_f32_sweeps": self.eig_f32_sweeps,
                "eig_fallbacks": self.eig_fallbacks,
                "ms_chol": self.ms_chol, "chol_flop": self.chol_flop}


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGS = {
    "chfsi_default_params": [ctypes.POINTER(Params)],
    "chfsi_create": [ctypes.POINTER(_P), _I, _P, ctypes.POINTER(Params)],
    "chfsi_solve": [_P, _P, _P, _I, _I, _I, _P, _D, _I, _P, _P, ctypes.POINTER(Info)],
    "chfsi_next_in_sequence": [_P, _P, _P, _P, _P, ctypes.POINTER(Info)],
    "chfsi_solve_batch": [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_I),
                          ctypes.POINTER(_I), _D, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I),
                          ctypes.POINTER(Info)],
    "chfsi_destroy": [_P],
    "chfsi_status_string": [_I],
    "chfsi_kernel_launches": [],
    "chfsi_fp64_peak": [_I, ctypes.POINTER(_D)],
    "chfsi_workspace_bytes": [_I, _I, _I, _I],
    "chfsi_gemm": [_P, ctypes.c_char, ctypes.c_char, _I, _I, _I, ctypes.POINTER(_D), _P, _I, _P, _I,
                   ctypes.POINTER(_D), _P, _I, _I],
    "chfsi_cholesky": [_P, _I, _P, _P],
    "chfsi_reduce": [_P, _I, _P, _P, _P],
    "chfsi_lanczos": [_P, _I, _P, _I, _I, _P, _P, _P, _P],
    "chfsi_filter": [_P, _I, _I, _P, _P, _I, _D, _D, _D, _I],
    "chfsi_filter_degrees": [_P, _I, _I, _P, _P, ctypes.POINTER(_I), _D, _D, _D, _I],
    "chfsi_filter_ritz": [_P, _I, _I, _P, _P, _P, _P, _I, _D, _D, _D],
    "chfsi_orthonormalize": [_P, _I, _I, _P, _I, _P],
    "chfsi_rayleigh_ritz": [_P, _I, _I, _P, _P, _P, _P],
    "chfsi_reduced_eig": [_P, _I, _P, _P, _P],
    "chfsi_reduced_eig_noalloc": [_P, _I, _P, _P, _P],
    "chfsi_residuals": [_P, _I, _I, _P, _P, _P, _P],
    "chfsi_degrees": [_P, _I, _P, _P, _D, _D, _D, _I, _I, _P],
    "chfsi_back_transform": [_P, _I, _I, _P, _P, _P],
}


def kernel_launches() -> int:
    return int(load().chfsi_kernel_launches())


def fp64_peak(device: int = 0) -> float:
    """Measured DFMA throughput of the device (TFLOP/s)."""
    out = _D()
    _check(load().chfsi_fp64_peak(device, ctypes.byref(out)), "chfsi_fp64_peak")
    return float(out.value)


def workspace_bytes(n, nev, nex, precision=CHFSI_PREC_MIXED) -> int:
    return int(load().chfsi_workspace_bytes(n, nev, nex, precision))


def exported_names():
    return list(_SIGS)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libchfsi.so (building it first when missing).  Raises when it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or build_if_missing:
        path = _build.build()
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = {"chfsi_status_string": ctypes.c_char_p, "chfsi_destroy": None,
                     "chfsi_kernel_launches": ctypes.c_ulonglong,
                     "chfsi_workspace_bytes": ctypes.c_size_t}.get(name, _I)
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        raise ChfsiError(status, where)


def _ptr(t) -> int | None:
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("device tensors (torch, CUDA) are required")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def colmajor(A, device="cuda"):
    """Upload the mathematical matrix A (rows x cols, numpy or torch) as a column-major
    complex128 device buffer (a torch tensor of shape (cols, rows))."""
    import torch
    t = torch.as_tensor(np.asarray(A) if not isinstance(A, torch.Tensor) else A)
    if t.dim() == 1:
        t = t[:, None]
    return t.to(torch.complex128).T.contiguous().to(device)


def to_numpy(t) -> np.ndarray:
    """Inverse of colmajor: device buffer of shape (cols, rows) -> numpy (rows, cols)."""
    return t.detach().cpu().numpy().T.copy()


def reduced_eig_noalloc(k, G, lam, W, stream=None) -> int:
    """Allocation-free reduced eigensolver (k <= 256); returns the chfsi_status code."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    return int(load().chfsi_reduced_eig_noalloc(_P(st.cuda_stream), k, _ptr(G), _ptr(lam), _ptr(W)))


def default_params(**kw) -> Params:
    p = Params()
    _check(load().chfsi_default_params(ctypes.byref(p)), "chfsi_default_params")
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Context:
    """One solver context (one sequence, one CUDA stream)."""

    def __init__(self, device: int = 0, stream=None, **params):
        import torch
        self.lib = load()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.params = default_params(**params)
        h = _P()
        _check(self.lib.chfsi_create(ctypes.byref(h), device, _P(self.stream.cuda_stream), ctypes.byref(self.params)),
               "chfsi_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.chfsi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- whole solves ---------------------------------------------------------------------
    def solve(self, H, S, n, nev, nex, X0=None, tol=1e-10, degree=0, evals=None, X=None):
        import torch
        evals = evals if evals is not None else torch.empty(nev, dtype=torch.float64, device=H.device)
        X = X if X is not None else torch.empty((nev, n), dtype=torch.complex128, device=H.device)
        info = Info()
        st = self.lib.chfsi_solve(self.h, _ptr(H), _ptr(S), n, nev, nex, _ptr(X0), tol, degree, _ptr(evals), _ptr(X),
                                  ctypes.byref(info))
        return st, evals, X, info

    def next_in_sequence(self, H_next, S_next=None, evals=None, X=None, nev=None, n=None):
        import torch
        evals = evals if evals is not None else torch.empty(nev, dtype=torch.float64, device=H_next.device)
        X = X if X is not None else torch.empty((nev, n), dtype=torch.complex128, device=H_next.device)
        info = Info()
        st = self.lib.chfsi_next_in_sequence(self.h, _ptr(H_next), _ptr(S_next), _ptr(evals), _ptr(X),
                                             ctypes.byref(info))
        return st, evals, X, info

    def solve_batch(self, Hs, Ss, ns, nevs, nexs, tol=1e-10, degree=0, evals=None, Xs=None):
        """Independent problems solved together (chfsi_solve_batch).  Hs, Ss: lists of device
        buffers (colmajor); returns (status of the call, per-problem statuses, evals, Xs, infos)."""
        import torch
        cnt = len(Hs)
        evals = evals if evals is not None else [torch.empty(nv, dtype=torch.float64, device=Hs[p].device)
                                                 for p, nv in enumerate(nevs)]
        Xs = Xs if Xs is not None else [torch.empty((nv, n), dtype=torch.complex128, device=Hs[p].device)
                                        for p, (n, nv) in enumerate(zip(ns, nevs))]
        arrP = lambda ts: (_P * cnt)(*[_ptr(t) for t in ts])
        arrI = lambda xs: (_I * cnt)(*[int(x) for x in xs])
        status = (_I * cnt)()
        infos = (Info * cnt)()
        st = self.lib.chfsi_solve_batch(self.h, cnt, arrP(Hs), arrP(Ss), arrI(ns), arrI(nevs), arrI(nexs), tol, degree,
                                        arrP(evals), arrP(Xs), status, infos)
        return st, list(status), evals, Xs, list(infos)

    # --- stages -------------------------------------------------------------------------------
    def gemm(self, opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, precision=CHFSI_PREC_FP64):
        al = (_D * 2)(complex(alpha).real, complex(alpha).imag)
        be = (_D * 2)(complex(beta).real, complex(beta).imag)
        _check(self.lib.chfsi_gemm(self.h, opA.encode(), opB.encode(), M, N, K, al, _ptr(A), lda, _ptr(B), ldb, be,
                                   _ptr(C), ldc, precision), "chfsi_gemm")

    def cholesky(self, n, S, L):
        _check(self.lib.chfsi_cholesky(self.h, n, _ptr(S), _ptr(L)), "chfsi_cholesky")

    def reduce(self, n, H, L, Hs):
        _check(self.lib.chfsi_reduce(self.h, n, _ptr(H), _ptr(L), _ptr(Hs)), "chfsi_reduce")

    def lanczos(self, n, Hs, steps, k, v0, alpha, beta, bounds):
        _check(self.lib.chfsi_lanczos(self.h, n, _ptr(Hs), steps, k, _ptr(v0), _ptr(alpha), _ptr(beta), _ptr(bounds)),
               "chfsi_lanczos")

    def filter(self, n, k, Hs, Y, m, a, b, a0, precision=CHFSI_PREC_FP64):
        _check(self.lib.chfsi_filter(self.h, n, k, _ptr(Hs), _ptr(Y), m, a, b, a0, precision), "chfsi_filter")

    def filter_degrees(self, n, k, Hs, Y, degrees, a, b, a0, precision=CHFSI_PREC_FP64):
        arr = (ctypes.c_int * k)(*[int(d) for d in degrees])
        _check(self.lib.chfsi_filter_degrees(self.h, n, k, _ptr(Hs), _ptr(Y), arr, a, b, a0, precision),
               "chfsi_filter_degrees")

    def filter_ritz(self, n, k, Hs, Y, lam, Z, m, a, b, a0):
        _check(self.lib.chfsi_filter_ritz(self.h, n, k, _ptr(Hs), _ptr(Y), _ptr(lam), _ptr(Z), m, a, b, a0),
               "chfsi_filter_ritz")

    def orthonormalize(self, n, nl, Ylocked, k, Y):
        _check(self.lib.chfsi_orthonormalize(self.h, n, nl, _ptr(Ylocked), k, _ptr(Y)), "chfsi_orthonormalize")

    def rayleigh_ritz(self, n, k, Hs, Y, lam, Z):
        _check(self.lib.chfsi_rayleigh_ritz(self.h, n, k, _ptr(Hs), _ptr(Y), _ptr(lam), _ptr(Z)),
               "chfsi_rayleigh_ritz")

    def reduced_eig(self, k, G, lam, W):
        _check(self.lib.chfsi_reduced_eig(self.h, k, _ptr(G), _ptr(lam), _ptr(W)), "chfsi_reduced_eig")

    def residuals(self, n, k, Z, Y, lam, res):
        _check(self.lib.chfsi_residuals(self.h, n, k, _ptr(Z), _ptr(Y), _ptr(lam), _ptr(res)), "chfsi_residuals")

    def degrees(self, k, lam, res, a, b, tol, m_min, m_max, deg):
        _check(self.lib.chfsi_degrees(self.h, k, _ptr(lam), _ptr(res), a, b, tol, m_min, m_max, _ptr(deg)),
               "chfsi_degrees")

    def back_transform(self, n, k, L, Y, X):
        _check(self.lib.chfsi_back_transform(self.h, n, k, _ptr(L), _ptr(Y), _ptr(X)), "chfsi_back_transform")
