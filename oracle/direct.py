"""O1: direct dense solver for H x = lam S x (test infrastructure only; see oracle/__init__).

The quantity ChFSI computes has a plain definition: the nev smallest eigenpairs of the
Hermitian-definite pencil (H, S) (Section 2, the generalized problems P^(l) of a FLAPW
self-consistent cycle; Algorithm 1 Ensure: the wanted eigenpairs).  This module writes that
definition out the textbook way:

1. S = L L^H by the Cholesky algorithm (the reduction "B = L L^T" of Section 3, read with
   ^H for complex Hermitian matrices).
2. H' = L^{-1} H L^{-H} by forward substitution (Section 3, standard form).
3. Householder reduction of H' to Hermitian tridiagonal form, then a diagonal unitary
   scaling that makes it real symmetric tridiagonal.
4. Implicit symmetric tridiagonal QR with Wilkinson shifts (C, oracle/tridiag.c).
5. Ascending sort; eigenvectors x = L^{-H} y.

Pins (tests/test_oracle_direct.py): prescribed spectra, 2x2 closed form, diagonal and
block-diagonal matrices, agreement with cyclic Jacobi (independent algorithm) and with
LAPACK via scipy.linalg.eigh (library special case), Sylvester inertia counts, brute-force
bisection on tiny matrices, S-orthonormality and residuals.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_lib = None


def _clib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.oracle_tridiag_qr.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int]
        _lib.oracle_tridiag_qr.restype = ctypes.c_int
        _lib.oracle_jacobi_hermitian.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        _lib.oracle_jacobi_hermitian.restype = ctypes.c_int
    return _lib


class NotPositiveDefinite(ValueError):
    pass


def cholesky(S: np.ndarray) -> np.ndarray:
    """Lower-triangular L with S = L L^H (column-by-column Cholesky).  Section 3 reduction.

    Raises NotPositiveDefinite on a non-positive pivot."""
    S = np.asarray(S, dtype=np.complex128)
    n = S.shape[0]
    L = np.zeros_like(S)
    for j in range(n):
        piv = S[j, j].real - np.sum(np.abs(L[j, :j]) ** 2)
        if not piv > 0.0:
            raise NotPositiveDefinite(f"pivot {j} = {piv}")
        L[j, j] = np.sqrt(piv)
        if j + 1 < n:
            L[j + 1:, j] = (S[j + 1:, j] - L[j + 1:, :j] @ L[j, :j].conj()) / L[j, j].real
    return L


def forward_solve(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with L X = B, L lower triangular (row-by-row forward substitution)."""
    n = L.shape[0]
    X = np.zeros(B.shape, dtype=np.complex128)
    for i in range(n):
        X[i] = (B[i] - L[i, :i] @ X[:i]) / L[i, i]
    return X


def backward_solve_h(L: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """X with L^H X = Y (back substitution on the upper-triangular L^H)."""
    n = L.shape[0]
    X = np.zeros(Y.shape, dtype=np.complex128)
    for i in range(n - 1, -1, -1):
        X[i] = (Y[i] - L[i + 1:, i].conj() @ X[i + 1:]) / np.conj(L[i, i])
    return X


def reduce_to_standard(H: np.ndarray, L: np.ndarray) -> np.ndarray:
    """H' = L^{-1} H L^{-H}, Hermitian part taken (Section 3, standard form)."""
    W = forward_solve(L, H)                 # L^{-1} H
    Hs = forward_solve(L, W.conj().T)       # L^{-1} (L^{-1} H)^H = L^{-1} H L^{-H}
    return 0.5 * (Hs + Hs.conj().T)


def householder_tridiagonal(A: np.ndarray):
    """A = Q T Q^H with T Hermitian tridiagonal.

    Returns (diag, offdiag, vs): diag real (n,), offdiag complex (n-1,) with
    T[k+1, k] = offdiag[k], and the unit Householder vectors vs[k] acting on rows k+1..n-1,
    Q = (I - 2 v_0 v_0^H)(I - 2 v_1 v_1^H)...  (Golub & Van Loan sec. 8.3.1)."""
    A = np.array(A, dtype=np.complex128, copy=True)
    n = A.shape[0]
    vs = []
    off = np.zeros(max(n - 1, 0), dtype=np.complex128)
    for k in range(n - 2):
        x = A[k + 1:, k].copy()
        nx = np.linalg.norm(x)
        ph = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -ph * nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv == 0.0:
            vs.append(None)
            off[k] = x[0]
            continue
        v /= nv
        vs.append(v)
        off[k] = alpha
        A[k + 1:, k] = 0.0
        A[k, k + 1:] = 0.0
        A22 = A[k + 1:, k + 1:]
        p = A22 @ v
        K = np.vdot(v, p).real
        w = 2.0 * p - 2.0 * K * v
        A22 -= np.outer(v, w.conj()) + np.outer(w, v.conj())
    if n >= 2:
        off[n - 2] = A[n - 1, n - 2]
    return np.real(np.diagonal(A)).copy(), off, vs


def tridiagonal_eig(d: np.ndarray, e: np.ndarray, vectors: bool = True):
    """Eigen-decomposition of the real symmetric tridiagonal (d, e) by implicit QR (C)."""
    n = d.size
    d = np.ascontiguousarray(d, dtype=np.float64).copy()
    e = np.ascontiguousarray(np.append(e, 0.0) if e.size < max(n, 1) else e, dtype=np.float64).copy()
    z = np.asfortranarray(np.eye(n)) if vectors else None
    rc = _clib().oracle_tridiag_qr(n, d.ctypes.data, e.ctypes.data,
                                   z.ctypes.data if vectors else None, n)
    if rc != 0:
        raise RuntimeError("tridiagonal QR did not converge")
    order = np.argsort(d, kind="stable")
    return (d[order], z[:, order]) if vectors else d[order]


def hermitian_eig(A: np.ndarray, vectors: bool = True):
    """All eigenpairs of a complex Hermitian matrix, ascending (Householder + implicit QR)."""
    n = A.shape[0]
    d, off, vs = householder_tridiagonal(A)
    # diagonal unitary D with D^H T D real: d_{j+1} = d_j * off_j / |off_j|
    ph = np.ones(n, dtype=np.complex128)
    for j in range(n - 1):
        ph[j + 1] = ph[j] * (off[j] / abs(off[j]) if off[j] != 0 else 1.0)
    res = tridiagonal_eig(d, np.abs(off), vectors)
    if not vectors:
        return res
    lam, z = res
    Y = ph[:, None] * z.astype(np.complex128)
    for k in range(len(vs) - 1, -1, -1):
        v = vs[k]
        if v is None:
            continue
        Y[k + 1:] -= 2.0 * np.outer(v, v.conj() @ Y[k + 1:])
    return lam, Y


def jacobi_eig(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """All eigenpairs by cyclic complex Jacobi (C), ascending.  Independent cross-check."""
    n = A.shape[0]
    a = np.asfortranarray(np.array(A, dtype=np.complex128))
    v = np.asfortranarray(np.zeros((n, n), dtype=np.complex128))
    w = np.zeros(n)
    rc = _clib().oracle_jacobi_hermitian(n, a.ctypes.data, v.ctypes.data, w.ctypes.data, tol, max_sweeps)
    if rc < 0:
        raise RuntimeError("Jacobi did not converge")
    order = np.argsort(w, kind="stable")
    return w[order], v[:, order]


def generalized_eig(H: np.ndarray, S: np.ndarray, nev: int | None = None, vectors: bool = True):
    """The nev smallest eigenpairs of H x = lam S x (all when nev is None), ascending.

    Eigenvectors are S-orthonormal: X^H S X = I."""
    L = cholesky(S)
    Hs = reduce_to_standard(H, L)
    if not vectors:
        lam = hermitian_eig(Hs, vectors=False)
        return lam if nev is None else lam[:nev]
    lam, Y = hermitian_eig(Hs, vectors=True)
    if nev is not None:
        lam, Y = lam[:nev], Y[:, :nev]
    return lam, backward_solve_h(L, Y)


def inertia_below(A: np.ndarray, sigma: float, B: np.ndarray | None = None) -> int:
    """Number of eigenvalues of A (or of the pencil (A, B)) below sigma.

    Sylvester's law of inertia: the count of negative pivots of the LDL^H factorisation of
    A - sigma B (no pivoting)."""
    M = np.array(A, dtype=np.complex128, copy=True)
    n = M.shape[0]
    M -= sigma * (np.eye(n) if B is None else B)
    neg = 0
    for j in range(n):
        dj = M[j, j].real
        if dj == 0.0:
            dj = 1e-300
        if dj < 0.0:
            neg += 1
        if j + 1 < n:
            col = M[j + 1:, j] / dj
            M[j + 1:, j + 1:] -= dj * np.outer(col, col.conj())
    return neg


def generalized_residuals(H, S, lam, X):
    """||H x_i - lam_i S x_i||_2 / ||H x_i||_2 per column (the acceptance measure)."""
    HX = H @ X
    R = HX - (S @ X) * lam[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(HX, axis=0)
