"""O2: Chebyshev filtered subspace iteration with locking, straight from Algorithm 1.

Test infrastructure only (see oracle/__init__).  Written step by step in the paper's order
(Section 3, Algorithm 1) on the standard-form matrix H (the paper's H^(l) = L^{-1} A L^{-H}),
in FP64, with numpy matrix products and numpy's Householder QR as library primitives.

Readings of the paper used here (each is also listed in the design notes):

* The filter is the scaled and shifted form of the three-term recurrence of Eq. (3term)
  (Zhou, Saad, Tiago & Chelikowsky 2006, cited in Section 3): with e = (b - a)/2,
  c = (b + a)/2 the recurrence runs on (H - cI)/e and is normalised at a0, so that
  Y_m = T_m((H - cI)/e) Y_0 / T_m((a0 - c)/e).  With c = 0, e = 1 it is Eq. (3term) itself
  up to that scalar normalisation.  The shift is the "update of the diagonal" of Section 3.
* Lanczos (Algorithm 1 line "Estimating the largest eigenvalue"; Zhou & Li 2011): k_L
  steps, no reorthogonalisation, start vector from the SplitMix64 generator; upper bound
  b = top Ritz value + |beta_{k_L}| |z_last| (the residual norm of the top Ritz pair, z its
  eigenvector of T) + 1e-3 of the Ritz spread.  The condition estimate of L (kappa_L_estimate)
  keeps the plainer bound max Ritz value + |beta_{k_L}|, which is never smaller.
* The block holds nev + nex vectors; the lower end a of the damped interval is the largest
  Ritz value of the block, a0 (the normalisation point) the smallest.
* Res(y, lam) is the relative residual ||H y - lam y|| / max(||H y||, 1e-4 ||H||) (||H||
  estimated by max(|a0|, |b|)); a pair locks when it is below tol / kappa_L, where
  kappa_L >= cond_2(L) makes the generalized relative residual ||A x - lam B x|| / ||A x||
  <= tol (kappa_L = 1 for a standard problem) for every eigenvalue with |lam| >= 1e-4 ||H||;
  nearer to zero the test is absolute, since a relative 1e-10 is below FP64's reach there.
* Locking follows the loop "for i = converged to nev": every active Ritz pair whose global
  index is below nev and whose residual passes is locked, contiguous or not.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import direct

# --- counter-based generator: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) ---------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of SplitMix64 seeded with `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix_uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [-0.5, 0.5): top 53 bits of each output, scaled by 2^-53, minus 0.5."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 - 0.5


def splitmix_complex_block(seed: int, n: int, k: int, stream: int) -> np.ndarray:
    """n x k complex block, column-major draw order; element (i, j) takes outputs
    2*(j*n + i) (real part) and 2*(j*n + i) + 1 (imaginary part) of stream `stream`
    (the stream offsets the counter by stream * 2^40)."""
    u = splitmix_uniform(seed, 2 * n * k, offset=stream << 40)
    z = u[0::2] + 1j * u[1::2]
    return z.reshape(k, n).T.copy()


# --- Algorithm 1, line "Estimating the largest eigenvalue" (Lanczos) ----------------------
def lanczos(H: np.ndarray, v0: np.ndarray, steps: int):
    """k-step Lanczos from v0 (normalised here), no reorthogonalisation.  H is anything
    with ``H @ v`` (a matrix or an operator object).

    Returns (alpha, beta): T = tridiag(beta[:-1], alpha, beta[:-1]); beta[-1] is the norm of
    the last residual vector."""
    steps = min(steps, v0.shape[0])
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    alpha = np.zeros(steps)
    beta = np.zeros(steps)
    b_prev = 0.0
    for j in range(steps):
        w = H @ v
        alpha[j] = np.vdot(v, w).real
        w = w - alpha[j] * v - b_prev * v_prev
        beta[j] = np.linalg.norm(w)
        if beta[j] == 0.0:
            return alpha[:j + 1], beta[:j + 1]
        v_prev, v, b_prev = v, w / beta[j], beta[j]
    return alpha, beta


def lanczos_bounds(alpha, beta, n: int, k: int):
    """(b_sup, a, a0) from a Lanczos run (first-solve a, a0; upper bound after Zhou & Li 2011).

    b_sup = mu_max + |beta_last| |z_last|: the top Ritz value plus the residual norm of its
    Ritz pair (z = the eigenvector of T for mu_max), plus a margin of 1e-3 of the Ritz
    spread; a0 = min Ritz value.  a estimates lambda_{k+1} from the Lanczos density of
    states: the Ritz values with the squared first components of their eigenvectors of T
    (the Gauss quadrature of the start vector's spectral measure, which for a random start
    approximates the eigenvalue distribution) give a cumulative distribution, and a is the
    first Ritz value (from the second on) whose cumulative weight reaches k / n, at most the
    second largest."""
    mu, Z = direct.tridiagonal_eig(np.asarray(alpha), np.asarray(beta[:-1]), vectors=True)
    kl = mu.size
    b_sup = mu[-1] + abs(beta[-1]) * abs(Z[-1, -1]) + 1e-3 * (mu[-1] - mu[0])
    cdf = np.cumsum(Z[0, :] ** 2)
    j = 1
    while j < kl - 2 and cdf[j] < k / n:
        j += 1
    return b_sup, mu[j], mu[0]


# --- Algorithm 1, line "Filtering the vectors" (Chebyshev filter, Eq. (3term)) -------------
def filter_coefficients(m: int, a: float, b: float, a0: float):
    """Per-step (alpha_j, beta_j, gamma_j), j = 1..m, of Y_j = alpha_j H Y_{j-1} +
    beta_j Y_{j-1} + gamma_j Y_{j-2} (the scaled recurrence written out)."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    sigma1 = e / (a0 - c)
    sigma = sigma1
    out = [(sigma1 / e, -c * sigma1 / e, 0.0)]
    for _ in range(2, m + 1):
        sig_new = 1.0 / (2.0 / sigma1 - sigma)
        out.append((2.0 * sig_new / e, -2.0 * sig_new * c / e, -sigma * sig_new))
        sigma = sig_new
    return out


def chebyshev_filter(H: np.ndarray, Y0: np.ndarray, m: int, a: float, b: float, a0: float) -> np.ndarray:
    """Y_m = T_m((H - cI)/e) Y_0 / T_m((a0 - c)/e) by the scaled three-term recurrence."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    sigma1 = e / (a0 - c)
    sigma = sigma1
    Y_prev = Y0
    Y = (sigma1 / e) * (H @ Y0 - c * Y0)
    for _ in range(2, m + 1):
        sig_new = 1.0 / (2.0 / sigma1 - sigma)
        Y_next = (2.0 * sig_new / e) * (H @ Y - c * Y) - (sigma * sig_new) * Y_prev
        Y_prev, Y, sigma = Y, Y_next, sig_new
    return Y


def chebyshev_filter_per_column(H, Y0, degrees, a, b, a0) -> np.ndarray:
    """Column i filtered with its own degree degrees[i] (same a, b, a0 for all)."""
    out = np.empty_like(Y0)
    for i, m in enumerate(degrees):
        out[:, i:i + 1] = chebyshev_filter(H, Y0[:, i:i + 1], int(m), a, b, a0)
    return out


def chebyshev_t(m: int, x: np.ndarray) -> np.ndarray:
    """Closed form of the Chebyshev polynomial of the first kind (for pins)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(m * np.arccos(x[inside]))
    big = x > 1.0
    out[big] = np.cosh(m * np.arccosh(x[big]))
    small = x < -1.0
    out[small] = (-1.0) ** m * np.cosh(m * np.arccosh(-x[small]))
    return out


# --- Algorithm 1, line "Re-orthonormalizing" (QR) -------------------------------------------
def orthonormalize(Y_locked: np.ndarray | None, Y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of the active block, orthogonal to the locked vectors.

    Householder QR (numpy/LAPACK) of [Y_locked | Y]; the phases of R's diagonal are moved
    into Q so that R has a positive diagonal, which makes Q unique."""
    nl = 0 if Y_locked is None else Y_locked.shape[1]
    full = Y if nl == 0 else np.hstack([Y_locked, Y])
    q, r = np.linalg.qr(full)
    d = np.diagonal(r)
    ph = np.where(d != 0, d / np.where(d != 0, np.abs(d), 1.0), 1.0)
    q = q * ph[None, :]
    return q[:, nl:]


# --- Algorithm 1, Rayleigh-Ritz lines --------------------------------------------------------
def rayleigh_ritz(H: np.ndarray, Q: np.ndarray):
    """G = Q^H H Q; G W = W Lam (ascending); returns (lam, Y = Q W, Z = H Y)."""
    Z = H @ Q
    G = Q.conj().T @ Z
    G = 0.5 * (G + G.conj().T)
    lam, W = direct.hermitian_eig(G)
    return lam, Q @ W, Z @ W


def residual_norms(Z: np.ndarray, Y: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """||H y_i - lam_i y_i||_2 per column, with Z = H Y (Algorithm 1, Res)."""
    return np.linalg.norm(Z - Y * lam[None, :], axis=0)


# --- per-vector degree (not in the paper) -----------------------------------------------------
def per_vector_degrees(lam, resid_rel, a, b, tol, m_min, m_max):
    """m_i = clamp(ceil(ln(tol / r_i) / ln(rho_i)), m_min, m_max) with the Chebyshev rate
    rho_i = 1 / (|t_i| + sqrt(t_i^2 - 1)), t_i = (lam_i - c) / e (rho_i = 1 inside [a, b])."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    out = np.empty(len(lam), dtype=np.int64)
    for i, (l, r) in enumerate(zip(lam, resid_rel)):
        t = abs((l - c) / e)
        if t <= 1.0 or r <= tol:
            out[i] = m_min if r <= tol else m_max
            continue
        rho = 1.0 / (t + math.sqrt(t * t - 1.0))
        need = math.log(tol / r) / math.log(rho)
        out[i] = int(min(max(math.ceil(need), m_min), m_max))
    return out


@dataclasses.dataclass
class ChFSIResult:
    lam: np.ndarray            # nev eigenvalues, ascending
    Y: np.ndarray              # n x nev eigenvectors of the standard-form matrix
    resid: np.ndarray          # relative residuals of the returned pairs
    iterations: int
    block_lam: np.ndarray      # Ritz values of the whole final block (seeding the next solve)
    block_Y: np.ndarray        # final block (locked + active), ascending
    bounds: tuple              # (a, b, a0) used last
    filter_column_steps: int


def chfsi(H: np.ndarray, nev: int, nex: int, Y0: np.ndarray, tol: float, degree: int,
          seed: int = 0, lanczos_steps: int = 20, max_iter: int = 50, kappa_L: float = 1.0,
          prev_bounds: tuple | None = None, degree_range: tuple | None = None) -> ChFSIResult:
    """Algorithm 1 on a standard-form Hermitian H, block of k = nev + nex columns.

    prev_bounds = (lam_1, lam_k) of the previous problem of a sequence (Algorithm 1 Require:
    the previous eigenvalues) or None for a first solve.  degree_range = (m_min, m_max)
    turns on per-vector degrees."""
    n = H.shape[0]
    k = nev + nex
    assert Y0.shape == (n, k)
    # Line 1: Lanczos estimate of the upper end of the spectrum
    v0 = splitmix_complex_block(seed, n, 1, stream=0)[:, 0]
    al, be = lanczos(H, v0, lanczos_steps)
    b_sup, a_l, a0_l = lanczos_bounds(al, be, n, k)
    if prev_bounds is None:
        a, a0 = a_l, a0_l
    else:
        a0, a = prev_bounds
        a0 = min(a0, a0_l)
    a0_init = a0
    tol_lock = tol / kappa_L

    Y_locked = np.zeros((n, 0), dtype=np.complex128)
    lam_locked = np.zeros(0)
    res_locked = np.zeros(0)
    Y = np.array(Y0, dtype=np.complex128, copy=True)
    degrees = np.full(k, degree, dtype=np.int64)
    col_steps = 0
    it = 0
    lam = np.zeros(0)
    while True:
        it += 1
        # Line 3: filter
        if degree_range is None:
            Y = chebyshev_filter(H, Y, degree, a, b_sup, a0)
            col_steps += degree * Y.shape[1]
        else:
            Y = chebyshev_filter_per_column(H, Y, degrees, a, b_sup, a0)
            col_steps += int(np.sum(degrees))
        # Line 4: QR (orthogonal to the locked vectors)
        Q = orthonormalize(Y_locked if Y_locked.shape[1] else None, Y)
        # Lines 5-7: Rayleigh-Ritz
        lam, Y, Z = rayleigh_ritz(H, Q)
        # relative to max(||H y||, 1e-4 ||H||): absolute for eigenvalues near 0, where a relative
        # residual of tol would lie below FP64's reach
        floor = 1e-4 * max(abs(a0_init), abs(b_sup))
        res = residual_norms(Z, Y, lam) / np.maximum(np.linalg.norm(Z, axis=0), floor)
        # Lines 8-12: deflation and locking, i = converged .. nev
        nl = Y_locked.shape[1]
        lock = np.zeros(Y.shape[1], dtype=bool)
        for i in range(0, max(nev - nl, 0)):
            if res[i] < tol_lock:
                lock[i] = True
        if lock.any():
            Y_locked = np.hstack([Y_locked, Y[:, lock]])
            lam_locked = np.concatenate([lam_locked, lam[lock]])
            res_locked = np.concatenate([res_locked, res[lock]])
        keep = ~lock
        # bounds for the next pass: a = largest Ritz value of the block, a0 = smallest seen
        a = float(lam[-1])
        a0 = min(a0, float(lam[0]))
        if degree_range is not None:
            degrees = per_vector_degrees(lam[keep], res[keep], a, b_sup, tol_lock, *degree_range)
        Y = Y[:, keep]
        lam_active = lam[keep]
        if Y_locked.shape[1] >= nev or it >= max_iter:
            break
    order = np.argsort(lam_locked, kind="stable")
    lam_out = lam_locked[order][:nev]
    Y_out = Y_locked[:, order][:, :nev]
    block_lam = np.concatenate([lam_locked, lam_active])
    block_Y = np.hstack([Y_locked, Y])
    border = np.argsort(block_lam, kind="stable")
    return ChFSIResult(lam=lam_out, Y=Y_out, resid=res_locked[order][:nev], iterations=it,
                       block_lam=block_lam[border], block_Y=block_Y[:, border],
                       bounds=(a, b_sup, a0), filter_column_steps=col_steps)


def kappa_L_estimate(L: np.ndarray, seed: int = 0, steps: int = 20) -> float:
    """Upper estimate of cond_2(L) = sqrt(lam_max(S) / lam_min(S)) from two Lanczos runs:
    on S = L L^H and on S^{-1} = L^{-H} L^{-1} (each bound = max Ritz value + |beta|).

    Pinned (tests/test_oracle_kappa.py) on S with cond(S) = 10 exactly: sqrt(10) <= estimate
    <= 2 sqrt(10) for any step count (each bound lies in [lam_max, 2 lam_max] since
    |beta| <= ||S||), and the estimate equals sqrt(10) when Lanczos runs to exhaustion."""
    n = L.shape[0]
    v0 = splitmix_complex_block(seed, n, 1, stream=1)[:, 0]

    class _Op:
        def __init__(self, f):
            self.f = f

        def __matmul__(self, x):
            return self.f(x)

    S_op = _Op(lambda x: L @ (L.conj().T @ x))
    Sinv_op = _Op(lambda x: direct.backward_solve_h(L, direct.forward_solve(L, x[:, None]))[:, 0])
    bounds = []
    for op in (S_op, Sinv_op):
        al, be = lanczos(op, v0, steps)
        mu = direct.tridiagonal_eig(al, be[:-1], vectors=False)
        bounds.append(mu[-1] + abs(be[-1]))
    return math.sqrt(bounds[0] * bounds[1])


def solve_generalized(H, S, nev, nex, Y0, tol, degree, seed=0, prev=None, **kw):
    """Generalized problem: reduce with the Cholesky factor (Section 3), run Algorithm 1 on
    H' = L^{-1} H L^{-H}, back-transform x = L^{-H} y.  prev = (L, result) of the previous
    problem of the sequence (S fixed) seeds the block and the bounds (Algorithm 1 Require)."""
    if prev is None:
        L = direct.cholesky(S)
        kap = kappa_L_estimate(L, seed)
    else:
        L, kap = prev[0], prev[2]
    Hs = direct.reduce_to_standard(H, L)
    if prev is not None:
        Y0 = prev[1].block_Y
        pb = (float(prev[1].block_lam[0]), float(prev[1].block_lam[-1]))
    else:
        pb = None
    res = chfsi(Hs, nev, nex, Y0, tol, degree, seed=seed, kappa_L=kap, prev_bounds=pb, **kw)
    X = direct.backward_solve_h(L, res.Y)
    return res.lam, X, res, (L, res, kap)
