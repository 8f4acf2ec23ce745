"""Pins of the oracle's direct solver (O1) against things other than itself:
closed forms, an independent algorithm (Jacobi), LAPACK (scipy) as a library special case,
prescribed spectra, Sylvester inertia and brute-force bisection."""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import direct
from paper_1305_5120_gb300 import synth


def rand_herm(n, seed):
    z = synth.complex_gaussian(synth.rng_for(seed, 77), (n, n))
    return synth.hermitian_part(z)


def test_two_by_two_closed_form():
    a, d, b = 1.3, -0.7, 0.4 - 0.9j
    A = np.array([[a, b], [np.conj(b), d]])
    mid, rad = (a + d) / 2, np.sqrt(((a - d) / 2) ** 2 + abs(b) ** 2)
    lam, Y = direct.hermitian_eig(A)
    assert np.allclose(lam, [mid - rad, mid + rad], atol=1e-15, rtol=0)
    assert np.allclose(A @ Y, Y * lam, atol=1e-14)
    # generalized 2x2 with diagonal S: det(A - lam S) = 0
    S = np.diag([2.0, 0.5])
    lg, X = direct.generalized_eig(A, S)
    for l in lg:
        assert abs(np.linalg.det(A - l * S)) < 1e-13


def test_diagonal_matrix():
    dvals = np.array([3.0, -1.0, 2.5, 0.0, -7.0, 1.0])
    lam, Y = direct.hermitian_eig(np.diag(dvals).astype(complex))
    assert np.array_equal(lam, np.sort(dvals))
    assert np.allclose(np.abs(Y), np.eye(6)[:, np.argsort(dvals)], atol=1e-15)


def test_toeplitz_tridiagonal_closed_form():
    # T = tridiag(e, d, e): lam_j = d + 2 e cos(j pi / (n + 1)), v_j(i) ~ sin(i j pi / (n + 1))
    n, d0, e0 = 57, 0.3, -1.7
    lam, Z = direct.tridiagonal_eig(np.full(n, d0), np.full(n - 1, e0))
    j = np.arange(1, n + 1)
    ref = np.sort(d0 + 2 * e0 * np.cos(j * np.pi / (n + 1)))
    assert np.abs(lam - ref).max() < 1e-13
    T = np.diag(np.full(n, d0)) + np.diag(np.full(n - 1, e0), 1) + np.diag(np.full(n - 1, e0), -1)
    assert np.abs(T @ Z - Z * lam).max() < 1e-13
    assert np.abs(Z.T @ Z - np.eye(n)).max() < 1e-13


def test_householder_reconstructs():
    A = rand_herm(23, 1)
    d, off, vs = direct.householder_tridiagonal(A)
    n = A.shape[0]
    T = np.diag(d).astype(complex) + np.diag(off, -1) + np.diag(off.conj(), 1)
    Q = np.eye(n, dtype=complex)
    for k, v in enumerate(vs):
        if v is None:
            continue
        Hk = np.eye(n, dtype=complex)
        Hk[k + 1:, k + 1:] -= 2 * np.outer(v, v.conj())
        Q = Q @ Hk
    assert np.abs(Q @ T @ Q.conj().T - A).max() < 1e-13


def test_agrees_with_jacobi():
    A = rand_herm(40, 2)
    lam1, Y1 = direct.hermitian_eig(A)
    lam2, Y2 = direct.jacobi_eig(A)
    assert np.abs(lam1 - lam2).max() < 1e-13
    # eigenvectors equal up to a phase per column (eigenvalues are simple here)
    ov = np.abs(np.sum(Y1.conj() * Y2, axis=0))
    assert np.abs(ov - 1).max() < 1e-11


def test_agrees_with_lapack():
    A = rand_herm(100, 3)
    S, _ = synth.spd_factor(100, 3)
    lam, X = direct.generalized_eig(A, S)
    ref = sl.eigh(A, S, eigvals_only=True)
    assert np.abs(lam - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(X.conj().T @ S @ X - np.eye(100)).max() < 1e-12


def test_prescribed_spectrum_pencil():
    p = synth.prescribed_pencil(160, 16, 50.0, 5)
    lam, X = direct.generalized_eig(p.H, p.S, nev=20)
    assert np.abs(lam - p.lam[:20]).max() < 1e-12 * 50
    r = direct.generalized_residuals(p.H, p.S, lam, X)
    assert r.max() < 1e-11


def test_cholesky_and_reduction():
    S, M = synth.spd_factor(60, 4)
    L = direct.cholesky(S)
    assert np.allclose(np.triu(L, 1), 0)
    assert np.all(np.diagonal(L).real > 0) and np.allclose(np.diagonal(L).imag, 0)
    assert np.abs(L @ L.conj().T - S).max() < 1e-14
    assert np.abs(L - sl.cholesky(S, lower=True)).max() < 1e-13
    H = rand_herm(60, 4)
    Hs = direct.reduce_to_standard(H, L)
    assert np.abs(L @ Hs @ L.conj().T - H).max() < 1e-13
    Y = synth.complex_gaussian(synth.rng_for(0, 9), (60, 3))
    X = direct.backward_solve_h(L, Y)
    assert np.abs(L.conj().T @ X - Y).max() < 1e-13


def test_cholesky_rejects_indefinite():
    A = np.diag([1.0, -1.0, 2.0]).astype(complex)
    with pytest.raises(direct.NotPositiveDefinite):
        direct.cholesky(A)


def test_inertia_counts():
    p = synth.prescribed_pencil(80, 8, 50.0, 6)
    sig = 0.5 * (p.lam[7] + p.lam[8])
    assert direct.inertia_below(p.H, sig, p.S) == 8
    assert direct.inertia_below(p.H, p.lam[0] - 1, p.S) == 0
    assert direct.inertia_below(p.H, p.lam[-1] + 1, p.S) == 80


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_brute_force_bisection(n):
    """Every eigenvalue of a tiny matrix found by bisection on inertia counts alone."""
    A = rand_herm(n, 10 + n)
    lo, hi = -np.abs(A).sum() - 1, np.abs(A).sum() + 1
    ref = []
    for j in range(n):
        a, b = lo, hi
        for _ in range(200):
            mid = 0.5 * (a + b)
            if direct.inertia_below(A, mid) <= j:
                a = mid
            else:
                b = mid
        ref.append(0.5 * (a + b))
    lam = direct.hermitian_eig(A, vectors=False)
    assert np.abs(lam - np.array(ref)).max() < 1e-13
