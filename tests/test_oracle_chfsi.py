"""Pins of the oracle's ChFSI (O2): the Chebyshev closed form, the paper's unscaled
recurrence (Eq. 3term) as a special case, prescribed spectra, invariants of Lanczos, QR and
Rayleigh-Ritz, the published SplitMix64 test vector, and agreement of the whole iteration
with the direct solver O1."""
import math

import numpy as np
import pytest

from oracle import chfsi, direct
from paper_1305_5120_gb300 import synth


def prescribed_standard(n, n_low, high, seed):
    lam = synth.prescribed_spectrum(n, n_low, high, seed)
    q = synth.haar_unitary(n, synth.rng_for(seed, 3))
    return synth.hermitian_part((q * lam[None, :]) @ q.conj().T), lam, q


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0 (Steele, Lea & Flood 2014; the reference seeding generator of
    # xoshiro/xoroshiro): first outputs 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f
    out = chfsi.splitmix64(0, 3)
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = chfsi.splitmix_uniform(7, 10000)
    assert u.min() >= -0.5 and u.max() < 0.5 and abs(u.mean()) < 0.02


def test_chebyshev_closed_form_matches_recurrence():
    x = np.linspace(-3, 3, 601)
    t_prev, t = np.ones_like(x), x.copy()
    for m in range(2, 26):
        t_prev, t = t, 2 * x * t - t_prev
        assert np.allclose(chfsi.chebyshev_t(m, x), t, rtol=1e-12, atol=1e-12)


def test_filter_on_prescribed_spectrum():
    n = 120
    H, lam, q = prescribed_standard(n, 12, 50.0, 1)
    Y0 = synth.start_block(n, 7, 1)
    a, b, a0 = 2.0, 50.5, -1.2
    m = 14
    Y = chfsi.chebyshev_filter(H, Y0, m, a, b, a0)
    e, c = (b - a) / 2, (b + a) / 2
    p = chfsi.chebyshev_t(m, (lam - c) / e) / chfsi.chebyshev_t(m, np.array([(a0 - c) / e]))[0]
    ref = q @ (p[:, None] * (q.conj().T @ Y0))
    assert np.abs(Y - ref).max() < 1e-10 * np.abs(ref).max()


def test_filter_reduces_to_paper_recurrence():
    """With c = 0, e = 1 (a = -1, b = 1) the scaled filter is Eq. (3term),
    C_{m+1} = 2 H C_m - C_{m-1}, C_0 = Y, C_1 = H Y, divided by T_m(a0)."""
    n = 50
    H, lam, q = prescribed_standard(n, 5, 1.0, 2)
    H = H / 1.0
    Y0 = synth.start_block(n, 3, 2)
    a0 = -1.3
    m = 9
    C_prev, C = Y0, H @ Y0
    for _ in range(2, m + 1):
        C_prev, C = C, 2 * H @ C - C_prev
    tm = chfsi.chebyshev_t(m, np.array([a0]))[0]
    Y = chfsi.chebyshev_filter(H, Y0, m, -1.0, 1.0, a0)
    assert np.abs(Y - C / tm).max() < 1e-12 * np.abs(C / tm).max()


def test_filter_coefficients_consistent():
    n = 40
    H, _, _ = prescribed_standard(n, 4, 20.0, 3)
    Y0 = synth.start_block(n, 5, 3)
    a, b, a0 = 1.0, 21.0, -1.1
    coef = chfsi.filter_coefficients(11, a, b, a0)
    Yp, Y = None, Y0
    for (al, be, ga) in coef:
        Yn = al * (H @ Y) + be * Y + (ga * Yp if Yp is not None else 0)
        Yp, Y = Y, Yn
    ref = chfsi.chebyshev_filter(H, Y0, 11, a, b, a0)
    assert np.abs(Y - ref).max() < 1e-12 * np.abs(ref).max()


def test_lanczos_bound_and_full_krylov():
    n = 300
    H, lam, _ = prescribed_standard(n, 30, 50.0, 4)
    v0 = chfsi.splitmix_complex_block(0, n, 1, 0)[:, 0]
    al, be = chfsi.lanczos(H, v0, 20)
    b_sup, a, a0 = chfsi.lanczos_bounds(al, be, n, 45)
    # an upper bound (the invariant the filter needs), and not a wild one: |beta| is at most
    # about half the spectral width for a converging Lanczos run
    assert lam[-1] <= b_sup <= lam[-1] + 0.5 * (lam[-1] - lam[0])
    assert lam[0] <= a0 < a < b_sup
    # full Krylov space of a small matrix: Ritz values are the eigenvalues
    H8, lam8, _ = prescribed_standard(8, 2, 5.0, 5)
    al, be = chfsi.lanczos(H8, chfsi.splitmix_complex_block(1, 8, 1, 0)[:, 0], 8)
    mu = direct.tridiagonal_eig(al, be[:-1], vectors=False)
    assert np.abs(mu - lam8).max() < 1e-10


def test_orthonormalize_properties():
    n = 90
    rng = synth.rng_for(0, 11)
    Yl = chfsi.orthonormalize(None, synth.complex_gaussian(rng, (n, 4)))
    Y = synth.complex_gaussian(rng, (n, 6))
    Q = chfsi.orthonormalize(Yl, Y)
    assert np.abs(Q.conj().T @ Q - np.eye(6)).max() < 1e-14
    assert np.abs(Yl.conj().T @ Q).max() < 1e-14
    # span([Yl, Q]) == span([Yl, Y])
    P = np.hstack([Yl, Q])
    assert np.abs(Y - P @ (P.conj().T @ Y)).max() < 1e-12
    # uniqueness: R = Q^H Y restricted part is upper triangular with positive diagonal
    R = Q.conj().T @ (Y - Yl @ (Yl.conj().T @ Y))
    assert np.abs(np.tril(R, -1)).max() < 1e-12
    assert np.all(np.diagonal(R).real > 0) and np.abs(np.diagonal(R).imag).max() < 1e-12


def test_rayleigh_ritz_exact_subspace():
    n = 70
    H, lam, q = prescribed_standard(n, 7, 30.0, 6)
    # a rotated basis of the invariant subspace of the 5 smallest eigenvalues
    W = synth.haar_unitary(5, synth.rng_for(6, 12))
    Qb = q[:, :5] @ W
    l, Y, Z = chfsi.rayleigh_ritz(H, Qb)
    assert np.abs(l - lam[:5]).max() < 1e-12
    assert chfsi.residual_norms(Z, Y, l).max() < 1e-12


def test_per_vector_degree_definition():
    lam = np.array([-0.9, -0.5, -0.01, 0.3])
    r = np.array([1e-3, 1e-6, 1e-2, 1e-12])
    a, b, tol = 2.0, 80.0, 1e-10
    m = chfsi.per_vector_degrees(lam, r, a, b, tol, 10, 25)
    e, c = (b - a) / 2, (b + a) / 2
    for i in range(3):
        t = abs((lam[i] - c) / e)
        rho = 1 / (t + math.sqrt(t * t - 1))
        need = math.log(tol / r[i]) / math.log(rho)
        if 10 < m[i] < 25:
            assert rho ** m[i] <= tol / r[i] * (1 + 1e-12) < rho ** (m[i] - 1)
        else:
            assert m[i] == (10 if need <= 10 else 25)
    assert m[3] == 10     # already converged: minimum degree


def test_chfsi_standard_prescribed():
    n, nev, nex = 200, 12, 6
    H, lam, _ = prescribed_standard(n, 20, 50.0, 7)
    Y0 = synth.start_block(n, nev + nex, 7)
    res = chfsi.chfsi(H, nev, nex, Y0, 1e-10, 16)
    assert np.abs(res.lam - lam[:nev]).max() < 1e-10 * max(1, np.abs(lam[:nev]).max())
    Z = H @ res.Y
    rel = np.linalg.norm(Z - res.Y * res.lam, axis=0) / np.linalg.norm(Z, axis=0)
    assert rel.max() < 1e-10
    assert np.abs(res.Y.conj().T @ res.Y - np.eye(nev)).max() < 1e-12


def test_chfsi_generalized_sequence_matches_direct():
    n, nev, nex = 160, 10, 5
    gen = synth.sequence(n, 16, 40.0, 3, seed=8)
    prev = None
    for step, p in gen:
        Y0 = synth.start_block(n, nev + nex, 8)
        lam, X, res, prev = chfsi.solve_generalized(p.H, p.S, nev, nex, Y0, 1e-10, 14, prev=prev)
        ref = direct.generalized_eig(p.H, p.S, nev=nev, vectors=False)
        assert np.abs(lam - ref).max() < 1e-10 * np.maximum(np.abs(ref), 1).max()
        assert direct.generalized_residuals(p.H, p.S, lam, X).max() <= 1e-10
        assert np.abs(X.conj().T @ p.S @ X - np.eye(nev)).max() < 1e-11
        sig = 0.5 * (ref[-1] + direct.generalized_eig(p.H, p.S, nev=nev + 1, vectors=False)[-1])
        assert direct.inertia_below(p.H, sig, p.S) == nev


def test_chfsi_per_vector_degree_converges():
    n, nev, nex = 150, 10, 4
    H, lam, _ = prescribed_standard(n, 15, 40.0, 9)
    Y0 = synth.start_block(n, nev + nex, 9)
    res = chfsi.chfsi(H, nev, nex, Y0, 1e-10, 12, degree_range=(6, 25))
    assert np.abs(res.lam - lam[:nev]).max() < 1e-10
