"""Host-side pieces of the sequence-correlation study (bench.py --workload seeding): the
S-inner-product angles between eigenvector sets, pinned by constructions whose angles are
known exactly."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

from paper_1305_5120_gb300 import synth  # noqa: E402


def s_matrix(n, seed):
    rng = synth.rng_for(seed, 1)
    Z = synth.complex_gaussian(rng, (n, n))
    return Z @ Z.conj().T / n + np.eye(n)


def s_orthonormal(n, k, S, seed):
    rng = synth.rng_for(seed, 2)
    L = np.linalg.cholesky(S)
    q, _ = np.linalg.qr(synth.complex_gaussian(rng, (n, k)))
    return np.linalg.solve(L.conj().T, q)   # X^H S X = I


def test_identical_and_phase_rotated_sets_have_zero_angles():
    n, k = 40, 6
    S = s_matrix(n, 1)
    X = s_orthonormal(n, k, S, 1)
    ph = np.exp(1j * np.linspace(0.3, 2.0, k))
    assert np.allclose(bench.s_angles(X, X * ph[None, :] * 3.0, S), 0.0, atol=1e-7)
    assert np.allclose(bench.s_principal_angles(X, X @ np.diag(ph), S), 0.0, atol=1e-7)


def test_known_rotation_angle():
    # x_0 rotated by phi towards an S-orthogonal direction: the angle is exactly phi
    n = 30
    S = s_matrix(n, 3)
    B = s_orthonormal(n, 2, S, 3)
    for phi in (0.1, 0.7, 1.3):
        Y = (np.cos(phi) * B[:, 0] + np.sin(phi) * B[:, 1])[:, None]
        a = bench.s_angles(B[:, :1], Y, S)
        pa = bench.s_principal_angles(B[:, :1], Y, S)
        assert abs(a[0] - phi) < 1e-10 and abs(pa[-1] - phi) < 1e-10


def test_principal_angles_ignore_the_basis_but_not_the_span():
    n, k = 50, 5
    S = s_matrix(n, 5)
    X = s_orthonormal(n, k + 1, S, 5)
    M = synth.complex_gaussian(synth.rng_for(5, 3), (k, k)) + 3 * np.eye(k)
    # same span, another basis: all principal angles zero
    assert bench.s_principal_angles(X[:, :k], X[:, :k] @ M, S).max() < 1e-7
    # one direction replaced by an S-orthogonal one: exactly one right angle
    Y = np.hstack([X[:, : k - 1], X[:, k:]])
    pa = bench.s_principal_angles(X[:, :k], Y, S)
    assert abs(pa[-1] - np.pi / 2) < 1e-7 and pa[:-1].max() < 1e-7
