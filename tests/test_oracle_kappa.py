"""Pins of the oracle's condition estimate of L (oracle.chfsi.kappa_L_estimate), which sets the
locking tolerance tol / kappa_L that makes ||H x - lam S x|| / ||H x|| <= tol hold for the
generalized problem (Section 3: H' = L^{-1} H L^{-H}, H x - lam S x = L (H' y - lam y)).

The estimate is sqrt(b(S) b(S^{-1})), b = max Ritz value + |beta_last| of a Lanczos run.
Mathematics fixes it from both sides: every Ritz value lies in [lam_min, lam_max] and
|beta| <= ||A||_2, so lam_max(A) <= b(A) <= 2 lam_max(A); with cond(S) = 10 exactly
(synth.spd_factor), sqrt(10) <= kappa <= 2 sqrt(10).  When the Krylov space is exhausted
(S with two distinct eigenvalues, two steps) the Ritz values are the eigenvalues and beta
vanishes, so the estimate equals sqrt(10) to rounding: that pins the formula itself (a
missing square root, one run instead of two, or S in place of S^{-1} all fail it)."""
import math

import numpy as np
import pytest

from oracle import chfsi, direct
from paper_1305_5120_gb300 import synth


def two_level_spd(n, lo, hi, seed):
    """S = V diag(s) V^H with s taking only the values lo and hi (both present)."""
    v = synth.haar_unitary(n, synth.rng_for(seed, 11))
    s = np.where(np.arange(n) % 3 == 0, hi, lo).astype(float)
    return synth.hermitian_part((v * s[None, :]) @ v.conj().T)


@pytest.mark.parametrize("lo,hi", [(2.0, 20.0), (0.5, 5.0), (1.0, 10.0)])
def test_exhausted_krylov_space_gives_exact_condition(lo, hi):
    S = two_level_spd(48, lo, hi, seed=3)
    L = direct.cholesky(S)
    kap = chfsi.kappa_L_estimate(L, seed=1, steps=2)
    assert abs(kap - math.sqrt(hi / lo)) <= 1e-10 * math.sqrt(hi / lo)


@pytest.mark.parametrize("n,steps,seed", [(60, 5, 0), (200, 10, 1), (300, 20, 2), (300, 20, 7)])
def test_estimate_brackets_cond_L(n, steps, seed):
    S, _ = synth.spd_factor(n, seed, cond=10.0)
    ev = np.linalg.eigvalsh(S)
    assert abs(ev[-1] / ev[0] - 10.0) < 1e-10          # the generator's promise
    L = direct.cholesky(S)
    kap = chfsi.kappa_L_estimate(L, seed=seed, steps=steps)
    assert math.sqrt(10.0) * (1 - 1e-12) <= kap <= 2.0 * math.sqrt(10.0)


def test_estimate_is_an_upper_bound_for_other_conditions():
    for cond in (2.0, 50.0, 400.0):
        S, _ = synth.spd_factor(150, 5, cond=cond)
        kap = chfsi.kappa_L_estimate(direct.cholesky(S), seed=5, steps=20)
        assert math.sqrt(cond) * (1 - 1e-12) <= kap <= 2.0 * math.sqrt(cond)
