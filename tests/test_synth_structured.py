"""The structured (FFT-built) pencils of the serving workload at scale: the recipe's
invariants, checked with LAPACK (scipy) on the CPU -- the eigenvalues of the pencil are the
prescribed ones, cond(S) = 10, the perturbation has unit 2-norm, and the unitaries spread
every basis vector over all coordinates (no near-diagonal H)."""
import numpy as np
import pytest
import scipy.linalg as sl

from paper_1305_5120_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n,seed", [(64, 1), (130, 7)])
def test_structured_pencil_has_the_prescribed_spectrum(n, seed):
    H, S, lam = synth.structured_pencil_device(n, n // 8, 50.0, seed, device="cpu")
    H, S, lam = H.numpy(), S.numpy(), lam.numpy()
    assert np.array_equal(H, H.conj().T) and np.array_equal(S, S.conj().T)
    ev = sl.eigh(H, S, eigvals_only=True)
    assert np.abs(ev - lam).max() <= 1e-13 * np.abs(lam).max()
    es = np.linalg.eigvalsh(S)
    assert abs(es.max() / es.min() - 10.0) < 1e-12
    # delocalised: H is far from diagonal
    assert np.linalg.norm(H - np.diag(np.diag(H))) > 0.3 * np.linalg.norm(H)


def test_structured_perturbation_unit_norm():
    E = synth.structured_perturbation_device(90, 4, 2, device="cpu").numpy()
    assert np.array_equal(E, E.conj().T)
    assert abs(np.abs(np.linalg.eigvalsh(E)).max() - 1.0) < 1e-13
