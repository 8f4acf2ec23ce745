"""The allocation-free reduced eigensolver (chfsi_reduced_eig_noalloc) against the
context-based one (chfsi_reduced_eig), through the C-ABI, on two calls in a row.

Callers that cannot allocate device memory use the allocation-free form; its scratch is a
fixed device array shared by all calls.  This file is collected last on purpose, and the
test must pass both alone in a fresh process (the first call does the per-device set-up)
and after every other test."""
import numpy as np
import pytest

from paper_1305_5120_gb300 import chfsi as lib
from paper_1305_5120_gb300 import synth

from gpu_util import phase_align, torch_cuda

pytestmark = pytest.mark.gpu


def herm(k, seed):
    return synth.hermitian_part(synth.complex_gaussian(synth.rng_for(seed, 700 + k), (k, k)))


@pytest.mark.parametrize("k", [47, 48, 240, 256])
def test_noalloc_matches_context_eigensolver_twice(k):
    torch = torch_cuda()
    ctx = lib.Context(device=0)
    for call, seed in enumerate([1, 2]):
        G = herm(k, seed)
        Gd = lib.colmajor(G)
        lam_ref = torch.empty(k, dtype=torch.float64, device="cuda")
        W_ref = torch.empty((k, k), dtype=torch.complex128, device="cuda")
        ctx.reduced_eig(k, Gd, lam_ref, W_ref)
        lam = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
        W = torch.full((k, k), np.nan, dtype=torch.complex128, device="cuda")
        st = lib.reduced_eig_noalloc(k, Gd, lam, W)
        assert st == 0, (call, lib.STATUS.get(st, st))
        l0, l1 = lam_ref.cpu().numpy(), lam.cpu().numpy()
        scale = max(1.0, np.abs(l0).max())
        assert np.abs(l1 - l0).max() < 1e-13 * scale
        W0, W1 = lib.to_numpy(W_ref), lib.to_numpy(W)
        assert np.abs(phase_align(W1, W0) - W0).max() < 1e-9
        assert np.abs(G @ W1 - W1 * l1).max() < 1e-12 * scale
        # the input is left untouched
        assert np.array_equal(lib.to_numpy(Gd), G)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_the_limit():
    torch = torch_cuda()
    k = 257
    G = torch.zeros((k, k), dtype=torch.complex128, device="cuda")
    lam = torch.empty(k, dtype=torch.float64, device="cuda")
    W = torch.empty((k, k), dtype=torch.complex128, device="cuda")
    assert lib.reduced_eig_noalloc(k, G, lam, W) == 1
