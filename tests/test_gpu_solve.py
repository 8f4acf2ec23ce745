"""Whole solves through the C-ABI (chfsi_solve / chfsi_next_in_sequence) against the
oracle: eigenvalues to 1e-10 relative (|d lam| <= 1e-10 max(|lam|, 1)), generalized
residuals ||Hx - lam Sx|| / ||Hx|| <= 1e-10, S-orthonormal eigenvectors, and the inertia
count that rules out a missed eigenvalue."""
import os

import numpy as np
import pytest

from oracle import chfsi as O2
from oracle import direct as O1
from paper_1305_5120_gb300 import chfsi as lib
from paper_1305_5120_gb300 import synth

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EV_TOL = 1e-10
RES_TOL = 1e-10


def check_pairs(H, S, lam, X, ref_lam, nev):
    assert lam.shape == (nev,)
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(lam - ref_lam[:nev]).max() <= EV_TOL * np.maximum(np.abs(ref_lam[:nev]), 1.0).max()
    r = O1.generalized_residuals(H, S, lam, X)
    assert r.max() <= RES_TOL, r.max()
    G = X.conj().T @ S @ X
    assert np.abs(G - np.eye(nev)).max() < 1e-11


def solve_once(prec, w, p, X0=None, per_vector=False):
    torch = torch_cuda()
    ctx = lib.Context(device=0, precision=prec, per_vector_degree=int(per_vector))
    k = w.nev + w.nex
    X0 = X0 if X0 is not None else synth.start_block(w.n, k, w.seed)
    st, ev, X, info = ctx.solve(lib.colmajor(p.H), lib.colmajor(p.S), w.n, w.nev, w.nex, lib.colmajor(X0), w.tol,
                                w.degree)
    torch.cuda.synchronize()
    return ctx, st, ev.cpu().numpy(), lib.to_numpy(X), info


@pytest.mark.parametrize("prec", [lib.CHFSI_PREC_FP64, lib.CHFSI_PREC_MIXED])
def test_single_n512(prec):
    w = synth.SINGLE_N512
    p = synth.prescribed_pencil(w.n, w.n_low, w.high, w.seed)
    ctx, st, lam, X, info = solve_once(prec, w, p)
    assert st == 0, lib.STATUS[st]
    check_pairs(p.H, p.S, lam, X, p.lam, w.nev)
    sig = 0.5 * (p.lam[w.nev - 1] + p.lam[w.nev])
    assert O1.inertia_below(p.H, sig, p.S) == w.nev
    assert info.iterations < 20 and info.locked == w.nev
    # the oracle ChFSI on the same start block converges to the same pairs
    lam_o, X_o, res_o, _ = O2.solve_generalized(p.H, p.S, w.nev, w.nex, synth.start_block(w.n, w.nev + w.nex, w.seed),
                                                w.tol, w.degree)
    assert np.abs(lam - lam_o).max() <= EV_TOL
    ctx.close()


def test_small_sequence_matches_direct_solver():
    torch = torch_cuda()
    n, nev, nex, steps = 300, 20, 8, 4
    ctx = lib.Context(device=0)
    prev = None
    for l, p in synth.sequence(n, 30, 40.0, steps, seed=3):
        H, S = lib.colmajor(p.H), lib.colmajor(p.S)
        if l == 0:
            st, ev, X, info = ctx.solve(H, S, n, nev, nex, lib.colmajor(synth.start_block(n, nev + nex, 3)), 1e-10, 16)
        else:
            st, ev, X, info = ctx.next_in_sequence(H, None, nev=nev, n=n)
        assert st == 0
        ref = O1.generalized_eig(p.H, p.S, nev=nev + 1, vectors=False)
        check_pairs(p.H, p.S, ev.cpu().numpy(), lib.to_numpy(X), ref, nev)
        if l > 0:
            assert info.iterations <= prev + 1
        prev = info.iterations
    ctx.close()


def test_sequence_with_changing_S():
    n, nev, nex = 200, 12, 6
    ctx = lib.Context(device=0)
    p0 = synth.prescribed_pencil(n, 20, 40.0, 4)
    st, ev, X, info = ctx.solve(lib.colmajor(p0.H), lib.colmajor(p0.S), n, nev, nex, None, 1e-10, 16)
    assert st == 0
    S1 = p0.S + 0.01 * synth.perturbation(n, 4, 50)
    H1 = p0.H + 0.01 * synth.perturbation(n, 4, 51)
    st, ev, X, info = ctx.next_in_sequence(lib.colmajor(H1), lib.colmajor(S1), nev=nev, n=n)
    assert st == 0
    ref = O1.generalized_eig(H1, S1, nev=nev, vectors=False)
    check_pairs(H1, S1, ev.cpu().numpy(), lib.to_numpy(X), ref, nev)
    ctx.close()


def load_golden_sequence():
    path = os.path.join(GOLDEN, "seq_n2000_evals.txt")
    if not os.path.exists(path):
        pytest.skip("golden eigenvalues not generated")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows[int(parts[0])] = np.array([float(x) for x in parts[1:]])
    return rows


@pytest.mark.parametrize("prec", [lib.CHFSI_PREC_FP64, lib.CHFSI_PREC_MIXED])
def test_sequence_n2000_against_golden(prec):
    """The n = 2000, 20-step sequence (the benchmark workload): every step's eigenvalues
    against the oracle's direct solver (stored by tests/golden/make_sequence_evals.py),
    residuals and S-orthonormality recomputed here in FP64."""
    torch = torch_cuda()
    gold = load_golden_sequence()
    w = synth.SEQ_N2000
    ctx = lib.Context(device=0, precision=prec)
    k = w.nev + w.nex
    refined = fallbacks = 0
    for l, p in synth.sequence(w.n, w.n_low, w.high, w.steps, w.seed):
        H, S = lib.colmajor(p.H), lib.colmajor(p.S)
        if l == 0:
            st, ev, X, info = ctx.solve(H, S, w.n, w.nev, w.nex, lib.colmajor(synth.start_block(w.n, k, w.seed)),
                                        w.tol, w.degree)
        else:
            st, ev, X, info = ctx.next_in_sequence(H, None, nev=w.nev, n=w.n)
        assert st == 0, (l, lib.STATUS[st])
        refined += info.eig_refined
        fallbacks += info.eig_fallbacks
        if l in gold:
            check_pairs(p.H, p.S, ev.cpu().numpy(), lib.to_numpy(X), gold[l], w.nev)
    ctx.close()
    if prec == lib.CHFSI_PREC_MIXED:
        # the reduced eigenproblems ran through the FP32 start + FP64 refinement, not the
        # fallback (FP64 Jacobi)
        assert refined >= 40 and fallbacks <= refined // 10, (refined, fallbacks)


def test_error_paths():
    torch = torch_cuda()
    ctx = lib.Context(device=0)
    n = 64
    p = synth.prescribed_pencil(n, 8, 10.0, 1)
    Sbad = np.diag(np.r_[np.ones(10), -1.0, np.ones(53)]).astype(complex)
    st, *_ = ctx.solve(lib.colmajor(p.H), lib.colmajor(Sbad), n, 8, 4, None, 1e-10, 10)
    assert st == 2
    st, *_ = ctx.solve(lib.colmajor(p.H), lib.colmajor(p.S), n, 60, 10, None, 1e-10, 10)   # nev+nex > n
    assert st == 1
    fresh = lib.Context(device=0)
    st, *_ = fresh.next_in_sequence(lib.colmajor(p.H), None, nev=8, n=n)
    assert st == 7
    # the context stays usable after an error
    st, ev, X, info = ctx.solve(lib.colmajor(p.H), lib.colmajor(p.S), n, 8, 4, None, 1e-10, 10)
    assert st == 0
    assert np.abs(ev.cpu().numpy() - p.lam[:8]).max() < 1e-10
    ctx.close()
    fresh.close()
