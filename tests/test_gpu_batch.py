"""Batched solves (chfsi_solve_batch): independent problems of uneven size advanced together,
the filter of every problem's iteration one grouped tensor-core launch per recurrence step.
Every problem must give what chfsi_solve gives on its own (the grouped launch runs each
problem's tiles exactly as the single launch does), and the prescribed spectrum.

The two tile widths of the filter step compute every output element in the same order, so
the autotuner's choice cannot change a result: pinned here by forcing each width."""
import os

import numpy as np
import pytest

from paper_1305_5120_gb300 import chfsi as lib
from paper_1305_5120_gb300 import synth

from gpu_util import floored_residuals, torch_cuda

pytestmark = pytest.mark.gpu


def problems(count, lo, hi, seed, device=False):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(lo, hi + 1))
        nev = max(4, int(round(n * rng.uniform(0.05, 0.15))))
        nex = max(2, int(round(0.2 * nev)))
        if device:
            H, S, lam = synth.prescribed_pencil_device(n, nev, 50.0, seed=seed * 100 + i)
            out.append((n, nev, nex, lib.colmajor(H), lib.colmajor(S), lam.cpu().numpy(), H, S))
        else:
            p = synth.prescribed_pencil(n, nev, 50.0, seed=seed * 100 + i)
            out.append((n, nev, nex, lib.colmajor(p.H), lib.colmajor(p.S), p.lam, p.H, p.S))
    return out


@pytest.mark.parametrize("prec,own_stream", [(lib.CHFSI_PREC_MIXED, True), (lib.CHFSI_PREC_MIXED, False),
                                             (lib.CHFSI_PREC_FP64, True)], ids=["mixed-graph", "mixed-default", "fp64"])
def test_batch_equals_single_solves(prec, own_stream):
    """On a created stream the grouped step launches are captured into a CUDA graph; on the
    default stream (not capturable) they are launched directly: same results either way."""
    torch = torch_cuda()
    probs = problems(5, 260, 700, seed=3)
    stream = torch.cuda.Stream() if own_stream else None
    ctx = lib.Context(device=0, precision=prec, stream=stream)
    st, sts, evals, Xs, infos = ctx.solve_batch([p[3] for p in probs], [p[4] for p in probs],
                                                [p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                                                1e-10, 20)
    assert st == 0 and all(s == 0 for s in sts), sts
    for q, (n, nev, nex, Hd, Sd, lam, H, S) in enumerate(probs):
        ev = evals[q].cpu().numpy()
        assert np.abs(ev - lam[:nev]).max() <= 1e-10 * max(1.0, np.abs(lam[:nev]).max())
        a, b, a0 = infos[q].bounds
        res, _ = floored_residuals(H, S, ev, lib.to_numpy(Xs[q]), max(abs(a0), abs(b)))
        assert res.max() <= 1e-10
        alone = lib.Context(device=0, precision=prec)
        s1, ev1, X1, i1 = alone.solve(Hd, Sd, n, nev, nex, None, 1e-10, 20)
        assert s1 == 0 and i1.iterations == infos[q].iterations
        assert np.abs(ev1.cpu().numpy() - ev).max() <= 1e-13 * max(1.0, np.abs(ev).max())
        alone.close()
    ctx.close()


def test_batch_kpoint_sizes_complete():
    torch = torch_cuda()
    probs = problems(6, 1500, 4000, seed=4, device=True)
    torch.cuda.synchronize()   # generated on the default stream; solved on another
    ctx = lib.Context(device=0, precision=lib.CHFSI_PREC_MIXED, check_inertia=1, stream=torch.cuda.Stream())
    st, sts, evals, Xs, infos = ctx.solve_batch([p[3] for p in probs], [p[4] for p in probs],
                                                [p[0] for p in probs], [p[1] for p in probs], [p[2] for p in probs],
                                                1e-10, 20)
    assert st == 0 and all(s == 0 for s in sts), sts
    for q, (n, nev, nex, Hd, Sd, lam, H, S) in enumerate(probs):
        ev = evals[q].cpu().numpy()
        assert np.abs(ev - lam[:nev]).max() <= 1e-10 * max(1.0, np.abs(lam[:nev]).max())
        assert infos[q].completeness == 2
        a, b, a0 = infos[q].bounds
        res, fl = floored_residuals(H, S, ev, Xs[q].T, max(abs(a0), abs(b)))
        assert res.max() <= 1e-10
    ctx.close()


def test_filter_tile_widths_agree():
    torch = torch_cuda()
    n, k, m = 700, 83, 12
    lam = synth.prescribed_spectrum(n, 70, 50.0, 5)
    q = synth.haar_unitary(n, synth.rng_for(5, 3))
    H = lib.colmajor(synth.hermitian_part((q * lam[None, :]) @ q.conj().T))
    Y0 = synth.start_block(n, k, 5)
    out = []
    try:
        for w in ("32", "64"):
            os.environ["CHFSI_FILTER_WIDTH"] = w
            ctx = lib.Context(device=0)
            Y = lib.colmajor(Y0)
            ctx.filter(n, k, H, Y, m, float(lam[100]), float(lam[-1] * 1.05), float(lam[0] - 0.1),
                       lib.CHFSI_PREC_MIXED)
            out.append(lib.to_numpy(Y))
            ctx.close()
    finally:
        os.environ.pop("CHFSI_FILTER_WIDTH", None)
    assert np.array_equal(out[0], out[1])
