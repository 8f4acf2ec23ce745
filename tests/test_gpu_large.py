"""The large single-problem workload (n = 13000, nev = 1300, nex = 260, degree chosen per
vector in [10, 25], mixed precision) and a per-vector-degree sequence, checked by
properties that hold at any size: the prescribed spectrum (exact eigenvalues of the
constructed pencil), generalized residuals ||Hx - lam Sx|| / ||Hx|| <= 1e-10 for every
returned pair, and S-orthonormality."""
import numpy as np
import pytest

from oracle import direct as O1
from paper_1305_5120_gb300 import chfsi as lib
from paper_1305_5120_gb300 import synth

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def check_device(H, S, lam_ref, ev, X, nev):
    torch = torch_cuda()
    Xm = X.T                                  # column-major buffer (nev, n) -> n x nev
    HX = H @ Xm
    R = HX - (S @ Xm) * ev[None, :]
    res = (torch.linalg.vector_norm(R, dim=0) / torch.linalg.vector_norm(HX, dim=0)).max().item()
    err = (ev - lam_ref[:nev]).abs().max().item()
    G = Xm.conj().T @ (S @ Xm)
    orth = (G - torch.eye(nev, dtype=G.dtype, device=G.device)).abs().max().item()
    return err, res, orth


@pytest.mark.parametrize("prec", [lib.CHFSI_PREC_FP64, lib.CHFSI_PREC_MIXED])
def test_per_vector_degree_sequence(prec):
    n, nev, nex = 400, 30, 10
    ctx = lib.Context(device=0, precision=prec, per_vector_degree=1, degree_min=6, degree_max=25)
    for l, p in synth.sequence(n, 40, 40.0, 3, seed=12):
        if l == 0:
            st, ev, X, info = ctx.solve(lib.colmajor(p.H), lib.colmajor(p.S), n, nev, nex,
                                        lib.colmajor(synth.start_block(n, nev + nex, 12)), 1e-10, 0)
        else:
            st, ev, X, info = ctx.next_in_sequence(lib.colmajor(p.H), None, nev=nev, n=n)
        assert st == 0
        ref = O1.generalized_eig(p.H, p.S, nev=nev, vectors=False)
        lam = ev.cpu().numpy()
        assert np.abs(lam - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())
        assert O1.generalized_residuals(p.H, p.S, lam, lib.to_numpy(X)).max() <= 1e-10
        # per-vector degrees: fewer column-steps than the full degree for every column
        assert info.filter_col_steps < info.iterations * (nev + nex) * 25
    ctx.close()


def test_large_n13000_per_vector_degree_mixed():
    torch = torch_cuda()
    w = synth.SEQ_N13000
    H, S, lam = synth.prescribed_pencil_device(w.n, w.n_low, w.high, w.seed)
    Hd, Sd = H.T.contiguous(), S.T.contiguous()      # column-major buffers
    ctx = lib.Context(device=0, precision=lib.CHFSI_PREC_MIXED, per_vector_degree=1, degree_min=10, degree_max=25)
    st, ev, X, info = ctx.solve(Hd, Sd, w.n, w.nev, w.nex, None, w.tol, 0)
    torch.cuda.synchronize()
    assert st == 0, lib.STATUS[st]
    err, res, orth = check_device(H, S, lam, ev, X, w.nev)
    assert err <= 1e-10 * max(1.0, lam[: w.nev].abs().max().item()), err
    assert res <= 1e-10, res
    assert orth <= 1e-11, orth
    ctx.close()
