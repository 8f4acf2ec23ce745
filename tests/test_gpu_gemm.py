"""chfsi_gemm (the complex product every stage is built from) in both precisions against an
extended-precision host product.

Bound: an FP64 GEMM satisfies |C - C_exact| <= K u sum_k |a_ik||b_kj| (u = 2^-53).  The
tensor-core expansion keeps 61 bits of every entry relative to its row (column) scale and
accumulates exactly, so it obeys the same form with K u replaced by ~ (2^-58 + u); both are
tested against 2^-44 sum|a||b| (the K u bound with a margin of 2^9 for K <= 6000), and
the typical (rms) error against 1e-15 of the rms of sum|a||b|."""
import numpy as np
import pytest

from paper_1305_5120_gb300 import chfsi as lib
from paper_1305_5120_gb300 import synth

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [  # M, N, K, opA, opB
    (1, 1, 1, "N", "N"), (37, 5, 29, "N", "N"), (130, 77, 300, "C", "N"), (200, 24, 333, "N", "C"),
    (512, 48, 512, "N", "N"), (240, 240, 2000, "C", "N"), (64, 64, 3000, "N", "N"), (2000, 240, 2000, "N", "N")]


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    c = lib.Context(device=0)
    yield c
    c.close()


def op(X, o):
    return X if o == "N" else X.conj().T


@pytest.mark.parametrize("prec", [lib.CHFSI_PREC_FP64, lib.CHFSI_PREC_MIXED])
@pytest.mark.parametrize("M,N,K,oa,ob", SHAPES)
def test_gemm(ctx, prec, M, N, K, oa, ob):
    rng = synth.rng_for(77, M * 7 + N * 3 + K)
    A = synth.complex_gaussian(rng, (M, K) if oa == "N" else (K, M))
    B = synth.complex_gaussian(rng, (K, N) if ob == "N" else (N, K))
    # entries of mixed magnitude within rows/columns (scale each row of A / column of B)
    A *= (10.0 ** rng.uniform(-3, 3, A.shape[0]))[:, None]
    B *= (10.0 ** rng.uniform(-3, 3, B.shape[1]))[None, :]
    C0 = synth.complex_gaussian(rng, (M, N))
    alpha, beta = 0.7 - 0.2j, -0.5 + 0.1j
    C = lib.colmajor(C0)
    ctx.gemm(oa, ob, M, N, K, alpha, lib.colmajor(A), A.shape[0], lib.colmajor(B), B.shape[0], beta, C, M, prec)
    got = lib.to_numpy(C)
    if M * N * K <= 2e7:
        Al, Bl = op(A, oa).astype(np.clongdouble), op(B, ob).astype(np.clongdouble)
        exact = (alpha * (Al @ Bl) + beta * C0.astype(np.clongdouble))
    else:   # large shapes: an FP64 host product (its own error is far inside the bound)
        exact = (alpha * (op(A, oa) @ op(B, ob)) + beta * C0).astype(np.clongdouble)
    err = np.abs(got.astype(np.clongdouble) - exact).astype(np.float64)
    bound = np.abs(alpha) * (np.abs(op(A, oa)) @ np.abs(op(B, ob))) + np.abs(beta) * np.abs(C0)
    assert np.all(err <= 2.0 ** -44 * bound + 1e-300), (err / bound).max()
    assert np.sqrt((err ** 2).mean()) <= 1e-15 * np.sqrt((bound ** 2).mean())
