"""Parity of each stage of the CUDA path (through the C-ABI) with the oracle, element by
element on the same seeded inputs, at sizes that span several tiles plus ragged tails."""
import numpy as np
import pytest

from oracle import chfsi as O2
from oracle import direct as O1
from paper_1305_5120_gb300 import chfsi as lib
from paper_1305_5120_gb300 import synth

from gpu_util import phase_align, rel_err, torch_cuda

pytestmark = pytest.mark.gpu

SIZES = [(200, 24), (333, 37), (512, 48)]


@pytest.fixture(scope="module", params=[lib.CHFSI_PREC_FP64, lib.CHFSI_PREC_MIXED], ids=["fp64", "mixed"])
def ctx(request):
    """Both precisions: in mixed mode the FP64 products of every stage run as the exact
    BF16-digit expansion on the tensor cores; the parity bounds are the same."""
    torch_cuda()
    c = lib.Context(device=0, precision=request.param)
    yield c
    c.close()


def std_problem(n, seed, n_low=None, high=50.0):
    n_low = n_low or max(4, n // 10)
    lam = synth.prescribed_spectrum(n, n_low, high, seed)
    q = synth.haar_unitary(n, synth.rng_for(seed, 3))
    return synth.hermitian_part((q * lam[None, :]) @ q.conj().T), lam, q


def dev(A):
    return lib.colmajor(A)


def empty(rows, cols, dtype=None):
    torch = torch_cuda()
    return torch.empty((cols, rows), dtype=dtype or torch.complex128, device="cuda")


@pytest.mark.parametrize("n", [64, 200, 333, 700])
def test_cholesky(ctx, n):
    """In mixed precision n > 256 takes the blocked factorisation (128-wide diagonal blocks on
    the FP64 pipe, panels and trailing updates as tensor-core products): 333 and 700 are
    ragged multiples of the block."""
    S, _ = synth.spd_factor(n, n)
    L = empty(n, n)
    ctx.cholesky(n, dev(S), L)
    Lg = lib.to_numpy(L)
    ref = O1.cholesky(S)
    assert np.abs(Lg - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(np.triu(Lg, 1)).max() == 0.0


@pytest.mark.parametrize("n,bad", [(64, 40), (600, 450)])
def test_cholesky_not_hpd(ctx, n, bad):
    S = np.diag(np.r_[np.ones(bad), -1.0, np.ones(n - bad - 1)]).astype(complex)
    L = empty(n, n)
    with pytest.raises(lib.ChfsiError) as e:
        ctx.cholesky(n, dev(S), L)
    assert e.value.status == 2


@pytest.mark.parametrize("n", [96, 333])
def test_reduce(ctx, n):
    p = synth.prescribed_pencil(n, n // 10, 50.0, 11)
    L = O1.cholesky(p.S)
    Hs = empty(n, n)
    ctx.reduce(n, dev(p.H), dev(L), Hs)
    ref = O1.reduce_to_standard(p.H, L)
    assert rel_err(lib.to_numpy(Hs), ref) < 1e-13


@pytest.mark.parametrize("n,k", SIZES)
def test_lanczos(ctx, n, k):
    torch = torch_cuda()
    H, lam, _ = std_problem(n, 21)
    steps = 20
    al = torch.empty(steps, dtype=torch.float64, device="cuda")
    be = torch.empty_like(al)
    bd = torch.empty(4, dtype=torch.float64, device="cuda")
    ctx.lanczos(n, dev(H), steps, k, None, al, be, bd)
    v0 = O2.splitmix_complex_block(0, n, 1, stream=0)[:, 0]
    ra, rb = O2.lanczos(H, v0, steps)
    assert np.abs(al.cpu().numpy() - ra).max() < 1e-10 * np.abs(lam).max()
    assert np.abs(be.cpu().numpy() - rb).max() < 1e-10 * np.abs(lam).max()
    b_sup, a, a0 = O2.lanczos_bounds(ra, rb, n, k)
    g = bd.cpu().numpy()
    assert abs(g[0] - b_sup) < 1e-10 * abs(b_sup)
    assert abs(g[1] - a) < 1e-9 * abs(b_sup) and abs(g[2] - a0) < 1e-9 * abs(b_sup)
    assert g[0] >= lam[-1]


@pytest.mark.parametrize("n,k", SIZES + [(130, 1)])
@pytest.mark.parametrize("m", [1, 2, 20])
def test_filter_fp64(ctx, n, k, m):
    H, lam, _ = std_problem(n, 31)
    Y0 = synth.start_block(n, k, 31)
    a, b, a0 = float(lam[int(1.2 * k)]), float(lam[-1] * 1.05), float(lam[0] - 0.1)
    Y = dev(Y0)
    ctx.filter(n, k, dev(H), Y, m, a, b, a0, lib.CHFSI_PREC_FP64)
    ref = O2.chebyshev_filter(H, Y0, m, a, b, a0)
    assert rel_err(lib.to_numpy(Y), ref) < 1e-11


def test_filter_per_vector_degree(ctx):
    n, k = 300, 29
    H, lam, _ = std_problem(n, 32)
    Y0 = synth.start_block(n, k, 32)
    deg = sorted(np.random.default_rng(1).integers(3, 17, k).tolist(), reverse=True)
    a, b, a0 = float(lam[40]), float(lam[-1] * 1.05), float(lam[0] - 0.1)
    Y = dev(Y0)
    ctx.filter_degrees(n, k, dev(H), Y, deg, a, b, a0, lib.CHFSI_PREC_FP64)
    ref = O2.chebyshev_filter_per_column(H, Y0, deg, a, b, a0)
    assert rel_err(lib.to_numpy(Y), ref) < 1e-11


@pytest.mark.parametrize("n,k,nl", [(200, 24, 0), (333, 37, 11), (512, 48, 32), (1000, 240, 16), (1200, 513, 0)])
def test_orthonormalize(ctx, n, k, nl):
    rng = synth.rng_for(5, n)
    Yl = O2.orthonormalize(None, synth.complex_gaussian(rng, (n, nl))) if nl else None
    Y0 = synth.complex_gaussian(rng, (n, k))
    Y = dev(Y0)
    ctx.orthonormalize(n, nl, dev(Yl) if nl else None, k, Y)
    ref = O2.orthonormalize(Yl, Y0)
    assert np.abs(lib.to_numpy(Y) - ref).max() < 1e-12


def test_orthonormalize_ill_conditioned(ctx):
    """A filtered block is far from orthogonal; the shifted CholQR path must still produce
    the unique Q (positive diagonal R)."""
    n, k = 400, 30
    H, lam, _ = std_problem(n, 6)
    Y0 = O2.chebyshev_filter(H, synth.start_block(n, k, 6), 20, float(lam[36]), float(lam[-1] * 1.05),
                             float(lam[0] - 0.05))
    Y = dev(Y0)
    ctx.orthonormalize(n, 0, None, k, Y)
    Q = lib.to_numpy(Y)
    assert np.abs(Q.conj().T @ Q - np.eye(k)).max() < 1e-12
    P = Q @ (Q.conj().T @ Y0)
    assert rel_err(P, Y0) < 1e-9
    R = Q.conj().T @ Y0
    assert np.all(np.diagonal(R).real > 0)


@pytest.mark.parametrize("k", [1, 2, 7, 48, 101, 240])
def test_reduced_eig(ctx, k):
    torch = torch_cuda()
    rng = synth.rng_for(9, k)
    G = synth.hermitian_part(synth.complex_gaussian(rng, (k, k)))
    lam = torch.empty(k, dtype=torch.float64, device="cuda")
    W = empty(k, k)
    ctx.reduced_eig(k, dev(G), lam, W)
    ref_l, ref_W = O1.hermitian_eig(G)
    lg = lam.cpu().numpy()
    assert np.abs(lg - ref_l).max() < 1e-13 * max(1.0, np.abs(ref_l).max())
    Wg = lib.to_numpy(W)
    assert np.abs(Wg.conj().T @ Wg - np.eye(k)).max() < 1e-13
    assert np.abs(G @ Wg - Wg * lg).max() < 1e-12 * np.abs(ref_l).max()
    assert np.abs(phase_align(Wg, ref_W) - ref_W).max() < 1e-9


def test_reduced_eig_near_diagonal(ctx):
    torch = torch_cuda()
    k = 240
    rng = synth.rng_for(10, 0)
    G = np.diag(np.sort(rng.uniform(-1, 80, k))).astype(complex)
    G = G + 1e-6 * synth.hermitian_part(synth.complex_gaussian(rng, (k, k)))
    lam = torch.empty(k, dtype=torch.float64, device="cuda")
    W = empty(k, k)
    ctx.reduced_eig(k, dev(G), lam, W)
    ref_l, _ = O1.hermitian_eig(G)
    assert np.abs(lam.cpu().numpy() - ref_l).max() < 1e-12 * 80


@pytest.mark.parametrize("n,k", SIZES)
def test_rayleigh_ritz_and_residuals(ctx, n, k):
    torch = torch_cuda()
    H, lam, _ = std_problem(n, 41)
    Q0 = O2.orthonormalize(None, O2.chebyshev_filter(H, synth.start_block(n, k, 41), 8, float(lam[int(1.3 * k)]),
                                                     float(lam[-1] * 1.05), float(lam[0] - 0.1)))
    Y = dev(Q0)
    Z = empty(n, k)
    lm = torch.empty(k, dtype=torch.float64, device="cuda")
    ctx.rayleigh_ritz(n, k, dev(H), Y, lm, Z)
    rl, rY, rZ = O2.rayleigh_ritz(H, Q0)
    lg = lm.cpu().numpy()
    assert np.abs(lg - rl).max() < 1e-12 * np.abs(lam).max()
    Yg = lib.to_numpy(Y)
    assert np.abs(phase_align(Yg, rY) - rY).max() < 1e-8
    Zg = lib.to_numpy(Z)
    assert np.abs(Zg - H @ Yg).max() < 1e-12 * np.abs(lam).max()
    res = torch.empty(k, dtype=torch.float64, device="cuda")
    ctx.residuals(n, k, Z, Y, lm, res)
    ref = O2.residual_norms(Zg, Yg, lg) / np.linalg.norm(Zg, axis=0)
    assert np.abs(res.cpu().numpy() - ref).max() <= 1e-14 * max(1.0, ref.max())


def test_degrees(ctx):
    torch = torch_cuda()
    k = 64
    rng = synth.rng_for(12, 0)
    lam = np.sort(rng.uniform(-1, 3, k))
    r = 10.0 ** rng.uniform(-12, -1, k)
    a, b, tol = 2.0, 80.0, 1e-10
    d = torch.empty(k, dtype=torch.int32, device="cuda")
    ctx.degrees(k, torch.tensor(lam, device="cuda"), torch.tensor(r, device="cuda"), a, b, tol, 10, 25, d)
    ref = O2.per_vector_degrees(lam, r, a, b, tol, 10, 25)
    assert np.array_equal(d.cpu().numpy(), ref)


@pytest.mark.parametrize("n,k", [(200, 24), (333, 37)])
def test_back_transform(ctx, n, k):
    S, _ = synth.spd_factor(n, 13)
    L = O1.cholesky(S)
    Y0 = synth.start_block(n, k, 13)
    X = empty(n, k)
    ctx.back_transform(n, k, dev(L), dev(Y0), X)
    ref = O1.backward_solve_h(L, Y0)
    assert rel_err(lib.to_numpy(X), ref) < 1e-13
