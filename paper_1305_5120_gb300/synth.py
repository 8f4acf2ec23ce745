"""Seeded synthetic inputs shaped like FLAPW generalized eigenproblem sequences (Section 2).

This module builds inputs only: it holds none of the solver's arithmetic and is the one
module that both the CUDA path's tests/benchmark and the oracle's tests draw inputs from.

Construction (prescribed spectrum, so that the eigenvalues of every first problem are known
exactly):

* ``S = V diag(s) V^H`` with ``V`` Haar-unitary and ``s = 1 + t g``: ``g`` holds the eigenvalues
  of a random Hermitian matrix ``G`` (sampled from the semicircle law on [-1, 1]) and ``t`` is
  chosen so that ``cond(S) = 10`` exactly, i.e. ``S = I + t G``.
* ``M = V diag(sqrt(s))`` satisfies ``S = M M^H``; with ``Q`` Haar-unitary,
  ``H = (M Q) diag(lam) (M Q)^H`` so that ``H x = lam S x`` has exactly the eigenvalues ``lam``
  (``M^H x`` is an eigenvector of ``Q diag(lam) Q^H``).  No Cholesky factor is needed here.
* Sequences: ``H_{l+1} = H_l + eps_l E_l``, ``eps_l = eps0 * decay**l``, with
  ``E_l = U_l diag(e) U_l^H`` Hermitian of unit 2-norm (``e`` semicircle samples rescaled so
  that ``max |e| = 1``), ``U_l`` Haar-unitary; ``S`` stays fixed.
* Start blocks: complex Gaussian entries, real and imaginary parts ~ N(0, 1/2).

Haar unitaries come from the QR factorisation of a complex Gaussian matrix with the phases of
R's diagonal moved into Q (Mezzadri, "How to generate random matrices from the classical
compact groups", 2007).  All matrices are returned as complex128 numpy arrays in the
mathematical orientation (``A[i, j]`` is row i, column j).
"""
from __future__ import annotations

import dataclasses
import numpy as np


def rng_for(seed: int, *stream: int) -> np.random.Generator:
    """Independent PCG64 stream for (seed, stream...)."""
    return np.random.default_rng(np.random.SeedSequence([int(seed), *[int(s) for s in stream]]))


def complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """Entries with independent real and imaginary parts ~ N(0, 1/2)."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def haar_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    z = complex_gaussian(rng, (n, n))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return q * ph[None, :]


def semicircle(rng: np.random.Generator, count: int) -> np.ndarray:
    """Samples of the Wigner semicircle density on [-1, 1] (rejection sampling)."""
    out = np.empty(0)
    while out.size < count:
        x = rng.uniform(-1.0, 1.0, 2 * count + 16)
        u = rng.uniform(0.0, 1.0, x.size)
        out = np.concatenate([out, x[u <= np.sqrt(1.0 - x * x)]])
    return out[:count]


def hermitian_part(a: np.ndarray) -> np.ndarray:
    return 0.5 * (a + a.conj().T)


@dataclasses.dataclass
class Pencil:
    """One generalized problem H x = lam S x (plus what built it)."""
    H: np.ndarray
    S: np.ndarray
    M: np.ndarray                    # any factor with S = M M^H (not a Cholesky factor)
    lam: np.ndarray | None = None    # exact eigenvalues (ascending) when prescribed


def spd_factor(n: int, seed: int, cond: float = 10.0):
    """S = I + t G with cond(S) = cond exactly; returns (S, M) with S = M M^H."""
    rng = rng_for(seed, 1)
    v = haar_unitary(n, rng)
    g = semicircle(rng, n)
    g[0], g[1] = -1.0, 1.0                 # pin the extremes so that cond(S) is exact
    t = (cond - 1.0) / (cond + 1.0)        # (1 + t) / (1 - t) = cond
    s = 1.0 + t * g
    S = hermitian_part((v * s[None, :]) @ v.conj().T)
    M = v * np.sqrt(s)[None, :]
    return S, M


def prescribed_spectrum(n: int, n_low: int, high: float, seed: int) -> np.ndarray:
    """n_low values uniform in [-1, 0], the remaining n - n_low uniform in [0.5, high]; sorted."""
    rng = rng_for(seed, 2)
    lam = np.concatenate([rng.uniform(-1.0, 0.0, n_low), rng.uniform(0.5, high, n - n_low)])
    return np.sort(lam)


def prescribed_pencil(n: int, n_low: int, high: float, seed: int, cond: float = 10.0) -> Pencil:
    S, M = spd_factor(n, seed, cond)
    lam = prescribed_spectrum(n, n_low, high, seed)
    q = haar_unitary(n, rng_for(seed, 3))
    mq = M @ q
    H = hermitian_part((mq * lam[None, :]) @ mq.conj().T)
    return Pencil(H=H, S=S, M=M, lam=lam)


def perturbation(n: int, seed: int, step: int) -> np.ndarray:
    """Random Hermitian E with ||E||_2 = 1 exactly."""
    rng = rng_for(seed, 100 + step)
    u = haar_unitary(n, rng)
    e = semicircle(rng, n)
    e = e / np.max(np.abs(e))
    return hermitian_part((u * e[None, :]) @ u.conj().T)


def sequence(n: int, n_low: int, high: float, steps: int, seed: int,
             eps0: float = 1e-2, decay: float = 0.7):
    """Yield (step, H_step) for a correlated sequence; S is fixed (returned first)."""
    p = prescribed_pencil(n, n_low, high, seed)
    H = p.H
    yield 0, p
    for l in range(1, steps):
        H = H + (eps0 * decay ** (l - 1)) * perturbation(n, seed, l - 1)
        yield l, Pencil(H=H, S=p.S, M=p.M, lam=None)


def start_block(n: int, k: int, seed: int) -> np.ndarray:
    return complex_gaussian(rng_for(seed, 4), (n, k))


# Workloads (sizes and spectra of the configurations the library is measured on).
@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    nev: int
    nex: int
    n_low: int
    high: float
    steps: int
    degree: int
    seed: int = 0
    tol: float = 1e-10


SINGLE_N512 = Workload("single n=512 nev=32 nex=16 m=20", 512, 32, 16, 32, 50.0, 1, 20)
SEQ_N2000 = Workload("sequence n=2000 x20 nev=200 nex=40 m=20", 2000, 200, 40, 200, 80.0, 20, 20)
SEQ_N13000 = Workload("sequence n=13000 x8 nev=1300 nex=260 m=10..25", 13000, 1300, 260, 1300, 80.0, 8, 20)


# Large problems: the same recipe generated on a CUDA device with torch (numpy's QR of an
# n = 13000 complex matrix takes minutes on host cores).  Inputs only: the factorisations
# here build the test matrices and are not part of the solver.
def _torch_haar(n, gen, device):
    import torch
    z = (torch.randn(n, n, generator=gen, device=device, dtype=torch.float64)
         + 1j * torch.randn(n, n, generator=gen, device=device, dtype=torch.float64)) * (0.5 ** 0.5)
    q, r = torch.linalg.qr(z)
    d = torch.diagonal(r)
    return q * (d / d.abs())[None, :]


def prescribed_pencil_device(n: int, n_low: int, high: float, seed: int, device="cuda", cond: float = 10.0):
    """(H, S, lam) as column-major-ready torch tensors on `device` (mathematical
    orientation, complex128); lam ascending, the exact eigenvalues of the pencil."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + 17)
    v = _torch_haar(n, gen, device)
    g = torch.from_numpy(semicircle(rng_for(seed, 1), n)).to(device)
    g[0], g[1] = -1.0, 1.0
    t = (cond - 1.0) / (cond + 1.0)
    s = 1.0 + t * g
    S = (v * s[None, :]) @ v.conj().T
    S = 0.5 * (S + S.conj().T)
    M = v * torch.sqrt(s)[None, :]
    lam = torch.from_numpy(prescribed_spectrum(n, n_low, high, seed)).to(device)
    q = _torch_haar(n, gen, device)
    mq = M @ q
    H = (mq * lam[None, :]) @ mq.conj().T
    H = 0.5 * (H + H.conj().T)
    return H, S, lam


def perturbation_device(n: int, seed: int, step: int, device="cuda"):
    """The sequence perturbation E of `perturbation` (Hermitian, unit 2-norm exactly), built
    with torch on `device` (mathematical orientation, complex128)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + 7919 * (step + 1) + 29)
    u = _torch_haar(n, gen, device)
    e = semicircle(rng_for(seed, 100 + step), n)
    e = torch.from_numpy(e / np.max(np.abs(e))).to(device)
    E = (u * e[None, :]) @ u.conj().T
    return 0.5 * (E + E.conj().T)



# Serving at scale (n up to 20000, hundreds of problems): the Haar recipe above costs O(n^3)
# per matrix (a QR and dense products), minutes at n = 20000.  Here the unitaries are
# structured, U = F D_b F D_a with F the unitary DFT and D_a, D_b diagonal matrices of random
# phases (two layers of phases and Fourier transforms spread every basis vector over all
# coordinates, as a Haar unitary does), and every matrix is formed by applying them to the
# columns of a matrix with FFTs: O(n^2 log n).  The pencil keeps the same law otherwise --
# S = V diag(s) V^H with cond(S) = 10 exactly, H = M W diag(lam) W^H M^H with M = V diag(sqrt(s))
# -- so its eigenvalues are exactly lam (up to the FFTs' rounding, ~1e-15 relative).
def _phases(n, gen, device):
    import torch
    t = torch.rand(n, generator=gen, device=device, dtype=torch.float64) * (2.0 * np.pi)
    return torch.polar(torch.ones_like(t), t)


class _FourierUnitary:
    def __init__(self, n, gen, device):
        self.da = _phases(n, gen, device)
        self.db = _phases(n, gen, device)

    def apply(self, x):        # U x for every column of x
        import torch
        y = torch.fft.fft(self.da[:, None] * x, dim=0, norm="ortho")
        return torch.fft.fft(self.db[:, None] * y, dim=0, norm="ortho")

    def apply_h(self, x):      # U^H x for every column of x
        import torch
        y = torch.conj(self.db)[:, None] * torch.fft.ifft(x, dim=0, norm="ortho")
        return torch.conj(self.da)[:, None] * torch.fft.ifft(y, dim=0, norm="ortho")

    def conjugate(self, d):    # U diag(d) U^H
        import torch
        eye = torch.eye(len(d), dtype=torch.complex128, device=d.device)
        return self.apply(d[:, None] * self.apply_h(eye))


def structured_pencil_device(n: int, n_low: int, high: float, seed: int, device="cuda", cond: float = 10.0):
    """(H, S, lam) like `prescribed_pencil_device`, with structured unitaries (above):
    O(n^2 log n) to build.  lam ascending, the exact eigenvalues of the pencil."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + 31)
    v = _FourierUnitary(n, gen, device)
    w = _FourierUnitary(n, gen, device)
    g = torch.from_numpy(semicircle(rng_for(seed, 1), n)).to(device)
    g[0], g[1] = -1.0, 1.0
    t = (cond - 1.0) / (cond + 1.0)
    s = (1.0 + t * g).to(torch.complex128)
    S = v.conjugate(s)
    S = 0.5 * (S + S.conj().T)
    lam = torch.from_numpy(prescribed_spectrum(n, n_low, high, seed)).to(device)
    C = w.conjugate(lam.to(torch.complex128))                 # W diag(lam) W^H
    r = torch.sqrt(s)
    T = r[:, None] * C * r[None, :]                           # diag(sqrt s) C diag(sqrt s)
    del C
    H = v.apply(torch.conj(v.apply(torch.conj(T).T)).T)       # V (V T^H)^H = V T V^H
    H = 0.5 * (H + H.conj().T)
    return H, S, lam


def structured_perturbation_device(n: int, seed: int, step: int, device="cuda"):
    """A Hermitian perturbation of unit 2-norm exactly, E = U diag(e) U^H with U structured."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + 7919 * (step + 1) + 37)
    u = _FourierUnitary(n, gen, device)
    e = semicircle(rng_for(seed, 100 + step), n)
    e = torch.from_numpy(e / np.max(np.abs(e))).to(device).to(torch.complex128)
    E = u.conjugate(e)
    return 0.5 * (E + E.conj().T)
