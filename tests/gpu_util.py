"""Helpers shared by the GPU tests (device setup, phase alignment)."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def phase_align(Y, Ref):
    """Multiply each column of Y by the unit phase that best aligns it with Ref."""
    ip = np.sum(Y.conj() * Ref, axis=0)
    ph = np.where(np.abs(ip) > 0, ip / np.abs(ip), 1.0)
    return Y * ph[None, :]


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def floored_residuals(H, S, lam, X, hnorm):
    """||H x - lam S x|| / max(||H x||, 1e-4 hnorm ||S x||) per column (torch tensors on the
    device, or numpy), and the mask of the columns where the floor decides.

    This is the acceptance measure the solver's lock test guarantees (Res = ||H'y - lam y|| /
    max(||H'y||, 1e-4 ||H'||), tol / kappa_L, with x = L^{-H} y): the relative residual
    ||Hx - lam Sx|| / ||Hx|| for |lam| >= 1e-4 ||H'||, and below that, where a relative 1e-10
    is beneath FP64's reach, the same bound against 1e-4 ||H'|| ||S x||."""
    try:
        import torch
        if isinstance(H, torch.Tensor):
            lam_t = torch.as_tensor(lam, device=H.device)
            HX, SX = H @ X, S @ X
            num = torch.linalg.vector_norm(HX - SX * lam_t[None, :], dim=0)
            nh = torch.linalg.vector_norm(HX, dim=0)
            fl = 1e-4 * hnorm * torch.linalg.vector_norm(SX, dim=0)
            return (num / torch.maximum(nh, fl)).cpu().numpy(), (fl > nh).cpu().numpy()
    except ImportError:  # pragma: no cover
        pass
    HX, SX = H @ X, S @ X
    num = np.linalg.norm(HX - SX * np.asarray(lam)[None, :], axis=0)
    nh = np.linalg.norm(HX, axis=0)
    fl = 1e-4 * hnorm * np.linalg.norm(SX, axis=0)
    return num / np.maximum(nh, fl), fl > nh
