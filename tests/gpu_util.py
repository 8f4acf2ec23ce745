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
