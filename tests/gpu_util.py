"""Shared helpers of the GPU parity tests (inputs come from the oracle and the
seeded generators; nothing here computes the method)."""
import numpy as np
import pytest


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def rel_err_cols(X, Xref):
    X = np.asarray(X, np.float64)
    Xref = np.asarray(Xref, np.float64)
    return np.linalg.norm(X - Xref, axis=0) / np.linalg.norm(Xref, axis=0)
