"""Helpers for the GPU tests: torch device arrays and oracle conversions."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def solver_lib():
    from paper_2211_08263_gb300 import wfft
    return wfft


def rel(a, b):
    """Relative L2 difference (complex-safe)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def to_dev(torch, arr, dtype):
    return torch.from_numpy(np.ascontiguousarray(arr)).to(device="cuda", dtype=dtype)


def oracle_field(prob, arr):
    from oracle.medium import field_to_oracle
    return field_to_oracle(prob, arr)


def abi_field(prob, arr):
    return np.asarray(arr).reshape(prob.ndim, prob.n[2], prob.n[1], prob.n[0])
