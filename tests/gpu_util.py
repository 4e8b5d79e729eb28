"""Helpers shared by the GPU tests (test infrastructure)."""
import numpy as np
import pytest

try:
    import torch
    HAS_GPU = torch.cuda.is_available()
except Exception:   # noqa: BLE001
    torch = None
    HAS_GPU = False


def need_gpu():
    if not HAS_GPU:
        pytest.skip("needs a CUDA GPU")
    from paper_2205_04194_gb300 import build
    build.build()


def rel2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def relinf(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()
