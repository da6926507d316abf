"""Helpers shared by the GPU tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_max(a, b, axis=None):
    """max |a - b| / max |b| (per row when axis is given)."""
    a = np.asarray(a)
    b = np.asarray(b)
    if axis is None:
        return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)
    num = np.max(np.abs(a - b), axis=axis)
    den = np.maximum(np.max(np.abs(b), axis=axis), 1e-300)
    return num / den
