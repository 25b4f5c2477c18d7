"""Helpers shared by the GPU tests (inputs only; no method arithmetic)."""
import numpy as np


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1))
