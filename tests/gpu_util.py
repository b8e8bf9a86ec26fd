"""Helpers for the GPU tests: host <-> device column-major copies."""
from __future__ import annotations

import numpy as np


def to_dev(A: np.ndarray):
    import torch

    import paper_1710_08471_gb300 as cq

    A = np.asarray(A, dtype=np.float64)
    if A.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(A)).cuda()
    t = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()  # (m, n) with stride (1, m)
    return cq.colmajor(t)


def to_host(X) -> np.ndarray:
    x = X.detach().cpu()
    if x.dim() == 1:
        return x.numpy().copy()
    return np.asfortranarray(x.numpy())


EPS = 2.0 ** -53
