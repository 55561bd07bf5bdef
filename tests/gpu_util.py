"""Helpers shared by the GPU parity tests (no solver arithmetic here)."""
import numpy as np
import torch

DEV = "cuda"


def T(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def empty(n, dtype=torch.float64):
    return torch.empty(n, dtype=dtype, device=DEV)


def H(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()
