"""Helpers for the GPU parity tests (imported only by tests marked gpu)."""
import numpy as np

import paper_2210_03179_gb300 as cm


def dev():
    import torch
    return torch.device("cuda:0")


def T(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), device=dev(), dtype=dtype or torch.float64)


def N(t):
    return t.detach().cpu().numpy().astype(np.float64)


def relerr(got, ref):
    ref = np.asarray(ref)
    scale = np.abs(ref).max()
    return float(np.abs(np.asarray(got) - ref).max() / (scale if scale > 0 else 1.0))


def empty(n, f32=False):
    import torch
    return torch.zeros(n, device=dev(), dtype=torch.float32 if f32 else torch.float64)
