"""Helpers shared by the GPU parity tests (marshalling only)."""
import math

import numpy as np


def dev():
    import torch
    return torch.device("cuda:0")


def to_gpu(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev())


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def make_ctx(n1, n2, nt, regnorm=1, beta=1e-2, gamma=math.inf, shear=0.0):
    from paper_1503_00757_gb300.binding import Context
    return Context(n1, n2, nt, regnorm=regnorm, beta=beta, gamma=gamma, shear=shear)
