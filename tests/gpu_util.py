"""Helpers shared by the GPU tests (array marshalling only)."""
import numpy as np
import torch


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def zeros(ny, nx):
    return torch.zeros((ny + 2, nx + 2), dtype=torch.float64, device="cuda")


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
