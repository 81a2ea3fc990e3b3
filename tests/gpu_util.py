"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import numpy as np
import torch

# Tolerances stated for the FP32 path and the BF16 tensor-core path.
TOL_OBJ_FP32 = 1e-5
TOL_GRAD_FP32 = 1e-4
TOL_BF16 = 3e-3


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_norm(got, ref):
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def gmm_dev(g):
    return [dev(a) for a in (g.x, g.alpha, g.mu, g.q, g.l)]


def status():
    return torch.zeros(1, dtype=torch.int32, device="cuda")
