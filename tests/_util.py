"""Helpers shared by the tests (no method arithmetic)."""
import numpy as np

TOL_COMP = 2e-6   # compensated FP32 vs the FP64 oracle, relative L2 per output
TOL_PLAIN = 1e-4  # plain FP32


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def to_dev(a, dev="cuda"):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def planar_to_rows(t, k):
    """[k, n] planar tensor -> numpy [n, k]."""
    return t.detach().cpu().numpy().reshape(k, -1).T.astype(np.float64)


def grad_rows(t):
    """[9, n] planar gradient -> numpy [n, 3, 3]."""
    return t.detach().cpu().numpy().T.reshape(-1, 3, 3).astype(np.float64)
