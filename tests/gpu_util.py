"""Helpers for the GPU parity tests (host side only)."""
import numpy as np


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_max(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_err(a, b):
    """The larger of the element-wise error (max |a - b| over max |b|) and
    the relative L2 error: a parity bound on it bounds every element."""
    return max(rel_max(a, b), rel_l2(a, b))


EPS = 2.220446049250313e-16


def floor_tol(c_ref, g, h, chi, alpha, base=1e-12):
    """Relative-residual tolerance at the FP64 rounding floor: A c is formed
    from values of size max|c|, so each cell of the residual carries about
    eps (alpha + 12 chi/h^2) max|c| of rounding; relative to the rms of g that
    is the floor. A few times it, and never below `base`."""
    rms = float(np.sqrt(np.mean(np.asarray(g) ** 2)))
    fl = 4.0 * EPS * (alpha + 12.0 * chi / h ** 2) * float(np.abs(c_ref).max()) / rms
    return max(base, fl)
