"""Peskin regularized-delta kernels (oracle; test infrastructure only).

Sec. III.A fixes a tensor-product kernel phi_w of support w*h built on the grid
(Eq. tensor_product) and satisfying the moment conditions of Eq. JS_invariance:
sum phi = 1, sum (q - r_k) phi = 0, sum phi^2 = const = Delta V^-1. The paper
does not print the formulas; it cites Peskin's review for the 4-point kernel
(Delta V = (8/3)^d h^d) and the 3-point kernel (Delta V = 2^d h^d). The
piecewise forms below are the published ones (Peskin, Acta Numerica 2002; the
3-point form of Roma, Peskin and Berger 1999), restated here.
"""
from __future__ import annotations

import numpy as np


def phi4(r):
    """Peskin 4-point kernel, argument in units of h, support |r| < 2."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    a = r < 1.0
    b = (r >= 1.0) & (r < 2.0)
    ra = r[a]
    out[a] = (3.0 - 2.0 * ra + np.sqrt(1.0 + 4.0 * ra - 4.0 * ra * ra)) / 8.0
    rb = r[b]
    out[b] = (5.0 - 2.0 * rb - np.sqrt(-7.0 + 12.0 * rb - 4.0 * rb * rb)) / 8.0
    return out


def phi3(r):
    """Peskin 3-point kernel, argument in units of h, support |r| < 3/2."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    a = r <= 0.5
    b = (r > 0.5) & (r < 1.5)
    ra = r[a]
    out[a] = (1.0 + np.sqrt(1.0 - 3.0 * ra * ra)) / 3.0
    rb = r[b]
    out[b] = (5.0 - 3.0 * rb - np.sqrt(1.0 - 3.0 * (1.0 - rb) ** 2)) / 6.0
    return out


KERNELS = {4: phi4, 3: phi3}
SUPPORT = {4: 2.0, 3: 1.5}
