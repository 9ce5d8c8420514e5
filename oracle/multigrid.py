"""Geometric-multigrid V-cycle definition (oracle; test infrastructure only).

Sec. III.E solves the Helmholtz/Poisson problem A c = g, A = alpha I - chi L,
with geometric multigrid V-cycles and uses them as preconditioners; the paper
takes the multigrid from a library and does not describe its internals. The
GPU library fixes these readings, and this module states them plainly:

* Levels: level l+1 halves every dimension of level l; coarsening continues
  while all dimensions are even and at least 4. Each level re-discretizes
  A_l = alpha I - chi L_{h_l} with h_l = 2^l h.
* Smoother: red-black Gauss-Seidel, red = cells with (i + j + k) even, each
  sweep updates red then black; nu1 sweeps before and nu2 after the coarse
  correction.
* Restriction: the mean of the 8 fine cells covering a coarse cell.
* Prolongation: cell-centred trilinear interpolation (weights 3/4, 1/4 per
  axis from the two nearest coarse centres).
* Coarsest level: solved exactly; when alpha = 0 with the pseudo-inverse, which
  is the restricted inverse of Appendix A (mean-zero in, mean-zero out).
  The FP32 V-cycle of the GPU library stops coarsening earlier, at the first
  level with at most 32768 cells and no side above 64, and solves that level
  exactly (``exact_cells`` / ``exact_side`` below); the FP64 V-cycle coarsens
  to the end.
* When alpha = 0 the right-hand side is first projected to mean zero and the
  returned field is projected to mean zero (Appendix A's restricted inverse).
"""
from __future__ import annotations

import numpy as np

from . import operators as op


def level_shapes(dims, h, exact_cells=None, exact_side=None):
    """List of ((nx, ny, nz), h_l) from finest to coarsest. With exact_cells
    (and exact_side), the list ends at the first level with at most
    exact_cells cells and no side above exact_side, if one exists."""
    out = [(tuple(int(v) for v in dims), float(h))]
    if exact_cells is not None:
        full = level_shapes(dims, h)
        for i, (d, _) in enumerate(full):
            if d[0] * d[1] * d[2] <= exact_cells and max(d) <= exact_side:
                return full[:i + 1]
        return full
    while True:
        d, hl = out[-1]
        if all(v % 2 == 0 and v >= 4 for v in d):
            out.append((tuple(v // 2 for v in d), 2.0 * hl))
        else:
            return out


def _colour_masks(shape):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    red = ((i + j + k) % 2) == 0
    return red, ~red


def rbgs_half_sweep(x, b, h, chi, alpha, colour):
    """Gauss-Seidel update of every cell of one colour (0 = red, 1 = black) of
    A x = b, in place: each such cell solves its own row of A x = b with its
    six neighbours (all of the other colour) held at their current values."""
    mask = _colour_masks(x.shape)[colour]
    diag = alpha + 6.0 * chi / (h * h)
    off = chi / (h * h)
    nb = np.zeros_like(x)
    for ax in range(3):
        nb += np.roll(x, 1, axis=ax) + np.roll(x, -1, axis=ax)
    x[mask] = ((b + off * nb) / diag)[mask]
    return x


def rbgs_sweep(x, b, h, chi, alpha):
    """One red-black Gauss-Seidel sweep on A x = b (in place): the red half
    from the old black values, then the black half from the new red values."""
    rbgs_half_sweep(x, b, h, chi, alpha, 0)
    rbgs_half_sweep(x, b, h, chi, alpha, 1)
    return x


def restrict(r):
    """8-cell mean."""
    nz, ny, nx = r.shape
    return r.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))


def _prolong_axis(e, axis):
    n = e.shape[axis]
    lo = np.roll(e, 1, axis=axis)    # coarse neighbour I-1
    hi = np.roll(e, -1, axis=axis)   # coarse neighbour I+1
    even = 0.75 * e + 0.25 * lo      # fine cell 2I
    odd = 0.75 * e + 0.25 * hi       # fine cell 2I+1
    out_shape = list(e.shape)
    out_shape[axis] = 2 * n
    out = np.empty(out_shape)
    sl_e = [slice(None)] * 3
    sl_o = [slice(None)] * 3
    sl_e[axis] = slice(0, 2 * n, 2)
    sl_o[axis] = slice(1, 2 * n, 2)
    out[tuple(sl_e)] = even
    out[tuple(sl_o)] = odd
    return out


def prolong(e):
    """Cell-centred trilinear interpolation to the next finer level."""
    out = e
    for ax in range(3):
        out = _prolong_axis(out, ax)
    return out


def coarse_solve(b, h, chi, alpha):
    """Exact coarsest solve (pseudo-inverse when alpha = 0): from the assembled
    dense matrix up to 512 cells, by the FFT Green's function above."""
    nz, ny, nx = b.shape
    n = b.size
    if n > 512:
        return op.green_apply(b, h, chi, alpha)
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = op.apply_A(e.reshape(b.shape), h, chi, alpha).ravel()
    if alpha == 0.0:
        # the minimum-norm least-squares solution: the pseudo-inverse applied
        # to b, computed directly (an explicit pinv loses accuracy on some
        # non-cubic singular operators)
        x = np.linalg.lstsq(A, b.ravel(), rcond=None)[0]
    else:
        x = np.linalg.solve(A, b.ravel())
    return x.reshape(b.shape)


def _vcycle(levels, l, b, x, chi, alpha, nu1, nu2):
    dims, h = levels[l]
    if l == len(levels) - 1:
        return coarse_solve(b, h, chi, alpha)
    for _ in range(nu1):
        rbgs_sweep(x, b, h, chi, alpha)
    r = b - op.apply_A(x, h, chi, alpha)
    bc = restrict(r)
    xc = _vcycle(levels, l + 1, bc, np.zeros_like(bc), chi, alpha, nu1, nu2)
    x += prolong(xc)
    for _ in range(nu2):
        rbgs_sweep(x, b, h, chi, alpha)
    return x


def vcycle(b, h, chi, alpha, x0=None, nu1=2, nu2=2, exact_cells=None, exact_side=None):
    """One V-cycle for A x = b from x0 (zero if None); returns the new x. The
    hierarchy follows level_shapes (exact_cells / exact_side as there)."""
    nz, ny, nx = b.shape
    levels = level_shapes((nx, ny, nz), h, exact_cells, exact_side)
    b = np.array(b, dtype=np.float64)
    if alpha == 0.0:
        b = b - b.mean()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    x = _vcycle(levels, 0, b, x, chi, alpha, nu1, nu2)
    if alpha == 0.0:
        x = x - x.mean()
    return x
