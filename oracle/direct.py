"""Exact solutions of the blob systems (oracle; test infrastructure only).

The paper's Krylov + multigrid solvers converge to the exact solution of a
linear system, so the oracle computes that solution directly.

* Diffusion-limited saddle point (Eq. saddle_point):
      A c + zeta S lambda = g,   xi J c = f,   A = alpha I - chi L.
  Schur elimination (Eqs. c_exact, r_schur): c = G (g - zeta S lambda),
  zeta M lambda = J G g - f/xi with M = J G S. When alpha = 0 the periodic A is
  singular; G is then the restricted (mean-zero) inverse, c gains an unknown
  constant cbar, and the solvability condition of Appendix A,
  zeta <S lambda> = <g>, i.e. sum(lambda) = h^3 sum(g) / zeta, closes the
  system (J 1 = 1 by the partition of unity in Eq. JS_invariance).
* Reaction-limited system (Eqs. unsteady_system, steady_state):
      (alpha I - chi L + S kappa J) c = g.
  With u = kappa * (J c): A c = g - S u. Eliminating c as above gives
  (I + kappa M) u = kappa J G g (alpha > 0) and, for alpha = 0, the extra
  unknown cbar with (I + kappa M) u - cbar kappa = kappa J G g and
  sum(u) = h^3 sum(g).
* ``dense_*``: brute-force assembly of the full (N_c + N) matrix from the
  operator definitions and a dense LU solve, for grids of a few hundred cells.
"""
from __future__ import annotations

import numpy as np

from . import operators as op


def schur_matrix(q, dims, h, chi, alpha, w=4):
    """M = J G S built column by column (N Green's-function solves)."""
    n = len(q)
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        col = op.green_apply(op.spread(e, q, dims, h, w), h, chi, alpha)
        M[:, j] = op.interp(col, q, h, w)
    return M


def solve_saddle(q, g, h, chi, alpha, zeta=1.0, xi=None, f=None, w=4, M=None):
    """Exact (c, lambda) of Eq. saddle_point; returns (c, lam, cbar)."""
    nz, ny, nx = g.shape
    dims = (nx, ny, nz)
    n = len(q)
    if xi is None:
        xi = zeta / h ** 3
    if f is None:
        f = np.zeros(n)
    if M is None:
        M = schur_matrix(q, dims, h, chi, alpha, w)
    rhs = op.interp(op.green_apply(g, h, chi, alpha), q, h, w) - f / xi
    if alpha > 0.0:
        lam = np.linalg.solve(zeta * M, rhs)
        cbar = 0.0
    else:
        K = np.zeros((n + 1, n + 1))
        K[:n, :n] = zeta * M
        K[:n, n] = -1.0
        K[n, :n] = 1.0
        b = np.concatenate([rhs, [h ** 3 * g.sum() / zeta]])
        sol = np.linalg.solve(K, b)
        lam, cbar = sol[:n], sol[n]
    c = op.green_apply(g - zeta * op.spread(lam, q, dims, h, w), h, chi, alpha) + cbar
    return c, lam, cbar


def solve_reaction(q, kappa, g, h, chi, alpha, w=4, M=None):
    """Exact c of (alpha I - chi L + S kappa J) c = g; returns (c, u, cbar)
    with u = kappa * (J c) the per-blob consumption rate."""
    nz, ny, nx = g.shape
    dims = (nx, ny, nz)
    n = len(q)
    kappa = np.asarray(kappa, dtype=np.float64)
    if M is None:
        M = schur_matrix(q, dims, h, chi, alpha, w)
    rhs = kappa * op.interp(op.green_apply(g, h, chi, alpha), q, h, w)
    B = np.eye(n) + kappa[:, None] * M
    if alpha > 0.0:
        u = np.linalg.solve(B, rhs)
        cbar = 0.0
    else:
        K = np.zeros((n + 1, n + 1))
        K[:n, :n] = B
        K[:n, n] = -kappa
        K[n, :n] = 1.0
        b = np.concatenate([rhs, [h ** 3 * g.sum()]])
        sol = np.linalg.solve(K, b)
        u, cbar = sol[:n], sol[n]
    c = op.green_apply(g - op.spread(u, q, dims, h, w), h, chi, alpha) + cbar
    return c, u, cbar


def dense_operator_matrices(q, dims, h, chi, alpha, w=4):
    """Dense A (N_c x N_c), S (N_c x N) and J (N x N_c) assembled by applying
    the operator definitions to unit vectors (tiny grids only)."""
    nx, ny, nz = dims
    nc = nx * ny * nz
    n = len(q)
    A = np.zeros((nc, nc))
    J = np.zeros((n, nc))
    for k in range(nc):
        e = np.zeros(nc)
        e[k] = 1.0
        e3 = e.reshape(nz, ny, nx)
        A[:, k] = op.apply_A(e3, h, chi, alpha).ravel()
        J[:, k] = op.interp(e3, q, h, w)
    S = np.zeros((nc, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        S[:, j] = op.spread(e, q, dims, h, w).ravel()
    return A, S, J


def dense_saddle(q, g, h, chi, alpha, zeta=1.0, xi=None, f=None, w=4):
    """Brute-force solve of [A zeta S; xi J 0][c; lambda] = [g; f]."""
    nz, ny, nx = g.shape
    n = len(q)
    if xi is None:
        xi = zeta / h ** 3
    if f is None:
        f = np.zeros(n)
    A, S, J = dense_operator_matrices(q, (nx, ny, nz), h, chi, alpha, w)
    nc = A.shape[0]
    K = np.zeros((nc + n, nc + n))
    K[:nc, :nc] = A
    K[:nc, nc:] = zeta * S
    K[nc:, :nc] = xi * J
    sol = np.linalg.solve(K, np.concatenate([g.ravel(), f]))
    return sol[:nc].reshape(g.shape), sol[nc:]


def dense_reaction(q, kappa, g, h, chi, alpha, w=4):
    """Brute-force solve of (A + S diag(kappa) J) c = g."""
    nz, ny, nx = g.shape
    A, S, J = dense_operator_matrices(q, (nx, ny, nz), h, chi, alpha, w)
    B = A + S @ (np.asarray(kappa)[:, None] * J)
    return np.linalg.solve(B, g.ravel()).reshape(g.shape)
