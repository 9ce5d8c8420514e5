"""Pins of the iterative CPU solver (oracle/cpu_solver.c), the timed CPU baseline.

Its V-cycle must equal the NumPy oracle's V-cycle (which is pinned by a
per-cell loop, its fixed point and the Green's function) and its solves must
reach the direct Schur solutions of oracle/direct.py (pinned by brute-force
dense solves) within the rounding floor of the tolerance asked for.
"""
import numpy as np
import pytest

from oracle import cpu_solver as cs, direct, multigrid as mg, operators as op
from synthetic import loguniform_rates, rsa_positions
from tests.gpu_util import floor_tol, rel_err


@pytest.fixture(scope="module", autouse=True)
def lib():
    cs.build()


@pytest.mark.parametrize("shape,shift", [((32, 24, 16), 0.0), ((16, 16, 16), 0.3), ((8, 20, 12), 0.0)])
def test_vcycle_equals_numpy_definition(shape, shift):
    rng = np.random.default_rng(81)
    b = rng.standard_normal(shape)
    x0 = rng.standard_normal(shape)
    h, chi = 0.7, 1.3
    for guess in (None, x0):
        got = cs.vcycle(b, h, chi, shift, x0=guess)
        want = mg.vcycle(b, h, chi, shift, x0=guess)
        assert rel_err(got, want) < 1e-13
    got = cs.vcycle(b, h, chi, shift, nu1=1, nu2=3)
    assert rel_err(got, mg.vcycle(b, h, chi, shift, nu1=1, nu2=3)) < 1e-13


CASES = [((16, 24, 32), 0.5, 1.3, 4), ((24, 24, 24), 1.0, 1.0, 3), ((20, 12, 16), 2.0, 0.7, 4)]


@pytest.mark.parametrize("dims,h,chi,w", CASES)
@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_reaction_solve_reaches_direct_solution(dims, h, chi, w, alpha):
    rng = np.random.default_rng(82)
    q = rsa_positions(9, dims, h, 3.0 * h, 83)
    kappa = loguniform_rates(len(q), 0.1, 10.0, 84)
    nx, ny, nz = dims
    g = 1.0 + 0.5 * rng.random((nz, ny, nx))
    c_ref, u_ref, _ = direct.solve_reaction(q, kappa, g, h, chi, alpha, w=w)
    tol = floor_tol(c_ref, g, h, chi, alpha, base=1e-12 if alpha == 0.0 else 1e-14)
    c, info = cs.solve_reaction(q, kappa, g, h, chi, alpha, w=w, tol=tol, max_iter=600)
    assert info["status"] == 0 and info["rel_residual"] <= tol
    assert info["threads"] >= 1 and info["vcycles"] == info["outer_iters"]
    assert rel_err(c, c_ref) < 1e-11
    assert rel_err(kappa * op.interp(c, q, h, w), u_ref) < 1e-10


@pytest.mark.parametrize("dims,h,chi,w", CASES)
@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_saddle_solve_reaches_direct_solution(dims, h, chi, w, alpha):
    rng = np.random.default_rng(85)
    q = rsa_positions(9, dims, h, 3.0 * h, 86)
    nx, ny, nz = dims
    g = 1.0 + 0.5 * rng.random((nz, ny, nx))
    f = 0.05 * rng.standard_normal(len(q))
    zeta = 0.6
    c_ref, lam_ref, _ = direct.solve_saddle(q, g, h, chi, alpha, zeta=zeta, f=f, w=w)
    # alpha > 0 has no large constant mode, so the solve can go below 1e-12
    tol = floor_tol(c_ref, g, h, chi, alpha, base=1e-12 if alpha == 0.0 else 1e-14)
    c, lam, info = cs.solve_saddle(q, g, h, chi, alpha, zeta=zeta, f=f, w=w, tol=tol, max_iter=600)
    assert info["status"] == 0 and info["rel_residual"] <= tol
    # Appendix A: seven V-cycles per outer iteration with n = 1, m = 5
    assert info["inner_iters"] == 5 * info["outer_iters"] and info["vcycles"] == 7 * info["outer_iters"]
    assert rel_err(c, c_ref) < 1e-11 and rel_err(lam, lam_ref) < 1e-11
    if alpha == 0.0:
        assert abs(lam.sum() - h ** 3 * g.sum() / zeta) < 1e-9 * abs(lam.sum())


def test_not_converged_is_reported():
    q = rsa_positions(6, (16, 16, 16), 1.0, 4.0, 87)
    g = np.ones((16, 16, 16))
    c, lam, info = cs.solve_saddle(q, g, 1.0, 1.0, 0.0, tol=1e-14, max_iter=2)
    assert info["status"] == 1 and info["outer_iters"] == 2 and info["rel_residual"] > 1e-14
    c, info = cs.solve_reaction(q, np.ones(6), g, 1.0, 1.0, 0.0, tol=1e-14, max_iter=3)
    assert info["status"] == 1 and info["outer_iters"] == 3
