"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: closed-form
values, exact invariants, brute-force dense solves, textbook Fourier
eigenvalues, or constants the paper prints (tests/golden/paper_constants.json).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import direct, kernels, multigrid as mg, operators as op, outputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


# ---------------------------------------------------------------- kernels
def test_peskin4_closed_form_points():
    # phi4 at r = 0, 1/2, 1, 3/2, 2 from the piecewise definition by hand.
    r = np.array([0.0, 0.5, 1.0, 1.5, 2.0, 2.5])
    want = [0.5, (2 + math.sqrt(2)) / 8, 0.25, (2 - math.sqrt(2)) / 8, 0.0, 0.0]
    np.testing.assert_allclose(kernels.phi4(r), want, rtol=0, atol=1e-16)
    np.testing.assert_allclose(kernels.phi3(np.array([0.0, 1.0, 1.5])), [2 / 3, 1 / 6, 0.0], atol=1e-16)


@pytest.mark.parametrize("w,sq", [(4, 3 / 8), (3, 1 / 2)])
def test_kernel_moment_conditions(w, sq):
    """Eq. JS_invariance: sum phi = 1, sum (q - r) phi = 0, sum phi^2 = 1/DeltaV."""
    rng = np.random.default_rng(11)
    j = np.arange(-5, 7)
    phi = kernels.KERNELS[w]
    for u in rng.random(50):
        v = phi(u - j)
        assert abs(v.sum() - 1) < 1e-15
        assert abs(((u - j) * v).sum()) < 1e-15
        assert abs((v * v).sum() - sq) < 1e-15
        if w == 4:
            assert abs(v[::2].sum() - 0.5) < 1e-15
    # Delta V = (sum phi^2)^-3 matches the printed (8/3)^3 h^3 and 2^3 h^3.
    key = "peskin4_volume_factor" if w == 4 else "peskin3_volume_factor"
    assert abs(1 / sq - GOLD[key]["value"]) < 1e-12


# ---------------------------------------------------------------- grid operator
def test_laplacian_fourier_eigenvalues():
    """A applied to a Fourier mode multiplies it by alpha + 4 chi/h^2 sum sin^2."""
    nx, ny, nz, h, chi, alpha = 8, 6, 10, 0.7, 1.3, 0.25
    k = (3, 1, 4)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = 2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz)
    mode = np.cos(ph) + 0.3 * np.sin(ph)
    lam = alpha + 4 * chi / h ** 2 * (math.sin(math.pi * k[0] / nx) ** 2 + math.sin(math.pi * k[1] / ny) ** 2
                                       + math.sin(math.pi * k[2] / nz) ** 2)
    np.testing.assert_allclose(op.apply_A(mode, h, chi, alpha), lam * mode, atol=1e-12)


def test_laplacian_point_stencil():
    c = np.zeros((6, 6, 6))
    c[2, 3, 4] = 1.0
    L = op.laplacian(c, 2.0)
    assert L[2, 3, 4] == -6 / 4
    for d in [(1, 3, 4), (3, 3, 4), (2, 2, 4), (2, 4, 4), (2, 3, 3), (2, 3, 5)]:
        assert L[d] == 1 / 4
    assert np.count_nonzero(L) == 7


@pytest.mark.parametrize("alpha", [0.0, 0.4])
def test_green_vs_dense(alpha):
    rng = np.random.default_rng(3)
    dims = (8, 4, 6)
    h, chi = 0.5, 2.0
    g = rng.standard_normal((6, 4, 8))
    A, _, _ = direct.dense_operator_matrices(np.zeros((0, 3)), dims, h, chi, alpha)
    if alpha == 0.0:
        want = np.linalg.lstsq(A, g.ravel(), rcond=None)[0]  # minimum-norm solution
    else:
        want = np.linalg.solve(A, g.ravel())
    got = op.green_apply(g, h, chi, alpha).ravel()
    np.testing.assert_allclose(got, want, atol=1e-12 * np.abs(want).max())
    if alpha == 0.0:
        assert abs(got.mean()) < 1e-14


def test_eigenvalues_vs_numpy_fft():
    """FFT of the point stencil column reproduces the closed-form eigenvalues."""
    dims = (8, 6, 4)
    h, chi, alpha = 1.5, 0.7, 0.2
    e = np.zeros((4, 6, 8))
    e[0, 0, 0] = 1.0
    col = op.apply_A(e, h, chi, alpha)
    np.testing.assert_allclose(np.real(np.fft.fftn(col)), op.helmholtz_eigenvalues(dims, h, chi, alpha), atol=1e-13)


# ---------------------------------------------------------------- J and S
def _blobs(n, dims, h, seed):
    rng = np.random.default_rng(seed)
    return rng.random((n, 3)) * np.array(dims) * h


def test_interp_reproduces_linear_fields():
    """Zeroth and first moments (Eq. JS_invariance) make J exact on constant and
    linear fields; this pins the cell-centre convention r_k = (k + 1/2) h."""
    dims = (16, 16, 16)
    h = 0.5
    rng = np.random.default_rng(5)
    q = 2.0 + rng.random((20, 3)) * 4.0      # supports stay inside, no wrap
    z, y, x = np.meshgrid((np.arange(16) + 0.5) * h, (np.arange(16) + 0.5) * h,
                          (np.arange(16) + 0.5) * h, indexing="ij")
    np.testing.assert_allclose(op.interp(np.ones((16, 16, 16)), q, h), 1.0, atol=1e-14)
    np.testing.assert_allclose(op.interp(x, q, h), q[:, 0], atol=1e-13)
    np.testing.assert_allclose(op.interp(y, q, h), q[:, 1], atol=1e-13)
    np.testing.assert_allclose(op.interp(z, q, h), q[:, 2], atol=1e-13)


@pytest.mark.parametrize("w", [4, 3])
def test_adjoint_mass_and_volume(w):
    dims = (12, 8, 10)
    h = 0.8
    q = _blobs(9, dims, h, 7)
    rng = np.random.default_rng(8)
    c = rng.standard_normal((10, 8, 12))
    lam = rng.standard_normal(9)
    S = op.spread(lam, q, dims, h, w)
    # S = h^-3 J^T (Sec. III.A): <J c, lam> = h^3 <c, S lam>
    assert abs(op.interp(c, q, h, w) @ lam - h ** 3 * np.sum(c * S)) < 1e-12
    # spreading preserves the total (Appendix A): h^3 sum S lam = sum lam
    assert abs(h ** 3 * S.sum() - lam.sum()) < 1e-12
    # J S 1 = Delta V^-1 for one blob (Eq. dV_JS), with Delta V = (8/3)^3 h^3 or 2^3 h^3
    one = op.interp(op.spread(np.ones(1), q[:1], dims, h, w), q[:1], h, w)[0]
    dv = (8 / 3) ** 3 if w == 4 else 8.0
    assert abs(one * dv * h ** 3 - 1) < 1e-12


def test_spread_brute_force_loop():
    """Spread compared with a pure-Python loop over cells and blobs."""
    dims = (5, 4, 6)
    h = 1.0
    q = np.array([[0.2, 3.9, 5.5], [2.5, 1.0, 2.25]])
    lam = np.array([1.5, -0.75])
    got = op.spread(lam, q, dims, h)
    want = np.zeros((6, 4, 5))
    for k in range(6):
        for j in range(4):
            for i in range(5):
                for b in range(2):
                    wgt = 1.0
                    for ax, (idx, n) in enumerate(((i, 5), (j, 4), (k, 6))):
                        d = q[b, ax] - (idx + 0.5)
                        d -= n * round(d / n)
                        wgt *= sum(float(kernels.phi4(np.array([d + m * n]))[0]) for m in (-1, 0, 1))
                    want[k, j, i] += lam[b] * wgt
    np.testing.assert_allclose(got, want, atol=1e-15)


# ---------------------------------------------------------------- direct solves
@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_saddle_schur_vs_dense(alpha):
    dims = (8, 8, 8)
    h, chi, zeta = 0.75, 1.7, 0.6
    rng = np.random.default_rng(21)
    q = np.array([[1.3, 2.7, 4.1], [4.5, 5.2, 0.9], [3.0, 0.4, 2.2]]) * h
    g = rng.standard_normal((8, 8, 8))
    f = rng.standard_normal(3)
    c, lam, _ = direct.solve_saddle(q, g, h, chi, alpha, zeta=zeta, f=f)
    cd, ld = direct.dense_saddle(q, g, h, chi, alpha, zeta=zeta, f=f)
    np.testing.assert_allclose(c, cd, atol=1e-12 * np.abs(cd).max())
    np.testing.assert_allclose(lam, ld, atol=1e-12 * np.abs(ld).max())


@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_reaction_schur_vs_dense(alpha):
    dims = (8, 8, 8)
    h, chi = 1.25, 0.9
    rng = np.random.default_rng(22)
    q = np.array([[1.3, 2.7, 4.1], [4.5, 5.2, 0.9], [3.0, 0.4, 2.2]]) * h
    kappa = np.array([0.3, 4.0, 0.0])
    g = rng.standard_normal((8, 8, 8))
    c, u, _ = direct.solve_reaction(q, kappa, g, h, chi, alpha)
    cd = direct.dense_reaction(q, kappa, g, h, chi, alpha)
    np.testing.assert_allclose(c, cd, atol=1e-12 * np.abs(cd).max())
    np.testing.assert_allclose(u, kappa * op.interp(cd, q, h), atol=1e-11 * np.abs(u).max())


def test_saddle_invariants():
    """Sum lambda = h^3 sum g / zeta (Appendix A) and J c = f / xi."""
    dims = (16, 16, 16)
    h, chi, zeta = 1.0, 1.0, 2.0
    q = _blobs(6, dims, h, 31)
    rng = np.random.default_rng(32)
    g = 1.0 + 0.2 * rng.standard_normal((16, 16, 16))
    f = 0.1 * rng.standard_normal(6)
    c, lam, _ = direct.solve_saddle(q, g, h, chi, 0.0, zeta=zeta, f=f)
    xi = zeta / h ** 3
    assert abs(lam.sum() - h ** 3 * g.sum() / zeta) < 1e-10 * abs(lam.sum())
    np.testing.assert_allclose(op.interp(c, q, h), f / xi, atol=1e-12)
    res = op.apply_A(c, h, chi, 0.0) + zeta * op.spread(lam, q, dims, h) - g
    assert np.abs(res).max() < 1e-11


def test_reaction_steady_balance():
    dims = (16, 16, 16)
    q = _blobs(5, dims, 1.0, 41)
    kappa = np.array([0.1, 1.0, 10.0, 3.0, 0.5])
    g = np.ones((16, 16, 16))
    c, u, _ = direct.solve_reaction(q, kappa, g, 1.0, 1.0, 0.0)
    assert abs(np.sum(kappa * op.interp(c, q, 1.0)) - g.sum()) < 1e-9 * g.sum()


def test_single_blob_finite_rate_shift():
    """Sec. III.D: for one periodic blob with a uniform source, c_P - c_0 is the
    constant lambda/kappa (here lambda = s V_Omega = 1)."""
    L = 16
    q = np.array([[7.3, 8.6, 8.1]])
    g = np.full((L, L, L), 1.0 / L ** 3)
    c0, lam, _ = direct.solve_saddle(q, g, 1.0, 1.0, 0.0)
    assert abs(lam[0] - 1.0) < 1e-12
    for kappa in (0.5, 7.0):
        cP, u, _ = direct.solve_reaction(q, np.array([kappa]), g, 1.0, 1.0, 0.0)
        np.testing.assert_allclose(cP - c0, 1.0 / kappa, atol=1e-11)


def test_cubic_lattice_equal_rates():
    L = 16
    from synthetic import lattice_positions
    q = lattice_positions((L, L, L), 1.0, 8, offset=(0.3, 0.3, 0.3))
    g = np.ones((L, L, L))
    c, lam, _ = direct.solve_saddle(q, g, 1.0, 1.0, 0.0)
    np.testing.assert_allclose(lam, lam.mean(), rtol=1e-11)


@pytest.mark.parametrize("w,key,tol", [(4, "reaction_radius_4pt_node", 0.015), (3, "reaction_radius_3pt_node", 0.01)])
def test_smoluchowski_reaction_radius(w, key, tol):
    """Sec. IV.A: single periodic blob at a grid node, s = 1/V_Omega; solving
    Eq. a_phi's series for a at L = 64 recovers the printed radius."""
    L = 64
    q = np.array([[L / 2, L / 2, L / 2]])
    g = np.full((L, L, L), 1.0 / L ** 3)
    c, lam, _ = direct.solve_saddle(q, g, 1.0, 1.0, 0.0, w=w)
    aL = outputs.reaction_radius(lam, c, 1.0)
    k = GOLD["radius_series_coefficient"]["value"]
    a = outputs.radius_from_series(aL, L, 1.0, k)
    assert abs(a - GOLD[key]["value"]) < tol * GOLD[key]["value"]
    # a_L decreases towards a as L grows (Eq. a_phi, positive correction)
    assert aL > a


# ---------------------------------------------------------------- multigrid
def test_transfer_operators_exact_on_linear():
    """Restriction (8-cell mean) and trilinear prolongation are exact on
    linear fields away from the periodic seam; both keep constants."""
    n = 8
    zc, yc, xc = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5, np.arange(n) + 0.5, indexing="ij")
    lin_c = 2.0 * xc - 0.5 * yc + 0.25 * zc           # coarse centres, spacing 2h, h = 1/2
    fine = mg.prolong(lin_c)
    zf, yf, xf = np.meshgrid((np.arange(2 * n) + 0.5) / 2, (np.arange(2 * n) + 0.5) / 2,
                             (np.arange(2 * n) + 0.5) / 2, indexing="ij")
    lin_f = 2.0 * xf - 0.5 * yf + 0.25 * zf
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(fine[inner], lin_f[inner], atol=1e-13)
    np.testing.assert_allclose(mg.restrict(lin_f), lin_c, atol=1e-13)
    np.testing.assert_allclose(mg.prolong(np.full((4, 4, 4), 3.0)), 3.0, atol=0)


def _rbgs_loop(x, b, h, chi, alpha):
    """One red-black Gauss-Seidel sweep written cell by cell: every red cell
    (i + j + k even) from its neighbours' current values, then every black
    cell, which then sees the red cells' new values."""
    nz, ny, nx = x.shape
    diag = alpha + 6.0 * chi / (h * h)
    off = chi / (h * h)
    for colour in (0, 1):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    if (i + j + k) % 2 != colour:
                        continue
                    s = (x[k, j, (i - 1) % nx] + x[k, j, (i + 1) % nx] + x[k, (j - 1) % ny, i]
                         + x[k, (j + 1) % ny, i] + x[(k - 1) % nz, j, i] + x[(k + 1) % nz, j, i])
                    x[k, j, i] = (b[k, j, i] + off * s) / diag
    return x


@pytest.mark.parametrize("alpha", [0.0, 0.35])
def test_rbgs_sweep_red_then_black_per_cell(alpha):
    """Sec. III.E smoother reading: the oracle's red-black sweep equals a
    per-cell loop that updates red cells, then black cells from the new red
    values (a Jacobi-ordered or colour-swapped sweep differs from it), on a
    non-cubic periodic grid; after the red half every red row of A x = b holds
    to rounding, and after the black half every black row does."""
    rng = np.random.default_rng(71)
    shape = (6, 4, 8)  # (nz, ny, nx)
    h, chi = 0.8, 1.3
    x0 = rng.standard_normal(shape)
    b = rng.standard_normal(shape)
    want = _rbgs_loop(x0.copy(), b, h, chi, alpha)
    got = mg.rbgs_sweep(x0.copy(), b, h, chi, alpha)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)
    k, j, i = np.meshgrid(np.arange(6), np.arange(4), np.arange(8), indexing="ij")
    red = (i + j + k) % 2 == 0
    x = x0.copy()
    mg.rbgs_half_sweep(x, b, h, chi, alpha, 0)
    r = b - op.apply_A(x, h, chi, alpha)
    assert np.abs(r[red]).max() < 1e-13 and np.abs(r[~red]).max() > 1e-3
    np.testing.assert_array_equal(x[~red], x0[~red])
    mg.rbgs_half_sweep(x, b, h, chi, alpha, 1)
    np.testing.assert_array_equal(x, got)
    r = b - op.apply_A(x, h, chi, alpha)
    assert np.abs(r[~red]).max() < 1e-13
    # the two plausible mistakes differ from the definition
    jac = x0.copy()
    nb = sum(np.roll(x0, s, axis=a) for a in range(3) for s in (1, -1))
    upd = (b + chi / h ** 2 * nb) / (alpha + 6 * chi / h ** 2)
    jac[red] = upd[red]
    jac[~red] = upd[~red]
    assert np.abs(jac - got).max() > 1e-3
    swapped = x0.copy()
    mg.rbgs_half_sweep(swapped, b, h, chi, alpha, 1)
    mg.rbgs_half_sweep(swapped, b, h, chi, alpha, 0)
    assert np.abs(swapped - got).max() > 1e-3


def test_level_shapes():
    assert [d for d, _ in mg.level_shapes((32, 32, 32), 1.0)] == [(32,) * 3, (16,) * 3, (8,) * 3, (4,) * 3, (2,) * 3]
    assert [d[0] for d, _ in mg.level_shapes((160, 160, 160), 1.0)] == [160, 80, 40, 20, 10, 5]
    assert [d[0] for d, _ in mg.level_shapes((96, 96, 96), 1.0)] == [96, 48, 24, 12, 6, 3]
    # the FP32 V-cycle's hierarchy: it ends at the first level of <= 32768 cells with no side above 64
    ex = dict(exact_cells=32768, exact_side=64)
    assert [d[0] for d, _ in mg.level_shapes((256,) * 3, 1.0, **ex)] == [256, 128, 64, 32]
    assert [d[0] for d, _ in mg.level_shapes((160,) * 3, 1.0, **ex)] == [160, 80, 40, 20]
    assert [d for d, _ in mg.level_shapes((32, 32, 32), 1.0, **ex)] == [(32,) * 3]
    # no level qualifies (a side stays above 64): the full hierarchy
    assert [d for d, _ in mg.level_shapes((256, 8, 2), 1.0, **ex)] == [(256, 8, 2)]


@pytest.mark.parametrize("exact", [{}, dict(exact_cells=32768, exact_side=64)])
@pytest.mark.parametrize("alpha", [0.0, 0.05])
def test_vcycle_fixed_point_and_reduction(alpha, exact):
    """A V-cycle started from the exact solution returns it; from zero it
    reduces the residual by at least the 5x the paper quotes (Sec. III.E);
    both for the full hierarchy and the one ending in an exact 16^3 level."""
    n, h, chi = 32, 1.0, 1.0
    rng = np.random.default_rng(51)
    x = rng.standard_normal((n, n, n))
    if alpha == 0.0:
        x -= x.mean()
    b = op.apply_A(x, h, chi, alpha)
    np.testing.assert_allclose(mg.vcycle(b, h, chi, alpha, x0=x, **exact), x, atol=1e-11)
    b2 = rng.standard_normal((n, n, n))
    if alpha == 0.0:
        b2 -= b2.mean()
    y = mg.vcycle(b2, h, chi, alpha, **exact)
    red = np.linalg.norm(b2) / np.linalg.norm(b2 - op.apply_A(y, h, chi, alpha))
    assert red >= GOLD["vcycle_residual_reduction"]["min"]


@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_coarse_solve_large_level_by_brute_force(alpha):
    """Levels above 512 cells are solved through the FFT Green's function:
    checked against the assembled dense operator at 10 x 10 x 8 (800 cells)."""
    rng = np.random.default_rng(62)
    shape = (8, 10, 10)
    b = rng.standard_normal(shape)
    if alpha == 0.0:
        b -= b.mean()
    h, chi = 2.0, 1.3
    n = b.size
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = op.apply_A(e.reshape(shape), h, chi, alpha).ravel()
    want = np.linalg.lstsq(A, b.ravel(), rcond=None)[0]  # minimum-norm solution when singular
    np.testing.assert_allclose(mg.coarse_solve(b, h, chi, alpha).ravel(), want, atol=1e-12)


def test_coarse_solve_vs_fft_green():
    rng = np.random.default_rng(61)
    b = rng.standard_normal((2, 2, 2))
    b -= b.mean()
    np.testing.assert_allclose(mg.coarse_solve(b, 16.0, 1.0, 0.0), op.green_apply(b, 16.0, 1.0, 0.0), atol=1e-13)
    b3 = rng.standard_normal((3, 3, 3))
    np.testing.assert_allclose(mg.coarse_solve(b3, 4.0, 1.0, 0.2), op.green_apply(b3, 4.0, 1.0, 0.2), atol=1e-13)
    # a non-cubic singular coarsest level (the (64, 48, 40) hierarchy ends at 8 x 6 x 5)
    b4 = rng.standard_normal((5, 6, 8))
    b4 -= b4.mean()
    np.testing.assert_allclose(mg.coarse_solve(b4, 8.0, 2.0, 0.0), op.green_apply(b4, 8.0, 2.0, 0.0), atol=1e-12)


def test_radius_series_inversion():
    """outputs.radius_from_series inverts Eq. a_phi (through its quadratic
    term): checked against the positive real root of the cubic
    a + k a^2 / (L h) + k^2 a^3 / (L h)^2 - a_L = 0 found by numpy.roots, for
    several box sizes, spacings and radii. The printed coefficient is the one
    in tests/golden."""
    k = GOLD["radius_series_coefficient"]["value"]
    assert outputs.RADIUS_SERIES_COEFFICIENT == k
    for aL, L, h in [(1.62, 16, 1.0), (1.43, 32, 1.0), (1.30, 128, 1.0), (0.74, 20, 0.5), (2.9, 16, 2.0)]:
        s = 1.0 / (L * h)
        roots = np.roots([k * k * s * s, k * s, 1.0, -aL])
        real = [r.real for r in roots if abs(r.imag) < 1e-12 and r.real > 0]
        assert len(real) == 1
        a = outputs.radius_from_series(aL, L, h)
        assert abs(a - real[0]) < 1e-13 * aL
        x = k * a * s
        assert abs(a * (1 + x + x * x) - aL) < 1e-13 * aL


def test_extrapolated_radius_is_first_order():
    """outputs.extrapolated_radius (Sec. IV.A: a ~ a_L - 2.84 a_L^2 / (L h))
    is the exact inverse of Eq. a_phi up to terms of second order in a/(L h):
    with a_L built from the series for a known a, its error divided by
    a (k a / (L h))^2 tends to a constant (-1 from the expansion
    a_L - k a_L^2/(L h) = a (1 - x^2 - 3 x^3 + ...), x = k a / (L h)), so doubling
    L quarters the error."""
    k = GOLD["radius_series_coefficient"]["value"]
    a = 1.27
    errs = []
    for L in (64, 128, 256, 512, 1024):
        x = k * a / L
        aL = a * (1 + x + x * x)
        e = outputs.extrapolated_radius(aL, L, 1.0) - a
        errs.append(e)
        assert abs(e / (a * x * x) + 1.0) < 4.0 * x  # next term: -3 x
    for e1, e2 in zip(errs, errs[1:]):
        assert 3.5 < e1 / e2 < 4.5
    # the paper's L = 128 study: the first-order form is within 0.1 % of the series inverse
    aL = a * (1 + k * a / 128 + (k * a / 128) ** 2)
    assert abs(outputs.extrapolated_radius(aL, 128, 1.0) - outputs.radius_from_series(aL, 128, 1.0)) < 1e-3 * a


def test_outputs_formulae():
    # Eq. beta_P_disc at phi -> 0 with s = 1/V: beta0 -> (4 pi a chi cbar)^-1 (Eq. beta0_low_phi)
    a, chi, V = 1.27, 1.0, 1e9
    cbar = 1.0 / (4 * math.pi * a * chi)
    b = outputs.beta0(cbar, 1.0 / V, a, chi, 1, V)
    assert abs(b - 1.0) < 1e-6
    assert abs(outputs.beta0_cubic_fit(0.0) - 1.0) < 1e-15


def test_translational_invariance_of_radius():
    """Sec. IV.A: moving the blob relative to the grid changes the reaction
    radius by about 1.5% (4-point) and 5% (3-point); the 4-point average is
    about 1.255h (caption of Fig. FarFieldDecay). L = 64, blob displaced from a
    cell centre along several directions."""
    L = 64
    offsets = [(0, 0, 0), (0.5, 0, 0), (0.5, 0.5, 0), (0.5, 0.5, 0.5)]
    res = {}
    for w in (4, 3):
        vals = []
        for d in offsets:
            q = np.array([[L / 2 + 0.5 + d[0], L / 2 + 0.5 + d[1], L / 2 + 0.5 + d[2]]])
            g = np.full((L, L, L), 1.0 / L ** 3)
            c, lam, _ = direct.solve_saddle(q, g, 1.0, 1.0, 0.0, w=w)
            vals.append(outputs.radius_from_series(outputs.reaction_radius(lam, c, 1.0), L, 1.0))
        res[w] = np.array(vals)
    v4, v3 = res[4], res[3]
    assert (v4.max() - v4.min()) / v4.mean() < 2 * GOLD["translational_variation_4pt"]["value"]
    assert abs(v4.mean() - GOLD["reaction_radius_4pt_average"]["value"]) < 0.01 * GOLD["reaction_radius_4pt_average"]["value"]
    var3 = (v3.max() - v3.min()) / v3.mean()
    assert 0.4 * GOLD["translational_variation_3pt"]["value"] < var3 < 1.5 * GOLD["translational_variation_3pt"]["value"]
    assert (v4.max() - v4.min()) / v4.mean() < var3   # the 4-point kernel is the more invariant one


@pytest.mark.parametrize("L,spacing", [(32, 8), (48, 12)])
def test_cubic_lattice_rate_matches_fit(L, spacing):
    """Sec. IV.B: a cubic array of blobs (at grid nodes, a = 1.27h) follows
    the paper's cubic-lattice fit Eq. beta_cubic (with its b = -0.92,
    c = 17.4) at low packing fraction."""
    from synthetic import lattice_positions
    q = lattice_positions((L, L, L), 1.0, spacing)
    V = L ** 3
    g = np.full((L, L, L), 1.0 / V)
    c, lam, _ = direct.solve_saddle(q, g, 1.0, 1.0, 0.0)
    a = GOLD["reaction_radius_4pt_node"]["value"]
    phi = len(q) * (4 * math.pi * a ** 3 / 3) / V
    b0 = outputs.beta0(c.mean(), 1.0 / V, a, 1.0, len(q), V)
    fit = outputs.beta0_cubic_fit(phi, GOLD["cubic_fit_b"]["value"], GOLD["cubic_fit_c"]["value"])
    assert abs(b0 - fit) < 0.01 * fit


def test_penalty_form_converges_to_saddle_point():
    """Sec. II.B: the reaction-limited system with a uniform rate kappa is a
    penalty form of the diffusion-limited saddle point; lambda = kappa J c of
    the reaction solution approaches the saddle point's multipliers as kappa
    grows, with an error that falls like 1/kappa."""
    from oracle import direct
    from synthetic import rsa_positions
    q = rsa_positions(5, (16, 16, 16), 1.0, 4.0, 8)
    g = np.ones((16, 16, 16))
    _, lam, _ = direct.solve_saddle(q, g, 1.0, 1.0, 0.0)
    errs = []
    for kappa in (1e2, 1e3, 1e4):
        _, u, _ = direct.solve_reaction(q, np.full(len(q), kappa), g, 1.0, 1.0, 0.0)
        errs.append(np.linalg.norm(u - lam) / np.linalg.norm(lam))
    assert errs[0] < 0.2
    assert 7.0 < errs[0] / errs[1] < 13.0 and 7.0 < errs[1] / errs[2] < 13.0
