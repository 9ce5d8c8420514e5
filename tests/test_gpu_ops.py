"""Op-level parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: apply_L, J and S differ from the oracle only in summation order
(a few ulp of the largest term), so they must agree to 1e-14 relative (max
norm). The V-cycle chains about 4 log2(n) kernels, each adding such rounding,
and must agree to 1e-12.
"""
import numpy as np
import pytest

from oracle import multigrid as mg, operators as op
from synthetic import rsa_positions
from tests.gpu_util import dev, host, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibrd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1306_3159_gb300 import build
    build.build()
    import paper_1306_3159_gb300 as p
    return p


CASES = [((32, 32, 32), 1.0, 1.0, 0.0), ((20, 12, 24), 0.7, 1.3, 0.25), ((8, 8, 8), 1.0, 1.0, 0.0),
         ((64, 48, 40), 1.0, 2.0, 0.05)]


@pytest.mark.parametrize("dims,h,chi,alpha", CASES)
def test_apply_L(ibrd, dims, h, chi, alpha):
    g = ibrd.Grid(*dims, h=h, chi=chi, alpha=alpha)
    nx, ny, nz = dims
    c = np.random.default_rng(1).standard_normal((nz, ny, nx))
    y = host(g.apply_L(dev(c)))
    assert rel_max(y, op.apply_A(c, h, chi, alpha)) < 1e-14


def _exact_residual(b, c, h, chi, alpha):
    """r = b - (diag c - off * sum of the 6 neighbours) in exact rational
    arithmetic on the library's double coefficients (off = chi / h^2, diag =
    alpha + 6 off, as the library rounds them)."""
    from fractions import Fraction as F
    off = chi / (h * h)
    diag = alpha + 6.0 * off
    to_q = np.vectorize(F, otypes=[object])
    cq = to_q(c)
    s = sum(np.roll(cq, sh, axis=a) for a in range(3) for sh in (1, -1))
    return to_q(b) - (F(diag) * cq - F(off) * s)


def _abs_err(r, exact):
    from fractions import Fraction as F
    return np.vectorize(lambda g, e: float(abs(F(float(g)) - e)), otypes=[float])(r, exact)


# dims, h, chi, alpha, whether the fixed-point form applies (nx % 32 == 0 and ny % 8 == 0)
RESID_CASES = [((32, 8, 4), 1.0, 1.0, 0.0, True), ((64, 32, 12), 0.5, 1.3, 0.7, True),
               ((96, 16, 8), 1.0, 2.0, 0.0, True), ((20, 12, 24), 0.7, 1.3, 0.25, False)]


@pytest.mark.parametrize("dims,h,chi,alpha,fx", RESID_CASES)
@pytest.mark.parametrize("field", ["random", "cancelling"])
def test_residual_against_exact_arithmetic(ibrd, dims, h, chi, alpha, fx, field):
    """ibrd_residual (the grid part of every FP64 residual of the solvers)
    against r = b - A c in exact rational arithmetic, cell by cell. Where the
    fixed-point form applies the error is within 2^-52 of |r| + |alpha c| +
    chi/h^2 |L c| plus 2^-55 chi/h^2 max|c| from the scaling (bounded here by
    2^-50 and 2^-54), and with alpha = 0 on a smooth field of size 1e6 (the
    neighbour sums cancel to 1e-4 of their terms, as near convergence) it is
    over ten times below the FP64 stencil's error. Elsewhere the FP64
    stencil's bound holds (2^-49 of diag |c| + chi/h^2 sum |c_nb| + |b|)."""
    nx, ny, nz = dims
    rng = np.random.default_rng(5 + nx)
    off = chi / (h * h)
    if field == "random":
        c = rng.standard_normal((nz, ny, nx))
        b = rng.standard_normal((nz, ny, nx))
    else:
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        smooth = np.sin(2 * np.pi * i / nx) * np.cos(2 * np.pi * j / ny) + np.sin(2 * np.pi * k / nz)
        c = 1e6 + 1e2 * smooth + 1e-3 * rng.standard_normal((nz, ny, nx))
        b = op.apply_A(c, h, chi, alpha) + 1e-3 * rng.standard_normal((nz, ny, nx))
    g = ibrd.Grid(*dims, h=h, chi=chi, alpha=alpha)
    r = host(g.residual(dev(b), dev(c)))
    exact = _exact_residual(b, c, h, chi, alpha)
    err = _abs_err(r, exact)
    nb_abs_diff = sum(np.abs(np.roll(c, sh, axis=a) - c) for a in range(3) for sh in (1, -1))
    nb_abs = sum(np.abs(np.roll(c, sh, axis=a)) for a in range(3) for sh in (1, -1))
    if fx:
        bound = 2.0 ** -50 * (np.abs(b) + abs(alpha) * np.abs(c) + off * nb_abs_diff) \
            + 2.0 ** -54 * off * np.abs(c).max()
    else:
        bound = 2.0 ** -49 * (np.abs(b) + (alpha + 6 * off) * np.abs(c) + off * nb_abs)
    assert (err <= bound).all(), float((err / bound).max())
    if fx and field == "cancelling" and alpha == 0.0:
        err64 = _abs_err(b - op.apply_A(c, h, chi, alpha), exact)
        assert err.max() < 0.1 * err64.max(), (err.max(), err64.max())


def test_residual_special_values(ibrd):
    """The fixed-point residual's edges: integer fields with binary
    coefficients come out exact; c = 0 gives b bit for bit; a NaN in c makes
    its cell and its six neighbours NaN and leaves the rest finite; c beyond
    the fixed-point window (1e300) takes the FP64 stencil, within its bound;
    right-hand sides of very different sizes (1e-30 next to 1) stay within the
    fixed-point bound."""
    dims = (64, 16, 8)
    nx, ny, nz = dims
    rng = np.random.default_rng(77)
    g = ibrd.Grid(*dims, h=1.0, chi=1.0, alpha=0.5)
    c = rng.integers(-2 ** 20, 2 ** 20, (nz, ny, nx)).astype(np.float64)
    b = rng.integers(-2 ** 20, 2 ** 20, (nz, ny, nx)).astype(np.float64)
    r = host(g.residual(dev(b), dev(c)))
    assert np.array_equal(r, b - op.apply_A(c, 1.0, 1.0, 0.5))  # every value exact in FP64 here
    bf = rng.standard_normal((nz, ny, nx))
    assert np.array_equal(host(g.residual(dev(bf), dev(np.zeros_like(bf)))), bf)
    cn = rng.standard_normal((nz, ny, nx))
    cn[3, 5, 7] = np.nan
    rn = host(g.residual(dev(bf), dev(cn)))
    bad = np.zeros_like(rn, dtype=bool)
    for (kk, jj, ii) in [(3, 5, 7), (2, 5, 7), (4, 5, 7), (3, 4, 7), (3, 6, 7), (3, 5, 6), (3, 5, 8)]:
        bad[kk, jj, ii] = True
    assert np.isnan(rn[bad]).all() and np.isfinite(rn[~bad]).all()
    cc = 1e300 * rng.standard_normal((nz, ny, nx))
    rr = host(g.residual(dev(bf), dev(cc)))
    nb = sum(np.abs(np.roll(cc, sh, axis=a)) for a in range(3) for sh in (1, -1))
    assert (np.abs(rr - (bf - op.apply_A(cc, 1.0, 1.0, 0.5))) <= 2.0 ** -49 * (np.abs(bf) + 6.5 * np.abs(cc) + nb)).all()
    bt = np.where(rng.random((nz, ny, nx)) < 0.1, 1e-30, 1.0)
    rt = host(g.residual(dev(bt), dev(bf)))
    exact = _exact_residual(bt, bf, 1.0, 1.0, 0.5)
    d = sum(np.abs(np.roll(bf, sh, axis=a) - bf) for a in range(3) for sh in (1, -1))
    assert (_abs_err(rt, exact) <= 2.0 ** -50 * (np.abs(bt) + 0.5 * np.abs(bf) + d) + 2.0 ** -54 * np.abs(bf).max()).all()


def _blobs(dims, h, n, seed):
    q = np.random.default_rng(seed).random((n, 3)) * np.array(dims) * h
    # include grid nodes, the domain edge and wrapped coordinates
    extra = np.array([[0.0, 0.0, 0.0], [dims[0] * h - 1e-9, 0.5 * h, dims[2] * h * 0.5],
                      [-0.3 * h, dims[1] * h + 0.2 * h, 2.0 * h]])
    return np.vstack([q, extra])


@pytest.mark.parametrize("dims,h", [((32, 32, 32), 1.0), ((20, 12, 24), 0.7), ((8, 8, 8), 1.0)])
@pytest.mark.parametrize("kernel", [4, 3])
def test_interp_and_spread(ibrd, dims, h, kernel):
    nx, ny, nz = dims
    q = _blobs(dims, h, 37, 2)
    g = ibrd.Grid(*dims, h=h, kernel=kernel)
    g.set_blobs(dev(q))
    rng = np.random.default_rng(3)
    c = rng.standard_normal((nz, ny, nx))
    lam = rng.standard_normal(len(q))
    qw = q % (np.array(dims) * h)
    assert rel_max(host(g.interp(dev(c))), op.interp(c, qw, h, kernel)) < 1e-14
    s_ref = op.spread(lam, qw, dims, h, kernel)
    s1 = host(g.spread(dev(lam)))
    assert rel_max(s1, s_ref) < 1e-14
    # deterministic: bitwise identical on repeat
    assert np.array_equal(host(g.spread(dev(lam))), s1)
    # accumulate adds onto the existing field
    base = rng.standard_normal((nz, ny, nx))
    out = dev(base)
    g.spread(dev(lam), out, accumulate=True)
    assert rel_max(host(out), base + s_ref) < 1e-14


def test_spread_interp_no_blobs(ibrd):
    import torch
    g = ibrd.Grid(16, 16, 16)
    g.set_blobs(torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    out = g.spread(torch.zeros(0, dtype=torch.float64, device="cuda"), g.field(5.0))
    assert float(out.abs().max()) == 0.0


def test_spread_many_blobs_per_tile(ibrd):
    """Dense packing: about 20 blobs per 8^3 tile (overlapping supports)."""
    dims = (32, 32, 32)
    q = np.random.default_rng(9).random((1500, 3)) * 32.0
    g = ibrd.Grid(*dims)
    g.set_blobs(dev(q))
    lam = np.random.default_rng(10).standard_normal(1500)
    assert rel_max(host(g.spread(dev(lam))), op.spread(lam, q, dims, 1.0)) < 1e-13


@pytest.mark.parametrize("dims,h,chi,alpha", CASES)
@pytest.mark.parametrize("zero", [True, False])
def test_vcycle(ibrd, dims, h, chi, alpha, zero):
    nx, ny, nz = dims
    rng = np.random.default_rng(4)
    b = rng.standard_normal((nz, ny, nx))
    x0 = rng.standard_normal((nz, ny, nx))
    g = ibrd.Grid(*dims, h=h, chi=chi, alpha=alpha)
    xd = dev(x0)
    g.vcycle(dev(b), xd, zero_initial_guess=zero)
    want = mg.vcycle(b, h, chi, alpha, x0=None if zero else x0)
    assert rel_max(host(xd), want) < 1e-12


def test_vcycle_reduction_matches_paper(ibrd):
    """Sec. III.E quotes a 5-10x residual reduction per V-cycle."""
    n = 64
    rng = np.random.default_rng(5)
    b = rng.standard_normal((n, n, n))
    b -= b.mean()
    g = ibrd.Grid(n, n, n)
    x = host(g.vcycle(dev(b)))
    red = np.linalg.norm(b) / np.linalg.norm(b - op.apply_A(x, 1.0, 1.0, 0.0))
    assert red > 5.0


def test_set_blobs_rejects_nonfinite(ibrd):
    g = ibrd.Grid(16, 16, 16)
    q = np.array([[1.0, 2.0, np.nan]])
    with pytest.raises(ibrd.IbrdError) as e:
        g.set_blobs(dev(q))
    assert e.value.status == 6


@pytest.mark.parametrize("dims,alpha", [((64, 64, 64), 0.0), ((32, 32, 32), 0.1), ((128, 64, 32), 0.0)])
def test_vcycle_f32(ibrd, dims, alpha):
    """The FP32 V-cycle of the mixed-precision solves against the FP64 oracle
    definition: FP32 rounding (2^-24 per operation, amplified by about ten
    smoothing and transfer steps) bounds the difference near 1e-6 relative."""
    import torch
    nx, ny, nz = dims
    rng = np.random.default_rng(7)
    b = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    g = ibrd.Grid(*dims, alpha=alpha)
    x = g.vcycle_f32(torch.from_numpy(b).cuda())
    # the FP32 hierarchy ends at an exact level of at most 32768 cells
    want = mg.vcycle(b.astype(np.float64), 1.0, 1.0, alpha, exact_cells=32768, exact_side=64)
    assert rel_max(x.cpu().numpy().astype(np.float64), want) < 2e-5


@pytest.mark.parametrize("dims,alpha", [((16, 16, 16), 0.0), ((12, 8, 20), 0.3), ((40, 40, 40), 0.0),
                                        ((24, 24, 24), 0.0), ((40, 40, 20), 0.2), ((64, 64, 8), 0.0),
                                        ((32, 32, 32), 0.1), ((64, 32, 16), 0.0)])
def test_vcycle_f32_exact_level(ibrd, dims, alpha):
    """FP32 V-cycles whose hierarchy ends in the exact Hartley-transform solve:
    at 16^3 and 12 x 8 x 20 the finest level itself is exact (one CTA; the
    result is the FFT Green's function solution); at 40^3 the exact level is
    10^3 below two smoothed levels; 24^3, 32^3, 40 x 40 x 20, 64 x 32 x 16 and
    64 x 64 x 8 are exact levels above 4096 cells (three launches: plane
    transforms, column transforms with the scaling, plane transforms; lines
    of 16 and 32 values register-blocked, the others generic)."""
    import torch
    nx, ny, nz = dims
    rng = np.random.default_rng(17)
    b = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    g = ibrd.Grid(*dims, alpha=alpha)
    x = g.vcycle_f32(torch.from_numpy(b).cuda()).cpu().numpy().astype(np.float64)
    want = mg.vcycle(b.astype(np.float64), 1.0, 1.0, alpha, exact_cells=32768, exact_side=64)
    assert rel_max(x, want) < 2e-5
    if nx * ny * nz <= 32768:
        bb = b.astype(np.float64)
        if alpha == 0.0:
            bb = bb - bb.mean()
        assert rel_max(x, op.green_apply(bb, 1.0, 1.0, alpha)) < 2e-5


def test_vcycle_smoother_variants_agree(ibrd):
    """Grids whose finest levels use the fused one-pass sweep and grids small
    enough to run entirely in the single-CTA coarse V-cycle follow the same
    definition (checked against the oracle at both sizes)."""
    for dims in [(256, 16, 8), (16, 16, 16)]:
        nx, ny, nz = dims
        b = np.random.default_rng(8).standard_normal((nz, ny, nx))
        g = ibrd.Grid(*dims)
        assert rel_max(host(g.vcycle(dev(b))), mg.vcycle(b, 1.0, 1.0, 0.0)) < 1e-12


TUNE_DIMS = (128, 64, 80)  # levels 128x64x80, 64x32x40 (FP32 exact level 32x16x20); FP64 coarsens to 8x4x5
TUNE_LEVELS = [(128, 64, 80), (64, 32, 40), (32, 16, 20)]


def _vcycle_both(ibrd, g, seed):
    import torch
    nx, ny, nz = TUNE_DIMS
    b = np.random.default_rng(seed).standard_normal((nz, ny, nx))
    x64 = host(g.vcycle(dev(b)))
    x32 = g.vcycle_f32(torch.from_numpy(b.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    assert rel_max(x64, mg.vcycle(b, 1.0, 1.0, 0.0)) < 1e-12
    b32 = b.astype(np.float32).astype(np.float64)
    assert rel_max(x32, mg.vcycle(b32, 1.0, 1.0, 0.0, exact_cells=32768, exact_side=64)) < 2e-5


@pytest.mark.parametrize("tx,zc", [(32, 2), (32, 3), (64, 7), (64, 80), (0, 12)])
def test_vcycle_tuned_shapes(ibrd, tx, zc):
    """Launch shapes the autotuner may keep (tile width 32 or 64, z-march depths
    with a ragged last chunk, down to one CTA per column) give the V-cycle of
    the oracle definition, FP64 and FP32, on every level that runs the sweep
    kernels."""
    g = ibrd.Grid(*TUNE_DIMS)
    for (nx, ny, nz) in TUNE_LEVELS:
        t32 = tx if (tx != 64 or nx % 64 == 0) else 32
        ibrd.ibrd_tune_set(g.handle, 4, 0, nx, ny, nz, t32, zc)
        ibrd.ibrd_tune_set(g.handle, 4, 1, nx, ny, nz, 0, max(1, zc // 2))
        ibrd.ibrd_tune_set(g.handle, 8, 0, nx, ny, nz, 32 if tx else 0, zc)
    _vcycle_both(ibrd, g, 21)


def test_autotune_report_and_parity(ibrd):
    """The autotuner times every level that runs the sweep kernels, keeps a
    shape only when it is faster than the built-in one, reuses its results for
    a second handle of the same grid, and leaves the V-cycle's definition
    unchanged."""
    g = ibrd.Grid(*TUNE_DIMS)
    rep = ibrd.ibrd_autotune(g.handle, -1, retune=True)
    seen = {(r["elem_bytes"], r["kind"], (r["nx"], r["ny"], r["nz"])) for r in rep}
    assert (4, 0, TUNE_LEVELS[0]) in seen and (4, 0, TUNE_LEVELS[1]) in seen and (4, 1, TUNE_LEVELS[0]) in seen
    assert (8, 0, TUNE_LEVELS[2]) in seen and (4, 0, TUNE_LEVELS[2]) not in seen  # FP32 exact level
    for r in rep:
        assert 0 < r["us_tuned"] <= r["us_default"] and r["cached"] == 0
        assert (r["zc"] == 0) == (r["us_tuned"] == r["us_default"])
    _vcycle_both(ibrd, g, 22)
    g2 = ibrd.Grid(*TUNE_DIMS)
    rep2 = ibrd.ibrd_autotune(g2.handle, -1)
    assert all(r["cached"] == 1 for r in rep2) and len(rep2) == len(rep)
    ibrd.ibrd_tune_clear(g.handle)
    _vcycle_both(ibrd, g, 23)


# Levels with rows of 128 or 256 cells (ny a multiple of 8, nz even) run the
# row-resident FP32 sweep: (256, 16, 8) and (128, 8, 4) are both levels of the
# first grid; (128, 8, 4) is a single 8-row tile whose halo rows wrap onto it,
# with four planes in z.
ROWS_CASES = [((256, 16, 8), 0.0), ((128, 8, 4), 0.0), ((256, 24, 16), 0.3), ((128, 40, 16), 0.0)]


def _levels(dims):
    out = [tuple(dims)]
    while all(v % 2 == 0 and v >= 4 for v in out[-1]):
        out.append(tuple(v // 2 for v in out[-1]))
    return out


@pytest.mark.parametrize("dims,alpha", ROWS_CASES)
@pytest.mark.parametrize("zc", [0, 2, 3, 5, 64])
def test_vcycle_f32_row_kernel(ibrd, dims, alpha, zc):
    """The row-resident FP32 sweep (one warp per x-row, plane ring fed by TMA
    tensor-map boxes, bounded mbarrier waits) inside the FP32 V-cycle gives the
    oracle's V-cycle within FP32 rounding, for the built-in z-march depth and
    depths with ragged last chunks, down to two planes per CTA; singular
    (alpha = 0: the kernel's per-CTA sums feed the mean projection) and
    shifted."""
    import torch
    nx, ny, nz = dims
    rng = np.random.default_rng(31 + zc)
    b = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    g = ibrd.Grid(*dims, alpha=alpha)
    if zc:
        for (lx, ly, lz) in _levels(dims):
            if lx in (128, 256) and ly % 8 == 0 and lz % 2 == 0 and lz >= 4:
                ibrd.ibrd_tune_set(g.handle, 4, 0, lx, ly, lz, lx, zc)
    x = g.vcycle_f32(torch.from_numpy(b).cuda()).cpu().numpy().astype(np.float64)
    want = mg.vcycle(b.astype(np.float64), 1.0, 1.0, alpha, exact_cells=32768, exact_side=64)
    assert rel_max(x, want) < 2e-5


@pytest.mark.parametrize("dims,alpha", ROWS_CASES + [((256, 64, 32), 0.0)])
@pytest.mark.parametrize("nu1,nu2,zero", [(1, 1, True), (1, 2, True), (2, 1, True), (1, 1, False)])
def test_vcycle_f32_sweep_counts(ibrd, dims, alpha, nu1, nu2, zero):
    """The FP32 V-cycle with the sweep counts of the solves' preconditioners:
    with one pre-smoothing sweep from zero on levels with 128- or 256-cell rows
    that sweep and the residual restriction run as one row-resident kernel
    (one pass over b, writing x and the coarse right-hand side); against the
    oracle's V-cycle with the same counts, from zero and from a guess."""
    import torch
    nx, ny, nz = dims
    rng = np.random.default_rng(61 + nu1 + 2 * nu2)
    b = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    x0 = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    g = ibrd.Grid(*dims, alpha=alpha)
    x = torch.from_numpy(x0).cuda()
    g.vcycle_f32(torch.from_numpy(b).cuda(), x, zero_initial_guess=zero, nu1=nu1, nu2=nu2)
    want = mg.vcycle(b.astype(np.float64), 1.0, 1.0, alpha, x0=None if zero else x0.astype(np.float64), nu1=nu1,
                     nu2=nu2, exact_cells=32768, exact_side=64)
    assert rel_max(x.cpu().numpy().astype(np.float64), want) < 2e-5


def _rows_levels(dims):
    return [lv for lv in _levels(dims) if lv[0] in (128, 256) and lv[1] % 8 == 0 and lv[2] % 2 == 0 and lv[2] >= 4]


@pytest.mark.parametrize("dims,alpha", ROWS_CASES + [((256, 64, 32), 0.0)])
@pytest.mark.parametrize("nu2,zero", [(1, True), (2, True), (1, False)])
@pytest.mark.parametrize("zc", [0, 2, 6])
def test_prolongation_fused_into_row_sweep(ibrd, dims, alpha, nu2, zero, zc):
    """On levels the row-resident sweep serves, the V-cycle adds the coarse-grid
    correction (the trilinear prolongation of the coarse solution, Sec. III.E)
    inside the first post-smoothing sweep, whose x reads then see x + P x_c,
    instead of writing the corrected field with a separate kernel first. The
    result equals, bit for bit, the V-cycle with the fusion switched off level
    by level (same sweep kernel and CTAs, so the same per-CTA sums feed the mean
    projection when alpha = 0), for one and two post-sweeps, from zero and from
    a guess, at the built-in z-march depth and at depths with ragged last chunks
    (nz = 8, 16, 32 with 6 planes per CTA); and it is the oracle's V-cycle
    within FP32 rounding."""
    import torch
    nx, ny, nz = dims
    rng = np.random.default_rng(71 + nu2 + 3 * zc)
    b = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    x0 = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    out = []
    for fused in (True, False):
        g = ibrd.Grid(*dims, alpha=alpha)
        for (lx, ly, lz) in _rows_levels(dims):
            if zc:
                ibrd.ibrd_tune_set(g.handle, 4, 0, lx, ly, lz, lx, zc)
            if not fused:
                ibrd.ibrd_tune_set(g.handle, 4, 2, lx, ly, lz, 1, 0)
        x = torch.from_numpy(x0).cuda()
        g.vcycle_f32(torch.from_numpy(b).cuda(), x, zero_initial_guess=zero, nu1=1, nu2=nu2)
        out.append(x.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    want = mg.vcycle(b.astype(np.float64), 1.0, 1.0, alpha, x0=None if zero else x0.astype(np.float64), nu1=1,
                     nu2=nu2, exact_cells=32768, exact_side=64)
    assert rel_max(out[0].astype(np.float64), want) < 2e-5


def test_prolongation_switch_arguments(ibrd):
    """The fusion switch is an FP32-only, hand-set entry: tx 0 or 1, zc 0."""
    g = ibrd.Grid(128, 16, 8)
    ibrd.ibrd_tune_set(g.handle, 4, 2, 128, 16, 8, 1, 0)
    ibrd.ibrd_tune_set(g.handle, 4, 2, 128, 16, 8, 0, 0)
    for bad in [(8, 2, 128, 16, 8, 1, 0), (4, 2, 128, 16, 8, 2, 0), (4, 2, 128, 16, 8, 1, 3),
                (4, 3, 128, 16, 8, 0, 0)]:
        with pytest.raises(ibrd.IbrdError):
            ibrd.ibrd_tune_set(g.handle, *bad)


def test_bounded_wait_gives_up_with_timeout_status(ibrd):
    """A bound of zero polls makes every plane wait of the row sweep give up:
    each CTA drains its copies in flight and stops, and the FP32 V-cycle and a
    solve in the refinement mode report IBRD_ERR_TIMEOUT instead of hanging or
    returning a wrong answer as a success. With the bound restored the same
    handle solves to the oracle's solution."""
    import torch
    from oracle import direct
    from synthetic import rsa_positions
    dims = (128, 16, 8)
    q = rsa_positions(4, dims, 1.0, 4.0, 41)
    gsrc = np.ones((8, 16, 128))
    g = ibrd.Grid(*dims)
    g.set_blobs(dev(q))
    b = torch.from_numpy(np.random.default_rng(42).standard_normal((8, 16, 128)).astype(np.float32)).cuda()
    ibrd.ibrd_set_wait_limit(g.handle, 0)
    with pytest.raises(ibrd.IbrdError) as e:
        g.vcycle_f32(b)
    assert e.value.status == 7
    with pytest.raises(ibrd.IbrdError) as e:
        g.solve_saddle(dev(gsrc), tol=1e-10, precision=ibrd.IBRD_MIXED_REFINE, max_iter=50)
    assert e.value.status == 7
    ibrd.ibrd_set_wait_limit(g.handle, 1 << 24)
    c, lam, info = g.solve_saddle(dev(gsrc), tol=1e-10, precision=ibrd.IBRD_MIXED_REFINE, max_iter=400)
    c_ref, lam_ref, _ = direct.solve_saddle(q, gsrc, 1.0, 1.0, 0.0)
    assert rel_max(host(c), c_ref) < 1e-8 and rel_max(host(lam), lam_ref) < 1e-8
    torch.cuda.synchronize()
