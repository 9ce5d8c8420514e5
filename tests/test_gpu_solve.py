"""Solve-level parity of the CUDA path with the FP64 oracle's exact solutions.

The FP64 GPU path solves to a relative true residual of 1e-12. That is near
the rounding floor of FP64 here: in the steady periodic case c carries a large
constant cbar (about 1e3 for a unit source at 32^3), and A c is formed from
values of that size, so its rounding is about 6 eps cbar per cell, i.e. a
relative residual of a few 1e-13. The error in c and lambda is bounded by the
condition number on mean-zero fields (about 30 at 32^3) times the residual
relative to ||c||, far below the 1e-11 relative error the tests require. The mixed FP32
path solves to 1e-10 and must be within 1e-8 of the exact solution.
"""
import math

import numpy as np
import pytest

from oracle import direct, operators as op, outputs
from synthetic import workload, loguniform_rates, lattice_positions, rsa_positions
from tests.gpu_util import dev, host, rel_err, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibrd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1306_3159_gb300 import build
    build.build()
    import paper_1306_3159_gb300 as p
    return p


@pytest.fixture(scope="module")
def small():
    w = workload("small")
    M = direct.schur_matrix(w.q, w.dims, w.h, w.chi, 0.0)
    return w, M


EPS = 2.220446049250313e-16


def floor_tol(c_ref, g, h, chi, alpha, base=1e-12):
    """Relative-residual tolerance at the FP64 rounding floor: A c is formed
    from values of size max|c|, so each cell of the residual carries about
    eps (alpha + 12 chi/h^2) max|c| of rounding; relative to the rms of g that
    is the floor. A few times it, and never below `base`."""
    rms = float(np.sqrt(np.mean(np.asarray(g) ** 2)))
    fl = 4.0 * EPS * (alpha + 12.0 * chi / h ** 2) * float(np.abs(c_ref).max()) / rms
    return max(base, fl)


def _grid(ibrd, w, alpha=0.0, kernel=4):
    g = ibrd.Grid(*w.dims, h=w.h, chi=w.chi, alpha=alpha, kernel=kernel)
    g.set_blobs(dev(w.q))
    return g


# Precision 1 (FP64 FGMRES, FP32 preconditioner) and 2 (FP64 refinement
# around FP32 FGMRES) both stop on the FP64 true residual, so both reach the
# FP64 tolerances too.
SOLVE_CASES = [(0, 1e-12, 1e-11), (1, 1e-10, 1e-8), (1, 1e-12, 1e-11), (2, 1e-10, 1e-8), (2, 1e-12, 1e-11)]


@pytest.mark.parametrize("precision,tol,err", SOLVE_CASES)
@pytest.mark.parametrize("precond", [0, 2])
def test_saddle_small(ibrd, small, precision, tol, err, precond):
    """precond 0: the approximate Schur preconditioner; 2: the library's
    default choice by blob count (48 blobs: the diagonal one)."""
    w, M = small
    c_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0, M=M)
    g = _grid(ibrd, w)
    tol = max(tol, floor_tol(c_ref, w.g, w.h, w.chi, 0.0))
    c, lam, info = g.solve_saddle(dev(w.g), tol=tol, precision=precision, max_iter=400, precond=precond)
    assert info["precond"] == (0 if precond == 0 else 1)
    assert info["rel_residual"] <= tol
    assert (info["refinements"] >= 1) == (precision == 2)
    assert rel_err(host(c), c_ref) < err
    assert rel_err(host(lam), lam_ref) < err
    # Appendix A solvability: sum lambda = h^3 sum g / zeta
    assert abs(info["sum_lambda"] - w.g.sum()) < 1e-9 * w.g.sum()
    K_ref = outputs.overall_rate(lam_ref, c_ref)
    assert abs(info["rate_K"] - K_ref) < err * abs(K_ref)
    a_ref = outputs.reaction_radius(lam_ref, c_ref, w.chi)
    assert abs(info["a_L"] - a_ref) < err * abs(a_ref)


@pytest.mark.parametrize("precision,tol,err", SOLVE_CASES)
@pytest.mark.parametrize("alpha", [0.0, 0.2])
def test_reaction_small(ibrd, small, precision, tol, err, alpha):
    w, M0 = small
    M = M0 if alpha == 0.0 else None
    c_ref, u_ref, _ = direct.solve_reaction(w.q, w.kappa, w.g, w.h, w.chi, alpha, M=M)
    g = _grid(ibrd, w, alpha)
    tol = max(tol, floor_tol(c_ref, w.g, w.h, w.chi, alpha))
    c, info = g.solve_reaction(dev(w.kappa), dev(w.g), tol=tol, precision=precision, max_iter=400)
    assert info["rel_residual"] <= tol
    assert rel_err(host(c), c_ref) < err
    assert abs(info["sum_lambda"] - u_ref.sum()) < err * abs(u_ref.sum())


@pytest.mark.parametrize("precision", [0, 2])
def test_single_pass_gram_schmidt(ibrd, small, precision):
    """Classical Gram-Schmidt without the second pass (reorth_eta = 0): each
    new basis vector is scaled inside the pass that subtracts its projections
    and its exact norm recorded as the stored vector's scale; up to 7 basis
    vectors the reductions, that bookkeeping and the Givens step run in the
    last CTA of the two Gram-Schmidt launches, from the eighth on in separate
    kernels. The FP64 solves to 1e-12 run one long restart cycle and so take
    both; both modes reach the oracle's solutions at 1e-11."""
    w, M = small
    c_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0, M=M)
    g = _grid(ibrd, w)
    tol = max(1e-12, floor_tol(c_ref, w.g, w.h, w.chi, 0.0))
    c, lam, info = g.solve_saddle(dev(w.g), tol=tol, precision=precision, max_iter=400, reorth_eta=0.0,
                                  precond=0)
    assert info["rel_residual"] <= tol and info["reorths"] == 0
    assert rel_err(host(c), c_ref) < 1e-11 and rel_err(host(lam), lam_ref) < 1e-11
    cr_ref, u_ref, _ = direct.solve_reaction(w.q, w.kappa, w.g, w.h, w.chi, 0.0, M=M)
    tol = max(1e-12, floor_tol(cr_ref, w.g, w.h, w.chi, 0.0))
    cr, info = g.solve_reaction(dev(w.kappa), dev(w.g), tol=tol, precision=precision, max_iter=400,
                                reorth_eta=0.0, nu1=1, nu2=1)
    assert info["rel_residual"] <= tol and info["reorths"] == 0
    assert rel_err(host(cr), cr_ref) < 1e-11
    if precision == 0:
        assert info["outer_iters"] >= 9, info["outer_iters"]


def test_saddle_alpha_positive_nonunit_scales(ibrd):
    """alpha > 0, h != 1, chi != 1, zeta != 1 and a nonzero f."""
    dims, h, chi, alpha, zeta = (24, 16, 20), 0.5, 1.7, 0.8, 0.3
    q = rsa_positions(12, dims, h, 3.0 * h, 12)
    rng = np.random.default_rng(13)
    gsrc = rng.standard_normal((20, 16, 24))
    f = 0.1 * rng.standard_normal(12)
    c_ref, lam_ref, _ = direct.solve_saddle(q, gsrc, h, chi, alpha, zeta=zeta, f=f)
    g = ibrd.Grid(*dims, h=h, chi=chi, alpha=alpha)
    g.set_blobs(dev(q))
    # alpha > 0: no large constant mode, so the solve can go below 1e-12
    c, lam, info = g.solve_saddle(dev(gsrc), f=dev(f), tol=1e-14, zeta=zeta, max_iter=400)
    assert rel_err(host(c), c_ref) < 1e-11
    assert rel_err(host(lam), lam_ref) < 1e-11


def test_saddle_tiny_single_blob(ibrd):
    """32^3, one blob at a sub-cell offset from the box centre, tol 1e-10."""
    w = workload("tiny")
    c_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0)
    g = _grid(ibrd, w)
    c, lam, info = g.solve_saddle(dev(w.g), tol=floor_tol(c_ref, w.g, 1.0, 1.0, 0.0), max_iter=400)
    assert rel_err(host(c), c_ref) < 1e-11
    assert abs(host(lam)[0] - lam_ref[0]) < 1e-11 * abs(lam_ref[0])


def test_saddle_diagonal_preconditioner(ibrd, small):
    w, M = small
    c_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0, M=M)
    g = _grid(ibrd, w)
    tol = floor_tol(c_ref, w.g, w.h, w.chi, 0.0)
    c, lam, info = g.solve_saddle(dev(w.g), tol=tol, precond=1, restart=60, max_iter=2000)
    assert rel_err(host(lam), lam_ref) < 1e-11


def test_auto_preconditioner_choice_and_kept_gamma(ibrd):
    """IBRD_PRECOND_AUTO (the default) picks the diagonal preconditioner up to
    512 blobs in the mixed modes and up to 2048 in FP64, above them the
    approximate Schur one with the block-preconditioned inner GMRES (the plain
    inner GMRES when alpha > 0); the diagonal preconditioner's gamma, computed
    once per handle, is kept when the blobs change and the solve still reaches
    the oracle's solution for the new configuration."""
    dims = (32, 32, 32)
    g = ibrd.Grid(*dims)
    src = np.ones((32, 32, 32))
    q1 = rsa_positions(20, dims, 1.0, 3.0, 71)
    q2 = rsa_positions(30, dims, 1.0, 3.0, 72)
    for q in (q1, q2):
        g.set_blobs(dev(q))
        c_ref, lam_ref, _ = direct.solve_saddle(q, src, 1.0, 1.0, 0.0)
        tol = floor_tol(c_ref, src, 1.0, 1.0, 0.0)
        c, lam, info = g.solve_saddle(dev(src), tol=tol, max_iter=600, precision=2)
        assert info["precond"] == 1
        assert rel_err(host(c), c_ref) < 1e-11 and rel_err(host(lam), lam_ref) < 1e-11
    big = ibrd.Grid(64, 64, 64)
    q3 = rsa_positions(600, (64, 64, 64), 1.0, 3.0, 73)
    big.set_blobs(dev(q3))
    src3 = dev(np.ones((64, 64, 64)))
    assert big.solve_saddle(src3, tol=1e-8, precision=2, max_iter=600)[2]["precond"] == 3
    assert big.solve_saddle(src3, tol=1e-8, precision=0, max_iter=600)[2]["precond"] == 1
    shifted = ibrd.Grid(64, 64, 64, alpha=0.1)
    shifted.set_blobs(dev(q3))
    assert shifted.solve_saddle(src3, tol=1e-8, precision=2, max_iter=600)[2]["precond"] == 0


@pytest.mark.parametrize("precision,tol,err", [(0, 1e-12, 1e-11), (2, 1e-10, 1e-8), (2, 1e-12, 1e-11)])
def test_saddle_block_preconditioner(ibrd, small, precision, tol, err):
    """IBRD_PRECOND_BLOCK: the approximate Schur preconditioner (Appendix A)
    whose inner GMRES runs on P M~ with P the sparse approximate inverse of
    M = J A^-1 S from the periodic Green's function of the box (and gamma on
    the diagonal). The saddle solve of the 48-blob workload reaches the
    oracle's direct solution (FP64 and refinement modes), reports the
    preconditioner that ran, and with one inner iteration takes fewer outer
    iterations than the plain inner GMRES."""
    w, M = small
    c_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0, M=M)
    g = _grid(ibrd, w)
    tol = max(tol, floor_tol(c_ref, w.g, w.h, w.chi, 0.0))
    outer = {}
    for pc in (0, 3):
        c, lam, info = g.solve_saddle(dev(w.g), tol=tol, precision=precision, max_iter=400, precond=pc,
                                      schur_inner=1)
        assert info["precond"] == pc and info["rel_residual"] <= tol
        assert rel_err(host(c), c_ref) < err and rel_err(host(lam), lam_ref) < err
        assert abs(info["sum_lambda"] - w.g.sum()) < 1e-9 * w.g.sum()
        outer[pc] = info["outer_iters"]
    assert outer[3] < outer[0], outer


def test_block_preconditioner_follows_the_blobs(ibrd):
    """The block preconditioner is rebuilt when the blobs move: a handle that
    solved one configuration with it and then another gives, bit for bit,
    the solve of a handle that saw only the second one with the same gamma
    (gamma is kept per handle, so the second handle takes it from the first
    configuration through a diagonal-preconditioned solve). An explicit
    block_cutoff solves too, to the oracle's solution, and a non-finite one
    is rejected."""
    dims = (64, 64, 32)
    src = np.ones((32, 64, 64))
    q1 = rsa_positions(300, dims, 1.0, 3.0, 81)
    q2 = rsa_positions(300, dims, 1.0, 3.0, 82)
    kw = dict(tol=1e-9, precision=2, max_iter=600, schur_inner=2)
    a = ibrd.Grid(*dims)
    a.set_blobs(dev(q1))
    a.solve_saddle(dev(src), precond=3, **kw)
    a.set_blobs(dev(q2))
    ca, la, ia = a.solve_saddle(dev(src), precond=3, **kw)
    b = ibrd.Grid(*dims)
    b.set_blobs(dev(q1))
    b.solve_saddle(dev(src), precond=1, **kw)
    b.set_blobs(dev(q2))
    cb, lb, ib = b.solve_saddle(dev(src), precond=3, **kw)
    assert ia["outer_iters"] == ib["outer_iters"]
    assert np.array_equal(host(ca), host(cb)) and np.array_equal(host(la), host(lb))
    c_ref, lam_ref, _ = direct.solve_saddle(q2, src, 1.0, 1.0, 0.0)
    c, lam, info = a.solve_saddle(dev(src), precond=3, block_cutoff=9.0, **kw)
    assert info["precond"] == 3
    assert rel_err(host(c), c_ref) < 1e-7 and rel_err(host(lam), lam_ref) < 1e-7
    with pytest.raises(ibrd.IbrdError):
        a.solve_saddle(dev(src), precond=3, block_cutoff=float("nan"), **kw)


def test_single_blob_finite_rate_shift(ibrd):
    """Sec. III.D: c_P - c_0 = 1/kappa, a constant field (one periodic blob)."""
    L = 16
    q = np.array([[7.3, 8.6, 8.1]])
    gsrc = np.full((L, L, L), 1.0 / L ** 3)
    g = ibrd.Grid(L, L, L)
    g.set_blobs(dev(q))
    c0, lam, _ = g.solve_saddle(dev(gsrc), tol=floor_tol(np.full(1, 0.2), gsrc, 1.0, 1.0, 0.0), max_iter=400)
    for kappa in (0.5, 7.0):
        tol = floor_tol(np.full(1, 0.2 + 1.0 / kappa), gsrc, 1.0, 1.0, 0.0)
        cP, _ = g.solve_reaction(dev(np.array([kappa])), dev(gsrc), tol=tol, max_iter=400)
        d = host(cP) - host(c0)
        assert np.abs(d - 1.0 / kappa).max() < 1e-9


def test_guess_and_not_converged(ibrd, small):
    w, _ = small
    g = _grid(ibrd, w)
    import paper_1306_3159_gb300 as p
    c = g.field()
    lam = dev(np.zeros(len(w.q)))
    info = p.ibrd_solve_saddle(g.handle, dev(w.g), None, c, lam, p.ibrd_default_opts(tol=1e-14, max_iter=2),
                               raise_on_error=False)
    assert info["status"] == 4 and info["outer_iters"] == 2
    # restart from the returned iterate
    info2 = p.ibrd_solve_saddle(g.handle, dev(w.g), None, c, lam,
                                p.ibrd_default_opts(tol=1e-9, max_iter=400, use_guess=1))
    assert info2["status"] == 0 and info2["rel_residual"] <= 1e-9


def test_nonfinite_source_reported(ibrd, small):
    w, _ = small
    g = _grid(ibrd, w)
    bad = w.g.copy()
    bad[1, 2, 3] = np.nan
    import paper_1306_3159_gb300 as p
    info = p.ibrd_solve_reaction(g.handle, dev(w.kappa), dev(bad), g.field(), p.ibrd_default_opts(),
                                 raise_on_error=False)
    assert info["status"] == 6
    with pytest.raises(p.IbrdError) as e:
        g.solve_reaction(dev(-w.kappa), dev(w.g))
    assert e.value.status == 6


def _residual_oracle(q, kappa, gsrc, c, lam, h, chi, alpha, zeta=1.0):
    """Relative true residual of a GPU solution, computed with the oracle's
    operator definitions (a property that holds at any size)."""
    dims = gsrc.shape[::-1]
    if lam is None:
        r = gsrc - (op.apply_A(c, h, chi, alpha) + op.spread(kappa * op.interp(c, q, h), q, dims, h))
        return np.linalg.norm(r) / np.linalg.norm(gsrc)
    r1 = gsrc - (op.apply_A(c, h, chi, alpha) + zeta * op.spread(lam, q, dims, h))
    r2 = -(zeta / h ** 3) * op.interp(c, q, h)
    return math.sqrt(np.sum(r1 ** 2) + np.sum(r2 ** 2)) / np.linalg.norm(gsrc)


def test_full_size_properties(ibrd):
    """256^3 with 4096 RSA blobs (spacing 4h), as timed by the benchmark: the
    oracle recomputes the true residual of both solves, and the Appendix A
    balance sum(lambda) = h^3 sum(g) holds."""
    w = workload("scale")
    g = _grid(ibrd, w)
    for precision in (1, 2):
        c, lam, info = g.solve_saddle(dev(w.g), tol=1e-8, precision=precision, max_iter=2000)
        ch, lh = host(c), host(lam)
        assert _residual_oracle(w.q, None, w.g, ch, lh, 1.0, 1.0, 0.0) < 2e-8
        assert abs(lh.sum() - w.g.sum()) < 1e-6 * w.g.sum()
        c2, info2 = g.solve_reaction(dev(w.kappa), dev(w.g), tol=1e-8, precision=precision, max_iter=2000)
        assert _residual_oracle(w.q, w.kappa, w.g, host(c2), None, 1.0, 1.0, 0.0) < 2e-8


def test_graph_replay_matches_direct_launches(ibrd, small):
    """Preconditioner applications replayed from captured CUDA graphs give
    the same iterates, bit for bit, as direct launches (every kernel is
    deterministic), for both solves and all three precision modes."""
    import torch
    w, _ = small
    g = _grid(ibrd, w)
    for precision in (0, 1, 2):
        outs = []
        for graphs in (0, 1, 1, 1):  # direct, first encounter, capture, replay
            c, lam, info = g.solve_saddle(dev(w.g), tol=1e-9, precision=precision, graphs=graphs)
            c2, info2 = g.solve_reaction(dev(w.kappa), dev(w.g), tol=1e-9, precision=precision, graphs=graphs)
            outs.append((host(c), host(lam), host(c2), info["outer_iters"], info["vcycles"], info2["vcycles"]))
        for o in outs[1:]:
            assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])
            assert np.array_equal(o[2], outs[0][2])
            assert o[3:] == outs[0][3:]
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", [0, 2])
def test_batch_matches_single_solves(ibrd, precision):
    """Batched solves of uneven realisations (grid sides 32-64, 4-200 blobs),
    each handle on its own stream and run concurrently from the library's host
    threads, give bit for bit the iterates of the same solves run one at a
    time; the smallest reaction problem also matches the oracle's exact
    solution."""
    import torch
    from synthetic import batch_workloads
    ws = batch_workloads(6, sides=(32, 40, 48, 64), n_lo=4, n_hi=200, seed=12)
    streams = [torch.cuda.Stream() for _ in ws]
    grids = [ibrd.Grid(*w.dims, h=w.h, chi=w.chi, stream=s.cuda_stream) for w, s in zip(ws, streams)]
    qs, ks, gs = [dev(w.q) for w in ws], [dev(w.kappa) for w in ws], [dev(w.g) for w in ws]
    cb = [torch.zeros_like(x) for x in gs]
    cs = [torch.zeros_like(x) for x in gs]
    lb = [torch.zeros(len(w.q), dtype=torch.float64, device="cuda") for w in ws]
    c1s, c2s, l2s = [torch.zeros_like(x) for x in gs], [torch.zeros_like(x) for x in gs], [torch.zeros_like(x) for x in lb]
    torch.cuda.synchronize()  # the handles' streams do not wait for torch's
    for g, q in zip(grids, qs):
        g.set_blobs(q)
    opts = ibrd.ibrd_default_opts(tol=1e-10, precision=precision, max_iter=400)
    hs = [g.handle for g in grids]
    rb = ibrd.ibrd_solve_reaction_batch(hs, ks, gs, cb, opts, threads=4)
    sb = ibrd.ibrd_solve_saddle_batch(hs, gs, None, cs, lb, opts, threads=3)
    for i, g in enumerate(grids):
        c1, c2, l2 = c1s[i], c2s[i], l2s[i]
        r1 = ibrd.ibrd_solve_reaction(g.handle, ks[i], gs[i], c1, opts)
        s1 = ibrd.ibrd_solve_saddle(g.handle, gs[i], None, c2, l2, opts)
        assert torch.equal(c1, cb[i]) and torch.equal(c2, cs[i]) and torch.equal(l2, lb[i])
        for a, b in ((r1, rb[i]), (s1, sb[i])):
            assert a["status"] == b["status"] == 0
            assert (a["outer_iters"], a["vcycles"], a["rel_residual"]) == (b["outer_iters"], b["vcycles"],
                                                                            b["rel_residual"])
    k = min(range(len(ws)), key=lambda i: ws[i].dims[0] ** 3 + len(ws[i].q))
    w = ws[k]
    c_ref, _, _ = direct.solve_reaction(w.q, w.kappa, w.g, w.h, w.chi, 0.0)
    assert rel_err(host(cb[k]), c_ref) < 1e-8
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", [0, 2])
def test_saddle_warm_start(ibrd, small, precision):
    """Saddle solves started from a guess of lambda (uniform share, the exact
    multipliers with 1 % noise, and an all-zero guess, which falls back to the
    uniform share) and the grid field built from it by Appendix A steps 3-5,
    or from the penalty form (a reaction-limited solve with a large rate),
    reach the tolerance and the oracle's solution; the exact multipliers never
    cost more iterations than a zero start."""
    import torch
    w, M = small
    c_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0, M=M)
    g = _grid(ibrd, w)
    tol = max(1e-12, floor_tol(c_ref, w.g, w.h, w.chi, 0.0))
    err = 1e-11
    noise = np.random.default_rng(3).standard_normal(len(lam_ref))
    _, _, cold = g.solve_saddle(dev(w.g), tol=tol, precision=precision, max_iter=400)
    for guess, lam0 in [(1, None), (2, lam_ref * (1 + 0.01 * noise)), (2, np.zeros_like(lam_ref)), (2, lam_ref),
                        (3, None)]:
        lam = dev(lam0) if lam0 is not None else None
        c, lam, info = g.solve_saddle(dev(w.g), lam=lam, tol=tol, precision=precision, max_iter=400,
                                      lambda_guess=guess, warm_cycles=3)
        assert info["rel_residual"] <= tol
        assert rel_err(host(c), c_ref) < err and rel_err(host(lam), lam_ref) < err
        if lam0 is not None and np.array_equal(lam0, lam_ref):
            assert info["outer_iters"] <= cold["outer_iters"]
    torch.cuda.synchronize()


def test_batch_reports_each_problem(ibrd):
    """A failing problem does not stop the others: a NaN source gives
    IBRD_ERR_NONFINITE for its problem only, a handle without blobs gives
    IBRD_ERR_STATE for a saddle solve, and the batch returns the first failure
    in index order while the other problems are solved."""
    import torch
    from synthetic import batch_workloads
    ws = batch_workloads(3, sides=(32,), n_lo=8, n_hi=20, seed=21)
    streams = [torch.cuda.Stream() for _ in ws]
    grids = [ibrd.Grid(*w.dims, stream=s.cuda_stream) for w, s in zip(ws, streams)]
    gs = [dev(w.g) for w in ws]
    gs[1][0, 0, 0] = float("nan")
    ks = [dev(w.kappa) for w in ws]
    cs = [torch.zeros_like(x) for x in gs]
    ls = [torch.zeros(len(w.q), dtype=torch.float64, device="cuda") for w in ws]
    qs = [dev(w.q) for w in ws]
    torch.cuda.synchronize()
    for i in (0, 1):
        grids[i].set_blobs(qs[i])
    opts = ibrd.ibrd_default_opts(tol=1e-10)
    hs = [g.handle for g in grids]
    out = ibrd.ibrd_solve_reaction_batch(hs[:2], ks[:2], gs[:2], cs[:2], opts, threads=2, raise_on_error=False)
    assert [o["status"] for o in out] == [0, 6] and out[0]["rel_residual"] <= 1e-10
    with pytest.raises(ibrd.IbrdError) as e:
        ibrd.ibrd_solve_saddle_batch(hs, [gs[0], gs[2], gs[2]], None, cs, ls, opts, threads=3)
    assert e.value.status == 8  # problem 2 has no blobs; problems 0 and 1 are solved
    out = ibrd.ibrd_solve_saddle_batch(hs, [gs[0], gs[2], gs[2]], None, cs, ls, opts, threads=3,
                                       raise_on_error=False)
    assert [o["status"] for o in out] == [0, 0, 8]
    torch.cuda.synchronize()


def test_degenerate_inputs(ibrd):
    """No blobs: the reaction-limited solve with alpha > 0 is the Helmholtz
    solve (the oracle's FFT Green's function), with alpha = 0 it has no
    solution and is refused (IBRD_ERR_ARG), and a saddle solve needs blobs
    (IBRD_ERR_STATE). Two coincident blobs make J rank-deficient: the field
    c is still unique and matches the oracle's solution for the merged blob,
    and the two multipliers share the merged one's."""
    import torch
    dims = (24, 16, 20)
    rng = np.random.default_rng(31)
    gsrc = 1.0 + 0.3 * rng.standard_normal((20, 16, 24))
    g = ibrd.Grid(*dims, alpha=0.5)
    kappa = torch.zeros(0, dtype=torch.float64, device="cuda")
    c, info = g.solve_reaction(kappa, dev(gsrc), tol=1e-13, max_iter=200)
    assert rel_err(host(c), op.green_apply(gsrc, 1.0, 1.0, 0.5)) < 1e-11
    g0 = ibrd.Grid(*dims)
    with pytest.raises(ibrd.IbrdError) as e:
        g0.solve_reaction(kappa, dev(gsrc), tol=1e-10)
    assert e.value.status == 1
    with pytest.raises(ibrd.IbrdError) as e:
        g0.solve_saddle(dev(gsrc), tol=1e-10)
    assert e.value.status == 8
    # coincident blobs
    w = workload("small")
    q3 = w.q[:3]
    q4 = np.vstack([q3, q3[:1]])
    c_ref, lam_ref, _ = direct.solve_saddle(q3, w.g, w.h, w.chi, 0.0)
    gc = ibrd.Grid(*w.dims)
    gc.set_blobs(dev(q4))
    c, lam, info = _saddle_status(ibrd, gc, w.g, 1e-11)
    assert info["status"] == 0, info["status"]
    lam = host(lam)
    assert rel_err(host(c), c_ref) < 1e-9
    assert abs(lam[0] + lam[3] - lam_ref[0]) < 1e-9 * abs(lam_ref).max()
    assert np.abs(lam[1:3] - lam_ref[1:3]).max() < 1e-9 * abs(lam_ref).max()
    torch.cuda.synchronize()


def _saddle_status(ibrd, grid, gsrc, tol):
    import torch
    c = grid.field()
    lam = torch.zeros(grid.n_blobs, dtype=torch.float64, device="cuda")
    info = ibrd.ibrd_solve_saddle(grid.handle, dev(gsrc), None, c, lam, ibrd.ibrd_default_opts(tol=tol, max_iter=400),
                                  raise_on_error=False)
    return c, lam, info


def test_solve_many_mixed_kinds(ibrd, small):
    """The two solves of one configuration (reaction-limited and saddle point),
    each on its own handle and stream with its own options, run together by
    ibrd_solve_many (each item setting its blobs and downloading its solution
    to pinned host memory): bit for bit the results of the separate calls, and
    the oracle's solutions."""
    import torch
    w, M = small
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ga = ibrd.Grid(*w.dims, stream=sa.cuda_stream)
    gb = ibrd.Grid(*w.dims, stream=sb.cuda_stream)
    q, k, src = dev(w.q), dev(w.kappa), dev(w.g)
    c1, c2, c3, c4 = (torch.zeros_like(src) for _ in range(4))
    l2, l4 = torch.zeros(len(w.q), dtype=torch.float64, device="cuda"), \
        torch.zeros(len(w.q), dtype=torch.float64, device="cuda")
    h1 = torch.zeros(src.shape, dtype=torch.float64).pin_memory()
    h2 = torch.zeros(src.shape, dtype=torch.float64).pin_memory()
    hl = torch.zeros(len(w.q), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    ro = ibrd.ibrd_default_opts(tol=1e-10, precision=2, max_iter=400, mg_cycles=1, nu1=1, nu2=1)
    so = ibrd.ibrd_default_opts(tol=1e-10, precision=2, max_iter=400, schur_inner=3, lambda_guess=1)
    # the items set the blobs themselves and download their solutions
    out = ibrd.ibrd_solve_many([dict(kind="reaction", grid=ga.handle, kappa=k, rhs=src, c=c1, opts=ro, q=q,
                                     c_host=h1),
                                dict(kind="saddle", grid=gb.handle, rhs=src, c=c2, lam=l2, opts=so, q=q,
                                     c_host=h2, lam_host=hl)], threads=2)
    gb.n_blobs = ga.n_blobs = len(w.q)
    assert torch.equal(h1, c1.cpu()) and torch.equal(h2, c2.cpu()) and torch.equal(hl, l2.cpu())
    r = ibrd.ibrd_solve_reaction(ga.handle, k, src, c3, ro)
    s_ = ibrd.ibrd_solve_saddle(gb.handle, src, None, c4, l4, so)
    assert torch.equal(c1, c3) and torch.equal(c2, c4) and torch.equal(l2, l4)
    assert out[0]["outer_iters"] == r["outer_iters"] and out[1]["outer_iters"] == s_["outer_iters"]
    c_ref, u_ref, _ = direct.solve_reaction(w.q, w.kappa, w.g, w.h, w.chi, 0.0, M=M)
    cs_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0, M=M)
    assert rel_err(host(c1), c_ref) < 1e-8 and rel_err(host(c2), cs_ref) < 1e-8 and rel_err(host(l2), lam_ref) < 1e-8
    torch.cuda.synchronize()


RANDOM_SHAPES = [(16, 24, 32), (40, 24, 16), (48, 48, 16), (32, 64, 16), (24, 24, 24), (20, 40, 12)]


@pytest.mark.parametrize("seed", range(6))
def test_random_configurations(ibrd, seed):
    """Seeded random configurations: grid shape, spacing h, diffusion
    coefficient chi, blob count (RSA, spacing 3h), kernel width, shift alpha
    and precision mode drawn per case; both solves against the oracle's exact
    solutions within 1e-11 (element-wise and in L2)."""
    import torch
    rng = np.random.default_rng(1000 + seed)
    dims = RANDOM_SHAPES[seed]
    n = int(rng.integers(1, 40))
    w_k = int(rng.choice([3, 4]))
    alpha = float(rng.choice([0.0, 0.3]))
    precision = int(rng.integers(0, 3))
    h = float(rng.choice([0.5, 1.0, 2.0]))
    chi = float(rng.choice([0.7, 1.0, 1.3]))
    q = rsa_positions(n, dims, h, 3.0 * h, 2000 + seed)
    n = len(q)
    kappa = loguniform_rates(n, 0.1, 10.0, 3000 + seed)
    nx, ny, nz = dims
    gsrc = 1.0 + 0.5 * rng.random((nz, ny, nx))
    g = ibrd.Grid(*dims, h=h, chi=chi, alpha=alpha, kernel=w_k)
    g.set_blobs(dev(q))
    case = (dims, h, chi, n, w_k, alpha, precision)
    c_ref, lam_ref, _ = direct.solve_saddle(q, gsrc, h, chi, alpha, w=w_k)
    # alpha > 0 has no large constant mode: solve below 1e-12, so that the
    # residual bounds the 1e-11 error whatever the conditioning of the case
    base = 1e-12 if alpha == 0.0 else 1e-14
    tol = floor_tol(c_ref, gsrc, h, chi, alpha, base=base)
    c, lam, info = g.solve_saddle(dev(gsrc), tol=tol, precision=precision, max_iter=600)
    assert info["rel_residual"] <= tol, case
    # every precision mode forms its stopping residual in FP64 and is solved
    # here to the FP64 rounding floor, so all of them meet the FP64 bar
    assert rel_err(host(c), c_ref) < 1e-11 and rel_err(host(lam), lam_ref) < 1e-11, case
    cr_ref, u_ref, _ = direct.solve_reaction(q, kappa, gsrc, h, chi, alpha, w=w_k)
    tol = floor_tol(cr_ref, gsrc, h, chi, alpha, base=base)
    cr, info = g.solve_reaction(dev(kappa), dev(gsrc), tol=tol, precision=precision, max_iter=600)
    assert info["rel_residual"] <= tol, case
    assert rel_err(host(cr), cr_ref) < 1e-11, case
    torch.cuda.synchronize()


def test_backward_euler_steps(ibrd, small):
    """Eq. unsteady_system as time stepping: three backward-Euler steps
    (alpha = 1/dt, right-hand side c^n / dt + s) of the reaction-limited
    system from c = 0, each against the oracle's exact step."""
    import torch
    w, _ = small
    dt = 2.0
    alpha = 1.0 / dt
    g = _grid(ibrd, w, alpha)
    c_ref = np.zeros_like(w.g)
    c = torch.zeros_like(dev(w.g))
    for _ in range(3):
        rhs_ref = c_ref / dt + w.g
        c_ref, _, _ = direct.solve_reaction(w.q, w.kappa, rhs_ref, w.h, w.chi, alpha)
        rhs = c / dt + dev(w.g)
        c, info = g.solve_reaction(dev(w.kappa), rhs, tol=max(1e-12, floor_tol(c_ref, rhs_ref, w.h, w.chi, alpha)),
                                   max_iter=400)
        assert rel_err(host(c), c_ref) < 1e-11
    torch.cuda.synchronize()


def test_device_terminated_graph_solve(ibrd, small):
    """opts.graphs = 2: from the second solve of a configuration on, a
    refinement-mode solve is ONE CUDA graph launch whose refinement steps,
    restart cycles and Krylov iterations are conditional nodes decided on the
    device. It gives bit for bit the iterates, iteration counts, refinement
    counts, residual and history of the host-driven loop (graphs = 1), for the
    reaction solve from zero and the saddle solve from a uniform-share warm
    start, on a grid whose finest level runs the row-resident kernels; and the
    oracle's solutions."""
    import torch
    dims = (128, 32, 16)
    q = rsa_positions(12, dims, 1.0, 4.0, 91)
    kappa = loguniform_rates(len(q), 0.1, 10.0, 92)
    src = 1.0 + 0.2 * np.random.default_rng(93).standard_normal((16, 32, 128))
    g = ibrd.Grid(*dims)
    g.set_blobs(dev(q))
    common = dict(tol=1e-10, precision=2, max_iter=600, restart=10, nu1=1, nu2=1, inner_tol=1e-3)
    out = {}
    for graphs in (1, 2, 2, 2):  # host loop; first encounter (host); graph built and launched; replay
        c, info = g.solve_reaction(dev(kappa), dev(src), graphs=graphs, **common)
        c2, lam, info2 = g.solve_saddle(dev(src), graphs=graphs, lambda_guess=1, warm_cycles=1, schur_inner=3,
                                        **common)
        out.setdefault(graphs, []).append((host(c), info, host(c2), host(lam), info2))
    ref = out[1][0]
    for run in out[2]:
        assert np.array_equal(run[0], ref[0]) and np.array_equal(run[2], ref[2]) and np.array_equal(run[3], ref[3])
        for a, b in ((run[1], ref[1]), (run[4], ref[4])):
            assert a["status"] == b["status"] == 0
            for k in ("outer_iters", "refinements", "vcycles", "rel_residual"):
                assert a[k] == b[k], (k, a[k], b[k])
            assert np.array_equal(a["history"], b["history"])
    c_ref, _, _ = direct.solve_reaction(q, kappa, src, 1.0, 1.0, 0.0)
    assert rel_err(out[2][-1][0], c_ref) < 1e-8
    # limits and faults end the device loop with the host loop's statuses
    info = ibrd.ibrd_solve_reaction(g.handle, dev(kappa), dev(src), g.field(),
                                    ibrd.ibrd_default_opts(graphs=2, **dict(common, max_iter=3)),
                                    raise_on_error=False)
    info = ibrd.ibrd_solve_reaction(g.handle, dev(kappa), dev(src), g.field(),
                                    ibrd.ibrd_default_opts(graphs=2, **dict(common, max_iter=3)),
                                    raise_on_error=False)
    assert info["status"] == 4 and info["outer_iters"] == 3
    ibrd.ibrd_set_wait_limit(g.handle, 0)
    for _ in range(2):  # host loop, then the graph (rebuilt: the bound is baked into its kernels)
        info = ibrd.ibrd_solve_reaction(g.handle, dev(kappa), dev(src), g.field(),
                                        ibrd.ibrd_default_opts(graphs=2, **common), raise_on_error=False)
        assert info["status"] == 7
    ibrd.ibrd_set_wait_limit(g.handle, 1 << 24)
    torch.cuda.synchronize()


def test_batch_as_one_graph(ibrd):
    """Batched refinement-mode solves with opts.graphs = 2: the first call runs
    the problems' host loops, the second records every problem's whole
    device-terminated solve into ONE graph (one branch per problem) and
    launches it, the third replays it. Every call gives, bit for bit, the
    iterates and reports of the same solves run one at a time, for reaction
    solves of uneven realisations (grid sides 32-64, 4-200 blobs) and
    warm-started saddle solves."""
    import torch
    from synthetic import batch_workloads
    ws = batch_workloads(5, sides=(32, 40, 48, 64), n_lo=4, n_hi=200, seed=14)
    streams = [torch.cuda.Stream() for _ in ws]
    grids = [ibrd.Grid(*w.dims, h=w.h, chi=w.chi, stream=s.cuda_stream) for w, s in zip(ws, streams)]
    ks, gs = [dev(w.kappa) for w in ws], [dev(w.g) for w in ws]
    torch.cuda.synchronize()
    for g, w in zip(grids, ws):
        g.set_blobs(dev(w.q))
    hs = [g.handle for g in grids]
    ro = dict(tol=1e-10, precision=2, max_iter=600, nu1=1, nu2=1, inner_tol=1e-3)
    so = dict(ro, lambda_guess=1, warm_cycles=1, schur_inner=3)
    singles = []
    for i, g in enumerate(grids):
        c = torch.zeros_like(gs[i])
        r = ibrd.ibrd_solve_reaction(g.handle, ks[i], gs[i], c, ibrd.ibrd_default_opts(graphs=1, **ro))
        c2, lam = torch.zeros_like(gs[i]), torch.zeros(len(ws[i].q), dtype=torch.float64, device="cuda")
        s1 = ibrd.ibrd_solve_saddle(g.handle, gs[i], None, c2, lam, ibrd.ibrd_default_opts(graphs=1, **so))
        singles.append((c, r, c2, lam, s1))
    torch.cuda.synchronize()
    for call in range(3):
        cb = [torch.zeros_like(x) for x in gs]
        rb = ibrd.ibrd_solve_reaction_batch(hs, ks, gs, cb, ibrd.ibrd_default_opts(graphs=2, **ro), threads=3)
        cs = [torch.zeros_like(x) for x in gs]
        lb = [torch.zeros(len(w.q), dtype=torch.float64, device="cuda") for w in ws]
        sb = ibrd.ibrd_solve_saddle_batch(hs, gs, None, cs, lb, ibrd.ibrd_default_opts(graphs=2, **so), threads=3)
        torch.cuda.synchronize()
        for i in range(len(ws)):
            c, r, c2, lam, s1 = singles[i]
            assert torch.equal(cb[i], c) and torch.equal(cs[i], c2) and torch.equal(lb[i], lam), (call, i)
            for a, b in ((rb[i], r), (sb[i], s1)):
                assert a["status"] == b["status"] == 0
                for k in ("outer_iters", "refinements", "vcycles", "rel_residual"):
                    assert a[k] == b[k], (call, i, k, a[k], b[k])
    k = min(range(len(ws)), key=lambda i: ws[i].dims[0] ** 3 + len(ws[i].q))
    w = ws[k]
    c_ref, _, _ = direct.solve_reaction(w.q, w.kappa, w.g, w.h, w.chi, 0.0)
    assert rel_err(host(cb[k]), c_ref) < 1e-8
    torch.cuda.synchronize()
