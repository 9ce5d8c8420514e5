"""The benchmark configurations beyond the timed one, as parity cases.

* Mixed precision at 64^3 (the 512^3 placement rule scaled to 64 blobs,
  spacing 3h): the FP64 GPU path and both mixed-precision modes against the
  oracle's exact saddle solution.
* Mixed precision at 512^3 with 32768 blobs (spacing 3h), diffusion-limited,
  solved to 1e-10: the two mixed-precision modes against the FP64 GPU path in
  c, lambda and the mean rate K (the bar for mixed precision is 1e-8).
"""
import numpy as np
import pytest

from oracle import direct, outputs
from synthetic import workload
from tests.gpu_util import dev, floor_tol, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibrd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1306_3159_gb300 import build
    build.build()
    import paper_1306_3159_gb300 as p
    return p


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_mixed64_against_oracle(ibrd, precision):
    w = workload("mixed64")
    c_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0)
    g = ibrd.Grid(*w.dims, h=w.h, chi=w.chi)
    g.set_blobs(dev(w.q))
    tol = floor_tol(c_ref, w.g, w.h, w.chi, 0.0)
    c, lam, info = g.solve_saddle(dev(w.g), tol=tol, precision=precision, max_iter=2000)
    assert info["status"] == 0 and info["rel_residual"] <= tol
    assert rel_err(host(c), c_ref) < 1e-11
    assert rel_err(host(lam), lam_ref) < 1e-11
    K_ref = outputs.overall_rate(lam_ref, c_ref)
    assert abs(info["rate_K"] - K_ref) < 1e-11 * abs(K_ref)


@pytest.mark.parametrize("precision", [0, 2])
def test_mixed64_with_forced_launch_shapes(ibrd, precision):
    """The same solve with non-default sweep launch shapes on every smoothed
    level (tile width 32, z-march depth 3 with a ragged last chunk; the
    stencil pass of the sweep from zero with depth 5): the solution is the
    oracle's, as with the built-in shapes."""
    w = workload("mixed64")
    c_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0)
    g = ibrd.Grid(*w.dims, h=w.h, chi=w.chi)
    g.set_blobs(dev(w.q))
    for side in (64, 32, 16):
        for elem in (4, 8):
            ibrd.ibrd_tune_set(g.handle, elem, 0, side, side, side, 32, 3)
        ibrd.ibrd_tune_set(g.handle, 4, 1, side, side, side, 0, 5)
    tol = floor_tol(c_ref, w.g, w.h, w.chi, 0.0)
    c, lam, info = g.solve_saddle(dev(w.g), tol=tol, precision=precision, max_iter=2000)
    assert info["status"] == 0 and info["rel_residual"] <= tol
    assert rel_err(host(c), c_ref) < 1e-11 and rel_err(host(lam), lam_ref) < 1e-11


def test_mixed512_modes_against_fp64(ibrd):
    w = workload("mixed")
    g = ibrd.Grid(*w.dims, h=w.h, chi=w.chi)
    g.set_blobs(dev(w.q))
    src = dev(w.g)
    c64, lam64, i64 = g.solve_saddle(src, tol=1e-10, precision=0, max_iter=3000)
    assert i64["status"] == 0
    c64h, lam64h, K64 = host(c64), host(lam64), i64["rate_K"]
    del c64, lam64
    for precision in (1, 2):
        c, lam, info = g.solve_saddle(src, tol=1e-10, precision=precision, max_iter=3000)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-10
        err_c = rel_err(host(c), c64h)
        err_l = rel_err(host(lam), lam64h)
        err_k = abs(info["rate_K"] - K64) / abs(K64)
        print(f"512^3, 32768 blobs, precision {precision}: error vs FP64 GPU c {err_c:.2e} lambda {err_l:.2e} "
              f"K {err_k:.2e} ({info['outer_iters']} iterations, {info['refinements']} refinements)")
        assert err_c < 1e-8 and err_l < 1e-8 and err_k < 1e-8
