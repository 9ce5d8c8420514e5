"""Physics checks of the CUDA path against numbers the paper prints
(Sec. IV.A and IV.B), at sizes the paper used."""
import math

import numpy as np
import pytest

from oracle import outputs
from synthetic import lattice_positions
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibrd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1306_3159_gb300 import build
    build.build()
    import paper_1306_3159_gb300 as p
    return p


def _radius(ibrd, L, q, w=4):
    g = ibrd.Grid(L, L, L, kernel=w)
    g.set_blobs(dev(np.asarray(q, dtype=np.float64)))
    src = np.full((L, L, L), 1.0 / L ** 3)
    # relative residual 1e-8: the source is 1/L^3, so the FP64 floor of the
    # relative residual is near 1e-9 here, and c-bar (hence a) is fixed to
    # far more digits than the percent-level checks below need
    c, lam, info = g.solve_saddle(dev(src), tol=1e-8, max_iter=500)
    aL = info["sum_lambda"] / (4 * math.pi * 1.0 * info["cbar"])
    return aL, outputs.radius_from_series(aL, L, 1.0)


def test_reaction_radius_at_node_L128(ibrd):
    """A blob at a grid node in a periodic 128^3 box: Eq. a_phi's series gives
    a = 1.27h (4-point) within 1.5%."""
    L = 128
    aL, a = _radius(ibrd, L, [[L / 2, L / 2, L / 2]])
    assert abs(a - 1.27) < 0.015 * 1.27
    assert aL > a


def test_translational_variation_L128(ibrd):
    """Sec. IV.A at L = 128: the 4-point radius varies by about 1.5% as the
    blob moves relative to the grid, the 3-point one by about 5%."""
    L = 128
    offsets = [(0, 0, 0), (0.5, 0, 0), (0.5, 0.5, 0), (0.5, 0.5, 0.5), (0.25, 0.25, 0.25)]
    var = {}
    for w in (4, 3):
        a = np.array([_radius(ibrd, L, [[L / 2 + 0.5 + d[0], L / 2 + 0.5 + d[1], L / 2 + 0.5 + d[2]]], w)[1]
                      for d in offsets])
        var[w] = (a.max() - a.min()) / a.mean()
        if w == 4:
            assert abs(a.mean() - 1.255) < 0.01 * 1.255
    assert var[4] < 0.03 and 0.02 < var[3] < 0.075 and var[4] < var[3]


def test_cubic_lattice_rate_L64(ibrd):
    """Sec. IV.B: 512 blobs on a cubic lattice of spacing 8h in 64^3 follow
    Eq. beta_cubic within 1%."""
    L, sp = 64, 8
    q = lattice_positions((L, L, L), 1.0, sp)
    g = ibrd.Grid(L, L, L)
    g.set_blobs(dev(q))
    V = L ** 3
    src = np.full((L, L, L), 1.0 / V)
    c, lam, info = g.solve_saddle(dev(src), tol=1e-8, max_iter=500)
    a = 1.27
    phi = len(q) * (4 * math.pi * a ** 3 / 3) / V
    b0 = outputs.beta0(info["cbar"], 1.0 / V, a, 1.0, len(q), V)
    fit = outputs.beta0_cubic_fit(phi)
    assert abs(b0 - fit) < 0.01 * fit
    # every blob of the lattice sees the same environment: equal rates
    lh = host(lam)
    assert np.abs(lh - lh.mean()).max() < 1e-6 * abs(lh.mean())


def test_reaction_radius_sweep_over_box_size(ibrd):
    """Sec. IV.A: a single blob at a node in periodic boxes of side L = 16,
    32, 64, 128. The measured a_L falls with L toward the isolated blob's
    radius (Eq. a_phi: a_L = a (1 + x + x^2 + ...), x = 2.84 a / L), and the
    series removes the box-size dependence: the corrected radii agree within
    1 % of each other and lie in 1.24h-1.30h."""
    rows = []
    for L in (16, 32, 64, 128):
        aL, a = _radius(ibrd, L, [[L / 2, L / 2, L / 2]])
        rows.append((L, aL, a))
    aLs = [r[1] for r in rows]
    corr = np.array([r[2] for r in rows])
    assert all(x > y for x, y in zip(aLs, aLs[1:])) and all(r[1] > r[2] for r in rows), rows
    assert np.all((corr > 1.24) & (corr < 1.30)), rows
    assert (corr.max() - corr.min()) / corr.mean() < 0.01, rows


# Cubic lattices of blobs at grid nodes (Sec. IV.B, Fig. PerDisp): (grid side,
# lattice spacing). A lattice of spacing s is the periodic tiling of one blob
# in an s^3 box, so each case is also checked against the oracle's direct
# solve of that single cell.
LATTICES = [(64, 4), (80, 5), (96, 6), (64, 8), (80, 10), (96, 12), (64, 16)]


@pytest.mark.parametrize("L,sp", LATTICES)
def test_cubic_lattice_phi_sweep(ibrd, L, sp):
    """Sec. IV.B, Eq. beta_cubic, packing fractions 0.002-0.134 (the paper's
    range is 0 < phi < 0.15): the GPU solve of a cubic lattice gives the mean
    concentration of the oracle's single periodic cell within 1e-8, and
    beta_0 follows the paper's fit to Lu's data within 1 % for phi < 0.02 and
    within 5 % above (where the supports of neighbouring blobs come within a
    few cells of each other)."""
    from oracle import direct
    q = lattice_positions((L, L, L), 1.0, sp)
    g = ibrd.Grid(L, L, L)
    g.set_blobs(dev(q))
    V = L ** 3
    src = np.full((L, L, L), 1.0 / V)
    c, lam, info = g.solve_saddle(dev(src), tol=1e-10, max_iter=500)
    a = 1.27
    phi = len(q) * (4 * math.pi * a ** 3 / 3) / V
    # the oracle's single cell: one blob at a node of an sp^3 box, same source density
    v1 = sp ** 3
    c1, _, _ = direct.solve_saddle(np.zeros((1, 3)), np.full((sp, sp, sp), 1.0 / V), 1.0, 1.0, 0.0)
    assert abs(info["cbar"] - c1.mean()) < 1e-8 * abs(c1.mean())
    b0 = outputs.beta0(info["cbar"], 1.0 / V, a, 1.0, len(q), V)
    fit = outputs.beta0_cubic_fit(phi)
    assert abs(b0 / fit - 1.0) < (0.01 if phi < 0.02 else 0.05), (phi, b0, fit)
    assert v1 * len(q) == V


def test_finite_rate_omega_linear_in_P(ibrd):
    """Sec. IV.D (Fig. finite_P_fit right): one blob (4-point kernel, at a
    node) in a periodic box, steady reaction-limited solves at P = 4 pi chi a /
    kappa from 0.1 to 10. Eq. Omega's Omega = [s a^2 (1 - phi) / (3 phi chi
    cbar)]^-1 is linear in P: for one periodic blob Sec. III.D gives c_P - c_0
    = lambda / kappa exactly, so Omega = beta_0^-1 + P / (1 - phi), with
    beta_0 from the diffusion-limited solve; Lu's approximation (Eq.
    beta_P_theory) has slope (1 - phi), the same to O(phi). The paper uses
    L = 100 grid cells; this multigrid needs sides that halve to a coarsest
    level of at most 512 cells, so L = 128 (phi = 4e-6) stands in."""
    L = 128
    a = 1.27
    V = L ** 3
    phi = (4 * math.pi * a ** 3 / 3) / V
    q = np.array([[L / 2, L / 2, L / 2]])
    g = ibrd.Grid(L, L, L)
    g.set_blobs(dev(q))
    src = dev(np.full((L, L, L), 1.0 / V))
    # the source is 1/V, so the FP64 floor of the relative residual is near
    # 1e-8 here (c is of order 1); cbar is still fixed to far more digits than
    # the 1e-6 checks below need
    _, _, info0 = g.solve_saddle(src, tol=2e-8, max_iter=500)
    omega0 = 1.0 / outputs.beta0(info0["cbar"], 1.0 / V, a, 1.0, 1, V)
    Ps = [0.1, 0.3, 1.0, 3.0, 10.0]
    om = []
    for P in Ps:
        kappa = 4 * math.pi * 1.0 * a / P
        _, info = g.solve_reaction(dev(np.array([kappa])), src, tol=2e-8, max_iter=500)
        om.append(1.0 / outputs.beta0(info["cbar"], 1.0 / V, a, 1.0, 1, V))
    om = np.array(om)
    np.testing.assert_allclose(om - omega0, np.array(Ps) / (1 - phi), rtol=1e-6)
    slope, icept = np.polyfit(Ps, om, 1)
    assert abs(slope - 1 / (1 - phi)) < 1e-6 and abs(icept - omega0) < 1e-6 * omega0
    # Eq. beta_P_theory: beta_P = (1 + P) / Omega against (1 + P) / (beta_0^-1 + (1 - phi) P)
    beta_p = (1 + np.array(Ps)) / om
    theory = (1 + np.array(Ps)) / (omega0 + (1 - phi) * np.array(Ps))
    assert np.abs(beta_p / theory - 1).max() < 5 * phi * max(Ps)
