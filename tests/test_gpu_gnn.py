"""The learned multiplier predictor's CUDA kernels against its FP64 definition
(oracle/gnn.py), through the C ABI: neighbour sets exactly, the FP32 forward
pass, loss and gradient within FP32 rounding, Adam's update, the bfloat16
tensor-core prediction against the definition with bfloat16 operands,
training, and its use as the warm start of a saddle solve."""
import numpy as np
import pytest

from oracle import direct, gnn
from synthetic import rsa_positions, workload
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


def _theta(seed):
    th = gnn.init_params(seed)
    p = gnn.unpack(th)
    rng = np.random.default_rng(seed + 100)
    for k in gnn.BIASES:
        p[k] = rng.uniform(-0.3, 0.3, size=p[k].shape)
    p["o0"] = np.array([0.2])
    # the FP32 model holds FP32 weights: give the reference the same values
    return gnn.pack(p).astype(np.float32).astype(np.float64)


def _config(n, side, seed, spacing=2.0):
    q = rsa_positions(n, (side, side, side), 1.0, spacing, seed)
    return q, np.array([side, side, side], dtype=np.float64)


# 40 / 8: five cells of the cell list per axis; 40 / 10 and 30 / 9.99: three
# (the fewest it takes, the last with cells barely longer than R); 20 / 9.5:
# two, so all pairs are screened; one blob: no neighbour at all
@pytest.mark.parametrize("n,side,R", [(200, 40, 8.0), (500, 40, 10.0), (150, 30, 9.99), (37, 20, 9.5),
                                      (1, 24, 6.0)])
def test_neighbours_exact(ibrd, n, side, R):
    q, box = _config(n, side, 3)
    m = ibrd.GNN(R, 64)
    cnt, idx, dist = m.neighbours(dev(q), box)
    cnt, idx, dist = host(cnt), host(idx), host(dist)
    nb, rr = gnn.neighbours(q, box, R)
    for i in range(n):
        assert cnt[i] == len(nb[i])
        assert list(idx[i, :cnt[i]]) == list(nb[i])
        # distances from FP32 coordinates: within a few ulps of the box side
        assert np.abs(dist[i, :cnt[i]] - rr[i]).max(initial=0.0) < 4e-6 * side


@pytest.mark.parametrize("box,R", [((40.0, 30.0, 50.0), 9.0), ((40.0, 18.0, 50.0), 8.5)])
def test_neighbours_non_cubic_box_and_shifted_positions(ibrd, box, R):
    """A box with three different sides (4 x 3 x 5 cells of the cell list; with
    18 along y only two fit, so all pairs are screened) and blobs given
    anywhere within a few box lengths of the origin: the lists are the FP64
    minimum-image definition's, and so is the forward pass."""
    box = np.array(box)
    q = rsa_positions(150, tuple(box), 1.0, 2.0, 17)
    rng = np.random.default_rng(4)
    q = q + box * rng.integers(-3, 4, size=q.shape)
    m = ibrd.GNN(R, 64)
    cnt, idx, dist = (host(t) for t in m.neighbours(dev(q), box))
    nb, rr = gnn.neighbours(q, box, R)
    for i in range(len(q)):
        assert cnt[i] == len(nb[i])
        assert list(idx[i, :cnt[i]]) == list(nb[i])
        assert np.abs(dist[i, :cnt[i]] - rr[i]).max(initial=0.0) < 4e-6 * box.max()
    th = _theta(3)
    m.set_params(th.astype(np.float32))
    y = host(m.forward(dev(q), box)).astype(np.float64)
    y_ref, _ = gnn.forward(th, q, box, R)
    assert np.abs(y - y_ref).max() < 2e-5 * max(1.0, np.abs(y_ref).max())


def test_forward_loss_gradient_and_adam(ibrd):
    import torch
    q, box = _config(300, 48, 5)
    R = 10.0
    th = _theta(7)
    lam = np.exp(np.random.default_rng(2).normal(0.0, 0.15, size=len(q)))
    m = ibrd.GNN(R, 64)
    m.set_params(th)
    qd, ld = dev(q), dev(lam)
    y = host(m.forward(qd, box)).astype(np.float64)
    y_ref, _ = gnn.forward(th, q, box, R)
    assert np.abs(y - y_ref).max() < 2e-5 * max(1.0, np.abs(y_ref).max())
    L, g = m.loss_grad(qd, box, ld)
    L_ref, g_ref = gnn.loss_and_grad(th, q, box, R, lam)
    assert abs(L - L_ref) < 1e-4 * L_ref
    g = host(g).astype(np.float64)
    off = 0
    for name, shape in gnn.LAYOUT:
        k = int(np.prod(shape))
        a, b = g[off:off + k], g_ref[off:off + k]
        # FP32 sums over blobs and edges: 1e-4 of the block, or 1e-6 of the
        # whole gradient for blocks that are sums of nearly cancelling terms
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b) + 1e-6 * np.linalg.norm(g_ref), name
        off += k
    # one Adam step from zero moments against the reference update
    m.adam_step(torch.from_numpy(g.astype(np.float32)).cuda(), 1e-3)
    th1 = m.get_params().astype(np.float64)
    z = np.zeros_like(th)
    want, _, _ = gnn.adam_step(th, g.astype(np.float32).astype(np.float64), z, z, 1, 1e-3)
    assert np.abs(th1 - want).max() < 1e-6
    # prediction: softmax of y scaled to the total, on the tensor-core path
    lam0 = host(m.predict(qd, box, 123.0))
    assert abs(lam0.sum() - 123.0) < 1e-9 * 123.0
    th1 = gnn.pack(gnn.unpack(th1))
    assert rel_err(lam0, gnn.predict(th1, q, box, R, 123.0, bf16_products=True)) < 2e-4


@pytest.mark.parametrize("n,side,R", [(500, 40, 10.0), (300, 48, 10.0), (37, 20, 9.5), (1, 24, 6.0)])
def test_predict_bfloat16_tensor_cores(ibrd, n, side, R):
    """The inference path (bfloat16 operands on mma.sync, FP32 accumulation)
    against the definition with bfloat16-rounded operands and exact sums: 500
    blobs have about 33 neighbours each (three 16-edge tiles, the last ragged),
    and none of the blob counts fills whole 16-blob node tiles. It must also be
    much closer to that definition than to the exact FP64 one, which it
    differs from by bfloat16 rounding (about 1e-3 of lambda)."""
    q, box = _config(n, side, 5)
    th = _theta(7)
    m = ibrd.GNN(R, 64)
    m.set_params(th.astype(np.float32))
    lam0 = host(m.predict(dev(q), box, 123.0))
    want = gnn.predict(th, q, box, R, 123.0, bf16_products=True)
    exact = gnn.predict(th, q, box, R, 123.0)
    err = rel_err(lam0, want)
    assert err < 2e-4, err
    gap = rel_err(want, exact)
    if gap > 1e-5:
        assert err < 0.25 * gap, (err, gap)
    # the FP32 forward of the same model stays on the exact definition
    y = host(m.forward(dev(q), box)).astype(np.float64)
    y_ref, _ = gnn.forward(th, q, box, R)
    assert np.abs(y - y_ref).max() < 2e-5 * max(1.0, np.abs(y_ref).max())


def test_predict_full_size_workload(ibrd):
    """The benchmark's evaluation case: the 256^3 workload's 4096 blobs with
    the cutoff 24h and the library's seeded weights; the tensor-core
    prediction against the definition with bfloat16 operands, every blob."""
    w = workload("scale")
    R = 24.0
    box = np.array([256.0, 256.0, 256.0])
    m = ibrd.GNN(R, 256)
    m.init_params(1)
    th = m.get_params().astype(np.float64)
    total = float(w.g.sum())
    lam0 = host(m.predict(dev(w.q), box, total))
    want = gnn.predict(th, w.q, box, R, total, bf16_products=True)
    assert rel_err(lam0, want) < 2e-4
    y = host(m.forward(dev(w.q), box)).astype(np.float64)
    y_ref, _ = gnn.forward(th, w.q, box, R)
    assert np.abs(y - y_ref).max() < 2e-5 * max(1.0, np.abs(y_ref).max())


def test_too_many_neighbours_is_an_argument_error(ibrd):
    q, box = _config(60, 20, 9, spacing=1.0)
    m = ibrd.GNN(9.9, 4)
    with pytest.raises(ibrd.IbrdError) as e:
        m.forward(dev(q), box)
    assert e.value.status == 1


def test_training_reduces_the_loss(ibrd):
    """Targets made by a teacher network of the same form: training a fresh
    model on 12 configurations lowers the loss several-fold."""
    R = 10.0
    teacher = _theta(11)
    qs, boxes, lams = [], [], []
    for s in range(12):
        q, box = _config(120, 40, 40 + s)
        y, _ = gnn.forward(teacher, q, box, R)
        qs.append(dev(q))
        boxes.append(box)
        lams.append(dev(np.exp(y - y.mean())))
    m = ibrd.GNN(R, 64)
    m.set_params(gnn.init_params(3).astype(np.float32))
    losses = m.train(qs, boxes, lams, epochs=30, lr=3e-3)
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.25 * losses[0]


def test_learned_warm_start_saddle(ibrd):
    """Multipliers from GPU saddle solves train the model; its prediction on a
    new configuration starts a saddle solve that reaches the oracle's exact
    solution within 1e-11."""
    import torch
    d, h = (32, 32, 32), 1.0
    box = np.array([32.0, 32.0, 32.0])
    R = 12.0
    qs, lams = [], []
    for s in range(6):
        q = rsa_positions(40, d, h, 4.0, 60 + s)
        g = ibrd.Grid(*d)
        g.set_blobs(dev(q))
        _, lam, info = g.solve_saddle(dev(np.ones((32, 32, 32))), tol=1e-10, precision=0)
        assert info["status"] == 0
        qs.append(dev(q))
        lams.append(lam)
    m = ibrd.GNN(R, 64)
    m.set_params(gnn.init_params(5).astype(np.float32))
    losses = m.train(qs, [box] * len(qs), lams, epochs=20, lr=2e-3)
    assert losses[-1] < losses[0]
    w = workload("small")
    c_ref, lam_ref, _ = direct.solve_saddle(w.q, w.g, w.h, w.chi, 0.0)
    lam0 = m.predict(dev(w.q), box, float(w.g.sum()))
    g = ibrd.Grid(*w.dims)
    g.set_blobs(dev(w.q))
    tol = floor_tol(c_ref, w.g, w.h, w.chi, 0.0)
    c, lam, info = g.solve_saddle(dev(w.g), lam=lam0, tol=tol, precision=2, lambda_guess=2, max_iter=400)
    assert info["rel_residual"] <= tol
    assert rel_err(host(c), c_ref) < 1e-11 and rel_err(host(lam), lam_ref) < 1e-11
    torch.cuda.synchronize()


def test_seeded_init(ibrd):
    """The library's seeded initial parameters: reproducible, seed-dependent,
    within +-1/sqrt(fan in), biases zero."""
    m = ibrd.GNN(8.0, 16)
    m.init_params(9)
    a = m.get_params()
    m.init_params(9)
    b = m.get_params()
    m.init_params(10)
    c = m.get_params()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    p = gnn.unpack(a.astype(np.float64))
    lims = [("W0", 0.25), ("o", 0.125)]
    for l in range(1, gnn.LAYERS + 1):
        lims += [(f"E{l}", 0.25), (f"W{l}", 0.125), (f"V{l}", 0.125)]
    for name, lim in lims:
        assert np.abs(p[name]).max() <= lim and np.abs(p[name]).max() > 0.9 * lim
    for name in gnn.BIASES + ["o0"]:
        assert not p[name].any()
