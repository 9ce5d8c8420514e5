"""Pins of the learned multiplier predictor's FP64 definition (oracle/gnn.py)
against facts that do not come from the oracle itself: central finite
differences for every gradient block, a k-d tree for the neighbour lists,
the symmetries of the network, the cutoff's continuity, and Adam's first step
in closed form."""
import numpy as np
import pytest

from oracle import gnn


def _config(n=14, side=20.0, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, side, size=(n, 3)), np.array([side, side, side])


def _theta(seed=1):
    th = gnn.init_params(seed)
    # non-zero biases so that both sides of every relu are exercised
    p = gnn.unpack(th)
    rng = np.random.default_rng(seed + 100)
    for k in gnn.BIASES:
        p[k] = rng.uniform(-0.3, 0.3, size=p[k].shape)
    p["o0"] = np.array([0.2])
    return gnn.pack(p)


def test_layout_size():
    # embedding, three layers (filter E, e; W, V, c), output
    assert gnn.n_params() == (64 * 16 + 64) + 3 * (64 * 16 + 64 + 2 * 64 * 64 + 64) + 64 + 1


def test_bf16_rounding_matches_torch():
    """The oracle's bfloat16 rounding (nearest, ties to even, of the FP32
    value) against torch's float32 -> bfloat16 conversion."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    v = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -0.0, 2.0 ** -130]])
    want = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(gnn.bf16(v), want)


def test_bf16_forward_is_close_and_exact_on_representable_values():
    """Inference with bfloat16 operands stays within a few bfloat16 ulps of
    the exact forward, and equals it when every weight is representable and
    the inputs of each product happen to be too (a zero-layer check: with all
    layer weights zero only biases and the exact embedding act)."""
    q, box = _config()
    th = _theta()
    y, _ = gnn.forward(th, q, box, 8.0)
    yb, _ = gnn.forward(th, q, box, 8.0, bf16_products=True)
    assert not np.array_equal(y, yb)
    assert np.abs(y - yb).max() < 3 * 2.0 ** -8 * (np.abs(y).max() + 1.0)
    p = gnn.unpack(th)
    for l in range(1, gnn.LAYERS + 1):
        for k in ("E", "W", "V"):
            p[f"{k}{l}"] = np.zeros_like(p[f"{k}{l}"])
    t0 = gnn.pack(p)
    assert np.array_equal(gnn.forward(t0, q, box, 8.0)[0], gnn.forward(t0, q, box, 8.0, bf16_products=True)[0])


def test_neighbours_match_kdtree():
    scipy = pytest.importorskip("scipy.spatial")
    q, box = _config(40, 24.0, 3)
    R = 8.0
    nb, rr = gnn.neighbours(q, box, R)
    tree = scipy.cKDTree(q, boxsize=box)
    for i in range(len(q)):
        want = sorted(j for j in tree.query_ball_point(q[i], R - 1e-12) if j != i)
        assert list(nb[i]) == want
        d = q[nb[i]] - q[i]
        d -= box * np.round(d / box)
        assert np.allclose(rr[i], np.linalg.norm(d, axis=1))


@pytest.mark.parametrize("block", [name for name, _ in gnn.LAYOUT])
def test_gradient_central_differences(block):
    q, box = _config()
    R = 8.0
    th = _theta()
    lam = np.exp(np.random.default_rng(5).normal(0, 0.2, size=len(q)))
    _, grad = gnn.loss_and_grad(th, q, box, R, lam)
    off = 0
    for name, shape in gnn.LAYOUT:
        n = int(np.prod(shape))
        if name == block:
            break
        off += n
    rng = np.random.default_rng(7)
    idx = off + rng.choice(n, size=min(n, 12), replace=False)
    eps = 1e-6
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (gnn.loss(tp, q, box, R, lam) - gnn.loss(tm, q, box, R, lam)) / (2 * eps)
        assert abs(fd - grad[k]) <= 1e-6 * max(1e-3, abs(fd)), (name, k, fd, grad[k])


def test_permutation_and_translation():
    q, box = _config(20, 22.0, 9)
    R = 9.0
    th = _theta(2)
    y, _ = gnn.forward(th, q, box, R)
    perm = np.random.default_rng(1).permutation(len(q))
    yp, _ = gnn.forward(th, q[perm], box, R)
    assert np.allclose(yp, y[perm], rtol=0, atol=1e-12)
    qs = np.mod(q + np.array([7.3, -2.1, 15.9]), box)
    ys, _ = gnn.forward(th, qs, box, R)
    assert np.allclose(ys, y, rtol=0, atol=1e-12)
    # a reflection of the box maps every distance to itself
    yr, _ = gnn.forward(th, np.mod(-q, box), box, R)
    assert np.allclose(yr, y, rtol=0, atol=1e-12)


def test_cutoff_is_continuous():
    box = np.array([30.0, 30.0, 30.0])
    R = 8.0
    th = _theta(3)
    ys = []
    for d in (R - 1e-7, R + 1e-7):
        q = np.array([[5.0, 5.0, 5.0], [5.0 + d, 5.0, 5.0], [20.0, 20.0, 20.0]])
        ys.append(gnn.forward(th, q, box, R)[0])
    assert np.abs(ys[0] - ys[1]).max() < 1e-9
    assert np.allclose(gnn.basis(np.array([R]), R), 0.0)


def test_isolated_blobs_share_equally():
    # no neighbours: every y equals the network's constant output
    q = np.array([[1.0, 1.0, 1.0], [15.0, 15.0, 15.0], [1.0, 15.0, 8.0]])
    lam = gnn.predict(_theta(4), q, np.array([30.0, 30.0, 30.0]), 6.0, 12.0)
    assert np.allclose(lam, 4.0, rtol=0, atol=1e-12)


def test_exact_prediction_has_zero_loss_and_gradient():
    q, box = _config(10, 18.0, 11)
    R = 7.0
    th = _theta(5)
    y, _ = gnn.forward(th, q, box, R)
    lam = 3.0 * np.exp(y)
    L, grad = gnn.loss_and_grad(th, q, box, R, lam)
    assert L < 1e-28 and np.abs(grad).max() < 1e-13
    assert abs(gnn.predict(th, q, box, R, 5.0).sum() - 5.0) < 1e-12


def test_adam_first_step_closed_form():
    # from zero moments, step 1 moves every parameter by lr * g / (|g| + eps)
    rng = np.random.default_rng(2)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    z = np.zeros(50)
    new, m1, m2 = gnn.adam_step(th, g, z, z, 1, 0.01)
    assert np.allclose(th - new, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m1, 0.1 * g) and np.allclose(m2, 0.001 * g * g)
