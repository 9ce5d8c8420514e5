"""FP64 reference of the learned multiplier predictor (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use
this module; the product path never imports it.

The paper leaves the Schur complement J A^-1 S of the diffusion-limited
saddle point (Eq. saddle_point) without a good preconditioner for many blobs
and names that as open (Sec. III.E, Sec. V). This module defines, in plain
NumPy, a small graph network over each blob's neighbours that predicts the
relative sink strengths lambda_i / <lambda> of a configuration, which serve
as the initial guess of the multipliers. The definition below is what the
CUDA kernels compute; it is written out step by step so that a reader can
check it.

Graph. Blobs i and j (j != i) are neighbours when the minimum-image distance
r_ij of their centres in the periodic box is below the cutoff R (R at most
half of the shortest box side, so the minimum image is unique).

Features. With s = r / R, a smooth cutoff f_c(s) = (1 - s)^2 and K = 16
Gaussian radial bases centred at mu_k = k / (K - 1) with width
sigma = 1.5 / (K - 1):

    b_k(r)  = f_c(s) exp(-((s - mu_k) / sigma)^2)

Network (width H = 64, L = 3 message-passing layers):

    x_i    = sum_j b(r_ij)                                       (K)
    a0_i   = W0 x_i + c0,          h0_i = relu(a0_i)             (H)
    for l = 1 .. L:
      P_ij = E_l b(r_ij) + e_l,    F_ij = relu(P_ij)             (H, per edge)
      m_i  = sum_j f_c(s_ij) F_ij * h_{l-1,j}                    (H, elementwise)
      a_i  = W_l m_i + V_l h_{l-1,i} + c_l
      h_{l,i} = h_{l-1,i} + relu(a_i)
    y_i    = o . h_{L,i} + o0

Inference on tensor cores (forward(..., bf16=True)): the operands of the
dense products E_l b, W_l m and V_l h -- the weights and the vectors they
multiply -- are rounded to bfloat16 (the nearest, ties to even, of their
FP32 values), the products summed exactly and the biases, relus and
residual sums kept at full precision; the embedding and output stay exact.

Prediction: lambda0_i = T exp(y_i) / sum_k exp(y_k), with T the total the
solvability condition fixes (zeta sum lambda = h^3 sum g, Appendix A).

Loss of one configuration with solved multipliers lambda (all > 0):
t_i = log lambda_i, r_i = (y_i - <y>) - (t_i - <t>), L = <r^2>.

Optimizer: Adam with bias correction.
"""
from __future__ import annotations

import numpy as np

H = 64
K = 16
LAYERS = 3
SIGMA = 1.5 / (K - 1)
MU = np.arange(K, dtype=np.float64) / (K - 1)

# Flat parameter layout shared with the library: name, shape.
LAYOUT = [("W0", (H, K)), ("c0", (H,))]
for _l in range(1, LAYERS + 1):
    LAYOUT += [(f"E{_l}", (H, K)), (f"e{_l}", (H,)), (f"W{_l}", (H, H)), (f"V{_l}", (H, H)), (f"c{_l}", (H,))]
LAYOUT += [("o", (H,)), ("o0", (1,))]
BIASES = ["c0"] + [f"{n}{l}" for l in range(1, LAYERS + 1) for n in ("e", "c")]


def n_params() -> int:
    return int(sum(np.prod(s) for _, s in LAYOUT))


def unpack(theta: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in LAYOUT:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in LAYOUT])


def init_params(seed: int) -> np.ndarray:
    """Seeded initial weights: uniform in +-1/sqrt(fan_in) (biases 0, o0 0)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in LAYOUT:
        if len(shape) == 2:
            lim = 1.0 / np.sqrt(shape[1])
            p[name] = rng.uniform(-lim, lim, size=shape)
        elif name == "o":
            p[name] = rng.uniform(-1.0 / np.sqrt(H), 1.0 / np.sqrt(H), size=shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)


def bf16(v) -> np.ndarray:
    """The bfloat16 nearest to each value's FP32 rounding (ties to even), as
    float64: the top 16 bits of the FP32 pattern after rounding."""
    f = np.asarray(v, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def neighbours(q: np.ndarray, box, R: float):
    """Per blob, the neighbours j != i with minimum-image distance < R, in
    increasing j, and those distances (brute force over all pairs)."""
    q = np.asarray(q, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    n = len(q)
    lists, dists = [], []
    for i in range(n):
        d = q - q[i]
        d -= box * np.round(d / box)
        r = np.sqrt((d ** 2).sum(1))
        js = [j for j in range(n) if j != i and r[j] < R]
        lists.append(np.array(js, dtype=np.int64))
        dists.append(r[js])
    return lists, dists


def basis(r: np.ndarray, R: float) -> np.ndarray:
    """b_k(r) for an array of distances: shape (len(r), K)."""
    s = np.asarray(r, dtype=np.float64)[:, None] / R
    fc = (1.0 - s) ** 2
    return fc * np.exp(-((s - MU[None, :]) / SIGMA) ** 2)


def cutoff(r: np.ndarray, R: float) -> np.ndarray:
    return (1.0 - np.asarray(r, dtype=np.float64) / R) ** 2


def forward(theta: np.ndarray, q: np.ndarray, box, R: float, bf16_products: bool = False):
    """Outputs y (N,) and the intermediate values the gradient needs."""
    p = unpack(theta)
    rd = bf16 if bf16_products else (lambda v: v)
    nb, rr = neighbours(q, box, R)
    n = len(q)
    x = np.zeros((n, K))
    for i in range(n):
        if len(nb[i]):
            x[i] = basis(rr[i], R).sum(0)
    a0 = x @ p["W0"].T + p["c0"]
    h = [np.maximum(a0, 0.0)]
    ms, as_ = [], []
    for l in range(1, LAYERS + 1):
        E, e, W, V, c = p[f"E{l}"], p[f"e{l}"], p[f"W{l}"], p[f"V{l}"], p[f"c{l}"]
        m = np.zeros((n, H))
        for i in range(n):
            if len(nb[i]):
                P = rd(basis(rr[i], R)) @ rd(E).T + e
                m[i] = (cutoff(rr[i], R)[:, None] * np.maximum(P, 0.0) * h[-1][nb[i]]).sum(0)
        a = rd(m) @ rd(W).T + rd(h[-1]) @ rd(V).T + c
        ms.append(m)
        as_.append(a)
        h.append(h[-1] + np.maximum(a, 0.0))
    y = h[-1] @ p["o"] + p["o0"][0]
    cache = dict(p=p, nb=nb, rr=rr, x=x, a0=a0, h=h, m=ms, a=as_)
    return y, cache


def predict(theta, q, box, R, total, bf16_products: bool = False):
    """lambda0_i = total * softmax(y)_i."""
    y, _ = forward(theta, q, box, R, bf16_products)
    e = np.exp(y - y.max())
    return total * e / e.sum()


def loss(theta, q, box, R, lam):
    y, _ = forward(theta, q, box, R)
    t = np.log(np.asarray(lam, dtype=np.float64))
    r = (y - y.mean()) - (t - t.mean())
    return float(np.mean(r ** 2))


def loss_and_grad(theta, q, box, R, lam):
    """L and dL/dtheta (flat, LAYOUT order) by the chain rule through forward."""
    y, c = forward(theta, q, box, R)
    p = c["p"]
    n = len(y)
    t = np.log(np.asarray(lam, dtype=np.float64))
    r = (y - y.mean()) - (t - t.mean())
    L = float(np.mean(r ** 2))
    dy = 2.0 * r / n                       # r already has mean zero
    g = {k: np.zeros_like(v) for k, v in p.items()}
    g["o"] = dy @ c["h"][-1]
    g["o0"] = np.array([dy.sum()])
    dh = dy[:, None] * p["o"][None, :]     # dL/dh_L
    for l in range(LAYERS, 0, -1):
        E, e, W, V = p[f"E{l}"], p[f"e{l}"], p[f"W{l}"], p[f"V{l}"]
        hprev, m, a = c["h"][l - 1], c["m"][l - 1], c["a"][l - 1]
        da = dh * (a > 0)
        g[f"W{l}"] = da.T @ m
        g[f"V{l}"] = da.T @ hprev
        g[f"c{l}"] = da.sum(0)
        dm = da @ W
        dprev = dh + da @ V               # the residual path and V's
        for i in range(n):
            if not len(c["nb"][i]):
                continue
            b = basis(c["rr"][i], R)
            fc = cutoff(c["rr"][i], R)
            P = b @ E.T + e
            F = np.maximum(P, 0.0)
            # m_i = sum_j fc_ij F_ij * h_{l-1,j}
            dprev[c["nb"][i]] += fc[:, None] * F * dm[i][None, :]
            dP = fc[:, None] * dm[i][None, :] * hprev[c["nb"][i]] * (P > 0)
            g[f"E{l}"] += dP.T @ b
            g[f"e{l}"] += dP.sum(0)
        dh = dprev
    da0 = dh * (c["a0"] > 0)
    g["W0"] = da0.T @ c["x"]
    g["c0"] = da0.sum(0)
    return L, pack(g)


def adam_step(theta, grad, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns the new theta, m1, m2."""
    m1 = beta1 * m1 + (1.0 - beta1) * grad
    m2 = beta2 * m2 + (1.0 - beta2) * grad * grad
    mh = m1 / (1.0 - beta1 ** step)
    vh = m2 / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m1, m2
