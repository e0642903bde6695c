"""FP64 reference of the per-pixel denoiser MLP (test infrastructure only).

y = rgb + cov s_out (W4 h3 + b4),  h_l = relu(W_l h_{l-1} + b_l),  h_0 = (t(x) - mu) * is,
14 -> 64 -> 64 -> 64 -> 3, t the identity except for feature 12 (luminance
variance) entering as its square root; mu, is, s_out fixed standardisation
constants stored after the weights; cov = feature 13 (hit fraction).  The kernels
round weights, inputs and hidden activations to FP16 and accumulate in FP32;
this reference takes the same FP16 roundings (numpy float16, round to
nearest even) and does all arithmetic in FP64.  Plain numpy matrix products
serve as the steps.
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 14, 64, 3
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NH)), ("b3", (NH,)),
         ("W4", (NOUT, NH)), ("b4", (NOUT,)), ("mu", (NIN,)), ("is", (NIN,)), ("sout", (1,))]
TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")
N_WEIGHTS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SIZES])


def h16(x):
    return np.asarray(x, np.float64).astype(np.float16).astype(np.float64)


def transform(aov):
    x = np.asarray(aov, np.float64).reshape(-1, NIN).copy()
    x[:, 12] = np.sqrt(np.maximum(x[:, 12], 0.0))
    return x


def init_weights(seed=0, scale_out=0.1, aov=None, sout=1.0):
    """He-uniform hidden layers, a small output layer (the net starts near the
    identity); standardisation from the features aov (or mu = 0, is = 1)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            fan_in = shape[1]
            lim = np.sqrt(6.0 / fan_in) * (scale_out if name == "W4" else 1.0)
            d[name] = rng.uniform(-lim, lim, shape)
        else:
            d[name] = np.zeros(shape)
    d["is"][:] = 1.0
    d["sout"][:] = sout
    if aov is not None:
        x = transform(aov)
        d["mu"] = x.mean(0)
        d["is"] = 1.0 / np.maximum(x.std(0), 1e-6)
    return pack(d).astype(np.float32)


def inputs(aov, P):
    return h16((transform(aov) - P["mu"]) * P["is"])


def forward(w, aov):
    """Returns y [n, 3] and the cache for backward."""
    P = unpack(np.asarray(w, np.float64))
    W = {k: (h16(v) if k.startswith("W") else v) for k, v in P.items()}
    x = inputs(aov, P)
    a1 = x @ W["W1"].T + W["b1"]
    h1 = h16(np.maximum(a1, 0))
    a2 = h1 @ W["W2"].T + W["b2"]
    h2 = h16(np.maximum(a2, 0))
    a3 = h2 @ W["W3"].T + W["b3"]
    h3 = h16(np.maximum(a3, 0))
    raw = np.asarray(aov, np.float64).reshape(-1, NIN)
    cov = raw[:, 13:14]
    y = raw[:, :3] + cov * W["sout"][0] * (h3 @ W["W4"].T + W["b4"])
    return y, dict(W=W, x=x, a1=a1, a2=a2, a3=a3, h1=h1, h2=h2, h3=h3, cov=cov)


def input_adjoint(w, aov, d_out):
    """J^T d_out with J = dy/d(rgb features), the other features held constant.

    Same rounding points as the kernel: each pixel's d_out is scaled to unit
    maximum and rounded to FP16, and every layer's adjoint is rounded to FP16
    before the next product."""
    _, c = forward(w, aov)
    W = c["W"]
    d = np.asarray(d_out, np.float64).reshape(-1, 3)
    s = np.abs(d).max(1, keepdims=True)
    inv = np.where(s > 0, 1.0 / np.where(s > 0, s, 1.0), 0.0)
    g3 = h16((h16(d * inv) @ W["W4"]) * (c["a3"] > 0))
    g2 = h16((g3 @ W["W3"]) * (c["a2"] > 0))
    g1 = h16((g2 @ W["W2"]) * (c["a1"] > 0))
    gx = (g1 @ W["W1"]) * s * W["sout"][0] * W["is"] * c["cov"]
    return d + gx[:, :3]


def loss_and_grad(w, aov, target):
    """Mean over pixels of |y - target|^2 and its gradient w.r.t. the packed weights
    (through the FP16-rounded weights, rounding treated as identity)."""
    y, c = forward(w, aov)
    W = c["W"]
    n = y.shape[0]
    e = y - np.asarray(target, np.float64).reshape(-1, 3)
    loss = float(np.sum(e * e) / n)
    gy = 2.0 * e / n * W["sout"][0] * c["cov"]
    g = {"W4": gy.T @ c["h3"], "b4": gy.sum(0), "mu": np.zeros(NIN), "is": np.zeros(NIN), "sout": np.zeros(1)}
    g3 = (gy @ W["W4"]) * (c["a3"] > 0)
    g["W3"], g["b3"] = g3.T @ c["h2"], g3.sum(0)
    g2 = (g3 @ W["W3"]) * (c["a2"] > 0)
    g["W2"], g["b2"] = g2.T @ c["h1"], g2.sum(0)
    g1 = (g2 @ W["W2"]) * (c["a1"] > 0)
    g["W1"], g["b1"] = g1.T @ c["x"], g1.sum(0)
    return loss, pack(g)


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return w, m, v
