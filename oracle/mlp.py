"""FP64 oracle of the warm-start network — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. The CUDA library shares no code with it.

The paper starts FCM from random memberships (Sec. 2.1, Algorithm 1 step 2);
it has no learned initialisation. The network here maps a slice's grey-level
histogram to initial centers V^0:

  input  f = [h_0 .. h_255, onehot(C)_1 .. onehot(C)_8]   (264 values)
         h_b = (# pixels with round(clip(x, 0, 255)) == b) / n
  layer 1  z1 = W1 f + b1,  a1 = GELU(z1)                 (128)
  layer 2  z2 = W2 a1 + b2, a2 = GELU(z2)                 (128)
  layer 3  y  = W3 a2 + b3                                (8)
  V^0 = sort(255 * y[:C])

  GELU(z) = z * Phi(z) = z/2 * (1 + erf(z / sqrt(2)))
  loss    = sum_{b, j < C_b} (y_bj - t_bj)^2 / sum_b C_b   (masked MSE)
  targets t_bj = (sorted converged centers of slice b) / 255 for j < C_b.

Training takes Adam steps (Kingma & Ba 2015, Algorithm 1) with bias
correction: for step t with gradient g,
  m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
  w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Weights are stored as W[out, in]. ``params`` is a dict of FP64 arrays W1, b1,
W2, b2, W3, b3. Pinned by ``tests/test_oracle_mlp.py``: finite differences of
the loss, closed values of GELU, a zero network's loss, a network with
hand-set weights whose outputs are exact (each pre-activation is 0, +-1 or far
into GELU's linear or zero regime), histogram invariants, and the closed forms
of the first two Adam steps.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

D_HIST = 256
D_ONEHOT = 8
D_IN = D_HIST + D_ONEHOT
D_H = 128
D_OUT = 8
PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")
PARAM_SHAPES = {"W1": (D_H, D_IN), "b1": (D_H,), "W2": (D_H, D_H), "b2": (D_H,),
                "W3": (D_OUT, D_H), "b3": (D_OUT,)}


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    """d/dz z Phi(z) = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def features(x, C):
    """Input vector of one slice: normalised 256-bin histogram of the grey
    levels (rounded to the nearest integer, clipped to [0, 255]) and a one-hot
    encoding of C in 1..8."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    b = np.clip(np.rint(x), 0, 255).astype(np.int64)
    f = np.zeros(D_IN)
    f[:D_HIST] = np.bincount(b, minlength=D_HIST) / x.size
    f[D_HIST + C - 1] = 1.0
    return f


def forward(params, X):
    """Network output y [B, 8] and the intermediate values."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ params["W1"].T + params["b1"]
    a1 = gelu(z1)
    z2 = a1 @ params["W2"].T + params["b2"]
    a2 = gelu(z2)
    y = a2 @ params["W3"].T + params["b3"]
    return y, (X, z1, a1, z2, a2)


def mask_of(Cs):
    Cs = np.asarray(Cs).reshape(-1)
    return (np.arange(D_OUT)[None, :] < Cs[:, None]).astype(np.float64)


def loss_and_grads(params, X, T, Cs):
    """Masked mean squared error and its gradient with respect to every
    parameter (backpropagation through the three layers)."""
    y, (X, z1, a1, z2, a2) = forward(params, X)
    M = mask_of(Cs)
    cnt = M.sum()
    r = (y - np.asarray(T, dtype=np.float64)) * M
    loss = float(np.sum(r * r) / cnt)
    dy = 2.0 * r / cnt
    g = {"W3": dy.T @ a2, "b3": dy.sum(0)}
    da2 = dy @ params["W3"]
    dz2 = da2 * gelu_grad(z2)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(0)
    da1 = dz2 @ params["W2"]
    dz1 = da1 * gelu_grad(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return loss, g


def predict_centers(params, X, Cs):
    """V^0 of every slice: the first C outputs times 255, sorted."""
    y, _ = forward(params, X)
    return [np.sort(255.0 * y[b, :C]) for b, C in enumerate(np.asarray(Cs).reshape(-1))]


def flat(params):
    return np.concatenate([np.asarray(params[k], dtype=np.float64).reshape(-1) for k in PARAM_ORDER])


def unflat(v):
    v = np.asarray(v, dtype=np.float64)
    out, o = {}, 0
    for k in PARAM_ORDER:
        size = int(np.prod(PARAM_SHAPES[k]))
        out[k] = v[o:o + size].reshape(PARAM_SHAPES[k])
        o += size
    return out


N_PARAMS = sum(int(np.prod(s)) for s in PARAM_SHAPES.values())


ADAM_B1 = 0.9
ADAM_B2 = 0.999
ADAM_EPS = 1e-8


def adam_step(params, grads, m, v, t, lr, b1=ADAM_B1, b2=ADAM_B2, eps=ADAM_EPS):
    """Adam step t (1-based) on every parameter, FP64; returns the new
    (params, m, v). ``m`` and ``v`` are dicts like ``params`` (zero before the
    first step)."""
    c1 = 1.0 - b1 ** t
    c2 = 1.0 - b2 ** t
    out_p, out_m, out_v = {}, {}, {}
    for k in PARAM_ORDER:
        g = np.asarray(grads[k], dtype=np.float64)
        mk = b1 * np.asarray(m[k], dtype=np.float64) + (1.0 - b1) * g
        vk = b2 * np.asarray(v[k], dtype=np.float64) + (1.0 - b2) * g * g
        out_p[k] = np.asarray(params[k], dtype=np.float64) - lr * (mk / c1) / (np.sqrt(vk / c2) + eps)
        out_m[k] = mk
        out_v[k] = vk
    return out_p, out_m, out_v


def zeros_like_params():
    return {k: np.zeros(PARAM_SHAPES[k]) for k in PARAM_ORDER}
