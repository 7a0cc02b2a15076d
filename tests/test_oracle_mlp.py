"""Pins of the FP64 warm-start-network oracle (CPU only).

* GELU at closed values: GELU(0) = 0, GELU(1) = Phi(1), GELU'(0) = 1/2,
  GELU(-z) = GELU(z) - z (odd part), and GELU' against a central difference.
* A network whose last layer is zero outputs b3: its loss is the masked mean of
  (b3 - t)^2, a closed form.
* The analytic gradient of every parameter against central finite differences
  of the loss (FP64, step 1e-6) on a small random batch.
* Histogram features sum to 1, are non-negative, and the one-hot part marks C.
* Planted mistakes in a copy of the backward pass (a dropped GELU factor, a
  transposed weight, an unmasked loss) break the finite-difference pin.
"""
import numpy as np
import pytest
from scipy.special import erf

from oracle import mlp


def rand_params(seed, scale=0.2):
    g = np.random.default_rng(seed)
    return {k: scale * g.standard_normal(s) for k, s in mlp.PARAM_SHAPES.items()}


def rand_batch(seed, B=6):
    g = np.random.default_rng(seed)
    X = np.abs(g.standard_normal((B, mlp.D_IN))) * 0.05
    Cs = g.integers(1, 9, size=B)
    X[:, mlp.D_HIST:] = 0.0
    X[np.arange(B), mlp.D_HIST + Cs - 1] = 1.0
    T = g.uniform(0, 1, (B, mlp.D_OUT))
    return X, T, Cs


def test_gelu_closed_values():
    Phi1 = 0.5 * (1.0 + erf(1.0 / np.sqrt(2.0)))
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(Phi1 - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    z = np.linspace(-4, 4, 33)
    assert np.allclose(mlp.gelu(-z), mlp.gelu(z) - z, atol=1e-14)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(fd, mlp.gelu_grad(z), atol=1e-8)


def test_zero_last_layer_loss_closed_form():
    p = rand_params(1)
    p["W3"][:] = 0.0
    X, T, Cs = rand_batch(2)
    L, _ = mlp.loss_and_grads(p, X, T, Cs)
    M = mlp.mask_of(Cs)
    ref = np.sum(((p["b3"][None, :] - T) ** 2) * M) / M.sum()
    assert abs(L - ref) <= 1e-14 * max(1.0, ref)


def _fd_check(grad_fn, p, X, T, Cs, n_probe=12, h=1e-6, seed=0):
    """Largest relative error of the analytic gradient on random coordinates."""
    L0, g = grad_fn(p, X, T, Cs)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for k in mlp.PARAM_ORDER:
        for _ in range(n_probe):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][idx] += h
            Lp, _ = mlp.loss_and_grads(q, X, T, Cs)
            q[k][idx] -= 2 * h
            Lm, _ = mlp.loss_and_grads(q, X, T, Cs)
            fd = (Lp - Lm) / (2 * h)
            an = g[k][idx]
            worst = max(worst, abs(fd - an) / max(1e-6, abs(fd) + abs(an)))
    return worst


def test_gradients_match_finite_differences():
    p = rand_params(3, scale=0.5)
    X, T, Cs = rand_batch(4)
    assert _fd_check(mlp.loss_and_grads, p, X, T, Cs) < 1e-6


def test_features_are_a_histogram():
    g = np.random.default_rng(9)
    x = g.uniform(-10, 270, 1001)
    f = mlp.features(x, 5)
    assert abs(f[:256].sum() - 1.0) < 1e-15 and f.min() >= 0
    assert f[256 + 4] == 1.0 and f[256:].sum() == 1.0
    assert f[0] == np.mean(np.rint(x) <= 0) and f[255] == np.mean(np.rint(x) >= 255)


def _mutant(kind):
    def grads(p, X, T, Cs):
        y, (X_, z1, a1, z2, a2) = mlp.forward(p, X)
        M = mlp.mask_of(Cs) if kind != "unmasked" else np.ones_like(y)
        cnt = mlp.mask_of(Cs).sum()
        r = (y - T) * M
        dy = 2.0 * r / cnt
        g = {"W3": dy.T @ a2, "b3": dy.sum(0)}
        da2 = dy @ p["W3"]
        dz2 = da2 * (1.0 if kind == "no_gelu_factor" else mlp.gelu_grad(z2))
        g["W2"] = dz2.T @ a1 if kind != "transposed" else (dz2.T @ a1).T
        g["b2"] = dz2.sum(0)
        da1 = dz2 @ p["W2"]
        dz1 = da1 * mlp.gelu_grad(z1)
        g["W1"] = dz1.T @ X_
        g["b1"] = dz1.sum(0)
        return float(np.sum(r * r) / cnt), g
    return grads


@pytest.mark.parametrize("kind", ["no_gelu_factor", "transposed", "unmasked"])
def test_planted_backward_mistakes_are_caught(kind):
    p = rand_params(5, scale=0.5)
    X, T, Cs = rand_batch(6)
    Cs[0] = 3  # some masked outputs
    assert _fd_check(_mutant(kind), p, X, T, Cs) > 1e-3
