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


# ---------------------------------------------------------------------------
# A network with hand-set weights whose outputs are exact numbers.
#
# Every pre-activation is 0, +-1, or at least 9 away from 0, where GELU is the
# identity or zero to within 9 * Phi(-9) ~ 1e-18. With Phi(1) the standard
# normal CDF at 1 (0.84134474606854293), GELU(1) = Phi(1) and
# GELU(-1) = -(1 - Phi(1)). Two input rows differ in f_0 (0.5 and 0).
#
#   layer 1  z1_0 = 2 f_0 + 9      -> a1_0 = 2 f_0 + 9
#            z1_1 = 3 f_1 - 20     -> a1_1 = 0
#            z1_2 = 1              -> a1_2 = Phi(1)
#            z1_3 = -1             -> a1_3 = Phi(1) - 1
#   layer 2  z2_0 = a1_0 + 5 a1_1 + 10          -> a2_0 = 2 f_0 + 19
#            z2_1 = -a1_0                        -> a2_1 = 0
#            z2_2 = a1_2 + a1_3 + 9              -> a2_2 = 8 + 2 Phi(1)
#   layer 3  y_0 = a2_0 / 100                    = (2 f_0 + 19) / 100
#            y_1 = a2_1 + a2_2 / 10              = (8 + 2 Phi(1)) / 10
#            y_2 = 0.25,  y_3 = -a2_0 / 50 + 1   = 1 - (2 f_0 + 19) / 50
# ---------------------------------------------------------------------------

PHI1 = 0.84134474606854293


def exact_net():
    p = {k: np.zeros(s) for k, s in mlp.PARAM_SHAPES.items()}
    p["W1"][0, 0], p["b1"][0] = 2.0, 9.0
    p["W1"][1, 1], p["b1"][1] = 3.0, -20.0
    p["b1"][2] = 1.0
    p["b1"][3] = -1.0
    p["W2"][0, 0], p["W2"][0, 1], p["b2"][0] = 1.0, 5.0, 10.0
    p["W2"][1, 0] = -1.0
    p["W2"][2, 2], p["W2"][2, 3], p["b2"][2] = 1.0, 1.0, 9.0
    p["W3"][0, 0] = 0.01
    p["W3"][1, 1], p["W3"][1, 2] = 1.0, 0.1
    p["b3"][2] = 0.25
    p["W3"][3, 0], p["b3"][3] = -0.02, 1.0
    return p


def exact_inputs():
    X = np.zeros((2, mlp.D_IN))
    X[0, 0], X[0, 1] = 0.5, 0.25
    X[1, 0], X[1, 1] = 0.0, 0.75
    X[0, mlp.D_HIST + 2] = 1.0   # C = 3
    X[1, mlp.D_HIST + 3] = 1.0   # C = 4
    return X


def exact_outputs():
    y = np.zeros((2, mlp.D_OUT))
    for r, f0 in enumerate((0.5, 0.0)):
        y[r, 0] = (2 * f0 + 19) / 100
        y[r, 1] = (8 + 2 * PHI1) / 10
        y[r, 2] = 0.25
        y[r, 3] = 1 - (2 * f0 + 19) / 50
    return y


def test_forward_of_a_hand_set_network_is_exact():
    y, _ = mlp.forward(exact_net(), exact_inputs())
    assert np.max(np.abs(y - exact_outputs())) <= 1e-14


def test_predicted_centers_of_the_hand_set_network():
    V = mlp.predict_centers(exact_net(), exact_inputs(), [3, 4])
    y = exact_outputs()
    assert np.allclose(V[0], 255.0 * np.array([0.2, 0.25, y[0, 1]]), rtol=0, atol=1e-12)
    assert np.allclose(V[1], 255.0 * np.array([0.19, 0.25, 1 - 0.38, y[1, 1]]), rtol=0, atol=1e-12)
    assert all(np.all(np.diff(v) > 0) for v in V)


def _forward_mutant(kind):
    """Copies of the oracle's forward pass with one composition mistake."""
    def fwd(p, X):
        z1 = X @ p["W1"].T + p["b1"]
        a1 = mlp.gelu(z1) if kind != "no_gelu_1" else z1
        W2 = p["W2"].T if kind == "W2_transposed" else p["W2"]
        z2 = a1 @ W2.T + (p["b2"] if kind != "bias_1_in_layer_2" else p["b1"])
        a2 = mlp.gelu(z2) if kind != "no_gelu_2" else z2
        if kind == "gelu_on_output":
            return mlp.gelu(a2 @ p["W3"].T + p["b3"])
        return a2 @ p["W3"].T + (p["b3"] if kind != "no_bias_3" else 0.0)
    return fwd


@pytest.mark.parametrize("kind", ["no_gelu_1", "no_gelu_2", "W2_transposed", "bias_1_in_layer_2",
                                  "gelu_on_output", "no_bias_3"])
def test_planted_forward_mistakes_are_caught(kind):
    y = _forward_mutant(kind)(exact_net(), exact_inputs())
    assert np.max(np.abs(y - exact_outputs())) > 1e-3


# ---------------------------------------------------------------------------
# Adam: the first two bias-corrected steps in closed form.
#   step 1: m_hat = g, v_hat = g^2       -> w moves by -lr g / (|g| + eps)
#   step 2 with g1 = 1, g2 = -1: m_hat = (0.09 - 0.1) / 0.19 = -1/19,
#          v_hat = (0.999 * 0.001 + 0.001) / (1 - 0.999^2) = 1
#                                         -> w moves by +lr / (19 (1 + eps))
#   step 2 with g1 = g2 = 2: m_hat = 2, v_hat = 4 -> w moves by -2 lr / (2 + eps)
# ---------------------------------------------------------------------------

def _grads(value):
    return {k: np.full(s, float(value)) for k, s in mlp.PARAM_SHAPES.items()}


def _two_steps(step_fn, g1, g2, lr):
    p0 = {k: np.full(s, 0.5) for k, s in mlp.PARAM_SHAPES.items()}
    z = mlp.zeros_like_params()
    p1, m, v = step_fn(p0, _grads(g1), z, mlp.zeros_like_params(), 1, lr)
    p2, _, _ = step_fn(p1, _grads(g2), m, v, 2, lr)
    return p0["b3"][0], p1["b3"][0], p2["b3"][0]


def test_adam_first_step_closed_form():
    lr = 1e-3
    for g in (3.0, -0.25, 1e-8):
        w0, w1, _ = _two_steps(mlp.adam_step, g, 0.0, lr)
        assert abs((w1 - w0) - (-lr * g / (abs(g) + 1e-8))) <= 1e-15
    w0, w1, _ = _two_steps(mlp.adam_step, 0.0, 0.0, lr)
    assert w1 == w0  # a zero gradient leaves the weight where it is


def test_adam_second_step_closed_form():
    lr = 1e-3
    _, w1, w2 = _two_steps(mlp.adam_step, 1.0, -1.0, lr)
    assert abs((w2 - w1) - lr / (19.0 * (1.0 + 1e-8))) <= 1e-15
    _, w1, w2 = _two_steps(mlp.adam_step, 2.0, 2.0, lr)
    assert abs((w2 - w1) - (-2.0 * lr / (2.0 + 1e-8))) <= 1e-15


def _adam_mutant(kind):
    def step(params, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        if kind == "betas_swapped":
            b1, b2 = b2, b1
        c1 = 1.0 - b1 ** t if kind != "no_bias_correction" else 1.0
        c2 = 1.0 - b2 ** t if kind != "no_bias_correction" else 1.0
        po, mo, vo = {}, {}, {}
        for k in mlp.PARAM_ORDER:
            g = grads[k]
            mk = b1 * m[k] + (1 - b1) * g
            vk = b2 * v[k] + (1 - b2) * g * g
            den = np.sqrt(vk / c2 + eps) if kind == "eps_inside_sqrt" else np.sqrt(vk / c2) + eps
            po[k] = params[k] - lr * (mk / c1) / den
            mo[k], vo[k] = mk, vk
        return po, mo, vo
    return step


@pytest.mark.parametrize("kind", ["no_bias_correction", "betas_swapped", "eps_inside_sqrt"])
def test_planted_adam_mistakes_are_caught(kind):
    lr = 1e-3
    bad = []
    for g in (3.0, 1e-8):
        w0, w1, _ = _two_steps(_adam_mutant(kind), g, 0.0, lr)
        bad.append(abs((w1 - w0) - (-lr * g / (abs(g) + 1e-8))) > 1e-9)
    _, w1, w2 = _two_steps(_adam_mutant(kind), 1.0, -1.0, lr)
    bad.append(abs((w2 - w1) - lr / (19.0 * (1.0 + 1e-8))) > 1e-9)
    assert any(bad)
