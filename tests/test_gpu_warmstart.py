"""The warm-start network on the GPU against its FP64 oracle, and what it
gains over the plain cold start (needs a GPU).

Parameters are drawn here (seeded numpy), set into the library, and given to
the oracle with the weight matrices rounded to BF16 as the library uses them
(biases stay FP32); nothing the oracle sees comes from the CUDA path.
"""
import os

import numpy as np
import pytest

import oracle
import phantom
from oracle import mlp
from parity import eps32

pytestmark = pytest.mark.gpu

TRAIN_OFFSET = 1_000_000


@pytest.fixture(scope="module")
def fcm():
    from paper_1601_00072_gb300 import _build
    _build.build()
    from paper_1601_00072_gb300.fcm import FCM
    h = FCM(0)
    yield h
    h.close()


def _cuda(a, dtype=np.float32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def bf16(a):
    """FP32 values rounded to BF16 (round to nearest even), as FP64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def random_params(seed, scale=0.15):
    g = np.random.default_rng(seed)
    return (scale * g.standard_normal(mlp.N_PARAMS)).astype(np.float32)


def oracle_params(p32):
    p = mlp.unflat(p32.astype(np.float64))
    for k in ("W1", "W2", "W3"):
        p[k] = bf16(p[k])
    return p


def batch_slices(indices):
    from paper_1601_00072_gb300.fcm import Slice
    out, host = [], []
    for i in indices:
        sp, img, _ = phantom.batch_slice(i)
        x = img.reshape(-1)
        u0 = phantom.dirichlet_u0((phantom.U0_FAMILY, i), sp.C, x.size)
        out.append(Slice(x=_cuda(x), C=sp.C, U0=_cuda(u0)))
        host.append((x, u0, sp.C))
    return out, host


def test_features_match_oracle(fcm):
    slices, host = batch_slices(range(8))
    F = fcm.features(slices).cpu().numpy()
    for k, (x, _, C) in enumerate(host):
        assert np.max(np.abs(F[k] - mlp.features(x, C))) <= 1e-7


def test_forward_matches_oracle(fcm):
    slices, host = batch_slices(range(16))
    p32 = random_params(1)
    fcm.set_model_params(p32)
    y = fcm.model_forward(fcm.features(slices)).cpu().numpy()
    X = np.stack([mlp.features(x, C) for x, _, C in host])
    yo, _ = mlp.forward(oracle_params(p32), X)
    assert np.max(np.abs(y - yo)) <= 1e-4 * (1.0 + np.max(np.abs(yo)))


def test_gradients_match_oracle(fcm):
    slices, host = batch_slices(range(24))
    p32 = random_params(2, scale=0.3)
    fcm.set_model_params(p32)
    g = np.random.default_rng(3)
    Cs = np.array([C for _, _, C in host], dtype=np.int32)
    T = g.uniform(0, 1, (len(host), 8)).astype(np.float32)
    loss, grad = fcm.model_loss_grad(fcm.features(slices), _cuda(T), _cuda(Cs, np.int32))
    X = np.stack([mlp.features(x, C) for x, _, C in host])
    lo, go = mlp.loss_and_grads(oracle_params(p32), X, T.astype(np.float64), Cs)
    assert abs(loss - lo) <= 1e-5 * max(1.0, lo)
    gg = mlp.unflat(grad.astype(np.float64))
    for k in mlp.PARAM_ORDER:
        rel = np.linalg.norm(gg[k] - go[k]) / max(1e-12, np.linalg.norm(go[k]))
        assert rel <= 1e-3, (k, rel)


def test_save_and_load_round_trip(fcm, tmp_path):
    fcm.model_init(11)
    a = fcm.model_params()
    path = tmp_path / "m.fcmw"
    fcm.model_save(str(path))
    fcm.model_init(12)
    assert not np.array_equal(fcm.model_params(), a)
    fcm.model_load(str(path))
    assert np.array_equal(fcm.model_params(), a)


def _gain(fcm, slices_cold, slices_warm):
    """Iterations of warm versus cold runs of the same slices and which warm
    runs pass the acceptance rule."""
    from paper_1601_00072_gb300 import warmstart
    fcm.run_batched(slices_cold)
    st, n_cold = fcm.run_batched_warm(slices_warm)
    cold_it = np.array([s.iters for s in slices_cold])
    warm_it = np.array([s.iters for s in slices_warm])
    return cold_it, warm_it, warmstart.accepted(slices_cold, slices_warm), n_cold


def _oracle_starts(i, starts):
    """Sorted converged centers and final J of the FP64 oracle from each
    seeded random start of generator slice i."""
    from paper_1601_00072_gb300 import warmstart
    sp, img, _ = phantom.batch_slice(i)
    x = img.reshape(-1)
    out = []
    for s in range(starts):
        u0 = phantom.dirichlet_u0(warmstart.u0_key(i, s), sp.C, x.size)
        o = oracle.fcm_quantized(x, sp.C, 2.0, eps32(1e-5), 300, U0=u0)
        out.append((np.sort(o["V"]), o["J"][-1]))
    return out


def test_training_on_the_gpu_saves_iterations(fcm):
    """Train a fresh network on 2048 generated slices (labels: the best of
    four cold starts of the library's FCM), then compare warm and cold starts
    on 128 slices of the batch workload, which training never saw."""
    from paper_1601_00072_gb300 import warmstart
    F, T, Cs, its = warmstart.labelled_set(fcm, range(TRAIN_OFFSET, TRAIN_OFFSET + 2048))
    # sampled labels against the oracle run from the same four starts: each
    # label is one of the oracle's converged solutions, nearly always its best
    best = 0
    for k in range(0, 2048, 128):
        sols = _oracle_starts(TRAIN_OFFSET + k, warmstart.STARTS)
        C = int(Cs[k])
        t = T[k, :C].cpu().numpy().astype(np.float64) * 255.0
        err = [np.max(np.abs(t - v) / np.maximum(v, 1.0)) for v, _ in sols]
        assert min(err) <= 1e-4, (k, err)
        Jmin = min(J for _, J in sols)
        best += any(e <= 1e-4 and J <= Jmin * (1 + 1e-5) for e, (_, J) in zip(err, sols))
    assert best >= 14, best
    fcm.model_init(0)
    l0, _ = fcm.model_loss_grad(F[:256], T[:256], Cs[:256])
    loss = fcm.model_train(F, T, Cs, epochs=120, batch=256, lr=2e-3, seed=0)
    assert loss < 0.2 * l0, (l0, loss)
    cold, _ = batch_slices(range(128))
    warm, _ = batch_slices(range(128))
    cold_it, warm_it, ok, n_cold = _gain(fcm, cold, warm)
    print(f"\ncold mean iters {cold_it.mean():.1f}, warm {warm_it.mean():.1f}, "
          f"accepted {ok.mean():.3f}, ran cold {n_cold}")
    assert warm_it.mean() < 0.85 * cold_it.mean()
    assert ok.mean() >= 0.85


@pytest.mark.skipif(not os.path.exists(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                                    "paper_1601_00072_gb300", "data", "warmstart.fcmw")),
                    reason="no trained model file")
def test_shipped_model_saves_iterations_on_the_batch(fcm):
    from paper_1601_00072_gb300 import warmstart
    fcm.model_load(warmstart.MODEL_PATH)
    cold, _ = batch_slices(range(512))
    warm, _ = batch_slices(range(512))
    cold_it, warm_it, ok, n_cold = _gain(fcm, cold, warm)
    print(f"\ncold mean iters {cold_it.mean():.1f}, warm {warm_it.mean():.1f}, "
          f"accepted {ok.mean():.3f}, ran cold {n_cold}")
    assert warm_it.mean() < 0.8 * cold_it.mean()
    assert ok.mean() >= 0.93


def test_unusable_predictions_fall_back_to_cold_start(fcm):
    p = np.zeros(mlp.N_PARAMS, dtype=np.float32)
    p[-8:] = 0.5  # every output 0.5: all predicted centers coincide
    fcm.set_model_params(p)
    cold, _ = batch_slices(range(8))
    warm, _ = batch_slices(range(8))
    fcm.run_batched(cold, tune=False)
    st, n_cold = fcm.run_batched_warm(warm, tune=False)
    assert n_cold == 8 and all(s.init == "U" for s in warm)
    for c, w in zip(cold, warm):
        assert c.iters == w.iters
        assert np.allclose(c.V.cpu().numpy(), w.V.cpu().numpy(), rtol=1e-6, atol=1e-5)
