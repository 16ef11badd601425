"""Pins of the router oracle (oracle.mlp): finite differences of the float64
network, closed forms of softmax cross-entropy and of Adam's first step, and
bfloat16 rounding against torch's own conversion."""
import numpy as np
import torch

from oracle import mlp


def _params(rng, d_in=6, h=5, m=4, scale=0.5):
    return {
        "W1": rng.standard_normal((h, d_in)) * scale, "b1": rng.standard_normal(h) * 0.1,
        "W2": rng.standard_normal((h, h)) * scale, "b2": rng.standard_normal(h) * 0.1,
        "W3": rng.standard_normal((m, h)) * scale, "b3": rng.standard_normal(m) * 0.1,
    }


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    x = rng.standard_normal((7, 6))
    q = rng.random((7, 4))
    q /= q.sum(1, keepdims=True)
    _, g, _ = mlp.loss_and_grads(p, x, q, bf16=False)
    eps = 1e-6
    for name, w in p.items():
        flat = w.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 6)):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = mlp.loss_and_grads(p, x, q, bf16=False)
            flat[idx] = old - eps
            lm, _, _ = mlp.loss_and_grads(p, x, q, bf16=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), name


def test_one_hot_cross_entropy_is_negative_log_softmax():
    rng = np.random.default_rng(1)
    p = _params(rng)
    x = rng.standard_normal((3, 6))
    q = np.eye(4)[[0, 2, 3]]
    loss, _, z = mlp.loss_and_grads(p, x, q, bf16=False)
    want = np.mean([np.log(np.exp(z[i]).sum()) - z[i, c] for i, c in enumerate([0, 2, 3])])
    assert abs(loss - want) < 1e-12


def test_round_bf16_matches_torch():
    rng = np.random.default_rng(2)
    a = np.concatenate([rng.standard_normal(5000).astype(np.float32) * 10,
                        np.array([0.0, -0.0, 1.0, 65504.0, 1e-30, 3.0e38], np.float32)])
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert (mlp.round_bf16(a) == want).all()


def test_adam_first_step_is_signed_lr():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    newp, st = mlp.adam(p, g, {}, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step = lr * g / (|g| + eps)
    want = p["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(newp["w"], want, rtol=0, atol=1e-15)
    assert st["t"] == 1


def test_topp_tie_order_and_targets():
    z = np.array([[1.0, 3.0, 3.0, 0.0], [5.0, 5.0, 5.0, 5.0]])
    assert mlp.topp(z, 3).tolist() == [[1, 2, 0], [0, 1, 2]]
    home = np.array([0, 1, 1, 2, 0])
    q = mlp.neighbour_partition_targets(np.array([[1, 2, 3, -1]]), home, 3)
    assert np.allclose(q, [[0.0, 2 / 3, 1 / 3]])  # normalised over the 3 valid labels
    assert np.allclose(mlp.label_targets(np.array([[-1, -1], [2, 2]]), 3), [[0, 0, 0], [0, 0, 1]])


def test_rows_without_target_have_no_gradient():
    rng = np.random.default_rng(4)
    p = _params(rng)
    x = rng.standard_normal((3, 6))
    q = np.zeros((3, 4))
    q[1, 2] = 1.0
    loss, g, z = mlp.loss_and_grads(p, x, q, bf16=False)
    _, g1, _ = mlp.loss_and_grads(p, x[1:2], q[1:2], bf16=False)
    # the two target-less rows change nothing but the 1/B normalisation
    for name in g:
        assert np.allclose(g[name] * 3, g1[name], rtol=1e-12, atol=1e-14)
