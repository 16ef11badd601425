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


def test_code_input_gradients_match_finite_differences():
    rng = np.random.default_rng(5)
    p = _params(rng)
    cb = 3
    p["W3"] = rng.standard_normal((4, 5 + cb)) * 0.5
    x = rng.standard_normal((6, 6))
    s = np.where(rng.random((6, cb)) < 0.5, 1.0, -1.0)
    q = rng.random((6, 4))
    q /= q.sum(1, keepdims=True)
    _, g, _ = mlp.loss_and_grads(p, x, q, bf16=False, s=s)
    eps = 1e-6
    for name, w in p.items():
        flat = w.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 8)):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = mlp.loss_and_grads(p, x, q, bf16=False, s=s)
            flat[idx] = old - eps
            lm, _, _ = mlp.loss_and_grads(p, x, q, bf16=False, s=s)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), name


def test_prior_weights_give_nearest_centre_routing(oracle_lib):
    """W3 = [0 | c_p / 2], b3 = 0: logits are bits/2 - Hamming distance (checked by a
    per-bit loop), and their top-t by (-z, p) is the C oracle's nearest-centre route."""
    rng = np.random.default_rng(6)
    n, m, bits, h = 40, 24, 128, 8
    codes = rng.integers(0, 2**63, size=(n, bits // 64), dtype=np.int64).view(np.uint64)
    cent = rng.integers(0, 2**63, size=(m, bits // 64), dtype=np.int64).view(np.uint64)
    cent[5] = cent[9]  # duplicate centres: equal logits, order by index
    s, cs = mlp.code_pm(codes, bits), mlp.code_pm(cent, bits)
    p = _params(rng, d_in=6, h=h, m=m)
    p["W3"] = np.concatenate([np.zeros((m, h)), cs / 2], axis=1)
    p["b3"] = np.zeros(m)
    z, _ = mlp.forward(p, rng.standard_normal((n, 6)), bf16=True, s=s)
    for i in range(0, n, 7):
        for c in range(m):
            d = sum(((int(codes[i, b // 64]) >> (b % 64)) & 1) != ((int(cent[c, b // 64]) >> (b % 64)) & 1)
                    for b in range(bits))
            assert z[i, c] == bits / 2 - d
    routes, _ = oracle_lib.route(codes, cent, 5)
    assert np.array_equal(mlp.topp(z, 5), routes)


def test_excluded_partition_is_left_out_of_the_softmax():
    """Leaving partition e out equals the plain loss of the network whose logit e
    is removed: checked against a hand-built softmax over the other columns and
    by finite differences."""
    rng = np.random.default_rng(7)
    p = _params(rng, m=5)
    x = rng.standard_normal((4, 6))
    ex = np.array([0, 3, 3, 1])
    lab = np.array([[0, 1, 2], [3, 3, 4], [1, -1, 3], [0, 2, 2]])
    q = mlp.label_targets(lab, 5, exclude=ex)
    assert np.allclose(q[1], [0, 0, 0, 0, 1]) and np.allclose(q[2], [0, 1, 0, 0, 0])
    loss, g, z = mlp.loss_and_grads(p, x, q, bf16=False, exclude=ex)
    want = 0.0
    for i in range(4):
        keep = [c for c in range(5) if c != ex[i]]
        lse = np.log(np.exp(z[i, keep]).sum())
        want -= sum(q[i, c] * (z[i, c] - lse) for c in keep)
    assert abs(loss - want / 4) < 1e-12
    eps = 1e-6
    for name in ("W3", "b3", "W1"):
        flat = p[name].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 5)):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = mlp.loss_and_grads(p, x, q, bf16=False, exclude=ex)
            flat[idx] = old - eps
            lm, _, _ = mlp.loss_and_grads(p, x, q, bf16=False, exclude=ex)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), name


# ---------------------------------------------------------------- shortlist head
def _params_code(rng, d_in=6, h=5, m=9, cb=64, scale=0.5):
    p = _params(rng, d_in, h, m, scale)
    p["W3"] = rng.standard_normal((m, h + cb)) * scale
    return p


def test_shortlist_gradients_match_finite_differences():
    rng = np.random.default_rng(10)
    p = _params_code(rng)
    B, Q, m = 6, 4, 9
    x = rng.standard_normal((B, 6))
    s = np.where(rng.random((B, 64)) < 0.5, 1.0, -1.0)
    cand = np.array([rng.permutation(m)[:Q] for _ in range(B)])
    cand[1, 3] = -1
    cand[4, 2:] = -1
    q = rng.random((B, Q)) * (cand >= 0)
    q[2] = 0.0  # a row without target
    q /= np.maximum(q.sum(1, keepdims=True), 1e-300)
    _, g, _ = mlp.shortlist_loss_and_grads(p, x, cand, q, bf16=False, s=s)
    eps = 1e-6
    for name, w in p.items():
        flat = w.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 9)):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _, _ = mlp.shortlist_loss_and_grads(p, x, cand, q, bf16=False, s=s)
            flat[idx] = old - eps
            lm, _, _ = mlp.shortlist_loss_and_grads(p, x, cand, q, bf16=False, s=s)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), name


def test_shortlist_of_every_partition_is_the_dense_softmax():
    """With every partition shortlisted (in index order) the shortlist head is the
    full softmax cross-entropy over all m logits: loss, gradients and logits equal
    the dense forms (which the finite-difference pin above checks)."""
    rng = np.random.default_rng(11)
    m, B = 7, 5
    p = _params_code(rng, m=m, cb=64)
    x = rng.standard_normal((B, 6))
    s = np.where(rng.random((B, 64)) < 0.5, 1.0, -1.0)
    labels = rng.integers(-1, m, size=(B, 6))
    cand = np.tile(np.arange(m), (B, 1))
    qs = mlp.shortlist_targets(labels, cand)
    qd = mlp.label_targets(labels, m)
    assert np.allclose(qs, qd)
    ls, gs, zs = mlp.shortlist_loss_and_grads(p, x, cand, qs, bf16=False, s=s)
    ld, gd, zd = mlp.loss_and_grads(p, x, qd, bf16=False, s=s)
    assert abs(ls - ld) < 1e-12
    assert np.allclose(zs, zd, rtol=0, atol=1e-12)
    for k in gd:
        assert np.allclose(gs[k], gd[k], rtol=0, atol=1e-12), k


def test_shortlist_targets_hand_worked():
    # row 0: labels 4, 4, 9 (9 not shortlisted) -> q = 1 on partition 4 (slot 1)
    # row 1: labels 3, 5, 5, 8 over shortlist [5, 3, 8] -> 2/4, 1/4, 1/4
    # row 2: no label shortlisted -> zero row
    labels = np.array([[4, 4, 9, -1], [3, 5, 5, 8], [1, 1, 2, 2]])
    cand = np.array([[7, 4, -1], [5, 3, 8], [6, 0, 3]])
    q = mlp.shortlist_targets(labels, cand)
    want = np.array([[0, 1, 0], [0.5, 0.25, 0.25], [0, 0, 0]])
    assert np.allclose(q, want)


def test_shortlist_select_hand_worked():
    z = np.array([[1.0, 3.0, 2.5, 0.0, 2.5]], np.float32)
    cand = np.array([[7, 2, 9, 4, 1]])
    # largest logit 3.0: with theta = 1 the threshold is 2.0; kept (by -z, then
    # partition): 2 (3.0), 1 (2.5), 9 (2.5); the home 7 is always slot 0
    assert mlp.shortlist_select(z, cand, 1.0, 4).tolist() == [[7, 2, 1, 9]]
    assert mlp.shortlist_select(z, cand, 1.0, 3).tolist() == [[7, 2, 1]]
    assert mlp.shortlist_select(z, cand, 0.4, 4).tolist() == [[7, 2, -1, -1]]
    assert mlp.shortlist_select(z, cand, 0.0, 2).tolist() == [[7, 2]]
    assert mlp.shortlist_select(z, cand, 10.0, 6).tolist() == [[7, 2, 1, 9, 4, -1]]
    # a missing candidate is never kept
    cand2 = np.array([[7, 2, -1, 4, 1]])
    assert mlp.shortlist_select(z, cand2, 10.0, 5).tolist() == [[7, 2, 1, 4, -1]]


def test_shortlist_prior_margin_rule_is_the_distance_gap_rule(oracle_lib):
    """With the prior weights at temperature a = 2^-3 (W3 = [0 | a (c_p - 1/2)],
    b3 = 0) the shortlisted logits are a (bits/2 - d(y, c_p)), and keeping the
    partitions within theta = a (delta + 1/2) of the largest logit keeps exactly
    the shortlisted centres within delta of the nearest one: checked against the C
    oracle's routes and distances."""
    import datagen
    rng = np.random.default_rng(12)
    bits, m, n, Q, h = 128, 40, 300, 8, 5
    codes = datagen.random_codes(n, bits, seed=5).numpy().view(np.uint64)
    cent = datagen.random_codes(m, bits, seed=6).numpy().view(np.uint64)
    r, d = oracle_lib.route(codes, cent, Q)
    a = 0.125
    p = _params(rng, 6, h, m)
    p["W3"] = np.concatenate([np.zeros((m, h)), a * (mlp.code_pm(cent, bits) / 2.0)], axis=1)
    p["b3"] = np.zeros(m)
    x = rng.standard_normal((n, 6))
    s = mlp.code_pm(codes, bits)
    z, _ = mlp.shortlist_forward(p, x, r, bf16=True, s=s)
    assert np.array_equal(z, a * (bits / 2.0 - d))
    for delta, pmax in ((0, 4), (3, 8), (6, 5)):
        sel = mlp.shortlist_select(z.astype(np.float32), r, a * (delta + 0.5), pmax)
        for i in range(n):
            want = [int(r[i, 0])] + [int(r[i, j]) for j in range(1, Q)
                                     if d[i, j] - d[i, 0] <= delta][:pmax - 1]
            want += [-1] * (pmax - len(want))
            assert sel[i].tolist() == want
