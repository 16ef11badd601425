"""GPU parity of the learned router: the tcgen05 BF16 GEMM against float64
matrix products, and the network's forward pass, loss, gradients, Adam step and
top-P routing against the float64 oracle (oracle.mlp) on bf16-rounded inputs.

Tolerances: the GPU accumulates in FP32 and rounds hidden activations to BF16
where the oracle rounds its float64 values, so an element near a BF16 rounding
boundary may differ by one BF16 ulp (2^-8 relative). Logits: max error <= 1e-2
of the largest logit; gradients: relative Frobenius error <= 2e-2 per tensor;
GEMM outputs: 1e-5 relative to the output's scale (FP32 accumulation)."""
import numpy as np
import pytest
import torch

import datagen
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bdg():
    from paper_2102_04656_b300 import build as b
    b.build()
    import paper_2102_04656_b300 as m
    m.lib()
    return m


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 136), (7, 1000, 512),
                                   (1000, 40, 10000), (129, 257, 8)])
def test_gemm_matches_float64(bdg, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = _bf16(rng.standard_normal((M, K)))
    B = _bf16(rng.standard_normal((N, K)))
    C, err = bdg.gemm_bf16(A.cuda(), B.cuda())
    ref = A.double().numpy() @ B.double().numpy().T
    scale = np.abs(ref).max() + 1e-30
    assert int(err.item()) == 0
    assert np.abs(C.cpu().numpy() - ref).max() <= 1e-5 * scale * max(1.0, np.sqrt(K / 64))


def test_gemm_epilogues(bdg):
    rng = np.random.default_rng(5)
    M, N, K = 200, 150, 96
    A = _bf16(rng.standard_normal((M, K)))
    B = _bf16(rng.standard_normal((N, K)))
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32))
    mask = _bf16(rng.standard_normal((M, N)))
    ref = A.double().numpy() @ B.double().numpy().T
    # bias + relu, bf16 out
    Cb, _ = bdg.gemm_bf16(A.cuda(), B.cuda(), bias=bias.cuda(), relu=True, out="bf16")
    want = np.maximum(ref + bias.double().numpy(), 0)
    assert np.allclose(Cb.float().cpu().numpy(), want, rtol=2 ** -7, atol=1e-4)
    # mask (relu derivative) + column sums
    cs = torch.zeros(N, dtype=torch.float32, device="cuda")
    Cm, _ = bdg.gemm_bf16(A.cuda(), B.cuda(), mask=mask.cuda(), colsum=cs)
    wantm = ref * (mask.double().numpy() > 0)
    assert np.abs(Cm.cpu().numpy() - wantm).max() <= 1e-5 * np.abs(ref).max()
    assert np.allclose(cs.cpu().numpy(), wantm.sum(0), rtol=1e-4, atol=1e-3)


@pytest.mark.parametrize("relu", [True, False])
def test_gemm_whole_tile_bias_bf16_epilogue(bdg, relu):
    """Whole-tile shapes with bias and BF16 output take the direct epilogue
    (each thread stores its own row)."""
    rng = np.random.default_rng(9)
    M, N, K = 384, 256, 200
    A = _bf16(rng.standard_normal((M, K)))
    B = _bf16(rng.standard_normal((N, K)))
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32))
    Cb, err = bdg.gemm_bf16(A.cuda(), B.cuda(), bias=bias.cuda(), relu=relu, out="bf16")
    want = A.double().numpy() @ B.double().numpy().T + bias.double().numpy()
    if relu:
        want = np.maximum(want, 0)
    assert int(err.item()) == 0
    assert np.allclose(Cb.float().cpu().numpy(), want, rtol=2 ** -7, atol=1e-3)


def _net(seed, d=128, h1=64, h2=64, m=40):
    flat = datagen.router_init(d, h1, h2, m, seed)
    o = np.cumsum([0, h1 * d, h1, h2 * h1, h2, m * h2, m])
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    shapes = [(h1, d), (h1,), (h2, h1), (h2,), (m, h2), (m,)]
    params = {n: flat[o[i]:o[i + 1]].reshape(s).astype(np.float64)
              for i, (n, s) in enumerate(zip(names, shapes))}
    return flat, params


def _batch(B, d, m, kt, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, d)).astype(np.float32)
    lab = rng.integers(-1, m, (B, kt)).astype(np.int32)  # -1 entries are ignored
    lab[::17] = -1  # rows without any target
    return x, lab


def _q(lab, m):
    return omlp.label_targets(lab, m)


def test_router_forward_loss_and_gradients(bdg):
    d, h1, h2, m, B, kt = 128, 64, 64, 40, 256, 16
    flat, params = _net(11, d, h1, h2, m)
    r = bdg.Router(torch.from_numpy(flat).cuda(), d, h1, h2, m, max_batch=512)
    x, lab = _batch(B, d, m, kt, 3)
    xb = _bf16(x).cuda()
    z = r.forward(xb).cpu().numpy()
    z_o, _ = omlp.forward(params, x, bf16=True)
    assert np.abs(z - z_o).max() <= 1e-2 * np.abs(z_o).max()
    r.train_step(xb, torch.from_numpy(lab).cuda(), lr=0.0, apply_update=False)
    torch.cuda.synchronize()
    loss_o, g_o, _ = omlp.loss_and_grads(params, x, _q(lab, m), bf16=True)
    assert abs(float(r.loss.item()) - loss_o) <= 1e-3 * abs(loss_o)
    g = r.unpack(r.grads.cpu())
    for name in ["W1", "b1", "W2", "b2", "W3", "b3"]:
        a, b_ = g[name].double().numpy(), g_o[name]
        rel = np.linalg.norm(a - b_) / (np.linalg.norm(b_) + 1e-30)
        assert rel <= 2e-2, (name, rel)
    assert int(r.err.item()) == 0


def test_router_adam_step_and_training_lowers_loss(bdg):
    d, h1, h2, m, B, kt = 64, 32, 32, 24, 128, 8
    flat, params = _net(12, d, h1, h2, m)
    r = bdg.Router(torch.from_numpy(flat).cuda(), d, h1, h2, m, max_batch=128)
    x, lab = _batch(B, d, m, kt, 4)
    xb, lb = _bf16(x).cuda(), torch.from_numpy(lab).cuda()
    r.train_step(xb, lb, lr=1e-3, apply_update=True)
    torch.cuda.synchronize()
    _, g_o, _ = omlp.loss_and_grads(params, x, _q(lab, m), bf16=True)
    new_o, _ = omlp.adam(params, g_o, {}, lr=1e-3)
    new = r.unpack(r.params.cpu())
    for name in new_o:
        # one Adam step moves each weight by about lr * sign(g); compare the moves
        step_gpu = new[name].double().numpy() - params[name]
        step_o = new_o[name] - params[name]
        agree = np.mean(np.abs(step_gpu - step_o) <= 2e-4 + 0.05 * np.abs(step_o))
        assert agree >= 0.97, (name, agree)
    losses = []
    for _ in range(60):
        losses.append(float(r.train_step(xb, lb, lr=3e-3).item()))
    assert losses[-1] < 0.9 * losses[0]  # random targets: the loss falls, slowly


def test_router_route_top_p(bdg):
    d, h1, h2, m, N, P = 128, 64, 64, 48, 1000, 5
    flat, params = _net(13, d, h1, h2, m)
    r = bdg.Router(torch.from_numpy(flat).cuda(), d, h1, h2, m, max_batch=256)  # 4 chunks
    x = np.random.default_rng(6).standard_normal((N, d)).astype(np.float32)
    home = np.random.default_rng(7).integers(0, m, N).astype(np.int32)
    routes = r.route(_bf16(x).cuda(), torch.from_numpy(home).cuda(), P).cpu().numpy()
    z_o, _ = omlp.forward(params, x, bf16=True)
    assert (routes[:, 0] == home).all()
    for i in range(N):
        zz = z_o[i].copy()
        zz[home[i]] = -np.inf
        want = omlp.topp(zz[None, :], P - 1)[0]
        got = routes[i, 1:]
        assert len(set(got.tolist())) == P - 1 and home[i] not in set(got.tolist())
        if not np.array_equal(got, want):
            # a different pick is only allowed among near-ties of the float64 logits
            kth = np.sort(zz)[::-1][P - 2]
            tol = 1e-2 * np.abs(z_o[i]).max()
            assert np.all(zz[got] >= kth - tol)


def _rand_codes(n, bits, seed):
    c = datagen.random_codes(n, bits, seed)
    return c, c.numpy().view(np.uint64)


def test_router_code_input_forward_and_gradients(bdg):
    """Last layer over [h2 | code as +-1], one partition per row left out of the
    softmax: forward, loss and gradients against the oracle."""
    d, h1, h2, m, B, kt, bits = 64, 32, 48, 40, 256, 12, 128
    flat, params = _net(21, d, h1, h2, m)
    rng = np.random.default_rng(22)
    params["W3"] = rng.uniform(-0.1, 0.1, (m, h2 + bits))
    o = np.cumsum([0, h1 * d, h1, h2 * h1, h2])
    flat = np.concatenate([flat[:o[-1]], params["W3"].reshape(-1), params["b3"]]).astype(np.float32)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):  # the oracle sees the fp32 values
        params[k] = params[k].astype(np.float32).astype(np.float64)
    r = bdg.Router(torch.from_numpy(flat).cuda(), d, h1, h2, m, max_batch=256, code_bits=bits)
    x, lab = _batch(B, d, m, kt, 23)
    ct, cu = _rand_codes(B, bits, 24)
    s = omlp.code_pm(cu, bits)
    xb, cd = _bf16(x).cuda(), ct.cuda()
    z = r.forward(xb, codes=cd).cpu().numpy()
    z_o, _ = omlp.forward(params, x, bf16=True, s=s)
    assert np.abs(z - z_o).max() <= 1e-2 * np.abs(z_o).max()
    ex = np.random.default_rng(25).integers(0, m, B).astype(np.int32)
    lab[::5, 0] = ex[::5]  # labels naming the left-out partition are ignored
    r.train_step(xb, torch.from_numpy(lab).cuda(), lr=0.0, apply_update=False, codes=cd,
                 exclude=torch.from_numpy(ex).cuda())
    torch.cuda.synchronize()
    loss_o, g_o, _ = omlp.loss_and_grads(params, x, omlp.label_targets(lab, m, exclude=ex),
                                         bf16=True, s=s, exclude=ex)
    assert abs(float(r.loss.item()) - loss_o) <= 1e-3 * abs(loss_o)
    g = r.unpack(r.grads.cpu())
    for name in ["W1", "b1", "W2", "b2", "W3", "b3"]:
        a, b_ = g[name].double().numpy(), g_o[name]
        rel = np.linalg.norm(a - b_) / (np.linalg.norm(b_) + 1e-30)
        assert rel <= 2e-2, (name, rel)
    assert int(r.err.item()) == 0


def test_prior_router_routes_like_nearest_centres(bdg):
    """Untrained router with prior_params: its routes equal the oracle's
    nearest-centre routes exactly (home = nearest centre, then by (d, c))."""
    import oracle
    from paper_2102_04656_b300 import learned
    d, h1, h2, m, N, P, bits = 64, 32, 32, 96, 3000, 6, 256
    flat, _ = _net(31, d, h1, h2, m)
    ct, cu = _rand_codes(N, bits, 32)
    cent_t, cent_u = _rand_codes(m, bits, 33)
    cent_t[7] = cent_t[50]  # duplicate centres: ties broken by index
    cent_u = cent_t.numpy().view(np.uint64)
    init = learned.prior_params(torch.from_numpy(flat).cuda(), d, h1, h2, m, cent_t.cuda())
    r = bdg.Router(init, d, h1, h2, m, max_batch=1024, code_bits=bits)  # 3 chunks
    want, _ = oracle.route(cu, cent_u, P)
    x = _bf16(np.random.default_rng(34).standard_normal((N, d))).cuda()
    got = learned.learned_routes(r, x, torch.from_numpy(want[:, 0].copy()).cuda(), P,
                                 codes=ct.cuda()).cpu().numpy()
    assert np.array_equal(got, want)


# ---------------------------------------------------------------- shortlist head
def _code_net(seed, d, h1, h2, m, bits):
    flat, params = _net(seed, d, h1, h2, m)
    rng = np.random.default_rng(seed + 1)
    params["W3"] = rng.uniform(-0.1, 0.1, (m, h2 + bits))
    params["b3"] = rng.uniform(-0.2, 0.2, m)
    o = np.cumsum([0, h1 * d, h1, h2 * h1, h2])
    flat = np.concatenate([flat[:o[-1]], params["W3"].reshape(-1), params["b3"]]).astype(np.float32)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):  # the oracle sees the fp32 values
        params[k] = params[k].astype(np.float32).astype(np.float64)
    return flat, params


def _shortlist(B, m, Q, seed, holes=True):
    rng = np.random.default_rng(seed)
    cand = np.stack([rng.permutation(m)[:Q] for _ in range(B)]).astype(np.int32)
    if holes:
        cand[::7, Q - 1] = -1
        cand[3::11, 2:] = -1
    return cand


def test_shortlist_forward_loss_and_gradients(bdg):
    """Shortlist head: logits, loss and gradients of every parameter against the
    float64 oracle, with missing candidates and rows without a shortlisted label."""
    d, h1, h2, m, B, kt, bits, Q = 64, 32, 48, 64, 256, 16, 128, 8
    flat, params = _code_net(41, d, h1, h2, m, bits)
    r = bdg.Router(torch.from_numpy(flat).cuda(), d, h1, h2, m, max_batch=256, code_bits=bits)
    x, lab = _batch(B, d, m, kt, 42)
    ct, cu = _rand_codes(B, bits, 43)
    s = omlp.code_pm(cu, bits)
    cand = _shortlist(B, m, Q, 44)
    lab[1::4, :3] = cand[1::4, :3]  # make sure many rows have shortlisted labels
    xb, cd, cn = _bf16(x).cuda(), ct.cuda(), torch.from_numpy(cand).cuda()
    z = r.forward_shortlist(xb, cn, codes=cd).cpu().numpy()
    z_o, _ = omlp.shortlist_forward(params, x, cand, bf16=True, s=s)
    fin = np.isfinite(z_o)
    assert np.array_equal(np.isfinite(z), fin)
    assert np.abs(z[fin] - z_o[fin]).max() <= 1e-2 * np.abs(z_o[fin]).max()
    r.train_step_shortlist(xb, cn, torch.from_numpy(lab).cuda(), lr=0.0, apply_update=False,
                           codes=cd)
    torch.cuda.synchronize()
    q = omlp.shortlist_targets(lab, cand)
    assert (q.sum(1) == 0).any() and (q.sum(1) > 0).sum() > B // 2
    loss_o, g_o, _ = omlp.shortlist_loss_and_grads(params, x, cand, q, bf16=True, s=s)
    assert abs(float(r.loss.item()) - loss_o) <= 1e-3 * abs(loss_o)
    g = r.unpack(r.grads.cpu())
    for name in ["W1", "b1", "W2", "b2", "W3", "b3"]:
        a, b_ = g[name].double().numpy(), g_o[name]
        rel = np.linalg.norm(a - b_) / (np.linalg.norm(b_) + 1e-30)
        assert rel <= 2e-2, (name, rel)
    assert int(r.err.item()) == 0


@pytest.mark.parametrize("theta,pmax", [(0.0, 4), (0.3, 8), (1.5, 5), (100.0, 8)])
def test_shortlist_route_choice_bit_exact(bdg, theta, pmax):
    """The probe choice of bdg_router_route_shortlist equals the oracle's rule
    applied to the kernel's own FP32 logits (the decision is taken in FP32 on
    both sides); the logits equal those of the forward entry point."""
    d, h1, h2, m, N, bits, Q = 64, 32, 32, 304, 3000, 256, 8
    flat, params = _code_net(51, d, h1, h2, m, bits)
    r = bdg.Router(torch.from_numpy(flat).cuda(), d, h1, h2, m, max_batch=512, code_bits=bits)
    x = _bf16(np.random.default_rng(52).standard_normal((N, d))).cuda()
    ct, _ = _rand_codes(N, bits, 53)
    cand = _shortlist(N, m, Q, 54)
    cn = torch.from_numpy(cand).cuda()
    routes, z = r.route_shortlist(x, cn, theta, pmax, codes=ct.cuda(), logits=True)
    z = z.cpu().numpy()
    want = omlp.shortlist_select(z, cand, theta, pmax)
    assert np.array_equal(routes.cpu().numpy(), want)
    z2 = r.forward_shortlist(x[:512], cn[:512], codes=ct[:512].cuda()).cpu().numpy()
    assert np.array_equal(z2, z[:512])
    # processing the points in another order (here a permutation) changes nothing
    perm = torch.from_numpy(np.random.default_rng(55).permutation(N).astype(np.int32)).cuda()
    routes_p, z_p = r.route_shortlist(x, cn, theta, pmax, codes=ct.cuda(), logits=True,
                                      order=perm)
    assert torch.equal(routes_p, routes)
    assert np.array_equal(z_p.cpu().numpy(), z)


def test_shortlist_prior_routes_by_distance_gap(bdg):
    """Untrained router with the prior at scale 1/8: the probe choice with theta =
    (delta + 1/2) / 8 keeps exactly the shortlisted centres within delta of the
    nearest one (distances from bdg_route, whose parity with the oracle is
    tested), in (d, c) order."""
    from paper_2102_04656_b300 import learned
    d, h1, h2, m, N, bits, Q = 64, 32, 32, 1104, 4000, 256, 8
    flat, _ = _net(61, d, h1, h2, m)
    c = datagen.make_codes(datagen.MixtureSpec(N, 64, 30, bits, seed=62)).cuda()
    cent = datagen.random_codes(m, bits, seed=63).cuda()
    cent[9] = cent[400]
    cand, rdist = bdg.route(c, cent, Q)
    a = 0.125
    init = learned.prior_params(torch.from_numpy(flat).cuda(), d, h1, h2, m, cent, scale=a)
    r = bdg.Router(init, d, h1, h2, m, max_batch=512, code_bits=bits)
    x = _bf16(np.random.default_rng(64).standard_normal((N, d))).cuda()
    gap = (rdist - rdist[:, :1]).cpu().numpy()
    cn = cand.cpu().numpy()
    for delta, pmax in ((0, 3), (2, 8), (5, 6)):
        got = r.route_shortlist(x, cand, a * (delta + 0.5), pmax, codes=c).cpu().numpy()
        for i in range(N):
            want = [int(cn[i, 0])] + [int(cn[i, j]) for j in range(1, Q)
                                      if gap[i, j] <= delta][:pmax - 1]
            want += [-1] * (pmax - len(want))
            assert got[i].tolist() == want, (i, delta)
