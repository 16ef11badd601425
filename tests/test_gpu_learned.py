"""What the trained router gains over the method without it.

Same data, same Bk-means centres, same home partitions. The method of Section
3.2 probes a fixed number P of nearest centres per point; the cheapest P whose
graph reaches tie-aware recall@k >= 0.95 against exact brute-force rows
(bdg_knn_rows) is its operating point. The router scores each point's 8
nearest centres and keeps those within theta of its best logit (a variable
number of probes); theta is calibrated on held-out rows with known exact
neighbours, never on the judge's rows. At equal recall (>= 0.95 on the judge)
the learned routes must need clearly less Reduce-1 work (pairs = sum over
partitions of |V_p| |H_p|) than the fixed-P operating point. Training must fit:
the trained router's shortlist loss on its training rows is below the untrained
prior's. The exact rows themselves are checked against the CPU oracle on a few
points."""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bdg():
    from paper_2102_04656_b300 import build as b
    b.build()
    import paper_2102_04656_b300 as m
    m.lib()
    return m


def _recall(g, exact_d, rows):
    gd = g.dists[rows.long()]
    dk = exact_d[:, -1:]
    below = (gd < dk).sum(1)
    at = torch.minimum((gd == dk).sum(1), (exact_d == dk).sum(1))
    return float((below + at).sum().item()) / exact_d.numel()


def _pairs(routes, m):
    probes = routes >= 0
    hc = torch.bincount(routes[:, 0].long(), minlength=m).double()
    vc = torch.bincount(routes[probes].long(), minlength=m).double()
    return float((hc * vc).sum().item())


def test_learned_router_gains_over_fixed_nearest_centre_probes(bdg):
    from paper_2102_04656_b300 import learned
    spec = datagen.MixtureSpec(200_000, 128, 512, 256, seed=777)
    codes, feats = datagen.make_codes(spec, device="cuda", with_features=True)
    n, k, m, Q = spec.n, 32, 128, 8
    sample = torch.from_numpy(datagen.sample_ids(n, 64 * m, spec.seed + 3)).cuda()
    entry = torch.from_numpy(datagen.sample_ids(n, 256, spec.seed + 4).astype(np.int32)).cuda()
    cent, _ = bdg.bkmeans(codes, sample, m, 8)
    cand, cdist = bdg.route(codes, cent, Q)
    home = cand[:, 0].contiguous()
    xb = feats.to(torch.bfloat16).contiguous()

    # training rows and held-out rows: exact neighbours over all points
    S, V = 40_000, 8_000
    rows_tv = torch.from_numpy(datagen.sample_ids(n, S + V, spec.seed + 5)).cuda()
    tr, va = rows_tv[:S], rows_tv[S:]
    labels = learned.neighbour_labels_full(codes, tr.to(torch.int32), home, k, skip_home=False)
    base = torch.from_numpy(datagen.router_init(128, 256, 256, m, spec.seed + 5)).cuda()
    a = 0.25
    init = learned.prior_params(base, 128, 256, 256, m, cent, scale=a)
    cfg = learned.TrainConfig(hidden=(256, 256), batch=2048, epochs=6, lr=1e-3)
    prior_loss = learned.prior_scale_loss(xb[tr].contiguous(), codes[tr].contiguous(),
                                          cand[tr].contiguous(), labels, m, base, cent, (a,),
                                          hidden=(256, 256), batch=2048)[a]
    router = learned.train_router_shortlist(xb[tr].contiguous(), codes[tr].contiguous(),
                                            cand[tr].contiguous(), labels, m, init, cfg,
                                            seed=spec.seed + 5)
    fit = float(router.train_step_shortlist(xb[tr[:2048]].contiguous(),
                                            cand[tr[:2048]].contiguous(), labels[:2048],
                                            0.0, apply_update=False,
                                            codes=codes[tr[:2048]].contiguous()).item())
    assert fit < prior_loss, (fit, prior_loss)

    # calibration on the held-out rows (neighbour lists 16 beyond k)
    va_ids, va_d = bdg.knn_rows(codes, va.to(torch.int32).contiguous(), k + 16)
    xv, cv, qv = xb[va].contiguous(), codes[va].contiguous(), cand[va].contiguous()
    theta, _, _ = learned.calibrate(
        lambda th: router.route_shortlist(xv, qv, th, Q, codes=cv),
        [round(0.05 * i, 2) for i in range(0, 201)],
        lambda r: learned.tie_aware_recall(r, va_ids, va_d, home, k), 0.955)

    # the judge: other rows, exact over all points; checked against the CPU oracle
    rows = torch.from_numpy(datagen.sample_ids(n, 3000, spec.seed + 9).astype(np.int32)).cuda()
    ex_ids, ex_d = bdg.knn_rows(codes, rows, k)
    few = rows[:20].cpu().numpy().astype(np.int64)
    o_ids, o_d = oracle.knn_exact(codes.cpu().numpy().view(np.uint64), k, few)
    assert np.array_equal(ex_ids[:20].cpu().numpy(), o_ids)

    fixed = {}
    for P in (2, 3, 4, 5):
        r = cand[:, :P].contiguous()
        g = bdg.build_graph(codes, k, m=m, t=P, routes=r, entry=entry)
        fixed[P] = (_recall(g, ex_d, rows), _pairs(r, m))
        g.free()
    ok = [P for P in fixed if fixed[P][0] >= 0.95]
    assert ok, fixed
    P_best = min(ok)
    lr_routes = router.route_shortlist(xb, cand, theta, Q, codes=codes)
    assert torch.equal(lr_routes[:, 0], home)
    g = bdg.build_graph(codes, k, m=m, t=Q, routes=lr_routes, entry=entry)
    rec_ln, pairs_ln = _recall(g, ex_d, rows), _pairs(lr_routes, m)
    g.free()
    print("fixed P (recall, pairs):", fixed, "learned:", rec_ln, pairs_ln, "theta", theta)
    assert rec_ln >= 0.95, (rec_ln, fixed)
    assert pairs_ln <= 0.85 * fixed[P_best][1], (pairs_ln, P_best, fixed)
