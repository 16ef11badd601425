"""What the trained router gains over the method without it.

Same data, same Bk-means centres, same home partitions, same number P of probed
partitions per point: the divide-and-conquer graph built with the nearest-centre
probes of Section 3.2 against the graph built with the router's probes (home +
P - 1 learned picks). The router's last layer also takes the code as +-1 and
starts at the nearest-centre logits, so training starts from the method's own
routing. Recall@k of both is judged against exact brute-force rows
(bdg_knn_rows) on sampled points; the router must not lose recall, and it must
gain at the smaller P. The exact rows themselves are checked against the CPU
oracle on a few points."""
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


def _recall(g, exact_ids, exact_d, rows):
    gd = g.dists[rows.long()]
    dk = exact_d[:, -1:]
    below = (gd < dk).sum(1)
    at = torch.minimum((gd == dk).sum(1), (exact_d == dk).sum(1))
    return float((below + at).sum().item()) / exact_d.numel()


def test_learned_router_gains_over_nearest_centre_probes(bdg):
    from paper_2102_04656_b300 import learned
    spec = datagen.MixtureSpec(200_000, 128, 512, 256, seed=777)
    codes, feats = datagen.make_codes(spec, device="cuda", with_features=True)
    n, k, m = spec.n, 32, 128
    sample = torch.from_numpy(datagen.sample_ids(n, 64 * m, spec.seed + 3)).cuda()
    entry = torch.from_numpy(datagen.sample_ids(n, 256, spec.seed + 4).astype(np.int32)).cuda()
    cent, _ = bdg.bkmeans(codes, sample, m, 8)
    home = bdg.route(codes, cent, 1)[0][:, 0].contiguous()
    xb = feats.to(torch.bfloat16).contiguous()

    # training data: the exact neighbours (over all points) of a seeded sample,
    # their home partitions
    S = 40_000
    tr = torch.from_numpy(datagen.sample_ids(n, S, spec.seed + 5)).cuda()
    labels = learned.neighbour_labels_full(codes, tr.to(torch.int32), home, k)
    base = torch.from_numpy(datagen.router_init(128, 256, 256, m, spec.seed + 5)).cuda()
    init = learned.prior_params(base, 128, 256, 256, m, cent)
    cfg = learned.TrainConfig(hidden=(256, 256), batch=2048, epochs=6, lr=1e-3)
    losses = []
    router = learned.train_router(xb[tr].contiguous(), labels, m, init, cfg, seed=spec.seed + 5,
                                  log=lambda ep, l: losses.append(l), codes=codes[tr].contiguous(),
                                  home=home[tr].contiguous())
    assert losses[-1] < losses[0]

    # judge rows
    rows = torch.from_numpy(datagen.sample_ids(n, 2000, spec.seed + 9).astype(np.int32)).cuda()
    ex_ids, ex_d = bdg.knn_rows(codes, rows, k)
    # the judge agrees with the CPU oracle on a few rows
    few = rows[:20].cpu().numpy().astype(np.int64)
    o_ids, o_d = oracle.knn_exact(codes.cpu().numpy().view(np.uint64), k, few)
    assert np.array_equal(ex_ids[:20].cpu().numpy(), o_ids)

    res = {}
    for P in (2, 4):
        r_ex, _ = bdg.route(codes, cent, P)
        g_ex = bdg.build_graph(codes, k, m=m, t=P, routes=r_ex, entry=entry)
        r_ln = learned.learned_routes(router, xb, home, P, codes=codes)
        assert torch.equal(r_ln[:, 0], home)
        g_ln = bdg.build_graph(codes, k, m=m, t=P, routes=r_ln, entry=entry)
        res[P] = (_recall(g_ex, ex_ids, ex_d, rows), _recall(g_ln, ex_ids, ex_d, rows))
        g_ex.free()
        g_ln.free()
    print("recall exhaustive vs learned:", res)
    for P, (rec_ex, rec_ln) in res.items():
        assert rec_ln >= rec_ex - 0.002, (P, rec_ex, rec_ln)
    assert res[2][1] > res[2][0], res
