"""The continuous-batching server: requests submitted from several host threads
while batches are in flight come back with exactly the ids and squared
distances that the same queries get when searched alone (each query runs on its
own warp with its own ef, so batching must not change a result; the FP32
re-rank is compared bit for bit, well inside its 1e-5 tolerance). Admission
respects the memory budget and over-budget requests are refused."""
import threading

import numpy as np
import pytest
import torch

import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bdg():
    from paper_2102_04656_b300 import build as b
    b.build()
    import paper_2102_04656_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("efs,R,ef_max", [((64, 256), 100, 256), ((1024, 2048), 2048, 2048)])
def test_results_identical_alone_and_in_the_mix(bdg, efs, R, ef_max):
    spec = datagen.MixtureSpec(60_000, 128, 256, 256, seed=4242)
    codes, feats = datagen.make_codes(spec, device="cuda", with_features=True)
    qc, qf = datagen.make_codes(spec, device="cuda", n=3000, seed_offset=2, with_features=True)
    entry = torch.from_numpy(datagen.sample_ids(spec.n, 1024, 1).astype(np.int32)).cuda()
    g = bdg.build_graph(codes, 32, m=16, t=3, bk_sample=torch.from_numpy(
        datagen.sample_ids(spec.n, 1024, 2)).cuda(), bk_iters=6, entry=entry)
    k = 10
    ef_all = datagen.ef_mix(3000, efs, 3)
    qc_h, qf_h = qc.cpu().numpy(), qf.cpu().numpy()
    rng = np.random.default_rng(0)
    sizes = rng.integers(1, 200, 40)
    starts = np.concatenate([[0], np.cumsum(sizes)])[:-1] % (3000 - 200)
    budget = 250 * (8 * 4 + 4 * 128 + 4 + 8 * R + 8 * k)  # at most ~250 queries in flight
    srv = bdg.Server(g, feats, R=R, k=k, ef_max=ef_max, max_batch=256, n_streams=3,
                     memory_budget=budget)
    with pytest.raises(bdg.BDGError):
        srv.submit(qc_h[:300], qf_h[:300], ef_all[:300])  # more than max_batch
    reqs = [None] * len(sizes)

    def submitter(lo, hi):
        for i in range(lo, hi):
            s, n = int(starts[i]), int(sizes[i])
            reqs[i] = srv.submit(qc_h[s:s + n], qf_h[s:s + n], ef_all[s:s + n])

    th = [threading.Thread(target=submitter, args=(0, 20)),
          threading.Thread(target=submitter, args=(20, 40))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    out = [srv.wait(r) for r in reqs]
    st = srv.stats()
    assert st["queries"] == int(sizes.sum()) and st["batches"] >= 2 and st["in_flight_bytes"] == 0
    for i, (ids, d2, lat) in enumerate(out):
        s, n = int(starts[i]), int(sizes[i])
        a_ids, a_d2 = bdg.search_rerank(g, qc[s:s + n].contiguous(), qf[s:s + n].contiguous(),
                                        feats, torch.from_numpy(ef_all[s:s + n]).cuda(), R, k,
                                        ef_max=ef_max)
        assert np.array_equal(ids, a_ids.cpu().numpy()), i
        assert np.array_equal(d2, a_d2.cpu().numpy()), i
        assert lat > 0
    srv.free()
