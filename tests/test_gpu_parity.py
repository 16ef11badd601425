"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same
seeded inputs. Integer results (ids, distances, centres, routes, tie order,
expansion counts) must be bit-exact; the FP32 re-rank must agree with the
float64 oracle within 1e-5 relative, with ids equal except where the oracle's
own distances of the swapped ids lie within that tolerance."""
import os
import struct

import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def bdg():
    from paper_2102_04656_b300 import build as b
    b.build()
    import paper_2102_04656_b300 as m
    m.lib()
    return m


def _np(codes):
    return codes.cpu().numpy().view(np.uint64)


def _entry(n, s, seed):
    return datagen.sample_ids(n, min(n, s), seed).astype(np.int32)


def _build_exact(bdg, codes_t, k, seed=5, kernel="auto"):
    n = codes_t.shape[0]
    entry = torch.from_numpy(_entry(n, 64, seed)).cuda()
    return bdg.build_graph(codes_t, k, m=1, t=1, entry=entry, kernel=kernel), entry


def _oracle_graph(cn, k, m, t, sample, bk_iters):
    """The oracle's own graph for a build configuration (exact when m == 1)."""
    if m == 1:
        return oracle.knn_exact(cn, k)
    cent, _, _ = oracle.bkmeans(cn, sample, m, bk_iters)
    r, _ = oracle.route(cn, cent, t)
    return oracle.knn_partitioned(cn, r, k)


def _tc_ok(bits, k):
    return bits in (256, 512) and k <= 64


KERNELS = ["popc", "tc"]


# ------------------------------------------------------------------ exact kNN
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("bits,n,k", [(64, 1000, 8), (128, 777, 16), (256, 3001, 32),
                                      (512, 1500, 64), (1024, 700, 128), (256, 130, 100),
                                      (512, 4097, 1), (256, 2000, 63)])
def test_exact_knn_bit_exact(bdg, bits, n, k, kernel):
    if kernel == "tc" and not _tc_ok(bits, k):
        pytest.skip("tensor path: 256/512-bit codes and k <= 64")
    c = datagen.random_codes(n, bits, seed=bits + n)
    c[7] = c[3]  # duplicates: d = 0 ties resolved by id
    c[n - 1] = c[3]
    g, _ = _build_exact(bdg, c.cuda(), k, kernel=kernel)
    torch.cuda.synchronize()
    ids_o, dist_o = oracle.knn_exact(_np(c), k)
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


@pytest.mark.parametrize("kernel", KERNELS)
def test_exact_knn_all_equal_codes(bdg, kernel):
    # every pair ties at d = 0: the k nearest are the k smallest other ids, which
    # the tensor path finds by its word-level (distance, position) bound
    c = torch.zeros(300, 4, dtype=torch.int64)
    g, _ = _build_exact(bdg, c.cuda(), 32, kernel=kernel)
    ids_o, dist_o = oracle.knn_exact(_np(c), 32)
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("bits,k,m,t", [(512, 64, 1, 1), (256, 32, 1, 1), (512, 64, 8, 3),
                                        (256, 32, 12, 4), (512, 64, 2, 2), (256, 32, 2, 2)])
def test_heavy_ties_bit_exact(bdg, bits, k, m, t, kernel):
    """Codes drawn from 40 distinct values: every row meets long runs of equal
    distances, so the lists keep filling with ties at the k-th distance. With
    m = 2 the partitions hold ~3,000 homes each, so with 512-bit codes the
    tensor path sorts them into locality order and the ties at the k-th distance
    are cut by id rank."""
    n = 6000
    base = datagen.random_codes(40, bits, seed=bits + k)
    pick = np.random.default_rng(bits * 7 + m).integers(0, 40, n)
    c = base[torch.from_numpy(pick)]
    entry = torch.from_numpy(_entry(n, 64, 3)).cuda()
    if m == 1:
        g = bdg.build_graph(c.cuda(), k, m=1, t=1, entry=entry, kernel=kernel)
        ids_o, dist_o = oracle.knn_exact(_np(c), k)
    else:
        sample = datagen.sample_ids(n, 64 * m, 4)
        g = bdg.build_graph(c.cuda(), k, m=m, t=t, bk_sample=torch.from_numpy(sample).cuda(),
                            bk_iters=4, entry=entry, kernel=kernel)
        cent, _, _ = oracle.bkmeans(_np(c), sample, m, 4)
        r, _ = oracle.route(_np(c), cent, t)
        ids_o, dist_o = oracle.knn_partitioned(_np(c), r, k)
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


@pytest.mark.parametrize("kernel", KERNELS)
def test_many_small_partitions_256b(bdg, kernel):
    """Partitions of ~100 homes (many ragged tiles) with four probes per point."""
    spec = datagen.MixtureSpec(30000, 64, 500, 256, seed=31)
    c = datagen.make_codes(spec)
    n, m, t, k = spec.n, 300, 4, 32
    sample = datagen.sample_ids(n, 64 * m, 5)
    entry = torch.from_numpy(_entry(n, 64, 6)).cuda()
    g = bdg.build_graph(c.cuda(), k, m=m, t=t, bk_sample=torch.from_numpy(sample).cuda(),
                        bk_iters=4, entry=entry, kernel=kernel)
    cent, _, _ = oracle.bkmeans(_np(c), sample, m, 4)
    r, _ = oracle.route(_np(c), cent, t)
    ids_o, dist_o = oracle.knn_partitioned(_np(c), r, k)
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


def test_exact_knn_small_n_pads(bdg):
    c = datagen.random_codes(5, 256, seed=9)
    g, _ = _build_exact(bdg, c.cuda(), 4)
    ids_o, dist_o = oracle.knn_exact(_np(c), 4)
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


@pytest.mark.parametrize("kernel", KERNELS)
def test_exact_knn_mixture_20k_256b_k32(bdg, kernel):
    """The exact brute-force workload: N = 20k, 128-d mixture -> 256-bit, k = 32."""
    w = datagen.WORKLOADS["exact_20k_256b"]
    c = datagen.make_codes(w["spec"])
    g, _ = _build_exact(bdg, c.cuda(), w["k"], kernel=kernel)
    ids_o, dist_o = oracle.knn_exact(_np(c), w["k"])
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


# ------------------------------------------------------------------ Bk-means + routing
@pytest.mark.parametrize("bits,n,m,S,iters", [(256, 5000, 32, 2048, 8), (512, 3000, 7, 700, 3),
                                              (64, 1000, 1, 1000, 2), (1024, 800, 16, 800, 4)])
def test_bkmeans_bit_exact(bdg, bits, n, m, S, iters):
    spec = datagen.MixtureSpec(n, 64, 24, bits, seed=bits + m)
    c = datagen.make_codes(spec)
    sample = datagen.sample_ids(n, S, seed=77)
    cent, loss = bdg.bkmeans(c.cuda(), torch.from_numpy(sample).cuda(), m, iters)
    cent_o, loss_o, _ = oracle.bkmeans(_np(c), sample, m, iters)
    assert np.array_equal(_np(cent), cent_o)
    assert np.array_equal(loss.cpu().numpy(), loss_o)


def test_bkmeans_sample_id_out_of_range_reads_zero_code(bdg):
    """A sample id outside [0, n) cannot be checked before launch; the call
    still returns cleanly and reads that id as the all-zero code: the centres
    equal those of the same run on the codes with a zero row appended and the
    bad ids pointing at it."""
    n, bits, m, S, iters = 3000, 256, 12, 600, 4
    c = datagen.make_codes(datagen.MixtureSpec(n, 64, 24, bits, seed=31)).cuda()
    sample = datagen.sample_ids(n, S, seed=32)
    bad = sample.copy()
    bad[[5, 77, 301]] = [-3, n, 1 << 40]
    cent, loss = bdg.bkmeans(c, torch.from_numpy(bad).cuda(), m, iters)
    torch.cuda.synchronize()
    c0 = torch.cat([c, torch.zeros(1, c.shape[1], dtype=c.dtype, device=c.device)])
    fixed = sample.copy()
    fixed[[5, 77, 301]] = n
    cent_r, loss_r = bdg.bkmeans(c0, torch.from_numpy(fixed).cuda(), m, iters)
    assert torch.equal(cent, cent_r)
    assert torch.equal(loss, loss_r)


@pytest.mark.parametrize("bits,t", [(256, 5), (512, 1), (128, 16), (64, 3)])
def test_route_bit_exact(bdg, bits, t):
    c = datagen.random_codes(4001, bits, seed=bits)
    ce = datagen.random_codes(300, bits, seed=bits + 1)
    ce[17] = ce[250]  # duplicate centre: tie by index
    r, d = bdg.route(c.cuda(), ce.cuda(), t)
    r_o, d_o = oracle.route(_np(c), _np(ce), t)
    assert np.array_equal(r.cpu().numpy(), r_o)
    assert np.array_equal(d.cpu().numpy(), d_o)


@pytest.mark.parametrize("kernel", ["popc", "tc"])
@pytest.mark.parametrize("bits,n,m,t", [(256, 3000, 2000, 16), (512, 1500, 1100, 8),
                                        (256, 700, 1200, 1), (512, 4001, 256, 5),
                                        (256, 3001, 200, 8), (512, 700, 17, 1),
                                        (256, 129, 16, 3)])
def test_route_kernels_bit_exact(bdg, kernel, bits, n, m, t, monkeypatch):
    """Routing on the tensor cores (256/512-bit codes) and on the ALU give the
    oracle's routes and distances, ties by centre index (duplicate centres,
    ragged last centre tile, t up to 16). Up to 256 centres and t <= 8 the
    tensor path keeps every centre in shared memory (m = 17 and 200 are not
    multiples of 16; 129 and 4001 points leave a ragged last point tile)."""
    monkeypatch.setenv("BDG_KNN_KERNEL", kernel)
    c = datagen.make_codes(datagen.MixtureSpec(n, 64, 40, bits, seed=n + m))
    ce = datagen.random_codes(m, bits, seed=m)
    ce[5] = ce[m - 1]
    ce[6] = c[3]  # a centre equal to a point: distance 0, not a self pair
    r, d = bdg.route(c.cuda(), ce.cuda(), t)
    r_o, d_o = oracle.route(_np(c), _np(ce), t)
    assert np.array_equal(r.cpu().numpy(), r_o)
    assert np.array_equal(d.cpu().numpy(), d_o)


def test_routes_gap_bit_exact(bdg):
    c = datagen.make_codes(datagen.MixtureSpec(5000, 64, 40, 256, seed=81))
    ce = datagen.random_codes(1500, 256, seed=82)
    r, d = bdg.route(c.cuda(), ce.cuda(), 8)
    r_o, d_o = oracle.route(_np(c), _np(ce), 8)
    for delta in (-1, 0, 2, 5, 300):
        got = bdg.routes_gap(r.clone(), d, delta).cpu().numpy()
        assert np.array_equal(got, oracle.routes_gap(r_o, d_o, delta)), delta


# ------------------------------------------------------------------ partitioned build
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("bits,n,m,t,k", [(512, 20000, 16, 3, 64), (256, 9000, 40, 5, 32),
                                          (256, 3000, 8, 8, 16), (128, 5000, 64, 2, 8),
                                          (512, 20000, 4, 3, 64), (512, 30000, 8, 4, 32),
                                          (256, 30000, 8, 4, 32)])
def test_partitioned_build_bit_exact(bdg, bits, n, m, t, k, kernel):
    """Bk-means, routing and Reduce 1 against the oracle. The last three cases
    have partitions of 3,000-5,000 homes: with 512-bit codes the tensor path then
    streams the homes in locality order (nearest of 16 pivot homes) and round A
    spirals out from every item's own tile."""
    if kernel == "tc" and not _tc_ok(bits, k):
        pytest.skip("tensor path: 256/512-bit codes and k <= 64")
    spec = datagen.MixtureSpec(n, 64, 48, bits, seed=n + m)
    c = datagen.make_codes(spec)
    sample = datagen.sample_ids(n, min(n, 64 * m), seed=3)
    entry = torch.from_numpy(_entry(n, 64, 4)).cuda()
    g = bdg.build_graph(c.cuda(), k, m=m, t=t, bk_sample=torch.from_numpy(sample).cuda(),
                        bk_iters=8, entry=entry, kernel=kernel)
    cent_o, _, _ = oracle.bkmeans(_np(c), sample, m, 8)
    r_o, _ = oracle.route(_np(c), cent_o, t)
    ids_o, dist_o = oracle.knn_partitioned(_np(c), r_o, k)
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


@pytest.mark.parametrize("kernel", KERNELS)
def test_partitioned_with_given_routes_and_empty_home(bdg, kernel):
    # partition 3 is probed by visitors but is nobody's home: its lists are pads
    n, bits, k = 2000, 256, 16
    c = datagen.random_codes(n, bits, seed=12)
    rng = np.random.default_rng(1)
    home = rng.integers(0, 3, n)
    routes = np.stack([home, np.full(n, 3), (home + 1) % 3], 1).astype(np.int32)
    entry = torch.from_numpy(_entry(n, 32, 2)).cuda()
    g = bdg.build_graph(c.cuda(), k, m=4, t=3, routes=torch.from_numpy(routes).cuda(),
                        entry=entry, kernel=kernel)
    ids_o, dist_o = oracle.knn_partitioned(_np(c), routes, k)
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


_POP8 = None


def _hamming_rows(codes, ids):
    """Hamming distances between each row's point and its listed ids (on the
    device; test-side arithmetic, a byte-table popcount): int32 [n, k]."""
    global _POP8
    if _POP8 is None:
        _POP8 = torch.tensor([bin(b).count("1") for b in range(256)], dtype=torch.int32,
                             device=codes.device)
    n, k = ids.shape
    out = torch.empty(n, k, dtype=torch.int32, device=codes.device)
    cb = codes.view(torch.uint8).reshape(codes.shape[0], -1)
    for s in range(0, n, 16384):
        e = min(n, s + 16384)
        nb = cb[ids[s:e].long().clamp(min=0)]                 # [b, k, bytes]
        x = torch.bitwise_xor(nb, cb[s:e, None, :])
        out[s:e] = _POP8[x.long()].sum(2).to(torch.int32)
    return out


def _check_rows_valid(codes, ids, dists, routes, home):
    """Properties every row of a partitioned graph has, at any size: ids in
    range and never the point itself, no repeats, each neighbour's home among
    the point's probed partitions, distances equal to the Hamming distances
    recomputed from the codes, rows ascending by (d, id)."""
    n, k = ids.shape
    me = torch.arange(n, device=ids.device, dtype=torch.int32)[:, None]
    assert bool(((ids >= 0) & (ids < n)).all()), "padding or out-of-range id"
    assert not bool((ids == me).any()), "self pair"
    srt = torch.sort(ids, dim=1).values
    assert not bool((srt[:, 1:] == srt[:, :-1]).any()), "repeated id"
    nh = home[ids.long()]                                      # [n, k]
    assert bool((nh[:, :, None] == routes[:, None, :]).any(2).all()), "id outside C(i)"
    assert torch.equal(dists, _hamming_rows(codes, ids)), "distance != Hamming"
    d0, d1 = dists[:, :-1], dists[:, 1:]
    i0, i1 = ids[:, :-1], ids[:, 1:]
    assert bool(((d0 < d1) | ((d0 == d1) & (i0 < i1))).all()), "row not ascending by (d, id)"


@pytest.mark.slow
def test_partitioned_2m_512b_sampled_rows(bdg):
    """Full-size partitioned workload (N = 2M, 512-bit, m = 256, t = 5, k = 64), in
    the configuration the bench times (a build plan replayed from its CUDA graph,
    kernel chosen by the autotuner): centres and routes compared in full; every
    one of the 2M rows checked for the properties of a partitioned graph; 10,000
    rows (among them members of the largest partition, the first and the last
    point) compared with the oracle, which computes them one by one."""
    w = datagen.WORKLOADS["partitioned_2m_512b"]
    spec = w["spec"]
    c_dev = datagen.make_codes(spec, device="cuda")
    c = _np(c_dev)
    n, m, t, k = spec.n, w["m"], w["t"], w["k"]
    sample = datagen.sample_ids(n, 64 * m, spec.seed + 3)
    sample_t = torch.from_numpy(sample).cuda()
    entry = torch.from_numpy(_entry(n, 256, spec.seed + 4)).cuda()
    cent, _ = bdg.bkmeans(c_dev, sample_t, m, w["bk_iters"])
    plan = bdg.BuildPlan(c_dev, k, m=m, t=t, bk_sample=sample_t, bk_iters=w["bk_iters"],
                         entry=entry, kernel="auto")
    plan.run()
    plan.run()  # a replay, as timed
    torch.cuda.synchronize()
    g = plan.graph
    cent_o, _, _ = oracle.bkmeans(c, sample, m, w["bk_iters"])
    assert np.array_equal(_np(cent), cent_o)
    r_gpu, _ = bdg.route(c_dev, cent, t)
    r_o, _ = oracle.route(c, cent_o, t)
    assert np.array_equal(r_gpu.cpu().numpy(), r_o)
    home = r_gpu[:, 0].contiguous()
    _check_rows_valid(c_dev, g.ids, g.dists, r_gpu, home)
    big = int(torch.bincount(home.long(), minlength=m).argmax())
    members = torch.nonzero(home == big).flatten().cpu().numpy()
    rng = np.random.default_rng(99)
    rows = np.concatenate([datagen.sample_ids(n, 8000, 99),
                           rng.choice(members, size=min(2000, members.size), replace=False),
                           [0, n - 1]])
    rows = np.unique(rows)
    ids_o, dist_o = oracle.knn_partitioned(c, r_o, k, rows)
    rt = torch.from_numpy(rows).cuda()
    assert np.array_equal(g.ids[rt].cpu().numpy(), ids_o)
    assert np.array_equal(g.dists[rt].cpu().numpy(), dist_o)
    plan.free()


@pytest.mark.slow
def test_search_10m_256b_properties(bdg):
    """Full-size search workload (10M x 256-bit, degree 32, 100k queries, ef mixed
    over {64, 128, 256, 512}, R = 100), in the configuration the bench times
    (packed layout): properties that hold at any size, checked on sampled
    queries — every returned distance is the Hamming distance the oracle
    computes for that id, rows are strictly ascending by (d, id) with padding
    last, at most min(ef, R) entries — and the packed layout gives the same
    answers as the rows as built."""
    w = datagen.WORKLOADS["search_10m_256b"]
    spec = w["spec"]
    codes = datagen.make_codes(spec, device="cuda")
    qc = datagen.make_codes(spec, device="cuda", n=w["nq"], seed_offset=2)
    n = spec.n
    sample = torch.from_numpy(datagen.sample_ids(n, 64 * 1024, spec.seed + 3)).cuda()
    entry = torch.from_numpy(datagen.sample_ids(n, 16384, spec.seed + 4).astype(np.int32)).cuda()
    g = bdg.build_graph(codes, w["k"], m=1024, t=3, bk_sample=sample, bk_iters=8, entry=entry)
    efs = datagen.ef_mix(w["nq"], w["efs"], spec.seed + 6)
    ef = torch.from_numpy(efs).cuda()
    R = 10 * w["topk"]
    a_ids, a_d = bdg.search(g, qc, ef, R, ef_max=max(w["efs"]))
    bdg.pack_codes(g)
    b_ids, b_d = bdg.search(g, qc, ef, R, ef_max=max(w["efs"]))
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)
    rows = datagen.sample_ids(w["nq"], 500, 17)
    sel = torch.from_numpy(rows).cuda()
    ids, d = b_ids[sel].cpu().numpy(), b_d[sel].cpu().numpy()
    cn, qn = _np(codes.cpu()), _np(qc.cpu())
    for r, qi in enumerate(rows):
        valid = ids[r] >= 0
        nv = int(valid.sum())
        assert valid[:nv].all() and not valid[nv:].any()  # padding last
        assert nv <= min(int(efs[qi]), R)
        keys = [(int(dd), int(ii)) for dd, ii in zip(d[r][:nv], ids[r][:nv])]
        assert keys == sorted(set(keys))  # strictly ascending, no repeats
        for dd, ii in keys[:20]:
            assert dd == oracle.hamming(qn[qi], cn[ii])
        assert (d[r][nv:] == spec.bits + 1).all()


@pytest.mark.parametrize("bits,k", [(512, 64), (256, 32), (128, 16), (1024, 100)])
def test_knn_rows_bit_exact(bdg, bits, k):
    c = datagen.random_codes(6000, bits, seed=bits * 3)
    c[100] = c[4000]
    rows = np.array([0, 100, 4000, 5999, 17, 17, 6001, -3] + list(range(200, 330)), np.int32)
    ids, dist = bdg.knn_rows(c.cuda(), torch.from_numpy(rows).cuda(), k)
    valid = (rows >= 0) & (rows < 6000)
    ids_o, dist_o = oracle.knn_exact(_np(c), k, rows[valid].astype(np.int64))
    assert np.array_equal(ids.cpu().numpy()[valid], ids_o)
    assert np.array_equal(dist.cpu().numpy()[valid], dist_o)
    assert (ids.cpu().numpy()[~valid] == -1).all()


# ------------------------------------------------------------------ search
def _write_graph(path, ids, bits, entry):
    n, k = ids.shape
    with open(path, "wb") as f:
        f.write(struct.pack("<6i", 0x31474442, 1, n, bits, k, len(entry)))
        f.write(np.ascontiguousarray(ids, np.int32).tobytes())
        f.write(np.zeros_like(ids, dtype=np.int32).tobytes())
        f.write(np.ascontiguousarray(entry, np.int32).tobytes())


@pytest.mark.parametrize("efs,R", [((64, 128, 256, 512), 100), ((1, 7, 33), 40), ((300,), 10),
                                   ((1024, 2048), 2048), ((700, 1500), 100),
                                   ((513, 600, 1000), 64)])
def test_search_bit_exact_with_expansions(bdg, efs, R):
    """Pools of every size class, up to ef = 2,048 (the 64-chunk pool) with all
    2,048 keys written."""
    spec = datagen.MixtureSpec(12000, 128, 128, 256, seed=31)
    c = datagen.make_codes(spec)
    q = datagen.make_codes(spec, n=700, seed_offset=2)
    entry = _entry(spec.n, 256, 8)
    g = bdg.build_graph(c.cuda(), 32, m=1, t=1, entry=torch.from_numpy(entry).cuda())
    ef = datagen.ef_mix(700, efs, seed=5)
    ids, dist, ex = bdg.search(g, q.cuda(), torch.from_numpy(ef).cuda(), R, ef_max=max(efs),
                               expansions=True)
    g_o, _ = oracle.knn_exact(_np(c), 32)
    ids_o, dist_o, cnt_o = oracle.search(_np(c), g_o, entry, _np(q), ef, R)
    assert np.array_equal(ids.cpu().numpy(), ids_o)
    assert np.array_equal(dist.cpu().numpy(), dist_o)
    assert np.array_equal(ex.cpu().numpy(), cnt_o[:, 0])


@pytest.mark.parametrize("bits,deg", [(256, 32), (512, 64), (64, 16)])
def test_search_with_packed_codes_bit_exact(bdg, bits, deg):
    """The packed layout (neighbour codes stored next to the rows) changes where
    the search reads codes from, not what it finds: pools, results and expansion
    counts equal the unpacked graph's and the oracle's, also through the
    re-rank and the shard-merged search."""
    spec = datagen.MixtureSpec(6000, 64, 40, bits, seed=bits + deg)
    c = datagen.make_codes(spec)
    g, entry = _build_exact(bdg, c.cuda(), deg)
    q = datagen.make_codes(spec, n=300, seed_offset=2)
    efs = np.array([16, 64, 100, 7] * 75, np.int32)
    ef = torch.from_numpy(efs).cuda()
    a_ids, a_d, a_ex = bdg.search(g, q.cuda(), ef, 40, ef_max=100, expansions=True)
    bdg.pack_codes(g)
    bdg.pack_codes(g)  # a second call does nothing
    b_ids, b_d, b_ex = bdg.search(g, q.cuda(), ef, 40, ef_max=100, expansions=True)
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d) and torch.equal(a_ex, b_ex)
    g_o, _ = oracle.knn_exact(_np(c), deg)
    assert np.array_equal(g.ids.cpu().numpy(), g_o)
    ids_o, dist_o, cnt = oracle.search(_np(c), g_o, entry.cpu().numpy(), _np(q), efs, 40)
    assert np.array_equal(b_ids.cpu().numpy(), ids_o)
    assert np.array_equal(b_ex.cpu().numpy(), cnt[:, 0])
    s_ids, _ = bdg.search_sharded([g], q.cuda(), ef, 40, ef_max=100)
    assert torch.equal(s_ids, b_ids)


def test_pack_codes_padded_rows_and_budget(bdg):
    """Rows with padding (ids -1) search the same packed or not; a copy that does
    not fit the memory budget is refused and leaves the graph searchable."""
    n, bits, k = 3000, 256, 16
    c = datagen.random_codes(n, bits, seed=61)
    rng = np.random.default_rng(2)
    home = rng.integers(0, 300, n)
    routes = np.stack([home, (home + 1 + rng.integers(0, 299, n)) % 300], 1).astype(np.int32)
    entry = torch.from_numpy(_entry(n, 32, 3)).cuda()
    g = bdg.build_graph(c.cuda(), k, m=300, t=2, routes=torch.from_numpy(routes).cuda(),
                        entry=entry)
    assert (g.ids.cpu().numpy() < 0).any()  # tiny partitions leave padded rows
    q = datagen.random_codes(100, bits, seed=62).cuda()
    ef = torch.full((100,), 48, dtype=torch.int32).cuda()
    a_ids, a_d = bdg.search(g, q, ef, 30, ef_max=48)
    used = bdg.memory_in_use()
    bdg.set_memory_budget(used + 1024)
    try:
        with pytest.raises(bdg.BDGError):
            bdg.pack_codes(g)
    finally:
        bdg.set_memory_budget(0)
    b_ids, _ = bdg.search(g, q, ef, 30, ef_max=48)
    assert torch.equal(a_ids, b_ids)
    bdg.pack_codes(g)
    c_ids, c_d = bdg.search(g, q, ef, 30, ef_max=48)
    assert torch.equal(a_ids, c_ids) and torch.equal(a_d, c_d)


def test_search_on_loaded_adversarial_graphs(bdg, tmp_path):
    # line graph with thermometer codes + complete graph + disconnected pieces
    n = 64
    c = np.zeros((n, 1), np.uint64)
    for i in range(n):
        c[i, 0] = np.uint64((1 << i) - 1) if i < 64 else np.uint64(~0)
    line = np.array([[i - 1 if i > 0 else -1, i + 1 if i < n - 1 else -1] + [-1] * 30
                     for i in range(n)], np.int32)
    rng = np.random.default_rng(3)
    scram = np.array([rng.permutation(row) for row in line], np.int32)  # -1 anywhere in a row
    comp = np.array([[j for j in range(n) if j != i][:40] for i in range(n)], np.int32)
    split = np.array([[(i + 1) % 32 + (32 if i >= 32 else 0), -1] for i in range(n)], np.int32)
    q = c[[0, 12, 40, 63, 5]].copy()
    q[4, 0] ^= np.uint64(1 << 50)
    c_t = torch.from_numpy(c.view(np.int64)).cuda()
    for name, adj in [("line", line), ("scram", scram), ("complete", comp), ("split", split)]:
        entry = np.array([0, 33], np.int32)
        p = str(tmp_path / f"{name}.bdg")
        _write_graph(p, adj, 64, entry)
        g = bdg.load_graph(p, c_t)
        # ef_max = 1024: the same queries through the 1,024-key pool
        for efs, ef_max in (((1,), 64), ((2, 5), 64), ((64,), 64), ((1,), 1024),
                            ((2, 5, 64), 1024)):
            ef = datagen.ef_mix(len(q), efs, seed=1)
            ids, dist, ex = bdg.search(g, torch.from_numpy(q.view(np.int64)).cuda(),
                                       torch.from_numpy(ef).cuda(), 20, ef_max=ef_max,
                                       expansions=True)
            ids_o, dist_o, cnt_o = oracle.search(c, adj, entry, q, ef, 20)
            assert np.array_equal(ids.cpu().numpy(), ids_o), (name, efs, ef_max)
            assert np.array_equal(dist.cpu().numpy(), dist_o), (name, efs, ef_max)
            assert np.array_equal(ex.cpu().numpy(), cnt_o[:, 0]), (name, efs, ef_max)


def test_search_invalid_ef_rows_are_padding(bdg):
    c = datagen.random_codes(500, 128, seed=4)
    g, _ = _build_exact(bdg, c.cuda(), 16)
    ef = torch.tensor([0, 65, 10], dtype=torch.int32).cuda()
    ids, dist, ex = bdg.search(g, c[:3].cuda(), ef, 12, ef_max=64, expansions=True)
    ids, ex = ids.cpu().numpy(), ex.cpu().numpy()
    assert (ids[0] == -1).all() and (ids[1] == -1).all() and ex[0] == -1 and ex[1] == -1
    assert ids[2, 0] == 2 and ex[2] > 0


def test_graph_save_load_roundtrip(bdg, tmp_path):
    c = datagen.random_codes(900, 256, seed=8).cuda()
    g, _ = _build_exact(bdg, c, 8)
    p = str(tmp_path / "g.bdg")
    g.save(p)
    h = bdg.load_graph(p, c)
    assert torch.equal(g.ids, h.ids) and torch.equal(g.dists, h.dists)


# ------------------------------------------------------------------ re-rank
def _check_rerank(ids, d2, feats, qf, cand, k):
    ids_o, d64 = oracle.rerank(feats, qf, cand, k, "f64")
    ids = ids.cpu().numpy()
    d2 = d2.cpu().numpy().astype(np.float64)
    fin = np.isfinite(d64)
    assert np.array_equal(np.isfinite(d2), fin)
    assert np.allclose(d2[fin], d64[fin], rtol=RTOL, atol=0)
    for r in range(ids.shape[0]):
        if np.array_equal(ids[r], ids_o[r]):
            continue
        # an id swap is only allowed between near-equal distances
        diff = ids[r] != ids_o[r]
        assert np.allclose(d2[r][diff], d64[r][diff], rtol=RTOL, atol=0)
        assert set(ids[r][diff]) <= set(ids_o[r][diff]) | set(cand[r])


@pytest.mark.parametrize("D,R,k", [(128, 100, 10), (256, 64, 32), (512, 37, 5), (1024, 1, 1),
                                   (128, 2048, 10)])
def test_rerank_within_tolerance(bdg, D, R, k):
    rng = np.random.default_rng(D + R)
    feats = rng.standard_normal((3000, D)).astype(np.float32)
    qf = rng.standard_normal((257, D)).astype(np.float32)
    cand = np.array([rng.permutation(3000)[:R] for _ in range(257)], np.int32)
    cand[5, : R // 2] = -1  # short rows
    ids, d2 = bdg.rerank(torch.from_numpy(feats).cuda(), torch.from_numpy(qf).cuda(),
                         torch.from_numpy(cand).cuda(), k)
    _check_rerank(ids, d2, feats, qf, cand, k)


def test_search_rerank_end_to_end(bdg):
    spec = datagen.MixtureSpec(8000, 128, 64, 256, seed=41)
    c, x = datagen.make_codes(spec, with_features=True)
    qc, qx = datagen.make_codes(spec, n=300, seed_offset=2, with_features=True)
    entry = _entry(spec.n, 128, 6)
    g = bdg.build_graph(c.cuda(), 32, m=1, t=1, entry=torch.from_numpy(entry).cuda())
    ef = datagen.ef_mix(300, (64, 128), seed=2)
    ids, d2 = bdg.search_rerank(g, qc.cuda(), qx.cuda(), x.cuda(), torch.from_numpy(ef).cuda(),
                                100, 10, ef_max=128)
    g_o, _ = oracle.knn_exact(_np(c), 32)
    cand_o, _, _ = oracle.search(_np(c), g_o, entry, _np(qc), ef, 100)
    _check_rerank(ids, d2, x.numpy(), qx.numpy(), cand_o, 10)


# ------------------------------------------------------------------ build plans (CUDA graphs)
@pytest.mark.parametrize("kernel", ["auto", "popc", "tc"])
def test_build_plan_replays_bit_exact(bdg, kernel, tmp_path, monkeypatch):
    monkeypatch.setenv("BDG_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    spec = datagen.MixtureSpec(12000, 64, 48, 512, seed=515)
    c = datagen.make_codes(spec).cuda()
    sample = torch.from_numpy(datagen.sample_ids(spec.n, 1024, 3)).cuda()
    entry = torch.from_numpy(_entry(spec.n, 64, 4)).cuda()
    plan = bdg.BuildPlan(c, 64, m=16, t=3, bk_sample=sample, bk_iters=6, entry=entry,
                         kernel=kernel)
    cent_o, _, _ = oracle.bkmeans(_np(c.cpu()), sample.cpu().numpy(), 16, 6)
    r_o, _ = oracle.route(_np(c.cpu()), cent_o, 3)
    ids_o, dist_o = oracle.knn_partitioned(_np(c.cpu()), r_o, 64)
    for _ in range(2):  # replays give the same exact graph
        plan.run()
        torch.cuda.synchronize()
        assert np.array_equal(plan.graph.ids.cpu().numpy(), ids_o)
        assert np.array_equal(plan.graph.dists.cpu().numpy(), dist_o)
        assert plan.kernel_ms() > 0
    if kernel == "auto":
        assert plan.tuned_ms["popc"] > 0 and plan.tuned_ms["tc"] > 0
        assert (tmp_path / "tune.txt").exists()
    # the plan re-reads the codes: new contents give the new graph
    c2 = datagen.random_codes(spec.n, 512, seed=9).cuda()
    c.copy_(c2)
    plan.run()
    torch.cuda.synchronize()
    cent2, _, _ = oracle.bkmeans(_np(c2.cpu()), sample.cpu().numpy(), 16, 6)
    r2, _ = oracle.route(_np(c2.cpu()), cent2, 3)
    ids2, _ = oracle.knn_partitioned(_np(c2.cpu()), r2, 64)
    assert np.array_equal(plan.graph.ids.cpu().numpy(), ids2)
    plan.free()


def test_build_plan_run_host_bit_exact(bdg, tmp_path, monkeypatch):
    """bdg_build_plan_run_host: host codes in, host rows out, on a side stream;
    two different code sets in a row give their own oracle graphs."""
    monkeypatch.setenv("BDG_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    n, bits, k, m, t = 6000, 256, 16, 8, 3
    dev = datagen.random_codes(n, bits, seed=1).cuda()
    sample = torch.from_numpy(datagen.sample_ids(n, 512, 3)).cuda()
    entry = torch.from_numpy(_entry(n, 32, 4)).cuda()
    plan = bdg.BuildPlan(dev, k, m=m, t=t, bk_sample=sample, bk_iters=4, entry=entry)
    st = torch.cuda.Stream()
    for seed in (21, 22):
        spec = datagen.MixtureSpec(n, 64, 30, bits, seed=seed)
        hc = datagen.make_codes(spec).pin_memory()
        hi = torch.empty(n, k, dtype=torch.int32).pin_memory()
        hd = torch.empty(n, k, dtype=torch.int32).pin_memory()
        plan.run_host(hc, hi, hd, stream=st)
        st.synchronize()
        cent_o, _, _ = oracle.bkmeans(_np(hc), sample.cpu().numpy(), m, 4)
        r_o, _ = oracle.route(_np(hc), cent_o, t)
        ids_o, dist_o = oracle.knn_partitioned(_np(hc), r_o, k)
        assert np.array_equal(hi.numpy(), ids_o)
        assert np.array_equal(hd.numpy(), dist_o)
    with pytest.raises(ValueError):
        plan.run_host(hc.cuda(), hi, hd)
    plan.free()


@pytest.mark.parametrize("world", [2, 3])
def test_partition_sharded_build_merge_bit_exact(bdg, world):
    """The compute steps of the partition-sharded build on one GPU: each rank's
    build over its LPT-assigned partitions (other slots -1), then the merge of
    the ranks' partial rows (bdg_merge_lists) equals the single build and the
    oracle; the collective between them is tested with gloo ranks on CPU."""
    from paper_2102_04656_b300 import distributed as D
    n, bits, k, m, t = 12000, 256, 32, 20, 4
    c = datagen.make_codes(datagen.MixtureSpec(n, 64, 30, bits, seed=90 + world))
    ce = datagen.random_codes(m, bits, seed=91)
    cd = c.cuda()
    routes, _ = bdg.route(cd, ce.cuda(), t)
    entry = torch.from_numpy(_entry(n, 32, 2)).cuda()
    hc, vc = D.partition_counts(routes, m)
    owner = D.assign_partitions(hc.cpu().numpy(), vc.cpu().numpy(), world)
    parts_i, parts_d = [], []
    for rank in range(world):
        g = bdg.build_graph(cd, k, m=m, t=t, routes=D.rank_routes(routes, owner, rank),
                            entry=entry)
        parts_i.append(g.ids.clone())
        parts_d.append(g.dists.clone())
        g.free()
    mi, md = bdg.merge_lists(torch.stack(parts_i).contiguous(), torch.stack(parts_d).contiguous(),
                             bits)
    ids_o, dist_o = oracle.knn_partitioned(_np(c), routes.cpu().numpy(), k)
    assert np.array_equal(mi.cpu().numpy(), ids_o)
    assert np.array_equal(md.cpu().numpy(), dist_o)


# ------------------------------------------------------------------ size classes
def _class_routes(seed):
    """Routes over 24 partitions whose home sets fall in all three size classes
    (>= 4096, 512..4095, < 512 homes), t = 3 distinct partitions per point."""
    rng = np.random.default_rng(seed)
    sizes = [5000, 4096, 3000, 2100, 900, 512, 511, 400, 300, 200, 100, 60, 30, 8, 1, 0,
             700, 1500, 2500, 350, 45, 3, 2, 77]
    home = np.repeat(np.arange(24), sizes)
    rng.shuffle(home)
    n = home.size
    r = np.empty((n, 3), np.int32)
    r[:, 0] = home
    for i in range(n):
        r[i, 1:] = rng.choice(np.setdiff1d(np.arange(24), [home[i]]), 2, replace=False)
    return r


@pytest.mark.parametrize("kmap", [("tc", "popc32", "popc"), ("popc", "tc", "popc32"),
                                  ("popc32", "popc32", "tc")])
def test_size_class_variants_bit_exact(bdg, kmap):
    """A build whose partition size classes run on different Reduce-1 variants
    (tensor cores, popcount with 64- and 32-visitor sub-tiles) equals the oracle."""
    r = _class_routes(7)
    n, k = r.shape[0], 32
    c = datagen.make_codes(datagen.MixtureSpec(n, 64, 40, 256, seed=700 + len(kmap[0])))
    entry = torch.from_numpy(_entry(n, 32, 2)).cuda()
    g = bdg.build_graph(c.cuda(), k, m=24, t=3, routes=torch.from_numpy(r).cuda(), entry=entry,
                        class_kernel=kmap)
    ids_o, dist_o = oracle.knn_partitioned(_np(c), r, k)
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


def test_build_plan_tunes_each_size_class(bdg, tmp_path, monkeypatch):
    """The plan's autotuner times every variant on every size class, keeps the
    fastest per class, caches the choice and builds the oracle's graph."""
    monkeypatch.setenv("BDG_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    r = _class_routes(8)
    n, k = r.shape[0], 32
    c = datagen.make_codes(datagen.MixtureSpec(n, 64, 40, 256, seed=801)).cuda()
    rt = torch.from_numpy(r).cuda()
    entry = torch.from_numpy(_entry(n, 32, 2)).cuda()
    plan = bdg.BuildPlan(c, k, m=24, t=3, routes=rt, entry=entry, kernel="auto")
    plan.run()
    torch.cuda.synchronize()
    ids_o, dist_o = oracle.knn_partitioned(_np(c.cpu()), r, k)
    assert np.array_equal(plan.graph.ids.cpu().numpy(), ids_o)
    assert np.array_equal(plan.graph.dists.cpu().numpy(), dist_o)
    for cl in plan.classes:
        assert set(cl["tuned_ms"]) == {"popc", "tc", "popc32"}
        assert cl["variant"] == min(cl["tuned_ms"], key=cl["tuned_ms"].get)
    line = (tmp_path / "tune.txt").read_text().split()
    assert line[0].startswith("classes2|") and len(line) == 1 + 3 + 9
    plan.free()
    # a second plan of the same shape takes the cached choice without timing
    plan2 = bdg.BuildPlan(c, k, m=24, t=3, routes=rt, entry=entry, kernel="auto")
    assert [cl["variant"] for cl in plan2.classes] == [cl["variant"] for cl in plan.classes]
    assert all(not cl["tuned_ms"] for cl in plan2.classes)
    plan2.run()
    torch.cuda.synchronize()
    assert np.array_equal(plan2.graph.ids.cpu().numpy(), ids_o)
    plan2.free()


# ------------------------------------------------------------------ coarse_num (Section 3.2)
def _skewed_routes(n, m, t, seed):
    """Routes with Zipf-skewed homes and random further slots (repeats allowed:
    the rule only sums the counts of the slots it keeps)."""
    rng = np.random.default_rng(seed)
    w = rng.zipf(1.5, m).astype(np.float64)
    r = rng.integers(0, m, (n, t)).astype(np.int32)
    if n:
        r[:, 0] = rng.choice(m, n, p=w / w.sum())
    return r


@pytest.mark.parametrize("n,m,t,coarse", [(5000, 40, 7, 300), (20000, 13000, 5, 4),
                                          (3000, 64, 1, 10), (0, 8, 3, 5), (4000, 30, 16, 0),
                                          (4000, 30, 4, 10 ** 12), (100003, 256, 8, 2500)])
def test_routes_coarse_bit_exact(bdg, n, m, t, coarse):
    r = _skewed_routes(n, m, t, seed=n + m)
    rt = torch.from_numpy(r).cuda()
    cnt = bdg.routes_coarse(rt, m, coarse)
    r_o, cnt_o = oracle.routes_coarse(r, m, coarse)
    assert np.array_equal(cnt.cpu().numpy(), cnt_o)
    assert np.array_equal(rt.cpu().numpy(), r_o)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("bits,n,m,t,k,coarse", [(512, 20000, 16, 6, 64, 3500),
                                                 (256, 9000, 40, 8, 32, 700),
                                                 (128, 5000, 64, 4, 8, 150)])
def test_partitioned_build_coarse_num_bit_exact(bdg, bits, n, m, t, k, coarse, kernel):
    if kernel == "tc" and not _tc_ok(bits, k):
        pytest.skip("tensor path: 256/512-bit codes and k <= 64")
    spec = datagen.MixtureSpec(n, 64, 48, bits, seed=n + m + 1)
    c = datagen.make_codes(spec)
    sample = datagen.sample_ids(n, min(n, 64 * m), seed=3)
    entry = torch.from_numpy(_entry(n, 64, 4)).cuda()
    g = bdg.build_graph(c.cuda(), k, m=m, t=t, bk_sample=torch.from_numpy(sample).cuda(),
                        bk_iters=8, entry=entry, kernel=kernel, coarse_num=coarse)
    cent_o, _, _ = oracle.bkmeans(_np(c), sample, m, 8)
    r_o, _ = oracle.route(_np(c), cent_o, t)
    rc_o, _ = oracle.routes_coarse(r_o, m, coarse)
    kept = (rc_o >= 0).sum(1)
    assert kept.min() < kept.max()  # the number of probed partitions varies
    ids_o, dist_o = oracle.knn_partitioned(_np(c), rc_o, k)
    assert np.array_equal(g.ids.cpu().numpy(), ids_o)
    assert np.array_equal(g.dists.cpu().numpy(), dist_o)


def test_build_plan_coarse_num_bit_exact(bdg, tmp_path, monkeypatch):
    monkeypatch.setenv("BDG_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    spec = datagen.MixtureSpec(12000, 64, 48, 512, seed=516)
    c = datagen.make_codes(spec).cuda()
    sample = torch.from_numpy(datagen.sample_ids(spec.n, 1024, 3)).cuda()
    entry = torch.from_numpy(_entry(spec.n, 64, 4)).cuda()
    plan = bdg.BuildPlan(c, 64, m=16, t=5, bk_sample=sample, bk_iters=6, entry=entry,
                         coarse_num=2000)
    cent_o, _, _ = oracle.bkmeans(_np(c.cpu()), sample.cpu().numpy(), 16, 6)
    r_o, _ = oracle.route(_np(c.cpu()), cent_o, 5)
    rc_o, _ = oracle.routes_coarse(r_o, 16, 2000)
    ids_o, dist_o = oracle.knn_partitioned(_np(c.cpu()), rc_o, 64)
    for _ in range(2):
        plan.run()
        torch.cuda.synchronize()
        assert np.array_equal(plan.graph.ids.cpu().numpy(), ids_o)
        assert np.array_equal(plan.graph.dists.cpu().numpy(), dist_o)
    plan.free()


def test_coarse_num_rejects_given_routes(bdg):
    c = datagen.random_codes(500, 256, seed=2).cuda()
    r = torch.zeros(500, 2, dtype=torch.int32, device="cuda")
    r[:, 1] = 1
    entry = torch.from_numpy(_entry(500, 16, 1)).cuda()
    with pytest.raises(bdg.BDGError):
        bdg.build_graph(c, 8, m=2, t=2, routes=r, entry=entry, coarse_num=100)


# ------------------------------------------------------------------ neighbourhood propagation
@pytest.mark.parametrize("bits,n,m,t,k,rounds", [(512, 20000, 16, 2, 32, 1), (256, 12000, 30, 2, 64, 2),
                                                 (128, 5000, 8, 1, 16, 1), (64, 3000, 6, 2, 100, 1)])
def test_propagate_bit_exact(bdg, bits, n, m, t, k, rounds):
    spec = datagen.MixtureSpec(n, 64, 40, bits, seed=bits + n + k)
    c = datagen.make_codes(spec)
    sample = datagen.sample_ids(n, min(n, 64 * m), 7)
    entry = torch.from_numpy(_entry(n, 64, 8)).cuda()
    g = bdg.build_graph(c.cuda(), k, m=m, t=t, bk_sample=torch.from_numpy(sample).cuda(),
                        bk_iters=4, entry=entry)
    base = g.ids.cpu().numpy()
    p = bdg.propagate(g, rounds)
    torch.cuda.synchronize()
    ids_o, _ = _oracle_graph(_np(c), k, m, t, sample, 4)
    assert np.array_equal(base, ids_o)
    for _ in range(rounds):
        ids_o, dist_o = oracle.propagate(_np(c), ids_o)
    assert np.array_equal(p.ids.cpu().numpy(), ids_o)
    assert np.array_equal(p.dists.cpu().numpy(), dist_o)
    assert np.array_equal(g.ids.cpu().numpy(), base)  # the input graph is untouched


def test_propagate_padded_rows(bdg):
    """A graph with more neighbours asked for than exist (padding rows)."""
    c = datagen.random_codes(40, 256, seed=77)
    g, _ = _build_exact(bdg, c.cuda(), 39)
    p = bdg.propagate(g, 1)
    g_o, _ = oracle.knn_exact(_np(c), 39)
    assert np.array_equal(g.ids.cpu().numpy(), g_o)
    ids_o, dist_o = oracle.propagate(_np(c), g_o)
    assert np.array_equal(p.ids.cpu().numpy(), ids_o)
    assert np.array_equal(p.dists.cpu().numpy(), dist_o)


# ------------------------------------------------------------------ pruning (Section 3.4)
@pytest.mark.parametrize("bits,n,m,t,k,L", [(512, 20000, 16, 3, 64, 50), (256, 12000, 30, 2, 32, 32),
                                            (256, 12000, 30, 2, 32, 1), (1024, 3000, 1, 1, 128, 64),
                                            (64, 5000, 8, 2, 16, 7)])
def test_prune_bit_exact(bdg, bits, n, m, t, k, L):
    spec = datagen.MixtureSpec(n, 64, 40, bits, seed=bits + n + k + L)
    c = datagen.make_codes(spec)
    sample = datagen.sample_ids(n, min(n, 64 * m), 7)
    entry = torch.from_numpy(_entry(n, 64, 8)).cuda()
    g = bdg.build_graph(c.cuda(), k, m=m, t=t, bk_sample=torch.from_numpy(sample).cuda(),
                        bk_iters=4, entry=entry)
    base = g.ids.cpu().numpy()
    p = bdg.prune(g, L)
    g_o, _ = _oracle_graph(_np(c), k, m, t, sample, 4)
    assert np.array_equal(base, g_o)
    ids_o, dist_o = oracle.prune(_np(c), g_o, L)
    assert p.ids.shape == (n, L)
    assert np.array_equal(p.ids.cpu().numpy(), ids_o)
    assert np.array_equal(p.dists.cpu().numpy(), dist_o)
    assert np.array_equal(g.ids.cpu().numpy(), base)  # the input graph is untouched
    if L >= 32:
        assert (ids_o < 0).any()  # occlusion removed edges


def test_prune_adversarial_rows(bdg, tmp_path):
    """Loaded rows in no order, with -1, out-of-range ids, self ids and repeats;
    all-equal codes (nothing occludes)."""
    n, k, bits = 3000, 48, 256
    rng = np.random.default_rng(4)
    for codes in (datagen.random_codes(n, bits, seed=5),
                  torch.full((n, bits // 64), 0x1234, dtype=torch.int64)):
        ids = rng.integers(-3, n + 5, (n, k)).astype(np.int32)
        ids[::5, 3] = np.arange(0, n, 5)
        ids[:, 7] = ids[:, 9]
        ids[100] = -1
        path = str(tmp_path / "adv.bdg")
        _write_graph(path, ids, bits, np.arange(16))
        g = bdg.load_graph(path, codes.cuda())
        for L in (40, 5):
            p = bdg.prune(g, L)
            ids_o, dist_o = oracle.prune(_np(codes), ids, L)
            assert np.array_equal(p.ids.cpu().numpy(), ids_o)
            assert np.array_equal(p.dists.cpu().numpy(), dist_o)


def test_prune_rejects_bad_L(bdg):
    c = datagen.random_codes(500, 256, seed=2).cuda()
    g, _ = _build_exact(bdg, c, 8)
    for L in (0, 9):
        with pytest.raises(bdg.BDGError):
            bdg.prune(g, L)


def test_prune_then_search_bit_exact(bdg):
    """The pruned graph (padded rows) searched: equal to the oracle's search on it."""
    spec = datagen.MixtureSpec(8000, 64, 40, 256, seed=91)
    c = datagen.make_codes(spec)
    g, entry = _build_exact(bdg, c.cuda(), 32)
    p = bdg.prune(g, 24)
    q = datagen.random_codes(64, 256, seed=92)
    ef = torch.full((64,), 64, dtype=torch.int32).cuda()
    ids, dist = bdg.search(p, q.cuda(), ef, 40, ef_max=64)
    g_o, _ = oracle.knn_exact(_np(c), 32)
    p_o, _ = oracle.prune(_np(c), g_o, 24)
    assert np.array_equal(p.ids.cpu().numpy(), p_o)
    ids_o, dist_o, _ = oracle.search(_np(c), p_o, entry.cpu().numpy(), _np(q),
                                     np.full(64, 64), 40)
    assert np.array_equal(ids.cpu().numpy(), ids_o)
    assert np.array_equal(dist.cpu().numpy(), dist_o)


# ------------------------------------------------------------------ multi-shard (Section 3.4)
@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("bits,n,S,m,t,k", [(512, 20003, 4, 16, 3, 32), (256, 9001, 3, 1, 1, 16),
                                            (128, 6000, 7, 12, 2, 8)])
def test_build_and_search_sharded_bit_exact(bdg, bits, n, S, m, t, k, kernel):
    if kernel == "tc" and not _tc_ok(bits, k):
        pytest.skip("tensor path: 256/512-bit codes and k <= 64")
    spec = datagen.MixtureSpec(n, 64, 48, bits, seed=n + S)
    c = datagen.make_codes(spec)
    cn = _np(c)
    off = oracle.shard_offsets(n, S)
    assert list(off) == bdg.shard_offsets(n, S)
    sample = datagen.sample_ids(n, min(n, 64 * m), seed=3)
    entries = np.stack([_entry(int(off[s + 1] - off[s]), 32, 10 + s) for s in range(S)])
    graphs = bdg.build_sharded(c.cuda(), k, S, torch.from_numpy(entries).cuda(), m=m, t=t,
                               bk_sample=torch.from_numpy(sample).cuda(), bk_iters=6,
                               kernel=kernel)
    cent_o = oracle.bkmeans(cn, sample, m, 6)[0] if m > 1 else None
    graphs_o = []
    for s in range(S):
        sl = cn[off[s]:off[s + 1]]
        if m > 1:
            r_o, _ = oracle.route(sl, cent_o, t)
            ids_o, dist_o = oracle.knn_partitioned(sl, r_o, k)
        else:
            ids_o, dist_o = oracle.knn_exact(sl, k)
        assert np.array_equal(graphs[s].ids.cpu().numpy(), ids_o), s
        assert np.array_equal(graphs[s].dists.cpu().numpy(), dist_o), s
        graphs_o.append(ids_o)
    q = datagen.make_codes(spec, n=300, seed_offset=2)
    efs = np.array([16, 64, 100, 7] * 75, np.int32)
    R = 40
    ids, dist = bdg.search_sharded(graphs, q.cuda(), torch.from_numpy(efs).cuda(), R, ef_max=100)
    ids_o, dist_o = oracle.search_sharded(cn, graphs_o, list(entries), _np(q), efs, R)
    assert np.array_equal(ids.cpu().numpy(), ids_o)
    assert np.array_equal(dist.cpu().numpy(), dist_o)
    for g in graphs:
        g.free()


def test_search_sharded_one_shard_equals_search(bdg):
    c = datagen.random_codes(5000, 256, seed=21).cuda()
    g, _ = _build_exact(bdg, c, 16)
    q = datagen.random_codes(200, 256, seed=22).cuda()
    ef = torch.tensor([3, 50, 0, 65] * 50, dtype=torch.int32).cuda()  # 0 and 65: invalid rows
    a_ids, a_d = bdg.search(g, q, ef, 30, ef_max=64)
    b_ids, b_d = bdg.search_sharded([g], q, ef, 30, ef_max=64)
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)


def test_sharded_argument_errors(bdg):
    c = datagen.random_codes(400, 256, seed=23).cuda()
    e = torch.zeros(2, 4, dtype=torch.int32).cuda()
    with pytest.raises(bdg.BDGError):
        bdg.build_sharded(c, 8, 0, e[:0])
    with pytest.raises(bdg.BDGError):
        bdg.build_sharded(c, 250, 2, e)  # k >= shard size
    g, _ = _build_exact(bdg, c, 8)
    q = c[:4]
    ef = torch.full((4,), 8, dtype=torch.int32).cuda()
    with pytest.raises(bdg.BDGError):
        bdg.search_sharded([g] * 33, q, ef, 8, ef_max=8)
    with pytest.raises(bdg.BDGError):
        bdg.search_sharded([g] * 7, q, ef, 1000, ef_max=8)  # S R > 6144
