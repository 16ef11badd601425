"""Pins of the CPU oracle against things other than itself: per-bit brute force,
metric axioms, the +-1 dot-product identity, hand-worked fixtures under
tests/golden/, closed forms and invariants (Section 3 / 3.2 / 3.5 of the paper)."""
import os

import numpy as np
import pytest

import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_codes(n, bits, seed):
    return datagen.random_codes(n, bits, seed).numpy().view(np.uint64)


def _bits(c, bits):
    return datagen.unpack_bits(c, bits).astype(np.int64)


# ---------------------------------------------------------------- Hamming
@pytest.mark.parametrize("bits", [64, 128, 256, 512])
def test_hamming_matches_per_bit_count(oracle_lib, bits):
    c = _rand_codes(40, bits, 7 + bits)
    b = _bits(c, bits)
    for i in range(0, 40, 3):
        for j in range(1, 40, 5):
            want = int((b[i] != b[j]).sum())
            assert oracle_lib.hamming(c[i], c[j]) == want


def test_hamming_metric_axioms(oracle_lib):
    c = _rand_codes(60, 256, 3)
    rng = np.random.default_rng(0)
    for _ in range(300):
        i, j, l = rng.integers(0, 60, 3)
        dij = oracle_lib.hamming(c[i], c[j])
        assert oracle_lib.hamming(c[i], c[i]) == 0
        assert dij == oracle_lib.hamming(c[j], c[i])
        assert dij <= oracle_lib.hamming(c[i], c[l]) + oracle_lib.hamming(c[l], c[j])


def test_hamming_pm1_dot_identity(oracle_lib):
    # with s = 2y - 1 in {-1, +1}: <s_a, s_b> = bits - 2 d(a, b)
    bits = 512
    c = _rand_codes(20, bits, 11)
    s = 2 * _bits(c, bits) - 1
    dot = s @ s.T
    for i in range(20):
        for j in range(20):
            assert (bits - dot[i, j]) // 2 == oracle_lib.hamming(c[i], c[j])


# ---------------------------------------------------------------- exact kNN
def _read_knn_golden():
    rows = {}
    codes = None
    with open(os.path.join(GOLDEN, "knn_tiny.txt")) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    codes = np.array([int(x, 16) for x in lines[0].split()], dtype=np.uint64)[:, None]
    for ln in lines[1:]:
        p, rest = ln.split(":")
        pairs = [tuple(int(v) for v in tok.split(",")) for tok in rest.split()]
        rows[int(p)] = pairs
    return codes, rows


def test_knn_exact_hand_worked_fixture(oracle_lib):
    codes, rows = _read_knn_golden()
    ids, dist = oracle_lib.knn_exact(codes, 2)
    for p, pairs in rows.items():
        assert [(int(a), int(b)) for a, b in zip(ids[p], dist[p])] == pairs


def test_knn_exact_pads_when_k_exceeds_candidates(oracle_lib):
    codes, _ = _read_knn_golden()
    ids, dist = oracle_lib.knn_exact(codes, 7)
    assert (ids[:, 5:] == -1).all() and (ids[:, 6] == -1).all()
    assert (dist[:, 5:] == 65).all()
    assert (ids[:, :5] >= 0).all()


@pytest.mark.parametrize("bits,n,k", [(64, 200, 8), (256, 300, 32), (512, 150, 16)])
def test_knn_exact_brute_force_and_separation(oracle_lib, bits, n, k):
    c = _rand_codes(n, bits, 100 + bits)
    # add exact duplicates so that d = 0 ties with id tie-break are exercised
    c[5] = c[17]
    c[40] = c[17]
    b = _bits(c, bits)
    full = (b[:, None, :] != b[None, :, :]).sum(2)  # per-bit brute force
    ids, dist = oracle_lib.knn_exact(c, k)
    for i in range(n):
        d = full[i].copy()
        order = [j for j in np.lexsort((np.arange(n), d)) if j != i][:k]
        assert list(ids[i]) == order
        assert list(dist[i]) == [int(d[j]) for j in order]
        # separation: every returned key is below every key left out
        keys = d.astype(np.int64) * (1 << 32) + np.arange(n)
        keys[i] = -1
        kept = keys[ids[i]]
        rest = np.setdiff1d(np.arange(n), np.append(ids[i], i))
        assert kept.max() < keys[rest].min()


def test_knn_exact_all_equal_codes_is_pure_id_order(oracle_lib):
    c = np.zeros((50, 4), np.uint64)
    ids, dist = oracle_lib.knn_exact(c, 10)
    for i in range(50):
        want = [j for j in range(50) if j != i][:10]
        assert list(ids[i]) == want
        assert (dist[i] == 0).all()


# ---------------------------------------------------------------- Bk-means
def test_bkmeans_hand_worked_fixture(oracle_lib):
    vals = {}
    with open(os.path.join(GOLDEN, "bkmeans_tiny.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            key, rest = ln.split(":")
            vals[key.strip()] = rest.split()
    codes = np.array([int(x, 16) for x in vals["codes"]], np.uint64)[:, None]
    sample = np.array([int(x) for x in vals["sample"]], np.int64)
    cent, loss, assign = oracle_lib.bkmeans(codes, sample, 2, 1)
    assert [int(x) for x in cent[:, 0]] == [int(x, 16) for x in vals["centroids"]]
    assert list(loss) == [int(x) for x in vals["loss"]]
    assert list(assign) == [int(x) for x in vals["assign"]]


def test_bkmeans_loss_non_increasing(oracle_lib):
    spec = datagen.MixtureSpec(3000, 32, 16, 128, seed=5)
    c = datagen.make_codes(spec).numpy().view(np.uint64)
    sample = datagen.sample_ids(3000, 2000, 9)
    _, loss, _ = oracle_lib.bkmeans(c, sample, 16, 8)
    assert all(loss[i + 1] <= loss[i] for i in range(len(loss) - 1))
    assert loss[-1] < loss[0]


def test_bkmeans_single_centre_is_bitwise_majority(oracle_lib):
    bits = 128
    c = _rand_codes(101, bits, 21)  # odd count: no ties
    sample = np.arange(101, dtype=np.int64)
    cent, _, _ = oracle_lib.bkmeans(c, sample, 1, 1)
    maj = (_bits(c, bits).sum(0) * 2 > 101).astype(np.uint8)
    assert (datagen.unpack_bits(cent, bits)[0] == maj).all()


def test_bkmeans_tie_keeps_previous_bit(oracle_lib):
    # two codes, one centre: every differing bit is a 1-of-2 tie -> keeps init bits
    c = _rand_codes(2, 128, 33)
    cent, _, _ = oracle_lib.bkmeans(c, np.array([1, 0], np.int64), 1, 3)
    assert (cent[0] == c[1]).all()


def test_bkmeans_recovers_planted_centres(oracle_lib):
    bits, m, per = 256, 8, 50
    rng = np.random.default_rng(4)
    centres = _rand_codes(m, bits, 44)
    cb = _bits(centres, bits)
    pts = []
    for j in range(m):
        for _ in range(per):
            b = cb[j].copy()
            flip = rng.choice(bits, 10, replace=False)
            b[flip] ^= 1
            pts.append(b)
    pts = np.array(pts, np.uint64)
    packed = np.zeros((len(pts), bits // 64), np.uint64)
    for w in range(bits // 64):
        for s in range(64):
            packed[:, w] |= pts[:, w * 64 + s] << np.uint64(s)
    sample = np.array([j * per for j in range(m)] + [i for i in range(m * per) if i % per],
                      np.int64)
    cent, _, assign = oracle_lib.bkmeans(packed, sample, m, 2)
    assert (cent == centres).all()
    assert (assign[:m] == np.arange(m)).all()


# ---------------------------------------------------------------- routing + partitioned graph
def test_route_matches_brute_force(oracle_lib):
    bits = 256
    c = _rand_codes(120, bits, 51)
    ce = _rand_codes(13, bits, 52)
    ce[4] = ce[9]  # duplicate centre: tie broken by centre index
    r, d = oracle_lib.route(c, ce, 5)
    full = (_bits(c, bits)[:, None, :] != _bits(ce, bits)[None, :, :]).sum(2)
    for i in range(120):
        order = np.lexsort((np.arange(13), full[i]))[:5]
        assert list(r[i]) == list(order)
        assert list(d[i]) == [int(full[i, o]) for o in order]


def test_partitioned_probe_all_equals_exact(oracle_lib):
    spec = datagen.MixtureSpec(600, 32, 8, 128, seed=61)
    c = datagen.make_codes(spec).numpy().view(np.uint64)
    ce, _, _ = oracle_lib.bkmeans(c, datagen.sample_ids(600, 600, 62), 6, 4)
    r, _ = oracle_lib.route(c, ce, 6)  # t = m: every partition is probed
    ids_p, dist_p = oracle_lib.knn_partitioned(c, r, 16)
    ids_e, dist_e = oracle_lib.knn_exact(c, 16)
    assert (ids_p == ids_e).all() and (dist_p == dist_e).all()
    r1 = np.zeros((600, 1), np.int32)  # m = 1
    ids_1, _ = oracle_lib.knn_partitioned(c, r1, 16)
    assert (ids_1 == ids_e).all()


def test_partitioned_rows_lie_in_candidate_set(oracle_lib):
    spec = datagen.MixtureSpec(800, 32, 8, 128, seed=71)
    c = datagen.make_codes(spec).numpy().view(np.uint64)
    ce, _, _ = oracle_lib.bkmeans(c, datagen.sample_ids(800, 512, 72), 8, 4)
    r, _ = oracle_lib.route(c, ce, 2)
    ids, dist = oracle_lib.knn_partitioned(c, r, 8)
    home = r[:, 0]
    b = _bits(c, 128)
    for i in range(0, 800, 7):
        cand = [j for j in range(800) if j != i and home[j] in set(r[i])]
        d = {j: int((b[i] != b[j]).sum()) for j in cand}
        want = sorted(cand, key=lambda j: (d[j], j))[:8]
        got = [int(x) for x in ids[i] if x >= 0]
        assert got == want
        assert all(int(x) in set(cand) for x in got)


# ---------------------------------------------------------------- search
def _thermometer(n, bits=64):
    c = np.zeros((n, bits // 64), np.uint64)
    for i in range(n):
        for b in range(i):
            c[i, b // 64] |= np.uint64(1) << np.uint64(b % 64)
    return c


def test_search_hand_worked_greedy_walk(oracle_lib):
    # 16 points on a line (thermometer codes: d(i, j) = |i - j|), graph = i-1, i+1;
    # entry sample {0}; query at 12; ef = 1 walks 0 -> 1 -> ... -> 12:
    # 13 expansions, 1 + 13 distance evaluations (entry + nodes 1..13), result (12, 0).
    c = _thermometer(16)
    g = np.array([[i - 1 if i > 0 else -1, i + 1 if i < 15 else -1] for i in range(16)],
                 np.int32)
    ids, dist, cnt = oracle_lib.search(c, g, np.array([0], np.int32), c[12:13], 1, 1)
    assert ids[0, 0] == 12 and dist[0, 0] == 0
    assert list(cnt[0]) == [13, 14]


def test_search_complete_graph_equals_brute_force(oracle_lib):
    n, bits = 90, 256
    c = _rand_codes(n, bits, 81)
    g = np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)
    q = _rand_codes(12, bits, 82)
    ids, dist, cnt = oracle_lib.search(c, g, np.array([3, 50], np.int32), q, n, n)
    full = (_bits(q, bits)[:, None, :] != _bits(c, bits)[None, :, :]).sum(2)
    for i in range(12):
        order = np.lexsort((np.arange(n), full[i]))
        assert list(ids[i]) == list(order)
        assert list(dist[i]) == [int(full[i, o]) for o in order]
    assert (cnt[:, 1] == n + 1).all()  # entry sample (2) + every other point once


def test_search_pads_short_pools(oracle_lib):
    c = _thermometer(4)
    g = np.array([[1, -1], [0, -1], [3, -1], [2, -1]], np.int32)  # two components
    ids, dist, _ = oracle_lib.search(c, g, np.array([0], np.int32), c[1:2], 8, 5)
    assert list(ids[0]) == [1, 0, -1, -1, -1]
    assert list(dist[0]) == [0, 1, 65, 65, 65]


# ---------------------------------------------------------------- re-rank
def test_rerank_integer_grid_exact(oracle_lib):
    # integer-valued features: squared L2 is exact in both precisions
    f = np.array([[0, 0], [1, 0], [0, 2], [3, 4], [1, 1], [1, 0]], np.float32)
    qf = np.array([[1, 0]], np.float32)
    cand = np.array([[3, 5, 2, 1, -1, 0, 4]], np.int32)
    for prec in ("f32", "f64"):
        ids, d = oracle_lib.rerank(f, qf, cand, 4, prec)
        assert list(ids[0]) == [1, 5, 0, 4]  # d = 0, 0 (id tie), 1, 1 (id tie)
        assert list(d[0]) == [0, 0, 1, 1]


def test_rerank_f32_within_tolerance_of_f64(oracle_lib):
    rng = np.random.default_rng(3)
    f = rng.standard_normal((500, 128)).astype(np.float32)
    qf = rng.standard_normal((20, 128)).astype(np.float32)
    cand = np.array([rng.permutation(500)[:100] for _ in range(20)], np.int32)
    i32, d32 = oracle_lib.rerank(f, qf, cand, 10, "f32")
    i64, d64 = oracle_lib.rerank(f, qf, cand, 10, "f64")
    brute = ((qf[:, None, :].astype(np.float64) - f[cand].astype(np.float64)) ** 2).sum(2)
    for q in range(20):
        order = cand[q][np.lexsort((cand[q], brute[q]))][:10]
        assert list(i64[q]) == list(order)
    assert np.allclose(d32, d64, rtol=1e-5, atol=0)


# ---------------------------------------------------------------- recall (Eq. 3)
def test_recall_definitions(oracle_lib):
    exact = np.array([[1, 2, 3, 4]])
    assert oracle_lib.recall_ids(np.array([[4, 3, 9, 1]]), exact) == 0.75
    ed = np.array([[1, 2, 2, 2]])
    assert oracle_lib.recall_tie_aware(np.array([[1, 2, 2, 2]]), ed) == 1.0
    assert oracle_lib.recall_tie_aware(np.array([[1, 2, 3, 3]]), ed) == 0.5


# ---------------------------------------------------------------- propagation
def _read_propagate_golden():
    with open(os.path.join(GOLDEN, "propagate_tiny.txt")) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    codes = np.array([[int(x, 16)] for x in lines[0].split()], dtype=np.uint64)
    n = codes.shape[0]
    g_in = np.array([[int(v) for v in ln.split(":")[1].split()] for ln in lines[1:1 + n]],
                    dtype=np.int32)
    want_ids, want_d = [], []
    for ln in lines[1 + n:1 + 2 * n]:
        pairs = [p.split(",") for p in ln.split(":")[1].split()]
        want_ids.append([int(a) for a, _ in pairs])
        want_d.append([int(b) for _, b in pairs])
    return codes, g_in, np.array(want_ids, np.int32), np.array(want_d, np.int32)


def test_propagate_hand_worked_fixture(oracle_lib):
    codes, g_in, want_ids, want_d = _read_propagate_golden()
    ids, d = oracle_lib.propagate(codes, g_in)
    assert np.array_equal(ids, want_ids)
    assert np.array_equal(d, want_d)


def test_propagate_brute_force_with_padding(oracle_lib):
    """Against a direct set enumeration, on random graphs with padding and self ids."""
    rng = np.random.default_rng(12)
    n, k, bits = 70, 5, 128
    c = _rand_codes(n, bits, 21)
    b = _bits(c, bits)
    g = rng.integers(0, n, (n, k)).astype(np.int32)
    g[rng.random((n, k)) < 0.15] = -1
    g[3, 0] = 3  # a point listed as its own neighbour is not a candidate of itself
    ids, d = oracle_lib.propagate(c, g)
    for x in range(n):
        cand = {int(z) for z in g[x] if z >= 0 and z != x}
        for z in g[x]:
            if z >= 0:
                cand |= {int(y) for y in g[z] if y >= 0 and y != x}
        keys = sorted((int((b[x] != b[y]).sum()), y) for y in cand)[:k]
        want_i = [y for _, y in keys] + [-1] * (k - len(keys))
        want_d = [dd for dd, _ in keys] + [bits + 1] * (k - len(keys))
        assert ids[x].tolist() == want_i and d[x].tolist() == want_d, x


def test_propagate_keeps_the_exact_graph_and_improves_rows(oracle_lib):
    """The exact graph is a fixed point; on an approximate graph no row's k-th key
    grows, and every row is drawn from its old list and its second floor."""
    spec = datagen.MixtureSpec(1500, 32, 12, 256, seed=44)
    c = datagen.make_codes(spec).numpy().view(np.uint64)
    k = 8
    ex_i, ex_d = oracle_lib.knn_exact(c, k)
    ids, d = oracle_lib.propagate(c, ex_i)
    assert np.array_equal(ids, ex_i) and np.array_equal(d, ex_d)
    cent, _, _ = oracle_lib.bkmeans(c, np.arange(0, 1500, 3, dtype=np.int64), 20, 4)
    r, _ = oracle_lib.route(c, cent, 2)  # two probes: lists reach into neighbouring partitions
    ap_i, ap_d = oracle_lib.knn_partitioned(c, r, k)
    ids, d = oracle_lib.propagate(c, ap_i)
    key = lambda dd, ii: dd.astype(np.int64) * (1 << 32) + (ii.astype(np.int64) & 0xffffffff)
    assert (key(d[:, -1], ids[:, -1]) <= key(ap_d[:, -1], ap_i[:, -1])).all()
    assert (d[:, -1] < ap_d[:, -1]).any()  # the round found better neighbours somewhere
    for x in range(0, 1500, 97):
        pool = set(ap_i[x].tolist())
        for z in ap_i[x]:
            if z >= 0:
                pool |= set(ap_i[z].tolist())
        assert set(ids[x].tolist()) <= pool


# ---------------------------------------------------------------- coarse_num
def _read_coarse_golden():
    with open(os.path.join(GOLDEN, "routes_coarse_tiny.txt")) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    routes, counts, cases, cur = [], None, {}, None
    for ln in lines:
        if ln.startswith("counts:"):
            counts = np.array([int(v) for v in ln.split(":")[1].split()], np.int32)
        elif ln.startswith("coarse"):
            cur = int(ln.split()[1])
            cases[cur] = []
        elif cur is None:
            routes.append([int(v) for v in ln.split(":")[1].split()])
        else:
            cases[cur].append([int(v) for v in ln.split(":")[1].split()])
    return (np.array(routes, np.int32), counts,
            {c: np.array(r, np.int32) for c, r in cases.items()})


def test_routes_coarse_hand_worked_fixture(oracle_lib):
    routes, counts, cases = _read_coarse_golden()
    for coarse, want in cases.items():
        got, cnt = oracle_lib.routes_coarse(routes, 4, coarse)
        assert np.array_equal(cnt, counts)
        assert np.array_equal(got, want), coarse


def test_routes_gap_hand_worked(oracle_lib):
    # point 0: centres 3, 1, 4 at 10, 12, 17 -> delta 2 keeps 3, 1; delta 7 keeps all
    # point 1: centres 2, 0, 1 at 5, 5, 6 (a tie with the home) -> delta 0 keeps 2, 0
    routes = np.array([[3, 1, 4], [2, 0, 1]], np.int32)
    rdist = np.array([[10, 12, 17], [5, 5, 6]], np.int32)
    assert oracle_lib.routes_gap(routes, rdist, 2).tolist() == [[3, 1, -1], [2, 0, 1]]
    assert oracle_lib.routes_gap(routes, rdist, 0).tolist() == [[3, -1, -1], [2, 0, -1]]
    assert oracle_lib.routes_gap(routes, rdist, 7).tolist() == [[3, 1, 4], [2, 0, 1]]
    assert oracle_lib.routes_gap(routes, rdist, -1).tolist() == [[3, -1, -1], [2, -1, -1]]


def test_routes_gap_against_per_bit_distances(oracle_lib):
    """Kept slots are exactly those whose centre's per-bit Hamming distance to
    the point exceeds the home centre's by at most delta; they form a prefix of
    the nearest-centre order; more delta never keeps fewer."""
    import datagen
    bits, n, m, t = 128, 400, 30, 6
    c = datagen.random_codes(n, bits, seed=71).numpy().view(np.uint64)
    ce = datagen.random_codes(m, bits, seed=72).numpy().view(np.uint64)
    r, d = oracle_lib.route(c, ce, t)
    ub, ucb = datagen.unpack_bits(c, bits), datagen.unpack_bits(ce, bits)
    prev = None
    for delta in (-1, 0, 1, 3, 8, bits):
        got = oracle_lib.routes_gap(r, d, delta)
        for i in range(n):
            dd = [int((ub[i] != ucb[r[i, s]]).sum()) for s in range(t)]
            want = [int(r[i, s]) if s == 0 or dd[s] - dd[0] <= delta else -1 for s in range(t)]
            assert got[i].tolist() == want
        nk = (got >= 0).sum(1)
        assert np.array_equal(got >= 0, np.arange(t)[None, :] < nk[:, None])
        if prev is not None:
            assert (nk >= prev).all()
        prev = nk


def _random_routes(n, m, t, seed):
    rng = np.random.default_rng(seed)
    sizes = rng.zipf(1.6, m).astype(np.float64)  # skewed partition sizes
    home = rng.choice(m, n, p=sizes / sizes.sum()).astype(np.int32)
    r = np.empty((n, t), np.int32)
    for i in range(n):
        others = rng.permutation(np.setdiff1d(np.arange(m), [home[i]]))[:t - 1]
        r[i, 0], r[i, 1:] = home[i], others
    return r


def test_routes_coarse_invariants(oracle_lib):
    """Kept slots form a prefix; the prefix before the last kept slot holds fewer
    than coarse_num points; a cut prefix holds at least coarse_num; the home
    counts are the histogram of slot 0; coarse_num <= 1 keeps only the home and
    coarse_num > n keeps everything; more coarse_num never keeps fewer slots."""
    n, m, t = 3000, 40, 7
    r = _random_routes(n, m, t, 5)
    hist = np.bincount(r[:, 0], minlength=m)
    prev = None
    for coarse in (0, 1, 50, 120, 300, 800, n + 1):
        got, cnt = oracle_lib.routes_coarse(r, m, coarse)
        assert np.array_equal(cnt, hist)
        kept = got >= 0
        assert kept[:, 0].all()
        assert np.array_equal(got[kept], r[kept])
        nk = kept.sum(1)
        assert np.array_equal(kept, np.arange(t)[None, :] < nk[:, None])  # a prefix
        held = np.cumsum(hist[r], axis=1)  # points held by the first s + 1 slots
        before_last = np.where(nk > 1, held[np.arange(n), np.maximum(nk - 2, 0)], 0)
        assert (before_last[nk > 1] < coarse).all()
        cut = nk < t
        assert (held[np.arange(n), nk - 1][cut] >= coarse).all()
        if coarse <= 1:
            assert (nk == 1).all()
        if coarse > n:
            assert (nk == t).all()
        if prev is not None:
            assert (nk >= prev).all()
        prev = nk


def test_partitioned_unused_slots_probe_nothing(oracle_lib):
    """A -1 slot contributes no neighbours: the rows equal those of the routes
    with every -1 slot replaced by the home (a repeat adds no candidate), and a
    direct set enumeration."""
    n, m, t, k, bits = 400, 12, 4, 6, 128
    c = _rand_codes(n, bits, 31)
    r = _random_routes(n, m, t, 6)
    got_r, _ = oracle_lib.routes_coarse(r, m, 60)
    assert (got_r < 0).any() and (got_r[:, 1] >= 0).any()
    filled = np.where(got_r >= 0, got_r, got_r[:, :1])
    ids, d = oracle_lib.knn_partitioned(c, got_r, k)
    ids2, d2 = oracle_lib.knn_partitioned(c, filled, k)
    assert np.array_equal(ids, ids2) and np.array_equal(d, d2)
    bitsm = _bits(c, bits)
    for i in range(0, n, 37):
        parts = set(int(p) for p in got_r[i] if p >= 0)
        cand = [(int((bitsm[i] != bitsm[j]).sum()), j) for j in range(n)
                if j != i and int(r[j, 0]) in parts]
        cand.sort()
        want = cand[:k] + [(bits + 1, -1)] * max(0, k - len(cand))
        assert [j for _, j in want] == list(ids[i]) and [dd for dd, _ in want] == list(d[i])


# ---------------------------------------------------------------- pruning
def _read_prune_golden():
    with open(os.path.join(GOLDEN, "prune_tiny.txt")) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    codes = np.array([[int(x, 16)] for x in lines[0].split()], dtype=np.uint64)
    n = codes.shape[0]
    g_in = np.array([[int(v) for v in ln.split(":")[1].split()] for ln in lines[1:1 + n]],
                    dtype=np.int32)
    cases, i = {}, 1 + n
    while i < len(lines):
        L = int(lines[i].split()[1])
        rows = [[p.split(",") for p in ln.split(":")[1].split()] for ln in lines[i + 1:i + 1 + n]]
        cases[L] = (np.array([[int(a) for a, _ in r] for r in rows], np.int32),
                    np.array([[int(b) for _, b in r] for r in rows], np.int32))
        i += 1 + n
    return codes, g_in, cases


def test_prune_hand_worked_fixture(oracle_lib):
    codes, g_in, cases = _read_prune_golden()
    assert set(cases) == {4, 2}
    for L, (want_ids, want_d) in cases.items():
        ids, d = oracle_lib.prune(codes, g_in, L)
        assert np.array_equal(ids, want_ids), L
        assert np.array_equal(d, want_d), L


def test_prune_line_keeps_the_two_sides(oracle_lib):
    """Codes with i ones (d(i, j) = |i - j|) and complete rows: every interior
    point keeps exactly its two line neighbours, the ends keep one."""
    n = 40
    codes = np.array([[(1 << i) - 1] for i in range(n)], dtype=np.uint64)
    g = np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)
    ids, d = oracle_lib.prune(codes, g, 8)
    for i in range(n):
        want = [i - 1, i + 1] if 0 < i < n - 1 else ([1] if i == 0 else [n - 2])
        got = [int(v) for v in ids[i] if v >= 0]
        assert got == want, i
        assert (d[i, :len(want)] == 1).all() and (d[i, len(want):] == 65).all()


def test_prune_equal_codes_keep_first_L_by_id(oracle_lib):
    """All codes equal: every distance is 0 and nothing is strictly closer, so
    the first L candidates by id are kept."""
    n, k, L = 30, 12, 7
    codes = np.full((n, 2), 0x5A5A, dtype=np.uint64)
    rng = np.random.default_rng(3)
    g = np.stack([rng.permutation(np.setdiff1d(np.arange(n), [i]))[:k] for i in range(n)]
                 ).astype(np.int32)
    ids, d = oracle_lib.prune(codes, g, L)
    for i in range(n):
        assert list(ids[i]) == sorted(g[i])[:L]
    assert (d == 0).all()


@pytest.mark.parametrize("bits,n,k,L", [(64, 300, 20, 10), (256, 200, 32, 32), (128, 150, 16, 3)])
def test_prune_characterisation(oracle_lib, bits, n, k, L):
    """On random rows (with -1, self ids and repeats): the kept ids are a
    subsequence of the distinct candidates in (d, id) order; no kept id is
    occluded by one kept before it; every candidate skipped before the walk
    stopped has an occluder kept before it; the walk stops only at L kept."""
    c = _rand_codes(n, bits, 41 + n)
    rng = np.random.default_rng(n)
    g = rng.integers(-1, n, (n, k)).astype(np.int32)
    g[::7, 0] = np.arange(0, n, 7)  # self ids
    g[:, 1] = g[:, 2]  # repeats
    ids, d = oracle_lib.prune(c, g, L)
    b = _bits(c, bits)
    dist = lambda i, j: int((b[i] != b[j]).sum())
    for x in range(n):
        cand = sorted({(dist(x, int(y)), int(y)) for y in g[x] if 0 <= y < n and y != x})
        kept = [int(v) for v in ids[x] if v >= 0]
        assert all(v == -1 for v in ids[x][len(kept):])
        pos = [cand.index((dist(x, y), y)) for y in kept]
        assert pos == sorted(pos) and len(set(kept)) == len(kept)
        for a, y in enumerate(kept):
            assert d[x, a] == dist(x, y)
            assert all(dist(z, y) >= dist(x, y) for z in kept[:a])
        last = pos[-1] if len(kept) == L else len(cand) - 1
        for j, (dxy, y) in enumerate(cand[:last + 1]):
            if y in kept:
                continue
            before = [z for z, p in zip(kept, pos) if p < j]
            assert any(dist(z, y) < dxy for z in before), (x, y)


# ---------------------------------------------------------------- multi-shard search
def test_shard_offsets_cover_contiguously(oracle_lib):
    for n, S in ((10, 3), (1000, 7), (5, 5), (8, 1)):
        off = oracle_lib.shard_offsets(n, S)
        assert off[0] == 0 and off[-1] == n and (np.diff(off) >= n // S).all()
        assert (np.diff(off) <= -(-n // S)).all()


def test_search_sharded_one_shard_is_search(oracle_lib):
    n, bits = 300, 128
    c = _rand_codes(n, bits, 91)
    rng = np.random.default_rng(9)
    g = np.array([rng.permutation(np.setdiff1d(np.arange(n), [i]))[:12] for i in range(n)],
                 np.int32)
    e = np.array([0, 100, 200], np.int32)
    q = _rand_codes(20, bits, 92)
    ef = np.array([5, 40] * 10)
    a_ids, a_d, _ = oracle_lib.search(c, g, e, q, ef, 30)
    b_ids, b_d = oracle_lib.search_sharded(c, [g], [e], q, ef, 30)
    assert np.array_equal(a_ids, b_ids) and np.array_equal(a_d, b_d)


def test_search_sharded_complete_shards_equal_brute_force(oracle_lib):
    """Complete graph per shard and ef >= shard size: each shard returns its
    exact first keys, so the merged answer is the exact first R over all n."""
    n, bits, S, R = 150, 256, 4, 25
    c = _rand_codes(n, bits, 93)
    c[77] = c[12]  # a duplicate code across shards: ties by global id
    off = oracle_lib.shard_offsets(n, S)
    graphs, entries = [], []
    for s in range(S):
        ns = int(off[s + 1] - off[s])
        graphs.append(np.array([[j for j in range(ns) if j != i] for i in range(ns)], np.int32))
        entries.append(np.array([0], np.int32))
    q = np.concatenate([_rand_codes(9, bits, 94), c[12:13]])
    ids, d = oracle_lib.search_sharded(c, graphs, entries, q, n, R)
    full = (_bits(q, bits)[:, None, :] != _bits(c, bits)[None, :, :]).sum(2)
    for i in range(q.shape[0]):
        order = np.lexsort((np.arange(n), full[i]))[:R]
        assert list(ids[i]) == list(order)
        assert list(d[i]) == [int(full[i, o]) for o in order]
    assert list(ids[-1][:2]) == [12, 77]
