"""CPU oracle for the Binary Distributed Graph hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct statements of what the method computes, written
from the paper (Zhao et al., "Large-Scale Visual Search with Binary Distributed
Graph at Alibaba"): Hamming distance and k-NN lists (Section 3), Bk-means
(Section 3.2, Eq. 1-2), nearest-centre routing and the single-pass
divide-and-conquer graph (Section 3.2), best-first search with a long-link entry
sample (Section 3.5), the real-valued re-rank (Section 3.5), the coarse_num
rule (Section 3.2), neighbourhood propagation (Section 3.3), occlusion pruning
(Section 3.4), recall (Eq. 3) and
the MLP router's forward/backward (``oracle.mlp``; the paper has no router).

Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may
import this package. It shares no code with the CUDA library and never imports
it. The numeric work is in ``bdg_oracle.c`` (compiled with gcc here by
``build()``); this module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bdg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile bdg_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _codes(c) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(c))
    if c.dtype == np.int64:
        c = c.view(np.uint64)
    assert c.dtype == np.uint64 and c.ndim == 2
    return c


def threads() -> int:
    """Number of OpenMP threads the oracle uses."""
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def hamming(a, b) -> int:
    a = np.ascontiguousarray(np.asarray(a).reshape(-1)).view(np.uint64)
    b = np.ascontiguousarray(np.asarray(b).reshape(-1)).view(np.uint64)
    lib = _load()
    lib.or_hamming.restype = ctypes.c_int32
    return int(lib.or_hamming(_p(a), _p(b), ctypes.c_int32(a.size)))


def knn_exact(codes, k: int, qidx=None):
    """Exact k-NN lists (ids int32 [nq, k], dists int32 [nq, k]) of points qidx."""
    c = _codes(codes)
    n, w = c.shape
    q = np.arange(n, dtype=np.int64) if qidx is None else np.ascontiguousarray(qidx, np.int64)
    ids = np.empty((q.size, k), np.int32)
    dist = np.empty((q.size, k), np.int32)
    _load().or_knn_exact(_p(c), ctypes.c_int64(n), ctypes.c_int32(w), ctypes.c_int32(k),
                         _p(q), ctypes.c_int64(q.size), _p(ids), _p(dist))
    return ids, dist


def bkmeans(codes, sample, m: int, iters: int):
    """Bk-means on codes[sample]: returns (centroids uint64 [m, W], loss int64 [iters+1],
    final assignment int32 [S])."""
    c = _codes(codes)
    s = np.ascontiguousarray(sample, np.int64)
    assert s.size >= m
    w = c.shape[1]
    cent = np.empty((m, w), np.uint64)
    loss = np.empty(iters + 1, np.int64)
    assign = np.empty(s.size, np.int32)
    _load().or_bkmeans(_p(c), ctypes.c_int32(w), _p(s), ctypes.c_int64(s.size),
                       ctypes.c_int32(m), ctypes.c_int32(iters), _p(cent), _p(loss), _p(assign))
    return cent, loss, assign


def route(codes, centroids, t: int):
    """t nearest centres per point by (d, c): (routes int32 [n, t], dists int32 [n, t])."""
    c = _codes(codes)
    ce = _codes(centroids)
    n, w = c.shape
    m = ce.shape[0]
    r = np.empty((n, t), np.int32)
    d = np.empty((n, t), np.int32)
    _load().or_route(_p(c), ctypes.c_int64(n), ctypes.c_int32(w), _p(ce), ctypes.c_int32(m),
                     ctypes.c_int32(t), _p(r), _p(d))
    return r, d


def routes_coarse(routes, m: int, coarse_num: int):
    """The coarse_num rule of Section 3.2 applied to t-nearest-centre routes
    [n, t]: (routes with the dropped slots set to -1, home counts int32 [m])."""
    rt = np.ascontiguousarray(routes, np.int32)
    n, t = rt.shape
    out = np.empty_like(rt)
    cnt = np.empty(m, np.int32)
    _load().or_routes_coarse(_p(rt), ctypes.c_int64(n), ctypes.c_int32(t), ctypes.c_int32(m),
                             ctypes.c_int64(coarse_num), _p(out), _p(cnt))
    return out, cnt


def routes_gap(routes, rdist, delta: int):
    """The distance-gap rule (not in the paper): t-nearest-centre routes [n, t]
    with every slot s >= 1 whose centre lies more than delta farther than the
    home's centre set to -1."""
    rt = np.ascontiguousarray(routes, np.int32)
    rd = np.ascontiguousarray(rdist, np.int32)
    n, t = rt.shape
    out = np.empty_like(rt)
    _load().or_routes_gap(_p(rt), _p(rd), ctypes.c_int64(n), ctypes.c_int32(t),
                          ctypes.c_int32(delta), _p(out))
    return out


def knn_partitioned(codes, routes, k: int, qidx=None):
    """Divide-and-conquer graph rows of points qidx given routes [n, t] (slot 0 =
    home; a slot holding -1 probes nothing)."""
    c = _codes(codes)
    n, w = c.shape
    rt = np.ascontiguousarray(routes, np.int32)
    t = rt.shape[1]
    q = np.arange(n, dtype=np.int64) if qidx is None else np.ascontiguousarray(qidx, np.int64)
    ids = np.empty((q.size, k), np.int32)
    dist = np.empty((q.size, k), np.int32)
    _load().or_knn_partitioned(_p(c), ctypes.c_int64(n), ctypes.c_int32(w), _p(rt),
                               ctypes.c_int32(t), ctypes.c_int32(k), _p(q),
                               ctypes.c_int64(q.size), _p(ids), _p(dist))
    return ids, dist


def propagate(codes, ids_in, k: int | None = None):
    """One round of neighbourhood propagation (Section 3.3): (ids, dists) int32 [n, k]."""
    c = _codes(codes)
    n, w = c.shape
    g = np.ascontiguousarray(ids_in, np.int32)
    k = g.shape[1] if k is None else k
    assert g.shape == (n, k)
    ids = np.empty((n, k), np.int32)
    dist = np.empty((n, k), np.int32)
    _load().or_propagate(_p(c), ctypes.c_int64(n), ctypes.c_int32(w), _p(g), ctypes.c_int32(k),
                         _p(ids), _p(dist))
    return ids, dist


def prune(codes, ids_in, L: int):
    """Occlusion pruning of Section 3.4 (FANNG's rule) of every row to at most L
    edges: (ids, dists) int32 [n, L]."""
    c = _codes(codes)
    n, w = c.shape
    g = np.ascontiguousarray(ids_in, np.int32)
    assert g.shape[0] == n
    k = g.shape[1]
    ids = np.empty((n, L), np.int32)
    dist = np.empty((n, L), np.int32)
    _load().or_prune(_p(c), ctypes.c_int64(n), ctypes.c_int32(w), _p(g), ctypes.c_int32(k),
                     ctypes.c_int32(L), _p(ids), _p(dist))
    return ids, dist


def search(codes, graph, entry, queries, ef, R: int):
    """Best-first search: (ids int32 [nq, R], dists int32 [nq, R], counters int64 [nq, 2])."""
    c = _codes(codes)
    n, w = c.shape
    g = np.ascontiguousarray(graph, np.int32)
    deg = g.shape[1]
    e = np.ascontiguousarray(entry, np.int32)
    qc = _codes(queries)
    nq = qc.shape[0]
    efa = np.ascontiguousarray(np.broadcast_to(np.asarray(ef, np.int32), (nq,)))
    ids = np.empty((nq, R), np.int32)
    dist = np.empty((nq, R), np.int32)
    cnt = np.empty((nq, 2), np.int64)
    _load().or_search(_p(c), ctypes.c_int64(n), ctypes.c_int32(w), _p(g), ctypes.c_int32(deg),
                      _p(e), ctypes.c_int32(e.size), _p(qc), ctypes.c_int64(nq), _p(efa),
                      ctypes.c_int32(R), _p(ids), _p(dist), _p(cnt))
    return ids, dist, cnt


def shard_offsets(n: int, S: int) -> np.ndarray:
    """Contiguous shards of Section 3.4: shard s holds points [off[s], off[s+1])
    with off[s] = floor(s * n / S)."""
    return np.array([(s * n) // S for s in range(S + 1)], np.int64)


def search_sharded(codes, graphs, entries, queries, ef, R: int):
    """Search over a multi-shard index (Sections 3.4 and 4): every shard s (its
    points codes[off[s]:off[s+1]], its own graph with local ids and its own
    entry sample) answers the query with ``search``; local ids become global
    (+ off[s]); the answer is the first min(ef, R) of all shards' keys by
    (d, global id), padded to R with (-1, bits + 1).
    Returns (ids, dists) int32 [nq, R]."""
    c = _codes(codes)
    S = len(graphs)
    off = shard_offsets(c.shape[0], S)
    qc = _codes(queries)
    nq, bits = qc.shape[0], 64 * c.shape[1]
    efa = np.broadcast_to(np.asarray(ef, np.int64), (nq,))
    parts = []
    for s in range(S):
        ids_s, d_s, _ = search(c[off[s]:off[s + 1]], graphs[s], entries[s], qc, ef, R)
        parts.append((np.where(ids_s >= 0, ids_s + off[s], -1), d_s))
    out_ids = np.full((nq, R), -1, np.int32)
    out_d = np.full((nq, R), bits + 1, np.int32)
    for q in range(nq):
        keys = [(int(d_s[q, r]), int(ids_s[q, r])) for ids_s, d_s in parts
                for r in range(R) if ids_s[q, r] >= 0]
        keys.sort()
        for r, (d, i) in enumerate(keys[:max(0, min(int(efa[q]), R))]):
            out_ids[q, r], out_d[q, r] = i, d
    return out_ids, out_d


def rerank(feats, qfeats, cand, k: int, precision: str = "f32"):
    """Re-rank candidates cand [nq, R] by squared L2: (ids int32 [nq, k], d [nq, k])."""
    f = np.ascontiguousarray(feats, np.float32)
    qf = np.ascontiguousarray(qfeats, np.float32)
    cd = np.ascontiguousarray(cand, np.int32)
    nq, R = cd.shape
    D = f.shape[1]
    ids = np.empty((nq, k), np.int32)
    if precision == "f32":
        d = np.empty((nq, k), np.float32)
        fn = _load().or_rerank_f32
    else:
        d = np.empty((nq, k), np.float64)
        fn = _load().or_rerank_f64
    fn(_p(f), ctypes.c_int32(D), _p(qf), _p(cd), ctypes.c_int64(nq), ctypes.c_int32(R),
       ctypes.c_int32(k), _p(ids), _p(d))
    return ids, d


def recall_ids(got, exact) -> float:
    """Eq. 3: mean over rows of |got_i intersect exact_i| / k (ids; -1 ignored)."""
    got = np.asarray(got)
    exact = np.asarray(exact)
    k = exact.shape[1]
    tot = 0
    for a, b in zip(got, exact):
        tot += len(set(a[a >= 0].tolist()) & set(b[b >= 0].tolist()))
    return tot / (k * exact.shape[0])


def recall_tie_aware(got_dist, exact_dist) -> float:
    """Tie-aware recall: a returned neighbour counts if its distance is below the
    exact k-th distance; neighbours at exactly the k-th distance count up to the
    number of such neighbours in the exact list (Eq. 3 with ties resolved by value)."""
    got_dist = np.asarray(got_dist)
    exact_dist = np.asarray(exact_dist)
    k = exact_dist.shape[1]
    dk = exact_dist[:, -1:]
    below = (got_dist < dk).sum(1)
    at = np.minimum((got_dist == dk).sum(1), (exact_dist == dk).sum(1))
    return float((below + at).sum() / (k * exact_dist.shape[0]))
