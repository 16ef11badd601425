"""Python binding of the B300 Binary Distributed Graph library (include/bdg.h).

Argument marshalling only: every step of the build and the search runs in the
CUDA kernels of libbdg.so. torch supplies device memory and the current CUDA
stream. The library must be built (``paper_2102_04656_b300.build.build()``);
importing works without it, but every call raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

__all__ = [
    "BDGError", "lib", "route", "bkmeans", "build_graph", "Graph", "search", "rerank",
    "search_rerank", "load_graph", "set_memory_budget", "memory_in_use", "knn_rows",
    "launch_count", "gemm_bf16", "Router", "Server", "BuildPlan",
]

_LIB = None
_c_void_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


class BDGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bdg status {status}: {msg}")
        self.status = status


class _Partitions(ctypes.Structure):
    _fields_ = [
        ("m", _i32), ("t", _i32), ("centroids", _c_void_p), ("bk_sample", _c_void_p),
        ("bk_sample_size", _i64), ("bk_iters", _i32), ("routes", _c_void_p),
        ("entry", _c_void_p), ("n_entry", _i32), ("tile_visitors", _i32), ("kernel", _i32),
        ("coarse_num", _i64), ("class_kernel", _i32 * 3),
    ]


def lib():
    """Load libbdg.so from the package's _build folder (raises if it is not built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libbdg.so is not built ({_build.LIB}); run "
                              "paper_2102_04656_b300.build.build()")
        L = ctypes.CDLL(_build.LIB)
        L.bdg_last_error.restype = ctypes.c_char_p
        L.bdg_memory_in_use.restype = ctypes.c_uint64
        L.bdg_set_memory_budget.argtypes = [ctypes.c_uint64]
        L.bdg_route.argtypes = [_c_void_p, _i64, _i32, _c_void_p, _i32, _i32, _c_void_p,
                                _c_void_p, _c_void_p]
        L.bdg_routes_coarse.argtypes = [_c_void_p, _i64, _i32, _i32, _i64, _c_void_p, _c_void_p]
        L.bdg_routes_gap.argtypes = [_c_void_p, _c_void_p, _i64, _i32, _i32, _c_void_p]
        L.bdg_merge_lists.argtypes = [_c_void_p, _c_void_p, _i32, _i64, _i32, _i32, _c_void_p,
                                      _c_void_p, _c_void_p]
        L.bdg_bkmeans.argtypes = [_c_void_p, _i64, _i32, _c_void_p, _i64, _i32, _i32, _c_void_p,
                                  _c_void_p, _c_void_p]
        L.bdg_build_graph.argtypes = [_c_void_p, _i64, _i32, _i32, ctypes.POINTER(_Partitions),
                                      _c_void_p, ctypes.POINTER(_c_void_p)]
        L.bdg_graph_info.argtypes = [_c_void_p, ctypes.POINTER(_c_void_p),
                                     ctypes.POINTER(_c_void_p), ctypes.POINTER(_i64),
                                     ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
        L.bdg_graph_free.argtypes = [_c_void_p]
        L.bdg_graph_free.restype = None
        L.bdg_graph_save.argtypes = [_c_void_p, ctypes.c_char_p]
        L.bdg_graph_load.argtypes = [ctypes.c_char_p, _c_void_p, ctypes.POINTER(_c_void_p)]
        L.bdg_search.argtypes = [_c_void_p, _c_void_p, _i64, _c_void_p, _i32, _i32, _c_void_p,
                                 _c_void_p, _c_void_p, _c_void_p]
        L.bdg_rerank.argtypes = [_c_void_p, _i64, _i32, _c_void_p, _c_void_p, _i64, _i32, _i32,
                                 _c_void_p, _c_void_p, _c_void_p]
        L.bdg_launch_count.restype = _i64
        L.bdg_profile_enable.argtypes = [_i32]
        L.bdg_profile_enable.restype = None
        L.bdg_profile_reset.restype = None
        L.bdg_profile_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(_i64)]
        L.bdg_knn_rows.argtypes = [_c_void_p, _i64, _i32, _c_void_p, _i64, _i32, _c_void_p,
                                   _c_void_p, _c_void_p]
        L.bdg_search_rerank.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i32, _i64,
                                        _c_void_p, _i32, _i32, _i32, _c_void_p, _c_void_p,
                                        _c_void_p, _c_void_p, _c_void_p]
        _LIB = L
    return _LIB


def _check(status: int):
    if status != 0:
        raise BDGError(status, lib().bdg_last_error().decode(errors="replace"))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name, ndim=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dims")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _codes(codes, name="codes"):
    _dev(codes, torch.int64, name, 2)  # raw 64-bit words (uint64 bit patterns)
    return codes, 64 * codes.shape[1]


def set_memory_budget(nbytes: int):
    _check(lib().bdg_set_memory_budget(int(nbytes)))


def memory_in_use() -> int:
    return int(lib().bdg_memory_in_use())


def route(codes, centroids, t: int, stream=None):
    """t nearest centres per point by (distance, centre): (routes, dists) int32 [n, t]."""
    codes, bits = _codes(codes)
    _codes(centroids, "centroids")
    n, m = codes.shape[0], centroids.shape[0]
    routes = torch.empty(n, t, dtype=torch.int32, device=codes.device)
    rdist = torch.empty(n, t, dtype=torch.int32, device=codes.device)
    _check(lib().bdg_route(_ptr(codes), n, bits, _ptr(centroids), m, t, _ptr(routes),
                           _ptr(rdist), _stream(stream)))
    return routes, rdist


def routes_coarse(routes, m: int, coarse_num: int, stream=None):
    """The coarse_num rule of Section 3.2 (bdg_routes_coarse) on routes int32
    [n, t], in place: the slots a point does not need become -1. Returns the
    home counts int32 [m]."""
    _dev(routes, torch.int32, "routes", 2)
    cnt = torch.empty(m, dtype=torch.int32, device=routes.device)
    _check(lib().bdg_routes_coarse(_ptr(routes), routes.shape[0], routes.shape[1], m, coarse_num,
                                   _ptr(cnt), _stream(stream)))
    return cnt


def routes_gap(routes, rdist, delta: int, stream=None):
    """The distance-gap rule (bdg_routes_gap) on routes int32 [n, t], in place:
    slots whose centre lies more than delta farther than the home's become -1."""
    _dev(routes, torch.int32, "routes", 2)
    _dev(rdist, torch.int32, "rdist", 2)
    if rdist.shape != routes.shape:
        raise ValueError("rdist must have the shape of routes")
    _check(lib().bdg_routes_gap(_ptr(routes), _ptr(rdist), routes.shape[0], routes.shape[1],
                                int(delta), _stream(stream)))
    return routes


def merge_lists(ids, dists, bits: int, stream=None):
    """First k of the union of S partial rows per point by (distance, id)
    (bdg_merge_lists): ids/dists int32 [S, n, k] (disjoint candidate sets, -1 =
    padding) -> (ids, dists) int32 [n, k]."""
    _dev(ids, torch.int32, "ids", 3)
    _dev(dists, torch.int32, "dists", 3)
    S, n, k = ids.shape
    oi = torch.empty(n, k, dtype=torch.int32, device=ids.device)
    od = torch.empty(n, k, dtype=torch.int32, device=ids.device)
    _check(lib().bdg_merge_lists(_ptr(ids), _ptr(dists), S, n, k, bits, _ptr(oi), _ptr(od),
                                 _stream(stream)))
    return oi, od


def knn_rows(codes, rows, k: int, stream=None):
    """Exact k-NN rows of the points ``rows`` over all codes: (ids, dists) int32 [nrows, k]."""
    codes, bits = _codes(codes)
    _dev(rows, torch.int32, "rows", 1)
    nr = rows.numel()
    ids = torch.empty(nr, k, dtype=torch.int32, device=codes.device)
    dist = torch.empty(nr, k, dtype=torch.int32, device=codes.device)
    _check(lib().bdg_knn_rows(_ptr(codes), codes.shape[0], bits, _ptr(rows), nr, k, _ptr(ids),
                              _ptr(dist), _stream(stream)))
    return ids, dist


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().bdg_launch_count())


def bkmeans(codes, sample, m: int, iters: int, stream=None):
    """Bk-means on codes[sample]: (centroids int64 [m, W], loss int64 [iters + 1])."""
    codes, bits = _codes(codes)
    _dev(sample, torch.int64, "sample", 1)
    cent = torch.empty(m, codes.shape[1], dtype=torch.int64, device=codes.device)
    loss = torch.empty(iters + 1, dtype=torch.int64, device=codes.device)
    _check(lib().bdg_bkmeans(_ptr(codes), codes.shape[0], bits, _ptr(sample), sample.numel(), m,
                             iters, _ptr(cent), _ptr(loss), _stream(stream)))
    return cent, loss


class _CudaArray:
    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": typestr, "data": (ptr, False), "version": 3,
            "strides": None, "stream": None,
        }
        self._owner = owner


class Graph:
    """A k-NN graph owned by the library (freed with the object). ``codes`` is
    borrowed and kept alive here."""

    def __init__(self, handle, codes, feats=None):
        self._h = ctypes.c_void_p(handle)
        self.codes = codes
        self.feats = feats
        ids, dists = ctypes.c_void_p(), ctypes.c_void_p()
        n, k, bits = _i64(), _i32(), _i32()
        _check(lib().bdg_graph_info(self._h, ctypes.byref(ids), ctypes.byref(dists),
                                    ctypes.byref(n), ctypes.byref(k), ctypes.byref(bits)))
        self.n, self.k, self.bits = n.value, k.value, bits.value
        dev = codes.device
        self.ids = torch.as_tensor(_CudaArray(ids.value, (self.n, self.k), "<i4", self), device=dev)
        self.dists = torch.as_tensor(_CudaArray(dists.value, (self.n, self.k), "<i4", self),
                                     device=dev)

    @property
    def handle(self):
        return self._h

    def save(self, path: str):
        _check(lib().bdg_graph_save(self._h, path.encode()))

    def free(self):
        """Release the device rows now; ``ids``/``dists`` become unusable."""
        if self._h is not None and self._h.value:
            self.ids = self.dists = None
            lib().bdg_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


KERNELS = {"auto": 0, "popc": 1, "tc": 2}


VARIANTS = {"follow": 0, "popc": 1, "tc": 2, "popc32": 3}


def build_graph(codes, k: int, m: int = 1, t: int = 1, centroids=None, bk_sample=None,
                bk_iters: int = 8, routes=None, entry=None, tile_visitors: int = 0,
                kernel: str = "auto", coarse_num: int = 0, class_kernel=None,
                stream=None) -> Graph:
    """Single-pass divide-and-conquer k-NN graph (exact when m == 1).

    kernel: "auto", "popc" (XOR + POPC) or "tc" (tcgen05 FP8 +-1 tensor cores).
    coarse_num > 0: each point probes the shortest prefix of its t nearest
    centres holding at least coarse_num points (Section 3.2).
    class_kernel: optional 3 variant names ("follow", "popc", "tc", "popc32"),
    one per partition size class (|H_p| >= 4096, 512..4095, < 512)."""
    codes, bits = _codes(codes)
    if entry is None:
        raise ValueError("entry (long-link sample ids, int32 CUDA tensor) is required")
    _dev(entry, torch.int32, "entry", 1)
    P = _Partitions()
    P.m, P.t = m, t
    P.centroids = None if centroids is None else _codes(centroids, "centroids")[0].data_ptr()
    P.bk_sample = None if bk_sample is None else _dev(bk_sample, torch.int64, "bk_sample",
                                                      1).data_ptr()
    P.bk_sample_size = 0 if bk_sample is None else bk_sample.numel()
    P.bk_iters = bk_iters
    P.routes = None if routes is None else _dev(routes, torch.int32, "routes", 2).data_ptr()
    P.entry = entry.data_ptr()
    P.n_entry = entry.numel()
    P.tile_visitors = tile_visitors
    P.kernel = KERNELS[kernel]
    P.coarse_num = coarse_num
    if class_kernel is not None:
        for i, v in enumerate(class_kernel):
            P.class_kernel[i] = VARIANTS[v]
    h = ctypes.c_void_p()
    _check(lib().bdg_build_graph(_ptr(codes), codes.shape[0], bits, k, ctypes.byref(P),
                                 _stream(stream), ctypes.byref(h)))
    return Graph(h.value, codes)


def propagate(g: Graph, rounds: int = 1, stream=None) -> Graph:
    """Neighbourhood propagation (see bdg_graph_propagate): a new Graph."""
    L = lib()
    if not getattr(L, "_prop_sigs", False):
        L.bdg_graph_propagate.argtypes = [_c_void_p, _i32, _c_void_p, ctypes.POINTER(_c_void_p)]
        L._prop_sigs = True
    h = ctypes.c_void_p()
    _check(L.bdg_graph_propagate(g._h, int(rounds), _stream(stream), ctypes.byref(h)))
    return Graph(h.value, g.codes)


def pack_codes(g: Graph, stream=None) -> Graph:
    """Store the neighbours' codes next to the graph's rows for faster search
    (see bdg_graph_pack_codes; N * k * bits / 8 bytes of device memory). Returns g."""
    lb = lib()
    if not getattr(lb, "_pack_sigs", False):
        lb.bdg_graph_pack_codes.argtypes = [_c_void_p, _c_void_p]
        lb._pack_sigs = True
    _check(lb.bdg_graph_pack_codes(g.handle, _stream(stream)))
    return g


def prune(g: Graph, L: int, stream=None) -> Graph:
    """Occlusion pruning to at most L edges per point (see bdg_graph_prune): a new Graph."""
    lb = lib()
    if not getattr(lb, "_prune_sigs", False):
        lb.bdg_graph_prune.argtypes = [_c_void_p, _i32, _c_void_p, ctypes.POINTER(_c_void_p)]
        lb._prune_sigs = True
    h = ctypes.c_void_p()
    _check(lb.bdg_graph_prune(g._h, int(L), _stream(stream), ctypes.byref(h)))
    return Graph(h.value, g.codes)


def load_graph(path: str, codes) -> Graph:
    codes, _ = _codes(codes)
    h = ctypes.c_void_p()
    _check(lib().bdg_graph_load(path.encode(), _ptr(codes), ctypes.byref(h)))
    return Graph(h.value, codes)


def search(g: Graph, queries, ef, R: int, ef_max: int | None = None, expansions: bool = False,
           stream=None):
    """Best-first graph search: (ids, dists) int32 [nq, R] (+ expansions int32 [nq])."""
    queries, _ = _codes(queries, "queries")
    _dev(ef, torch.int32, "ef", 1)
    nq = queries.shape[0]
    if ef_max is None:
        raise ValueError("ef_max (host bound on ef over the batch) is required")
    ids = torch.empty(nq, R, dtype=torch.int32, device=queries.device)
    dist = torch.empty(nq, R, dtype=torch.int32, device=queries.device)
    ex = torch.empty(nq, dtype=torch.int32, device=queries.device) if expansions else None
    _check(lib().bdg_search(g.handle, _ptr(queries), nq, _ptr(ef), ef_max, R, _ptr(ids),
                            _ptr(dist), _ptr(ex), _stream(stream)))
    return (ids, dist, ex) if expansions else (ids, dist)


def _shard_sigs(lb):
    if not getattr(lb, "_shard_sigs", False):
        lb.bdg_build_sharded.argtypes = [_c_void_p, _i64, _i32, _i32, ctypes.POINTER(_Partitions),
                                         _i32, _c_void_p, ctypes.POINTER(_c_void_p)]
        lb.bdg_search_sharded.argtypes = [ctypes.POINTER(_c_void_p), _i32, _c_void_p, _i64,
                                          _c_void_p, _i32, _i32, _c_void_p, _c_void_p, _c_void_p]
        lb._shard_sigs = True
    return lb


def shard_offsets(n: int, S: int) -> list:
    """Shard s of a multi-shard build holds points [off[s], off[s+1])."""
    return [(s * n) // S for s in range(S + 1)]


def build_sharded(codes, k: int, S: int, entries, m: int = 1, t: int = 1, centroids=None,
                  bk_sample=None, bk_iters: int = 8, kernel: str = "auto", coarse_num: int = 0,
                  stream=None) -> list:
    """Multi-shard build (bdg_build_sharded): S graphs over contiguous shards,
    Bk-means once. entries: int32 [S, n_entry] local entry ids per shard."""
    codes, bits = _codes(codes)
    _dev(entries, torch.int32, "entries", 2)
    if entries.shape[0] != S:
        raise ValueError("entries must hold one sample per shard")
    P = _Partitions()
    P.m, P.t = m, t
    P.centroids = None if centroids is None else _codes(centroids, "centroids")[0].data_ptr()
    P.bk_sample = None if bk_sample is None else _dev(bk_sample, torch.int64, "bk_sample",
                                                      1).data_ptr()
    P.bk_sample_size = 0 if bk_sample is None else bk_sample.numel()
    P.bk_iters = bk_iters
    P.routes = None
    P.entry = entries.data_ptr()
    P.n_entry = entries.shape[1]
    P.tile_visitors = 0
    P.kernel = KERNELS[kernel]
    P.coarse_num = coarse_num
    hs = (_c_void_p * S)()
    _check(_shard_sigs(lib()).bdg_build_sharded(_ptr(codes), codes.shape[0], bits, k,
                                                ctypes.byref(P), S, _stream(stream), hs))
    off = shard_offsets(codes.shape[0], S)
    return [Graph(hs[s], codes[off[s]:off[s + 1]]) for s in range(S)]


def search_sharded(graphs, queries, ef, R: int, ef_max: int, stream=None):
    """Search over a multi-shard index (bdg_search_sharded): (ids, dists) int32
    [nq, R] with global ids (shard s's ids offset by the earlier shards' sizes)."""
    queries, _ = _codes(queries, "queries")
    _dev(ef, torch.int32, "ef", 1)
    nq = queries.shape[0]
    ids = torch.empty(nq, R, dtype=torch.int32, device=queries.device)
    dist = torch.empty(nq, R, dtype=torch.int32, device=queries.device)
    hs = (_c_void_p * len(graphs))(*[g.handle for g in graphs])
    _check(_shard_sigs(lib()).bdg_search_sharded(hs, len(graphs), _ptr(queries), nq, _ptr(ef),
                                                 ef_max, R, _ptr(ids), _ptr(dist),
                                                 _stream(stream)))
    return ids, dist


def rerank(feats, qfeats, cand, k: int, stream=None):
    """FP32 squared-L2 re-rank of candidates: (ids int32 [nq, k], d2 float32 [nq, k])."""
    _dev(feats, torch.float32, "feats", 2)
    _dev(qfeats, torch.float32, "qfeats", 2)
    _dev(cand, torch.int32, "cand", 2)
    nq, R = cand.shape
    ids = torch.empty(nq, k, dtype=torch.int32, device=cand.device)
    d2 = torch.empty(nq, k, dtype=torch.float32, device=cand.device)
    _check(lib().bdg_rerank(_ptr(feats), feats.shape[0], feats.shape[1], _ptr(qfeats), _ptr(cand),
                            nq, R, k, _ptr(ids), _ptr(d2), _stream(stream)))
    return ids, d2


def search_rerank(g: Graph, queries, qfeats, feats, ef, R: int, k: int, ef_max: int,
                  stream=None):
    """Search then re-rank: (ids int32 [nq, k], d2 float32 [nq, k])."""
    queries, _ = _codes(queries, "queries")
    _dev(ef, torch.int32, "ef", 1)
    _dev(feats, torch.float32, "feats", 2)
    _dev(qfeats, torch.float32, "qfeats", 2)
    nq = queries.shape[0]
    dev = queries.device
    cand = torch.empty(nq, R, dtype=torch.int32, device=dev)
    cdist = torch.empty(nq, R, dtype=torch.int32, device=dev)
    ids = torch.empty(nq, k, dtype=torch.int32, device=dev)
    d2 = torch.empty(nq, k, dtype=torch.float32, device=dev)
    _check(lib().bdg_search_rerank(g.handle, _ptr(queries), _ptr(qfeats), _ptr(feats),
                                   feats.shape[1], nq, _ptr(ef), ef_max, R, k, _ptr(cand),
                                   _ptr(cdist), _ptr(ids), _ptr(d2), _stream(stream)))
    return ids, d2


# ----------------------------------------------------------------------------- router
def _router_sigs(L):
    if getattr(L, "_router_sigs", False):
        return
    L.bdg_gemm_bf16.argtypes = [_c_void_p, _c_void_p, _i32, _i32, _i32, _c_void_p, _c_void_p,
                                _i32, _c_void_p, _c_void_p, _c_void_p, _c_void_p, _c_void_p]
    L.bdg_router_create.argtypes = [_i32, _i32, _i32, _i32, _i32, _c_void_p, _i32,
                                    ctypes.POINTER(_c_void_p)]
    L.bdg_router_free.argtypes = [_c_void_p]
    L.bdg_router_free.restype = None
    L.bdg_router_info.argtypes = [_c_void_p, ctypes.POINTER(_c_void_p), ctypes.POINTER(_c_void_p),
                                  ctypes.POINTER(_i64), ctypes.POINTER(_c_void_p),
                                  ctypes.POINTER(_c_void_p)]
    L.bdg_router_forward.argtypes = [_c_void_p, _c_void_p, _c_void_p, _i32, _c_void_p,
                                     _c_void_p]
    L.bdg_router_train_step.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i32,
                                        _c_void_p, _i32, ctypes.c_float, _i32, _c_void_p]
    L.bdg_router_route.argtypes = [_c_void_p, _c_void_p, _c_void_p, _i64, _c_void_p, _i32,
                                   _c_void_p, _c_void_p]
    L.bdg_router_forward_shortlist.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i32,
                                               _i32, _c_void_p, _c_void_p]
    L.bdg_router_train_step_shortlist.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p,
                                                  _i32, _c_void_p, _i32, _i32, ctypes.c_float,
                                                  _i32, _c_void_p]
    L.bdg_router_route_shortlist.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i32,
                                             _i64, ctypes.c_float, _i32, _c_void_p, _c_void_p,
                                             _c_void_p, _c_void_p]
    L._router_sigs = True


def gemm_bf16(A, B, bias=None, mask=None, relu=False, out="f32", colsum=None, stream=None):
    """C = epilogue(A @ B^T) on the library's tcgen05 BF16 GEMM (FP32 accumulation)."""
    L = lib()
    _router_sigs(L)
    _dev(A, torch.bfloat16, "A", 2)
    _dev(B, torch.bfloat16, "B", 2)
    M, K = A.shape
    N = B.shape[0]
    dev = A.device
    of = torch.empty(M, N, dtype=torch.float32, device=dev) if out in ("f32", "both") else None
    ob = torch.empty(M, N, dtype=torch.bfloat16, device=dev) if out in ("bf16", "both") else None
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(L.bdg_gemm_bf16(_ptr(A), _ptr(B), M, N, K, _ptr(bias), _ptr(mask), int(relu),
                           _ptr(of), _ptr(ob), _ptr(colsum), _ptr(err), _stream(stream)))
    return (of if out == "f32" else ob if out == "bf16" else (of, ob)), err


class Router:
    """The BF16 MLP partition router (see include/bdg.h): d_in -> h1 -> h2, then
    [h2 | code as +-1] -> m logits (code_bits = 0: h2 -> m)."""

    def __init__(self, init_params, d_in: int, h1: int, h2: int, m: int, max_batch: int,
                 code_bits: int = 0):
        L = lib()
        _router_sigs(L)
        _dev(init_params, torch.float32, "init_params", 1)
        h = ctypes.c_void_p()
        _check(L.bdg_router_create(d_in, h1, h2, m, code_bits, _ptr(init_params), max_batch,
                                   ctypes.byref(h)))
        self._h = h
        self.d_in, self.h1, self.h2, self.m, self.max_batch = d_in, h1, h2, m, max_batch
        self.code_bits = code_bits
        p, g, lo, er = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        n = _i64()
        _check(L.bdg_router_info(h, ctypes.byref(p), ctypes.byref(g), ctypes.byref(n),
                                 ctypes.byref(lo), ctypes.byref(er)))
        dev = init_params.device
        self.n_params = n.value
        self.params = torch.as_tensor(_CudaArray(p.value, (n.value,), "<f4", self), device=dev)
        self.grads = torch.as_tensor(_CudaArray(g.value, (n.value,), "<f4", self), device=dev)
        self.loss = torch.as_tensor(_CudaArray(lo.value, (1,), "<f4", self), device=dev)
        self.err = torch.as_tensor(_CudaArray(er.value, (1,), "<i4", self), device=dev)

    def unpack(self, flat):
        """Split a packed parameter vector into W1, b1, W2, b2, W3, b3 views."""
        d, a, b, m = self.d_in, self.h1, self.h2, self.m
        bs = b + self.code_bits
        sizes = [a * d, a, b * a, b, m * bs, m]
        shapes = [(a, d), (a,), (b, a), (b,), (m, bs), (m,)]
        out, o = {}, 0
        for name, sz, sh in zip(["W1", "b1", "W2", "b2", "W3", "b3"], sizes, shapes):
            out[name] = flat[o:o + sz].view(*sh)
            o += sz
        return out

    def _codes(self, codes, n):
        if self.code_bits == 0:
            return None
        if codes is None:
            raise ValueError("this router takes the points' codes as input")
        _dev(codes, torch.int64, "codes", 2)
        if codes.shape[0] != n or codes.shape[1] * 64 != self.code_bits:
            raise ValueError(f"codes: expected [{n}, {self.code_bits // 64}]")
        return codes

    def forward(self, x, codes=None, stream=None):
        _dev(x, torch.bfloat16, "x", 2)
        c = self._codes(codes, x.shape[0])
        z = torch.empty(x.shape[0], self.m, dtype=torch.float32, device=x.device)
        _check(lib().bdg_router_forward(self._h, _ptr(x), _ptr(c), x.shape[0], _ptr(z),
                                        _stream(stream)))
        return z

    def train_step(self, x, labels, lr: float, apply_update: bool = True, codes=None,
                   exclude=None, stream=None):
        """exclude: optional int32 [B], a partition per row left out of its softmax."""
        _dev(x, torch.bfloat16, "x", 2)
        _dev(labels, torch.int32, "labels", 2)
        c = self._codes(codes, x.shape[0])
        if exclude is not None:
            _dev(exclude, torch.int32, "exclude", 1)
        _check(lib().bdg_router_train_step(self._h, _ptr(x), _ptr(c), _ptr(labels),
                                           labels.shape[1], _ptr(exclude), x.shape[0], float(lr),
                                           int(apply_update), _stream(stream)))
        return self.loss

    def route(self, x, home, P: int, codes=None, stream=None):
        _dev(x, torch.bfloat16, "x", 2)
        _dev(home, torch.int32, "home", 1)
        c = self._codes(codes, x.shape[0])
        routes = torch.empty(x.shape[0], P, dtype=torch.int32, device=x.device)
        _check(lib().bdg_router_route(self._h, _ptr(x), _ptr(c), x.shape[0], _ptr(home), P,
                                      _ptr(routes), _stream(stream)))
        return routes

    # ---- shortlist head: the last layer on each point's Q candidate partitions
    def _cand(self, cand, n):
        _dev(cand, torch.int32, "cand", 2)
        if cand.shape[0] != n:
            raise ValueError(f"cand: expected {n} rows")
        return cand

    def forward_shortlist(self, x, cand, codes=None, stream=None):
        """Logits of the shortlisted partitions: float32 [B, Q] (-inf where cand < 0)."""
        _dev(x, torch.bfloat16, "x", 2)
        B = x.shape[0]
        c = self._codes(codes, B)
        cand = self._cand(cand, B)
        z = torch.empty(B, cand.shape[1], dtype=torch.float32, device=x.device)
        _check(lib().bdg_router_forward_shortlist(self._h, _ptr(x), _ptr(c), _ptr(cand),
                                                  cand.shape[1], B, _ptr(z), _stream(stream)))
        return z

    def train_step_shortlist(self, x, cand, labels, lr: float, apply_update: bool = True,
                             codes=None, stream=None):
        """One step of softmax cross-entropy over each row's shortlist."""
        _dev(x, torch.bfloat16, "x", 2)
        _dev(labels, torch.int32, "labels", 2)
        B = x.shape[0]
        c = self._codes(codes, B)
        cand = self._cand(cand, B)
        _check(lib().bdg_router_train_step_shortlist(self._h, _ptr(x), _ptr(c), _ptr(cand),
                                                     cand.shape[1], _ptr(labels),
                                                     labels.shape[1], B, float(lr),
                                                     int(apply_update), _stream(stream)))
        return self.loss

    def route_shortlist(self, x, cand, theta: float, pmax: int, codes=None, logits=False,
                        order=None, stream=None):
        """Probed partitions int32 [N, pmax] (-1 = none): the home cand[:, 0], then
        the shortlisted partitions within theta of the largest shortlisted logit.
        With logits=True also returns the float32 [N, Q] logits. order: optional
        int32 [N] permutation the points are processed in (e.g. by home)."""
        _dev(x, torch.bfloat16, "x", 2)
        N = x.shape[0]
        c = self._codes(codes, N)
        cand = self._cand(cand, N)
        if order is not None:
            _dev(order, torch.int32, "order", 1)
            if order.numel() != N:
                raise ValueError("order must hold N entries")
        routes = torch.empty(N, pmax, dtype=torch.int32, device=x.device)
        z = (torch.empty(N, cand.shape[1], dtype=torch.float32, device=x.device)
             if logits else None)
        _check(lib().bdg_router_route_shortlist(self._h, _ptr(x), _ptr(c), _ptr(cand),
                                                cand.shape[1], N, float(theta), pmax,
                                                _ptr(order), _ptr(routes), _ptr(z),
                                                _stream(stream)))
        return (routes, z) if logits else routes

    def free(self):
        if self._h is not None and self._h.value:
            self.params = self.grads = self.loss = self.err = None
            lib().bdg_router_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ----------------------------------------------------------------------------- serving
class Server:
    """Continuous-batching search server (see bdg_server_* in include/bdg.h)."""

    def __init__(self, graph: Graph, feats, R: int, k: int, ef_max: int, max_batch: int = 4096,
                 n_streams: int = 4, memory_budget: int = 0):
        L = lib()
        if not getattr(L, "_server_sigs", False):
            L.bdg_server_create.argtypes = [_c_void_p, _c_void_p, _i32, _i32, _i32, _i32, _i32,
                                            _i32, ctypes.c_uint64, ctypes.POINTER(_c_void_p)]
            L.bdg_server_submit.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p, _i32,
                                            ctypes.POINTER(_i64)]
            L.bdg_server_wait.argtypes = [_c_void_p, _i64, _c_void_p, _c_void_p,
                                          ctypes.POINTER(ctypes.c_double), _i32]
            L.bdg_server_stats.argtypes = [_c_void_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                           ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_uint64)]
            L.bdg_server_free.argtypes = [_c_void_p]
            L.bdg_server_free.restype = None
            L._server_sigs = True
        _dev(feats, torch.float32, "feats", 2)
        self.graph, self.feats, self.k = graph, feats, k
        h = ctypes.c_void_p()
        _check(L.bdg_server_create(graph.handle, _ptr(feats), feats.shape[1], R, k, ef_max,
                                   max_batch, n_streams, int(memory_budget), ctypes.byref(h)))
        self._h = h

    def submit(self, queries, qfeats, ef) -> int:
        """queries int64/uint64 [nq, W], qfeats float32 [nq, D], ef int32 [nq] (host numpy)."""
        import numpy as np
        q = np.ascontiguousarray(queries).view(np.uint64)
        qf = np.ascontiguousarray(qfeats, dtype=np.float32)
        e = np.ascontiguousarray(ef, dtype=np.int32)
        rid = _i64()
        _check(lib().bdg_server_submit(self._h, q.ctypes.data_as(_c_void_p),
                                       qf.ctypes.data_as(_c_void_p), e.ctypes.data_as(_c_void_p),
                                       q.shape[0], ctypes.byref(rid)))
        return rid.value, q.shape[0]

    def wait(self, req, timeout_ms: int = 60000):
        """Returns (ids int32 [nq, k], d2 float32 [nq, k], latency_ms)."""
        import numpy as np
        rid, nq = req
        ids = np.empty((nq, self.k), np.int32)
        d2 = np.empty((nq, self.k), np.float32)
        lat = ctypes.c_double()
        _check(lib().bdg_server_wait(self._h, rid, ids.ctypes.data_as(_c_void_p),
                                     d2.ctypes.data_as(_c_void_p), ctypes.byref(lat), timeout_ms))
        return ids, d2, lat.value

    def stats(self):
        b, q, p = _i64(), _i64(), _i64()
        m = ctypes.c_uint64()
        _check(lib().bdg_server_stats(self._h, ctypes.byref(b), ctypes.byref(q), ctypes.byref(p),
                                      ctypes.byref(m)))
        return {"batches": b.value, "queries": q.value, "pending": p.value,
                "in_flight_bytes": m.value}

    def free(self):
        if self._h is not None and self._h.value:
            lib().bdg_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ----------------------------------------------------------------------------- build plans
class BuildPlan:
    """A build captured once into a CUDA graph (bdg_build_plan_*): run() replays
    the whole build; kernel "auto" lets the library's autotuner pick the Reduce-1
    kernel. Arrays passed here are re-read by every run and must stay alive."""

    def __init__(self, codes, k: int, m: int = 1, t: int = 1, centroids=None, bk_sample=None,
                 bk_iters: int = 8, routes=None, entry=None, kernel: str = "auto",
                 coarse_num: int = 0, stream=None):
        L = lib()
        if not getattr(L, "_plan_sigs", False):
            L.bdg_build_plan_create.argtypes = [_c_void_p, _i64, _i32, _i32,
                                                ctypes.POINTER(_Partitions), _c_void_p,
                                                ctypes.POINTER(_c_void_p)]
            L.bdg_build_plan_run.argtypes = [_c_void_p, _c_void_p]
            L.bdg_build_plan_run_host.argtypes = [_c_void_p, _c_void_p, _c_void_p, _c_void_p,
                                                  _c_void_p]
            L.bdg_build_plan_kernel_ms.argtypes = [_c_void_p, ctypes.POINTER(ctypes.c_float)]
            L.bdg_build_plan_info.argtypes = [_c_void_p, ctypes.POINTER(_c_void_p),
                                              ctypes.POINTER(_i32),
                                              ctypes.POINTER(ctypes.c_float),
                                              ctypes.POINTER(ctypes.c_float)]
            L.bdg_build_plan_classes.argtypes = [_c_void_p, ctypes.POINTER(_i32),
                                                 ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                                 ctypes.POINTER(ctypes.c_float)]
            L.bdg_build_plan_free.argtypes = [_c_void_p]
            L.bdg_build_plan_free.restype = None
            L._plan_sigs = True
        codes, bits = _codes(codes)
        _dev(entry, torch.int32, "entry", 1)
        self._keep = (codes, centroids, bk_sample, routes, entry)
        P = _Partitions()
        P.m, P.t = m, t
        P.centroids = None if centroids is None else centroids.data_ptr()
        P.bk_sample = None if bk_sample is None else bk_sample.data_ptr()
        P.bk_sample_size = 0 if bk_sample is None else bk_sample.numel()
        P.bk_iters = bk_iters
        P.routes = None if routes is None else routes.data_ptr()
        P.entry = entry.data_ptr()
        P.n_entry = entry.numel()
        P.tile_visitors = 0
        P.kernel = KERNELS[kernel]
        P.coarse_num = coarse_num
        h = ctypes.c_void_p()
        _check(L.bdg_build_plan_create(_ptr(codes), codes.shape[0], bits, k, ctypes.byref(P),
                                       _stream(stream), ctypes.byref(h)))
        self._h = h
        gp, kern = ctypes.c_void_p(), _i32()
        mp, mt = ctypes.c_float(), ctypes.c_float()
        _check(L.bdg_build_plan_info(h, ctypes.byref(gp), ctypes.byref(kern), ctypes.byref(mp),
                                     ctypes.byref(mt)))
        self.kernel = {1: "popc", 2: "tc"}[kern.value]
        self.tuned_ms = {"popc": mp.value, "tc": mt.value}
        var = (_i32 * 3)()
        lo, hi = (_i32 * 3)(), (_i32 * 3)()
        ms = (ctypes.c_float * 9)()
        _check(L.bdg_build_plan_classes(h, var, lo, hi, ms))
        names = {1: "popc", 2: "tc", 3: "popc32"}
        self.classes = [{"size_lo": lo[c], "size_hi": hi[c], "variant": names[var[c]],
                         "tuned_ms": {names[v + 1]: round(ms[v * 3 + c], 3) for v in range(3)
                                      if ms[v * 3 + c] >= 0}} for c in range(3)]
        self.graph = _PlanGraph(gp.value, codes, self)

    def run(self, stream=None):
        _check(lib().bdg_build_plan_run(self._h, _stream(stream)))

    def run_host(self, host_codes, host_ids, host_dists=None, stream=None):
        """One build from host memory (bdg_build_plan_run_host): host_codes int64
        [N, W] and host_ids / host_dists int32 [N, k] CPU tensors (page-locked for
        asynchronous copies); asynchronous on `stream`."""
        for t, nm, dt in ((host_codes, "host_codes", torch.int64),
                          (host_ids, "host_ids", torch.int32),
                          (host_dists, "host_dists", torch.int32)):
            if t is not None and (t.is_cuda or not t.is_contiguous() or t.dtype != dt):
                raise ValueError(f"{nm} must be a contiguous CPU {dt} tensor")
        if tuple(host_codes.shape) != tuple(self._keep[0].shape):
            raise ValueError("host_codes must have the shape of the plan's codes")
        if tuple(host_ids.shape) != (self.graph.n, self.graph.k):
            raise ValueError("host_ids must be [N, k]")
        if host_dists is not None and tuple(host_dists.shape) != tuple(host_ids.shape):
            raise ValueError("host_dists must be [N, k]")
        _check(lib().bdg_build_plan_run_host(self._h, ctypes.c_void_p(host_codes.data_ptr()),
                                             ctypes.c_void_p(host_ids.data_ptr()),
                                             None if host_dists is None else
                                             ctypes.c_void_p(host_dists.data_ptr()),
                                             _stream(stream)))

    def kernel_ms(self) -> float:
        ms = ctypes.c_float()
        _check(lib().bdg_build_plan_kernel_ms(self._h, ctypes.byref(ms)))
        return ms.value

    def free(self):
        if self._h is not None and self._h.value:
            self.graph = None
            lib().bdg_build_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _PlanGraph(Graph):
    """The graph owned by a build plan (freed with the plan, not on its own)."""

    def __init__(self, handle, codes, plan):
        super().__init__(handle, codes)
        self._plan = plan

    def free(self):
        self._h = None

    def __del__(self):
        pass
