"""The bench's multi-GPU host logic on CPU: two gloo ranks (one process each)
rendezvous like torchrun ranks, build their own seeded inputs (independent
problems: weak scaling, no collective on the data path), and agree on the
slowest rank's time and the whole-job throughput."""
import hashlib
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import datagen
    got_ws, got_rank, _ = bench._dist()
    assert (got_ws, got_rank) == (ws, rank)
    # each rank draws its own problem from a rank-shifted seed
    w = dict(datagen.WORKLOADS["exact_20k_256b"])
    w["spec"] = datagen.MixtureSpec(2000, 32, 8, 256, seed=5)
    w["m"] = 4
    _, codes, _, _ = bench._build_inputs(w, "cpu", seed_shift=rank)
    h = torch.tensor([int(hashlib.sha256(codes.numpy().tobytes()).hexdigest()[:12], 16)],
                     dtype=torch.int64)
    hs = [torch.zeros_like(h) for _ in range(ws)]
    dist.all_gather(hs, h)
    bench._barrier(ws)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    ms_max = bench._max_over_ranks(ms, ws, "cpu")
    out[rank] = (ms_max, bench._job_mpoints_per_s(2000, ws, ms_max), len({int(x) for x in hs}))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_job_throughput():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms_max, mpts, distinct = res[0]
    assert ms_max == 15.0
    assert mpts == pytest.approx(2000 * 2 / 0.015 / 1e6)
    assert distinct == 2  # the two ranks built different problems


# ---------------------------------------------------------------- partition-sharded build
def _merge_rows_np(ids, dists, k, bits):
    """Test double of the merge: first k of the union of the partial rows by
    (distance, id), padding (-1, bits + 1)."""
    S, n, _ = ids.shape
    out_i = np.full((n, k), -1, np.int32)
    out_d = np.full((n, k), bits + 1, np.int32)
    for i in range(n):
        keys = sorted((int(dists[s, i, j]), int(ids[s, i, j])) for s in range(S)
                      for j in range(ids.shape[2]) if ids[s, i, j] >= 0)[:k]
        for j, (d, x) in enumerate(keys):
            out_i[i, j], out_d[i, j] = x, d
    return out_i, out_d


def _sharded_rank_main(rank, ws, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist

    import datagen
    import oracle
    from paper_2102_04656_b300 import distributed as D
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    n, bits, k, m, t = 1500, 128, 8, 12, 3
    codes = datagen.make_codes(datagen.MixtureSpec(n, 32, 10, bits, seed=41))
    cn = codes.numpy().view(np.uint64)
    cent = datagen.random_codes(m, bits, seed=42).numpy().view(np.uint64)
    routes_np, _ = oracle.route(cn, cent, t)
    routes = torch.from_numpy(routes_np)

    def build_fn(c, k_, m_, t_, r, entry):  # the oracle stands in for the GPU build
        ids, d = oracle.knn_partitioned(cn, r.numpy(), k_)
        return torch.from_numpy(ids), torch.from_numpy(d)

    def merge_fn(pi, pd):
        i, d = _merge_rows_np(pi.numpy(), pd.numpy(), k, bits)
        return torch.from_numpy(i), torch.from_numpy(d)

    lo, ids, d = D.sharded_build(codes, k, m, routes, None, ws, rank, bits,
                                 build_fn=build_fn, merge_fn=merge_fn)
    out[rank] = (lo, ids.numpy().tolist(), d.numpy().tolist())
    dist.destroy_process_group()


def test_partition_sharded_build_on_two_gloo_ranks_equals_one_process():
    """Two ranks split the partitions by LPT, each builds its partitions' partial
    rows, one all-to-all hands every point's rows to its owner, the owner merges:
    the blocks put together equal the single-process graph (oracle) bit for bit."""
    import numpy as np

    import datagen
    import oracle
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_sharded_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    n, bits, k, m, t = 1500, 128, 8, 12, 3
    cn = datagen.make_codes(datagen.MixtureSpec(n, 32, 10, bits, seed=41)).numpy().view(np.uint64)
    cent = datagen.random_codes(m, bits, seed=42).numpy().view(np.uint64)
    r, _ = oracle.route(cn, cent, t)
    ids_o, d_o = oracle.knn_partitioned(cn, r, k)
    got_i = np.concatenate([np.array(res[rk][1], np.int32) for rk in range(ws)])
    got_d = np.concatenate([np.array(res[rk][2], np.int32) for rk in range(ws)])
    assert [res[rk][0] for rk in range(ws)] == [0, 750]
    assert np.array_equal(got_i, ids_o)
    assert np.array_equal(got_d, d_o)


def test_lpt_assignment_balances_work():
    """Every partition goes to one rank; partitions in decreasing work each to the
    least loaded rank: no rank ends above the least loaded one by more than the
    largest single item, and a hand-worked case."""
    import numpy as np

    from paper_2102_04656_b300.distributed import assign_partitions
    # work 10, 9, 8, 7, 1 over 2 ranks: 10 -> r0, 9 -> r1, 8 -> r1 (9 < 10), 7 -> r0, 1 -> r0
    own = assign_partitions([10, 9, 8, 7, 1], [1, 1, 1, 1, 1], 2)
    assert own.tolist() == [0, 1, 1, 0, 0]
    rng = np.random.default_rng(3)
    hc, vc = rng.integers(0, 5000, 300), rng.integers(0, 20000, 300)
    for world in (2, 3, 8):
        own = assign_partitions(hc, vc, world)
        load = np.bincount(own, weights=hc.astype(float) * vc, minlength=world)
        assert load.max() - load.min() <= (hc.astype(float) * vc).max()
        assert set(own.tolist()) <= set(range(world))
