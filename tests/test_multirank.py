"""The bench's multi-GPU host logic on CPU: two gloo ranks (one process each)
rendezvous like torchrun ranks, build their own seeded inputs (independent
problems: weak scaling, no collective on the data path), and agree on the
slowest rank's time and the whole-job throughput."""
import hashlib
import os
import socket
import sys

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
