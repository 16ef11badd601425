"""Learned routing for the divide-and-conquer build: training data, the training
loop and the routes, on top of the C ABI (every step runs in libbdg.so kernels;
this module only orders the calls).

Training targets: for a seeded sample of points, their exact k nearest
neighbours within the sample (an exact, m = 1 build of the sample's codes) and
the home partition of each neighbour; the router learns to put probability on
the partitions where a point's neighbours live. Routes keep the nearest centre
as the home (slot 0) so the home sets H_p are the same as with exhaustive
routing; only the other P - 1 probed partitions come from the network.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import Router, build_graph


@dataclasses.dataclass
class TrainConfig:
    hidden: tuple = (512, 512)
    batch: int = 4096
    epochs: int = 4
    lr: float = 1e-3
    k_labels: int = 32


def neighbour_labels(codes_sample, home_sample, k: int, entry=None, skip_home: bool = True):
    """Home partitions of each sample point's exact k nearest neighbours within
    the sample: int32 [S, k]. -1 marks a missing neighbour and, with skip_home,
    a neighbour living in the point's own home partition: the home is always
    probed, so the router only has to learn where the other neighbours live."""
    if entry is None:
        entry = torch.zeros(1, dtype=torch.int32, device=codes_sample.device)
    g = build_graph(codes_sample, k, m=1, t=1, entry=entry)
    ids = g.ids.long()
    lab = torch.where(ids >= 0, home_sample[ids.clamp(min=0)], torch.full_like(ids, -1))
    if skip_home:
        lab = torch.where(lab == home_sample[:, None], torch.full_like(lab, -1), lab)
    out = lab.to(torch.int32).contiguous()
    g.free()
    return out


def train_router(feats_bf16, labels, m: int, init_params, cfg: TrainConfig, seed: int,
                 log=None) -> Router:
    """Train a router on (features, labels) with Adam for cfg.epochs epochs of
    shuffled batches (seeded order). Returns the trained Router."""
    S, d = feats_bf16.shape
    h1, h2 = cfg.hidden
    B = min(cfg.batch, S - S % 8)
    r = Router(init_params, d, h1, h2, m, max_batch=max(B, 8))
    rng = np.random.default_rng(seed)
    for ep in range(cfg.epochs):
        order = torch.from_numpy(rng.permutation(S)).to(feats_bf16.device)
        last = None
        for s in range(0, S - B + 1, B):
            idx = order[s:s + B]
            last = r.train_step(feats_bf16[idx].contiguous(), labels[idx].contiguous(), cfg.lr)
        if log is not None and last is not None:
            log(ep, float(last.item()))
    return r


def learned_routes(router: Router, feats_bf16, home, P: int):
    """int32 [N, P]: home first, then the router's P - 1 best other partitions."""
    return router.route(feats_bf16, home.to(torch.int32).contiguous(), P)
