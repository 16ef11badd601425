"""Learned routing for the divide-and-conquer build: training data, the training
loop and the routes, on top of the C ABI (every step runs in libbdg.so kernels;
this module only orders the calls).

Training targets: for a seeded sample of points, their exact k nearest
neighbours within the sample (an exact, m = 1 build of the sample's codes) and
the home partition of each neighbour; the router learns to put probability on
the partitions where a point's neighbours live. Routes keep the nearest centre
as the home (slot 0) so the home sets H_p are the same as with exhaustive
routing; only the other P - 1 probed partitions come from the network.

With the code input (``prior_params``), the last layer also sees the point's
code as +-1 and starts with the centres in its code columns and zeros
elsewhere: the untrained router routes exactly like the nearest-centre rule,
and training moves it from there towards where the neighbours actually live.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import Router, build_graph, knn_rows


@dataclasses.dataclass
class TrainConfig:
    hidden: tuple = (512, 512)
    batch: int = 4096
    epochs: int = 4
    lr: float = 1e-3
    k_labels: int = 32


def prior_params(base_flat, d_in: int, h1: int, h2: int, m: int, centres, scale: float = 1.0):
    """Packed router parameters with a code input of the last layer: W1, b1, W2,
    b2 from ``base_flat`` (a packed d_in -> h1 -> h2 -> m vector), W3 =
    [0 | scale (2 c_p - 1) / 2] with c_p the bits of centre p, b3 = 0. The logits
    are then scale (bits / 2 - d(y, c_p)). centres: int64 [m, W] packed codes.
    A power-of-two scale keeps the BF16 weights and FP32 sums exact."""
    W = centres.shape[1]
    bits = 64 * W
    n12 = h1 * d_in + h1 + h2 * h1 + h2
    shifts = torch.arange(64, device=centres.device, dtype=torch.int64)
    cb = ((centres[:, :, None] >> shifts) & 1).reshape(m, bits).to(torch.float32)
    w3 = torch.cat([torch.zeros(m, h2, device=centres.device), scale * (cb - 0.5)], dim=1)
    return torch.cat([base_flat[:n12].to(centres.device, torch.float32), w3.reshape(-1),
                      torch.zeros(m, device=centres.device)]).contiguous()


def neighbour_labels_full(codes, rows, home, k: int, skip_home: bool = True):
    """Home partitions of the exact k nearest neighbours, over all N points, of
    the sample points ``rows`` (int32 [S]): int32 [S, k]. -1 marks a neighbour
    living in the point's own home partition (with skip_home)."""
    ids, _ = knn_rows(codes, rows, k)
    ids = ids.long()
    lab = torch.where(ids >= 0, home[ids.clamp(min=0)], torch.full_like(ids, -1))
    if skip_home:
        lab = torch.where(lab == home[rows.long()][:, None], torch.full_like(lab, -1), lab)
    return lab.to(torch.int32).contiguous()


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
                 log=None, codes=None, home=None) -> Router:
    """Train a router on (features, labels) with Adam for cfg.epochs epochs of
    shuffled batches (seeded order). With ``codes`` (int64 [S, W]) the last
    layer also takes the codes (init_params then holds W3 [m, h2 + 64 W], e.g.
    from prior_params). With ``home`` (int32 [S]) each row's home partition,
    probed anyway, is left out of its softmax. Returns the trained Router."""
    S, d = feats_bf16.shape
    h1, h2 = cfg.hidden
    B = min(cfg.batch, S - S % 8)
    cbits = 0 if codes is None else 64 * codes.shape[1]
    r = Router(init_params, d, h1, h2, m, max_batch=max(B, 8), code_bits=cbits)
    rng = np.random.default_rng(seed)
    for ep in range(cfg.epochs):
        order = torch.from_numpy(rng.permutation(S)).to(feats_bf16.device)
        last = None
        for s in range(0, S - B + 1, B):
            idx = order[s:s + B]
            cx = None if codes is None else codes[idx].contiguous()
            hx = None if home is None else home[idx].to(torch.int32).contiguous()
            last = r.train_step(feats_bf16[idx].contiguous(), labels[idx].contiguous(), cfg.lr,
                                codes=cx, exclude=hx)
        if log is not None and last is not None:
            log(ep, float(last.item()))
    return r


def learned_routes(router: Router, feats_bf16, home, P: int, codes=None):
    """int32 [N, P]: home first, then the router's P - 1 best other partitions."""
    return router.route(feats_bf16, home.to(torch.int32).contiguous(), P, codes=codes)


# ---------------------------------------------------------------------------
# Shortlist routing: the router scores only each point's Q nearest centres (the
# Map step's shortlist, slot 0 = home) and chooses how many of them to probe.
def train_router_shortlist(feats_bf16, codes, cand, labels, m: int, init_params,
                           cfg: TrainConfig, seed: int, log=None) -> Router:
    """Train the shortlist head (and the layers below it) with Adam on
    (features, codes, shortlist, labels): labels are the homes of each row's
    exact neighbours, home included. Seeded batch order. Returns the Router."""
    S, d = feats_bf16.shape
    h1, h2 = cfg.hidden
    B = min(cfg.batch, S - S % 8)
    r = Router(init_params, d, h1, h2, m, max_batch=max(B, 8), code_bits=64 * codes.shape[1])
    rng = np.random.default_rng(seed)
    for ep in range(cfg.epochs):
        order = torch.from_numpy(rng.permutation(S)).to(feats_bf16.device)
        last = None
        for s in range(0, S - B + 1, B):
            idx = order[s:s + B]
            last = r.train_step_shortlist(feats_bf16[idx].contiguous(), cand[idx].contiguous(),
                                          labels[idx].contiguous(), cfg.lr,
                                          codes=codes[idx].contiguous())
        if log is not None and last is not None:
            log(ep, float(last.item()))
    return r


def prior_scale_loss(feats_bf16, codes, cand, labels, m: int, base_flat, centres, scales,
                     hidden=(512, 512), batch: int = 4096):
    """Shortlist cross-entropy of the untrained prior (logits a (bits/2 - d)) at
    each scale a, on the first rows of the given set (no update): {a: loss}."""
    d = feats_bf16.shape[1]
    h1, h2 = hidden
    B = min(batch, feats_bf16.shape[0] - feats_bf16.shape[0] % 8)
    out = {}
    for a in scales:
        init = prior_params(base_flat, d, h1, h2, m, centres, scale=a)
        r = Router(init, d, h1, h2, m, max_batch=B, code_bits=64 * codes.shape[1])
        loss = r.train_step_shortlist(feats_bf16[:B].contiguous(), cand[:B].contiguous(),
                                      labels[:B].contiguous(), 0.0, apply_update=False,
                                      codes=codes[:B].contiguous())
        out[a] = float(loss.item())
        r.free()
    return out


def label_recall(routes, labels):
    """Share of the rows' labels (homes of their exact neighbours, -1 ignored)
    found among the rows' probed partitions: the id-based recall of a
    partitioned build for those rows (a neighbour is found exactly when its home
    is probed). routes: int32 [S, P] (-1 = none), labels: int32 [S, k]."""
    hit = (labels[:, :, None] == routes[:, None, :]) & (routes[:, None, :] >= 0)
    valid = labels >= 0
    return float((hit.any(2) & valid).sum().item()) / max(1, int(valid.sum().item()))


def tie_aware_recall(routes, ids, dists, home, k: int):
    """Tie-aware recall@k of a partitioned build for rows whose exact neighbour
    lists are known beyond k (ids/dists int32 [S, k'] with k' > k, ascending):
    a listed neighbour is found exactly when its home is probed; with d_k the
    exact k-th distance, the row's result counts the found neighbours below d_k
    plus, at d_k, as many found ones as the exact top k holds there (the listed
    neighbours stand in for all points at d_k). routes: int32 [S, P] (-1 = none)."""
    nh = home[ids.long().clamp(min=0)]
    found = ((nh[:, :, None] == routes[:, None, :]) & (routes[:, None, :] >= 0)).any(2)
    found &= ids >= 0
    dk = dists[:, k - 1:k]
    below = (found & (dists < dk)).sum(1)
    at_found = (found & (dists == dk)).sum(1)
    at_exact = (dists[:, :k] == dk).sum(1)
    return float((below + torch.minimum(at_found, at_exact)).sum().item()) / (ids.shape[0] * k)


def calibrate(choose, values, score, target: float):
    """The first value (in the given order, cheapest first) whose routes reach
    score(routes) >= target on the held-out rows; the last value if none does.
    choose(v) -> routes of the held-out rows. Returns (value, score, mean probes)."""
    best = None
    for v in values:
        r = choose(v)
        rec = score(r)
        best = (v, rec, float((r >= 0).sum(1).float().mean().item()))
        if rec >= target:
            break
    return best
