"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no distances, no selection, no clustering). Everything the
method itself draws at random (the Bk-means sample, the long-link entry sample,
the per-query ef mix) is produced here and passed to both sides as an input.

Workload recipe (stand-in for the paper's proprietary image features, Section 3.1
and Table 1, which are not available):
  * features x = mu_c + sigma * eps, c ~ U{0..C-1} (uniform weights),
    mu ~ N(0, 1)^D per component, eps ~ N(0, I_D), sigma = 0.3;
  * codes y_j = [<x, r_j> > 0] with r_j ~ N(0, I_D) seeded random projections
    (a stand-in for the learned LPH hash of Section 3.1);
  * bit j of a code lives in 64-bit word j // 64 at bit position j % 64
    (least-significant bit first), one row of W = bits / 64 words per point.
Seeds follow one scheme per workload: base seed for the mixture, +1 for the
projections, +2 for queries, +3 for the Bk-means sample, +4 for the entry
sample, +5 for the router, +6 for arrivals.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

__all__ = [
    "MixtureSpec", "mixture_features", "projections", "sign_pack",
    "make_codes", "sample_ids", "ef_mix", "unpack_bits", "random_codes",
    "WORKLOADS",
]


@dataclasses.dataclass(frozen=True)
class MixtureSpec:
    n: int
    dim: int
    components: int
    bits: int
    sigma: float = 0.3
    seed: int = 1000


# Named workloads (sizes of the paper-shaped synthetic inputs).
WORKLOADS = {
    # exact brute-force graph, N=20k, 128-d features -> 256-bit codes, k=32
    "exact_20k_256b": dict(spec=MixtureSpec(20_000, 128, 64, 256, seed=1000), k=32),
    # partitioned build, N=2M, 256-d features -> 512-bit codes, m=256, t=5, k=64
    "partitioned_2m_512b": dict(spec=MixtureSpec(2_000_000, 256, 1024, 512, seed=1001),
                                k=64, m=256, t=5, bk_iters=8),
    # learned-routed build, N=100M, 128-d -> 256-bit codes, m=10k, P=8, k=32
    "learned_100m_256b": dict(spec=MixtureSpec(100_000_000, 128, 4096, 256, seed=1002),
                              k=32, m=10_000, t=8, bk_iters=8),
    # graph search, N=10M, 128-d -> 256-bit codes, degree 32, 100k queries
    "search_10m_256b": dict(spec=MixtureSpec(10_000_000, 128, 4096, 256, seed=1003),
                            k=32, nq=100_000, efs=(64, 128, 256, 512), topk=10),
}


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def mixture_features(spec: MixtureSpec, device="cpu", n: int | None = None,
                     seed_offset: int = 0, chunk: int = 1 << 20):
    """Gaussian-mixture features, float32 [n, dim], and component labels int64 [n].

    The component centres always come from ``spec.seed`` so that queries drawn
    with another ``seed_offset`` (e.g. +2) come from the same mixture.
    """
    n = spec.n if n is None else n
    g_mu = _gen(spec.seed, device)
    mu = torch.randn(spec.components, spec.dim, generator=g_mu, device=device)
    g = _gen(spec.seed * 7919 + 17 + seed_offset, device)
    comp = torch.randint(0, spec.components, (n,), generator=g, device=device)
    x = torch.empty(n, spec.dim, dtype=torch.float32, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        eps = torch.randn(e - s, spec.dim, generator=g, device=device)
        x[s:e] = mu[comp[s:e]] + spec.sigma * eps
    return x, comp


def projections(spec: MixtureSpec, device="cpu") -> torch.Tensor:
    """Random projection matrix float32 [dim, bits], r_j ~ N(0, I)."""
    g = _gen(spec.seed + 1, device)
    return torch.randn(spec.dim, spec.bits, generator=g, device=device)


def sign_pack(x: torch.Tensor, r: torch.Tensor, chunk: int | None = None) -> torch.Tensor:
    """Pack [<x, r_j> > 0] into uint64-compatible int64 words, LSB-first.

    Returns an int64 tensor [n, bits // 64] holding the raw 64-bit patterns
    (view it as uint64 on the host with ``.numpy().view(np.uint64)``).
    """
    n, bits = x.shape[0], r.shape[1]
    assert bits % 64 == 0
    if chunk is None:
        chunk = (1 << 20) if x.is_cuda else (1 << 14)
    w = bits // 64
    out = torch.empty(n, w, dtype=torch.int64, device=x.device)
    shifts = torch.arange(64, device=x.device, dtype=torch.int64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        b = (x[s:e] @ r > 0).to(torch.int64).view(e - s, w, 64)
        out[s:e] = (b << shifts).sum(dim=2)  # disjoint powers of two: sum == OR
    return out


def make_codes(spec: MixtureSpec, device="cpu", n: int | None = None, seed_offset: int = 0,
               with_features: bool = False):
    """Features -> packed codes for a workload. Returns codes (int64 [n, W]) and
    optionally the float32 features."""
    x, _ = mixture_features(spec, device=device, n=n, seed_offset=seed_offset)
    r = projections(spec, device=device)
    codes = sign_pack(x, r)
    return (codes, x) if with_features else codes


def random_codes(n: int, bits: int, seed: int, device="cpu") -> torch.Tensor:
    """Uniformly random packed codes int64 [n, bits // 64] (for edge-case tests)."""
    g = _gen(seed, device)
    w = bits // 64
    lo = torch.randint(0, 1 << 32, (n, w), generator=g, device=device, dtype=torch.int64)
    hi = torch.randint(0, 1 << 32, (n, w), generator=g, device=device, dtype=torch.int64)
    return (hi << 32) | lo


def sample_ids(n: int, s: int, seed: int) -> np.ndarray:
    """First ``s`` ids of a seeded permutation of 0..n-1 (int64, host)."""
    rng = np.random.default_rng(seed)
    if s >= n:
        return rng.permutation(n).astype(np.int64)
    return rng.choice(n, size=s, replace=False).astype(np.int64)


def ef_mix(nq: int, choices, seed: int) -> np.ndarray:
    """Per-query ef drawn uniformly from ``choices`` (int32, host)."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(choices, dtype=np.int32), size=nq).astype(np.int32)


def unpack_bits(codes: np.ndarray, bits: int) -> np.ndarray:
    """[n, W] uint64 -> [n, bits] uint8 of 0/1 following the LSB-first layout."""
    c = np.ascontiguousarray(codes).view(np.uint64)
    n, w = c.shape
    sh = np.arange(64, dtype=np.uint64)
    b = (c[:, :, None] >> sh) & np.uint64(1)
    return b.reshape(n, w * 64)[:, :bits].astype(np.uint8)


def router_init(d_in: int, h1: int, h2: int, m: int, seed: int) -> np.ndarray:
    """Seeded initial router parameters, packed W1 b1 W2 b2 W3 b3 (float32):
    every weight and bias uniform in +-1/sqrt(fan_in)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((d_in, h1), (h1, h2), (h2, m)):
        bound = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, size=fan_out * fan_in))
        parts.append(rng.uniform(-bound, bound, size=fan_out))
    return np.concatenate(parts).astype(np.float32)
