"""MLP router oracle (float64, numpy) -- TEST INFRASTRUCTURE ONLY.

The paper routes each point to its t nearest binary centres (Section 3.2) and has
no learned router; this network is the learned alternative that picks the top-P
partitions instead. The oracle states the network and its gradients plainly:

  h1 = relu(x W1^T + b1)          x: [B, d_in]
  h2 = relu(h1 W2^T + b2)
  z  = [h2 | s] W3^T + b3         z: [B, m] logits, one per partition
  loss = -(1/B) sum_i sum_p q_ip log softmax(z_i)_p

where s is the point's code written as +-1 (a set bit is +1), an optional
input of the last layer (without it, z = h2 W3^T + b3). With the code columns
of W3 set to c_p / 2 (centre p as +-1) and everything else in W3 and b3 zero,
z_p = <s, c_p> / 2 = bits / 2 - d(y, c_p): the nearest-centre rule of
Section 3.2 written as logits.

with q_i the target distribution over partitions: the empirical distribution of
the partitions given as point i's labels (the homes of its exact neighbours).
A row without any label has no target and contributes neither loss nor
gradient. Optionally one partition per row (its home, which is probed anyway)
is left out: the softmax runs over the other partitions and labels naming it
are ignored. Gradients are the analytic chain rule;
``adam`` is Kingma & Ba's update with bias correction.

With ``bf16=True`` the float64 computation rounds to bfloat16 (round to nearest,
ties to even) exactly where a bf16 pipeline stores a tensor: the inputs, the
weights, h1, h2 and the logit gradient and hidden-layer gradients that feed the
backward products. Everything else stays float64.
"""
from __future__ import annotations

import numpy as np


def round_bf16(a) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def _q(a, bf16):
    return round_bf16(a) if bf16 else np.asarray(a, dtype=np.float64)


def code_pm(codes_u64, bits):
    """Packed codes (uint64 [n, bits/64], LSB-first) as +-1 float64 [n, bits]."""
    c = np.asarray(codes_u64, dtype=np.uint64)
    out = np.empty((c.shape[0], bits), np.float64)
    for b in range(bits):
        bit = (c[:, b // 64] >> np.uint64(b % 64)) & np.uint64(1)
        out[:, b] = np.where(bit == 1, 1.0, -1.0)
    return out


def forward(params, x, bf16=True, s=None):
    """Returns (z, cache). params: dict W1,b1,W2,b2,W3,b3 (float arrays);
    s: optional +-1 code input [B, cb] of the last layer (W3 is then [m, h2 + cb])."""
    W1, W2, W3 = (_q(params[k], bf16) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (np.asarray(params[k], np.float64) for k in ("b1", "b2", "b3"))
    x = _q(x, bf16)
    a1 = x @ W1.T + b1
    h1 = _q(np.maximum(a1, 0.0), bf16)
    a2 = h1 @ W2.T + b2
    h2 = _q(np.maximum(a2, 0.0), bf16)
    u = h2 if s is None else np.concatenate([h2, np.asarray(s, np.float64)], axis=1)
    z = u @ W3.T + b3
    return z, dict(x=x, h1=h1, h2=h2, u=u, W1=W1, W2=W2, W3=W3)


def softmax(z):
    z = np.asarray(z, np.float64)
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def loss_and_grads(params, x, q, bf16=True, s=None, exclude=None):
    """Mean soft-target cross-entropy and its gradients w.r.t. every parameter.
    exclude: optional int [B], a partition per row left out of its softmax (q must
    be zero there, e.g. from label_targets with the same exclude)."""
    z, c = forward(params, x, bf16, s)
    B = z.shape[0]
    zs = z.copy()
    if exclude is not None:
        zs[np.arange(B), np.asarray(exclude)] = -np.inf
    p = softmax(zs)
    q = np.asarray(q, np.float64)
    has = (q.sum(axis=1) > 0)[:, None]  # rows with a target
    logp = np.log(np.maximum(p, 1e-300))
    loss = float(-np.where(q > 0, q * logp, 0.0).sum() / B)
    dz = (p - q) / B * has
    dzq = _q(dz, bf16)
    g = {}
    g["W3"] = dzq.T @ c["u"]
    g["b3"] = dz.sum(0)
    h2n = c["h2"].shape[1]
    dh2 = (dzq @ c["W3"][:, :h2n]) * (c["h2"] > 0)
    dh2q = _q(dh2, bf16)
    g["W2"] = dh2q.T @ c["h1"]
    g["b2"] = dh2.sum(0)
    dh1 = (dh2q @ c["W2"]) * (c["h1"] > 0)
    dh1q = _q(dh1, bf16)
    g["W1"] = dh1q.T @ c["x"]
    g["b1"] = dh1.sum(0)
    return loss, g, z


def adam(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (bias-corrected) on float64 copies; returns new params, state."""
    t = state.get("t", 0) + 1
    newp, news = {}, {"t": t}
    for k, w in params.items():
        gk = np.asarray(grads[k], np.float64)
        m = beta1 * state.get("m_" + k, 0.0) + (1 - beta1) * gk
        v = beta2 * state.get("v_" + k, 0.0) + (1 - beta2) * gk * gk
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        newp[k] = np.asarray(w, np.float64) - lr * mh / (np.sqrt(vh) + eps)
        news["m_" + k], news["v_" + k] = m, v
    return newp, news


def topp(z, P):
    """First P partitions of sort over (-z_p, p) per row."""
    z = np.asarray(z, np.float64)
    out = np.empty((z.shape[0], P), np.int32)
    for i, row in enumerate(z):
        order = np.lexsort((np.arange(row.size), -row))
        out[i] = order[:P]
    return out


def label_targets(labels, m, exclude=None):
    """q_ip = #{labels of row i equal to p} / #{valid labels of row i}, a label
    being valid when it is in [0, m) and not exclude[i] (a row without valid
    labels gets q = 0)."""
    labels = np.asarray(labels)
    B = labels.shape[0]
    q = np.zeros((B, m), np.float64)
    for i in range(B):
        ex = -1 if exclude is None else int(exclude[i])
        valid = [int(p) for p in labels[i] if 0 <= p < m and p != ex]
        for p in valid:
            q[i, p] += 1.0 / len(valid)
    return q


def neighbour_partition_targets(knn_ids, home, m):
    """Targets from neighbour lists: the labels are home(j) for the listed
    neighbours j (ids -1 ignored)."""
    knn_ids = np.asarray(knn_ids)
    labels = np.where(knn_ids >= 0, np.asarray(home)[np.maximum(knn_ids, 0)], -1)
    return label_targets(labels, m)


# ---------------------------------------------------------------------------
# Shortlist head. The router's last layer is evaluated only on a shortlist of
# candidate partitions per point: cand[i] = the Q nearest centres of point i in
# the order of Section 3.2's Map step (cand[i, 0] = its home), -1 = no
# candidate. Same parameters as above; only the softmax runs over the shortlist:
#
#   z_ij = [h2_i | s_i] . W3[cand_ij] + b3[cand_ij]      (j < Q, -inf where cand_ij < 0)
#   loss = -(1/B) sum_i sum_j q_ij log softmax(z_i)_j
#   q_ij = #{labels of i equal to cand_ij} / #{labels of i found in cand_i}
#
# A row none of whose labels is shortlisted has no target (no loss, no gradient).
# The logit gradient dz stays at full precision (the CUDA path keeps it in
# FP32); dh2 is rounded where the pipeline stores it (bf16), like the dense path.

def shortlist_forward(params, x, cand, bf16=True, s=None):
    """Shortlisted logits z [B, Q] (-inf for cand < 0) and the cache."""
    W1, W2, W3 = (_q(params[k], bf16) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (np.asarray(params[k], np.float64) for k in ("b1", "b2", "b3"))
    x = _q(x, bf16)
    h1 = _q(np.maximum(x @ W1.T + b1, 0.0), bf16)
    h2 = _q(np.maximum(h1 @ W2.T + b2, 0.0), bf16)
    u = h2 if s is None else np.concatenate([h2, np.asarray(s, np.float64)], axis=1)
    cand = np.asarray(cand)
    B, Q = cand.shape
    z = np.full((B, Q), -np.inf)
    for i in range(B):
        for j in range(Q):
            p = int(cand[i, j])
            if p >= 0:
                z[i, j] = u[i] @ W3[p] + b3[p]
    return z, dict(x=x, h1=h1, h2=h2, u=u, W1=W1, W2=W2, W3=W3)


def shortlist_targets(labels, cand):
    """q [B, Q]: the share of row i's labels naming cand[i, j], among its labels
    that name any shortlisted partition (zero row if none does)."""
    labels = np.asarray(labels)
    cand = np.asarray(cand)
    B, Q = cand.shape
    q = np.zeros((B, Q), np.float64)
    for i in range(B):
        hits = [j for lab in labels[i] for j in range(Q)
                if cand[i, j] >= 0 and int(lab) == int(cand[i, j])]
        for j in hits:
            q[i, j] += 1.0 / len(hits)
    return q


def shortlist_loss_and_grads(params, x, cand, q, bf16=True, s=None):
    """Mean soft-target cross-entropy over the shortlist and its gradients."""
    z, c = shortlist_forward(params, x, cand, bf16, s)
    cand = np.asarray(cand)
    B, Q = z.shape
    p = softmax(z)  # exp(-inf) = 0: a missing candidate gets probability 0
    q = np.asarray(q, np.float64)
    has = (q.sum(axis=1) > 0)[:, None]
    logp = np.log(np.maximum(p, 1e-300))
    loss = float(-np.where(q > 0, q * logp, 0.0).sum() / B)
    dz = (p - q) / B * has
    g = {"W3": np.zeros_like(c["W3"]), "b3": np.zeros(c["W3"].shape[0])}
    h2n = c["h2"].shape[1]
    dh2 = np.zeros_like(c["h2"])
    for i in range(B):
        for j in range(Q):
            pj = int(cand[i, j])
            if pj < 0:
                continue
            g["W3"][pj] += dz[i, j] * c["u"][i]
            g["b3"][pj] += dz[i, j]
            dh2[i] += dz[i, j] * c["W3"][pj, :h2n]
    dh2 = dh2 * (c["h2"] > 0)
    dh2q = _q(dh2, bf16)
    g["W2"] = dh2q.T @ c["h1"]
    g["b2"] = dh2.sum(0)
    dh1 = (dh2q @ c["W2"]) * (c["h1"] > 0)
    dh1q = _q(dh1, bf16)
    g["W1"] = dh1q.T @ c["x"]
    g["b1"] = dh1.sum(0)
    return loss, g, z


def shortlist_select(z, cand, theta, pmax):
    """Partitions probed per point (int32 [B, pmax], -1 = none): slot 0 is
    cand[i, 0] (the home, always probed); then the other shortlisted partitions
    whose logit is within theta of the row's largest shortlisted logit, by
    (-z, partition) ascending, at most pmax - 1 of them. The comparison is made
    in the precision of z (float32 logits give float32 decisions)."""
    z = np.asarray(z)
    cand = np.asarray(cand)
    B, Q = z.shape
    out = np.full((B, pmax), -1, np.int32)
    for i in range(B):
        out[i, 0] = cand[i, 0]
        valid = [j for j in range(Q) if cand[i, j] >= 0]
        zmax = max(z[i, j] for j in valid)
        thr = zmax - z.dtype.type(theta)
        keep = [j for j in valid if j >= 1 and z[i, j] >= thr]
        keep.sort(key=lambda j: (-z[i, j], int(cand[i, j])))
        for r, j in enumerate(keep[:pmax - 1]):
            out[i, 1 + r] = cand[i, j]
    return out
