"""Sharding of independent recompressions across GPUs (one process per GPU).

The pairs of a batch are independent (no data moves between them), so the
only multi-GPU step is the partition: pairs go to ranks by LPT (longest
processing time first: sort by predicted flops, give each pair to the rank
with the least load so far), which keeps the largest rank load within
4/3 - 1/(3 N) of the optimum (Graham 1969). Predicted flops follow the
Section 4 cost model with the clamped ranks. After the run one all-gather
collects every pair's status word and output ranks on every rank.
"""
from __future__ import annotations

from typing import List, Sequence

from . import costmodel


def pair_ranks(Y, Z, opts):
    """(n, r, s, ell) of one pair: mode sizes, bond ranks of Y and Z and the
    clamped sketch ranks of the plan (the reading of Algorithm 4's ranks the
    library uses: l_k = min(l_req, r_k s_k, left / right mode products), then
    l_k <= l_{k-1} n_{k-1} and l_k <= n_k l_{k+1})."""
    n = [int(c.shape[1]) for c in Y]
    r = [1] + [int(c.shape[2]) for c in Y]
    s = [1] + [int(c.shape[2]) for c in Z]
    d = len(n)
    if opts.get("sketch_rank", 0) > 0:
        lreq = int(opts["sketch_rank"])
    elif opts.get("max_rank", 0) > 0:
        lreq = int(opts["max_rank"]) + int(opts.get("oversample", 10))
    else:
        lreq = max(a * b for a, b in zip(r, s))
    ell = [1] * (d + 1)
    for k in range(1, d):
        left = right = 1
        for j in range(k):
            left *= n[j]
        for j in range(k, d):
            right *= n[j]
        ell[k] = min(lreq, r[k] * s[k], left, right)
    for k in range(1, d):
        ell[k] = min(ell[k], ell[k - 1] * n[k - 1])
    for k in range(d - 1, 0, -1):
        ell[k] = min(ell[k], n[k] * ell[k + 1])
    return n, r, s, ell


def predicted_flops(Y, Z, opts) -> float:
    n, r, s, ell = pair_ranks(Y, Z, opts)
    hp, sw = costmodel.hatt1_flops(n, r, s, ell)
    return hp + sw


def lpt_partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of `costs` split into `world` lists by LPT; ties go to the
    lowest rank, equal costs keep their input order (deterministic, so every
    rank computes the same partition without communicating)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        w = min(range(world), key=lambda q: (load[q], q))
        parts[w].append(i)
        load[w] += float(costs[i])
    return [sorted(p) for p in parts]


def gather_records(records, world: int, device=None):
    """All-gather of per-pair records (lists of ints: pair index, status,
    ranks...) from every rank; returns the concatenation in rank order. Uses
    the default process group (NCCL between GPUs, gloo on CPU)."""
    if world <= 1:
        return list(records)
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, list(records))
    merged = []
    for part in out:
        merged.extend(part)
    return merged
