"""Power iteration for the largest entry of a TT tensor (Section 5, Example 3)
through the libhatt C ABI: X_0 = the all-ones tensor at unit norm, then for
t = 0, 1, ...: P = HaTT-1(Y ⊙ X_t) with sketch rank `rank` (seed + t),
lambda_t = <P, X_t> (the Rayleigh estimate of max(Y), X_t having unit norm),
X_{t+1} = P / ||P||. Every contraction, norm and scaling runs in the
library's kernels; this module only sequences the calls."""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import torch

from . import binding


def largest_entry(Y: Sequence[torch.Tensor], iters: int = 100, rank: int = 5, seed: int = 0,
                  precision: int = binding.TT_FP64) -> Tuple[torch.Tensor, List[torch.Tensor]]:
    """Y: CUDA float64 cores (r_k, n_k, r_{k+1}), Y >= 0. Returns the estimates
    lambda_0..lambda_{iters-1} (a CUDA float64 tensor) and the last iterate."""
    dev = Y[0].device
    n = [int(c.shape[1]) for c in Y]
    X = [torch.ones((1, m, 1), dtype=torch.float64, device=dev) for m in n]
    total = math.prod(float(m) for m in n)
    binding.tt_scale(X[0], torch.tensor([math.sqrt(total)], dtype=torch.float64, device=dev))
    lams = torch.empty(iters, dtype=torch.float64, device=dev)
    for t in range(iters):
        P = binding.tt_hadamard_recompress(Y, X, sketch_rank=rank, seed=seed + t,
                                           precision=precision)
        lams[t:t + 1].copy_(binding.tt_dot(P, X))
        binding.tt_scale(P[-1], binding.tt_norm(P))
        X = P
    return lams, X
