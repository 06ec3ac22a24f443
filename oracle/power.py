"""Power iteration for the largest entry of a TT tensor (Section 5, Example 3;
the iteration of Espig et al. 2020), plain float64 numpy. TEST INFRASTRUCTURE
ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's baseline leg.

For a nonnegative tensor Y the map X -> Y ⊙ X is a diagonal operator whose
largest eigenvalue is max(Y), with an eigenvector concentrated on that entry.
Starting from the all-ones tensor (unit-normalized), each iteration forms
P = Y ⊙ X_t recompressed by HaTT-1 with sketch rank l (the paper uses l = 5),
takes the Rayleigh estimate lambda_t = <P, X_t> (X_t has unit norm), and
normalizes X_{t+1} = P / ||P||. Reading: the sketch of iteration t uses seed
`seed + t`; the paper states neither the seeds nor the estimate it reports,
and the Rayleigh quotient is the standard choice."""
from __future__ import annotations

import numpy as np

from . import hatt
from . import tt


def power_iteration_largest(Y, iters=100, rank=5, seed=0):
    """Returns (lambdas, X): the estimates lambda_0..lambda_{iters-1} of max(Y)
    and the last normalized iterate."""
    d = len(Y)
    n = [int(c.shape[1]) for c in Y]
    X = [np.ones((1, m, 1)) for m in n]
    X[0] = X[0] / np.sqrt(float(np.prod([float(m) for m in n])))
    lams = []
    for t in range(iters):
        P = hatt.hadamard_recompress(Y, X, sketch_rank=rank, seed=seed + t)
        lams.append(tt.tt_dot(P, X))
        nrm = tt.tt_norm(P)
        P = [np.array(c) for c in P]
        P[-1] = P[-1] / nrm
        X = P
    return lams, X


def separable_max(g):
    """max over the grid of sum_k g[k](x_k): the sum of the per-coordinate
    maxima (the terms are independent)."""
    return float(sum(np.max(v) for v in g))
