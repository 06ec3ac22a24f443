"""TT-Rounding (Algorithm 1, after Oseledets 2011) and the truncation rule.

Reading of Algorithm 1: the right-to-left pass is an LQ factorization of
H(B_k) (a QR of its transpose) that pushes the triangular factor into core
k-1. The left-to-right pass QR-factors V(B_k), truncates the SVD of the
triangular factor and multiplies Sigma V^T into the *orthogonalized* core
B_{k+1} produced by the first pass (the printed line uses A_{k+1}, which would
discard the orthogonalization; the standard algorithm uses B_{k+1}).

Truncation rule (the paper is fixed-rank only; the tolerance form follows
Oseledets): with delta = tol * ||A||_F / sqrt(d-1), keep at each bond the
smallest rank rho >= 1 whose discarded tail sum_{i>=rho} sigma_i^2 <= delta^2,
then cap rho by max_rank.
"""
from __future__ import annotations

import numpy as np

from .tt import H, V


def choose_rank(sigma, delta, max_rank):
    """Smallest rho >= 1 with sum_{i >= rho} sigma_i^2 <= delta^2, capped by
    max_rank (sigma sorted in decreasing order)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    m = sigma.size
    if m == 0:
        return 0
    sq = sigma ** 2
    # tail[rho] = sum_{i >= rho} sigma_i^2, tail[m] = 0
    tail = np.concatenate([np.cumsum(sq[::-1])[::-1], [0.0]])
    rho = m
    for cand in range(1, m + 1):
        if tail[cand] <= delta * delta:
            rho = cand
            break
    if max_rank is not None and max_rank > 0:
        rho = min(rho, int(max_rank))
    return max(1, rho)


def tt_round(A, max_rank=0, tol=0.0):
    """Algorithm 1: right-to-left orthogonalization, then left-to-right
    QR + truncated SVD. Returns (cores, ranks)."""
    d = len(A)
    B = [np.array(c, dtype=np.float64) for c in A]
    if d == 1:
        return B, [1, 1]
    # right-to-left orthogonalization: H(B_k) = L Q^T
    for k in range(d - 1, 0, -1):
        a, n, b = B[k].shape
        q, r = np.linalg.qr(H(B[k]).T)          # H(B_k)^T = Q R
        B[k] = q.T.reshape(q.shape[1], n, b)
        B[k - 1] = np.einsum("aib,cb->aic", B[k - 1], r)   # V(B_{k-1}) R^T
    nrm = float(np.linalg.norm(B[0]))
    delta = tol * nrm / np.sqrt(d - 1)
    for k in range(d - 1):
        a, n, b = B[k].shape
        q, r = np.linalg.qr(V(B[k]))
        u, s, vt = np.linalg.svd(r, full_matrices=False)
        rho = choose_rank(s, delta, max_rank)
        B[k] = (q @ u[:, :rho]).reshape(a, n, rho)
        B[k + 1] = np.einsum("ab,bic->aic", s[:rho, None] * vt[:rho], B[k + 1])
    return B, [1] + [int(c.shape[2]) for c in B]


def tt_svd(full, max_rank=0, tol=0.0):
    """TT-SVD of a dense tensor (sequential truncated SVDs of unfoldings,
    Oseledets 2011), with the same truncation rule. Tiny cases only."""
    shape = full.shape
    d = len(shape)
    nrm = float(np.linalg.norm(full))
    delta = tol * nrm / np.sqrt(max(d - 1, 1))
    cores = []
    c = full.reshape(1, -1)
    rprev = 1
    for k in range(d - 1):
        c = c.reshape(rprev * shape[k], -1)
        u, s, vt = np.linalg.svd(c, full_matrices=False)
        rho = choose_rank(s, delta, max_rank)
        cores.append(u[:, :rho].reshape(rprev, shape[k], rho))
        c = s[:rho, None] * vt[:rho]
        rprev = rho
    cores.append(c.reshape(rprev, shape[-1], 1))
    return cores
