"""Algorithmic flop counts of one HaTT-1 recompression (Section 4, Table 4.1).

Counts follow the paper's per-operation costs with the actual (clamped) ranks
of every core instead of uniform maxima:
  HPCRL-1 step k (W^{(k+1)} -> W^{(k)}):  n r s l' (2 r' + 2 s' - 2) + 2 n r s l' l - r s l
  left-to-right step k, m = l n rows:     m l' (2 r's' - 1)          (C W)
                                          4 m l'^2 - 4 l'^3 / 3      (econ QR, Q only)
                                          r's' l' (2 m - 1)          (M = Q^T C)
                                          n' r's' l' (2 r' + 2 s' - 2) (core update)
where primes denote the right bond of core k (or core k+1 for the update).
The truncation sweep added by this library is counted separately.
"""
from __future__ import annotations


def hatt1_flops(n, r, s, ell):
    """(hpcrl_flops, sweep_flops) for mode sizes n[0..d-1] and bond ranks
    r, s, ell[0..d] of Y, Z and the sketch."""
    d = len(n)
    hp = 0.0
    for k in range(1, d):
        rk, sk, lk = r[k], s[k], ell[k]
        r1, s1, l1 = r[k + 1], s[k + 1], ell[k + 1]
        hp += n[k] * rk * sk * l1 * (2 * r1 + 2 * s1 - 2) + 2.0 * n[k] * rk * sk * l1 * lk - rk * sk * lk
    sw = 0.0
    for k in range(d - 1):
        rows = ell[k] * n[k]
        lp = ell[k + 1]
        rsp = r[k + 1] * s[k + 1]
        sw += rows * lp * (2 * rsp - 1)
        sw += 4.0 * rows * lp * lp - 4.0 * lp ** 3 / 3.0
        sw += rsp * lp * (2 * rows - 1)
        sw += n[k + 1] * rsp * lp * (2 * r[k + 1] + 2 * s[k + 1] - 2)
    return hp, sw


def hatt1_contraction_flops(n, r, s, ell):
    """The part of hatt1_flops that the HaTT contractions themselves carry
    (HPCRL, C W, M = Q^T C, core update), i.e. everything but the QR term:
    the work of the launches the library tags as method products."""
    hp, sw = hatt1_flops(n, r, s, ell)
    d = len(n)
    for k in range(d - 1):
        rows = ell[k] * n[k]
        lp = ell[k + 1]
        sw -= 4.0 * rows * lp * lp - 4.0 * lp ** 3 / 3.0
    return hp + sw


def truncation_flops(n, ell):
    """Leading-order flops of the right-to-left truncation sweep as implemented:
    per core k >= 1 the Gram B B^T and the projection U^T B (2 l^2 N each,
    N = n_k l_{k+1}), about 18 l^3 for the eigen refinement, and the update of
    core k-1 (2 l_{k-1} n_{k-1} l^2)."""
    d = len(n)
    f = 0.0
    for k in range(1, d):
        l = ell[k]
        N = n[k] * ell[k + 1]
        f += 4.0 * l * l * N + 18.0 * l ** 3 + 2.0 * ell[k - 1] * n[k - 1] * l * l
    return f


def pkp_rounding_flops(n, r, s):
    """Table 4.1 TT-Rounding cost on the explicit PKP ranks r_k s_k (uniform
    leading-order form summed core by core): n (5 R^3 + 6 R^2 l + 2 R l^2) with
    R = r s and l the target rank taken as R (no truncation)."""
    d = len(n)
    f = 0.0
    for k in range(1, d - 1):
        R = r[k] * s[k]
        f += n[k] * (5.0 * R ** 3 + 6.0 * R ** 3 + 2.0 * R ** 3)
    return f
