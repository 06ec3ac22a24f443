"""Pins for TT-Rounding (Algorithm 1) and the truncation rule."""
import numpy as np

from oracle import rounding, tt
from paper_2410_04385_gb300 import workloads as wl


def test_choose_rank_rule():
    s = np.array([10.0, 1.0, 0.1, 0.01])
    # tails: rho=1 -> 1+0.01+0.0001, rho=2 -> 0.0101, rho=3 -> 1e-4, rho=4 -> 0
    assert rounding.choose_rank(s, 0.0, 0) == 4
    assert rounding.choose_rank(s, 0.011, 0) == 3     # delta^2 = 1.21e-4 >= 1e-4
    assert rounding.choose_rank(s, 0.1, 0) == 3       # delta^2 = 0.01 < 0.0101
    assert rounding.choose_rank(s, 0.1006, 0) == 2    # delta^2 = 0.01012 >= 0.0101
    assert rounding.choose_rank(s, 1.0, 0) == 2       # delta^2 = 1 < 1.0101
    assert rounding.choose_rank(s, 1.01, 0) == 1      # delta^2 = 1.0201 >= 1.0101
    assert rounding.choose_rank(s, 0.0, 3) == 3
    assert rounding.choose_rank(np.zeros(3), 0.0, 0) == 1


def test_tt_round_exact_low_rank_matches_tt_svd_ranks():
    # sum of two rank-2 TTs padded to rank 8: true ranks are <= 4
    d, n = 5, 6
    A = tt.tt_add(wl.sin_sum_tt(d, n, "sin"), wl.sin_sum_tt(d, n, "cos"), 0.5)
    G = wl.gaussian_tt([n] * d, [1, 2, 2, 2, 2, 1], seed=9)
    A = tt.tt_add(A, G, 1.0)           # ranks 6, full-rank-ish part from G
    full = tt.tt_full(A)
    B, rk = rounding.tt_round(A, 0, 1e-13)
    ref = rounding.tt_svd(full, 0, 1e-13)
    assert rk == tt.ranks(ref)
    assert np.linalg.norm(tt.tt_full(B) - full) <= 1e-12 * np.linalg.norm(full)


def test_tt_round_tolerance_bound():
    d, n = 5, 5
    A = wl.gaussian_tt([n] * d, [1, 5, 6, 6, 5, 1], seed=10)
    full = tt.tt_full(A)
    for tol in (1e-1, 3e-1):
        B, rk = rounding.tt_round(A, 0, tol)
        err = np.linalg.norm(tt.tt_full(B) - full) / np.linalg.norm(full)
        assert err <= tol * (1 + 1e-10)
        # TT-SVD of the dense tensor with the same rule picks the same ranks
        ref = rounding.tt_svd(full, 0, tol)
        assert rk == tt.ranks(ref)


def test_tt_round_max_rank():
    A = wl.gaussian_tt([4] * 6, [1, 4, 6, 6, 6, 4, 1], seed=12)
    B, rk = rounding.tt_round(A, 3, 0.0)
    assert max(rk) == 3
    # rank-3 truncation is quasi-optimal: error at most sqrt(d-1) times the best per-bond tails
    full = tt.tt_full(A)
    err = np.linalg.norm(tt.tt_full(B) - full)
    tails = []
    for k in range(1, 6):
        sv = np.linalg.svd(full.reshape(4 ** k, -1), compute_uv=False)
        tails.append(np.sum(sv[3:] ** 2))
    assert err <= np.sqrt(np.sum(tails)) * (1 + 1e-10)
