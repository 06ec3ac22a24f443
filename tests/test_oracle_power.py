"""Pins of the oracle's power iteration (Example 3)."""
import numpy as np
import pytest

from oracle import power as opower
from oracle import tt as ott
from paper_2410_04385_gb300 import workloads as wl


@pytest.mark.parametrize("gfun", [wl.qing_grid, wl.alpine_grid])
def test_separable_max_is_the_brute_force_max(gfun):
    g = gfun(4)
    full = ott.tt_full(wl.separable_sum_tt(g))
    assert np.max(full) == pytest.approx(opower.separable_max(g), rel=1e-14)


def test_exact_sketch_reproduces_dense_power_iteration():
    """With a sketch that covers every bond (d = 3, n = 10: l = 10) each
    recompression is exact, so X_t is the dense y^t normalized and the
    estimate must be lambda_t = sum y^(2t+1) / sum y^(2t)."""
    g = wl.alpine_grid(3)
    Y = wl.separable_sum_tt(g)
    y = ott.tt_full(Y).ravel()
    lams, X = opower.power_iteration_largest(Y, iters=12, rank=10)
    for t, lam in enumerate(lams):
        expect = np.sum(y ** (2 * t + 1)) / np.sum(y ** (2 * t))
        assert lam == pytest.approx(expect, rel=1e-12)
    xt = y ** 12 / np.linalg.norm(y ** 12)
    assert np.allclose(ott.tt_full(X).ravel(), xt, atol=1e-12)


def test_rank5_iteration_approaches_the_max():
    g = wl.alpine_grid(4)
    lams, _ = opower.power_iteration_largest(wl.separable_sum_tt(g), iters=100, rank=5)
    true = opower.separable_max(g)
    assert abs(lams[-1] - true) <= 1e-3 * true
    assert abs(lams[-1] - true) < abs(lams[9] - true)
