"""GPU parity of the power iteration of Example 3 (largest entry of the Qing
and Alpine TTs) against the oracle's iteration with the same sketches."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import power as opower
from oracle import tt as ott
from paper_2410_04385_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def B():
    from paper_2410_04385_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    return binding


def to_gpu(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


@pytest.mark.parametrize("gfun", [wl.qing_grid, wl.alpine_grid])
def test_iterates_match_oracle(B, gfun):
    from paper_2410_04385_gb300 import power_iteration as pi
    Y = wl.separable_sum_tt(gfun(10))
    lams_g, Xg = pi.largest_entry(to_gpu(Y), iters=30, rank=5, seed=11)
    lams_o, Xo = opower.power_iteration_largest(Y, iters=30, rank=5, seed=11)
    lg = lams_g.cpu().numpy()
    assert np.allclose(lg, lams_o, rtol=1e-10, atol=0)
    X = [c.cpu().numpy() for c in Xg]
    assert ott.tt_diff_norm(X, Xo) <= 1e-10


def test_exact_sketch_gives_dense_power_iteration(B):
    from paper_2410_04385_gb300 import power_iteration as pi
    g = wl.alpine_grid(3)
    Y = wl.separable_sum_tt(g)
    y = ott.tt_full(Y).ravel()
    lams, _ = pi.largest_entry(to_gpu(Y), iters=12, rank=10)
    for t, lam in enumerate(lams.cpu().numpy()):
        assert lam == pytest.approx(np.sum(y ** (2 * t + 1)) / np.sum(y ** (2 * t)), rel=1e-12)


def test_scale_rejects_bad_arguments(B):
    lib = B.load()
    import ctypes
    assert lib.tt_scale(None, 4, None, None) == 3
    assert lib.tt_scale(None, -1, None, None) == 3
    assert lib.tt_scale(None, 0, None, None) == 0
