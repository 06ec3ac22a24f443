"""GPU parity of HaTT-2 (HPCRL-2, Eq. (3.7)) through the C ABI against the
FP64 oracle, which takes a full SVD of every W^{(k)}.

The GPU path reads the singular values off the Gram matrix W^T W, so a cut
decision can only differ from the oracle's when a ratio sigma_j / sigma_1
lies within rounding of ep: every case checks, with the oracle's singular
values, that each ratio is at least 1e-3 away from ep (relatively), so both
sides keep the same terms. Tensors are compared (gauges are not unique),
relative Frobenius difference <= 1e-10: the kept directions agree to
~1e-15 / gap, and the result is that of the same rank-R sketches.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hatt as ohatt
from oracle import philox as ophilox
from oracle import tt as ott
from paper_2410_04385_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

REL_TOL = 1e-10


@pytest.fixture(scope="module")
def B():
    from paper_2410_04385_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    return binding


def to_gpu(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def run_gpu(B, Y, Z, **opts):
    return [c.cpu().numpy() for c in B.tt_hadamard_recompress(to_gpu(Y), to_gpu(Z), **opts)]


def rel_diff(X, A):
    return ott.tt_diff_norm(X, A) / max(ott.tt_norm(A), 1e-300)


def cut_margin(Y, Z, sketch_rank, seed, ep):
    """Smallest |sigma_j / sigma_1 / ep - 1| over the matrices HPCRL-2 cuts,
    the kept ranks, and the largest condition number of a tall sketch."""
    n = [c.shape[1] for c in Y]
    ell = ohatt.plan_ranks(n, ott.ranks(Y), ott.ranks(Z), sketch_rank)
    W, kept = ohatt.hpcrl2(Y, Z, ophilox.sketch_tt(seed, n, ell), ep)
    m, cond = np.inf, 1.0
    for k in range(1, len(Y)):
        sv = np.linalg.svd(W[k], compute_uv=False)
        if k >= 2:
            m = min(m, float(np.min(np.abs(sv / sv[0] / ep - 1.0))))
        if W[k].shape[0] >= W[k].shape[1]:
            cond = max(cond, float(sv[0] / max(sv[-1], 1e-300)))
    return m, kept, cond


def small_random():
    n = [6, 5, 7, 4, 6, 5]
    return (wl.gaussian_tt(n, [1, 4, 5, 6, 5, 3, 1], 11),
            wl.gaussian_tt(n, [1, 3, 4, 3, 4, 2, 1], 12))


def test_hatt2_ep_zero_equals_hatt1(B):
    """P6 on the GPU: ep = 0 keeps every term."""
    Y, Z = small_random()
    X1 = run_gpu(B, Y, Z, sketch_rank=12, seed=3)
    X2 = run_gpu(B, Y, Z, sketch_rank=12, seed=3, variant=2, ep=0.0)
    A = ohatt.hadamard_recompress(Y, Z, sketch_rank=12, seed=3)
    assert rel_diff(X2, X1) <= 1e-12
    assert rel_diff(X2, A) <= 1e-12


@pytest.mark.parametrize("which", ["random", "sin"])
@pytest.mark.parametrize("ep,sketch", [(3e-2, 12), (0.3, 12), (0.3, 6), (0.95, 4)])
@pytest.mark.parametrize("seed", [0, 1])
def test_hatt2_matches_oracle(B, which, ep, sketch, seed):
    """The sketches must keep full column rank for the result to be unique
    (checked: condition number < 1e6); with a rank-deficient sketch the QR
    completes the basis arbitrarily (next test)."""
    if which == "random":
        Y, Z = small_random()
    else:
        Y, Z, _ = wl.workload_small_sin_times_random()
    margin, kept, cond = cut_margin(Y, Z, sketch, seed, ep)
    assert margin > 1e-3 and cond < 1e6
    X = run_gpu(B, Y, Z, sketch_rank=sketch, seed=seed, variant=2, ep=ep)
    A = ohatt.hadamard_recompress(Y, Z, sketch_rank=sketch, seed=seed, variant=2, ep=ep)
    assert rel_diff(X, A) <= REL_TOL


@pytest.mark.parametrize("which", ["random", "sin"])
def test_hatt2_rank_deficient_sketch_gives_a_projection(B, which):
    """ep = 0.95 keeps one term per step, so with n_k < l the sketches W^{(k)}
    have rank n_k < l: the range of each QR factor is only partly fixed and
    the result is not unique. Any valid result is still the orthogonal
    projection of Y * Z onto the span of its left-orthonormal interface, so
    ||X|| <= ||A|| and ||A - X||^2 = ||A||^2 - ||X||^2 (A = Y * Z), and it
    keeps at least the oracle's accuracy up to the arbitrary directions."""
    if which == "random":
        Y, Z = small_random()
    else:
        Y, Z, _ = wl.workload_small_sin_times_random()
    _, kept, cond = cut_margin(Y, Z, 12, 0, 0.95)
    assert max(kept) == 1 and cond > 1e12
    X = run_gpu(B, Y, Z, sketch_rank=12, seed=0, variant=2, ep=0.95)
    A = ott.tt_full(Y) * ott.tt_full(Z)
    Xf = ott.tt_full(X)
    na, nx, ne = np.linalg.norm(A), np.linalg.norm(Xf), np.linalg.norm(A - Xf)
    assert np.all(np.isfinite(Xf))
    assert nx <= na * (1 + 1e-12)
    assert abs(ne ** 2 - (na ** 2 - nx ** 2)) <= 1e-10 * na ** 2


def test_hatt2_several_tiles_with_truncation(B):
    """Ranks and modes that span several GEMM tiles, a ragged sketch rank,
    and the final tolerance truncation on top of the truncated sketches."""
    n = [16, 12, 20, 16, 12, 16, 20]
    Y = wl.gaussian_tt(n, [1, 14, 22, 30, 25, 18, 9, 1], 21)
    Z = wl.gaussian_tt(n, [1, 5, 7, 6, 8, 6, 3, 1], 22)
    ep = 0.5
    margin, kept, cond = cut_margin(Y, Z, 45, 5, ep)
    assert margin > 1e-3 and cond < 1e6 and max(kept) < 45
    X = run_gpu(B, Y, Z, sketch_rank=45, seed=5, variant=2, ep=ep, max_rank=30, tol=1e-8)
    A = ohatt.hadamard_recompress(Y, Z, sketch_rank=45, seed=5, variant=2, ep=ep, max_rank=30,
                                  tol=1e-8)
    assert ott.ranks(X) == ott.ranks(A)
    assert rel_diff(X, A) <= REL_TOL


def test_hatt2_captured_replays_equal_eager(B):
    """The kept ranks R_k stay in device memory (the contractions read them
    there), so a call can be captured in a CUDA graph: replays give the eager
    result, which matches the oracle. The workspace is filled with NaN before
    each run, so a contraction that read a column past R_k (the buffers are
    laid out for R_k = l_{k+1}) would show."""
    Y, Z = small_random()
    ep = 0.3
    margin, kept, cond = cut_margin(Y, Z, 12, 0, ep)
    assert margin > 1e-3 and cond < 1e6 and min(kept[2:-1]) < 12
    h = B.HadamardRecompressor(to_gpu(Y), to_gpu(Z), sketch_rank=12, seed=0, variant=2, ep=ep)
    h.workspace.fill_(255)
    h.run()
    torch.cuda.synchronize()
    X_eager = [c.cpu().numpy().copy() for c in h.result()]
    A = ohatt.hadamard_recompress(Y, Z, sketch_rank=12, seed=0, variant=2, ep=ep)
    assert rel_diff(X_eager, A) <= REL_TOL
    h.capture()
    for _ in range(2):
        h.workspace.fill_(255)
        for t in h.out_bufs:
            t.fill_(float("nan"))
        h.replay()
        torch.cuda.synchronize()
        X = [c.cpu().numpy() for c in h.result()]
        assert rel_diff(X, X_eager) <= 1e-13


def test_hatt2_in_the_stream_lane_batch(B):
    """Variant 2 pairs (and a HaTT-1 pair) in one batched call over library
    streams: each equals its oracle result."""
    Y1, Z1 = small_random()
    Y2, Z2, _ = wl.workload_small_sin_times_random()
    cases = [(Y1, Z1, dict(sketch_rank=12, seed=0, variant=2, ep=0.3)),
             (Y2, Z2, dict(sketch_rank=12, seed=1, variant=2, ep=3e-2)),
             (Y1, Z1, dict(sketch_rank=12, seed=1)),
             (Y2, Z2, dict(sketch_rank=6, seed=0, variant=2, ep=0.3))]
    for Y, Z, o in cases:
        if o.get("variant") == 2:
            margin, _, cond = cut_margin(Y, Z, o["sketch_rank"], o["seed"], o["ep"])
            assert margin > 1e-3 and cond < 1e6
    h = B.BatchRecompressor([(to_gpu(Y), to_gpu(Z), o) for Y, Z, o in cases], lanes=3)
    h.run()
    torch.cuda.synchronize()
    for j, (Y, Z, o) in enumerate(cases):
        X = [c.cpu().numpy() for c in h.result(j)]
        A = ohatt.hadamard_recompress(Y, Z, **o)
        assert rel_diff(X, A) <= REL_TOL
