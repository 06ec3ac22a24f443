"""GPU tests of the batched task engine (tt_batched_*): one persistent launch
over many uneven pairs.

  * FP64: every pair's result equals the oracle's HaTT-1 result for the same
    sketch seed (relative Frobenius difference <= 1e-12), and the single-pair
    entry point's result to the same tolerance; two runs agree bitwise.
  * FP32 sketch products: every pair within the mixed-mode bound against the
    exact product (reading C7) and close to the single-pair FP32 result.
  * A CUDA graph of one run replays to the same result.
  * Bounded waits: with a poll cap of 1 the waits run out and the status says
    so (TT_ERR_TIMEOUT) without hanging; the next run with the normal cap is
    correct again.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hatt as ohatt
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


def uneven_pairs(count, seed, precision=0):
    """Small uneven pairs: orders 2-6, modes {3, 8, 16, 17}, inner ranks 1-9,
    sketch rank = 2 max(r) (no truncation), Gaussian cores."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        d = int(rng.integers(2, 7))
        n = int(rng.choice([3, 8, 16, 17]))
        ry = [1] + [int(v) for v in rng.integers(1, 10, size=d - 1)] + [1]
        rz = [1] + [int(v) for v in rng.integers(1, 10, size=d - 1)] + [1]
        Y = wl.gaussian_tt([n] * d, ry, int(rng.integers(1 << 30)))
        Z = wl.gaussian_tt([n] * d, rz, int(rng.integers(1 << 30)))
        ell = 2 * max(max(ry), max(rz))
        out.append((Y, Z, dict(sketch_rank=ell, max_rank=ell, oversample=0, seed=100 + j,
                               precision=precision)))
    return out


def to_gpu(pairs):
    return [([torch.from_numpy(c).cuda() for c in Y], [torch.from_numpy(c).cuda() for c in Z], o)
            for Y, Z, o in pairs]


def host(cores):
    return [c.detach().cpu().numpy() for c in cores]


def rel_diff(X, Xo):
    return ott.tt_diff_norm(X, Xo) / ott.tt_norm(Xo)


def test_fp64_batch_matches_the_oracle_and_single_calls(B):
    pairs = uneven_pairs(24, 1)
    gp = to_gpu(pairs)
    eng = B.BatchedRecompressor(gp, autotune=True)
    eng.run()
    torch.cuda.synchronize()
    assert eng.status() == 0
    first = [host(eng.result(j)) for j in range(len(pairs))]
    for j, (Y, Z, o) in enumerate(pairs):
        opts = {k: v for k, v in o.items() if k != "precision"}
        Xo = ohatt.hadamard_recompress(Y, Z, **opts)
        assert rel_diff(first[j], Xo) <= 1e-12, j
        Xs = host(B.tt_hadamard_recompress(gp[j][0], gp[j][1], **o))
        assert rel_diff(first[j], Xs) <= 1e-12, j
    eng.run()
    torch.cuda.synchronize()
    for j in range(len(pairs)):
        for a, b in zip(first[j], host(eng.result(j))):
            assert np.array_equal(a, b)
    info = eng.info()
    assert info["tasks"] >= info["stages"] > 0 and info["blocks"] >= 152


def test_fp32_sketch_batch_within_the_mixed_bound(B):
    pairs = uneven_pairs(12, 2, precision=B.TT_MIXED_FP32)
    gp = to_gpu(pairs)
    eng = B.BatchedRecompressor(gp, autotune=False)
    eng.run()
    torch.cuda.synchronize()
    assert eng.status() == 0
    for j, (Y, Z, o) in enumerate(pairs):
        A = ott.hadamard_pkp(Y, Z)
        opts = {k: v for k, v in o.items() if k != "precision"}
        e64 = ott.tt_rel_error(ohatt.hadamard_recompress(Y, Z, **opts), A)
        e32 = ott.tt_rel_error(ohatt.hadamard_recompress(Y, Z, fmt="fp32", **opts), A)
        X = host(eng.result(j))
        assert ott.tt_rel_error(X, A) <= 10 * max(e64, e32, 1e-12), j
        Xs = host(B.tt_hadamard_recompress(gp[j][0], gp[j][1], **o))
        assert rel_diff(X, Xs) <= 10 * max(e64, e32, 1e-12), j


def test_graph_replay_of_a_run(B):
    pairs = uneven_pairs(8, 3)
    eng = B.BatchedRecompressor(to_gpu(pairs))
    eng.run()
    torch.cuda.synchronize()
    ref = [host(eng.result(j)) for j in range(len(pairs))]
    for j in range(len(pairs)):
        for c in eng.out_bufs[j]:
            c.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            eng.run(stream=s)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert eng.status() == 0
    for j in range(len(pairs)):
        for a, b in zip(ref[j], host(eng.result(j))):
            assert np.array_equal(a, b)


def test_bounded_waits_report_a_timeout_and_recover(B):
    pairs = uneven_pairs(16, 4)
    eng = B.BatchedRecompressor(to_gpu(pairs), autotune=False)
    eng.run(spin_cap=1)
    torch.cuda.synchronize()
    assert eng.status() == B.TT_ERR_TIMEOUT
    assert B.status_string(B.TT_ERR_TIMEOUT).startswith("a bounded device wait")
    eng.run()
    torch.cuda.synchronize()
    assert eng.status() == 0
    Y, Z, o = pairs[0]
    Xo = ohatt.hadamard_recompress(Y, Z, **{k: v for k, v in o.items() if k != "precision"})
    assert rel_diff(host(eng.result(0)), Xo) <= 1e-12
