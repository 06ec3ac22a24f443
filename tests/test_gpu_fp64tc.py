"""GPU parity of TT_FP64_TC: every product of at least 2e7 flops with
max(M, N) >= 128 and K >= 128 runs on the BF16 tensor cores from 6-bit slices
with exact FP32 accumulation, so the result must meet the same FP64 parity
bar as the native path (relative 1e-12 against the oracle), and agree with
the native FP64 path to that bar."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hatt as ohatt
from oracle import tt as ott
from paper_2410_04385_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

REL_TOL = 1e-12


@pytest.fixture(scope="module")
def B():
    from paper_2410_04385_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    return binding


def to_gpu(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def to_np(cores):
    return [c.detach().cpu().numpy() for c in cores]


def rel_diff(X, A):
    return ott.tt_diff_norm(X, A) / max(ott.tt_norm(A), 1e-300)


def test_full_size_d20_matches_oracle(B):
    Y, Z, o = wl.workload_random_d20()
    h = B.HadamardRecompressor(to_gpu(Y), to_gpu(Z), seed=9, precision=B.TT_FP64_TC, **o)
    h.run()
    torch.cuda.synchronize()
    X = to_np(h.result())
    Xo, info = ohatt.hadamard_recompress(Y, Z, seed=9, return_info=True, **o)
    assert ott.ranks(X) == info["ranks"]
    assert rel_diff(X, Xo) <= REL_TOL
    assert B.device_error() == 0


@pytest.mark.parametrize("shape", [
    (6, 32, 20, 20, 60),      # every left-to-right product qualifies
    (5, 24, 33, 17, 70),      # ragged tiles in M, N and K
    (4, 64, 16, 24, 100),     # wide left factor, split K pieces (K > 448)
])
def test_matches_native_fp64(B, shape):
    d, n, r, s, ell = shape
    Y = wl.gaussian_tt([n] * d, [1] + [r] * (d - 1) + [1], 51)
    Z = wl.gaussian_tt([n] * d, [1] + [s] * (d - 1) + [1], 52)
    Yg, Zg = to_gpu(Y), to_gpu(Z)
    X64 = to_np(B.tt_hadamard_recompress(Yg, Zg, sketch_rank=ell, seed=3))
    Xtc = to_np(B.tt_hadamard_recompress(Yg, Zg, sketch_rank=ell, seed=3, precision=B.TT_FP64_TC))
    assert ott.ranks(Xtc) == ott.ranks(X64)
    assert rel_diff(Xtc, X64) <= REL_TOL
    assert B.device_error() == 0


def test_with_truncation_matches_oracle(B):
    n = [16] * 6
    Y = wl.gaussian_tt(n, [1, 16, 24, 24, 24, 16, 1], 61)
    Z = wl.gaussian_tt(n, [1, 12, 12, 12, 12, 12, 1], 62)
    X = to_np(B.tt_hadamard_recompress(to_gpu(Y), to_gpu(Z), max_rank=60, sketch_rank=80, seed=4,
                                       precision=B.TT_FP64_TC))
    Xo = ohatt.hadamard_recompress(Y, Z, max_rank=60, sketch_rank=80, seed=4)
    assert ott.ranks(X) == ott.ranks(Xo)
    assert rel_diff(X, Xo) <= REL_TOL
