"""Failure detection through the C ABI, without faulting the GPU: non-finite
values made on the host in input cores reach the device health word
(tt_device_status -> TT_ERR_NONFINITE) for the single-pair recompression, the
TT rounding and the batched task engine, whose other pairs stay correct; a
clean call afterwards reports TT_OK (the word is cleared on read)."""
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
    binding.device_status()          # start from a clear word
    return binding


def gpu(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def pair(seed=1):
    Y = wl.gaussian_tt([8] * 5, [1, 4, 5, 3, 4, 1], seed)
    Z = wl.gaussian_tt([8] * 5, [1, 3, 2, 5, 2, 1], seed + 1)
    return Y, Z


@pytest.mark.parametrize("which, core, value", [("Y", 2, np.nan), ("Z", 0, np.inf),
                                                ("Y", 4, -np.inf), ("Z", 3, np.nan)])
def test_nonfinite_input_is_reported(B, which, core, value):
    Y, Z = pair()
    bad = Y if which == "Y" else Z
    bad[core] = bad[core].copy()
    bad[core][0, 1, 0] = value
    B.tt_hadamard_recompress(gpu(Y), gpu(Z), sketch_rank=10, seed=3)
    torch.cuda.synchronize()
    assert B.device_status() == B.TT_ERR_NONFINITE
    Y, Z = pair()
    X = B.tt_hadamard_recompress(gpu(Y), gpu(Z), sketch_rank=10, seed=3)
    torch.cuda.synchronize()
    assert B.device_status() == B.TT_OK
    Xo = ohatt.hadamard_recompress(Y, Z, sketch_rank=10, seed=3)
    Xh = [c.cpu().numpy() for c in X]
    assert ott.tt_diff_norm(Xh, Xo) <= 1e-12 * ott.tt_norm(Xo)


def test_nonfinite_input_to_rounding_is_reported(B):
    A = wl.gaussian_tt([6] * 4, [1, 5, 7, 4, 1], 9)
    A[1] = A[1].copy()
    A[1][2, 3, 1] = np.nan
    B.tt_round(gpu(A), max_rank=3)
    torch.cuda.synchronize()
    assert B.device_status() == B.TT_ERR_NONFINITE
    assert B.device_status() == B.TT_OK


def test_engine_reports_a_nonfinite_pair_and_keeps_the_others(B):
    pairs = []
    for j in range(6):
        Y, Z = pair(10 + 2 * j)
        if j == 2:
            Z[1] = Z[1].copy()
            Z[1][0, 0, 0] = np.inf
        pairs.append((Y, Z, dict(sketch_rank=10, max_rank=10, oversample=0, seed=50 + j)))
    eng = B.BatchedRecompressor([(gpu(Y), gpu(Z), o) for Y, Z, o in pairs], autotune=False)
    eng.run()
    torch.cuda.synchronize()
    assert eng.status() == B.TT_ERR_NONFINITE
    for j in (0, 5):
        Y, Z, o = pairs[j]
        Xo = ohatt.hadamard_recompress(Y, Z, **o)
        Xh = [c.cpu().numpy() for c in eng.result(j)]
        assert ott.tt_diff_norm(Xh, Xo) <= 1e-12 * ott.tt_norm(Xo)
