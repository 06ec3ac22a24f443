"""GPU parity of the low-precision sketch modes (HPCRL-1 products with FP32,
TF32 or BF16 operands and FP32 accumulation; everything else FP64) against
the oracle's emulation of the same rounding, following the error model that
governs them: a perturbed sketch W + E keeps range(C_k (W + E)) inside
range(C_k), so the result is exact where the sketch rank covers the left
factor, and otherwise carries an error of the order of the format's unit
roundoff on top of the range-finder error. Errors are measured against the
exact product Y ⊙ Z."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hatt as ohatt
from oracle import tt as ott
from paper_2410_04385_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

FMT = {1: "fp32", 2: "tf32", 3: "bf16"}
UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


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
    X = B.tt_hadamard_recompress(to_gpu(Y), to_gpu(Z), **opts)
    return [c.cpu().numpy() for c in X]


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_full_rank_sketch_error_follows_the_format(B, prec):
    """Config-1 shapes (sin x random, d = 6, n = 8), sketch = PKP rank: the
    error against the dense product is a few unit roundoffs of the format, as
    in the oracle's emulation."""
    Y, Z, _ = wl.workload_small_sin_times_random()
    A = ott.tt_full(Y) * ott.tt_full(Z)
    fmt = FMT[prec]
    Xg = run_gpu(B, Y, Z, sketch_rank=12, seed=0, precision=prec)
    Xo = ohatt.hadamard_recompress(Y, Z, sketch_rank=12, seed=0, fmt=fmt)
    err_g = np.linalg.norm(ott.tt_full(Xg) - A) / np.linalg.norm(A)
    err_o = np.linalg.norm(ott.tt_full(Xo) - A) / np.linalg.norm(A)
    assert ott.ranks(Xg) == ott.ranks(Xo)
    assert err_g <= 30 * UNIT_ROUNDOFF[fmt]
    assert err_g <= 10 * max(err_o, 1e-14) and err_o <= 10 * max(err_g, 1e-14)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_exact_where_the_sketch_covers_the_left_factor(B, prec):
    Y = wl.gaussian_tt([4, 4, 4], [1, 2, 2, 1], 21)
    Z = wl.gaussian_tt([4, 4, 4], [1, 2, 2, 1], 22)
    A = ott.tt_full(Y) * ott.tt_full(Z)
    Xg = run_gpu(B, Y, Z, seed=5, precision=prec)
    assert ott.ranks(Xg) == [1, 4, 4, 1]
    assert np.linalg.norm(ott.tt_full(Xg) - A) <= 1e-13 * np.linalg.norm(A)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_rank_deficient_sketch_meets_the_per_config_bound(B, prec):
    """Sketch rank 14 below the PKP rank 30 (d = 8, n = 6): the GPU error
    against Y ⊙ Z stays within 10 x max(FP64 error, emulated error, tol)."""
    n = [6] * 8
    Y = wl.gaussian_tt(n, [1, 5, 6, 6, 6, 6, 6, 5, 1], 31)
    Z = wl.gaussian_tt(n, [1, 4, 5, 5, 5, 5, 5, 4, 1], 32)
    A = ott.hadamard_pkp(Y, Z)
    fmt = FMT[prec]
    Xg = run_gpu(B, Y, Z, sketch_rank=14, seed=7, precision=prec)
    e64 = ott.tt_rel_error(ohatt.hadamard_recompress(Y, Z, sketch_rank=14, seed=7), A)
    eem = ott.tt_rel_error(ohatt.hadamard_recompress(Y, Z, sketch_rank=14, seed=7, fmt=fmt), A)
    eg = ott.tt_rel_error(Xg, A)
    assert 0 < e64 < 1
    assert eg <= 10 * max(e64, eem)


def test_no_device_wait_ran_out(B):
    """The tensor-core products wait on an mbarrier with a bounded loop; none
    of the runs above may have hit the bound."""
    assert B.device_error() == 0


def test_tensor_core_products_match_simt_rounding_model(B):
    """The TF32 / BF16 products run on tcgen05; their result equals the
    exact product of the rounded operands up to FP32 accumulation, checked
    through a one-core-deep chain against the emulation on a shape that
    spans several 128-row tiles, a ragged N and split K."""
    n = [40, 40, 40]
    Y = wl.gaussian_tt(n, [1, 37, 29, 1], 41)
    Z = wl.gaussian_tt(n, [1, 23, 31, 1], 42)
    for prec in (2, 3):
        Xg = run_gpu(B, Y, Z, sketch_rank=40, seed=9, precision=prec)
        Xo = ohatt.hadamard_recompress(Y, Z, sketch_rank=40, seed=9, fmt=FMT[prec])
        A = ott.tt_full(Y) * ott.tt_full(Z)
        eg = np.linalg.norm(ott.tt_full(Xg) - A) / np.linalg.norm(A)
        eo = np.linalg.norm(ott.tt_full(Xo) - A) / np.linalg.norm(A)
        assert eg <= 10 * max(eo, 1e-14) and eo <= 10 * max(eg, 1e-14)
    assert B.device_error() == 0


def test_rejects_unknown_precision(B):
    Y, Z, _ = wl.workload_small_sin_times_random()
    with pytest.raises(B.HattError):
        run_gpu(B, Y, Z, sketch_rank=12, precision=5)     # past TT_FP64_TC = 4
