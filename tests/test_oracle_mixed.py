"""Pins of the oracle's low-precision sketch emulation (CPU).

round_operand must reproduce the binary32, TF32 and BF16 roundings exactly
(hand-computed ties, torch's CPU bfloat16 conversion as an independent
library routine, error bounds). A low-precision sketch is not exact even at
the separation rank: where the sketch rank is below the rank of the left
factor C_k (the last bond of the config-1 shapes: l = 8 < 10), exactness
rests on the columns of C_k W lying in the range of the full unfolding,
which holds for the exact W only; W + E adds C_k E outside it, so the error
scales with the format's unit roundoff."""
import numpy as np
import pytest

from oracle import hatt as ohatt
from oracle import tt as ott
from paper_2410_04385_gb300 import workloads as wl

q = ohatt.round_operand


def test_bf16_ties_to_even_and_tf32_ties_away():
    # bf16 keeps 7 mantissa bits: ulp(1) = 2^-7
    assert q(1 + 2.0 ** -8, "bf16") == 1.0                      # tie -> even (down)
    assert q(1 + 3 * 2.0 ** -8, "bf16") == 1 + 2.0 ** -6        # tie -> even (up)
    assert q(1 + 2.0 ** -8 + 2.0 ** -20, "bf16") == 1 + 2.0 ** -7
    assert q(-(1 + 3 * 2.0 ** -8), "bf16") == -(1 + 2.0 ** -6)
    # tf32 keeps 10 mantissa bits: ulp(1) = 2^-10, ties away from zero
    assert q(1 + 2.0 ** -11, "tf32") == 1 + 2.0 ** -10
    assert q(-(1 + 2.0 ** -11), "tf32") == -(1 + 2.0 ** -10)
    assert q(1 + 2.0 ** -11 - 2.0 ** -23, "tf32") == 1.0
    # binary32 first: 1 + 2^-30 is below half an ulp of binary32
    assert q(1 + 2.0 ** -30, "fp32") == 1.0
    assert q(1 + 2.0 ** -23, "fp32") == 1 + 2.0 ** -23
    assert q(0.1, "fp64") == 0.1


def test_bf16_matches_torch_cpu_conversion():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(20000) * 10.0 ** np.random.default_rng(1).uniform(-20, 20, 20000)
    f32 = torch.from_numpy(x.astype(np.float32))
    ref = f32.to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(q(x, "bf16"), ref)


@pytest.mark.parametrize("fmt,bits", [("fp32", 23), ("tf32", 10), ("bf16", 7)])
def test_rounding_error_bounds_idempotence_symmetry(fmt, bits):
    x = np.random.default_rng(2).standard_normal(50000) * 10.0 ** np.random.default_rng(3).uniform(-30, 30, 50000)
    y = q(x, fmt)
    # one rounding to `bits` mantissa bits (plus the binary32 one): half an ulp each
    bound = 2.0 ** -(bits + 1) + 2.0 ** -24
    assert np.all(np.abs(y - x) <= bound * np.abs(x) * (1 + 1e-12))
    assert np.array_equal(q(y, fmt), y)
    assert np.array_equal(q(-x, fmt), -y)
    if fmt != "fp32":                                   # the result is representable
        mant = np.frexp(y)[0] * 2.0 ** (bits + 1)
        assert np.all(mant == np.round(mant))


UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.mark.parametrize("fmt", ohatt.FORMATS)
def test_sketch_precision_sets_the_error_of_a_full_rank_sketch(fmt):
    """Config-1 shapes, sketch rank = the PKP rank after the clamps, checked
    against the dense product: exact in FP64, and within 30 unit roundoffs of
    the format otherwise (about 3 are observed), never exact below FP64 at
    this size."""
    Y, Z, o = wl.workload_small_sin_times_random()
    X = ohatt.hadamard_recompress(Y, Z, sketch_rank=12, seed=0, fmt=fmt)
    A = ott.tt_full(Y) * ott.tt_full(Z)
    err = np.linalg.norm(ott.tt_full(X) - A) / np.linalg.norm(A)
    if fmt == "fp64":
        assert err <= 1e-13
    else:
        assert 1e-3 * UNIT_ROUNDOFF[fmt] < err <= 30 * UNIT_ROUNDOFF[fmt]


def test_low_precision_sketch_is_exact_where_sketch_rank_covers_the_left_factor():
    """With every l_k at least the rank of the left factor (here the clamp
    l_k <= r_k s_k is never active below the unfolding ranks: d = 3, n = 4,
    ranks 2 x 2, sketch = PKP rank 4 = n), range(C_k W) = range(C_k) for any
    nonsingular W, so even a BF16 sketch reproduces Y ⊙ Z to rounding."""
    Y = wl.gaussian_tt([4, 4, 4], [1, 2, 2, 1], 21)
    Z = wl.gaussian_tt([4, 4, 4], [1, 2, 2, 1], 22)
    A = ott.tt_full(Y) * ott.tt_full(Z)
    for fmt in ohatt.FORMATS:
        X = ohatt.hadamard_recompress(Y, Z, seed=5, fmt=fmt)
        assert ott.ranks(X) == [1, 4, 4, 1]
        assert np.linalg.norm(ott.tt_full(X) - A) <= 1e-13 * np.linalg.norm(A)


def test_low_precision_sketch_changes_a_rank_deficient_result_boundedly():
    """Below the separation rank the sketch precision matters, but a BF16
    sketch is just another random test matrix: its range-finder error stays
    within a small factor of the FP64 one (C7's bound uses a factor 10)."""
    n = [6] * 6
    Y = wl.gaussian_tt(n, [1, 4, 5, 5, 5, 4, 1], 11)
    Z = wl.gaussian_tt(n, [1, 3, 4, 4, 4, 3, 1], 12)
    A = ott.hadamard_pkp(Y, Z)
    errs = {}
    for fmt in ("fp64", "bf16"):
        X = ohatt.hadamard_recompress(Y, Z, sketch_rank=10, seed=3, fmt=fmt)
        errs[fmt] = ott.tt_rel_error(X, A)
    assert 0 < errs["fp64"] < 1
    assert errs["bf16"] <= 10 * errs["fp64"]
