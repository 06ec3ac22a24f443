"""GPU parity: libhatt kernels (through the C ABI) against the FP64 oracle.

Tolerances: FP64 path vs FP64 oracle, relative Frobenius difference of the
reconstructed tensors <= 1e-12 (both sides use the same Philox sketch; the
tensors, not the cores, are compared because QR / truncation gauges are not
unique). Integer work (Philox words, ranks) is compared exactly.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hatt as ohatt
from oracle import philox as ophilox
from oracle import rounding as oround
from oracle import tt as ott
from paper_2410_04385_gb300 import workloads as wl
from tests.conftest import read_kat

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


def run_gpu(B, Y, Z, **opts):
    return to_np(B.tt_hadamard_recompress(to_gpu(Y), to_gpu(Z), **opts))


# ---------------------------------------------------------------- RNG ---

def test_philox_known_answers_bit_exact(B, golden_dir):
    rows = read_kat(os.path.join(golden_dir, "philox4x32_10_kat.txt"))
    for ctr, key, out in rows:
        c = torch.tensor(np.array(ctr, dtype=np.uint32).view(np.int32).reshape(1, 4)).cuda()
        got = B.tt_philox4x32_10(c, key[0], key[1]).cpu().numpy().view(np.uint32).ravel()
        assert [int(v) for v in got] == out


def test_philox_many_counters_bit_exact(B):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(4099, 4), dtype=np.uint64).astype(np.uint32)
    key = (0xDEADBEEF, 0x01234567)
    got = B.tt_philox4x32_10(torch.tensor(ctr.view(np.int32)).cuda(), *key).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), ophilox.philox4x32_10(ctr, key))


@pytest.mark.parametrize("seed", [0, 7, 2 ** 40 + 3])
def test_sketch_cores_match_oracle(B, seed):
    n = [8, 3, 17, 1, 5]
    ell = [1, 8, 13, 7, 5, 1]
    got = to_np(B.tt_sketch_tt(n, ell, seed=seed))
    ref = ophilox.sketch_tt(seed, n, ell)
    for g, r in zip(got, ref):
        assert g.shape == r.shape
        assert np.max(np.abs(g - r)) <= 1e-14 * np.max(np.abs(r))


# ---------------------------------------------------------- dot / norm ---

@pytest.mark.parametrize("shape", [
    ([3, 4, 5], [1, 2, 3, 1], [1, 4, 2, 1]),
    ([17, 1, 33, 8], [1, 5, 7, 3, 1], [1, 1, 9, 20, 1]),
    ([64] * 6, [1, 30, 40, 40, 40, 30, 1], [1, 20, 20, 20, 20, 20, 1]),
])
def test_dot_and_norm(B, shape):
    n, ra, rb = shape
    A = wl.gaussian_tt(n, ra, 1)
    Bt = wl.gaussian_tt(n, rb, 2)
    g = B.tt_dot(to_gpu(A), to_gpu(Bt)).item()
    ref = ott.tt_dot(A, Bt)
    assert abs(g - ref) <= 1e-12 * ott.tt_norm(A) * ott.tt_norm(Bt)
    gn = B.tt_norm(to_gpu(A)).item()
    assert abs(gn - ott.tt_norm(A)) <= 1e-12 * ott.tt_norm(A)


def test_dot_order_one(B):
    A = wl.gaussian_tt([9], [1, 1], 3)
    C = wl.gaussian_tt([9], [1, 1], 4)
    assert np.isclose(B.tt_dot(to_gpu(A), to_gpu(C)).item(), ott.tt_dot(A, C), rtol=1e-13)


# ------------------------------------------------------------- HaTT-1 ---

def test_small_workload_vs_oracle_and_brute_force(B):
    Y, Z, o = wl.workload_small_sin_times_random(seed=0)
    X = run_gpu(B, Y, Z, seed=0, **o)
    Xo, info = ohatt.hadamard_recompress(Y, Z, seed=0, return_info=True, **o)
    assert ott.ranks(X) == info["ranks"]
    assert rel_diff(X, Xo) <= REL_TOL
    dense = ott.tt_full(Y) * ott.tt_full(Z)
    assert np.linalg.norm(ott.tt_full(X) - dense) <= 1e-13 * np.linalg.norm(dense) * 10


def test_sin_times_cos_rank_two(B):
    Y, Z, o = wl.workload_small_sin_times_cos()
    X = run_gpu(B, Y, Z, seed=2, **o)
    assert ott.ranks(X) == [1, 2, 2, 2, 2, 2, 1]
    d, n = 6, 8
    S = sum(np.meshgrid(*([wl.uniform_grid(n)] * d), indexing="ij"))
    assert np.allclose(ott.tt_full(X), 0.5 * np.sin(2 * S), atol=1e-12)
    assert abs(ott.tt_norm(X) ** 2 - 32768.0) <= 1e-9


@pytest.mark.parametrize("case", range(8))
def test_hatt_random_shapes_no_truncation(B, case):
    """Shapes spanning several GEMM tiles and ragged tails; every core compared
    as a tensor, and the result must be left-orthogonal."""
    rng = np.random.default_rng(100 + case)
    d = int(rng.integers(2, 8))
    n = [int(v) for v in rng.choice([1, 3, 7, 16, 17, 33], size=d)]
    r = [1] + [int(v) for v in rng.integers(1, 25, size=d - 1)] + [1]
    s = [1] + [int(v) for v in rng.integers(1, 25, size=d - 1)] + [1]
    Y = wl.gaussian_tt(n, r, 200 + case)
    Z = wl.gaussian_tt(n, s, 300 + case)
    sk = int(rng.integers(1, 70))
    X = run_gpu(B, Y, Z, sketch_rank=sk, seed=case)
    Xo = ohatt.hadamard_recompress(Y, Z, sketch_rank=sk, seed=case)
    assert ott.ranks(X) == ott.ranks(Xo)
    assert rel_diff(X, Xo) <= REL_TOL
    assert ott.is_left_orthogonal(X, atol=1e-12)


def test_exact_recompression_reproduces_product(B):
    n = [5, 4, 6, 3, 5]
    Y = wl.gaussian_tt(n, [1, 3, 4, 2, 3, 1], 11)
    Z = wl.gaussian_tt(n, [1, 2, 3, 3, 2, 1], 12)
    X = run_gpu(B, Y, Z, seed=4)                       # sketch rank = PKP rank
    dense = ott.tt_full(Y) * ott.tt_full(Z)
    assert np.linalg.norm(ott.tt_full(X) - dense) <= 1e-13 * np.linalg.norm(dense) * 10


def test_square_is_rank_deficient_but_exact(B):
    """Y ⊙ Y: the PKP sketch has exactly dependent columns (r(r+1)/2 < r^2),
    which exercises the shifted Cholesky-QR passes."""
    n = [6] * 5
    Y = wl.gaussian_tt(n, [1, 3, 3, 3, 3, 1], 13)
    X = run_gpu(B, Y, Y, seed=5)
    Xo = ohatt.hadamard_recompress(Y, Y, seed=5)
    dense = ott.tt_full(Y) ** 2
    assert np.linalg.norm(ott.tt_full(X) - dense) <= 1e-12 * np.linalg.norm(dense)
    assert rel_diff(X, Xo) <= REL_TOL


def test_order_one_two_and_unit_modes(B):
    Y1, Z1 = wl.gaussian_tt([9], [1, 1], 1), wl.gaussian_tt([9], [1, 1], 2)
    X1 = run_gpu(B, Y1, Z1)
    assert np.allclose(X1[0], Y1[0] * Z1[0], rtol=1e-15, atol=0)
    Y2, Z2 = wl.gaussian_tt([5, 6], [1, 3, 1], 3), wl.gaussian_tt([5, 6], [1, 2, 1], 4)
    X2 = run_gpu(B, Y2, Z2, sketch_rank=6)
    assert rel_diff(X2, ohatt.hadamard_recompress(Y2, Z2, sketch_rank=6)) <= REL_TOL
    Y3 = wl.gaussian_tt([3, 1, 4, 1], [1, 2, 3, 2, 1], 5)
    Z3 = wl.gaussian_tt([3, 1, 4, 1], [1, 3, 2, 2, 1], 6)
    X3 = run_gpu(B, Y3, Z3, sketch_rank=20)
    assert rel_diff(X3, ohatt.hadamard_recompress(Y3, Z3, sketch_rank=20)) <= REL_TOL


@pytest.mark.parametrize("tol,max_rank", [(1e-2, 0), (1e-6, 0), (0.0, 5), (1e-3, 7)])
def test_truncation_vs_oracle(B, tol, max_rank):
    n = [6] * 6
    Y = wl.gaussian_tt(n, [1, 4, 4, 4, 4, 4, 1], 21)
    Z = wl.gaussian_tt(n, [1, 3, 4, 4, 3, 3, 1], 22)
    A = ott.hadamard_pkp(Y, Z)
    X = run_gpu(B, Y, Z, sketch_rank=16, tol=tol, max_rank=max_rank, seed=3)
    Xo, info = ohatt.hadamard_recompress(Y, Z, sketch_rank=16, tol=tol, max_rank=max_rank, seed=3,
                                         return_info=True)
    assert ott.ranks(X) == info["ranks"]
    # both are truncations of the same sketched tensor with the same rule
    assert rel_diff(X, Xo) <= max(REL_TOL, 2 * tol * 1e-3)
    if max_rank:
        assert max(ott.ranks(X)) <= max_rank


def test_random_d20_full_size(B):
    """The d = 20, n = 32, rank-20 x rank-20 workload (target 40, sketch 50)
    in the launch configuration of the benchmark."""
    Y, Z, o = wl.workload_random_d20()
    h = B.HadamardRecompressor(to_gpu(Y), to_gpu(Z), seed=9, **o)
    h.run()
    torch.cuda.synchronize()
    X = to_np(h.result())
    Xo, info = ohatt.hadamard_recompress(Y, Z, seed=9, return_info=True, **o)
    assert ott.ranks(X) == info["ranks"] == [1] + [32] + [40] * 17 + [32] + [1]
    assert rel_diff(X, Xo) <= REL_TOL
    # a second run on the same buffers is bitwise identical (fixed reduction order)
    h.run()
    torch.cuda.synchronize()
    X2 = to_np(h.result())
    for a, b in zip(X, X2):
        assert np.array_equal(a, b)


# ------------------------------------------------------------- rounding ---

def test_round_exact_rank(B):
    d, n = 6, 7
    A = ott.tt_add(wl.sin_sum_tt(d, n, "sin"), wl.gaussian_tt([n] * d, [1, 2, 3, 3, 3, 2, 1], 5))
    Bg = to_np(B.tt_round(to_gpu(A), 0, 1e-13))
    Bo, rk = oround.tt_round(A, 0, 1e-13)
    assert ott.ranks(Bg) == rk
    assert rel_diff(Bg, A) <= 1e-12


@pytest.mark.parametrize("tol", [1e-1, 1e-4])
def test_round_tolerance(B, tol):
    n = [5] * 6
    A = wl.gaussian_tt(n, [1, 5, 8, 9, 8, 5, 1], 31)
    Bg = to_np(B.tt_round(to_gpu(A), 0, tol))
    assert rel_diff(Bg, A) <= tol * (1 + 1e-9)
    Bo, rk = oround.tt_round(A, 0, tol)
    assert max(ott.ranks(Bg)) <= max(rk) + 1


def test_round_of_pkp_matches_hatt(B):
    """Rounding the explicit PKP product and HaTT with an exact sketch give the
    same tensor (Y ⊙ Z itself)."""
    n = [4] * 5
    Y = wl.gaussian_tt(n, [1, 3, 3, 3, 3, 1], 41)
    Z = wl.gaussian_tt(n, [1, 3, 3, 3, 3, 1], 42)
    A = ott.hadamard_pkp(Y, Z)
    Bg = to_np(B.tt_round(to_gpu(A), 0, 1e-14))
    assert rel_diff(Bg, A) <= 1e-12


def hard_spectrum_tt(kind):
    """A TT whose middle bond has a graded spectrum (twelve decades) or
    clusters {1, 1e-3, 1e-6, 0} of six singular values each: the FP32 eigen
    start of the truncation cannot resolve these, so the FP64 refinement and
    its closing orthonormalization carry the accuracy."""
    d, n, r = 5, 6, 24
    A = wl.gaussian_tt([n] * d, [1, 6, r, r, 6, 1], 77)
    if kind == "graded":
        s = 10.0 ** (-np.linspace(0.0, 12.0, r))
    else:
        s = np.repeat([1.0, 1e-3, 1e-6, 0.0], r // 4)
    A[1] = A[1] * s[None, None, :]
    return A


@pytest.mark.parametrize("kind,tol", [("graded", 1e-9), ("graded", 1e-5), ("clustered", 1e-12)])
def test_round_hard_spectra(B, kind, tol):
    A = hard_spectrum_tt(kind)
    Bg = to_np(B.tt_round(to_gpu(A), 0, tol))
    Bo, rk = oround.tt_round(A, 0, tol)
    assert ott.ranks(Bg) == rk
    assert rel_diff(Bg, A) <= tol * (1 + 1e-6) + 1e-13
    assert rel_diff(Bg, Bo) <= tol + 1e-13
    if kind == "clustered":
        assert rk[2] == 18                      # the six zero singular values are dropped


def test_round_cut_below_resolution_is_conservative(B):
    """tol = 1e-11 puts the cut near sigma^2 ~ 1e-24 ||X||^2, below what two
    Gram levels resolve in FP64: ranks may exceed the SVD's, never fall
    below them, and the error bound holds."""
    A = hard_spectrum_tt("graded")
    tol = 1e-11
    Bg = to_np(B.tt_round(to_gpu(A), 0, tol))
    _, rk = oround.tt_round(A, 0, tol)
    assert all(a >= b for a, b in zip(ott.ranks(Bg), rk))
    assert rel_diff(Bg, A) <= tol


def test_round_without_truncation_keeps_exact_zero_directions_exact(B):
    """Six singular values of a bond are exactly zero, so the left-to-right
    Cholesky QR meets exactly zero columns: they must be null columns of an
    otherwise unshifted factorization, and a round that changes no rank must
    reproduce the input to rounding."""
    A = hard_spectrum_tt("clustered")
    Bg = to_np(B.tt_round(to_gpu(A), 24, 0.0))
    assert rel_diff(Bg, A) <= 1e-13


def test_kernel_timer_times_every_gemm_launch(B):
    """One eager recompression under the kernel timer: every FP64 GEMM launch
    gets a positive duration and the flop count of its shape; the launches
    outside the capacity run untimed; a captured replay records nothing."""
    Y, Z, o = wl.workload_small_sin_times_random()
    Yg, Zg = to_gpu(Y), to_gpu(Z)
    h = B.HadamardRecompressor(Yg, Zg, seed=0, **o)
    B.kernel_timer_start(4096)
    h.run()
    torch.cuda.synchronize()
    ms, fl, recorded = B.kernel_timer_stop(4096)
    assert recorded == len(ms) > 10
    assert all(0.0 < t < 100.0 for t in ms)
    assert all(f > 0 and f == int(f) and int(f) % 2 == 0 for f in fl)
    B.kernel_timer_start(3)
    h.run()
    torch.cuda.synchronize()
    ms3, _, rec3 = B.kernel_timer_stop(3)
    assert rec3 == 3 and len(ms3) == 3
    h.capture()
    B.kernel_timer_start(16)
    h.replay()
    torch.cuda.synchronize()
    _, _, rec_graph = B.kernel_timer_stop(16)
    assert rec_graph == 0
