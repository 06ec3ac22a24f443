"""Pins for the HaTT-1 oracle: brute force, closed forms, the RandOrth twin,
Theorem 3.1 and exact TT identities."""
import numpy as np
import pytest

from oracle import flops, hatt, philox, randorth, rounding, tt
from paper_2410_04385_gb300 import workloads as wl


def _rand_pair(n, r, s, seed):
    return wl.gaussian_tt(n, r, seed), wl.gaussian_tt(n, s, seed + 1000)


# ----------------------------------------------------------------- plan ---

def test_plan_small_workload():
    n = [8] * 6
    r = [1, 2, 2, 2, 2, 2, 1]
    s = [1, 5, 5, 5, 5, 5, 1]
    assert hatt.plan_ranks(n, r, s, 12) == [1, 8, 10, 10, 10, 8, 1]


@pytest.mark.parametrize("seed", range(6))
def test_plan_constraints(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.integers(2, 7))
    n = [int(v) for v in rng.integers(1, 5, size=d)]
    r = [1] + [int(v) for v in rng.integers(1, 6, size=d - 1)] + [1]
    s = [1] + [int(v) for v in rng.integers(1, 6, size=d - 1)] + [1]
    ell = hatt.plan_ranks(n, r, s, int(rng.integers(1, 30)))
    assert ell[0] == ell[-1] == 1
    for k in range(1, d):
        assert 1 <= ell[k] <= r[k] * s[k]
        assert ell[k] <= ell[k - 1] * n[k - 1]
        assert ell[k] <= n[k] * ell[k + 1]


# ----------------------------------------------------- W definition (3.1) ---

def _dense_right_part(cores):
    """H(T_{k:d}) as a dense (r_k, prod n) matrix."""
    t = cores[0]
    for c in cores[1:]:
        t = np.tensordot(t, c, axes=([t.ndim - 1], [0]))
    return t.reshape(t.shape[0], -1)


def test_sketch_matches_definition_3_1():
    n = [3, 2, 4, 3]
    Y, Z = _rand_pair(n, [1, 2, 3, 2, 1], [1, 3, 2, 2, 1], seed=20)
    ell = hatt.plan_ranks(n, tt.ranks(Y), tt.ranks(Z), 5)
    R = philox.sketch_tt(4, n, ell)
    A = tt.hadamard_pkp(Y, Z)
    W = hatt.hpcrl1_contract(Y, Z, R, normalize=False)
    for k in range(1, 4):
        ref = _dense_right_part(A[k:]) @ _dense_right_part(R[k:]).T
        assert np.allclose(W[k], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_two_hpcrl_codings_agree():
    n = [3, 4, 2, 5, 3]
    Y, Z = _rand_pair(n, [1, 3, 2, 4, 3, 1], [1, 2, 3, 2, 4, 1], seed=21)
    ell = hatt.plan_ranks(n, tt.ranks(Y), tt.ranks(Z), 6)
    R = philox.sketch_tt(9, n, ell)
    Wa = hatt.hpcrl1_wlwr(Y, Z, R)
    Wb = hatt.hpcrl1_contract(Y, Z, R)
    for k in range(1, 5):
        assert np.allclose(Wa[k], Wb[k], rtol=1e-12, atol=1e-14)


def test_two_core_update_codings_agree():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((5, 3 * 4))
    y = rng.standard_normal((3, 6, 2))
    z = rng.standard_normal((4, 6, 3))
    assert np.allclose(hatt.core_update_paper(M, y, z), hatt.core_update_contract(M, y, z),
                       rtol=1e-13, atol=1e-13)
    # and both equal M times the explicit PKP core
    ref = (M @ tt.H(tt.pkp_core(y, z))).reshape(5, 6, 6)
    assert np.allclose(hatt.core_update_contract(M, y, z), ref, rtol=1e-13, atol=1e-13)


# ------------------------------------------------- RandOrth twin (P3) ---

@pytest.mark.parametrize("seed", [30, 31, 32])
def test_hatt_equals_randorth_on_explicit_pkp(seed):
    rng = np.random.default_rng(seed)
    d = 5
    n = [int(v) for v in rng.integers(3, 7, size=d)]
    r = [1] + [int(v) for v in rng.integers(2, 5, size=d - 1)] + [1]
    s = [1] + [int(v) for v in rng.integers(2, 5, size=d - 1)] + [1]
    Y, Z = _rand_pair(n, r, s, seed)
    ell = hatt.plan_ranks(n, r, s, 6)
    R = philox.sketch_tt(seed, n, ell)
    A = tt.hadamard_pkp(Y, Z)
    Xr, Wr = randorth.randorth(A, R)
    Wh = hatt.hpcrl1_contract(Y, Z, R)
    for k in range(1, d):
        assert np.allclose(Wh[k], Wr[k], rtol=1e-12, atol=1e-14)
    Xh = hatt.hatt1_sweep(Y, Z, Wh)
    for a, b in zip(Xh, Xr):
        assert a.shape == b.shape
        assert np.allclose(a, b, rtol=1e-9, atol=1e-11 * np.abs(b).max())
    assert tt.tt_diff_norm(Xh, Xr) <= 1e-12 * tt.tt_norm(Xr)


def test_paper_form_equals_contract_form_end_to_end():
    n = [4, 3, 5, 4]
    Y, Z = _rand_pair(n, [1, 3, 4, 2, 1], [1, 2, 2, 3, 1], seed=40)
    Xa = hatt.hadamard_recompress(Y, Z, sketch_rank=5, seed=1, coding="paper")
    Xb = hatt.hadamard_recompress(Y, Z, sketch_rank=5, seed=1, coding="contract")
    assert tt.tt_diff_norm(Xa, Xb) <= 1e-13 * tt.tt_norm(Xb)


# ---------------------------------------------- brute force / exactness ---

def test_small_workload_brute_force():
    Y, Z, o = wl.workload_small_sin_times_random(seed=0)
    X, info = hatt.hadamard_recompress(Y, Z, seed=0, return_info=True, **o)
    assert info["ell"] == [1, 8, 10, 10, 10, 8, 1]
    dense = tt.tt_full(Y) * tt.tt_full(Z)          # 8^6 entries
    err = np.linalg.norm(tt.tt_full(X) - dense) / np.linalg.norm(dense)
    assert err <= 1e-13
    assert max(info["ranks"]) <= 10


@pytest.mark.parametrize("seed", [50, 51, 52, 53])
def test_exact_when_sketch_rank_is_pkp_rank(seed):
    """Theorem 3.1 with the range-finder argument: l_k >= separation rank
    reproduces Y ⊙ Z to rounding for any sketch."""
    rng = np.random.default_rng(seed)
    d = int(rng.integers(2, 6))
    n = [int(v) for v in rng.integers(2, 6, size=d)]
    r = [1] + [int(v) for v in rng.integers(1, 4, size=d - 1)] + [1]
    s = [1] + [int(v) for v in rng.integers(1, 4, size=d - 1)] + [1]
    Y, Z = _rand_pair(n, r, s, seed)
    X = hatt.hadamard_recompress(Y, Z, sketch_rank=100, seed=seed)
    dense = tt.tt_full(Y) * tt.tt_full(Z)
    assert np.linalg.norm(tt.tt_full(X) - dense) <= 1e-13 * np.linalg.norm(dense) * d


def test_order_one_and_two():
    Y1 = wl.gaussian_tt([7], [1, 1], 1)
    Z1 = wl.gaussian_tt([7], [1, 1], 2)
    X1 = hatt.hadamard_recompress(Y1, Z1, sketch_rank=3)
    assert np.allclose(tt.tt_full(X1), tt.tt_full(Y1) * tt.tt_full(Z1), rtol=1e-15)
    Y2 = wl.gaussian_tt([5, 6], [1, 3, 1], 3)
    Z2 = wl.gaussian_tt([5, 6], [1, 2, 1], 4)
    X2 = hatt.hadamard_recompress(Y2, Z2, sketch_rank=6)
    assert np.allclose(tt.tt_full(X2), tt.tt_full(Y2) * tt.tt_full(Z2), rtol=1e-12, atol=1e-14)


def test_mode_size_one():
    Y = wl.gaussian_tt([3, 1, 4, 1], [1, 2, 3, 2, 1], 5)
    Z = wl.gaussian_tt([3, 1, 4, 1], [1, 3, 2, 2, 1], 6)
    X = hatt.hadamard_recompress(Y, Z, sketch_rank=20)
    dense = tt.tt_full(Y) * tt.tt_full(Z)
    assert np.linalg.norm(tt.tt_full(X) - dense) <= 1e-13 * np.linalg.norm(dense)


# ---------------------------------------------------- closed forms (P4) ---

def test_sin_times_cos_closed_form():
    Y, Z, o = wl.workload_small_sin_times_cos()
    X, info = hatt.hadamard_recompress(Y, Z, seed=2, return_info=True, **o)
    d, n = 6, 8
    S = sum(np.meshgrid(*([wl.uniform_grid(n)] * d), indexing="ij"))
    assert np.allclose(tt.tt_full(X), 0.5 * np.sin(2 * S), atol=1e-13)
    # rank 2 everywhere after the tol = 1e-12 truncation
    assert info["ranks"] == [1, 2, 2, 2, 2, 2, 1]
    # ||Y ⊙ Z||^2 = 8^6 * 1/4 * 1/2 = 32768 exactly; <Y ⊙ Z, 1> = 0
    assert abs(tt.tt_norm(X) ** 2 - 32768.0) <= 1e-10
    assert abs(tt.tt_dot(X, wl.ones_tt([n] * d))) <= 1e-9


def test_theorem_3_1_sketch_rank_bound():
    """Theorem 3.1, rank W^{(k)} <= separation rank, holds for a minimal TT
    representation: ½ sin(2 sum x) rounded to its minimal ranks 2."""
    Y, Z, _ = wl.workload_small_sin_times_cos()
    A_min, rk = rounding.tt_round(tt.hadamard_pkp(Y, Z), 0, 1e-14)
    assert rk == [1, 2, 2, 2, 2, 2, 1]
    n = tt.modes(Y)
    R = philox.sketch_tt(8, n, [1] + [4] * 5 + [1])
    W = randorth.partial_contraction_rl(A_min, R)
    for k in range(1, 6):
        sv = np.linalg.svd(W[k], compute_uv=False)
        assert np.sum(sv > 1e-12 * sv[0]) <= 2


def test_pkp_sketch_rank_exceeds_separation_rank_but_unfolding_sketch_does_not():
    """With the non-minimal PKP representation the right factor H(A_{k:d})
    spans sin^2, sin cos, cos^2 of the right sum: rank 3 > 2, so W^{(k)} from
    HPCRL has rank 3. The sketch of the unfolding, A_<k> H(R_{k:d})^T, still
    has rank <= 2, which is what exact recompression needs."""
    Y, Z, _ = wl.workload_small_sin_times_cos()
    n = tt.modes(Y)
    ell = hatt.plan_ranks(n, tt.ranks(Y), tt.ranks(Z), 12)
    R = philox.sketch_tt(8, n, ell)
    W = hatt.hpcrl1_contract(Y, Z, R, normalize=False)
    full = tt.tt_full(Y) * tt.tt_full(Z)
    for k in range(1, 6):
        sv = np.linalg.svd(W[k], compute_uv=False)
        assert np.sum(sv > 1e-12 * sv[0]) == 3
        unf = full.reshape(8 ** k, -1)
        sk = unf @ _dense_right_part(R[k:]).T
        sv2 = np.linalg.svd(sk, compute_uv=False)
        assert np.sum(sv2 > 1e-12 * sv2[0]) <= 2


# ------------------------------------------------- TT identities (P5) ---

def test_identities_on_exact_recompression():
    n = [4, 5, 3, 4, 5]
    Y, Z = _rand_pair(n, [1, 3, 2, 3, 2, 1], [1, 2, 3, 2, 2, 1], seed=60)
    X = hatt.hadamard_recompress(Y, Z, sketch_rank=100, seed=3)
    ones = wl.ones_tt(n)
    # <Y ⊙ Z, 1> = <Y, Z>
    assert np.isclose(tt.tt_dot(X, ones), tt.tt_dot(Y, Z), rtol=1e-12)
    # ||Y ⊙ Z||^2 = <Y ⊙ Y, Z ⊙ Z>
    lhs = tt.tt_norm(X) ** 2
    rhs = tt.tt_dot(tt.hadamard_pkp(Y, Y), tt.hadamard_pkp(Z, Z))
    assert np.isclose(lhs, rhs, rtol=1e-12)
    # left-orthogonal output; the norm sits in the last core
    assert tt.is_left_orthogonal(X, atol=1e-13)
    assert np.isclose(np.linalg.norm(X[-1]), tt.tt_norm(X), rtol=1e-13)


# ---------------------------------------------------------- truncation ---

def test_truncation_honours_tolerance_and_matches_rounding():
    n = [5] * 5
    Y, Z = _rand_pair(n, [1, 3, 3, 3, 3, 1], [1, 3, 3, 3, 3, 1], seed=70)
    A = tt.hadamard_pkp(Y, Z)
    nA = tt.tt_norm(A)
    for tol in (1e-1, 1e-3):
        X, info = hatt.hadamard_recompress(Y, Z, sketch_rank=100, tol=tol, seed=1,
                                           return_info=True)
        err = tt.tt_diff_norm(X, A) / nA
        assert err <= tol * (1 + 1e-8)
        _, rk = rounding.tt_round(A, 0, tol)
        # exact sketch + exact truncation -> the same rank profile as TT-Rounding
        assert info["ranks"] == rk


def test_truncation_max_rank():
    n = [6] * 6
    Y, Z = _rand_pair(n, [1, 4, 4, 4, 4, 4, 1], [1, 4, 4, 4, 4, 4, 1], seed=71)
    X, info = hatt.hadamard_recompress(Y, Z, max_rank=5, sketch_rank=12, seed=2,
                                       return_info=True)
    assert max(info["ranks"]) <= 5
    assert tt.ranks(X) == info["ranks"]


# ------------------------------------------------------------ cost model ---

def test_flop_model_matches_table_4_1():
    d, n, r, s, l = 20, 32, 20, 20, 50
    ell = [1] + [l] * (d - 1) + [1]
    rr = [1] + [r] * (d - 1) + [1]
    hp, lr = flops.hatt1_flops([n] * d, rr, rr, ell)
    table = flops.table41_hatt1(d, n, r, s, l)
    # boundary cores have rank 1 and the -1 / -4/3 terms are dropped by the table
    assert abs((hp + lr) / table - 1.0) < 0.08


def test_speedup_closed_form_vs_randorth():
    # SP(l) = (4rs + 6l)/(4r + 4s + 6l); at l = r = s: (4r + 6)/14 (Section 4)
    for r in (5, 10, 20):
        d, n, l, s = 10, 8, r, r
        ro = (d - 2) * n * (4 * r ** 2 * s ** 2 * l + 6 * r * s * l ** 2)
        sp = ro / flops.table41_hatt1(d, n, r, s, l)
        assert np.isclose(sp, (4 * r + 6) / 14)


def test_package_cost_model_agrees_with_oracle_flop_model():
    from paper_2410_04385_gb300 import costmodel
    rng = np.random.default_rng(5)
    for _ in range(5):
        d = int(rng.integers(2, 12))
        n = [int(v) for v in rng.integers(1, 40, size=d)]
        r = [1] + [int(v) for v in rng.integers(1, 30, size=d - 1)] + [1]
        s = [1] + [int(v) for v in rng.integers(1, 30, size=d - 1)] + [1]
        ell = hatt.plan_ranks(n, r, s, int(rng.integers(1, 80)))
        a = costmodel.hatt1_flops(n, r, s, ell)
        b = flops.hatt1_flops(n, r, s, ell)
        assert np.allclose(a, b, rtol=1e-12)


def test_hatt2_with_ep_zero_equals_hatt1():
    """P6: with ep = 0 every nonzero singular value is kept, so HPCRL-2 forms
    the same sketches as HPCRL-1 and HaTT-2 equals HaTT-1 (same sketch)."""
    n = [5, 4, 6, 3, 5]
    Y = wl.gaussian_tt(n, [1, 3, 4, 4, 2, 1], 71)
    Z = wl.gaussian_tt(n, [1, 2, 3, 2, 3, 1], 72)
    W1 = hatt.hpcrl1_contract(Y, Z, philox.sketch_tt(4, n, hatt.plan_ranks(n, tt.ranks(Y), tt.ranks(Z), 7)))
    W2, kept = hatt.hpcrl2(Y, Z, philox.sketch_tt(4, n, hatt.plan_ranks(n, tt.ranks(Y), tt.ranks(Z), 7)), 0.0)
    for a, b in zip(W1[1:-1], W2[1:-1]):
        assert np.allclose(a, b, atol=1e-12 * np.abs(a).max())
    X1 = hatt.hadamard_recompress(Y, Z, sketch_rank=7, seed=4)
    X2 = hatt.hadamard_recompress(Y, Z, sketch_rank=7, seed=4, variant=2, ep=0.0)
    assert tt.tt_diff_norm(X1, X2) <= 1e-12 * tt.tt_norm(X1)


def test_hatt2_truncation_keeps_range_until_ep_is_large():
    """Y = sin(sum x) (rank 2) times a random rank-5 TT has TT ranks of 10 at
    most. Truncating W^{(k)} only shortens the next contraction: while the
    n*R rank-one terms still span the range, HaTT-2 stays exact, and the kept
    ranks R fall as ep grows. At ep = 0.95 only the dominant direction
    survives and the result is far off."""
    Y, Z, _ = wl.workload_small_sin_times_random()
    A = tt.tt_full(Y) * tt.tt_full(Z)
    n = [c.shape[1] for c in Y]
    ell = hatt.plan_ranks(n, tt.ranks(Y), tt.ranks(Z), 12)
    kept_prev = None
    for ep in (1e-12, 1e-2, 3e-1, 0.95):
        X = hatt.hadamard_recompress(Y, Z, sketch_rank=12, seed=0, variant=2, ep=ep)
        err = np.linalg.norm(tt.tt_full(X) - A) / np.linalg.norm(A)
        _, kept = hatt.hpcrl2(Y, Z, philox.sketch_tt(0, n, ell), ep)
        if kept_prev is not None:
            assert all(a <= b for a, b in zip(kept, kept_prev))
        kept_prev = kept
        if ep < 0.5:
            assert err <= 1e-13
        else:
            assert err > 1e-2 and max(kept) == 1


def test_hatt2_step_is_the_kronecker_definition_on_the_truncated_sketch():
    """Against the defining formula with explicit partial Kronecker cores
    A_k(i) = Y_k(i) (x) Z_k(i) (what HaTT never forms): every HPCRL-2 step is
    W^{(k-1)} = sum_i A_k(i) W~ R_k(i)^T / ||.||_F with W~ the rank-R_k
    truncated SVD of W^{(k)}, the R_k the recursion reports. ep = 0.3 cuts in
    the middle of the spectra, so the truncation is active at every step."""
    n = [4, 5, 3, 4, 5]
    Y = wl.gaussian_tt(n, [1, 3, 4, 3, 2, 1], 81)
    Z = wl.gaussian_tt(n, [1, 2, 3, 4, 2, 1], 82)
    ell = hatt.plan_ranks(n, tt.ranks(Y), tt.ranks(Z), 8)
    R = philox.sketch_tt(6, n, ell)
    W, kept = hatt.hpcrl2(Y, Z, R, 0.3)
    cut = 0
    for k in range(len(n) - 1, 0, -1):
        u, sv, vt = np.linalg.svd(W[k + 1], full_matrices=False)
        Rk = kept[k + 1]
        cut += Rk < len(sv)
        Wt = (u[:, :Rk] * sv[:Rk]) @ vt[:Rk]
        E = sum(np.kron(Y[k][:, i, :], Z[k][:, i, :]) @ Wt @ R[k][:, i, :].T for i in range(n[k]))
        E = E / np.linalg.norm(E)
        assert np.allclose(W[k], E, rtol=0, atol=1e-13)
    assert cut >= 2


def test_hatt_accuracy_below_the_numerical_rank_within_the_randomized_bound():
    """At a target rank r below the numerical rank the paper states no bound.
    A bound that holds in expectation follows from two published results: a
    rank-(r+p) Gaussian range finder leaves at most sqrt(1 + r/(p-1)) times
    the optimal tail at a bond (Halko, Martinsson, Tropp 2011, Thm 10.5), and
    a TT built by successive projections errs by at most the root sum of
    squares of its bond errors (Oseledets 2011, Thm 2.2). So
    ||A - X|| <= sqrt(sum_k (1 + r/(p-1)) tail_k(r)^2) in expectation, tail_k
    the optimal rank-r error of the k-th unfolding. Checked with a factor 2
    over five seeds on products of smooth TTs with decaying spectra; a
    transposed operand or a wrong index gives errors of order one."""
    d, n, p = 6, 8, 10
    for trial in range(2):
        Y = wl.smooth_tt(d, n, 6, seed=10 + trial)
        Z = wl.smooth_tt(d, n, 6, seed=20 + trial)
        A = tt.tt_full(Y) * tt.tt_full(Z)
        na = np.linalg.norm(A)
        for r in (3, 8):
            tails = [np.sqrt(np.sum(np.linalg.svd(A.reshape(n ** k, -1), compute_uv=False)[r:] ** 2))
                     for k in range(1, d)]
            bound = np.sqrt(np.sum((1.0 + r / (p - 1.0)) * np.square(tails)))
            lower = max(tails)
            for seed in range(5):
                X = hatt.hadamard_recompress(Y, Z, max_rank=r, oversample=p, seed=seed)
                err = np.linalg.norm(tt.tt_full(X) - A)
                assert lower * (1 - 1e-12) <= err <= 2.0 * bound
                assert max(tt.ranks(X)) <= r
            assert lower > 1e-3 * na          # the target is really below the numerical rank
