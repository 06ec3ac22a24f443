"""Pins for the oracle's TT basics (Section 2.1-2.2) against dense brute force."""
import numpy as np

from oracle import tt
from paper_2410_04385_gb300 import workloads as wl


def _dense_grid_sum(d, n):
    x = wl.uniform_grid(n)
    grids = np.meshgrid(*([x] * d), indexing="ij")
    return sum(grids)


def test_sin_cos_generators_match_closed_form():
    d, n = 4, 5
    S = _dense_grid_sum(d, n)
    assert np.allclose(tt.tt_full(wl.sin_sum_tt(d, n, "sin")), np.sin(S), atol=1e-14)
    assert np.allclose(tt.tt_full(wl.sin_sum_tt(d, n, "cos")), np.cos(S), atol=1e-14)
    assert tt.ranks(wl.sin_sum_tt(d, n)) == [1, 2, 2, 2, 1]


def test_fourier_generator_matches_function():
    d, n = 3, 4
    coef = np.array([1.5, -0.25, 2.0])
    N = n ** d
    # mode 1 fastest: flat index i_1 + i_2 n + i_3 n^2, t = 2 pi (1 + flat) / N
    idx = np.arange(N)
    t = 2 * np.pi * (1 + idx) / N
    ys = sum(c * np.sin((j + 1) * t) for j, c in enumerate(coef))
    yc = sum(c * np.cos((j + 1) * t) for j, c in enumerate(coef))
    Ts = tt.tt_full(wl.fourier_series_tt(d, n, coef, "sin"))
    Tc = tt.tt_full(wl.fourier_series_tt(d, n, coef, "cos"))
    # dense TT is row-major in (i_1, ..., i_d); flat index with mode 1 fastest
    Ts_flat = Ts.transpose(range(d - 1, -1, -1)).ravel()
    Tc_flat = Tc.transpose(range(d - 1, -1, -1)).ravel()
    assert np.allclose(Ts_flat, ys, atol=1e-12)
    assert np.allclose(Tc_flat, yc, atol=1e-12)


def test_pkp_gives_hadamard_product():
    Y = wl.gaussian_tt([3, 4, 2, 5], [1, 2, 3, 4, 1], seed=1)
    Z = wl.gaussian_tt([3, 4, 2, 5], [1, 3, 1, 2, 1], seed=2)
    A = tt.hadamard_pkp(Y, Z)
    assert tt.ranks(A) == [1, 6, 3, 8, 1]
    assert np.allclose(tt.tt_full(A), tt.tt_full(Y) * tt.tt_full(Z), rtol=1e-13, atol=1e-15)


def test_pkp_entry_formula():
    y = np.arange(2 * 3 * 4, dtype=float).reshape(2, 3, 4)
    z = np.arange(5 * 3 * 2, dtype=float).reshape(5, 3, 2) - 7
    p = tt.pkp_core(y, z)
    for a in range(2):
        for b in range(5):
            for i in range(3):
                for a1 in range(4):
                    for b1 in range(2):
                        assert p[a * 5 + b, i, a1 * 2 + b1] == y[a, i, a1] * z[b, i, b1]


def test_dot_norm_and_diff_vs_dense():
    Y = wl.gaussian_tt([4, 3, 5, 2], [1, 3, 2, 4, 1], seed=3)
    Z = wl.gaussian_tt([4, 3, 5, 2], [1, 2, 5, 3, 1], seed=4)
    fy, fz = tt.tt_full(Y), tt.tt_full(Z)
    assert np.isclose(tt.tt_dot(Y, Z), np.sum(fy * fz), rtol=1e-13)
    assert np.isclose(tt.tt_norm(Y), np.linalg.norm(fy), rtol=1e-13)
    assert np.isclose(tt.tt_diff_norm(Y, Z), np.linalg.norm(fy - fz), rtol=1e-12)


def test_diff_norm_is_stable_below_sqrt_eps():
    Y = wl.gaussian_tt([6] * 5, [1, 4, 4, 4, 4, 1], seed=5)
    eps = 1e-13
    Y2 = [c.copy() for c in Y]
    Y2[2] = Y2[2] * (1 + eps)
    rel = tt.tt_diff_norm(Y, Y2) / tt.tt_norm(Y)
    assert abs(rel / eps - 1.0) < 1e-2


def test_left_orthogonalize():
    Y = wl.gaussian_tt([3, 4, 5, 3], [1, 3, 4, 2, 1], seed=6)
    L = tt.left_orthogonalize(Y)
    assert tt.is_left_orthogonal(L, atol=1e-13)
    assert np.allclose(tt.tt_full(L), tt.tt_full(Y), atol=1e-13)
    assert np.isclose(np.linalg.norm(L[-1]), np.linalg.norm(tt.tt_full(Y)), rtol=1e-13)


def test_bond_singular_values_equal_those_of_the_dense_unfoldings():
    A = wl.gaussian_tt([3, 4, 5, 3], [1, 2, 6, 3, 1], 5)
    full = tt.tt_full(A)
    sv = tt.bond_singular_values(A)
    for k in range(1, 4):
        dense = np.linalg.svd(full.reshape(int(np.prod(full.shape[:k])), -1), compute_uv=False)
        m = len(sv[k - 1])
        assert np.allclose(sv[k - 1], dense[:m], rtol=1e-12, atol=1e-14 * dense[0])
        assert np.all(dense[m:] <= 1e-12 * dense[0])
