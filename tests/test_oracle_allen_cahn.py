"""Pins of the oracle's Allen-Cahn pieces against dense arithmetic."""
import numpy as np
import pytest

from oracle import allen_cahn as ac
from oracle import tt as ott


def dense_laplacian(U, h):
    out = np.zeros_like(U)
    for ax in range(U.ndim):
        out += (np.roll(U, -1, ax) - 2 * U + np.roll(U, 1, ax)) / (h * h)
    return out


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_laplacian_tt_is_the_dense_stencil(d):
    n, h = 7, 0.3
    u = [np.random.default_rng(d).standard_normal(s) for s in
         [(1 if k == 0 else 3, n, 1 if k == d - 1 else 3) for k in range(d)]]
    L = ac.laplacian_tt(u, h)
    assert np.allclose(ott.tt_full(L), dense_laplacian(ott.tt_full(u), h), atol=1e-9)
    if d > 1:
        assert ott.ranks(L)[1:-1] == [6] * (d - 1)


def test_second_difference_annihilates_constants_and_is_periodic():
    D = ac.second_difference(8, 0.5)
    assert np.allclose(D @ np.ones(8), 0)
    assert D[0, 7] == D[7, 0] == 4.0
    x = 2 * np.pi * np.arange(64) / 64
    # exact on sin(kx) up to the symbol 2(cos(kh) - 1)/h^2
    h = 2 * np.pi / 64
    assert np.allclose(ac.second_difference(64, h) @ np.sin(3 * x), 2 * (np.cos(3 * h) - 1) / h ** 2 * np.sin(3 * x))


def test_lincomb_tt_is_the_dense_combination():
    rng = np.random.default_rng(4)
    shapes = lambda r: [(1, 5, r), (r, 5, r + 1), (r + 1, 5, 1)]
    T = [[rng.standard_normal(s) for s in shapes(r)] for r in (1, 2, 4)]
    coef = [0.5, -2.0, 3.0]
    S = ac.lincomb_tt(T, coef)
    assert np.allclose(ott.tt_full(S), sum(c * ott.tt_full(t) for c, t in zip(coef, T)))
    assert ott.ranks(S) == [1, 7, 10, 1]


def test_initial_condition_is_the_sum_of_sines():
    d, n = 3, 8
    u = ac.initial_condition(d, n, seed=5)
    K = np.random.default_rng(5).integers(1, 4, size=(4, d))
    x = 2 * np.pi * np.arange(n) / n
    G = np.meshgrid(*([x] * d), indexing="ij")
    dense = sum(np.prod([np.sin(K[j, i] * G[i]) for i in range(d)], axis=0) for j in range(4))
    assert np.allclose(ott.tt_full(u), dense)


def test_tt_time_stepping_matches_dense_explicit_euler():
    """d = 2, n = 16: with sketch and rounding ranks that cover every bond
    (no truncation error), ten TT steps equal ten dense explicit Euler steps,
    and the discrete energy decreases."""
    d, n, eps, dt = 2, 16, 0.1, 1e-3
    h = 2 * np.pi / n
    u = ac.initial_condition(d, n, seed=1)
    U = ott.tt_full(u)
    for w in range(10):
        u, _ = ac.step(u, h, eps, dt, max_rank=16, tol=1e-14, hatt_tol=0.0, seed=10 * w)
        U = U + dt * (eps * eps * dense_laplacian(U, h) + U - U ** 3)
    assert np.allclose(ott.tt_full(u), U, atol=1e-10)


def test_energy_formula_and_decay_on_dense_grid():
    d, n, eps, dt = 2, 16, 0.1, 1e-3
    h = 2 * np.pi / n
    u = ac.initial_condition(d, n, seed=2)
    prev = None
    for w in range(5):
        U = ott.tt_full(u)
        u2 = ott.hadamard_pkp(u, u)                      # exact u^2 for the energy
        E = ac.energy(u, u2, h, eps, n, d)
        dense = h ** d * (0.5 * eps ** 2 * np.sum(-U * dense_laplacian(U, h)) + 0.25 * np.sum((U ** 2 - 1) ** 2))
        assert E == pytest.approx(dense, rel=1e-12)
        if prev is not None:
            assert E < prev
        prev = E
        u, _ = ac.step(u, h, eps, dt, max_rank=16, tol=1e-14, hatt_tol=0.0, seed=w)
