"""Seeded synthetic TT inputs shaped like the HaTT paper's experiments.

This module holds input generators only: it builds TT cores from closed-form
functions or seeded random numbers. It contains none of the recompression
arithmetic (no Hadamard products, contractions, QR, rounding or norms), so the
CPU oracle and the CUDA path can both draw their inputs from it without sharing
any of the method.

Every core is a C-ordered float64 numpy array of shape (r_{k-1}, n_k, r_k),
r_0 = r_d = 1 (the TT format of Section 2.2, Eq. (2.1)-(2.2)).
"""
from __future__ import annotations

import numpy as np


def uniform_grid(n: int) -> np.ndarray:
    """Points 2*pi*j/n, j = 0..n-1 (a uniform grid over [0, 2*pi))."""
    return 2.0 * np.pi * np.arange(n, dtype=np.float64) / n


def gaussian_tt(n, ranks, seed: int):
    """Random TT with i.i.d. N(0, 1/(n_k r_k)) cores, r_k the right rank.

    With that variance E||Y||_F^2 = 1 for any order, so the "unit-norm" random
    operands of the paper's random-TT experiments are reproduced in scale.
    `n` is a list of mode sizes, `ranks` the d+1 bond ranks (ends equal to 1).
    """
    n = [int(v) for v in n]
    ranks = [int(v) for v in ranks]
    d = len(n)
    assert len(ranks) == d + 1 and ranks[0] == 1 and ranks[-1] == 1
    rng = np.random.default_rng(seed)
    cores = []
    for k in range(d):
        std = 1.0 / np.sqrt(n[k] * ranks[k + 1])
        cores.append(rng.standard_normal((ranks[k], n[k], ranks[k + 1])) * std)
    return cores


def uniform_tt(n, ranks, seed: int):
    """Random uniform TT: cores with i.i.d. U[0, 1] entries (Definition 2.1)."""
    rng = np.random.default_rng(seed)
    d = len(n)
    return [rng.random((int(ranks[k]), int(n[k]), int(ranks[k + 1]))) for k in range(d)]


def sin_sum_tt(d: int, n: int, phase: str = "sin"):
    """Rank-2 TT of sin(x_1+...+x_d) (phase="sin") or cos(x_1+...+x_d) on the
    uniform grid. Built from the angle-addition identities:
    the state [sin S_k, cos S_k] with S_k = x_1+...+x_k is carried left to right.
    """
    x = uniform_grid(n)
    s, c = np.sin(x), np.cos(x)
    if d == 1:
        f = s if phase == "sin" else c
        return [f.reshape(1, n, 1).copy()]
    first = np.stack([s, c], axis=-1).reshape(1, n, 2)
    mid = np.empty((2, n, 2))
    mid[0, :, 0], mid[0, :, 1] = c, -s
    mid[1, :, 0], mid[1, :, 1] = s, c
    last = np.empty((2, n, 1))
    if phase == "sin":
        last[0, :, 0], last[1, :, 0] = c, s
    else:
        last[0, :, 0], last[1, :, 0] = -s, c
    return [first] + [mid.copy() for _ in range(d - 2)] + [last]


def ones_tt(n):
    """Rank-1 TT of the all-ones tensor."""
    return [np.ones((1, int(m), 1)) for m in n]


def smooth_tt(d: int, n: int, rank: int, seed: int, terms: int = 8, rho: float = 0.5,
              gauge: bool = True):
    """Smooth TT with decaying spectrum: Y = sum_j rho^(j-1) prod_k f_jk(x_k),
    f_jk(x) = sum_{q<terms} a cos(w x + phi), w uniform in {1..6}, a ~ N(0,1),
    phi ~ U[0, 2pi); each f_jk is scaled to unit 2-norm over the grid, so
    ||Y|| is close to 1. The diagonal-core representation is made dense with
    random orthogonal gauges G_k <- O_{k-1}^T G_k O_k, which leave the tensor
    unchanged.
    """
    rng = np.random.default_rng(seed)
    x = uniform_grid(n)
    R = int(rank)
    f = np.zeros((d, R, n))
    for k in range(d):
        for j in range(R):
            w = rng.integers(1, 7, size=terms)
            a = rng.standard_normal(terms)
            ph = rng.uniform(0.0, 2.0 * np.pi, size=terms)
            v = (a[:, None] * np.cos(w[:, None] * x[None, :] + ph[:, None])).sum(0)
            f[k, j] = v / np.linalg.norm(v)
    weights = rho ** np.arange(R)
    cores = []
    for k in range(d):
        if k == 0:
            g = (weights[:, None] * f[0]).T.reshape(1, n, R)
        elif k == d - 1:
            g = f[k].reshape(R, n, 1).copy()
        else:
            g = np.zeros((R, n, R))
            for j in range(R):
                g[j, :, j] = f[k, j]
        cores.append(g)
    if d == 1:
        return [(weights[:, None] * f[0]).sum(0).reshape(1, n, 1)]
    if gauge:
        gauges = [np.ones((1, 1))]
        for k in range(1, d):
            q, rr = np.linalg.qr(rng.standard_normal((R, R)))
            gauges.append(q * np.sign(np.diag(rr))[None, :])
        gauges.append(np.ones((1, 1)))
        for k in range(d):
            g = cores[k]
            g = np.einsum("ab,bic->aic", gauges[k].T, g)
            g = np.einsum("aic,cd->aid", g, gauges[k + 1])
            cores[k] = np.ascontiguousarray(g)
    return cores


def fourier_series_tt(d: int, n: int, coef, kind: str = "sin"):
    """TT of t -> sum_j coef[j-1] * kind(j t), t = 2*pi*(1 + sum_k i_k n^k)/n^d
    (mode 1 fastest), the folding of the paper's Fourier-series example.
    Each sin(jt)/cos(jt) is a rank-2 TT in the folded digits; the sum is
    formed exactly by stacking the terms block-diagonally (rank 2*J).
    """
    coef = np.asarray(coef, dtype=np.float64)
    J = coef.size
    N = float(n) ** d
    i = np.arange(n, dtype=np.float64)
    # t = 2*pi*(1 + sum_k i_k n^k)/N = theta_0 + sum_k theta_k(i_k)
    cores = []
    R = 2 * J
    for k in range(d):
        ang = np.zeros((J, n))
        for j in range(1, J + 1):
            base = 2.0 * np.pi * j / N
            ang[j - 1] = base * (i * n ** k + (1.0 if k == 0 else 0.0))
        s, c = np.sin(ang), np.cos(ang)
        if k == 0:
            g = np.zeros((1, n, R))
            g[0, :, 0::2] = s.T
            g[0, :, 1::2] = c.T
        elif k == d - 1:
            g = np.zeros((R, n, 1))
            if kind == "sin":
                g[0::2, :, 0] = c * coef[:, None]
                g[1::2, :, 0] = s * coef[:, None]
            else:
                g[0::2, :, 0] = -s * coef[:, None]
                g[1::2, :, 0] = c * coef[:, None]
        else:
            g = np.zeros((R, n, R))
            for j in range(J):
                g[2 * j, :, 2 * j] = c[j]
                g[2 * j, :, 2 * j + 1] = -s[j]
                g[2 * j + 1, :, 2 * j] = s[j]
                g[2 * j + 1, :, 2 * j + 1] = c[j]
        cores.append(g)
    return cores


def ranks_of(cores):
    """Bond ranks [r_0, ..., r_d] of a core list."""
    return [int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]


def modes_of(cores):
    return [int(c.shape[1]) for c in cores]


# --- named workloads -------------------------------------------------------

def workload_small_sin_times_random(seed: int = 0):
    """d=6, n=8: Y = sin(sum x) (rank 2), Z = Gaussian TT with inner ranks 5.
    Sketch rank 12, max rank 10, tol 1e-12."""
    d, n = 6, 8
    Y = sin_sum_tt(d, n, "sin")
    Z = gaussian_tt([n] * d, [1] + [5] * (d - 1) + [1], seed)
    return Y, Z, dict(max_rank=10, tol=1e-12, sketch_rank=12)


def workload_small_sin_times_cos():
    """d=6, n=8: Y = sin(sum x), Z = cos(sum x); the product is
    0.5*sin(2 sum x), of TT rank 2."""
    d, n = 6, 8
    return sin_sum_tt(d, n, "sin"), sin_sum_tt(d, n, "cos"), dict(max_rank=10, tol=1e-12,
                                                                  sketch_rank=12)


def workload_random_d20(seed_y: int = 1, seed_z: int = 2):
    """d=20, n=32, all inner ranks 20 for both operands (PKP rank 400);
    target rank 40 with an oversampled sketch of rank 50."""
    d, n, r = 20, 32, 20
    rk = [1] + [r] * (d - 1) + [1]
    return (gaussian_tt([n] * d, rk, seed_y), gaussian_tt([n] * d, rk, seed_z),
            dict(max_rank=40, tol=0.0, sketch_rank=50))


def workload_smooth_d50(seed_y: int = 3, seed_z: int = 4):
    """d=50, n=64, ranks 40, smooth cores; target rank 80, sketch 90, tol 1e-8."""
    d, n, r = 50, 64, 40
    return (smooth_tt(d, n, r, seed_y), smooth_tt(d, n, r, seed_z),
            dict(max_rank=80, tol=1e-8, sketch_rank=90))


def workload_batch_uneven(count: int = 256, seed: int = 7, d_range=(10, 40), n_choices=(16, 32, 64),
                          r_range=(8, 48)):
    """Many independent pairs of uneven order, mode size and rank: per pair
    d uniform in d_range, one mode size from n_choices, every inner rank of
    Y and of Z uniform in r_range, Gaussian cores; sketch rank = target rank
    = 2 max(r_Y, r_Z) (clamped by the plan to the PKP ranks and unfolding
    sizes), so no truncation sweep follows. Returns a list of (Y, Z, opts)."""
    rng = np.random.default_rng(seed)
    pairs = []
    for j in range(count):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        n = int(rng.choice(n_choices))
        ry = [1] + [int(v) for v in rng.integers(r_range[0], r_range[1] + 1, size=d - 1)] + [1]
        rz = [1] + [int(v) for v in rng.integers(r_range[0], r_range[1] + 1, size=d - 1)] + [1]
        Y = gaussian_tt([n] * d, ry, int(rng.integers(1 << 30)))
        Z = gaussian_tt([n] * d, rz, int(rng.integers(1 << 30)))
        target = 2 * max(max(ry), max(rz))
        pairs.append((Y, Z, dict(sketch_rank=target, max_rank=target, oversample=0)))
    return pairs


def separable_sum_tt(g):
    """TT of f(x_1..x_d) = sum_k g[k](x_k) (g: list of d vectors of length n)
    in the rank-d form of a d-term canonical decomposition: bond ranks
    {1, d, ..., d, 1}; term j is the product over k of g[k] if k == j and of
    ones otherwise, carried on bond index j (diagonal inner cores)."""
    d = len(g)
    n = len(g[0])
    cores = []
    for k in range(d):
        a = 1 if k == 0 else d
        b = 1 if k == d - 1 else d
        c = np.zeros((a, n, b))
        for j in range(d):
            vec = np.asarray(g[k], dtype=np.float64) if j == k else np.ones(n)
            c[0 if k == 0 else j, :, 0 if k == d - 1 else j] = vec
        cores.append(c)
    return cores


def qing_grid(d: int, n: int = 10):
    """Per-coordinate terms of the Qing function (x_i - i)^2, i = 1..d, on a
    uniform grid of n points over [-500, 500] (endpoints included)."""
    x = np.linspace(-500.0, 500.0, n)
    return [(x - (k + 1)) ** 2 for k in range(d)]


def alpine_grid(d: int, n: int = 10):
    """Per-coordinate terms |x sin x + 0.1 x| of the Alpine function on a
    uniform grid of n points over [-2.5 pi, 2.5 pi]."""
    x = np.linspace(-2.5 * np.pi, 2.5 * np.pi, n)
    return [np.abs(x * np.sin(x) + 0.1 * x) for _ in range(d)]


def ones_tt_list(d: int, n: int = 10):
    """The all-ones TT (rank 1), the power iteration's start."""
    return [np.ones((1, n, 1)) for _ in range(d)]
