"""Allen-Cahn time stepping in TT format (Section 5, Example 4), plain float64
numpy. TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke()
and bench.py's baseline leg.

Equation u_t = eps^2 Lap u + u - u^3 on the periodic box [0, 2 pi)^d, second
order central differences with n points per axis (h = 2 pi / n). Reading:
the paper integrates a relaxed discrete-variational-derivative scheme with
QTT / DMRG solvers (third-party solvers); here the time integrator is
explicit Euler with the Laplacian applied (not solved),
  u^{w+1} = (1 + dt) u^w + dt eps^2 Lap_h u^w - dt (u^w)^3,
which is stable for dt eps^2 4 d / h^2 < 2; u^2 and u^3 = u^2 ⊙ u are HaTT-1
recompressions and every step ends with TT rounding at a relative tolerance.
The discrete energy
  E = h^d [ eps^2 / 2 (-<u, Lap_h u>) + 1/4 (<u^2, u^2> - 2 <u, u> + n^d) ]
is the quantity whose decay is checked."""
from __future__ import annotations

import numpy as np

from . import hatt
from . import rounding
from . import tt


def second_difference(n, h):
    """Periodic 3-point second difference (n x n): (u_{i+1} - 2 u_i + u_{i-1}) / h^2."""
    D = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    D[0, -1] = D[-1, 0] = 1.0
    return D / (h * h)


def laplacian_tt(u, h):
    """Lap_h u = sum_k I x .. x D_k x .. x I applied to the TT u, as a TT of
    ranks 2 r_k: core k = [[u_k, D u_k], [0, u_k]] (first core the top row,
    last core the right column)."""
    d = len(u)
    if d == 1:
        D = second_difference(u[0].shape[1], h)
        return [np.einsum("ij,ajb->aib", D, u[0])]
    out = []
    for k, c in enumerate(u):
        a, n, b = c.shape
        Dc = np.einsum("ij,ajb->aib", second_difference(n, h), c)
        if k == 0:
            out.append(np.concatenate([c, Dc], axis=2))                  # 1 x n x 2b
        elif k == d - 1:
            out.append(np.concatenate([Dc, c], axis=0))                  # 2a x n x 1
        else:
            blk = np.zeros((2 * a, n, 2 * b))
            blk[:a, :, :b] = c
            blk[:a, :, b:] = Dc
            blk[a:, :, b:] = c
            out.append(blk)
    return out


def lincomb_tt(terms, coef):
    """sum_j coef[j] * terms[j] as one TT with block-diagonal cores (ranks add;
    the coefficients scale the first cores)."""
    d = len(terms[0])
    if d == 1:
        return [sum(c * t[0] for c, t in zip(coef, terms))]
    out = []
    for k in range(d):
        if k == 0:
            out.append(np.concatenate([c * t[0] for c, t in zip(coef, terms)], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([t[-1] for t in terms], axis=0))
        else:
            A = sum(t[k].shape[0] for t in terms)
            Bd = sum(t[k].shape[2] for t in terms)
            n = terms[0][k].shape[1]
            blk = np.zeros((A, n, Bd))
            ia = ib = 0
            for t in terms:
                a, _, b = t[k].shape
                blk[ia:ia + a, :, ib:ib + b] = t[k]
                ia += a
                ib += b
            out.append(blk)
    return out


def initial_condition(d, n, terms=4, seed=0):
    """sum_{j<terms} prod_i sin(k_ij x_i), k_ij uniform in {1, 2, 3}, as a TT
    of ranks {1, terms, ..., terms, 1} (x_i = 2 pi m / n)."""
    rng = np.random.default_rng(seed)
    K = rng.integers(1, 4, size=(terms, d))
    x = 2.0 * np.pi * np.arange(n) / n
    cores = []
    for i in range(d):
        a = 1 if i == 0 else terms
        b = 1 if i == d - 1 else terms
        c = np.zeros((a, n, b))
        for j in range(terms):
            c[0 if i == 0 else j, :, 0 if i == d - 1 else j] = np.sin(K[j, i] * x)
        cores.append(c)
    return cores


def energy(u, u2, h, eps, n, d):
    """Discrete energy from u and (an approximation of) u^2."""
    lap = laplacian_tt(u, h)
    grad = -tt.tt_dot(u, lap)
    quart = tt.tt_dot(u2, u2) - 2.0 * tt.tt_dot(u, u) + float(n) ** d
    return h ** d * (0.5 * eps * eps * grad + 0.25 * quart)


def step(u, h, eps, dt, max_rank, tol, hatt_tol, seed):
    """One explicit Euler step; returns (u_next, u2)."""
    u2 = hatt.hadamard_recompress(u, u, max_rank=max_rank, tol=hatt_tol, seed=seed)
    u3 = hatt.hadamard_recompress(u2, u, max_rank=max_rank, tol=hatt_tol, seed=seed + 1)
    w = lincomb_tt([u, laplacian_tt(u, h), u3], [1.0 + dt, dt * eps * eps, -dt])
    un, _ = rounding.tt_round(w, max_rank, tol)
    return un, u2
