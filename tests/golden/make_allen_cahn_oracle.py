"""Writes allen_cahn_oracle_samples.npz: the oracle's Allen-Cahn trajectory
(Section 5, Example 4; explicit Euler, u^2 and u^3 by HaTT-1 with rank cap 24
and tolerance 1e-10, TT rounding to rank 24 / tolerance 1e-8) on [0, 2 pi)^8,
n = 64, eps = 0.1, dt = 1e-3, from the seeded initial condition, held at rank
24 (padded back with zeros after every step, the shapes the GPU's fixed-rank
stepper keeps), with sketch seeds 10 + 2 w and 11 + 2 w in step w -- the
seeds the stepper's graph draws when it advances its seed offset by 2 per
replay. Stores the state after STEPS steps at 4000 seeded multi-indices, the
discrete energy every 10 steps, and for every step and bond the singular
values of the tensor the rounding truncates at its cut (largest, last kept,
first dropped), its rank there and its norm.

Only the oracle and the seeded generators run here (about a second per step).
The GPU test and bench.py read the stored samples.

    python tests/golden/make_allen_cahn_oracle.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import allen_cahn as oac  # noqa: E402
from oracle import hatt as ohatt  # noqa: E402
from oracle import rounding as orounding  # noqa: E402
from oracle import tt as ott  # noqa: E402

D, N, EPS, DT, RANK, STEPS, SEED = 8, 64, 0.1, 1e-3, 24, 100, 10
TOL, HATT_TOL = 1e-8, 1e-10
SAMPLES, INDEX_SEED = 4000, 77


def pad(u, rank):
    d = len(u)
    rk = [1] + [max(int(c.shape[2]), rank) for c in u[:-1]] + [1]
    out = []
    for k, c in enumerate(u):
        p = np.zeros((rk[k], c.shape[1], rk[k + 1]))
        p[: c.shape[0], :, : c.shape[2]] = c
        out.append(p)
    return out


def entries(cores, idx):
    M = np.ones((idx.shape[0], 1))
    for k, c in enumerate(cores):
        M = np.einsum("sa,sab->sb", M, c[:, idx[:, k], :].transpose(1, 0, 2))
    return M[:, 0]


def main(out=os.path.join(HERE, "allen_cahn_oracle_samples.npz")):
    h = 2.0 * np.pi / N
    u = pad(oac.initial_condition(D, N, seed=0), RANK)
    energies = []
    cut = []                       # per step and bond: sigma_1, sigma_rho, sigma_rho+1, rank, ||w||
    for w in range(STEPS):
        # the steps of oracle.allen_cahn.step, with the spectrum of the tensor
        # the rounding truncates (for the resolution bound of the GPU test)
        seed = SEED + 2 * w
        u2 = ohatt.hadamard_recompress(u, u, max_rank=RANK, tol=HATT_TOL, seed=seed)
        u3 = ohatt.hadamard_recompress(u2, u, max_rank=RANK, tol=HATT_TOL, seed=seed + 1)
        wt = oac.lincomb_tt([u, oac.laplacian_tt(u, h), u3], [1.0 + DT, DT * EPS * EPS, -DT])
        sv = ott.bond_singular_values(wt)
        un, rk = orounding.tt_round(wt, RANK, TOL)
        nw = ott.tt_norm(wt)
        cut.append([[v[0], v[rk[k + 1] - 1], v[rk[k + 1]] if len(v) > rk[k + 1] else 0.0, len(v), nw]
                    for k, v in enumerate(sv)])
        u = pad(un, RANK)
        if w % 10 == 9:
            energies.append(oac.energy(u, u2, h, EPS, N, D))
            print("step", w + 1, "energy", energies[-1], flush=True)
    idx = np.random.default_rng(INDEX_SEED).integers(0, N, size=(SAMPLES, D))
    np.savez_compressed(out, idx=idx.astype(np.uint8), u=entries(u, idx),
                        energy_every_10=np.array(energies), steps=np.array(STEPS),
                        cut=np.array(cut), norm_u=np.array(ott.tt_norm(u)))
    print("wrote", out)


if __name__ == "__main__":
    main()
