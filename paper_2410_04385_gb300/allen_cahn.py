"""Allen-Cahn time stepping in TT format (Section 5, Example 4) through the
libhatt C ABI: explicit Euler for u_t = eps^2 Lap u + u - u^3 on the periodic
box [0, 2 pi)^d with central differences,
  u^{w+1} = round( (1 + dt) u^w + dt eps^2 Lap_h u^w - dt (u^w)^3 ),
u^2 = HaTT-1(u ⊙ u) and u^3 = HaTT-1(u^2 ⊙ u) (never the explicit Kronecker
cores), tt_round at a relative tolerance after every step, and the discrete
energy E = h^d [eps^2/2 (-<u, Lap_h u>) + 1/4 (<u^2, u^2> - 2 <u, u> + n^d)].
The module only sequences library calls (each call synchronizes to learn the
data-dependent output ranks)."""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import torch

from . import binding


def energy(u: Sequence[torch.Tensor], u2: Sequence[torch.Tensor], h: float, eps: float) -> float:
    d = len(u)
    n = int(u[0].shape[1])
    lap = binding.tt_laplacian(u, 1.0 / (h * h))
    grad = -float(binding.tt_dot(u, lap).item())
    quart = float(binding.tt_dot(u2, u2).item()) - 2.0 * float(binding.tt_dot(u, u).item()) + float(n) ** d
    return h ** d * (0.5 * eps * eps * grad + 0.25 * quart)


def step(u: Sequence[torch.Tensor], h: float, eps: float, dt: float, max_rank: int, tol: float,
         hatt_tol: float, seed: int, precision: int = binding.TT_FP64
         ) -> Tuple[List[torch.Tensor], List[torch.Tensor]]:
    """One explicit Euler step; returns (u_next, u^2)."""
    u2 = binding.tt_hadamard_recompress(u, u, max_rank=max_rank, tol=hatt_tol, seed=seed,
                                        precision=precision)
    u3 = binding.tt_hadamard_recompress(u2, u, max_rank=max_rank, tol=hatt_tol, seed=seed + 1,
                                        precision=precision)
    lap = binding.tt_laplacian(u, 1.0 / (h * h))
    w = binding.tt_lincomb([u, lap, u3], [1.0 + dt, dt * eps * eps, -dt])
    un = binding.tt_round(w, max_rank, tol)
    return [c.contiguous() for c in un], u2
