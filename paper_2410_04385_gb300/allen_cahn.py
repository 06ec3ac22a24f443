"""Allen-Cahn time stepping in TT format (Section 5, Example 4) through the
libhatt C ABI: explicit Euler for u_t = eps^2 Lap u + u - u^3 on the periodic
box [0, 2 pi)^d with central differences,
  u^{w+1} = round( (1 + dt) u^w + dt eps^2 Lap_h u^w - dt (u^w)^3 ),
u^2 = HaTT-1(u ⊙ u) and u^3 = HaTT-1(u^2 ⊙ u) (never the explicit Kronecker
cores), tt_round at a relative tolerance after every step, and the discrete
energy E = h^d [eps^2/2 (-<u, Lap_h u>) + 1/4 (<u^2, u^2> - 2 <u, u> + n^d)].
`step` sequences library calls (each call synchronizes to learn the
data-dependent output ranks); `FixedRankStepper` keeps every shape fixed and
replays one captured step."""
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


def pad_ranks(u: Sequence[torch.Tensor], rank: int) -> List[torch.Tensor]:
    """The same TT with every inner rank raised to `rank` by zero rows and
    columns (no rank is lowered)."""
    d = len(u)
    rk = [1] + [max(int(c.shape[2]), rank) for c in u[:-1]] + [1]
    out = []
    for k, c in enumerate(u):
        p = torch.zeros((rk[k], c.shape[1], rk[k + 1]), dtype=c.dtype, device=c.device)
        p[: c.shape[0], :, : c.shape[2]] = c
        out.append(p)
    return out


class FixedRankStepper:
    """Explicit Euler steps with every shape fixed, so one step can be captured
    in a CUDA graph and replayed: u is held at the padded rank `rank` (zero
    past the ranks the rounding keeps), both HaTT-1 calls and the rounding run
    with fixed_ranks=1, and the Laplacian, the combination and the rounding
    write into buffers planned once. With fresh_seeds the sketches of step w
    use the keys seed + 2 w and seed + 1 + 2 w: a device counter (the calls'
    seed_offset) that every step, graph replays included, advances by 2;
    without it every step uses seed and seed + 1."""

    def __init__(self, u0: Sequence[torch.Tensor], h: float, eps: float, dt: float, rank: int,
                 tol: float, hatt_tol: float, hatt_rank: int, seed: int,
                 precision: int = binding.TT_FP64, fresh_seeds: bool = False):
        self.h, self.eps, self.dt = h, eps, dt
        self.u = [c.contiguous().clone() for c in pad_ranks(u0, rank)]
        ranks = [int(self.u[0].shape[0])] + [int(c.shape[2]) for c in self.u]
        dev = self.u[0].device
        self.seed_counter = torch.zeros(1, dtype=torch.int64, device=dev) if fresh_seeds else None
        self.h1 = binding.HadamardRecompressor(self.u, self.u, max_rank=hatt_rank, tol=hatt_tol,
                                               seed=seed, precision=precision, fixed_ranks=1,
                                               seed_offset=self.seed_counter)
        self.u2 = self.h1.result()
        self.h2 = binding.HadamardRecompressor(self.u2, self.u, max_rank=hatt_rank, tol=hatt_tol,
                                               seed=seed + 1, precision=precision, fixed_ranks=1,
                                               seed_offset=self.seed_counter)
        self.u3 = self.h2.result()
        self.lap = binding.tt_laplacian(self.u, 1.0 / (h * h))
        self.coef = [1.0 + dt, dt * eps * eps, -dt]
        self.w = binding.tt_lincomb([self.u, self.lap, self.u3], self.coef)
        self.rnd = binding.Rounder(self.w, max_rank=rank, tol=tol, fixed_ranks=1)
        self.un = self.rnd.result()
        if [int(self.un[0].shape[0])] + [int(c.shape[2]) for c in self.un] != ranks:
            raise ValueError("the rounding bound differs from the padded rank: lower `rank` to "
                             "at most the mode-size products")
        self.graph = None

    def step(self):
        """One step, enqueued on the current stream (nothing is read back)."""
        self.h1.run()
        self.h2.run()
        binding.tt_laplacian(self.u, 1.0 / (self.h * self.h), out=self.lap)
        binding.tt_lincomb([self.u, self.lap, self.u3], self.coef, out=self.w)
        self.rnd.run()
        for a, b in zip(self.u, self.un):
            a.copy_(b)
        if self.seed_counter is not None:
            self.seed_counter.add_(2)

    def capture(self):
        """Capture one step in a CUDA graph. The eager warm-up before the
        capture is a real step: u has advanced by one step on return."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def energy(self) -> float:
        return energy(self.u, self.u2, self.h, self.eps)
