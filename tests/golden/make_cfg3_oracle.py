"""Writes cfg3_oracle_samples.npz: the FP64 oracle's HaTT-1 result for the
smooth d = 50, n = 64, rank-40 workload (sketch rank 90, target rank 80,
tol 1e-8, sketch seed 9), once with exact FP64 sketch products and once with
each emulated low-precision format (FP32, TF32, BF16 operands of the HPCRL-1
products, reading C6 / C7), sampled at 4000 seeded multi-indices, together
with the exact entries Y * Z there. Also the untruncated FP64 result (sketch
rank 90, no truncation sweep) at the same indices, once by each of the
oracle's two codings of HPCRL-1 and the core update, and per bond its singular
values at the cut (ranks rho and rho + 1 of the truncated result) with the
sketch rank there, from which the GPU test derives the resolution bound of a
Gram-based truncation.

Only the oracle and the seeded input generators run here (about 100 s per
format on eight cores). The GPU parity test at full configuration size and
the per-precision comparison of bench.py read the stored samples: the oracle
itself is too slow to run inside them.

    python tests/golden/make_cfg3_oracle.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import hatt as ohatt  # noqa: E402
from oracle import tt as ott  # noqa: E402
from paper_2410_04385_gb300 import workloads  # noqa: E402

SKETCH_SEED = 9
SAMPLES = 4000
INDEX_SEED = 2024
FORMATS = ("fp64", "fp32", "tf32", "bf16")


def sample_indices(d: int, n: int) -> np.ndarray:
    return np.random.default_rng(INDEX_SEED).integers(0, n, size=(SAMPLES, d))


def entries(cores, idx):
    """Entries of a TT at the multi-indices idx (samples x d)."""
    M = np.ones((idx.shape[0], 1))
    for k, c in enumerate(cores):
        M = np.einsum("sa,sab->sb", M, c[:, idx[:, k], :].transpose(1, 0, 2))
    return M[:, 0]


def main(out=os.path.join(HERE, "cfg3_oracle_samples.npz")):
    Y, Z, opts = workloads.workload_smooth_d50()
    d, n = len(Y), int(Y[0].shape[1])
    idx = sample_indices(d, n)
    rec = {"idx": idx.astype(np.uint8), "exact": entries(Y, idx) * entries(Z, idx)}
    Xu = ohatt.hadamard_recompress(Y, Z, seed=SKETCH_SEED, sketch_rank=opts["sketch_rank"])
    rec["x_fp64_notrunc"] = entries(Xu, idx)
    # the same sketch through the oracle's second coding of HPCRL-1 and the core
    # update (the paper's W_L / W_R form, Eq. (3.4)-(3.5), and Eq. (3.10)): its
    # difference to the first coding is the rounding sensitivity of the result
    Xp = ohatt.hadamard_recompress(Y, Z, seed=SKETCH_SEED, sketch_rank=opts["sketch_rank"],
                                   coding="paper")
    rec["x_fp64_notrunc_paper"] = entries(Xp, idx)
    del Xp
    rec["ranks_fp64_notrunc"] = np.array(ott.ranks(Xu))
    sv = ott.bond_singular_values(Xu)
    rec["sv_first"] = np.array([v[0] for v in sv])
    rec["norm_notrunc"] = np.array(ott.tt_norm(Xu))
    print("untruncated ranks", ott.ranks(Xu)[:4], flush=True)
    for fmt in FORMATS:
        X = ohatt.hadamard_recompress(Y, Z, seed=SKETCH_SEED, fmt=fmt, **opts)
        rec[f"x_{fmt}"] = entries(X, idx)
        rec[f"ranks_{fmt}"] = np.array(ott.ranks(X))
        rec[f"norm_{fmt}"] = np.array(ott.tt_norm(X))
        if fmt == "fp64":
            rho = ott.ranks(X)
            rec["sv_cut"] = np.array([[v[rho[k + 1] - 1], v[rho[k + 1]] if len(v) > rho[k + 1] else 0.0]
                                      for k, v in enumerate(sv)])
            rec["ell_bond"] = np.array([len(v) for v in sv])
        print(fmt, "ranks", ott.ranks(X)[:4], "norm", ott.tt_norm(X), flush=True)
    np.savez_compressed(out, **rec)
    print("wrote", out)


if __name__ == "__main__":
    main()
