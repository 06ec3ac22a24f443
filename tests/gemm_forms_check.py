"""Subprocess body of tests/test_gpu_gemm_forms.py and tests/test_gpu_qr_forms.py:
runs HaTT and TT rounding through the C ABI with the FP64 GEMM form chosen by
the environment (HATT_GEMM_FORM=pair: the paired-column kernel on every
product), or with the first-use tuner switched off (argument "model": the
model's plan only), and the Cholesky QR form chosen by the environment
(HATT_QR_FORM=steps: a launch per step), and prints one JSON line of relative
differences to the FP64 oracle and a SHA-256 of the d = 20 result."""
import hashlib
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import hatt as ohatt  # noqa: E402
from oracle import rounding as oround  # noqa: E402
from oracle import tt as ott  # noqa: E402
from paper_2410_04385_gb300 import binding as B  # noqa: E402
from paper_2410_04385_gb300 import workloads as wl  # noqa: E402


def gpu(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def host(cores):
    return [c.cpu().numpy() for c in cores]


def rel(X, A):
    return ott.tt_diff_norm(X, A) / max(ott.tt_norm(A), 1e-300)


def main():
    B.load()
    if len(sys.argv) > 1 and sys.argv[1] == "model":
        B.gemm_autotune(False)
    out = {}
    # the benchmark workload: HPCRL, QR, projection and core-update products
    Y, Z, o = wl.workload_random_d20()
    h = B.HadamardRecompressor(gpu(Y), gpu(Z), seed=9, **o)
    h.run()
    torch.cuda.synchronize()
    X = host(h.result())
    Xo, info = ohatt.hadamard_recompress(Y, Z, seed=9, return_info=True, **o)
    out["d20_rel"] = rel(X, Xo)
    out["d20_sha"] = hashlib.sha256(b"".join(np.ascontiguousarray(c).tobytes() for c in X)).hexdigest()
    out["d20_ranks_equal"] = ott.ranks(X) == info["ranks"]
    # truncation by tolerance (Gram, eigen-solve and truncation products)
    n = [6] * 6
    Yt = wl.gaussian_tt(n, [1, 4, 4, 4, 4, 4, 1], 21)
    Zt = wl.gaussian_tt(n, [1, 3, 4, 4, 3, 3, 1], 22)
    Xt = host(B.tt_hadamard_recompress(gpu(Yt), gpu(Zt), sketch_rank=16, tol=1e-4, seed=3))
    Xto, info_t = ohatt.hadamard_recompress(Yt, Zt, sketch_rank=16, tol=1e-4, seed=3,
                                            return_info=True)
    out["trunc_rel"] = rel(Xt, Xto)
    out["trunc_ranks_equal"] = ott.ranks(Xt) == info_t["ranks"]
    # TT rounding of a rank-deficient tensor
    A = ott.tt_add(wl.sin_sum_tt(6, 7, "sin"), wl.gaussian_tt([7] * 6, [1, 2, 3, 3, 3, 2, 1], 5))
    Ar = host(B.tt_round(gpu(A), 0, 1e-13))
    Ao, rk = oround.tt_round(A, 0, 1e-13)
    out["round_rel_to_input"] = rel(Ar, A)
    out["round_ranks_equal"] = ott.ranks(Ar) == rk
    # uneven pairs through the single-pair entry point (many batched shapes;
    # the n = 16 ones, whose oracle runs take seconds)
    worst = 0.0
    pairs = [q for q in wl.workload_batch_uneven(count=12, seed=11) if q[0][0].shape[1] == 16][:4]
    for Yp, Zp, op in pairs:
        Xp = host(B.tt_hadamard_recompress(gpu(Yp), gpu(Zp), seed=4, **op))
        Xpo = ohatt.hadamard_recompress(Yp, Zp, seed=4, **op)
        worst = max(worst, rel(Xp, Xpo))
    out["uneven_rel_max"] = worst
    out["device_error"] = B.device_error()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
