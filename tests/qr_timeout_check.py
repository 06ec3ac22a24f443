"""Subprocess body of tests/test_gpu_qr_forms.py: with HATT_QR_SPIN_CAP=1 every
grid-barrier wait of the fused Cholesky QR gives up after one poll. Runs one
recompression (its QRs stop early and raise the timeout bit), reads the device
status, then runs a stream-lane batch (whose QRs are launched per step, with
no grid barrier) and compares it with the oracle: the context stays usable.
Prints one JSON line."""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import hatt as ohatt  # noqa: E402
from oracle import tt as ott  # noqa: E402
from paper_2410_04385_gb300 import binding as B  # noqa: E402
from paper_2410_04385_gb300 import workloads as wl  # noqa: E402


def gpu(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def main():
    B.load()
    out = {}
    n = [8] * 6
    Y = wl.gaussian_tt(n, [1, 5, 6, 6, 6, 4, 1], 31)
    Z = wl.gaussian_tt(n, [1, 4, 4, 5, 4, 3, 1], 32)
    B.device_status()                                 # clear
    h = B.HadamardRecompressor(gpu(Y), gpu(Z), sketch_rank=20, seed=2)
    h.run()
    torch.cuda.synchronize()
    out["status_after_fused"] = B.device_status()
    batch = B.BatchRecompressor([(gpu(Y), gpu(Z), dict(sketch_rank=20, seed=2))], lanes=2)
    batch.run()
    torch.cuda.synchronize()
    X = [c.cpu().numpy() for c in batch.result(0)]
    A = ohatt.hadamard_recompress(Y, Z, sketch_rank=20, seed=2)
    out["batch_rel"] = ott.tt_diff_norm(X, A) / ott.tt_norm(A)
    out["status_after_batch"] = B.device_status()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
