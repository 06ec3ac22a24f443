#!/usr/bin/env python3
"""HaTT benchmark: TT Hadamard recompressions per second on GB300.

One step = one HaTT-1 recompression (sketch generation, right-to-left HPCRL-1
sketches, left-to-right QR/projection pass and the truncation sweep) of the
d = 20, n = 32 random TT pair with all inner ranks 20 (PKP rank 400), sketch
rank 50, target rank 40, in FP64, through the libhatt C ABI. The launch
sequence of a step is captured once in a CUDA graph and replayed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hatt|reference]

Prints one JSON line (rank 0). Under torchrun every rank recompresses its own
pair (replicas, weak scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "TT Hadamard recompressions/sec at rel. error ≤1e-10, HaTT vs explicit-PKP round"
UNIT = "recompressions/s"
WORKLOAD = ("random TT pair d=20 n=32, inner ranks 20 x 20 (PKP rank 400), Gaussian cores "
            "N(0,1/(n r_k)) seeds 1,2; HaTT-1 sketch rank 50 (clamped 32 at the ends), "
            "target rank 40, tol 0, fp64")
SKETCH_SEED = 9
L2_FLUSH_BYTES = 256 << 20          # > 129 MB L2
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x FP64 FMA lanes/SM x 2 x max clock
FP64_PEAK_NOTE = ("derived: 152 SMs x 2 FP64 FMA lanes/SM/clk x 2 flop x 2070 MHz = 1.259 TFLOP/s; "
                  "a DFMA throughput loop measured 1.196 TFLOP/s on this GB300 pool")


GEMM_TIMING_STEPS = 3
CFG3_GOLDEN = os.path.join(ROOT, "tests", "golden", "cfg3_oracle_samples.npz")
AC_GOLDEN = os.path.join(ROOT, "tests", "golden", "allen_cahn_oracle_samples.npz")
GEMM_PROFILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                            "gemm_f64_kernel_d20_traffic.json")
GEMM_SOURCE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2410_04385_gb300",
                           "csrc", "k_gemm.cu")


def gemm_traffic_per_launch():
    """(DRAM bytes read + written per launch of the method GEMMs, note) from
    the committed ncu summary. The bytes are None when the kernel source has
    changed since the capture, and the note says so."""
    try:
        with open(GEMM_PROFILE) as f:
            prof = json.load(f)
        with open(GEMM_SOURCE, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError) as e:
        return None, f"no ncu record ({type(e).__name__})"
    if prof.get("source_sha256") != sha:
        return None, "stale: k_gemm.cu changed since the ncu capture; re-capture"
    return prof.get("dram_bytes_per_launch"), prof.get("note", "ncu capture")


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest per-rank value (the job's step time is its slowest rank's);
    identity on one rank. Uses the default process group (NCCL on GPUs)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms_per_step: float, world: int) -> float:
    """Whole-job recompressions per second: every rank recompresses its own
    pair per step (replicas), so N pairs per max-over-ranks step time."""
    return world * 1000.0 / ms_per_step


def sampled_entries(cores, idx):
    """Entries of a TT at the multi-indices idx (samples x d), float64."""
    import numpy as np
    M = np.ones((idx.shape[0], 1))
    for k, c in enumerate(cores):
        M = np.einsum("sa,sab->sb", M, c[:, idx[:, k], :].transpose(1, 0, 2))
    return M[:, 0]


def allen_cahn_initial(d, n, terms=4, seed=0):
    """sum_{j<terms} prod_i sin(k_ij x_i), k_ij in {1, 2, 3} (seeded), x_i =
    2 pi m / n, as a TT of ranks {1, terms, ..., terms, 1}."""
    import numpy as np
    rng = np.random.default_rng(seed)
    K = rng.integers(1, 4, size=(terms, d))
    x = 2.0 * np.pi * np.arange(n) / n
    cores = []
    for i in range(d):
        c = np.zeros((1 if i == 0 else terms, n, 1 if i == d - 1 else terms))
        for j in range(terms):
            c[0 if i == 0 else j, :, 0 if i == d - 1 else j] = np.sin(K[j, i] * x)
        cores.append(c)
    return cores


def run_allen_cahn(dev, d=8, n=64, steps=50, eps=0.1, dt=1e-3, graph_steps=1000, mixed_steps=100):
    """Example 4 on [0, 2 pi)^8, n = 64, eps = 0.1, dt = 1e-3: explicit Euler
    with u^2, u^3 by HaTT-1 (rank cap 24, tol 1e-10) and tt_round (cap 24, tol
    1e-8) each step. (1) The eager loop (data-dependent ranks, one library call
    sequence per step). (2) The fixed-rank variant (rank 24 held) with one step
    captured in a CUDA graph and replayed graph_steps times, fresh sketch seeds
    every replay; the state after 100 steps against the FP64 oracle's (4000
    stored samples), the energy every 100 steps. (3) The same graph with FP32
    sketch products for mixed_steps steps, against the same oracle state."""
    import math
    import numpy as np
    import torch
    from paper_2410_04385_gb300 import allen_cahn as ac
    from paper_2410_04385_gb300 import binding
    h = 2.0 * math.pi / n
    u = [torch.from_numpy(c).to(dev) for c in allen_cahn_initial(d, n)]
    energies = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for w in range(steps):
        u, u2 = ac.step(u, h, eps, dt, max_rank=24, tol=1e-8, hatt_tol=1e-10, seed=10 * w)
        if w % 10 == 9:
            energies.append(ac.energy(u, u2, h, eps))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = {"workload": f"u_t = eps^2 Lap u + u - u^3 on [0,2pi)^{d}, n={n}, eps={eps}, dt={dt}, "
                       f"explicit Euler, u^3 by two HaTT-1 calls, tt_round tol 1e-8",
           "eager": {"steps": steps, "ms_per_step": 1000.0 * wall / steps,
                     "max_rank": int(max(c.shape[2] for c in u)), "energy_every_10_steps": energies,
                     "energy_non_increasing": bool(all(b <= a * (1 + 1e-9)
                                                       for a, b in zip(energies, energies[1:])))}}
    gold = dict(np.load(AC_GOLDEN)) if os.path.exists(AC_GOLDEN) else None

    def sample_err(st):
        if gold is None:
            return None
        x = sampled_entries([c.cpu().numpy() for c in st.u], gold["idx"])
        return float(np.linalg.norm(x - gold["u"]) / np.linalg.norm(gold["u"]))

    def graph_run(precision, total):
        st = ac.FixedRankStepper([torch.from_numpy(c).to(dev) for c in allen_cahn_initial(d, n)], h,
                                 eps, dt, rank=24, tol=1e-8, hatt_tol=1e-10, hatt_rank=24, seed=10,
                                 precision=precision, fresh_seeds=True)
        st.capture()                                   # step 1
        genergies, ms, done, err100 = [], 0.0, 1, None
        while done < total:
            chunk = min(100 - done % 100 if done % 100 else 100, total - done)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(chunk):
                st.replay()
            b.record()
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
            done += chunk
            if done % 100 == 0:
                genergies.append(st.energy())
            if done == 100:
                err100 = sample_err(st)
        return st, {"steps": total, "ms_per_step": ms / max(total - 1, 1),
                    "energy_every_100_steps": genergies,
                    "energy_non_increasing": bool(all(y <= x * (1 + 1e-9)
                                                      for x, y in zip(genergies, genergies[1:]))),
                    "rel_error_vs_fp64_oracle_at_step_100": err100}

    st, g = graph_run(binding.TT_FP64, graph_steps)
    g.update({"timing": "CUDA events around each run of replays (energy read between them)",
              "sketch_seeds": "fresh every replay: keys seed + 2w, seed + 1 + 2w (device seed offset)",
              "oracle": "FP64 oracle's fixed-rank trajectory, 100 steps (tests/golden/"
                        "make_allen_cahn_oracle.py), relative error on 4000 sampled entries"})
    out["graph"] = g
    del st
    _, m = graph_run(binding.TT_MIXED_FP32, mixed_steps)
    m["precision"] = "FP32 sketch products (HPCRL), FP64 QR / projection / update / rounding"
    out["graph_mixed_fp32"] = m
    out["device_error"] = binding.device_error()
    return out


def run_power_iteration(workloads, dev, d=50, iters=100):
    """Example 3: largest entry of the Qing and Alpine TTs (d = 50, n = 10,
    ranks d) by 100 power iterations with HaTT-1 at sketch rank 5; wall time
    of the whole iteration (one synchronizing library call sequence per step)
    and the relative error of the last estimate against the exact maximum."""
    import numpy as np
    import torch
    from paper_2410_04385_gb300 import power_iteration as pi
    out = {"workload": f"Qing / Alpine TT, d={d}, n=10, ranks {d}, sketch rank 5, {iters} iterations"}
    for name, gfun in (("qing", workloads.qing_grid), ("alpine", workloads.alpine_grid)):
        g = gfun(d)
        Y = [torch.from_numpy(c).to(dev) for c in workloads.separable_sum_tt(g)]
        pi.largest_entry(Y, iters=2, rank=5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lams, _ = pi.largest_entry(Y, iters=iters, rank=5)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        true = float(sum(np.max(v) for v in g))    # separable sum: sum of per-coordinate maxima
        out[name] = {"s_per_run": wall, "iterations_per_s": iters / wall,
                     "rel_error_of_max": abs(float(lams[-1].item()) - true) / true}
    return out


def run_batch_cfg4(binding, workloads, dev, rank=0, world=1):
    """256 independent pairs (d in [10, 40], n in {16, 32, 64}, inner ranks in
    [8, 48], sketch rank = target rank = 2 max(r_Y, r_Z)) recompressed by ONE
    persistent launch of the task engine (FP32 sketch products, FP64 QR /
    projection / update, autotuned tiles), against the same pairs one after
    another in FP64 through the single-pair entry point on one stream. Device
    time of a whole batch each (CUDA events); the engine's results are checked
    against the sequential FP64 ones with TT inner products."""
    import torch
    from paper_2410_04385_gb300 import sharding
    pairs = workloads.workload_batch_uneven()
    out = {"workload": "256 TT pairs, d 10-40, n 16/32/64, ranks 8-48, sketch = target = 2 max(r)",
           "unit": "recompressions/s"}
    # pairs sharded over the ranks by LPT on predicted flops (no data-path collective)
    costs = [sharding.predicted_flops(Y, Z, o) for Y, Z, o in pairs]
    mine = sharding.lpt_partition(costs, world)[rank]
    mk = lambda prec, idx: [([torch.from_numpy(c).to(dev) for c in pairs[j][0]],
                             [torch.from_numpy(c).to(dev) for c in pairs[j][1]],
                             dict(pairs[j][2], precision=prec, seed=j)) for j in idx]
    gpu = mk(binding.TT_MIXED_FP32, mine)
    t0 = time.perf_counter()
    eng = binding.BatchedRecompressor(gpu, autotune=True) if gpu else None
    plan_s = time.perf_counter() - t0
    if eng is not None:
        eng.run()
    torch.cuda.synchronize()
    ms = []
    for _ in range(2):
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        if eng is not None:
            eng.run()
        s1.record()
        torch.cuda.synchronize()
        ms.append(max_over_ranks(s0.elapsed_time(s1), world, dev))
    status = eng.status() if eng is not None else 0
    prof = eng.profile() if eng is not None else {}
    records = [[j, status] + [int(v) for v in eng.Xd[q].r] for q, j in enumerate(mine)] if eng else []
    gathered = sharding.gather_records(records, world)
    out["engine"] = {"ms_per_batch": min(ms), "value": 1000.0 * len(pairs) / min(ms),
                     "launches_per_batch_per_gpu": 1, "status": status, "plan_and_autotune_s": plan_s,
                     "workspace_gb_rank0": (eng.workspace_bytes / 1e9) if eng else 0.0,
                     **(eng.info() if eng else {}),
                     "precision": "FP32 sketch products, FP64 QR / projection / update",
                     "sharding": f"LPT on predicted flops over {world} rank(s); pairs on rank 0: {len(mine)}",
                     "pairs_gathered": len(gathered),
                     "cta_time_fractions_rank0": prof,
                     "all_status_ok": all(rec[1] == 0 for rec in gathered)}
    if world > 1:
        out["scaling"] = "strong"
        del eng
        torch.cuda.empty_cache()
        return out
    res = [[c.clone() for c in eng.result(q)] for q in range(len(gpu))]
    del eng, gpu
    torch.cuda.empty_cache()
    seq_in = mk(binding.TT_FP64, range(len(pairs)))
    seq = binding.BatchRecompressor(seq_in, lanes=1)
    seq.run()                          # first calls: the library times its GEMM tilings
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    seq.run()
    s1.record()
    torch.cuda.synchronize()
    seq_ms = s0.elapsed_time(s1)
    out["sequential_fp64"] = {"ms_per_batch": seq_ms, "value": 1000.0 * len(pairs) / seq_ms,
                              "impl": "256 single-pair FP64 calls one after another on one stream"}
    worst = 0.0
    for j in range(len(pairs)):
        a, b = res[j], seq.result(j)
        aa = binding.tt_dot(a, a).item()
        bb = binding.tt_dot(b, b).item()
        ab = binding.tt_dot(a, b).item()
        worst = max(worst, (max(aa - 2 * ab + bb, 0.0) ** 0.5) / bb ** 0.5)
    out["max_rel_diff_engine_fp32_vs_sequential_fp64"] = worst
    out["speedup_engine_vs_sequential_fp64"] = seq_ms / min(ms)
    from paper_2410_04385_gb300 import costmodel
    sw = 0.0
    for Y, Z, o in pairs:
        n, r, s_, ell = sharding.pair_ranks(Y, Z, o)
        sw += costmodel.hatt1_flops(n, r, s_, ell)[1]
    ach = sw / (min(ms) * 1e-3) / 1e12
    out["engine_roofline"] = {"bound": "alu", "fp64_flops": sw, "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                              "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                              "note": "FP64 left-to-right pass (Section 4 model) over the batch time; the "
                                      "FP32 sketch products (HPCRL) run inside the same time"}
    out["device_error"] = binding.device_error()
    del seq, res
    torch.cuda.empty_cache()
    return out


def run_mixed_cfg3(binding, workloads, dev, samples=2000, steps=2):
    """Smooth TT pair d=50, n=64, ranks 40 (sketch 90, target 80, tol 1e-8) in
    every precision: device time per recompression (graph replay, CUDA events)
    and the relative error on sampled entries against the exact product."""
    import numpy as np
    import torch
    Y, Z, opts = workloads.workload_smooth_d50()
    idx = np.random.default_rng(0).integers(0, 64, size=(samples, len(Y)))
    exact = sampled_entries(Y, idx) * sampled_entries(Z, idx)
    Yg = [torch.from_numpy(c).to(dev) for c in Y]
    Zg = [torch.from_numpy(c).to(dev) for c in Z]
    out = {"workload": "smooth TT pair d=50, n=64, ranks 40, sketch 90, max rank 80, tol 1e-8",
           "error": f"relative, on {samples} sampled entries, against Y*Z", "per_precision": {}}
    gold = None
    if os.path.exists(CFG3_GOLDEN):
        gold = dict(np.load(CFG3_GOLDEN))
        out["oracle_comparison"] = ("relative difference on the 4000 entries stored by "
                                    "tests/golden/make_cfg3_oracle.py (FP64 oracle, same sketch seed; "
                                    "and the oracle emulating the sketch format); c7_bound = "
                                    "10 max(oracle FP64 error, emulated error, tol) against Y*Z")
    for prec, name in ((0, "fp64"), (1, "fp32"), (2, "tf32"), (3, "bf16")):
        h = binding.HadamardRecompressor(Yg, Zg, seed=SKETCH_SEED, precision=prec, **opts)
        h.run()
        h.capture()
        h.replay()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            h.replay()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        X = [c.cpu().numpy() for c in h.result()]
        x = sampled_entries(X, idx)
        err = float(np.sqrt(np.sum((x - exact) ** 2) / np.sum(exact ** 2)))
        out["per_precision"][name] = {"ms_per_recompression": min(ms), "rel_error_sampled": err,
                                      "max_rank": int(max(h.Xd.r))}
        if gold is not None:
            xg = sampled_entries(X, gold["idx"])
            ex = gold["exact"]
            rd = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
            e_emul = rd(gold[f"x_{name}"], ex)
            out["per_precision"][name].update({
                "rel_diff_vs_fp64_oracle": rd(xg, gold["x_fp64"]),
                "rel_diff_vs_emulated_oracle": rd(xg, gold[f"x_{name}"]),
                "rel_error_vs_exact_oracle_samples": rd(xg, ex),
                "oracle_fp64_error_vs_exact": rd(gold["x_fp64"], ex),
                "oracle_emulated_error_vs_exact": e_emul,
                "c7_bound": 10.0 * max(rd(gold["x_fp64"], ex), e_emul, 1e-8)})
        del h
    out["device_error"] = binding.device_error()
    return out


def run_hatt2_example1b(binding, workloads, dev, samples=20000, reps=5):
    """Example 1b: y = sum_{j<=60} a_j sin(j t), z = sum_j b_j cos(j t), a, b ~
    U[0.1, 10.1] (seeded), t on 20^7 points folded to a d = 7, n = 20 TT and
    rounded to 1e-14 (tt_round); HaTT-1 against HaTT-2 at l = 20 over the
    paper's ep values, and over l = 10..60 at ep = 1e-3. Wall time per call,
    eager and as a CUDA-graph replay (both variants keep their ranks on the
    device), and the relative error on sampled entries against the closed
    form y(t) z(t)."""
    import numpy as np
    import torch
    d, n, J = 7, 20, 60
    rng = np.random.default_rng(11)
    a, b = rng.uniform(0.1, 10.1, J), rng.uniform(0.1, 10.1, J)
    Yr = binding.tt_round([torch.from_numpy(c).to(dev) for c in workloads.fourier_series_tt(d, n, a, "sin")],
                          tol=1e-14)
    Zr = binding.tt_round([torch.from_numpy(c).to(dev) for c in workloads.fourier_series_tt(d, n, b, "cos")],
                          tol=1e-14)
    idx = rng.integers(0, n, size=(samples, d))
    t = 2.0 * np.pi * (1.0 + (idx * (float(n) ** np.arange(d))).sum(axis=1)) / float(n) ** d
    j = np.arange(1, J + 1)
    exact = (np.sin(np.outer(t, j)) @ a) * (np.cos(np.outer(t, j)) @ b)

    def one(ell, variant, ep):
        h = binding.HadamardRecompressor(Yr, Zr, sketch_rank=ell, seed=SKETCH_SEED, variant=variant,
                                         ep=ep)
        h.run()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            h.run()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        x = sampled_entries([c.cpu().numpy() for c in h.result()], idx)
        err = float(np.sqrt(np.sum((x - exact) ** 2) / np.sum(exact ** 2)))
        h.capture()
        h.replay()
        torch.cuda.synchronize()
        tg = []
        for _ in range(reps):
            t0 = time.perf_counter()
            h.replay()
            torch.cuda.synchronize()
            tg.append(time.perf_counter() - t0)
        xg = sampled_entries([c.cpu().numpy() for c in h.result()], idx)
        return {"variant": variant, "ep": ep if variant == 2 else None, "ell": ell,
                "ms_per_call": 1000.0 * float(np.median(ts)),
                "ms_per_graph_replay": 1000.0 * float(np.median(tg)), "rel_error_sampled": err,
                "graph_equals_eager": bool(np.array_equal(x, xg))}

    rows = [one(20, 1, 0.0)] + [one(20, 2, ep) for ep in (0.95, 1e-1, 4e-2, 1e-3, 1e-5, 1e-10, 1e-14)]
    sweep = [one(ell, v, 1e-3) for ell in (10, 20, 30, 40, 50, 60) for v in (1, 2)]
    return {"workload": "Fourier-series product (Example 1b): d=7, n=20, 60 terms each, inputs "
                        "rounded to 1e-14, no output truncation",
            "input_ranks": [[int(c.shape[0]) for c in Yr] + [1], [int(c.shape[0]) for c in Zr] + [1]],
            "error": f"relative, on {samples} sampled entries, against the closed form y(t) z(t)",
            "ep_sweep_l20": rows, "ell_sweep_ep1e-3": sweep}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["hatt", "reference"], default="hatt")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-pkp", action="store_true")
    p.add_argument("--no-power", action="store_true", help="skip the power iteration run")
    p.add_argument("--no-allen-cahn", action="store_true", help="skip the Allen-Cahn run")
    p.add_argument("--no-hatt2", action="store_true", help="skip the HaTT-1 / HaTT-2 comparison")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the 256-pair batched run (about a minute)")
    p.add_argument("--no-mixed", action="store_true",
                   help="skip the per-precision run of the smooth d=50 workload")
    p.add_argument("--cpu-leg", default=None, help=argparse.SUPPRESS)
    p.add_argument("--gpu-result", default=None, help=argparse.SUPPRESS)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    return p.parse_args()


# ------------------------------------------------------------ CPU oracle leg ---

def cpu_leg(out_path: str, seconds: float, gpu_result: str | None):
    """Runs in a fresh process: times the FP64 oracle on this host's cores on a
    bounded sample (whole recompressions of the bench workload) and, if given
    the GPU result, computes its relative difference to the oracle's result
    for the same sketch (the error gate of the metric)."""
    import numpy as np

    from oracle import hatt as ohatt
    from oracle import tt as ott
    from paper_2410_04385_gb300 import workloads

    Y, Z, opts = workloads.workload_random_d20()
    times = []
    Xo = None
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        Xo = ohatt.hadamard_recompress(Y, Z, seed=SKETCH_SEED, **opts)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all >= seconds and len(times) >= 3:
            break
    res = {"seconds_per_recompression": statistics.median(times), "runs": len(times),
           "wall_s": time.perf_counter() - t_all}
    if gpu_result:
        data = np.load(gpu_result)
        Xg = [data[f"c{k}"] for k in range(len(Xo))]
        res["rel_diff_vs_oracle"] = ott.tt_diff_norm(Xg, Xo) / ott.tt_norm(Xo)
        res["ranks_match"] = ott.ranks(Xg) == ott.ranks(Xo)
    with open(out_path, "w") as f:
        json.dump(res, f)


def run_cpu_leg(seconds: float, gpu_result: str | None):
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(cores)
    with tempfile.TemporaryDirectory() as td:
        out = os.path.join(td, "cpu.json")
        cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", out,
               "--cpu-seconds", str(seconds)]
        if gpu_result:
            cmd += ["--gpu-result", gpu_result]
        subprocess.run(cmd, check=True, env=env, cwd=ROOT)
        with open(out) as f:
            res = json.load(f)
    res["cores"] = cores
    return res


# ------------------------------------------------------------------ clocks ---

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------- PKP comparator ---

def pkp_round_gpu(Yg, Zg, max_rank):
    """Explicit-PKP TT-Rounding on the GPU (comparator only): PKP cores of rank
    r*s, then Algorithm 1 with cuSOLVER QR/SVD through torch.linalg in FP64."""
    import torch
    A = [torch.einsum("aib,cid->acibd", y, z).reshape(y.shape[0] * z.shape[0], y.shape[1],
                                                       y.shape[2] * z.shape[2])
         for y, z in zip(Yg, Zg)]
    d = len(A)
    B = [a.clone() for a in A]
    for k in range(d - 1, 0, -1):
        a, n, b = B[k].shape
        q, r = torch.linalg.qr(B[k].reshape(a, n * b).T)
        B[k] = q.T.reshape(q.shape[1], n, b)
        B[k - 1] = torch.einsum("aib,cb->aic", B[k - 1], r)
    for k in range(d - 1):
        a, n, b = B[k].shape
        q, r = torch.linalg.qr(B[k].reshape(a * n, b))
        u, s, vt = torch.linalg.svd(r, full_matrices=False)
        rho = min(max_rank, s.numel())
        B[k] = (q @ u[:, :rho]).reshape(a, n, rho)
        B[k + 1] = torch.einsum("ab,bic->aic", s[:rho, None] * vt[:rho], B[k + 1])
    return B


# ------------------------------------------------------------- reference ---

def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle timed on the host cores, each
    step one whole recompression of the same workload."""
    if rank != 0:
        return
    from oracle import hatt as ohatt
    from paper_2410_04385_gb300 import workloads
    Y, Z, opts = workloads.workload_random_d20()
    for _ in range(args.warmup):
        ohatt.hadamard_recompress(Y, Z, seed=SKETCH_SEED, **opts)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ohatt.hadamard_recompress(Y, Z, seed=SKETCH_SEED, **opts)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    cores = os.cpu_count() or 1
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "n/a (host CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} whole recompressions of the workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- main ---

def main():
    args = parse()
    if args.cpu_leg:
        cpu_leg(args.cpu_leg, args.cpu_seconds, args.gpu_result)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2410_04385_gb300 import binding, costmodel, workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    binding.load()

    Y, Z, opts = workloads.workload_random_d20()
    Yg = [torch.from_numpy(c).to(dev) for c in Y]
    Zg = [torch.from_numpy(c).to(dev) for c in Z]
    h = binding.HadamardRecompressor(Yg, Zg, seed=SKETCH_SEED, **opts)

    # a first call (the library times its GEMM tilings for shapes it has not
    # run yet), then the launches and wall time of one eager call, then the
    # same sequence captured in a graph
    h.run()
    torch.cuda.synchronize()
    c0 = binding.launch_count()
    t0 = time.perf_counter()
    h.run()
    torch.cuda.synchronize()
    eager_ms = 1000.0 * (time.perf_counter() - t0)
    launches_per_step = binding.launch_count() - c0
    h.capture()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        h.replay()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                       # L2 flush between steps, outside the events
        starts[i].record(stream)
        h.replay()
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = max_over_ranks(statistics.mean(step_ms), world, dev)
    value = job_throughput(ms, world)

    # ---- end to end through the C ABI with host buffers (pinned) ----
    Yh = [c.cpu().pin_memory() for c in Yg]
    Zh = [c.cpu().pin_memory() for c in Zg]
    res = h.result()
    ranks = h.Xd.r
    outs_h = [torch.empty(c.numel(), dtype=torch.float64).pin_memory() for c in res]
    h2d = sum(c.numel() * 8 for c in Yh + Zh)
    d2h = sum(c.numel() * 8 for c in outs_h) + 8 * len(ranks)
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(-2, args.steps):
        flush.zero_()
        if i >= 0:
            e_s[i].record(stream)
        for dst, src in zip(Yg + Zg, Yh + Zh):
            dst.copy_(src, non_blocking=True)
        h.replay()
        for dst, buf, c in zip(outs_h, h.out_bufs, res):
            dst.copy_(buf[: c.numel()], non_blocking=True)
        if i >= 0:
            e_e[i].record(stream)
    torch.cuda.synchronize()
    e2e_ms = statistics.mean(s.elapsed_time(e) for s, e in zip(e_s, e_e))

    # ---- dominant kernel: the FP64 GEMM, timed live with CUDA events ----
    # Eager steps under the library's kernel timer, each queued behind a
    # bounded GPU sleep so that the host has enqueued the whole step before
    # the GPU reaches it and no event pair brackets a host launch gap.
    cap = 8192
    sleep_cycles = int(2.1e9 * min(0.25, max(0.05, 3e-3 * eager_ms)))
    t_s = [torch.cuda.Event(enable_timing=True) for _ in range(GEMM_TIMING_STEPS)]
    t_e = [torch.cuda.Event(enable_timing=True) for _ in range(GEMM_TIMING_STEPS)]
    binding.kernel_timer_start(cap)
    for i in range(GEMM_TIMING_STEPS):
        torch.cuda._sleep(sleep_cycles)
        t_s[i].record(stream)
        h.run()
        t_e[i].record(stream)
    torch.cuda.synchronize()
    g_ms, g_fl, g_rec, g_role = binding.kernel_timer_stop(cap, with_roles=True)
    timed_steps_ms = sum(a.elapsed_time(b) for a, b in zip(t_s, t_e))
    gemm_ms = sum(g_ms)
    # the dominant kernel's roofline counts only the launches that compute the
    # HaTT contractions (always real work); the truncation products (Gram
    # matrices, projections; refinement products for c > 96, which a device
    # flag can turn into no-ops) are reported apart
    m_idx = [i for i, ro in enumerate(g_role) if ro == binding.TT_ROLE_METHOD]
    a_idx = [i for i, ro in enumerate(g_role) if ro != binding.TT_ROLE_METHOD]
    meth_ms = sum(g_ms[i] for i in m_idx)
    meth_flops = sum(g_fl[i] for i in m_idx)
    aux_ms = sum(g_ms[i] for i in a_idx)
    meth_tflops = meth_flops / (meth_ms * 1e-3) / 1e12
    traffic, traffic_note = gemm_traffic_per_launch()

    # ---- roofline of the whole step (one graph launch = one recompression) ----
    n = workloads.modes_of(Y)
    r = workloads.ranks_of(Y)
    s = workloads.ranks_of(Z)
    ell = [int(v) for v in h.bound]
    hp, sw = costmodel.hatt1_flops(n, r, s, ell)
    alg_flops = hp + sw
    contr_flops = costmodel.hatt1_contraction_flops(n, r, s, ell)
    achieved_tflops = alg_flops / (ms * 1e-3) / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "ranks_out": ranks,
                   "l2": "flushed between timed steps (256 MiB write, outside the events)",
                   "launch": "one CUDA graph replay per step", "parallelism": f"replicas x{world}"},
        "gpu_launches": launches_per_step * args.steps,
        "launches_per_step": launches_per_step,
        "eager_ms_per_step": eager_ms,
        "wall_s_timed_region": wall,
        "e2e": {"value": world * 1000.0 / e2e_ms, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu",
                     "kernel": "gemm_f64_kernel, launches computing the HaTT contractions (HPCRL S1-S3, "
                               "C_k W, Q^T C_k, the two core-update stages)",
                     "achieved": meth_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": meth_tflops / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "traffic_note": traffic_note,
                     "launches_timed": len(m_idx),
                     "avg_launch_us": 1e3 * meth_ms / max(len(m_idx), 1),
                     "algorithmic_flops_per_launch": meth_flops / max(len(m_idx), 1),
                     "algorithmic_flops_per_step": meth_flops / GEMM_TIMING_STEPS,
                     "section4_contraction_flops_per_step": contr_flops,
                     "share_of_step": meth_ms / timed_steps_ms,
                     "timing": "CUDA events around every launch on its own stream (library kernel "
                               "timer), eager steps queued behind a GPU sleep",
                     "peak_source": FP64_PEAK_NOTE},
        "gemm_aux": {"kernel": "gemm_f64_kernel, all other launches (truncation Gram matrices and "
                               "projections; the Cholesky QR computes its Gram matrix in its own "
                               "kernel)",
                     "launches_per_step": len(a_idx) / GEMM_TIMING_STEPS,
                     "share_of_step": aux_ms / timed_steps_ms,
                     "all_gemm_share_of_step": gemm_ms / timed_steps_ms},
        "roofline_step": {"bound": "alu", "kernel": "HaTT-1 step (graph of all libhatt kernels)",
                          "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": achieved_tflops / FP64_PEAK_TFLOPS,
                          "algorithmic_flops_per_step": alg_flops},
        "clocks": clocks,
    }

    # ---- explicit-PKP rounding on the same GPU (comparator) ----
    if not args.no_pkp and rank == 0:
        B = pkp_round_gpu(Yg, Zg, opts["max_rank"])
        torch.cuda.synchronize()
        reps = []
        for _ in range(2):
            t0 = time.perf_counter()
            B = pkp_round_gpu(Yg, Zg, opts["max_rank"])
            torch.cuda.synchronize()
            reps.append(time.perf_counter() - t0)
        pkp_s = min(reps)
        line["pkp_round"] = {"value": 1.0 / pkp_s, "unit": UNIT, "ms_per_recompression": 1e3 * pkp_s,
                             "impl": "explicit PKP cores (rank 400) + TT-Rounding (Algorithm 1) "
                                     "with torch.linalg (cuSOLVER) FP64 QR/SVD on the same GPU"}
        line["speedup_vs_pkp_round"] = (1000.0 / ms) * pkp_s
        del B

    # ---- mixed-precision sketches on the smooth d=50 workload ----
    if not args.no_mixed and rank == 0:
        line["mixed_cfg3"] = run_mixed_cfg3(binding, workloads, dev)

    # ---- many uneven pairs: batched over library streams vs one after another ----
    if not args.no_batch:
        b4 = run_batch_cfg4(binding, workloads, dev, rank, world)
        if rank == 0:
            line["batch_cfg4"] = b4

    # ---- power iteration for the largest entry (Example 3) ----
    if not args.no_power and rank == 0:
        line["power_iteration"] = run_power_iteration(workloads, dev)

    # ---- HaTT-1 against HaTT-2 on the Fourier-series product (Example 1b) ----
    if not args.no_hatt2 and rank == 0:
        line["hatt2_example1b"] = run_hatt2_example1b(binding, workloads, dev)

    # ---- Allen-Cahn time stepping (Example 4) ----
    if not args.no_allen_cahn and rank == 0:
        line["allen_cahn"] = run_allen_cahn(dev)

    # ---- CPU oracle baseline and the error gate ----
    if not args.no_cpu_baseline and rank == 0:
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "gpu_result.npz")
            np.savez(path, **{f"c{k}": c.cpu().numpy() for k, c in enumerate(res)})
            cpu = run_cpu_leg(args.cpu_seconds, path)
        line["cpu_baseline"] = {"value": 1.0 / cpu["seconds_per_recompression"], "unit": UNIT,
                                "cores": cpu["cores"], "kind": "oracle",
                                "sample": f"{cpu['runs']} whole recompressions of the workload "
                                          f"(numpy float64, {cpu['wall_s']:.1f} s)"}
        line["rel_error_vs_oracle"] = cpu["rel_diff_vs_oracle"]
        line["error_gate_1e-10"] = bool(cpu["rel_diff_vs_oracle"] <= 1e-10 and cpu["ranks_match"])

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
