"""Host-side tests of the C ABI: the library loads, exports every symbol that
include/hatt.h declares, and its planning / argument checks (host code only,
no kernel launches) agree with the oracle's rank plan."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import hatt as ohatt
from paper_2410_04385_gb300 import binding as B
from paper_2410_04385_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        libbuild.build()
    return B.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hatt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tt_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_path_entry_points():
    names = declared_functions()
    for want in ("tt_hadamard_recompress", "tt_round", "tt_dot", "tt_norm"):
        assert want in names
    assert len(names) >= 10


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    nm_names = set(B.EXPORTS)
    assert set(declared_functions()) <= nm_names


def test_status_strings(lib):
    for st in range(0, 9):
        assert len(B.status_string(st)) > 0
    assert B.status_string(99) == "unknown status"


def _plan(Yr, Zr, n, **opts):
    Yd = B.TT(n=n, r=Yr)
    Zd = B.TT(n=n, r=Zr)
    o = B.make_opts(**opts)
    d = len(n)
    bound = (ctypes.c_int64 * (d + 1))()
    ws = ctypes.c_size_t()
    st = B.load().tt_hadamard_recompress_plan(Yd.ref(), Zd.ref(), ctypes.byref(o), bound,
                                              ctypes.byref(ws))
    return st, [int(v) for v in bound], int(ws.value)


def test_plan_matches_oracle_small_workload(lib):
    n = [8] * 6
    st, bound, ws = _plan([1, 2, 2, 2, 2, 2, 1], [1, 5, 5, 5, 5, 5, 1], n, max_rank=10, tol=1e-12,
                          sketch_rank=12)
    assert st == 0
    assert bound == [1, 8, 10, 10, 10, 8, 1]
    assert ws > 0


@pytest.mark.parametrize("seed", range(8))
def test_plan_matches_oracle_random(lib, seed):
    rng = np.random.default_rng(seed)
    d = int(rng.integers(1, 8))
    n = [int(v) for v in rng.integers(1, 9, size=d)]
    r = [1] + [int(v) for v in rng.integers(1, 9, size=d - 1)] + [1]
    s = [1] + [int(v) for v in rng.integers(1, 9, size=d - 1)] + [1]
    mr = int(rng.integers(0, 20))
    sk = int(rng.integers(0, 40))
    st, bound, ws = _plan(r, s, n, max_rank=mr, sketch_rank=sk, oversample=5)
    assert st == 0
    lreq = ohatt.requested_sketch_rank(r, s, mr, sk, 5)
    assert bound == ohatt.plan_ranks(n, r, s, lreq)


@pytest.mark.parametrize("d,n,r,lreq", [(20, 32, 20, 50), (50, 64, 40, 90), (300, 2, 3, 9)])
def test_plan_long_chains_saturate_mode_products(lib, d, n, r, lreq):
    rk = [1] + [r] * (d - 1) + [1]
    st, bound, ws = _plan(rk, rk, [n] * d, sketch_rank=lreq)
    assert st == 0
    assert bound == ohatt.plan_ranks([n] * d, rk, rk, lreq)
    assert min(bound) >= 1


def test_plan_workspace_grows_with_size(lib):
    small = _plan([1] + [4] * 5 + [1], [1] + [4] * 5 + [1], [8] * 6, sketch_rank=8)[2]
    big = _plan([1] + [20] * 19 + [1], [1] + [20] * 19 + [1], [32] * 20, max_rank=40,
                sketch_rank=50)[2]
    assert big > small > 0


@pytest.mark.parametrize("case,expect", [
    ("order_mismatch", 1), ("mode_mismatch", 1), ("boundary_rank", 1), ("zero_mode", 1),
    ("negative_opt", 3), ("bad_precision", 3), ("bad_variant", 3), ("rank_too_big", 2),
    ("negative_ep", 3), ("ep_one", 3), ("ep_nan", 3),
])
def test_plan_rejects_bad_arguments(lib, case, expect):
    n = [4, 4, 4]
    Yr, Zr = [1, 3, 3, 1], [1, 2, 2, 1]
    opts = dict(sketch_rank=4)
    if case == "order_mismatch":
        Yd, Zd = B.TT(n=n, r=Yr), B.TT(n=[4, 4], r=[1, 2, 1])
    elif case == "mode_mismatch":
        Yd, Zd = B.TT(n=n, r=Yr), B.TT(n=[4, 5, 4], r=Zr)
    elif case == "boundary_rank":
        Yd, Zd = B.TT(n=n, r=[2, 3, 3, 1]), B.TT(n=n, r=Zr)
    elif case == "zero_mode":
        Yd, Zd = B.TT(n=[4, 0, 4], r=Yr), B.TT(n=[4, 0, 4], r=Zr)
    elif case == "rank_too_big":
        Yd = B.TT(n=[64] * 4, r=[1, 64, 64, 64, 1])
        Zd = B.TT(n=[64] * 4, r=[1, 64, 64, 64, 1])
        opts = dict(sketch_rank=200)
    else:
        Yd, Zd = B.TT(n=n, r=Yr), B.TT(n=n, r=Zr)
        if case == "negative_opt":
            opts = dict(max_rank=-1)
        elif case == "bad_precision":
            opts = dict(precision=7)
        elif case == "bad_variant":
            opts = dict(variant=5)
        elif case == "negative_ep":
            opts = dict(variant=2, ep=-1e-3)
        elif case == "ep_one":
            opts = dict(variant=2, ep=1.0)
        elif case == "ep_nan":
            opts = dict(variant=2, ep=float("nan"))
    o = B.make_opts(**opts)
    bound = (ctypes.c_int64 * 8)()
    ws = ctypes.c_size_t()
    st = B.load().tt_hadamard_recompress_plan(Yd.ref(), Zd.ref(), ctypes.byref(o), bound,
                                              ctypes.byref(ws))
    assert st == expect


def test_execute_rejects_small_workspace_before_launching(lib):
    # fake, never-dereferenced device addresses: the size check precedes any launch
    n = [4, 4, 4]
    Yd = B.TT(n=n, r=[1, 3, 3, 1])
    Zd = B.TT(n=n, r=[1, 2, 2, 1])
    Xd = B.TT(n=n, r=[1, 4, 4, 1])
    base = 1 << 40
    Yd.set_core_ptrs([base + k * (1 << 20) for k in range(3)])
    Zd.set_core_ptrs([base + (3 + k) * (1 << 20) for k in range(3)])
    Xd.set_core_ptrs([base + (6 + k) * (1 << 20) for k in range(3)])
    o = B.make_opts(sketch_rank=4)
    st = B.load().tt_hadamard_recompress(Yd.ref(), Zd.ref(), ctypes.byref(o), Xd.ref(),
                                         ctypes.c_void_p(base + (1 << 30)), 16, None)
    assert st == 4
    # misaligned workspace
    st = B.load().tt_hadamard_recompress(Yd.ref(), Zd.ref(), ctypes.byref(o), Xd.ref(),
                                         ctypes.c_void_p(base + (1 << 30) + 8), 1 << 30, None)
    assert st == 4
    # output aliasing an input core
    Xd.set_core_ptrs([base, base + (7 << 20), base + (8 << 20)])
    st = B.load().tt_hadamard_recompress(Yd.ref(), Zd.ref(), ctypes.byref(o), Xd.ref(),
                                         ctypes.c_void_p(base + (1 << 30)), 1 << 30, None)
    assert st == 1


def test_round_and_dot_plans(lib):
    n = [5, 6, 7]
    Ad = B.TT(n=n, r=[1, 4, 9, 1])
    bound = (ctypes.c_int64 * 4)()
    ws = ctypes.c_size_t()
    assert B.load().tt_round_plan(Ad.ref(), 0, 1e-8, bound, ctypes.byref(ws)) == 0
    assert [int(v) for v in bound] == [1, 4, 9, 1]
    assert ws.value > 0
    Bd = B.TT(n=n, r=[1, 2, 3, 1])
    assert B.load().tt_dot_plan(Ad.ref(), Bd.ref(), ctypes.byref(ws)) == 0
    Cd = B.TT(n=[5, 6, 8], r=[1, 2, 3, 1])
    assert B.load().tt_dot_plan(Ad.ref(), Cd.ref(), ctypes.byref(ws)) == 1


def test_kernel_timer_argument_checks(lib):
    """The timer's argument and state checks answer before any CUDA call
    (status 3 = TT_ERR_ARG)."""
    assert lib.tt_kernel_timer_start(0) == 3
    assert lib.tt_kernel_timer_start(-5) == 3
    assert lib.tt_kernel_timer_start((1 << 20) + 1) == 3
    ms = (ctypes.c_double * 4)()
    fl = (ctypes.c_double * 4)()
    cnt = ctypes.c_int64(-1)
    # no timer running
    assert lib.tt_kernel_timer_stop(ms, fl, 4, ctypes.byref(cnt)) == 3
    assert lib.tt_kernel_timer_stop(None, None, 4, None) == 3
    assert lib.tt_kernel_timer_stop(ms, fl, -1, None) == 3


def test_binding_entry_points_accept_every_option():
    """The Python wrappers pass every tt_opts field through (marshalling only)."""
    import inspect
    fields = {name for name, _ in B.OptsStruct._fields_}
    assert fields <= set(inspect.signature(B.make_opts).parameters)
    assert fields <= set(inspect.signature(B.tt_hadamard_recompress).parameters)
    assert (B.TT_FP64, B.TT_MIXED_FP32, B.TT_MIXED_TF32, B.TT_MIXED_BF16) == (0, 1, 2, 3)
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "hatt.h")).read()
    for name, v in (("TT_FP64", 0), ("TT_MIXED_FP32", 1), ("TT_MIXED_TF32", 2), ("TT_MIXED_BF16", 3)):
        assert re.search(rf"{name}\s*=\s*{v}\b", hdr)


def test_batch_plan_sums_per_lane_maxima(lib):
    """Host-only: the batch workspace is one region per lane, each the largest
    single-pair workspace of the pairs on that lane (pair j on lane j % lanes)."""
    pairs = []
    for j, (n, r) in enumerate([(8, 3), (16, 5), (4, 2), (8, 6), (32, 4)]):
        Y = B.TT(n=[n] * 4, r=[1, r, r, r, 1])
        Z = B.TT(n=[n] * 4, r=[1, r + 1, r + 1, r + 1, 1])
        pairs.append((Y, Z, B.make_opts(sketch_rank=2 * r)))
    single = []
    for Y, Z, o in pairs:
        bound = (ctypes.c_int64 * 5)()
        ws = ctypes.c_size_t()
        assert lib.tt_hadamard_recompress_plan(Y.ref(), Z.ref(), ctypes.byref(o), bound, ctypes.byref(ws)) == 0
        single.append((ws.value + 255) // 256 * 256)
    Ya = (B.TTStruct * 5)(*[p[0].s for p in pairs])
    Za = (B.TTStruct * 5)(*[p[1].s for p in pairs])
    Oa = (B.OptsStruct * 5)(*[p[2] for p in pairs])
    for lanes in (1, 2, 3, 5, 8):
        ws = ctypes.c_size_t()
        assert lib.tt_hadamard_recompress_batch_plan(5, Ya, Za, Oa, lanes, ctypes.byref(ws)) == 0
        expect = sum(max([single[j] for j in range(5) if j % lanes == l] or [0]) for l in range(lanes))
        assert ws.value == expect + 256
    ws = ctypes.c_size_t()
    assert lib.tt_hadamard_recompress_batch_plan(5, Ya, Za, Oa, 0, ctypes.byref(ws)) == 3
    assert lib.tt_hadamard_recompress_batch_plan(5, Ya, Za, Oa, 33, ctypes.byref(ws)) == 3
    assert lib.tt_hadamard_recompress_batch_plan(0, None, None, None, 4, ctypes.byref(ws)) == 0
    assert ws.value == 256
    bad = (B.OptsStruct * 5)(*[p[2] for p in pairs])
    bad[3].precision = 9
    assert lib.tt_hadamard_recompress_batch_plan(5, Ya, Za, bad, 2, ctypes.byref(ws)) == 3


def test_precision_range_is_checked_on_the_host(lib):
    """tt_opts.precision: 0..4 plan, anything else is TT_ERR_ARG (status 3)."""
    Y = B.TT(n=[4, 4, 4], r=[1, 2, 2, 1])
    Z = B.TT(n=[4, 4, 4], r=[1, 2, 2, 1])
    bound = (ctypes.c_int64 * 4)()
    ws = ctypes.c_size_t()
    for prec, expect in [(-1, 3), (0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (5, 3)]:
        o = B.make_opts(sketch_rank=4, precision=prec)
        assert lib.tt_hadamard_recompress_plan(Y.ref(), Z.ref(), ctypes.byref(o), bound, ctypes.byref(ws)) == expect


def test_hatt2_plan_and_batch_plan(lib):
    """HaTT-2 plans the same output bound as HaTT-1 and a workspace that also
    holds its own buffers; the batched entry point takes it (the kept ranks
    stay on the device), with a lane at least as large as the single plan."""
    n = [6] * 5
    Yr, Zr = [1, 4, 5, 5, 3, 1], [1, 3, 4, 2, 3, 1]
    st1, b1, w1 = _plan(Yr, Zr, n, sketch_rank=9)
    st2, b2, w2 = _plan(Yr, Zr, n, sketch_rank=9, variant=2, ep=1e-3)
    assert st1 == st2 == 0 and b1 == b2 and w2 > w1
    Yd, Zd = B.TT(n=n, r=Yr), B.TT(n=n, r=Zr)
    Ys = (B.TTStruct * 1)(Yd.s)
    Zs = (B.TTStruct * 1)(Zd.s)
    o = (B.OptsStruct * 1)(B.make_opts(sketch_rank=9, variant=2, ep=1e-3))
    bound = ctypes.c_size_t()
    assert B.load().tt_hadamard_recompress_batch_plan(1, Ys, Zs, o, 1, ctypes.byref(bound)) == 0
    assert bound.value >= w2


def test_fixed_ranks_plan_bounds(lib):
    """fixed_ranks = 1 reports the bound the output keeps: min(l_k, max_rank)
    for a truncating HaTT call, min(b_k, max_rank) for tt_round_ex; 0 keeps the
    unpadded bounds; other values are rejected."""
    n = [6] * 5
    Yr, Zr = [1, 4, 5, 5, 3, 1], [1, 3, 4, 2, 3, 1]
    st, b0, _ = _plan(Yr, Zr, n, max_rank=5, sketch_rank=9)
    st1, b1, _ = _plan(Yr, Zr, n, max_rank=5, sketch_rank=9, fixed_ranks=1)
    assert st == st1 == 0
    assert b1 == [min(v, 5) for v in b0] and max(b0) > 5
    st2, _, _ = _plan(Yr, Zr, n, max_rank=5, sketch_rank=9, fixed_ranks=2)
    assert st2 == 3
    A = B.TT(n=[8] * 4, r=[1, 8, 30, 8, 1])
    for fixed, cap in ((0, 6), (1, 6), (1, 0)):
        bound = (ctypes.c_int64 * 5)()
        ws = ctypes.c_size_t()
        assert lib.tt_round_ex_plan(A.ref(), cap, 1e-8, fixed, bound, ctypes.byref(ws)) == 0
        base = [1, 8, 30, 8, 1]
        want = [min(v, cap) for v in base] if (fixed and cap) else base
        want[0] = want[-1] = 1
        assert list(bound) == want
    bound = (ctypes.c_int64 * 5)()
    assert lib.tt_round_ex_plan(A.ref(), 6, 1e-8, 3, bound, ctypes.byref(ws)) == 3


def test_pad_ranks_keeps_the_tensor():
    """Host-only: zero padding raises every inner rank and leaves the tensor
    (the contraction of the cores) unchanged."""
    import torch
    from paper_2410_04385_gb300 import allen_cahn as ac
    g = torch.Generator().manual_seed(0)
    u = [torch.randn(1, 5, 2, generator=g, dtype=torch.float64),
         torch.randn(2, 5, 3, generator=g, dtype=torch.float64),
         torch.randn(3, 5, 1, generator=g, dtype=torch.float64)]
    p = ac.pad_ranks(u, 4)
    assert [tuple(c.shape) for c in p] == [(1, 5, 4), (4, 5, 4), (4, 5, 1)]
    full = lambda cs: torch.einsum("aib,bjc,ckd->ijk", *cs)
    assert torch.allclose(full(u), full(p), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("n,Yr,Zr", [
    ([5], [1, 1], [1, 1]),                     # d = 1: one core, no recursion
    ([4, 6], [1, 3, 1], [1, 2, 1]),            # d = 2: one HPCRL step on W^(2) = [1]
    ([1, 7, 1, 3], [1, 1, 2, 2, 1], [1, 1, 3, 2, 1]),   # unit modes clamp the sketch to 1
])
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("fixed", [0, 1])
def test_plan_edge_shapes_every_variant(lib, n, Yr, Zr, variant, fixed):
    """Host-only: planning (which walks the whole launch sequence without
    launching) accepts orders 1 and 2 and unit mode sizes in every variant and
    output mode, and reports bounds no larger than the mode products allow."""
    st, bound, ws = _plan(Yr, Zr, n, max_rank=3, tol=1e-10, sketch_rank=4, variant=variant,
                          ep=0.1, fixed_ranks=fixed)
    assert st == 0 and ws > 0
    d = len(n)
    assert bound[0] == 1 and bound[d] == 1
    for k in range(1, d):
        left = int(np.prod(n[:k]))
        assert 1 <= bound[k] <= left


def test_gemm_plan_arguments(lib):
    """tt_gemm_plan (host only): a workspace for the tile counters and any
    split-K scratch; unknown precision, K < 1, negative sizes and a null
    output are refused with TT_ERR_ARG, sizes past 2^31 with TT_ERR_SHAPE."""
    ws = ctypes.c_size_t()
    for prec in range(5):
        assert lib.tt_gemm_plan(prec, 300, 77, 4096, 1, ctypes.byref(ws)) == 0 and ws.value > 16384
    assert lib.tt_gemm_plan(5, 4, 4, 4, 1, ctypes.byref(ws)) == 3
    assert lib.tt_gemm_plan(-1, 4, 4, 4, 1, ctypes.byref(ws)) == 3
    assert lib.tt_gemm_plan(0, 4, 4, 0, 1, ctypes.byref(ws)) == 3
    assert lib.tt_gemm_plan(0, -4, 4, 4, 1, ctypes.byref(ws)) == 3
    assert lib.tt_gemm_plan(0, 4, 4, 4, 1, None) == 3
    assert lib.tt_gemm_plan(0, 1 << 20, 1 << 12, 4, 1, ctypes.byref(ws)) == 1
