"""Host-side tests of the batched task engine's planning call
(tt_batched_plan_create): output ranks, workspace size and the refusals.
Device addresses are stand-ins that the planner forms but never dereferences;
nothing is launched."""
import ctypes
import os

import pytest

from oracle import hatt as ohatt
from paper_2410_04385_gb300 import binding as B
from paper_2410_04385_gb300 import build as libbuild

BASE = 1 << 40


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        libbuild.build()
    return B.load()


def descriptors(specs):
    """specs: list of (n, rY, rZ, opts); fake core addresses, 1 MiB apart."""
    Yd, Zd, Xd, Od = [], [], [], []
    slot = 0
    for n, ry, rz, o in specs:
        d = len(n)
        y, z = B.TT(n=n, r=ry), B.TT(n=n, r=rz)
        x = B.TT(n=n, r=[1] * (d + 1))
        for t in (y, z, x):
            t.set_core_ptrs([BASE + (slot + k) * (1 << 20) for k in range(d)])
            slot += d
        Yd.append(y), Zd.append(z), Xd.append(x), Od.append(B.make_opts(**o))
    arr = lambda ts: (B.TTStruct * len(ts))(*[t.s for t in ts])
    return Yd, Zd, Xd, arr(Yd), arr(Zd), arr(Xd), (B.OptsStruct * len(Od))(*Od)


def create(specs):
    Yd, Zd, Xd, Ya, Za, Xa, Oa = descriptors(specs)
    plan = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    st = B.load().tt_batched_plan_create(len(specs), Ya, Za, Oa, Xa, ctypes.byref(plan),
                                         ctypes.byref(ws))
    ranks = [[int(v) for v in Xa[j].r[: len(specs[j][0]) + 1]] for j in range(len(specs))]
    if plan.value:
        B.load().tt_batched_plan_destroy(plan)
    return st, int(ws.value), ranks


def test_plan_writes_the_clamped_sketch_ranks(lib):
    specs = [([4, 5, 6, 3], [1, 3, 4, 2, 1], [1, 2, 5, 3, 1], dict(sketch_rank=7, seed=1)),
             ([8, 8], [1, 6, 1], [1, 5, 1], dict(max_rank=12, oversample=0, seed=2)),
             ([3, 16, 16, 16, 3], [1, 3, 9, 9, 3, 1], [1, 2, 8, 8, 2, 1], dict(seed=3))]
    st, ws, ranks = create(specs)
    assert st == 0 and ws > 0
    for (n, ry, rz, o), got in zip(specs, ranks):
        lreq = ohatt.requested_sketch_rank(ry, rz, o.get("max_rank", 0), o.get("sketch_rank", 0),
                                           o.get("oversample", 10))
        assert got == [int(v) for v in ohatt.plan_ranks(n, ry, rz, lreq)]


def test_workspace_grows_linearly_with_the_batch(lib):
    # every pair has its own region: the size is a fixed part plus one region per pair
    one = [([16] * 6, [1] + [5] * 5 + [1], [1] + [4] * 5 + [1], dict(sketch_rank=12))]
    sizes = []
    for k in (1, 2, 3, 5):
        st, ws, _ = create(one * k)
        assert st == 0
        sizes.append(ws)
    per = sizes[1] - sizes[0]
    assert per > 0
    assert abs((sizes[2] - sizes[1]) - per) <= 0.05 * per
    assert abs((sizes[3] - sizes[0]) - 4 * per) <= 0.05 * 4 * per


@pytest.mark.parametrize("opts, expect", [
    (dict(sketch_rank=8, max_rank=4), 3),          # needs the truncation sweep
    (dict(sketch_rank=8, tol=1e-10), 3),           # tolerance: truncation sweep
    (dict(sketch_rank=8, precision=2), 3),         # TF32 tensor-core products
    (dict(sketch_rank=8, variant=2, ep=0.1), 3),   # HaTT-2: device-side ranks, not in the engine
    (dict(sketch_rank=8, precision=1), 0),         # FP32 sketch products
])
def test_plan_refusals(lib, opts, expect):
    st, _, _ = create([([6, 6, 6], [1, 3, 3, 1], [1, 4, 4, 1], opts)])
    assert st == expect


def test_plan_rejects_mismatched_modes(lib):
    Yd, Zd, Xd, Ya, Za, Xa, Oa = descriptors([([5, 5, 5], [1, 2, 2, 1], [1, 2, 2, 1], {})])
    zbad = B.TT(n=[5, 4, 5], r=[1, 2, 2, 1])
    zbad.set_core_ptrs([BASE, BASE + 8, BASE + 16])
    Za = (B.TTStruct * 1)(zbad.s)
    plan, ws = ctypes.c_void_p(), ctypes.c_size_t()
    st = B.load().tt_batched_plan_create(1, Ya, Za, Oa, Xa, ctypes.byref(plan), ctypes.byref(ws))
    assert st == 1 and not plan.value
