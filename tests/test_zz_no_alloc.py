"""GPU test of tt_dot_noalloc, the inner product for callers that cannot
allocate device memory (for example a real-time loop that forbids allocation,
or a plugin whose host framework owns the GPU's memory). Its scratch is a fixed
per-GPU array inside the library, so the test checks that two calls in a row
on the same array give the same result as tt_dot with a caller-owned
workspace, and that a problem larger than the array is refused up front.

The file name sorts last so that a run stopping at the first failure has
already run every other test."""
import ctypes
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2410_04385_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

REL_TOL = 1e-12


@pytest.fixture(scope="module")
def B():
    from paper_2410_04385_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    return binding


def to_gpu(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def call_noalloc(B, A, C, out):
    Ad, Cd = B.TT(A), B.TT(C)
    st = B.load().tt_dot_noalloc(Ad.ref(), Cd.ref(), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("case", ["random_d20", "uneven_d6"])
def test_noalloc_dot_matches_tt_dot_on_two_calls(B, case):
    if case == "random_d20":
        Y, Z, _ = wl.workload_random_d20()
    else:
        Y = wl.gaussian_tt([64, 17, 33, 64, 5, 64], [1, 30, 7, 40, 12, 25, 1], 7)
        Z = wl.gaussian_tt([64, 17, 33, 64, 5, 64], [1, 40, 21, 3, 33, 9, 1], 8)
    A, C = to_gpu(Y), to_gpu(Z)
    ref = B.tt_dot(A, C).item()
    scale = B.tt_norm(A).item() * B.tt_norm(C).item()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        assert call_noalloc(B, A, C, out) == B.TT_OK
        assert abs(out.item() - ref) <= REL_TOL * scale
    # the Python wrapper, into a preallocated result
    out.fill_(float("nan"))
    assert B.tt_dot_noalloc(A, C, out=out) is out
    torch.cuda.synchronize()
    assert abs(out.item() - ref) <= REL_TOL * scale


def test_noalloc_dot_refuses_problems_beyond_its_scratch(B):
    # T = G H(B_k) alone needs 128 * 512 * 128 doubles = 64 MiB > 8 MiB
    n = [512, 512, 512]
    A = [torch.zeros((1, 512, 128), dtype=torch.float64, device="cuda"),
         torch.zeros((128, 512, 128), dtype=torch.float64, device="cuda"),
         torch.zeros((128, 512, 1), dtype=torch.float64, device="cuda")]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert call_noalloc(B, A, A, out) == 4          # TT_ERR_WORKSPACE
    assert B.status_string(4).startswith("workspace")
    assert n == [c.shape[1] for c in A]
