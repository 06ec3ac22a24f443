"""Thin ctypes binding of libhatt (include/hatt.h).

Argument marshalling only: torch supplies device memory and the current CUDA
stream; every arithmetic step runs in the library's CUDA kernels. The functions
keep the C names. If the compiled library is missing this module raises at
load time: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libhatt.so")

TT_OK = 0
TT_FP64 = 0
TT_MIXED_FP32 = 1
TT_MIXED_TF32 = 2
TT_MIXED_BF16 = 3
TT_FP64_TC = 4
TT_MAX_SMALL_RANK = 128


class TTStruct(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32),
        ("n", ctypes.POINTER(ctypes.c_int64)),
        ("r", ctypes.POINTER(ctypes.c_int64)),
        ("cores", ctypes.POINTER(ctypes.c_void_p)),
    ]


class OptsStruct(ctypes.Structure):
    _fields_ = [
        ("max_rank", ctypes.c_int64),
        ("tol", ctypes.c_double),
        ("sketch_rank", ctypes.c_int64),
        ("oversample", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("ep", ctypes.c_double),
        ("fixed_ranks", ctypes.c_int32),
        ("seed_offset", ctypes.c_void_p),
    ]


class HattError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed: status {status} ({msg})")
        self.status = status


_lib = None

EXPORTS = ("tt_hadamard_recompress_plan", "tt_hadamard_recompress", "tt_round_plan", "tt_round",
           "tt_round_ex_plan", "tt_round_ex",
           "tt_dot_plan", "tt_dot", "tt_dot_noalloc", "tt_norm", "tt_sketch_tt",
           "tt_philox4x32_10", "tt_launch_count", "tt_gemm_autotune", "tt_kernel_timer_start",
           "tt_kernel_timer_stop", "tt_kernel_timer_stop_ex", "tt_device_error", "tt_hadamard_recompress_batch_plan",
           "tt_hadamard_recompress_batch", "tt_scale", "tt_laplacian", "tt_lincomb",
           "tt_status_string", "tt_batched_plan_create", "tt_batched_plan_bind", "tt_batched_run",
           "tt_batched_status", "tt_batched_plan_info", "tt_batched_plan_destroy",
           "tt_batched_tune_cache", "tt_device_status", "tt_batched_profile", "tt_gemm_plan",
           "tt_gemm")


def load(path: Optional[str] = None):
    """Load libhatt.so (once). Raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libhatt.so not found at {p}; build it with "
                           "`python -m paper_2410_04385_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(p)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.tt_status_string.restype = ctypes.c_char_p
    lib.tt_status_string.argtypes = [ctypes.c_int]
    lib.tt_hadamard_recompress_plan.argtypes = [P(TTStruct), P(TTStruct), P(OptsStruct),
                                                P(ctypes.c_int64), P(ctypes.c_size_t)]
    lib.tt_hadamard_recompress.argtypes = [P(TTStruct), P(TTStruct), P(OptsStruct), P(TTStruct),
                                           vp, ctypes.c_size_t, vp]
    lib.tt_round_plan.argtypes = [P(TTStruct), ctypes.c_int64, ctypes.c_double, P(ctypes.c_int64),
                                  P(ctypes.c_size_t)]
    lib.tt_round.argtypes = [P(TTStruct), ctypes.c_int64, ctypes.c_double, P(TTStruct), vp,
                             ctypes.c_size_t, vp]
    lib.tt_round_ex_plan.argtypes = [P(TTStruct), ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                                     P(ctypes.c_int64), P(ctypes.c_size_t)]
    lib.tt_round_ex.argtypes = [P(TTStruct), ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                                P(TTStruct), vp, ctypes.c_size_t, vp]
    lib.tt_gemm_plan.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_int64, P(ctypes.c_size_t)]
    lib.tt_gemm.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                            ctypes.c_int64, vp, vp, vp, ctypes.c_double, vp, ctypes.c_size_t, vp]
    lib.tt_dot_plan.argtypes = [P(TTStruct), P(TTStruct), P(ctypes.c_size_t)]
    lib.tt_dot.argtypes = [P(TTStruct), P(TTStruct), vp, vp, ctypes.c_size_t, vp]
    lib.tt_dot_noalloc.argtypes = [P(TTStruct), P(TTStruct), vp, vp]
    lib.tt_norm.argtypes = [P(TTStruct), vp, vp, ctypes.c_size_t, vp]
    lib.tt_sketch_tt.argtypes = [ctypes.c_int32, P(ctypes.c_int64), P(ctypes.c_int64),
                                 ctypes.c_uint64, ctypes.c_uint32, P(ctypes.c_void_p), vp]
    lib.tt_philox4x32_10.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, vp, ctypes.c_int64, vp]
    lib.tt_launch_count.restype = ctypes.c_int64
    lib.tt_launch_count.argtypes = []
    lib.tt_kernel_timer_start.argtypes = [ctypes.c_int32]
    lib.tt_gemm_autotune.argtypes = [ctypes.c_int32]
    lib.tt_device_error.argtypes = [P(ctypes.c_int32)]
    lib.tt_device_status.argtypes = [P(ctypes.c_int32)]
    lib.tt_scale.argtypes = [vp, ctypes.c_int64, vp, vp]
    lib.tt_laplacian.argtypes = [P(TTStruct), ctypes.c_double, P(TTStruct), vp]
    lib.tt_lincomb.argtypes = [ctypes.c_int32, P(TTStruct), P(ctypes.c_double), P(TTStruct), vp]
    lib.tt_hadamard_recompress_batch_plan.argtypes = [ctypes.c_int32, P(TTStruct), P(TTStruct),
                                                      P(OptsStruct), ctypes.c_int32,
                                                      P(ctypes.c_size_t)]
    lib.tt_batched_plan_create.argtypes = [ctypes.c_int32, P(TTStruct), P(TTStruct),
                                           P(OptsStruct), P(TTStruct), P(vp), P(ctypes.c_size_t)]
    lib.tt_batched_plan_bind.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int32, vp]
    lib.tt_batched_run.argtypes = [vp, ctypes.c_int64, vp]
    lib.tt_batched_status.argtypes = [vp, vp, P(ctypes.c_int32)]
    lib.tt_batched_plan_info.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int32)]
    lib.tt_batched_plan_destroy.argtypes = [vp]
    lib.tt_batched_tune_cache.argtypes = [ctypes.c_char_p, ctypes.c_int32]
    lib.tt_batched_profile.argtypes = [vp, vp, P(ctypes.c_int64)]
    lib.tt_hadamard_recompress_batch.argtypes = [ctypes.c_int32, P(TTStruct), P(TTStruct),
                                                 P(OptsStruct), P(TTStruct), ctypes.c_int32, vp,
                                                 ctypes.c_size_t, vp]
    lib.tt_kernel_timer_stop.argtypes = [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int32,
                                         P(ctypes.c_int64)]
    lib.tt_kernel_timer_stop_ex.argtypes = [P(ctypes.c_double), P(ctypes.c_double),
                                            P(ctypes.c_int32), ctypes.c_int32, P(ctypes.c_int64)]
    for name in EXPORTS:
        getattr(lib, name)
    if path is None:
        _lib = lib
    return lib


def launch_count() -> int:
    """Kernels enqueued by libhatt in this process so far."""
    return int(load().tt_launch_count())


def gemm(A: torch.Tensor, B: torch.Tensor, precision=0, alpha=1.0, stream=None) -> torch.Tensor:
    """C = alpha A B through tt_gemm (A: [batch,] M x K, B: [batch,] K x N,
    contiguous CUDA float64); precision as tt_precision. Returns C (allocated
    here, with the workspace; enqueued on `stream`)."""
    for t in (A, B):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("A and B must be contiguous CUDA float64 tensors")
    squeeze = A.dim() == 2
    A3 = A.unsqueeze(0) if squeeze else A
    B3 = B.unsqueeze(0) if squeeze else B
    if A3.dim() != 3 or B3.dim() != 3 or A3.shape[0] != B3.shape[0] or A3.shape[2] != B3.shape[1]:
        raise ValueError("shapes do not chain")
    nb, M, K = (int(v) for v in A3.shape)
    N = int(B3.shape[2])
    lib = load()
    ws = ctypes.c_size_t()
    _check("tt_gemm_plan", lib.tt_gemm_plan(int(precision), M, N, K, nb, ctypes.byref(ws)))
    with torch.cuda.device(A.device):
        work = torch.empty(max(int(ws.value), 1), dtype=torch.uint8, device=A.device)
        C = torch.empty((nb, M, N), dtype=torch.float64, device=A.device)
        _check("tt_gemm", lib.tt_gemm(int(precision), M, N, K, nb, ctypes.c_void_p(A3.data_ptr()),
                                      ctypes.c_void_p(B3.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                                      float(alpha), ctypes.c_void_p(work.data_ptr()), int(ws.value),
                                      _stream_ptr(stream)))
        if stream is not None:
            work.record_stream(stream)
            C.record_stream(stream)
    return C[0] if squeeze else C


def tt_scale(x: torch.Tensor, divisor: torch.Tensor, stream=None) -> None:
    """x /= divisor[0] in place on the device (both CUDA float64)."""
    if x.dtype != torch.float64 or divisor.dtype != torch.float64 or not x.is_contiguous():
        raise ValueError("x and divisor must be contiguous CUDA float64 tensors")
    _check("tt_scale", load().tt_scale(ctypes.c_void_p(x.data_ptr()), x.numel(),
                                       ctypes.c_void_p(divisor.data_ptr()), _stream_ptr(stream)))


def tt_laplacian(A: Sequence[torch.Tensor], inv_h2: float, out=None,
                 stream=None) -> List[torch.Tensor]:
    """Periodic central-difference Laplacian of the TT A (ranks doubled);
    `out` may hold preallocated cores of the result's shapes."""
    Ad = TT(A)
    d, n, r = Ad.d, Ad.n, Ad.r
    rl = [1] + [2 * v for v in r[1:-1]] + [1] if d > 1 else [1, 1]
    if out is None:
        out = [torch.empty((rl[k], n[k], rl[k + 1]), dtype=torch.float64, device=A[0].device)
               for k in range(d)]
    Ld = TT(out)
    _check("tt_laplacian", load().tt_laplacian(Ad.ref(), float(inv_h2), Ld.ref(), _stream_ptr(stream)))
    return out


def tt_lincomb(terms: Sequence[Sequence[torch.Tensor]], coef: Sequence[float], out=None,
               stream=None) -> List[torch.Tensor]:
    """sum_j coef[j] terms[j] as one TT (block-diagonal cores); `out` may
    hold preallocated cores of the result's shapes."""
    Td = [TT(t) for t in terms]
    d, n = Td[0].d, Td[0].n
    rs = [sum(t.r[k] for t in Td) for k in range(d + 1)]
    rs[0] = rs[d] = 1
    if out is None:
        out = [torch.empty((rs[k], n[k], rs[k + 1]), dtype=torch.float64,
                           device=terms[0][0].device) for k in range(d)]
    Sd = TT(out)
    Ta = (TTStruct * len(Td))(*[t.s for t in Td])
    ca = (ctypes.c_double * len(coef))(*[float(c) for c in coef])
    _check("tt_lincomb", load().tt_lincomb(len(Td), Ta, ca, Sd.ref(), _stream_ptr(stream)))
    return out


def device_error() -> int:
    """Read and clear the device error word (synchronizes): nonzero when a
    bounded wait inside a kernel ran out since the last read."""
    v = ctypes.c_int32(0)
    _check("tt_device_error", load().tt_device_error(ctypes.byref(v)))
    return int(v.value)


def gemm_autotune(enable: bool) -> None:
    """First-use timing of FP64 GEMM tilings (tt_gemm_autotune); on by default."""
    _check("tt_gemm_autotune", load().tt_gemm_autotune(1 if enable else 0))


def kernel_timer_start(capacity: int) -> None:
    """Start timing the FP64 GEMM kernel launches (outside graph capture)
    with CUDA events on their own stream; see tt_kernel_timer_start."""
    _check("tt_kernel_timer_start", load().tt_kernel_timer_start(int(capacity)))


TT_ROLE_AUX = 0
TT_ROLE_METHOD = 1


def kernel_timer_stop(capacity: int, with_roles: bool = False):
    """Stop the timer; returns (ms, flops, recorded): per-launch durations in
    milliseconds and algorithmic flop counts of the first min(recorded,
    capacity) timed launches; with_roles adds the list of launch roles
    (TT_ROLE_METHOD / TT_ROLE_AUX) as a fourth item."""
    ms = (ctypes.c_double * max(capacity, 1))()
    fl = (ctypes.c_double * max(capacity, 1))()
    ro = (ctypes.c_int32 * max(capacity, 1))()
    cnt = ctypes.c_int64(0)
    _check("tt_kernel_timer_stop_ex",
           load().tt_kernel_timer_stop_ex(ms, fl, ro, int(capacity), ctypes.byref(cnt)))
    k = min(int(cnt.value), int(capacity))
    if with_roles:
        return list(ms[:k]), list(fl[:k]), int(cnt.value), list(ro[:k])
    return list(ms[:k]), list(fl[:k]), int(cnt.value)


def status_string(status: int) -> str:
    return load().tt_status_string(int(status)).decode()


def _check(fn: str, status: int):
    if status != TT_OK:
        raise HattError(fn, status, status_string(status))


def _stream_ptr(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class TT:
    """Host-side descriptor (tt_t) of a TT given as a list of CUDA float64 cores
    of shapes (r_k, n_k, r_{k+1}), or of shapes only (cores=None)."""

    def __init__(self, cores: Optional[Sequence[torch.Tensor]] = None, n=None, r=None,
                 pinned_ranks: bool = False):
        if cores is not None:
            for c in cores:
                if c.dtype != torch.float64 or not c.is_cuda or not c.is_contiguous():
                    raise ValueError("cores must be contiguous CUDA float64 tensors")
            n = [int(c.shape[1]) for c in cores]
            r = [int(cores[0].shape[0])] + [int(c.shape[2]) for c in cores]
        self.d = len(n)
        self.n_arr = (ctypes.c_int64 * self.d)(*n)
        if pinned_ranks:
            # page-locked rank array: the library's device-to-host rank copy is
            # then asynchronous and can be captured in a CUDA graph
            self.r_pinned = torch.tensor(list(r), dtype=torch.int64).pin_memory()
            self.r_arr = ctypes.cast(self.r_pinned.data_ptr(), ctypes.POINTER(ctypes.c_int64))
        else:
            self.r_pinned = None
            self.r_arr = (ctypes.c_int64 * (self.d + 1))(*r)
        self.core_arr = (ctypes.c_void_p * self.d)()
        self.cores = list(cores) if cores is not None else None
        if cores is not None:
            for k, c in enumerate(cores):
                self.core_arr[k] = c.data_ptr()
        self.s = TTStruct(self.d, self.n_arr, self.r_arr, self.core_arr)

    def set_core_ptrs(self, ptrs):
        for k, p in enumerate(ptrs):
            self.core_arr[k] = p

    @property
    def n(self):
        return [int(v) for v in self.n_arr]

    @property
    def r(self):
        return [int(self.r_arr[k]) for k in range(self.d + 1)]

    def ref(self):
        return ctypes.byref(self.s)


def make_opts(max_rank=0, tol=0.0, sketch_rank=0, oversample=10, seed=0, precision=TT_FP64,
              variant=1, ep=0.0, fixed_ranks=0, seed_offset=None):
    """seed_offset: None, or a CUDA uint64/int64 tensor of one element whose
    value the sketch adds to `seed` when it runs (graph replays)."""
    off = None if seed_offset is None else ctypes.c_void_p(seed_offset.data_ptr())
    return OptsStruct(int(max_rank), float(tol), int(sketch_rank), int(oversample),
                      int(seed) & 0xFFFFFFFFFFFFFFFF, int(precision), int(variant), float(ep),
                      int(fixed_ranks), off)


class HadamardRecompressor:
    """Plans once and owns the output buffers and workspace, so repeated calls
    (benchmarks, time stepping) allocate nothing. `run` enqueues on `stream`."""

    def __init__(self, Y: Sequence[torch.Tensor], Z: Sequence[torch.Tensor], **opts):
        lib = load()
        self.Yd = TT(Y)
        self.Zd = TT(Z)
        self.opts = make_opts(**opts)
        d = self.Yd.d
        self.bound = (ctypes.c_int64 * (d + 1))()
        ws = ctypes.c_size_t()
        _check("tt_hadamard_recompress_plan",
               lib.tt_hadamard_recompress_plan(self.Yd.ref(), self.Zd.ref(), ctypes.byref(self.opts),
                                               self.bound, ctypes.byref(ws)))
        self.workspace_bytes = int(ws.value)
        dev = Y[0].device
        self.workspace = torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=dev)
        n = self.Yd.n
        b = [int(v) for v in self.bound]
        self.out_bufs = [torch.empty(b[k] * n[k] * b[k + 1], dtype=torch.float64, device=dev)
                         for k in range(d)]
        self.Xd = TT(n=n, r=b, pinned_ranks=True)
        self.Xd.set_core_ptrs([t.data_ptr() for t in self.out_bufs])
        self.graph = None

    def rebind(self, Y: Sequence[torch.Tensor], Z: Sequence[torch.Tensor]):
        """Point at new input cores of the same shapes."""
        self.Yd.set_core_ptrs([c.data_ptr() for c in Y])
        self.Zd.set_core_ptrs([c.data_ptr() for c in Z])

    def run(self, stream=None):
        st = load().tt_hadamard_recompress(self.Yd.ref(), self.Zd.ref(), ctypes.byref(self.opts),
                                           self.Xd.ref(), ctypes.c_void_p(self.workspace.data_ptr()),
                                           self.workspace_bytes, _stream_ptr(stream))
        _check("tt_hadamard_recompress", st)

    def capture(self):
        """Capture one call in a CUDA graph (the library's launch sequence is
        fixed and allocation-free); replay with `replay()`."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(s)                      # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def result(self) -> List[torch.Tensor]:
        """Output cores as views (call after the stream has completed)."""
        r = self.Xd.r
        n = self.Xd.n
        return [self.out_bufs[k][: r[k] * n[k] * r[k + 1]].view(r[k], n[k], r[k + 1])
                for k in range(self.Xd.d)]


def tt_hadamard_recompress(Y, Z, max_rank=0, tol=0.0, sketch_rank=0, oversample=10, seed=0,
                           precision=TT_FP64, variant=1, ep=0.0, fixed_ranks=0, seed_offset=None,
                           stream=None) -> List[torch.Tensor]:
    """HaTT recompression of Y ⊙ Z; returns the output cores (synchronizes).
    precision: TT_FP64, TT_MIXED_FP32 / TF32 / BF16 or TT_FP64_TC;
    variant 1 = HaTT-1, 2 = HaTT-2 with threshold ep; seed_offset: None or a
    one-element CUDA int64 tensor added to the sketch key."""
    h = HadamardRecompressor(Y, Z, max_rank=max_rank, tol=tol, sketch_rank=sketch_rank,
                             oversample=oversample, seed=seed, precision=precision,
                             variant=variant, ep=ep, fixed_ranks=fixed_ranks,
                             seed_offset=seed_offset)
    h.run(stream)
    (stream or torch.cuda.current_stream()).synchronize()
    return [c.clone() for c in h.result()]


class Rounder:
    """tt_round_ex planned once for inputs of fixed shapes: owns the output
    buffers and the workspace, so `run` allocates nothing and (with
    fixed_ranks=1, which also keeps the output shapes fixed) can be captured
    in a CUDA graph."""

    def __init__(self, A: Sequence[torch.Tensor], max_rank=0, tol=0.0, fixed_ranks=0):
        lib = load()
        self.Ad = TT(A)
        self.max_rank, self.tol, self.fixed = int(max_rank), float(tol), int(fixed_ranks)
        d = self.Ad.d
        bound = (ctypes.c_int64 * (d + 1))()
        ws = ctypes.c_size_t()
        _check("tt_round_ex_plan", lib.tt_round_ex_plan(self.Ad.ref(), self.max_rank, self.tol,
                                                        self.fixed, bound, ctypes.byref(ws)))
        dev = A[0].device
        self.workspace_bytes = int(ws.value)
        self.workspace = torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=dev)
        n = self.Ad.n
        b = [int(v) for v in bound]
        self.out_bufs = [torch.empty(b[k] * n[k] * b[k + 1], dtype=torch.float64, device=dev)
                         for k in range(d)]
        self.Bd = TT(n=n, r=b, pinned_ranks=True)
        self.Bd.set_core_ptrs([t.data_ptr() for t in self.out_bufs])

    def run(self, stream=None):
        _check("tt_round_ex", load().tt_round_ex(self.Ad.ref(), self.max_rank, self.tol, self.fixed,
                                                 self.Bd.ref(),
                                                 ctypes.c_void_p(self.workspace.data_ptr()),
                                                 self.workspace_bytes, _stream_ptr(stream)))

    def result(self) -> List[torch.Tensor]:
        """Output cores as views (call after the stream has completed)."""
        r, n = self.Bd.r, self.Bd.n
        return [self.out_bufs[k][: r[k] * n[k] * r[k + 1]].view(r[k], n[k], r[k + 1])
                for k in range(self.Bd.d)]


def tt_round(A, max_rank=0, tol=0.0, fixed_ranks=0, stream=None) -> List[torch.Tensor]:
    """TT rounding of A (synchronizes); fixed_ranks=1 keeps the bound ranks
    min(b_k, max_rank), zero past the ranks kept."""
    h = Rounder(A, max_rank=max_rank, tol=tol, fixed_ranks=fixed_ranks)
    h.run(stream)
    (stream or torch.cuda.current_stream()).synchronize()
    return [c.clone() for c in h.result()]


def _dot_common(fn, A, B, stream):
    lib = load()
    Ad = TT(A)
    Bd = TT(B)
    ws = ctypes.c_size_t()
    _check("tt_dot_plan", lib.tt_dot_plan(Ad.ref(), Bd.ref(), ctypes.byref(ws)))
    dev = A[0].device
    work = torch.empty(max(int(ws.value), 1), dtype=torch.uint8, device=dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    if fn == "tt_dot":
        st = lib.tt_dot(Ad.ref(), Bd.ref(), ctypes.c_void_p(out.data_ptr()),
                        ctypes.c_void_p(work.data_ptr()), int(ws.value), _stream_ptr(stream))
    else:
        st = lib.tt_norm(Ad.ref(), ctypes.c_void_p(out.data_ptr()),
                         ctypes.c_void_p(work.data_ptr()), int(ws.value), _stream_ptr(stream))
    _check(fn, st)
    (stream or torch.cuda.current_stream()).synchronize()
    return out


def tt_dot(A, B, stream=None) -> torch.Tensor:
    """<A, B> as a 1-element CUDA tensor."""
    return _dot_common("tt_dot", A, B, stream)


def tt_dot_noalloc(A, B, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """<A, B> through tt_dot_noalloc: no device allocation inside the library
    (its scratch is a fixed per-GPU array). `out` may be preallocated so that
    the call allocates nothing on the Python side either."""
    Ad = TT(A)
    Bd = TT(B)
    dev = A[0].device
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=dev)
    elif out.device != dev or out.dtype != torch.float64 or out.numel() < 1:
        raise ValueError("out must be a float64 tensor on the cores' device")
    # the library takes its scratch array and stream from the current device
    with torch.cuda.device(dev):
        _check("tt_dot_noalloc", load().tt_dot_noalloc(Ad.ref(), Bd.ref(),
                                                       ctypes.c_void_p(out.data_ptr()),
                                                       _stream_ptr(stream)))
    return out


def tt_norm(A, stream=None) -> torch.Tensor:
    """||A||_F as a 1-element CUDA tensor."""
    return _dot_common("tt_norm", A, A, stream)


def tt_sketch_tt(n, ell, seed=0, pair=0, device="cuda", stream=None) -> List[torch.Tensor]:
    """Gaussian sketch TT of Definition 2.1, generated by the library."""
    lib = load()
    d = len(n)
    cores = [torch.empty((int(ell[k]), int(n[k]), int(ell[k + 1])), dtype=torch.float64,
                         device=device) for k in range(d)]
    ptrs = (ctypes.c_void_p * d)(*[c.data_ptr() for c in cores])
    _check("tt_sketch_tt", lib.tt_sketch_tt(d, (ctypes.c_int64 * d)(*n),
                                            (ctypes.c_int64 * (d + 1))(*ell), int(seed),
                                            int(pair), ptrs, _stream_ptr(stream)))
    (stream or torch.cuda.current_stream()).synchronize()
    return cores


def tt_philox4x32_10(ctr: torch.Tensor, key0: int, key1: int, stream=None) -> torch.Tensor:
    """Raw Philox4x32-10 blocks; ctr is an int32 CUDA tensor of shape (count, 4)
    holding the counter words' bit patterns. Returns the same shape."""
    if ctr.dtype != torch.int32 or ctr.dim() != 2 or ctr.shape[1] != 4 or not ctr.is_cuda:
        raise ValueError("ctr must be an int32 CUDA tensor of shape (count, 4)")
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    _check("tt_philox4x32_10", load().tt_philox4x32_10(
        ctypes.c_void_p(ctr.data_ptr()), int(key0) & 0xFFFFFFFF, int(key1) & 0xFFFFFFFF,
        ctypes.c_void_p(out.data_ptr()), int(ctr.shape[0]), _stream_ptr(stream)))
    (stream or torch.cuda.current_stream()).synchronize()
    return out


class BatchRecompressor:
    """Many independent pairs (uneven orders, modes, ranks) recompressed by one
    tt_hadamard_recompress_batch call over `lanes` library streams. Plans once
    and owns every output buffer and the lane workspace."""

    def __init__(self, pairs, lanes: int = 8):
        """pairs: list of (Y cores, Z cores, options dict) with CUDA float64 cores."""
        lib = load()
        self.count = len(pairs)
        self.lanes = int(lanes)
        self.Yd = [TT(Y) for Y, _, _ in pairs]
        self.Zd = [TT(Z) for _, Z, _ in pairs]
        self.opts = [make_opts(**o) for _, _, o in pairs]
        self.Xd, self.out_bufs = [], []
        for (Y, _, _), yd, zd, op in zip(pairs, self.Yd, self.Zd, self.opts):
            bound = (ctypes.c_int64 * (yd.d + 1))()
            ws = ctypes.c_size_t()
            _check("tt_hadamard_recompress_plan",
                   lib.tt_hadamard_recompress_plan(yd.ref(), zd.ref(), ctypes.byref(op), bound,
                                                   ctypes.byref(ws)))
            n, b = yd.n, [int(v) for v in bound]
            bufs = [torch.empty(b[k] * n[k] * b[k + 1], dtype=torch.float64, device=Y[0].device)
                    for k in range(yd.d)]
            xd = TT(n=n, r=b, pinned_ranks=True)
            xd.set_core_ptrs([t.data_ptr() for t in bufs])
            self.Xd.append(xd)
            self.out_bufs.append(bufs)
        self.Ya = (TTStruct * max(self.count, 1))(*[t.s for t in self.Yd])
        self.Za = (TTStruct * max(self.count, 1))(*[t.s for t in self.Zd])
        self.Xa = (TTStruct * max(self.count, 1))(*[t.s for t in self.Xd])
        self.Oa = (OptsStruct * max(self.count, 1))(*self.opts)
        ws = ctypes.c_size_t()
        _check("tt_hadamard_recompress_batch_plan",
               lib.tt_hadamard_recompress_batch_plan(self.count, self.Ya, self.Za, self.Oa,
                                                     self.lanes, ctypes.byref(ws)))
        self.workspace_bytes = int(ws.value)
        dev = pairs[0][0][0].device if pairs else torch.device("cuda")
        self.workspace = torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=dev)
        self.graph = None

    def run(self, stream=None):
        _check("tt_hadamard_recompress_batch",
               load().tt_hadamard_recompress_batch(self.count, self.Ya, self.Za, self.Oa, self.Xa,
                                                   self.lanes,
                                                   ctypes.c_void_p(self.workspace.data_ptr()),
                                                   self.workspace_bytes, _stream_ptr(stream)))

    def capture(self):
        """One batch call in a CUDA graph (the lanes fork from and join into the
        capturing stream); replay with `replay()`."""
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def result(self, j: int) -> List[torch.Tensor]:
        r, n = self.Xd[j].r, self.Xd[j].n
        return [self.out_bufs[j][k][: r[k] * n[k] * r[k + 1]].view(r[k], n[k], r[k + 1])
                for k in range(self.Xd[j].d)]


TT_ERR_NONFINITE = 6
TT_ERR_TIMEOUT = 7
TT_ERR_BREAKDOWN = 8
DEFAULT_SPIN_CAP = 1 << 26


def device_status() -> int:
    """Read and clear the device error word as a status (synchronizes):
    TT_OK, TT_ERR_TIMEOUT, TT_ERR_NONFINITE or TT_ERR_BREAKDOWN."""
    v = ctypes.c_int32(0)
    _check("tt_device_status", load().tt_device_status(ctypes.byref(v)))
    return int(v.value)


class BatchedRecompressor:
    """Many independent pairs recompressed by ONE persistent launch of the task
    engine (tt_batched_*). Plans once, owns every output buffer and the
    workspace; `run` enqueues the launch (capturable after construction)."""

    def __init__(self, pairs, autotune: bool = True, stream=None):
        """pairs: list of (Y cores, Z cores, options dict) with CUDA float64
        cores; options as tt_hadamard_recompress (no truncation: sketch rank =
        output rank), precision TT_FP64 or TT_MIXED_FP32."""
        lib = load()
        self.count = len(pairs)
        self.pairs = pairs                       # keeps the input tensors alive
        self.Yd = [TT(Y) for Y, _, _ in pairs]
        self.Zd = [TT(Z) for _, Z, _ in pairs]
        self.opts = [make_opts(**o) for _, _, o in pairs]
        self.Xd, self.out_bufs = [], []
        for (Y, _, _), yd, zd, op in zip(pairs, self.Yd, self.Zd, self.opts):
            bound = (ctypes.c_int64 * (yd.d + 1))()
            ws = ctypes.c_size_t()
            _check("tt_hadamard_recompress_plan",
                   lib.tt_hadamard_recompress_plan(yd.ref(), zd.ref(), ctypes.byref(op), bound,
                                                   ctypes.byref(ws)))
            n, b = yd.n, [int(v) for v in bound]
            bufs = [torch.empty(b[k] * n[k] * b[k + 1], dtype=torch.float64, device=Y[0].device)
                    for k in range(yd.d)]
            xd = TT(n=n, r=b, pinned_ranks=True)
            xd.set_core_ptrs([t.data_ptr() for t in bufs])
            self.Xd.append(xd)
            self.out_bufs.append(bufs)
        self.Ya = (TTStruct * self.count)(*[t.s for t in self.Yd])
        self.Za = (TTStruct * self.count)(*[t.s for t in self.Zd])
        self.Xa = (TTStruct * self.count)(*[t.s for t in self.Xd])
        self.Oa = (OptsStruct * self.count)(*self.opts)
        self.plan = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        _check("tt_batched_plan_create",
               lib.tt_batched_plan_create(self.count, self.Ya, self.Za, self.Oa, self.Xa,
                                          ctypes.byref(self.plan), ctypes.byref(ws)))
        self.workspace_bytes = int(ws.value)
        dev = pairs[0][0][0].device
        self.workspace = torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=dev)
        _check("tt_batched_plan_bind",
               lib.tt_batched_plan_bind(self.plan, ctypes.c_void_p(self.workspace.data_ptr()),
                                        self.workspace_bytes, 1 if autotune else 0,
                                        _stream_ptr(stream)))

    def run(self, spin_cap: int = DEFAULT_SPIN_CAP, stream=None):
        _check("tt_batched_run", load().tt_batched_run(self.plan, int(spin_cap), _stream_ptr(stream)))

    def status(self, stream=None) -> int:
        v = ctypes.c_int32(0)
        _check("tt_batched_status", load().tt_batched_status(self.plan, _stream_ptr(stream),
                                                             ctypes.byref(v)))
        return int(v.value)

    def info(self):
        st, tk, bl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check("tt_batched_plan_info", load().tt_batched_plan_info(self.plan, ctypes.byref(st),
                                                                   ctypes.byref(tk), ctypes.byref(bl)))
        return {"stages": int(st.value), "tasks": int(tk.value), "blocks": int(bl.value)}

    def profile(self, stream=None):
        """Sums over the CTAs of the last run's cycle counters (see
        tt_batched_profile) as a dict of fractions of the CTAs' time."""
        out = (ctypes.c_int64 * 24)()
        _check("tt_batched_profile", load().tt_batched_profile(self.plan, _stream_ptr(stream), out))
        total = max(int(out[0]), 1)
        kinds = ("sketch", "gemm", "norm_part", "norm", "first_core", "cholesky", "qr_apply", "set")
        res = {"wait_frac": out[1] / total, "ticket_frac": out[2] / total}
        for t, name in enumerate(kinds):
            res[f"{name}_frac"] = out[8 + t] / total
            res[f"{name}_tasks"] = int(out[16 + t])
        return res

    def result(self, j: int) -> List[torch.Tensor]:
        r, n = self.Xd[j].r, self.Xd[j].n
        return [self.out_bufs[j][k][: r[k] * n[k] * r[k + 1]].view(r[k], n[k], r[k + 1])
                for k in range(self.Xd[j].d)]

    def __del__(self):
        if getattr(self, "plan", None) is not None and self.plan.value and _lib is not None:
            _lib.tt_batched_plan_destroy(self.plan)
            self.plan = ctypes.c_void_p()


def batched_tune_cache(path: str, save: bool) -> None:
    """Save or load the engine's process-wide tile cache (text lines)."""
    _check("tt_batched_tune_cache", load().tt_batched_tune_cache(path.encode(), 1 if save else 0))
