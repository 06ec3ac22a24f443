"""Product-level checks of the contraction kernels through the C ABI
(tt_gemm), element by element, on shapes of the benchmark configurations:

* HPCRL S1 of the smooth d = 50 pair (batch 64 of 1600 x 90 x 90) and a
  long-K product (300 x 77 x 4096: several 128-row tiles, a ragged N, K
  split into slices).
* TT_MIXED_TF32 / TT_MIXED_BF16 run on the tcgen05 tensor cores, FP32
  accumulation per K slice; TT_MIXED_FP32 on the SIMT kernel with FP32
  operands. Every element must lie within the FP32 accumulation bound of the
  exact product of the operands rounded as the format prescribes (the
  oracle's round_operand):
      |C - A~ B~| <= gamma_K (|A~| |B~|),  gamma_K = K u / (1 - K u),
  with u = 2^-23 (one ulp per addition: the bound holds whether the
  accumulator rounds or truncates). A~ B~ and |A~| |B~| are formed in FP64
  (exact products of <= 24-bit mantissas, FP64 sums far below the bound).
* The operands are really rounded to the format: all-(1 + 2^-12) operands
  (TF32 keeps 10 mantissa bits, so they round to 1) and all-(1 + 2^-9)
  operands (BF16 keeps 7) give C = K to within K u, not K (1 + 2^-11) or
  K (1 + 2^-8) as unrounded operands would.
* TT_FP64 within the FP64 bound gamma_K with u = 2^-53, times 2."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hatt as ohatt

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

FMT = {1: "fp32", 2: "tf32", 3: "bf16"}
SHAPES = [(64, 1600, 90, 90), (1, 300, 77, 4096)]


@pytest.fixture(scope="module")
def B():
    import os
    from paper_2410_04385_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    return binding


def operands(shape, seed):
    nb, M, N, K = shape
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((nb, M, K)) * np.exp(rng.uniform(-2, 2, (nb, M, 1)))
    Bm = rng.standard_normal((nb, K, N)) * np.exp(rng.uniform(-2, 2, (nb, 1, N)))
    return A, Bm


def gamma(K, u):
    return K * u / (1.0 - K * u)


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("shape", SHAPES, ids=["hpcrl_s1_d50", "long_k"])
def test_low_precision_product_within_fp32_accumulation_bound(B, prec, shape):
    A, Bm = operands(shape, 7 + prec)
    C = B.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda(), precision=prec)
    torch.cuda.synchronize()
    C = C.cpu().numpy()
    Ar, Br = ohatt.round_operand(A, FMT[prec]), ohatt.round_operand(Bm, FMT[prec])
    ref = Ar @ Br
    scale = np.abs(Ar) @ np.abs(Br)
    K = shape[3]
    err = np.abs(C - ref)
    assert np.all(err <= gamma(K, 2.0 ** -23) * scale + 1e-300)
    assert B.device_error() == 0


@pytest.mark.parametrize("prec, x", [(2, 1.0 + 2.0 ** -12), (3, 1.0 + 2.0 ** -9)])
def test_operands_are_rounded_to_the_format(B, prec, x):
    K = 256
    A = np.full((1, 130, K), x)
    Bm = np.full((1, K, 33), x)
    C = B.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda(), precision=prec)
    torch.cuda.synchronize()
    C = C.cpu().numpy()
    assert np.all(np.abs(C - K) <= K * K * 2.0 ** -23)
    assert np.all(np.abs(C - K * x * x) > 0.5 * K * (x * x - 1.0))


@pytest.mark.parametrize("shape", SHAPES, ids=["hpcrl_s1_d50", "long_k"])
def test_fp64_product_within_fp64_bound(B, shape):
    A, Bm = operands(shape, 3)
    C = B.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda(), precision=0, alpha=0.5)
    torch.cuda.synchronize()
    C = C.cpu().numpy()
    ref = 0.5 * (A @ Bm)
    scale = 0.5 * (np.abs(A) @ np.abs(Bm))
    K = shape[3]
    assert np.all(np.abs(C - ref) <= 2 * gamma(K, 2.0 ** -53) * scale + 1e-300)
