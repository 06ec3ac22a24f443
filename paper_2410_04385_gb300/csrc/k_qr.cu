// Economy QR of the tall sketch S = C_k W^{(k)} (Algorithm 4) on GB300.
//
// Householder QR is a chain of rank-1 updates and would run on one SM at the
// FP64 rate of a single SM (~8 GFLOP/s on GB300). Cholesky QR instead spends
// almost all of its flops in two SM-parallel products (the Gram S^T S and
// S R^{-1}); only a c x c Cholesky factorization and triangular inverse run in
// one block. A pass is
//     G = S^T S,  R^T R = G (+ shift),  S <- S R^{-1}
// and passes repeat until G = I to working accuracy (Cholesky QR2 needs two
// passes for cond(S) < ~1e8). When the unshifted factorization breaks down
// (cond(S) >~ 1e8, or exactly dependent columns as in Y ⊙ Y or exact
// low-rank products), the pass uses the shift s = 11 (m c + c (c + 1)) u tr(G)
// of shifted Cholesky QR (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa,
// SIAM J. Sci. Comput. 2020); each shifted pass lifts the smallest singular
// values towards 1, so later passes converge. A column that is exactly zero
// stays zero (its Gram row and column vanish), which leaves a partial
// isometry whose zero columns carry nothing into the next core.
//
// All passes are launched unconditionally (fixed launch sequence, capturable
// in a CUDA graph); a device flag set by the convergence test turns the
// remaining launches into no-ops.
#include <algorithm>
#include "hatt_internal.cuh"

namespace hatt {
namespace {

constexpr int kPasses = 4;
constexpr int kCholThreads = 256;
constexpr int kTrmmThreads = 256;
constexpr int kTrmmRows = 16;
constexpr size_t kCholSmemMax = 200 * 1024;   // dynamic shared memory of the Cholesky block

// G (c x (c+1)) plus, when it fits, R^{-1} (c x c)
__host__ __device__ constexpr size_t chol_smem_doubles(int c, bool with_inv) {
  return (size_t)c * (c + 1) + (with_inv ? (size_t)c * c : 0);
}

// 1/sqrt(x) for finite x > 0: range reduction x = m 2^e with e even, an FP32
// seed for m, then two Newton-Raphson steps y <- y (3 - m y^2) / 2 in FP64
// (each squares the relative error: 2^-23 -> 2^-46 -> below FP64 rounding).
// A handful of dependent FP64 multiply-adds instead of the long FP64 sqrt and
// divide sequences, which sit on the Cholesky critical path once per column.
__device__ __forceinline__ double rsqrt_newton(double x) {
  int e;
  double m = frexp(x, &e);                 // m in [0.5, 1)
  if (e & 1) { m *= 2.0; e -= 1; }         // m in [0.5, 2), e even
  double y = (double)rsqrtf((float)m);
  y = y * fma(-0.5 * m, y * y, 1.5);
  y = y * fma(-0.5 * m, y * y, 1.5);
  return ldexp(y, -e / 2);
}

// Flag words (reset at the start of every QR):
//   flags[0] done:      no further pass is needed (read by the Gram GEMM and
//                       this kernel at the start of every later pass)
//   flags[1] skip_trmm: the S <- S R^{-1} launch of this pass is a no-op
//   flags[2] passes applied, flags[3] shifted passes (diagnostics)
__global__ void __launch_bounds__(kCholThreads)
chol_inv_kernel(const double *Gg, double *Rinv_g, int c, int m, int *flags) {
  if (flags[0]) {
    if (threadIdx.x == 0) flags[1] = 1;
    return;
  }
  extern __shared__ double sm[];
  const int ld = c + 1;
  double *G = sm;                                   // c x ld, upper triangle becomes R
  const bool inv_in_smem = chol_smem_doubles(c, true) * sizeof(double) <= kCholSmemMax;
  double *Ri = inv_in_smem ? sm + c * ld : Rinv_g;  // R^{-1}, ld = c
  __shared__ double s_diag_max, s_trace, s_dev;
  __shared__ double s_rinv[kMaxSmall];              // 1 / R_jj
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;           // 16 x 16 grid (kCholThreads = 256)

  // -- convergence test: G = I to working accuracy, except columns that are
  // exactly zero (a zero column stays zero through every pass). The test is
  // absolute on purpose: S of any scale (HaTT sketches of long chains reach
  // 1e-20 and below) is never mistaken for a converged basis.
  double dev = 0.0, dmax = 0.0, tr = 0.0;
  for (int e = tid; e < c * c; e += kCholThreads) {
    const int i = e / c, j = e % c;
    const double v = Gg[e];
    G[i * ld + j] = v;
    if (i == j) {
      dmax = fmax(dmax, v);
      tr += v;
      dev = fmax(dev, (v == 0.0) ? 0.0 : fabs(v - 1.0));
    } else {
      dev = fmax(dev, fabs(v));
    }
  }
  {
    __shared__ double red[kCholThreads];
    red[tid] = dev;
    __syncthreads();
    for (int w = kCholThreads / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
      __syncthreads();
    }
    if (tid == 0) s_dev = red[0];
    __syncthreads();
    red[tid] = dmax;
    __syncthreads();
    for (int w = kCholThreads / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
      __syncthreads();
    }
    if (tid == 0) s_diag_max = red[0];
    __syncthreads();
    red[tid] = tr;
    __syncthreads();
    for (int w = kCholThreads / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) s_trace = red[0];
    __syncthreads();
  }
  const double u = 1.1102230246251565e-16;
  if (s_dev <= 8.0 * c * u) {              // already orthonormal: nothing to apply
    if (tid == 0) { flags[0] = 1; flags[1] = 1; }
    return;
  }
  if (tid == 0) {
    flags[1] = 0;
    flags[2] += 1;
    // ||G - I||_max <= 0.1/c puts every eigenvalue of G in [0.9, 1.1]
    // (Gerschgorin): one more Cholesky QR pass orthonormalizes to working
    // accuracy, so this pass is the last one
    if (s_dev <= 0.1 / c) flags[0] = 1;
  }

  // -- Cholesky: first unshifted, then shifted if a pivot is not safely positive
  for (int attempt = 0; attempt < 2; ++attempt) {
    double shift = 0.0;
    if (attempt == 1) {
      shift = 11.0 * ((double)m * c + (double)c * (c + 1)) * u * s_trace;
      if (!(shift > 0.0)) shift = 1e-300;
      for (int e = tid; e < c * c; e += kCholThreads) {
        const int i = e / c, j = e % c;
        G[i * ld + j] = Gg[e] + (i == j ? shift : 0.0);
      }
      if (tid == 0) flags[3] += 1;
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    const double floor_piv = (attempt == 0) ? (double)c * u * s_diag_max : 0.0;
    for (int j = 0; j < c; ++j) {
      if (tid == 0) {
        double piv = G[j * ld + j];
        if (!(piv > floor_piv)) {
          if (attempt == 0) s_fail = 1;
          piv = fmax(shift, 1e-300);          // shifted attempt: never divide by zero
        }
        const double y = rsqrt_newton(piv);
        G[j * ld + j] = piv * y;              // R_jj = sqrt(piv)
        s_rinv[j] = y;
      }
      __syncthreads();
      if (s_fail) break;
      const double yj = s_rinv[j];
      for (int l = j + 1 + tid; l < c; l += kCholThreads) G[j * ld + l] *= yj;
      __syncthreads();
      // trailing update of the upper triangle on a 16 x 16 thread grid
      for (int i = j + 1 + ty; i < c; i += 16) {
        const double rji = G[j * ld + i];
        for (int l = i + tx; l < c; l += 16) G[i * ld + l] = fma(-rji, G[j * ld + l], G[i * ld + l]);
      }
      __syncthreads();
    }
    __syncthreads();
    if (!s_fail) break;
  }

  // -- triangular inverse, row by row from the bottom: Ri[i][j], j >= i.
  // One warp per entry: the lanes split the dot product sum_l R_il Ri_lj and
  // reduce with shuffles, so a row costs a few shuffle rounds instead of a
  // dependent chain of up to c FP64 multiply-adds.
  for (int e = tid; e < c * c; e += kCholThreads) {
    const int i = e / c, j = e % c;
    if (j < i) Ri[e] = 0.0;
  }
  const int warp = tid >> 5, lane = tid & 31;
  for (int i = c - 1; i >= 0; --i) {
    const double yi = s_rinv[i];
    for (int j = i + warp; j < c; j += kCholThreads / 32) {
      double s = 0.0;
      for (int l = i + 1 + lane; l <= j; l += 32) s = fma(G[i * ld + l], Ri[l * c + j], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) Ri[i * c + j] = ((j == i) ? 1.0 - s : -s) * yi;
    }
    __syncthreads();
  }
  if (inv_in_smem)
    for (int e = tid; e < c * c; e += kCholThreads) Rinv_g[e] = Ri[e];
}

// S[r][j] <- sum_{i <= j} S[r][i] Rinv[i][j], rows owned by one block (in place).
__global__ void __launch_bounds__(kTrmmThreads)
trmm_rows_kernel(double *S, int m, int c, long long ldS, const double *Rinv, const int *flags) {
  if (flags[1]) return;
  extern __shared__ double sm[];
  double *Rs = sm;                       // c x c
  double *Xs = sm + c * c;               // kTrmmRows x c
  const int r0 = blockIdx.x * kTrmmRows;
  const int rows = min(kTrmmRows, m - r0);
  for (int e = threadIdx.x; e < c * c; e += kTrmmThreads) Rs[e] = Rinv[e];
  for (int e = threadIdx.x; e < rows * c; e += kTrmmThreads) {
    const int r = e / c, j = e % c;
    Xs[r * c + j] = S[(long long)(r0 + r) * ldS + j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * c; e += kTrmmThreads) {
    const int r = e / c, j = e % c;
    double s = 0.0;
    for (int i = 0; i <= j; ++i) s = fma(Xs[r * c + i], Rs[i * c + j], s);
    S[(long long)(r0 + r) * ldS + j] = s;
  }
}

size_t chol_smem(int c) {
  const size_t with_inv = chol_smem_doubles(c, true) * sizeof(double);
  return with_inv <= kCholSmemMax ? with_inv : chol_smem_doubles(c, false) * sizeof(double);
}
size_t trmm_smem(int c) { return (size_t)(c * c + kTrmmRows * c) * sizeof(double); }

Gemm gram_desc(double *S, int m, int c, long long ldS, double *G, const int *flags) {
  Gemm g;
  g.M = c; g.N = c; g.K = m;
  g.A = S; g.sAm = 1; g.sAk = ldS;       // A(i, k) = S[k][i]
  g.B = S; g.sBk = ldS; g.sBn = 1;       // B(k, j) = S[k][j]
  g.C = G; g.sCm = c; g.sCn = 1;
  g.skip_dev = flags;
  return g;
}

}  // namespace

size_t qr_scratch_doubles(int m, int c) {
  Gemm g = gram_desc(nullptr, m, c, c, nullptr, nullptr);
  return (size_t)2 * c * c + gemm_scratch_doubles(g);
}

cudaError_t qr_inplace(double *S, int m, int c, long long ldS, double *scratch, int *flags,
                       cudaStream_t st) {
  if (c <= 0 || m <= 0) return cudaSuccess;
  if (c > kMaxSmall) return cudaErrorInvalidValue;
  double *G = scratch;
  double *Rinv = scratch + (size_t)c * c;
  double *gs = scratch + (size_t)2 * c * c;
  cudaError_t e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kCholSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(trmm_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trmm_smem(kMaxSmall));
  if (e != cudaSuccess) return e;
  const Gemm gd = gram_desc(S, m, c, ldS, G, flags);
  const int blocks = (m + kTrmmRows - 1) / kTrmmRows;
  for (int p = 0; p < kPasses; ++p) {
    e = gemm_f64(gd, gs, st);
    if (e != cudaSuccess) return e;
    chol_inv_kernel<<<1, kCholThreads, chol_smem(c), st>>>(G, Rinv, c, m, flags);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    trmm_rows_kernel<<<blocks, kTrmmThreads, trmm_smem(c), st>>>(S, m, c, ldS, Rinv, flags);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hatt
