// Economy QR of the tall sketch S = C_k W^{(k)} (Algorithm 4) on GB300.
//
// Householder QR is a chain of rank-1 updates and would run on one SM at the
// FP64 rate of a single SM (~8 GFLOP/s on GB300). Cholesky QR instead spends
// almost all of its flops in two SM-parallel steps (the Gram S^T S, and
// S R^{-1} as a forward substitution with one warp per row of S); only the
// c x c Cholesky factorization runs in one block. A pass is
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
// An S of exactly lower rank than c (a raw TT representation, a sketch of an
// exact low-rank product) has null directions at the rounding level, ~u ||S||.
// Each shifted pass multiplies them by about 1/sqrt(s / ||S||^2), i.e. by 1e4
// to 1e6 for the sizes here, so they need four shifted passes to reach unit
// size and then one or two plain ones: six passes in all. Stopping earlier
// leaves Q far from orthonormal, and the projection Q Q^T C of the callers
// then loses about 1e-9 of C.
//
// All passes are launched unconditionally (fixed launch sequence, capturable
// in a CUDA graph); a device flag set by the convergence test turns the
// remaining launches into no-ops.
#include <algorithm>
#include "hatt_internal.cuh"

namespace hatt {
namespace {

__device__ int g_qr_health = 0;   // kHealthNonfinite / kHealthBreakdown bits

constexpr int kPasses = 6;
constexpr int kCholThreads = 256;
constexpr int kTrsmThreads = 256;

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
//   flags[1] skip_apply: the S <- S R^{-1} launch of this pass is a no-op
//   flags[2] passes applied, flags[3] shifted passes (diagnostics)
__global__ void __launch_bounds__(kCholThreads)
chol_inv_kernel(const double *Gg, double *Ut_g, double *y_g, int c, int m, int *flags) {
  pdl_enter();
  if (flags[0]) {
    if (threadIdx.x == 0) flags[1] = 1;
    return;
  }
  extern __shared__ double sm[];
  const int ld = c + 1;
  double *G = sm;                                   // c x ld, upper triangle becomes R
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
  int bad = 0;
  for (int e = tid; e < c * c; e += kCholThreads) {
    const int i = e / c, j = e % c;
    const double v = Gg[e];
    bad |= !isfinite(v);
    G[i * ld + j] = v;
    if (i == j) {
      dmax = fmax(dmax, v);
      tr += v;
      dev = fmax(dev, (v == 0.0) ? 0.0 : fabs(v - 1.0));
    } else {
      dev = fmax(dev, fabs(v));
    }
  }
  // a non-finite Gram matrix (a non-finite input core or intermediate): record
  // it, leave S as it is and stop this QR (every later pass is a no-op)
  if (__syncthreads_or(bad)) {
    if (tid == 0) {
      atomicOr(&g_qr_health, kHealthNonfinite);
      flags[0] = 1;
      flags[1] = 1;
    }
    return;
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
        if (Gg[j * c + j] == 0.0) {
          // an exactly zero column of S: its Gram row and column vanish, so
          // R_jj = 1 leaves Q_j = 0 and couples nothing. Sending it to the
          // shifted attempt instead would make every pass shifted and leave
          // ||Q^T Q - I|| at the shift (~1e-11) on an otherwise benign S.
          piv = 1.0;
        } else if (!(piv > floor_piv)) {
          if (attempt == 0) s_fail = 1;
          else atomicOr(&g_qr_health, kHealthBreakdown);   // shifted and still not positive
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

  // -- publish R = D U~ as the unit upper triangle U~ (U~_jl = R_jl / R_jj)
  // and y_j = 1 / R_jj; the apply kernel solves with them, so no serial
  // triangular inverse is formed in this single block
  for (int i = ty; i < c; i += 16)
    for (int l = tx; l < c; l += 16)
      Ut_g[i * c + l] = (l > i) ? G[i * ld + l] * s_rinv[i] : (l == i ? 1.0 : 0.0);
  for (int i = tid; i < c; i += kCholThreads) y_g[i] = s_rinv[i];
}

// Q = S R^{-1} = (S U~^{-1}) D^{-1}, one warp per row, in place. Lane t holds
// columns t, t+32, t+64, t+96 of the row; step l broadcasts the finished x_l
// and every lane updates its later columns (x_j -= x_l U~_lj). The unit
// diagonal keeps divisions out of the chain; the final scaling by y = D^{-1}
// is one multiply per entry.
__global__ void __launch_bounds__(kTrsmThreads)
trsm_rows_kernel(double *S, int m, int c, long long ldS, const double *Ut, const double *y,
                 const int *flags) {
  pdl_enter();
  if (flags[1]) return;
  extern __shared__ double sm[];
  double *Us = sm;                       // c x c
  double *ys = sm + c * c;               // c
  for (int e = threadIdx.x; e < c * c; e += kTrsmThreads) Us[e] = Ut[e];
  for (int e = threadIdx.x; e < c; e += kTrsmThreads) ys[e] = y[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = kTrsmThreads / 32;
  for (int r = blockIdx.x * warps + (threadIdx.x >> 5); r < m; r += gridDim.x * warps) {
    double *row = S + (long long)r * ldS;
    double x0 = lane < c ? row[lane] : 0.0;
    double x1 = lane + 32 < c ? row[lane + 32] : 0.0;
    double x2 = lane + 64 < c ? row[lane + 64] : 0.0;
    double x3 = lane + 96 < c ? row[lane + 96] : 0.0;
    for (int l = 0; l < c; ++l) {
      const int slot = l >> 5;
      const double own = slot == 0 ? x0 : slot == 1 ? x1 : slot == 2 ? x2 : x3;
      const double xl = __shfl_sync(0xffffffffu, own, l & 31);
      const double *u = Us + l * c;
      if (lane > l && lane < c) x0 = fma(-xl, u[lane], x0);
      if (lane + 32 > l && lane + 32 < c) x1 = fma(-xl, u[lane + 32], x1);
      if (c > 64 && lane + 64 > l && lane + 64 < c) x2 = fma(-xl, u[lane + 64], x2);
      if (c > 96 && lane + 96 > l && lane + 96 < c) x3 = fma(-xl, u[lane + 96], x3);
    }
    if (lane < c) row[lane] = x0 * ys[lane];
    if (lane + 32 < c) row[lane + 32] = x1 * ys[lane + 32];
    if (lane + 64 < c) row[lane + 64] = x2 * ys[lane + 64];
    if (lane + 96 < c) row[lane + 96] = x3 * ys[lane + 96];
  }
}

size_t chol_smem(int c) { return (size_t)c * (c + 1) * sizeof(double); }
size_t trsm_smem(int c) { return (size_t)(c * c + c) * sizeof(double); }

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

cudaError_t qr_health_word(int *value, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_qr_health, sizeof(int));
  if (e == cudaSuccess && clear && *value != 0) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_qr_health, &zero, sizeof(int));
  }
  return e;
}

size_t qr_scratch_doubles(int m, int c) {
  Gemm g = gram_desc(nullptr, m, c, c, nullptr, nullptr);
  return (size_t)2 * c * c + c + gemm_scratch_doubles(g);
}

cudaError_t qr_inplace(double *S, int m, int c, long long ldS, double *scratch, int *flags,
                       cudaStream_t st) {
  if (c <= 0 || m <= 0) return cudaSuccess;
  if (c > kMaxSmall) return cudaErrorInvalidValue;
  double *G = scratch;
  double *Ut = scratch + (size_t)c * c;
  double *y = scratch + (size_t)2 * c * c;
  double *gs = scratch + (size_t)2 * c * c + c;
  cudaError_t e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)chol_smem(kMaxSmall));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(trsm_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsm_smem(kMaxSmall));
  if (e != cudaSuccess) return e;
  const Gemm gd = gram_desc(S, m, c, ldS, G, flags);
  const int blocks = std::max(1, std::min((m + kTrsmThreads / 32 - 1) / (kTrsmThreads / 32), 2 * 152));
  for (int p = 0; p < kPasses; ++p) {
    e = gemm_f64(gd, gs, st);
    if (e != cudaSuccess) return e;
    launch_k(chol_inv_kernel, 1, kCholThreads, chol_smem(c), st, G, Ut, y, c, m, flags);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    launch_k(trsm_rows_kernel, blocks, kTrsmThreads, trsm_smem(c), st, S, m, c, ldS, Ut, y, flags);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hatt
