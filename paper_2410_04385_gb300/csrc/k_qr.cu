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

// 1/sqrt(x) for x in [1e-30, 1e30] (a pivot pre-scaled by an even power of
// two): the FP32 seed and the same two Newton-Raphson steps as rsqrt_newton,
// without its range reduction. On GB300 a dependent FP64 instruction costs
// ~64 clocks and frexp / ldexp are long sequences: measured 1447 clocks for
// rsqrt_newton against ~450 for this, on the critical path of every column.
__device__ __forceinline__ double rsqrt_scaled(double x) {
  const double h = -0.5 * x;
  double y = (double)rsqrtf((float)x);
  y = y * fma(h, y * y, 1.5);
  y = y * fma(h, y * y, 1.5);
  return y;
}

// Warp reduction of the three convergence statistics; lane 0 holds the
// result. dev and dmax are maxima of non-negative doubles, taken on their bit
// patterns (integer order equals numeric order there), which keeps them off
// the FP64 unit.
__device__ __forceinline__ void warp_stats(long long &dev, long long &dmax, double &tr) {
  for (int o = 16; o > 0; o >>= 1) {
    dev = max(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
  }
}

// Pivot step of column j (thread 0 only): R_jj = sqrt(pivot) as y_j = 1/R_jj.
// An exactly zero column of S (zero Gram diagonal) gets R_jj = 1, which
// leaves Q_j = 0 and couples nothing; sending it to the shifted attempt
// instead would make every pass shifted and leave ||Q^T Q - I|| at the shift
// (~1e-11) on an otherwise benign S. A pivot not safely positive fails the
// unshifted attempt; in the shifted attempt it sets the breakdown bit and is
// clamped so that nothing divides by zero.
// sc = 2^-2k and unsc = 2^-k put the largest Gram diagonal near 1, so every
// pivot above the failure floor is a normal FP32 number once scaled.
__device__ __forceinline__ void chol_pivot(double *G, int ld, int j, const unsigned char *zero_col,
                                           double floor_piv, double shift, int attempt, double sc,
                                           double unsc, double *rinv, unsigned char *fail) {
  if (zero_col[j]) {
    rinv[j] = 1.0;
    return;
  }
  double piv = G[j * ld + j];
  if (!(piv > floor_piv)) {
    if (attempt == 0) fail[j] = 1;
    else atomicOr(&g_qr_health, kHealthBreakdown);
    piv = fmax(shift, 1e-300);
  }
  const double ps = piv * sc;
  rinv[j] = (ps >= 1e-30 && ps <= 1e30) ? rsqrt_scaled(ps) * unsc : rsqrt_newton(piv);
}

// Flag words (reset at the start of every QR):
//   flags[0] done:      no further pass is needed (read by the Gram GEMM and
//                       this kernel at the start of every later pass)
//   flags[1] skip_apply: the S <- S R^{-1} launch of this pass is a no-op
//   flags[2] passes applied, flags[3] shifted passes (diagnostics)
//
// One block: convergence test of G = S^T S, then the Cholesky factor R of G
// (shifted if the plain factorization breaks down), published as the unit
// upper triangle U~ = D^{-1} R and y = diag(D^{-1}), D = diag(R).
//
// Right-looking factorization with a one-column look-ahead: during the
// trailing update for column j, warp 0 first updates row j + 1 and thread 0
// takes the pivot of column j + 1 (the only serial step of the next column)
// while the other warps update the rest, so each column costs one barrier and
// the pivot's dependent FP64 chain overlaps the bulk of the update. Rows of R
// are not scaled in place: the update subtracts (G_ji y_j^2) G_jl, and the
// publication scales row j by y_j^2.
__global__ void __launch_bounds__(kCholThreads)
chol_inv_kernel(const double *Gg, double *Ut_g, double *y_g, int c, int m, int *flags) {
  pdl_enter();
  if (flags[0]) {
    if (threadIdx.x == 0) flags[1] = 1;
    return;
  }
  extern __shared__ double sm[];
  const int ld = c + 1;
  double *G = sm;                                   // c x ld, upper triangle is updated
  __shared__ double s_red[3][kCholThreads / 32];
  __shared__ double s_diag_max, s_trace, s_dev, s_sc, s_unsc;
  __shared__ double s_rinv[kMaxSmall];              // 1 / R_jj
  __shared__ unsigned char s_zero[kMaxSmall];       // column j of S is exactly zero
  __shared__ unsigned char s_failc[kMaxSmall];      // unshifted pivot j not safely positive
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tx = tid % 16, ty = tid / 16;           // 16 x 16 grid (kCholThreads = 256)

  // -- convergence test: G = I to working accuracy, except columns that are
  // exactly zero (a zero column stays zero through every pass). The test is
  // absolute on purpose: S of any scale (HaTT sketches of long chains reach
  // 1e-20 and below) is never mistaken for a converged basis.
  long long dev = 0, dmax = 0;          // bit patterns of non-negative doubles
  double tr = 0.0;
  int bad = 0;
  const int n = c * c;
  // entry e = i c + j of thread tid: (i, j) advanced by (di, dj) per step of
  // kCholThreads entries, with a carry, instead of a division per entry
  const int di = kCholThreads / c, dj = kCholThreads - (kCholThreads / c) * c;
  int ii = tid / c, jj = tid - (tid / c) * c;
  for (int e0 = tid; e0 < n; e0 += 4 * kCholThreads) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {         // four loads in flight per thread
      const int e = e0 + q * kCholThreads;
      v[q] = e < n ? Gg[e] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = e0 + q * kCholThreads;
      if (e >= n) break;
      const int i = ii, j = jj;
      ii += di;
      jj += dj;
      if (jj >= c) {
        jj -= c;
        ++ii;
      }
      const long long bits = __double_as_longlong(fabs(v[q]));
      bad |= bits >= 0x7ff0000000000000LL;                   // Inf or NaN
      G[i * ld + j] = v[q];
      if (i == j) {
        s_zero[i] = (v[q] == 0.0);
        dmax = max(dmax, bits);
        tr += v[q];
        if (v[q] != 0.0) dev = max(dev, __double_as_longlong(fabs(v[q] - 1.0)));
      } else {
        dev = max(dev, bits);
      }
    }
  }
  warp_stats(dev, dmax, tr);
  if (lane == 0) {
    s_red[0][warp] = __longlong_as_double(dev);
    s_red[1][warp] = __longlong_as_double(dmax);
    s_red[2][warp] = tr;
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
  if (tid == 0) {
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    for (int w = 0; w < kCholThreads / 32; ++w) {
      d0 = fmax(d0, s_red[0][w]);
      d1 = fmax(d1, s_red[1][w]);
      d2 += s_red[2][w];
    }
    s_dev = d0;
    s_diag_max = d1;
    s_trace = d2;
    // pivot scaling 2^-2k with the largest diagonal in [0.5, 2) after scaling;
    // the exponent is read off the bits (frexp / ldexp are long sequences on
    // this chain), with frexp / ldexp kept for subnormal or extreme values
    const long long bits = __double_as_longlong(d1);
    const int be = (int)((bits >> 52) & 0x7ff);
    int ex = 0;
    if (be > 0) ex = be - 1022;                 // d1 = m 2^ex, m in [0.5, 1)
    else if (d1 > 0.0) frexp(d1, &ex);
    const int k = ex / 2;
    s_sc = (-2 * k + 1023 >= 1 && -2 * k + 1023 <= 2046)
               ? __longlong_as_double((long long)(-2 * k + 1023) << 52) : ldexp(1.0, -2 * k);
    s_unsc = (-k + 1023 >= 1 && -k + 1023 <= 2046)
                 ? __longlong_as_double((long long)(-k + 1023) << 52) : ldexp(1.0, -k);
  }
  __syncthreads();
  const double u = 1.1102230246251565e-16;
  const double sc = s_sc, unsc = s_unsc;
  if (s_dev <= 8.0 * c * u) {              // already orthonormal: nothing to apply
    if (tid == 0) { flags[0] = 1; flags[1] = 1; }
    return;
  }

  // -- Cholesky: first unshifted, then shifted if a pivot is not safely positive.
  // A failed pivot of column j is recorded in s_failc[j] while column j - 1
  // is updated and read by every thread after that column's barrier, so all
  // threads leave the column loop at the same j.
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
    for (int j = tid; j < c; j += kCholThreads) s_failc[j] = 0;
    __syncthreads();
    const double floor_piv = (attempt == 0) ? (double)c * u * s_diag_max : 0.0;
    if (tid == 0) chol_pivot(G, ld, 0, s_zero, floor_piv, shift, attempt, sc, unsc, s_rinv, s_failc);
    __syncthreads();
    bool failed = false;
    for (int j = 0; j < c; ++j) {
      if (s_failc[j]) {
        failed = true;
        break;
      }
      const double yj = s_rinv[j];
      const double y2 = yj * yj;
      const double *rowj = G + j * ld;
      if (warp == 0 && j + 1 < c) {       // look-ahead: row j + 1, then its pivot
        const int i = j + 1;
        const double rji = rowj[i] * y2;
        for (int l = i + lane; l < c; l += 32) G[i * ld + l] = fma(-rji, rowj[l], G[i * ld + l]);
        __syncwarp();
        if (lane == 0) chol_pivot(G, ld, i, s_zero, floor_piv, shift, attempt, sc, unsc, s_rinv, s_failc);
      }
      // trailing update of the rows below by warps 1..7 on a 14 x 16 grid:
      // warp 0 carries the pivot chain and takes no share of it
      if (warp > 0) {
        const int bt = tid - 32, bx = bt % 16, by = bt / 16;
        for (int i = j + 2 + by; i < c; i += 14) {
          const double rji = rowj[i] * y2;
          for (int l = i + bx; l < c; l += 16) G[i * ld + l] = fma(-rji, rowj[l], G[i * ld + l]);
        }
      }
      __syncthreads();
    }
    if (!failed) break;
    __syncthreads();                      // all reads of G and s_failc done before the retry
  }

  // -- publish R = D U~ as the unit upper triangle U~ (U~_jl = R_jl / R_jj =
  // G_jl y_j^2 with G the updated Gram row) and y_j = 1 / R_jj; the apply
  // kernel solves with them, so no serial triangular inverse is formed in
  // this single block
  for (int i = ty; i < c; i += 16) {
    const double yi2 = s_rinv[i] * s_rinv[i];
    for (int l = tx; l < c; l += 16)
      Ut_g[i * c + l] = (l > i) ? G[i * ld + l] * yi2 : (l == i ? 1.0 : 0.0);
  }
  for (int i = tid; i < c; i += kCholThreads) y_g[i] = s_rinv[i];
  // this pass applies; ||G - I||_max <= 0.1/c puts every eigenvalue of G in
  // [0.9, 1.1] (Gerschgorin): one more Cholesky QR pass orthonormalizes to
  // working accuracy, so this pass is the last one. Written last: the
  // read-modify-write would otherwise sit on the first pivot's path.
  if (tid == 0) {
    flags[1] = 0;
    flags[2] += 1;
    if (s_dev <= 0.1 / c) flags[0] = 1;
  }
}

// Q = S R^{-1} = (S U~^{-1}) D^{-1}, one warp per row, in place. The unit
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
  const int ns = (c + 31) / 32;          // column slots in use (c <= 128)
  for (int r = blockIdx.x * warps + (threadIdx.x >> 5); r < m; r += gridDim.x * warps) {
    double *row = S + (long long)r * ldS;
    double x[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) x[s] = (s < ns && lane + 32 * s < c) ? row[lane + 32 * s] : 0.0;
    switch (ns) {
      case 1: trsm_row<1>(x, Us, c, lane); break;
      case 2: trsm_row<2>(x, Us, c, lane); break;
      case 3: trsm_row<3>(x, Us, c, lane); break;
      default: trsm_row<4>(x, Us, c, lane); break;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int col = lane + 32 * s;
      if (s < ns && col < c) row[col] = x[s] * ys[col];
    }
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
