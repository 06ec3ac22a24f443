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
// Two launch forms, the same passes:
//  * fused (qr_fused_kernel): all passes in one cooperative launch, one block
//    per SM, each block owning a contiguous slice of the rows of S. Grid
//    barriers separate the Gram partial sums, their reduction, the
//    factorization (block 0) and the apply; a converged QR stops at once, so
//    no launch and no no-op pass follows the convergence test. Used on
//    calls whose stream runs alone (single recompressions, rounding);
//  * launch per step: per pass the Gram shares, their sum, the
//    factorization and the apply, all passes launched unconditionally (fixed
//    launch sequence); a device flag set by the convergence test turns the
//    remaining launches into no-ops. Used by the batched entry point, whose
//    many streams would serialize on whole-GPU cooperative grids.
// Both run the same device code on the same row partition, so they give
// bitwise the same Q; both are capturable in a CUDA graph.
#include <algorithm>
#include <cstdlib>
#include <cstring>
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

// 1/x for x in [1e-30, 1e30] (a pivot pre-scaled by an even power of two):
// an FP32 reciprocal seed (rcp.approx, relative error below 2^-22), then two
// Newton-Raphson steps r <- r + r (1 - x r) in FP64, each two fused
// multiply-adds (the error squares per step: 2^-22 -> 2^-44 -> FP64
// rounding). Two dependent FP64 instructions fewer than rsqrt_scaled, and its
// result is the multiplier 1/R_jj^2 the trailing update uses directly.
__device__ __forceinline__ double rcp_scaled(double x) {
  float f;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"((float)x));
  double r = (double)f;
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
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

// Pivot step of column j (thread 0 only): R_jj = sqrt(pivot), stored as
// rinv2_j = 1/pivot, the multiplier of the trailing update, and the pivot
// itself; 1/R_jj is formed at publication, for all j at once and off the
// column chain. An exactly zero column of S (zero Gram diagonal) gets R_jj = 1,
// which leaves Q_j = 0 and couples nothing; sending it to the shifted attempt
// instead would make every pass shifted and leave ||Q^T Q - I|| at the shift
// (~1e-11) on an otherwise benign S. A pivot not safely positive fails the
// unshifted attempt; in the shifted attempt it sets the breakdown bit and is
// clamped so that nothing divides by zero.
// G is factorized scaled by sc = 2^-2k, which puts the largest Gram diagonal
// near 1 (exact: a power of two), so every pivot above the failure floor is a
// normal FP32 number and the chain carries no scaling; floor_piv and clamp
// (the value a failed pivot takes) are scaled alike.
__device__ __forceinline__ void chol_pivot(double *G, int ld, int j, const unsigned char *zero_col,
                                           double floor_piv, double clamp, int attempt,
                                           double *rinv2, double *pivots, unsigned char *fail) {
  if (zero_col[j]) {
    rinv2[j] = 1.0;
    pivots[j] = 1.0;
    return;
  }
  double piv = G[j * ld + j];
  if (!(piv > floor_piv)) {
    if (attempt == 0) fail[j] = 1;
    else atomicOr(&g_qr_health, kHealthBreakdown);
    piv = clamp;
  }
  pivots[j] = piv;
  rinv2[j] = (piv >= 1e-30 && piv <= 1e30) ? rcp_scaled(piv) : 1.0 / piv;
}

// Flag words (reset at the start of every QR):
//   flags[0] done:      no further pass is needed (read by the Gram GEMM and
//                       this kernel at the start of every later pass)
//   flags[1] skip_apply: the S <- S R^{-1} step of this pass is a no-op
//   flags[2] passes applied, flags[3] shifted passes (diagnostics)
//   flags[4] grid-barrier arrivals, flags[5] abort (fused form only)
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
// publication scales row j by y_j^2. G is read through L2 (__ldcg): in the
// fused form other blocks of the same launch wrote it.
__device__ __forceinline__ void chol_factor(const double *Gg, double *Ut_g, double *y_g, int c,
                                            int m, int *flags, double *sm) {
  const int ld = c + 1;
  double *G = sm;                                   // c x ld, upper triangle is updated
  __shared__ double s_red[3][kCholThreads / 32];
  __shared__ double s_diag_max, s_trace, s_dev, s_sc, s_unsc;
  __shared__ double s_rinv2[kMaxSmall];             // 1 / (sc R_jj^2)
  __shared__ double s_piv[kMaxSmall];               // sc R_jj^2 (the scaled pivot)
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
      v[q] = e < n ? __ldcg(Gg + e) : 0.0;
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
  for (int i = ty; i < c; i += 16)         // the factorization runs on sc G
    for (int j = tx; j < c; j += 16) G[i * ld + j] *= sc;

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
        G[i * ld + j] = (__ldcg(Gg + e) + (i == j ? shift : 0.0)) * sc;
      }
      if (tid == 0) flags[3] += 1;
    }
    for (int j = tid; j < c; j += kCholThreads) s_failc[j] = 0;
    __syncthreads();
    const double floor_piv = (attempt == 0) ? (double)c * u * s_diag_max * sc : 0.0;
    const double clamp = fmax(shift, 1e-300) * sc;
    if (tid == 0) chol_pivot(G, ld, 0, s_zero, floor_piv, clamp, attempt, s_rinv2, s_piv, s_failc);
    __syncthreads();
    bool failed = false;
    for (int j = 0; j < c; ++j) {
      if (s_failc[j]) {
        failed = true;
        break;
      }
      const double y2 = s_rinv2[j];
      const double *rowj = G + j * ld;
      if (warp == 0 && j + 1 < c) {       // look-ahead: row j + 1, then its pivot
        const int i = j + 1;
        const double rji = rowj[i] * y2;
        for (int l = i + lane; l < c; l += 32) G[i * ld + l] = fma(-rji, rowj[l], G[i * ld + l]);
        __syncwarp();
        if (lane == 0) chol_pivot(G, ld, i, s_zero, floor_piv, clamp, attempt, s_rinv2, s_piv, s_failc);
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
  // G_jl / G_jj with G the updated, scaled Gram row: the scale cancels) and
  // y_j = 1 / R_jj; the apply
  // kernel solves with them, so no serial triangular inverse is formed in
  // this single block
  for (int i = ty; i < c; i += 16) {
    const double yi2 = s_rinv2[i];
    for (int l = tx; l < c; l += 16)
      Ut_g[i * c + l] = (l > i) ? G[i * ld + l] * yi2 : (l == i ? 1.0 : 0.0);
  }
  for (int i = tid; i < c; i += kCholThreads) {
    double yi = 1.0;                      // 1 / R_ii (1 for an exactly zero column)
    if (!s_zero[i]) {                     // the pivot is sc R_ii^2, sc = unsc^2
      const double ps = s_piv[i];
      yi = ((ps >= 1e-30 && ps <= 1e30) ? rsqrt_scaled(ps) : rsqrt_newton(ps)) * unsc;
    }
    y_g[i] = yi;
  }
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

__global__ void __launch_bounds__(kCholThreads)
chol_inv_kernel(const double *Gg, double *Ut_g, double *y_g, int c, int m, int *flags) {
  pdl_enter();
  if (flags[0]) {
    if (threadIdx.x == 0) flags[1] = 1;
    return;
  }
  extern __shared__ double sm[];
  chol_factor(Gg, Ut_g, y_g, c, m, flags, sm);
}

// Q = S R^{-1} = (S U~^{-1}) D^{-1}, one warp per row, in place. The unit
// diagonal keeps divisions out of the chain; the final scaling by y = D^{-1}
// is one multiply per entry. Rows r_first, r_first + r_step, ... < r_end of
// this warp; U~ (Us) and y (ys) in shared memory.
// Two rows at once, their chains interleaved (the same operations on each
// row as trsm_row, so a row's result does not depend on its partner).
template <int NS>
__device__ __forceinline__ void trsm_row2(double (&x)[4], double (&z)[4], const double *Us, int c,
                                          int lane) {
#pragma unroll
  for (int s0 = 0; s0 < NS; ++s0) {
    const int lend = min(c, 32 * (s0 + 1));
    for (int l = 32 * s0; l < lend; ++l) {
      const double xl = __shfl_sync(0xffffffffu, x[s0], l & 31);
      const double zl = __shfl_sync(0xffffffffu, z[s0], l & 31);
      const double *u = Us + l * c;
#pragma unroll
      for (int s = s0; s < NS; ++s) {
        const int col = lane + 32 * s;
        if (col > l && col < c) {
          const double uv = u[col];
          x[s] = fma(-xl, uv, x[s]);
          z[s] = fma(-zl, uv, z[s]);
        }
      }
    }
  }
}

__device__ __forceinline__ void apply_rows(double *S, long long ldS, int c, const double *Us,
                                           const double *ys, int r_first, int r_end, int r_step) {
  const int lane = threadIdx.x & 31;
  const int ns = (c + 31) / 32;          // column slots in use (c <= 128)
  for (int r = r_first; r < r_end; r += 2 * r_step) {
    double *row = S + (long long)r * ldS;
    double *row2 = S + (long long)(r + r_step) * ldS;
    const bool two = r + r_step < r_end;   // the warp's next row: solved alongside
    double x[4], z[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const bool in = s < ns && lane + 32 * s < c;
      x[s] = in ? row[lane + 32 * s] : 0.0;
      z[s] = (in && two) ? row2[lane + 32 * s] : 0.0;
    }
    if (two) {
      switch (ns) {
        case 1: trsm_row2<1>(x, z, Us, c, lane); break;
        case 2: trsm_row2<2>(x, z, Us, c, lane); break;
        case 3: trsm_row2<3>(x, z, Us, c, lane); break;
        default: trsm_row2<4>(x, z, Us, c, lane); break;
      }
    } else {
      switch (ns) {
        case 1: trsm_row<1>(x, Us, c, lane); break;
        case 2: trsm_row<2>(x, Us, c, lane); break;
        case 3: trsm_row<3>(x, Us, c, lane); break;
        default: trsm_row<4>(x, Us, c, lane); break;
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int col = lane + 32 * s;
      if (s < ns && col < c) {
        row[col] = x[s] * ys[col];
        if (two) row2[col] = z[s] * ys[col];
      }
    }
  }
}

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
  const int warps = kTrsmThreads / 32;
  apply_rows(S, ldS, c, Us, ys, blockIdx.x * warps + (threadIdx.x >> 5), m, gridDim.x * warps);
}

// ------------------------------------------------------- the Gram matrix ---
// G = S^T S from per-block shares: block b of nb sums the rows [b p, b p + p)
// of S, p = ceil(m / nb), into the upper triangle (i <= j, c (c + 1) / 2
// entries) of its own share, and a warp then sums each entry over the nb
// shares. Both forms of the QR run these same device functions with the
// same nb (qr_blocks), so they compute bitwise the same G, and the same QR.
constexpr int kQrMaxBlocks = 160;       // >= the SMs of the device (152 on GB300)
constexpr int kQrRowTile = 16;          // rows of S staged per Gram step
constexpr int kQrMinRows = 4;           // rows per block at least (small m: fewer blocks)
// Gram entries a thread owns at most: c <= 64 and c <= kMaxSmall (two
// instantiations, so the common small case carries a quarter of the slots)
constexpr int kQrSlots64 = (64 * 65 / 2 + kCholThreads - 1) / kCholThreads;
constexpr int kQrMaxSlots = (kMaxSmall * (kMaxSmall + 1) / 2 + kCholThreads - 1) / kCholThreads;
constexpr long long kQrSpinCap = 1LL << 21;   // polls of one barrier wait (seconds)

// Row i and column j >= i of entry o of the upper triangle of a c x c matrix
// stored by rows (row i starts at i c - i (i - 1) / 2): the root of the
// quadratic, then exact integer correction.
__device__ __forceinline__ void upper_index(int o, int c, int &i, int &j) {
  const float b = 2.0f * c + 1.0f;
  i = (int)((b - sqrtf(b * b - 8.0f * o)) * 0.5f);
  i = max(0, min(i, c - 1));
  while (i + 1 < c && (i + 1) * c - (i + 1) * i / 2 <= o) ++i;
  while (i > 0 && i * c - i * (i - 1) / 2 > o) --i;
  j = i + (o - (i * c - i * (i - 1) / 2));
}

// Entries of a share this thread sums: t, t + 256, ... (nq of them, packed
// as i << 8 | j); nqw = the most any lane of the warp has (lane 0's). Each
// warp runs the multiply-adds of nqw slots by warp-uniform branches, as the
// GEMM does (a predicated-off DFMA costs as much as a full one).
template <int MAXQ>
struct GramSlots {
  int pk[MAXQ];
  int nq, nqw;
};

template <int MAXQ>
__device__ __forceinline__ void gram_slots(int c, GramSlots<MAXQ> &g) {
  const int tid = threadIdx.x;
  const int T = c * (c + 1) / 2;
  g.nq = max(0, (T - tid + kCholThreads - 1) / kCholThreads);
  g.nqw = __shfl_sync(0xffffffffu, g.nq, 0);
#pragma unroll
  for (int q = 0; q < MAXQ; ++q) {
    int i = 0, j = 0;
    if (q < g.nq) upper_index(tid + kCholThreads * q, c, i, j);
    g.pk[q] = (i << 8) | j;
  }
}

// This block's share of the rows [r0, r1) of S, into mine (T entries); sm
// holds kQrRowTile rows of S. S is read through L2 (another block of the
// fused launch may have written it).
template <int MAXQ>
__device__ __forceinline__ void gram_share(const double *S, long long ldS, int c, int r0, int r1,
                                           const GramSlots<MAXQ> &g, double *mine, double *sm) {
  const int tid = threadIdx.x;
  double acc[MAXQ];
#pragma unroll
  for (int q = 0; q < MAXQ; ++q) acc[q] = 0.0;
  for (int rt = r0; rt < r1; rt += kQrRowTile) {
    const int rows = min(kQrRowTile, r1 - rt);
    for (int e = tid; e < rows * c; e += kCholThreads) {
      const int rr = e / c;
      sm[e] = __ldcg(S + (long long)(rt + rr) * ldS + (e - rr * c));
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
      if (q < g.nqw) {
        const double *a = sm + (g.pk[q] >> 8), *b = sm + (g.pk[q] & 255);
        double v = acc[q];
#pragma unroll 4
        for (int r = 0; r < rows; ++r) v = fma(a[r * c], b[r * c], v);
        acc[q] = v;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < MAXQ; ++q)
    if (q < g.nq) mine[tid + kCholThreads * q] = acc[q];
}

// Entry t of G summed over the nb shares by one warp: lanes over shares in
// order, then a fixed shuffle tree; lane 0 writes G(i, j) and G(j, i).
__device__ __forceinline__ void gram_entry(const double *part, int nb, int c, int t, double *G) {
  const int lane = threadIdx.x & 31;
  const int T = c * (c + 1) / 2;
  constexpr int kPer = (kQrMaxBlocks + 31) / 32;
  double sh[kPer];                        // all loads in flight, then summed in share order
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int p = lane + 32 * k;
    sh[k] = p < nb ? __ldcg(part + (long long)p * T + t) : 0.0;
  }
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) v += sh[k];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) {
    int i, j;
    upper_index(t, c, i, j);
    G[i * c + j] = v;
    G[j * c + i] = v;
  }
}

// Launch per step: the shares (nb blocks), then their sum. Both do nothing
// once the QR has converged.
template <int MAXQ>
__global__ void __launch_bounds__(kCholThreads)
gram_share_kernel(const double *S, long long ldS, int m, int c, double *part, const int *flags) {
  pdl_enter();
  if (flags[0]) return;
  extern __shared__ double sm[];
  GramSlots<MAXQ> g;
  gram_slots(c, g);
  const int per = (m + gridDim.x - 1) / gridDim.x;
  const int r0 = min(m, (int)blockIdx.x * per), r1 = min(m, r0 + per);
  gram_share(S, ldS, c, r0, r1, g, part + (long long)blockIdx.x * (c * (c + 1) / 2), sm);
}

__global__ void __launch_bounds__(kCholThreads)
gram_sum_kernel(const double *part, int nb, int c, double *G, const int *flags) {
  pdl_enter();
  if (flags[0]) return;
  const int T = c * (c + 1) / 2;
  const int warps = gridDim.x * (kCholThreads / 32);
  for (int t = blockIdx.x * (kCholThreads / 32) + (threadIdx.x >> 5); t < T; t += warps)
    gram_entry(part, nb, c, t, G);
}

// ------------------------------------------------------------ fused form ---
// Grid barrier of the fused QR (cooperative launch: every block is resident).
// Arrivals count up in bar[0] (zero at the start of the QR); the e-th barrier
// waits for e * gridDim.x of them. A wait gives up after spin_cap polls,
// sets the timeout health bit and bar[1] (abort), and every block that sees
// bar[1] gives up too: the QR then stops with S partly processed, and the
// device status reports the timeout. Returns false in that case.
__device__ __forceinline__ bool grid_barrier(int *bar, int &epoch, long long spin_cap) {
  ++epoch;
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&bar[0], 1);
    const int target = epoch * (int)gridDim.x;
    volatile int *vb = bar;
    long long polls = 0;
    while (vb[0] < target) {
      if (vb[1] != 0) { ok = 0; break; }
      if (++polls > spin_cap) {
        atomicOr(&g_qr_health, kHealthTimeout);
        atomicExch(&bar[1], 1);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

// All passes of one Cholesky QR of S (m x c, leading dimension ldS) in one
// launch of nb blocks, block b owning the rows [b p, b p + p) of S. A pass:
//   1. the block's Gram share -> part[b];
//   2. barrier; each warp sums entries of G over the shares (gram_entry);
//   3. barrier; block 0: convergence test and factorization (chol_factor);
//   4. barrier; unless the pass found S orthonormal (or G non-finite),
//      R^{-1} applied to the block's own rows; if the factorization marked
//      the pass as the last, the QR ends here, else a barrier and the next
//      pass.
// The passes, G, tests and factorization are those of the launch-per-step
// form, bit for bit.
template <int MAXQ>
__global__ void __launch_bounds__(kCholThreads, 1)
qr_fused_kernel(double *S, int m, int c, long long ldS, double *G, double *Ut, double *y,
                double *part, int *flags, long long spin_cap) {
  pdl_enter();
  extern __shared__ double sm[];
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int kWarps = kCholThreads / 32;
  const int nb = gridDim.x, bid = blockIdx.x;
  const int per = (m + nb - 1) / nb;
  const int r0 = min(m, bid * per), r1 = min(m, r0 + per);
  const int T = c * (c + 1) / 2;
  GramSlots<MAXQ> g;
  gram_slots(c, g);
  int *bar = flags + 4;
  int epoch = 0;
  for (int pass = 0; pass < kPasses; ++pass) {
    gram_share(S, ldS, c, r0, r1, g, part + (long long)bid * T, sm);
    if (!grid_barrier(bar, epoch, spin_cap)) return;
    for (int t = bid * kWarps + warp; t < T; t += nb * kWarps) gram_entry(part, nb, c, t, G);
    if (!grid_barrier(bar, epoch, spin_cap)) return;
    if (bid == 0) chol_factor(G, Ut, y, c, m, flags, sm);
    if (!grid_barrier(bar, epoch, spin_cap)) return;
    const int done = __ldcg(flags), skip = __ldcg(flags + 1);
    if (skip) return;                      // orthonormal already (or a non-finite G)
    for (int e = tid; e < c * c; e += kCholThreads) sm[e] = __ldcg(Ut + e);
    for (int e = tid; e < c; e += kCholThreads) sm[c * c + e] = __ldcg(y + e);
    __syncthreads();
    apply_rows(S, ldS, c, sm, sm + c * c, r0 + warp, r1, kWarps);
    if (done) return;                      // this pass was the last one
    if (!grid_barrier(bar, epoch, spin_cap)) return;
  }
}

// SMs and cooperative-launch support of the current device, cached per
// device (0 SMs: unknown device).
void device_info(int &sms, bool &coop) {
  static int s_sms[64] = {};
  static signed char s_coop[64] = {};
  sms = 0;
  coop = false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  if (s_sms[dev] == 0) {
    int n = 0, co = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&co, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      return;
    }
    s_coop[dev] = co ? 1 : 0;
    s_sms[dev] = n;
  }
  sms = s_sms[dev];
  coop = s_coop[dev] != 0;
}

// Blocks (Gram shares) of a QR of m rows: at least kQrMinRows rows each, at
// most one per SM (the fused form keeps every block resident).
int qr_blocks(int m, int sms) {
  const int want = (m + kQrMinRows - 1) / kQrMinRows;
  return std::max(1, std::min({want, std::max(sms, 1), kQrMaxBlocks}));
}

// Test hooks, read once: HATT_QR_FORM=steps makes single calls use the
// launch-per-step form; HATT_QR_SPIN_CAP=<n> bounds each grid-barrier wait of
// the fused form to n polls (a small n makes the waits run out: the timeout
// status without a hang).
bool force_qr_steps() {
  static const bool v = [] {
    const char *e = getenv("HATT_QR_FORM");
    return e != nullptr && strcmp(e, "steps") == 0;
  }();
  return v;
}

long long qr_spin_cap() {
  static const long long v = [] {
    const char *e = getenv("HATT_QR_SPIN_CAP");
    const long long n = e ? atoll(e) : 0;
    return n > 0 ? n : kQrSpinCap;
  }();
  return v;
}

size_t chol_smem(int c) { return (size_t)c * (c + 1) * sizeof(double); }
size_t trsm_smem(int c) { return (size_t)(c * c + c) * sizeof(double); }
size_t gram_smem(int c) { return (size_t)kQrRowTile * c * sizeof(double); }

}  // namespace

cudaError_t qr_health_word(int *value, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_qr_health, sizeof(int));
  if (e == cudaSuccess && clear && *value != 0) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_qr_health, &zero, sizeof(int));
  }
  return e;
}

// G, U~, y, then the blocks' Gram shares.
size_t qr_scratch_doubles(int m, int c) {
  (void)m;
  return (size_t)2 * c * c + c + (size_t)kQrMaxBlocks * c * (c + 1) / 2;
}

cudaError_t qr_inplace(double *S, int m, int c, long long ldS, double *scratch, int *flags,
                       cudaStream_t st) {
  if (c <= 0 || m <= 0) return cudaSuccess;
  if (c > kMaxSmall) return cudaErrorInvalidValue;
  double *G = scratch;
  double *Ut = scratch + (size_t)c * c;
  double *y = scratch + (size_t)2 * c * c;
  double *part = scratch + (size_t)2 * c * c + c;
  int sms = 0;
  bool coop = false;
  device_info(sms, coop);
  if (sms <= 0) return cudaErrorInvalidDevice;
  const int nb = qr_blocks(m, sms);
  cudaError_t e = cudaMemsetAsync(flags, 0, 6 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const bool small = c <= 64;               // the kQrSlots64 instantiations
  if (coop && programmatic_launch() && !force_qr_steps()) {
    auto kernel = small ? qr_fused_kernel<kQrSlots64> : qr_fused_kernel<kQrMaxSlots>;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol_smem(kMaxSmall));
    if (e != cudaSuccess) return e;
    const size_t smem = std::max({chol_smem(c), trsm_smem(c), gram_smem(c)});
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(kCholThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kernel, S, m, c, ldS, G, Ut, y, part, flags, qr_spin_cap());
    note_launch();
    return e;
  }
  e = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)chol_smem(kMaxSmall));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(trsm_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)trsm_smem(kMaxSmall));
  if (e != cudaSuccess) return e;
  const int T = c * (c + 1) / 2;
  const int sum_blocks = std::max(1, std::min((T + 7) / 8, 2 * sms));
  const int blocks = std::max(1, std::min((m + kTrsmThreads / 32 - 1) / (kTrsmThreads / 32), 2 * sms));
  for (int p = 0; p < kPasses; ++p) {
    launch_k(small ? gram_share_kernel<kQrSlots64> : gram_share_kernel<kQrMaxSlots>, nb,
             kCholThreads, gram_smem(c), st, S, ldS, m, c, part, flags);
    note_launch();
    launch_k(gram_sum_kernel, sum_blocks, kCholThreads, 0, st, part, nb, c, G, flags);
    note_launch();
    launch_k(chol_inv_kernel, 1, kCholThreads, chol_smem(c), st, G, Ut, y, c, m, flags);
    note_launch();
    launch_k(trsm_rows_kernel, blocks, kTrsmThreads, trsm_smem(c), st, S, m, c, ldS, Ut, y, flags);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hatt
