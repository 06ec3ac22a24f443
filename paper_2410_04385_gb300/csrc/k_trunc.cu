// Right-to-left truncation sweep of a left-orthogonal TT (max_rank / tol).
//
// For core k with horizontal unfolding B = H(X_k) (la x N, N = n lb) and all
// cores to its left orthonormal, the singular values of B are those of the
// full unfolding at bond k. One step:
//   1. G = B B^T                                   (FP64 GEMM, all SMs)
//   2. eigenvectors of G in FP32 by tridiagonalization, bisection and inverse
//      iteration (one block; the FP32 pipe of GB300 is ~60x its FP64 pipe, and
//      this is the only serial stage)
//   3. three Ogita-Aishima refinement steps in FP64 (Ogita & Aishima, "Iterative
//      refinement for symmetric eigenvalue decomposition", JJIAM 2018):
//      R = I - U^T U, S = U^T G U, l_i = s_ii/(1 - r_ii),
//      E_ij = (s_ij + l_j r_ij)/(l_j - l_i) for separated pairs, r_ij/2 otherwise,
//      U <- U (I + E); quadratic convergence from the FP32 start. Three
//      closing steps with E = R/2 for every pair (Newton-Schulz, each squares
//      ||I - U^T U||) make U orthonormal to working accuracy whatever the
//      eigenvalue gaps: on graded or tightly clustered spectra the rotations
//      of the refinement can leave ||I - U^T U|| near 1e-2
//   4. B1 = U^T B (FP64 GEMM); e_i = ||row_i(B1)||^2 are the energies of the
//      directions u_i, computed from B itself (not from the squared Gram), so
//      the discarded tail sum_{dropped} e_i is accurate to O(u ||B||^2)
//   5. rho = smallest rank whose discarded tail <= delta^2, capped;
//      X_k <- rows of B1 scaled to unit norm, X_{k-1} <- X_{k-1} (U_rho Sigma_rho).
// The reconstruction U_rho U_rho^T B is an exact orthogonal projection of B,
// so the truncation error equals the computed tail whatever the accuracy of U.
// Everything stays in the padded la x n x lb layout; dropped rows/columns are
// zero, and the ranks live in device memory (no host synchronization).
#include <algorithm>
#include "hatt_internal.cuh"

namespace hatt {
namespace {

constexpr int kOaThreads = 1024;
constexpr int kThreads = 256;
constexpr int kRefineSteps = 3;   // Ogita-Aishima steps
constexpr int kOrthSteps = 3;     // closing Newton-Schulz steps
constexpr int kEigSteps = kRefineSteps + kOrthSteps;
constexpr double kConverged = 1e-9;

// 1/x for finite nonzero x: x = m 2^e with |m| in [0.5, 1), FP32 seed for 1/m,
// two Newton-Raphson steps y <- y (2 - m y) in FP64 (relative error 2^-23 ->
// 2^-46 -> FP64 rounding). Cheaper on GB300's FP64 unit than an IEEE divide.
__device__ __forceinline__ double rcp_newton(double x) {
  int e;
  const double m = frexp(x, &e);
  double y = (double)__frcp_rn((float)m);
  y = y * fma(-m, y, 2.0);
  y = y * fma(-m, y, 2.0);
  return ldexp(y, -e);
}

__device__ double block_sum(double v, double *red) {
  const int tid = threadIdx.x;
  red[tid] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Symmetric eigenvectors of the trace-scaled Gram matrix in FP32, one block,
// O(c^3) work in about 6c barrier-separated steps (cyclic Jacobi needs
// ~6 sweeps x (c - 1) rounds of O(c^2) updates and was the slowest kernel):
//   1. Householder tridiagonalization T = H^T A H (Golub & Van Loan 8.3.1):
//      for column k, v = x - alpha e_1, p = beta A v, w = p - (beta/2)(v^T p) v,
//      A <- A - v w^T - w v^T on the trailing block;
//   2. eigenvalues of T by bisection on Sturm counts, one thread per
//      eigenvalue (the i-th largest), from Gerschgorin bounds;
//   3. eigenvectors of T by two steps of inverse iteration, one thread per
//      eigenvalue, each a tridiagonal solve by Gaussian elimination with
//      partial pivoting (Golub & Van Loan 4.3);
//   4. modified Gram-Schmidt (twice) inside each cluster of eigenvalues closer
//      than 1e-3 of the spectral radius, where inverse iteration alone does
//      not give orthogonal vectors;
//   5. back-transformation Z <- H Z by the stored reflectors.
// Columns come out sorted by decreasing eigenvalue. The result only seeds the
// FP64 refinement, which needs a relative residual of ~1e-5 and an orthogonal
// start (within each cluster an arbitrary orthonormal basis is fine).
constexpr int kEigThreads = 256;
constexpr float kClusterRel = 1e-3f;

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lanes per dot product when n dot products share `threads` threads: the
// largest power of two <= 32 with lanes * n <= threads.
__device__ __forceinline__ int lanes_per_dot_n(int n, int threads) {
  int t = 32;
  while (t > 1 && t * n > threads) t >>= 1;
  return t;
}
__device__ __forceinline__ int lanes_per_dot(int n) { return lanes_per_dot_n(n, kEigThreads); }

// Sum over aligned groups of `lanes` lanes (a power of two dividing 32); every
// lane of the warp must call it.
__device__ __forceinline__ float group_sum_f(float v, int lanes) {
  for (int o = lanes >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Entry j of the start vector of eigenvector i: a hash of (i, j) mapped to
// [-1, 1). Start vectors must have independent projections on a cluster's
// eigenspace; a smooth pattern close to the all-ones vector does not (all of
// them project onto nearly the same direction), and Gram-Schmidt then keeps
// mostly the out-of-cluster error.
__device__ __forceinline__ float start_entry(int i, int j) {
  unsigned h = (unsigned)i * 0x9E3779B1u + (unsigned)j * 0x85EBCA77u + 0x165667B1u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return -1.0f + 2.0f * (float)(h & 0xffffffu) * (1.0f / 16777216.0f);
}

// Solve (T - lam I) z = b in place (b -> z), T with diagonal d and
// off-diagonal e, by Gaussian elimination with partial pivoting (Golub & Van
// Loan 4.3). The row being eliminated is carried in registers, so the sweep
// only stores the U factor (ua, udu, udu2) and the transformed right-hand side
// (kept in b); the back substitution reads them in reverse order, with loads
// that do not depend on its own recurrence.
__device__ void tridiag_shifted_solve(const float *d, const float *e, int c, float lam,
                                      float tiny, float *ua, float *udu, float *udu2, float *b) {
  // the pivoting choice is made with selects, not branches: the lanes of a
  // warp solve different systems and would otherwise run both paths
  float ac = d[0] - lam, duc = (c > 1) ? e[0] : 0.0f, bc = b[0];
  for (int j = 0; j + 1 < c; ++j) {
    const float an = d[j + 1] - lam, dun = (j + 2 < c) ? e[j + 1] : 0.0f, bn = b[j + 1];
    const float lo = e[j];                       // sub-diagonal entry of row j + 1
    const bool keep = fabsf(ac) >= fabsf(lo);    // else rows j and j + 1 swap
    const float acp = (ac == 0.0f) ? tiny : ac;
    const float piv = keep ? acp : lo;
    const float f = __fdividef(keep ? lo : ac, piv);
    ua[j] = piv;
    udu[j] = keep ? duc : an;
    udu2[j] = keep ? 0.0f : dun;
    b[j] = keep ? bc : bn;
    const float na = keep ? fmaf(-f, duc, an) : fmaf(-f, an, duc);
    const float nd = keep ? dun : -f * dun;
    const float nb = keep ? fmaf(-f, bc, bn) : fmaf(-f, bn, bc);
    ac = na; duc = nd; bc = nb;
  }
  ua[c - 1] = ac; udu[c - 1] = 0.0f; udu2[c - 1] = 0.0f; b[c - 1] = bc;
  // Back substitution. A shift equal to an eigenvalue leaves pivots near zero:
  // they are raised to +-tiny, and whenever a component exceeds 1e18 the whole
  // vector (solved and pending parts) is scaled by 1e-18 -- the system is
  // linear, so only the direction of z matters -- which keeps every
  // intermediate far from FP32 overflow.
  float z1 = 0.0f, z2 = 0.0f;                    // z_{j+1}, z_{j+2}
  for (int j = c - 1; j >= 0; --j) {
    float t = fmaf(-udu[j], z1, fmaf(-udu2[j], z2, b[j]));
    float piv = ua[j];
    if (fabsf(piv) < tiny) piv = piv < 0.0f ? -tiny : tiny;
    t = __fdividef(t, piv);
    if (fabsf(t) > 1e18f) {
      for (int q = 0; q < c; ++q) b[q] *= 1e-18f;
      z1 *= 1e-18f;
      z2 *= 1e-18f;
      t *= 1e-18f;
    }
    b[j] = t;
    z2 = z1;
    z1 = t;
  }
}

// Householder reflector of column k of A (rows k+1..c-1), by one warp:
// v = x - alpha e_1 with alpha = -sign(x_0) ||x|| in row k of Vh, tau[k] =
// 2 / v^T v (0 when x is already zero), d[k] = A_kk, e[k] = alpha.
__device__ __forceinline__ void householder_col(const float *A, int ld, int c, int k, float *Vh,
                                                float *d, float *e, float *tau, int lane) {
  const int m = c - k - 1;
  float *v = Vh + k * c;
  float s2 = 0.0f;
  for (int r = lane; r < m; r += 32) {
    const float x = A[(k + 1 + r) * ld + k];
    s2 = fmaf(x, x, s2);
  }
  s2 = warp_sum_f(s2);
  const float x0 = A[(k + 1) * ld + k];
  const bool skip = !(s2 > 1e-36f);
  const float alpha = skip ? x0 : -copysignf(sqrtf(s2), x0);
  const float v0 = x0 - alpha;
  const float vtv = s2 - x0 * x0 + v0 * v0;
  for (int r = lane; r < m; r += 32) v[r] = skip ? 0.0f : (r == 0 ? v0 : A[(k + 1 + r) * ld + k]);
  if (lane == 0) {
    d[k] = A[k * ld + k];
    e[k] = alpha;
    tau[k] = (skip || !(vtv > 0.0f)) ? 0.0f : 2.0f / vtv;
  }
}

constexpr int kSturmPts = 2;      // Sturm-count points per lane and multisection round
constexpr int kWarpCluster = 8;   // clusters up to this size are orthogonalized by one warp
constexpr int kBtCols = 8;        // eigenvector columns per warp in the back-transformation

// Back-transformation of columns i0 .. i0 + kBtCols - 1 of Z by the stored
// reflectors, one warp: lane l holds rows l + 32 t (t < TR, TR = 2 covers
// c <= 64), the reflectors applied from the last to the first with one warp
// sum per column each.
template <int TR>
__device__ __noinline__ void back_transform_cols(float *Z, int ld, const float *Vh,
                                                 const float *tau, int c, int i0, int lane) {
  float z[kBtCols][TR];
#pragma unroll
  for (int q = 0; q < kBtCols; ++q)
#pragma unroll
    for (int t = 0; t < TR; ++t) {
      const int r = lane + 32 * t, i = i0 + q;
      z[q][t] = (r < c && i < c) ? Z[r * ld + i] : 0.0f;
    }
  for (int k = c - 3; k >= 0; --k) {
    const float beta = tau[k];
    if (beta == 0.0f) continue;
    const float *v = Vh + k * c;                  // v[r - k - 1] for rows r > k
    float vr[TR];
#pragma unroll
    for (int t = 0; t < TR; ++t) {
      const int r = lane + 32 * t;
      vr[t] = (r > k && r < c) ? v[r - k - 1] : 0.0f;
    }
    float dq[kBtCols];
#pragma unroll
    for (int q = 0; q < kBtCols; ++q) {
      float acc = vr[0] * z[q][0];
#pragma unroll
      for (int t = 1; t < TR; ++t) acc = fmaf(vr[t], z[q][t], acc);
      dq[q] = acc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < kBtCols; ++q) dq[q] += __shfl_xor_sync(0xffffffffu, dq[q], o);
#pragma unroll
    for (int q = 0; q < kBtCols; ++q) {
      const float f = beta * dq[q];
#pragma unroll
      for (int t = 0; t < TR; ++t) z[q][t] = fmaf(-f, vr[t], z[q][t]);
    }
  }
#pragma unroll
  for (int q = 0; q < kBtCols; ++q)
#pragma unroll
    for (int t = 0; t < TR; ++t) {
      const int r = lane + 32 * t, i = i0 + q;
      if (r < c && i < c) Z[r * ld + i] = z[q][t];
    }
}

__global__ void __launch_bounds__(kEigThreads)
eig_tridiag32_kernel(const double *G, int c, double *U, const int *skip) {
  pdl_enter();
  if (skip && *skip) return;
  extern __shared__ float fs[];
  const int ld = c + 1;
  float *A = fs;                 // c x ld
  float *Z = A + c * ld;         // c x ld, eigenvectors (columns)
  float *Vh = Z + c * ld;        // c x c, reflector k in row k (length c-k-1)
  float *d = Vh + c * c;         // diagonal of T
  float *e = d + c;              // off-diagonal of T
  float *tau = e + c;            // reflector scales beta_k
  float *lam = tau + c;          // eigenvalues, decreasing
  float *p = lam + c;            // work vector
  float *p2 = p + c;             // work vector (second buffer of p)
  __shared__ double s_tr;
  __shared__ float s_scal[4];
  __shared__ int s_start[kMaxSmall + 1];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {                          // trace (FP64), one warp
    double tr = 0.0;
    for (int i = lane; i < c; i += 32) tr += G[i * c + i];
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (lane == 0) s_tr = tr;
  }
  __syncthreads();
  const double scale = s_tr > 0.0 ? 1.0 / s_tr : 1.0;
  for (int e2 = tid; e2 < c * c; e2 += kEigThreads) {
    const int i = e2 / c, j = e2 % c;
    A[i * ld + j] = (float)(0.5 * (G[i * c + j] + G[j * c + i]) * scale);
  }
  __syncthreads();

  // 1. tridiagonalization, two barriers per column. With p_k = beta_k A2 v_k
  // known, K = beta_k/2 v_k^T p_k and w = p_k - K v_k: warp 0 updates column
  // k + 1 (column 0 of A2) and forms reflector k + 1 while warps 1..7 apply
  // A2 -= v w^T + w v^T to the trailing block A2[1:, 1:]; after a barrier all
  // warps form p_{k+1} = beta_{k+1} A2' v_{k+1}. Row k + 1 right of the
  // diagonal is never read again and is not updated.
  {
    float *pc = p, *pn = p2;
    auto matvec = [&](int k1) {                             // pn = beta_k1 A2_k1 v_k1
      const int m = c - k1 - 1;
      const float *v = Vh + k1 * c;
      const int lanes = lanes_per_dot(m);
      const int i = tid / lanes, sub = tid % lanes;
      float sacc = 0.0f, sacc2 = 0.0f;
      if (i < m) {
        const float *row = A + (k1 + 1 + i) * ld + (k1 + 1);
        int j = sub;
        for (; j + lanes < m; j += 2 * lanes) {
          sacc = fmaf(row[j], v[j], sacc);
          sacc2 = fmaf(row[j + lanes], v[j + lanes], sacc2);
        }
        if (j < m) sacc = fmaf(row[j], v[j], sacc);
      }
      sacc = group_sum_f(sacc + sacc2, lanes);
      if (i < m && sub == 0) pn[i] = tau[k1] * sacc;
    };
    if (warp == 0 && c > 2) householder_col(A, ld, c, 0, Vh, d, e, tau, lane);
    __syncthreads();
    if (c > 2) matvec(0);
    __syncthreads();
    { float *t = pc; pc = pn; pn = t; }
    for (int k = 0; k + 2 < c; ++k) {
      const int m = c - k - 1;
      const float *v = Vh + k * c;
      const float beta = tau[k];
      float kd = 0.0f;                                      // K = beta/2 v^T p, every warp
      for (int r = lane; r < m; r += 32) kd = fmaf(v[r], pc[r], kd);
      const float K = 0.5f * beta * warp_sum_f(kd);
      if (warp == 0) {                                      // column k + 1, then reflector k + 1
        const float v0 = v[0], w0 = pc[0] - K * v0;
        for (int i = lane; i < m; i += 32) {
          const float vi = v[i], wi = pc[i] - K * vi;
          A[(k + 1 + i) * ld + (k + 1)] -= vi * w0 + wi * v0;
        }
        __syncwarp();
        if (k + 3 < c) householder_col(A, ld, c, k + 1, Vh, d, e, tau, lane);
      } else {                                              // trailing block, warps 1..7
        const int mm = m - 1;
        const int bt = tid - 32;
        const int lanes = lanes_per_dot_n(mm, kEigThreads - 32);
        const int r = bt / lanes, sub = bt % lanes;
        if (r < mm) {
          const float vi = v[r + 1], wi = pc[r + 1] - K * vi;
          float *row = A + (k + 2 + r) * ld + (k + 2);
          int j = sub;
          for (; j + lanes < mm; j += 2 * lanes) {
            const float wj = pc[j + 1] - K * v[j + 1], wj2 = pc[j + lanes + 1] - K * v[j + lanes + 1];
            row[j] -= vi * wj + wi * v[j + 1];
            row[j + lanes] -= vi * wj2 + wi * v[j + lanes + 1];
          }
          if (j < mm) {
            const float wj = pc[j + 1] - K * v[j + 1];
            row[j] -= vi * wj + wi * v[j + 1];
          }
        }
      }
      __syncthreads();
      if (k + 3 < c) matvec(k + 1);
      __syncthreads();
      float *t = pc; pc = pn; pn = t;
    }
  }
  if (tid == 0) {
    if (c >= 2) {
      d[c - 2] = A[(c - 2) * ld + (c - 2)];
      e[c - 2] = A[(c - 1) * ld + (c - 2)];
    }
    d[c - 1] = A[(c - 1) * ld + (c - 1)];
    e[c - 1] = 0.0f;
    // Gerschgorin interval and the smallest pivot allowed in Sturm counts
    float lo = 3.0e38f, hi = -3.0e38f, emax = 0.0f;
    for (int i = 0; i < c; ++i) {
      const float rad = (i > 0 ? fabsf(e[i - 1]) : 0.0f) + (i + 1 < c ? fabsf(e[i]) : 0.0f);
      lo = fminf(lo, d[i] - rad);
      hi = fmaxf(hi, d[i] + rad);
      if (i + 1 < c) {
        p[i] = e[i] * e[i];                                  // e^2 for the Sturm counts
        emax = fmaxf(emax, p[i]);
      }
    }
    s_scal[0] = lo;
    s_scal[1] = hi;
    s_scal[2] = 1e-35f * fmaxf(1.0f, emax);
  }
  __syncthreads();

  // 2. eigenvalues by multisection on Sturm counts: a group of G lanes per
  // eigenvalue (the i-th largest), each lane counting at kSturmPts points of
  // the bracket at once, so a round shrinks it G kSturmPts + 1 times (a
  // bisection step halves it) and the independent count chains hide each
  // other's division latency.
  const float glo = s_scal[0], ghi = s_scal[1], pivmin = s_scal[2];
  const float span = fmaxf(fabsf(glo), fabsf(ghi));
  {
    const int G = c <= 32 ? 8 : c <= 64 ? 4 : 2;
    const int i = tid / G, g = tid % G;
    const bool has = i < c;
    const int target = c - 1 - i;                           // count of smaller eigenvalues
    float a = glo, b = ghi;
    bool active = has;
    const float inv_n = 1.0f / (float)(G * kSturmPts + 1);
    for (int round = 0; round < 64 && __any_sync(0xffffffffu, active); ++round) {
      float na = a, nb = b;
      if (active) {
        float x[kSturmPts], q[kSturmPts];
        int cnt[kSturmPts];
#pragma unroll
        for (int t = 0; t < kSturmPts; ++t) {
          x[t] = fmaf(b - a, (float)(g + G * t + 1) * inv_n, a);
          q[t] = d[0] - x[t];
          cnt[t] = q[t] < 0.0f;
        }
        for (int j = 1; j < c; ++j) {
          const float dj = d[j], ej2 = p[j - 1];
#pragma unroll
          for (int t = 0; t < kSturmPts; ++t) {
            if (fabsf(q[t]) < pivmin) q[t] = -pivmin;
            q[t] = dj - x[t] - __fdividef(ej2, q[t]);
            cnt[t] += q[t] < 0.0f;
          }
        }
#pragma unroll
        for (int t = 0; t < kSturmPts; ++t) {
          if (cnt[t] <= target) na = fmaxf(na, x[t]);
          else nb = fminf(nb, x[t]);
        }
      }
      for (int o = 1; o < G; o <<= 1) {                     // group of G aligned lanes
        na = fmaxf(na, __shfl_xor_sync(0xffffffffu, na, o));
        nb = fminf(nb, __shfl_xor_sync(0xffffffffu, nb, o));
      }
      if (active) {
        a = na;
        b = nb;
        if (b - a <= 2.4e-7f * fmaxf(fmaxf(fabsf(a), fabsf(b)), 1e-7f * span)) active = false;
      }
    }
    if (has && g == 0) lam[i] = 0.5f * (a + b);
  }
  __syncthreads();
  // Shifts of equal (or nearly equal) eigenvalues are moved apart by 10 ulps
  // of the larger magnitude, as in LAPACK's inverse iteration: identical
  // shifts meet the same near-zero pivot and return the same vector, which
  // Gram-Schmidt would then annihilate (exact ties occur, e.g. the two equal
  // singular values of sin(a + b) = sin a cos b + cos a sin b).
  if (tid == 0)
    for (int i = 1; i < c; ++i) {
      const float pert = 6e-7f * fabsf(lam[i - 1]);
      if (lam[i - 1] - lam[i] < pert) lam[i] = lam[i - 1] - pert;
    }
  __syncthreads();

  // 3. inverse iteration, one thread per eigenvector (column i of Z)
  const float tiny = 1e-30f + 1e-13f * span;
  for (int i = tid; i < c; i += kEigThreads) {
    float a[kMaxSmall], du[kMaxSmall], du2[kMaxSmall], z[kMaxSmall];
    for (int j = 0; j < c; ++j) z[j] = start_entry(i, j);
    for (int it = 0; it < 2; ++it) {
      tridiag_shifted_solve(d, e, c, lam[i], tiny, a, du, du2, z);
      float mx = 0.0f;                             // scale by max |z_j| first: z.z
      for (int j = 0; j < c; ++j) mx = fmaxf(mx, fabsf(z[j]));   // may overflow
      const float sc = mx > 0.0f ? 1.0f / mx : 0.0f;
      float s = 0.0f;
      for (int j = 0; j < c; ++j) {
        z[j] *= sc;
        s = fmaf(z[j], z[j], s);
      }
      const float inv = s > 0.0f ? rsqrtf(s) : 0.0f;
      for (int j = 0; j < c; ++j) z[j] *= inv;
    }
    for (int j = 0; j < c; ++j) Z[j * ld + i] = z[j];
  }
  // cluster starts: lam decreasing, a new cluster where the gap exceeds the threshold
  for (int i = tid; i < c; i += kEigThreads)
    s_start[i] = (i == 0) || (lam[i - 1] - lam[i] > kClusterRel * span);
  if (tid == 0) s_start[c] = 1;
  __syncthreads();

  // 4. Gram-Schmidt (twice) within clusters. Clusters of up to kWarpCluster
  // vectors: modified Gram-Schmidt by one warp each, all such clusters at
  // once. Larger clusters (graded spectra put every eigenvalue below
  // kClusterRel of the largest into one): classical Gram-Schmidt by the whole
  // block, one vector at a time -- its projections on the earlier vectors of
  // the cluster spread over the warps, the update over the rows.
  for (int s0 = 0; s0 < c; ++s0) {
    if (!s_start[s0] || (s0 % (kEigThreads / 32)) != warp) continue;
    int t0 = s0 + 1;
    while (!s_start[t0]) ++t0;
    if (t0 - s0 > kWarpCluster) continue;
    for (int a = s0 + 1; a < t0; ++a) {
      for (int rep = 0; rep < 2; ++rep) {
        for (int b = s0; b < a; ++b) {
          float dot = 0.0f;
          for (int r = lane; r < c; r += 32) dot = fmaf(Z[r * ld + b], Z[r * ld + a], dot);
          dot = warp_sum_f(dot);
          for (int r = lane; r < c; r += 32) Z[r * ld + a] = fmaf(-dot, Z[r * ld + b], Z[r * ld + a]);
          __syncwarp();
        }
        float sn = 0.0f;
        for (int r = lane; r < c; r += 32) sn = fmaf(Z[r * ld + a], Z[r * ld + a], sn);
        sn = warp_sum_f(sn);
        const float inv = sn > 0.0f ? rsqrtf(sn) : 0.0f;
        for (int r = lane; r < c; r += 32) Z[r * ld + a] *= inv;
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int s0 = 0; s0 < c; ++s0) {                 // every thread takes the same branches
    if (!s_start[s0]) continue;
    int t0 = s0 + 1;
    while (!s_start[t0]) ++t0;
    if (t0 - s0 <= kWarpCluster) continue;
    for (int a = s0 + 1; a < t0; ++a) {
      for (int rep = 0; rep < 2; ++rep) {
        for (int bb = s0 + warp; bb < a; bb += kEigThreads / 32) {   // p[b - s0] = z_b . z_a
          float dot = 0.0f;
          for (int r = lane; r < c; r += 32) dot = fmaf(Z[r * ld + bb], Z[r * ld + a], dot);
          dot = warp_sum_f(dot);
          if (lane == 0) p[bb - s0] = dot;
        }
        __syncthreads();
        for (int r = tid; r < c; r += kEigThreads) {                  // z_a -= sum_b p_b z_b
          float za = Z[r * ld + a];
          for (int bb = s0; bb < a; ++bb) za = fmaf(-p[bb - s0], Z[r * ld + bb], za);
          Z[r * ld + a] = za;
        }
        __syncthreads();
      }
      if (warp == 0) {
        float sn = 0.0f;
        for (int r = lane; r < c; r += 32) sn = fmaf(Z[r * ld + a], Z[r * ld + a], sn);
        sn = warp_sum_f(sn);
        if (lane == 0) s_scal[3] = sn > 0.0f ? rsqrtf(sn) : 0.0f;
      }
      __syncthreads();
      const float inv = s_scal[3];
      for (int r = tid; r < c; r += kEigThreads) Z[r * ld + a] *= inv;
      __syncthreads();
    }
  }

  // 5. back-transformation Z <- H_0 ... H_{c-3} Z. The columns of Z are
  // independent: each warp takes kBtCols of them at a time, holds their
  // entries in registers (lane l: rows l, l + 32, l + 64, l + 96) and applies
  // the reflectors from the last to the first -- per reflector one warp sum
  // per column, no block barrier.
  for (int i0 = warp * kBtCols; i0 < c; i0 += (kEigThreads / 32) * kBtCols) {
    if (c <= 64) back_transform_cols<2>(Z, ld, Vh, tau, c, i0, lane);
    else back_transform_cols<4>(Z, ld, Vh, tau, c, i0, lane);
  }
  __syncthreads();
  for (int e2 = tid; e2 < c * c; e2 += kEigThreads) {
    const int r = e2 / c, i = e2 % c;
    U[e2] = (double)Z[r * ld + i];
  }
}

// One Ogita-Aishima step: given UtU (= U^T U), S (= U^T G U) and G, write
// Eout = I + E (so that the next U is U * Eout). The cluster threshold is
// floored at the rounding level of ||G||: eigenvalues that agree to working
// accuracy (exact degeneracies, e.g. the equal singular values of
// sin(2x+2y) = sin 2x cos 2y + cos 2x sin 2y) are only orthogonalized, never
// rotated by a quotient of two rounding errors.
// Rotations larger than 0.1 are not applied (the pair counts as clustered
// for this step). With orth_only set, every pair is treated as clustered: E = (I - U^T U)/2,
// one Newton-Schulz orthonormalization step (S and G are not read). A
// positive floor_norm replaces ||G||_F in the floor (the deflated matrix of
// the cluster levels has an exactly diagonal part that must not raise it).
//
// The quotient of a separated pair is formed in FP32 after scaling numerator
// and denominator by 1/||G||_F (the denominator exceeds 64 c u ||G||, so it
// stays in range): E only enters as U (I + E), so a relative error of 1e-7 in
// E adds 1e-7 * ||E|| to an error that the step squares anyway.
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kOaThreads)
oa_update_kernel(const double *UtU, const double *S, const double *G, int c, int orth_only,
                 double floor_norm, int *state, int step, int nsteps, double *Eout) {
  pdl_enter();
  if (state && state[step]) return;
  __shared__ double wred[3][kOaThreads / 32];
  __shared__ double lam[kMaxSmall];
  __shared__ double s_delta, s_inv;
  const int tid = threadIdx.x;
  if (!orth_only) {
    for (int i = tid; i < c; i += kOaThreads) lam[i] = S[i * c + i] / UtU[i * c + i];
    __syncthreads();
    double g2 = 0.0, r2 = 0.0, sd2 = 0.0;
    for (int i = tid / 32; i < c; i += kOaThreads / 32)
      for (int j = tid % 32; j < c; j += 32) {
        const int e = i * c + j;
        const double r = (i == j ? 1.0 : 0.0) - UtU[e];
        const double sd = S[e] - (i == j ? lam[i] : 0.0);
        g2 = fma(G[e], G[e], g2);
        r2 = fma(r, r, r2);
        sd2 = fma(sd, sd, sd2);
      }
    g2 = warp_sum_d(g2);
    r2 = warp_sum_d(r2);
    sd2 = warp_sum_d(sd2);
    if ((tid & 31) == 0) { wred[0][tid >> 5] = g2; wred[1][tid >> 5] = r2; wred[2][tid >> 5] = sd2; }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0, s = 0.0;
      for (int w = 0; w < kOaThreads / 32; ++w) { a += wred[0][w]; b += wred[1][w]; s += wred[2][w]; }
      const double u = 1.1102230246251565e-16;
      const double gn = sqrt(a);
      s_delta = fmax(2.0 * (sqrt(s) + gn * sqrt(b)), 64.0 * c * u * (floor_norm > 0.0 ? floor_norm : gn));
      s_inv = gn > 0.0 ? rcp_newton(gn) : 1.0;
    }
    __syncthreads();
  }
  const double delta = orth_only ? 0.0 : s_delta;
  const double inv = orth_only ? 1.0 : s_inv;
  double emax = 0.0;
  for (int i = tid / 32; i < c; i += kOaThreads / 32)
    for (int j = tid % 32; j < c; j += 32) {
      const int e = i * c + j;
      const double r = (i == j ? 1.0 : 0.0) - UtU[e];
      double E;
      E = 0.5 * r;
      if (!orth_only && i != j && fabs(lam[i] - lam[j]) > delta) {
        const float num = (float)(fma(lam[j], r, S[e]) * inv);
        const float den = (float)((lam[j] - lam[i]) * inv);
        const float q = __fdividef(num, den);
        // a first-order rotation above 0.1 belongs to a pair the current
        // iterate does not resolve yet: applying it would wreck the
        // orthogonality; the pair is treated as clustered for this step
        if (fabsf(q) <= 0.1f) E = (double)q;
      }
      emax = fmax(emax, fabs(E));
      Eout[e] = E + (i == j ? 1.0 : 0.0);
    }
  // Converged: after this correction (|E| <= kConverged) the error is
  // O(|E|^2 + 1e-7 |E|) ~ 1e-16, so every later step is skipped.
  if (!state) return;
  for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  __shared__ double wmax[kOaThreads / 32];
  if ((tid & 31) == 0) wmax[tid >> 5] = emax;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < kOaThreads / 32; ++w) m = fmax(m, wmax[w]);
    if (m <= kConverged)
      for (int j = step + 1; j < nsteps; ++j) state[j] = 1;
  }
}

// After an eigvecs run whose steps may have stopped early: the number of
// steps applied is the index of the first skipped step; if it is odd the
// result sits in Ub and is copied to Ua.
__global__ void select_result_kernel(const int *state, int nsteps, const double *Ub, double *Ua,
                                     int count) {
  pdl_enter();
  int applied = nsteps;
  for (int j = 0; j < nsteps; ++j)
    if (state[j]) { applied = j; break; }
  if ((applied & 1) == 0) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
    Ua[e] = Ub[e];
}

// ---------------------------------------------------------------------------
// Further levels (tolerance mode only). The FP32 start resolves eigenvalues
// only down to ~1e-7 of the matrix it is given, and the refinement cannot
// split what the start leaves mixed: its cluster test compares gaps with the
// size of the unresolved block itself (~1e-7 ||G||). Eigenvalues below that
// stay mixed after the first level. G1 = B1 B1^T, formed from the rotated rows
// B1 = U^T B, holds its entries to u times the row norms, so the low-energy
// rows can be diagonalized again on their own scale, and again below that:
//   level 0:  cluster C = {i : G1_ii < kLevelCut ||G1||_F}
//   level j:  cluster C = {i : G1_ii < kLevelCut s_{j-1}}
//   s_j = sum_{i in C} G1_ii,  H = G1[C, C] / s_j on the cluster,
//   H_ii = 1.25 + i/(2c) (distinct, above the cluster's spectrum, no
//   coupling) elsewhere,
// and the eigenvectors V of H (same FP32 start + FP64 refinement, floor taken
// from the cluster's norm, 1) rotate U <- U V. Each level resolves about
// seven decades of energy below its scale; its cut, 1e-6 of the scale, stays
// above what the previous level resolved. A level is skipped (V = I, and so
// are all later levels) when its cluster has fewer than two rows or fits
// under delta^2 as a whole, in which case the cut cannot fall inside it, or
// when the rank cap keeps fewer rows than lie above the cluster (the cut is
// then made above it).
//   flags[0] = this level (and every later one) skipped
//   flags[1] = skip the cross step (delta^2 > 1e-16 ||G1||_F: the level-one
//              leakage, ~u^2 ||G1|| / 1e-12, is then irrelevant); level 0
//   flags[2] = level 0 and the cross step skipped: B1 needs no recomputation
//   scale[0] = s of the last level applied
constexpr double kLevelCut = 1e-6;
constexpr int kLevels = 6;

// Outside stream capture the host reads flags[0] after each level's
// preparation and stops launching once a level is skipped (every later one
// would be too): one short synchronization instead of ~25 no-op launches
// per remaining level. Captured streams, and the batched entry point (whose
// lanes share one issuing thread), launch every level.
thread_local bool t_host_sync = true;

__global__ void __launch_bounds__(kThreads)
level_prep_kernel(const double *G1, int c, int cap, const double *delta2, int level,
                  double *scale, double *H, double *V, int *flags, int *eig_state) {
  pdl_enter();
  __shared__ double red[kThreads];
  __shared__ int inc[kMaxSmall];
  const int tid = threadIdx.x;
  const int prev_skip = level > 0 && flags[0];   // read by every thread before any write
  double f2 = 0.0;
  if (level == 0)
    for (int e = tid; e < c * c; e += kThreads) f2 = fma(G1[e], G1[e], f2);
  const double fn = sqrt(block_sum(f2, red));
  const double thr = kLevelCut * (level == 0 ? fn : scale[0]);
  double s = 0.0, m = 0.0;
  for (int i = tid; i < c; i += kThreads) {
    const double ei = G1[i * c + i];
    inc[i] = ei < thr;
    if (inc[i]) { s += ei; m += 1.0; }
  }
  s = block_sum(s, red);
  m = block_sum(m, red);
  const double d2 = delta2[0];
  const int skip = prev_skip || (m < 2.0) || !(s > d2) || (cap > 0 && c - (int)m >= cap);
  if (tid == 0) {
    flags[0] = skip;
    if (level == 0) {
      const int skip_cross = d2 > 1e-16 * fn;
      flags[1] = skip_cross;
      flags[2] = skip && skip_cross;
    }
    if (!skip) scale[0] = s;
  }
  if (tid < kEigSteps) eig_state[tid] = skip;
  const double inv_s = skip ? 0.0 : 1.0 / s;
  for (int e = tid; e < c * c; e += kThreads) {
    const int i = e / c, j = e % c;
    if (skip) {
      V[e] = (i == j) ? 1.0 : 0.0;
    } else if (inc[i] && inc[j]) {
      H[e] = G1[e] * inv_s;
    } else {
      H[e] = (i == j) ? 1.25 + 0.5 * (double)i / (double)c : 0.0;
    }
  }
}

// Cross step: one first-order Jacobi rotation for every pair whose energies
// differ by more than half the larger, computed from G1 = B1 B1^T (entries
// accurate relative to the row norms): E_ij = G1_ij / (G1_jj - G1_ii). It
// removes the leakage of high-energy directions into low-energy ones that the
// first level leaves at ~u ||G|| / gap. Rotations above 1e-2 are left out:
// they belong to pairs the Gram matrices could not resolve, where a
// first-order step would not converge. Eout = I + E (I when skipped).
__global__ void __launch_bounds__(kOaThreads)
cross_kernel(const double *G1, int c, const int *flags, double *Eout) {
  pdl_enter();
  const int skip = flags[1];
  for (int e = threadIdx.x; e < c * c; e += kOaThreads) {
    const int i = e / c, j = e % c;
    double v = (i == j) ? 1.0 : 0.0;
    if (!skip && i != j) {
      const double ei = G1[i * c + i], ej = G1[j * c + j];
      const double gap = ej - ei;
      if (fabs(gap) > 0.5 * fmax(ei, ej)) {
        const double q = G1[e] / gap;
        if (fabs(q) <= 1e-2) v = q;
      }
    }
    Eout[e] = v;
  }
}

__global__ void __launch_bounds__(kThreads)
rownorm_kernel(const double *B1, long long N, double *e) {
  pdl_enter();
  __shared__ double red[kThreads];
  const int row = blockIdx.x;
  double s = 0.0;
  for (long long j = threadIdx.x; j < N; j += kThreads) {
    const double v = B1[row * N + j];
    s = fma(v, v, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) e[row] = s;
}

// Sort energies, pick rho by the tolerance rule, cap, publish rank/perm/sigma.
__global__ void __launch_bounds__(kThreads)
rank_kernel(const double *e, int c, int cap, const double *delta2, long long *ranks, int k,
            int *perm, double *sigma) {
  pdl_enter();
  __shared__ double sorted[kMaxSmall];
  __shared__ double tails[kMaxSmall + 1];
  __shared__ long long keys[kMaxSmall];
  const int tid = threadIdx.x;
  // sort key: the energy, or -1 when it is not finite (NaN compares false
  // with everything, so without the key equal positions could repeat and
  // perm would not be a permutation); staged in shared memory once as the
  // order-preserving integer image of the double (x >= 0: its bits; x < 0:
  // the bits with the magnitude bits flipped), so the counting loop below
  // waits on no global load and compares on the integer pipe
  for (int i = tid; i < c; i += kThreads) {
    const double v = e[i];
    const long long b = __double_as_longlong(isfinite(v) ? v : -1.0);
    keys[i] = b ^ ((b >> 63) & 0x7fffffffffffffffLL);
  }
  __syncthreads();
  for (int i = tid; i < c; i += kThreads) {
    const long long ki = keys[i];
    int pos = 0;
    for (int j = 0; j < c; ++j) {
      const long long kj = keys[j];
      pos += (kj > ki) || (kj == ki && j < i);
    }
    const double ei = isfinite(e[i]) ? e[i] : -1.0;
    perm[pos] = i;
    sorted[pos] = ei;
    sigma[pos] = sqrt(fmax(ei, 0.0));
  }
  __syncthreads();
  if (tid == 0) {
    const double d2 = delta2[0];
    // tail[rho] = sum_{p >= rho} sorted[p]; smallest rho >= 1 with tail <= delta^2
    double tail = 0.0;
    int rho = c;
    tails[c] = 0.0;
    for (int p = c - 1; p >= 0; --p) {
      const double sp = sorted[p];
      tail += (sp > 0.0) ? sp : 0.0;
      tails[p] = tail;
    }
    for (int cand = 1; cand <= c; ++cand) {
      if (tails[cand] <= d2) { rho = cand; break; }
    }
    if (cap > 0) rho = min(rho, cap);
    rho = max(rho, 1);
    ranks[k] = rho;
  }
}

__global__ void newcore_kernel(const double *B1, int c, long long N, const int *perm,
                               const double *sigma, const long long *ranks, int k, double *Xk) {
  pdl_enter();
  const int rho = (int)ranks[k];
  const long long total = (long long)c * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / N);
    const long long col = t % N;
    double v = 0.0;
    if (j < rho) {
      const double s = sigma[j];
      if (s > 0.0) v = B1[(long long)perm[j] * N + col] / s;
    }
    Xk[t] = v;
  }
}

__global__ void kmat_kernel(const double *U, int c, const int *perm, const double *sigma,
                            const long long *ranks, int k, double *K) {
  pdl_enter();
  const int rho = (int)ranks[k];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < c * c; t += gridDim.x * blockDim.x) {
    const int l = t / c, j = t % c;
    K[t] = (j < rho) ? U[l * c + perm[j]] * sigma[j] : 0.0;
  }
}

__global__ void __launch_bounds__(kThreads)
delta2_kernel(const double *x, long long count, double tol, int d, double *out, double *partials,
              unsigned int *ticket) {
  pdl_enter();
  __shared__ double red[kThreads];
  __shared__ bool last;
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < count;
       e += (long long)gridDim.x * kThreads)
    s = fma(x[e], x[e], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) t += ((volatile double *)partials)[i];
  t = block_sum(t, red);
  if (threadIdx.x == 0) {
    out[0] = tol * tol * t / (double)(d > 1 ? d - 1 : 1);
    *ticket = 0u;
  }
}

struct RankTable {
  int count;
  long long r[kMaxOrder + 1];
};

__global__ void set_ranks_kernel(RankTable t, long long *ranks) {
  pdl_enter();
  for (int i = threadIdx.x; i < t.count; i += blockDim.x) ranks[i] = t.r[i];
}

size_t eig_smem(int c) { return ((size_t)2 * c * (c + 1) + (size_t)c * c + 6 * (size_t)c) * sizeof(float); }

struct Layout {
  double *G, *U0, *U1, *UtU, *T, *S, *E, *H, *V0, *V1, *B1, *e, *sigma, *K, *tmp, *gs, *scale;
  int *perm, *flags;
};

Layout carve(double *base, int la, long long N, long long mrows) {
  Layout L;
  const size_t c2 = (size_t)la * la;
  double *p = base;
  L.G = p; p += c2;
  L.U0 = p; p += c2;
  L.U1 = p; p += c2;
  L.UtU = p; p += c2;
  L.T = p; p += c2;
  L.S = p; p += c2;
  L.E = p; p += c2;
  L.K = p; p += c2;
  L.H = p; p += c2;
  L.V0 = p; p += c2;
  L.V1 = p; p += c2;
  L.flags = (int *)p; p += 12;       // 24 ints: level flags, two eigvecs states
  L.scale = p; p += 1;
  L.e = p; p += la;
  L.sigma = p; p += la;
  L.perm = (int *)p; p += la;
  L.B1 = p; p += (size_t)la * N;
  L.tmp = p; p += (size_t)mrows * la;
  L.gs = p;
  return L;
}

size_t carve_doubles(int la, long long N, long long mrows) {
  return (size_t)11 * la * la + 13 + 3 * (size_t)la + (size_t)la * N + (size_t)mrows * la;
}

Gemm g_gram(const double *B, int la, long long N, double *G) {
  Gemm g;
  g.M = la; g.N = la; g.K = (int)N;
  g.A = B; g.sAm = N; g.sAk = 1;
  g.B = B; g.sBk = 1; g.sBn = N;
  g.C = G; g.sCm = la; g.sCn = 1;
  return g;
}
Gemm g_tn(const double *U, const double *X, int la, long long ncols, long long ldx, double *C,
          long long ldc) {   // C = U^T X, U la x la, X la x ncols
  Gemm g;
  g.M = la; g.N = (int)ncols; g.K = la;
  g.A = U; g.sAm = 1; g.sAk = la;
  g.B = X; g.sBk = ldx; g.sBn = 1;
  g.C = C; g.sCm = ldc; g.sCn = 1;
  return g;
}
Gemm g_nn(const double *X, const double *Y, long long m, int k, int n, double *C) {
  Gemm g;
  g.M = (int)m; g.N = n; g.K = k;
  g.A = X; g.sAm = k; g.sAk = 1;
  g.B = Y; g.sBk = n; g.sBn = 1;
  g.C = C; g.sCm = n; g.sCn = 1;
  return g;
}

}  // namespace

size_t trunc_scratch_doubles(int la, int n, int lb, int lm, int nm) {
  const long long N = (long long)n * lb;
  const long long mrows = (long long)lm * nm;
  size_t gs = 0;
  gs = std::max(gs, gemm_scratch_doubles(g_gram(nullptr, la, N, nullptr)));
  gs = std::max(gs, gemm_scratch_doubles(g_tn(nullptr, nullptr, la, la, la, nullptr, la)));
  gs = std::max(gs, gemm_scratch_doubles(g_nn(nullptr, nullptr, la, la, la, nullptr)));
  gs = std::max(gs, gemm_scratch_doubles(g_tn(nullptr, nullptr, la, N, N, nullptr, N)));
  gs = std::max(gs, gemm_scratch_doubles(g_nn(nullptr, nullptr, mrows, la, la, nullptr)));
  return carve_doubles(la, N, mrows) + gs;
}

// Eigenvectors of the symmetric c x c matrix A (row-major, device): FP32
// start, kRefineSteps Ogita-Aishima steps and kOrthSteps Newton-Schulz steps
// in FP64, ping-ponging between Ua and Ub; the result lands in Ua.
// state[j] != 0 turns step j into no-ops (state[0] also the FP32 start): the
// caller clears state[0..kEigSteps) or sets it to skip everything, and a step
// whose correction is below kConverged sets the flags of all later steps.
static cudaError_t eigvecs(const double *A, int c, double *Ua, double *Ub, double floor_norm,
                           int *state, const Layout &L, cudaStream_t st) {
  cudaError_t e;
#define HATT_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  HATT_TRY(cudaFuncSetAttribute(eig_tridiag32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)eig_smem(kMaxSmall)));
  launch_k(eig_tridiag32_kernel, 1, kEigThreads, eig_smem(c), st, A, c, Ua, state);
  note_launch();
  HATT_TRY(cudaGetLastError());
  if (c <= kEigFusedMax) {          // all refinement steps in one cluster launch
    bool ok = false;
    HATT_TRY(refine_cluster_available(&ok));
    if (ok) return refine_cluster(A, c, Ua, floor_norm, state, st);
  }
  double *U = Ua, *Un = Ub;
  for (int it = 0; it < kEigSteps; ++it) {
    const int orth_only = (it >= kRefineSteps);   // closing steps: orthonormalize only
    Gemm g = g_tn(U, U, c, c, c, L.UtU, c);
    g.skip_dev = state + it;
    HATT_TRY(gemm_f64(g, L.gs, st));
    if (!orth_only) {
      g = g_nn(A, U, c, c, c, L.T);
      g.skip_dev = state + it;
      HATT_TRY(gemm_f64(g, L.gs, st));
      g = g_tn(U, L.T, c, c, c, L.S, c);
      g.skip_dev = state + it;
      HATT_TRY(gemm_f64(g, L.gs, st));
    }
    launch_k(oa_update_kernel, 1, kOaThreads, 0, st, L.UtU, L.S, A, c, orth_only, floor_norm, state, it,
                                                kEigSteps, L.E);
    note_launch();
    HATT_TRY(cudaGetLastError());
    g = g_nn(U, L.E, c, c, c, Un);
    g.skip_dev = state + it;
    HATT_TRY(gemm_f64(g, L.gs, st));
    std::swap(U, Un);
  }
  static_assert(kEigSteps % 2 == 0, "with every step applied the result is in Ua");
  launch_k(select_result_kernel, 4, kThreads, 0, st, state, kEigSteps, Ub, Ua, c * c);
  note_launch();
  HATT_TRY(cudaGetLastError());
#undef HATT_TRY
  return cudaSuccess;
}

cudaError_t trunc_step(double *Xk, int la, int n, int lb, double *Xkm1, int lm, int nm, int cap,
                       const double *delta2_dev, long long *ranks_dev, int k, bool deep,
                       double *scratch, cudaStream_t st) {
  if (la > kMaxSmall) return cudaErrorInvalidValue;
  const long long N = (long long)n * lb;
  const long long mrows = (long long)lm * nm;
  Layout L = carve(scratch, la, N, mrows);
  cudaError_t e;
#define HATT_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  int *state1 = L.flags + 8, *state2 = L.flags + 16;
  HATT_TRY(gemm_f64(g_gram(Xk, la, N, L.G), L.gs, st));
  HATT_TRY(cudaMemsetAsync(state1, 0, kEigSteps * sizeof(int), st));
  HATT_TRY(eigvecs(L.G, la, L.U0, L.U1, 0.0, state1, L, st));
  double *U = L.U0;
  HATT_TRY(gemm_f64(g_tn(U, Xk, la, N, N, L.B1, N), L.gs, st));
  if (deep) {
    // further levels on the low-energy rows of B1, then the cross step
    double *Ua = L.U0, *Ub = L.U1;       // Ua holds the current U
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HATT_TRY(cudaStreamIsCapturing(st, &cs));
    const bool host_exit = t_host_sync && cs == cudaStreamCaptureStatusNone;
    for (int level = 0; level < kLevels; ++level) {
      Gemm g = g_gram(L.B1, la, N, L.G);                                        // G1 = B1 B1^T
      if (level > 0) g.skip_dev = L.flags;
      HATT_TRY(gemm_f64(g, L.gs, st));
      launch_k(level_prep_kernel, 1, kThreads, 0, st, L.G, la, cap, delta2_dev, level, L.scale, L.H,
                                                L.V0, L.flags, state2);
      note_launch();
      HATT_TRY(cudaGetLastError());
      if (host_exit) {
        int skip = 0;
        HATT_TRY(cudaMemcpyAsync(&skip, L.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        HATT_TRY(cudaStreamSynchronize(st));
        if (skip) break;
      }
      HATT_TRY(eigvecs(L.H, la, L.V0, L.V1, 1.0, state2, L, st));
      HATT_TRY(gemm_f64(g_nn(Ua, L.V0, la, la, la, Ub), L.gs, st));              // Ub = Ua V
      g = g_tn(Ub, Xk, la, N, N, L.B1, N);                                      // B1 = Ub^T B
      g.skip_dev = L.flags;               // skipped level: V = I, B1 is already Ua^T B
      HATT_TRY(gemm_f64(g, L.gs, st));
      std::swap(Ua, Ub);
    }
    Gemm g = g_gram(L.B1, la, N, L.G);                                          // G1 = B1 B1^T
    g.skip_dev = L.flags + 1;
    HATT_TRY(gemm_f64(g, L.gs, st));
    launch_k(cross_kernel, 1, kOaThreads, 0, st, L.G, la, L.flags, L.E);
    note_launch();
    HATT_TRY(cudaGetLastError());
    HATT_TRY(gemm_f64(g_nn(Ua, L.E, la, la, la, Ub), L.gs, st));               // Ub = Ua (I + E)
    std::swap(Ua, Ub);
    for (int it = 0; it < 2; ++it) {                                            // orthonormalize
      HATT_TRY(gemm_f64(g_tn(Ua, Ua, la, la, la, L.UtU, la), L.gs, st));
      launch_k(oa_update_kernel, 1, kOaThreads, 0, st, L.UtU, L.S, L.G, la, 1, 0.0, nullptr, 0, 0, L.E);
      note_launch();
      HATT_TRY(cudaGetLastError());
      HATT_TRY(gemm_f64(g_nn(Ua, L.E, la, la, la, Ub), L.gs, st));
      std::swap(Ua, Ub);
    }
    g = g_tn(Ua, Xk, la, N, N, L.B1, N);                                        // B1 = U^T B
    g.skip_dev = L.flags + 2;
    HATT_TRY(gemm_f64(g, L.gs, st));
    U = Ua;
  }
  launch_k(rownorm_kernel, la, kThreads, 0, st, L.B1, N, L.e);
  note_launch();
  HATT_TRY(cudaGetLastError());
  launch_k(rank_kernel, 1, kThreads, 0, st, L.e, la, cap, delta2_dev, ranks_dev, k, L.perm, L.sigma);
  note_launch();
  HATT_TRY(cudaGetLastError());
  const long long tot = (long long)la * N;
  const int blocks = (int)std::min<long long>((tot + kThreads - 1) / kThreads, 8 * 152);
  launch_k(newcore_kernel, blocks, kThreads, 0, st, L.B1, la, N, L.perm, L.sigma, ranks_dev, k, Xk);
  note_launch();
  HATT_TRY(cudaGetLastError());
  launch_k(kmat_kernel, (la * la + kThreads - 1) / kThreads, kThreads, 0, st, U, la, L.perm, L.sigma,
                                                                         ranks_dev, k, L.K);
  note_launch();
  HATT_TRY(cudaGetLastError());
  HATT_TRY(gemm_f64(g_nn(Xkm1, L.K, mrows, la, la, L.tmp), L.gs, st));
  HATT_TRY(copy_f64(L.tmp, Xkm1, mrows * la, st));
#undef HATT_TRY
  return cudaSuccess;
}

// Eigenvectors of a symmetric c x c matrix G (columns of U), the same FP32
// start and FP64 refinement as the truncation sweep uses.
void set_host_sync(bool allowed) { t_host_sync = allowed; }

size_t sym_eig_scratch_doubles(int c) {
  size_t gs = 0;
  gs = std::max(gs, gemm_scratch_doubles(g_tn(nullptr, nullptr, c, c, c, nullptr, c)));
  gs = std::max(gs, gemm_scratch_doubles(g_nn(nullptr, nullptr, c, c, c, nullptr)));
  return carve_doubles(c, 1, 1) + gs;
}

cudaError_t sym_eig(const double *G, int c, double *U, double *scratch, cudaStream_t st) {
  if (c < 1 || c > kMaxSmall) return cudaErrorInvalidValue;
  Layout L = carve(scratch, c, 1, 1);
  int *state = L.flags + 8;
  cudaError_t e = cudaMemsetAsync(state, 0, kEigSteps * sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = eigvecs(G, c, L.U0, L.U1, 0.0, state, L, st);
  if (e != cudaSuccess) return e;
  return copy_f64(L.U0, U, (long long)c * c, st);
}

cudaError_t trunc_delta2(const double *x, long long count, double tol, int d, double *delta2_dev,
                         double *partials, unsigned int *ticket, cudaStream_t st) {
  const int blocks = (int)std::max<long long>(1, std::min<long long>((count + kThreads - 1) / kThreads, 2 * 152));
  launch_k(delta2_kernel, blocks, kThreads, 0, st, x, count, tol, d, delta2_dev, partials, ticket);
  note_launch();
  return cudaGetLastError();
}

cudaError_t set_ranks(long long *ranks_dev, const long long *ranks_host, int count,
                      cudaStream_t st) {
  if (count > kMaxOrder + 1) return cudaErrorInvalidValue;
  RankTable t;
  t.count = count;
  for (int i = 0; i < count; ++i) t.r[i] = ranks_host[i];
  launch_k(set_ranks_kernel, 1, 256, 0, st, t, ranks_dev);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hatt
