// Right-to-left truncation sweep of a left-orthogonal TT (max_rank / tol).
//
// For core k with horizontal unfolding B = H(X_k) (la x N, N = n lb) and all
// cores to its left orthonormal, the singular values of B are those of the
// full unfolding at bond k. One step:
//   1. G = B B^T                                   (FP64 GEMM, all SMs)
//   2. eigenvectors of G by cyclic Jacobi in FP32   (one block; the FP32 pipe
//      of GB300 is ~60x its FP64 pipe, and this is the only serial stage)
//   3. three Ogita-Aishima refinement steps in FP64 (Ogita & Aishima, "Iterative
//      refinement for symmetric eigenvalue decomposition", JJIAM 2018):
//      R = I - U^T U, S = U^T G U, l_i = s_ii/(1 - r_ii),
//      E_ij = (s_ij + l_j r_ij)/(l_j - l_i) for separated pairs, r_ij/2 otherwise,
//      U <- U (I + E); quadratic convergence from the FP32 start. A last
//      step with E = R/2 for every pair makes U orthonormal to working
//      accuracy whatever the eigenvalue gaps
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

constexpr int kJacThreads = 256;
constexpr int kMaxSweeps = 12;
constexpr int kOaThreads = 1024;
constexpr int kThreads = 256;
constexpr int kRefineSteps = 3;

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

// Cyclic Jacobi (round-robin ordering, c/2 disjoint rotations per round) on
// the trace-scaled Gram matrix in FP32. Output: U (c x c, FP64, columns =
// eigenvectors sorted by decreasing eigenvalue). A round computes its c/2
// rotations once, then applies both sides at once, 2 x 2 block by 2 x 2 block,
// from one copy of A into the other (J^T A J restricted to the rows of pair j
// and the columns of pair j' depends only on that block), so a round costs two
// barriers. The result only seeds the FP64 refinement, which converges
// quadratically from it.
__global__ void __launch_bounds__(kJacThreads)
jacobi_eig32_kernel(const double *G, int c, double *U) {
  extern __shared__ float fs[];
  const int ld = c + 1;
  float *Ab0 = fs;                // c x ld
  float *Ab1 = fs + c * ld;       // c x ld
  float *V = fs + 2 * c * ld;     // c x ld
  float *rc = V + c * ld;         // rotation cosines   [c/2 + 1]
  float *rs = rc + (c / 2 + 1);   // rotation sines
  int *pp = (int *)(rs + (c / 2 + 1));
  int *pq = pp + (c / 2 + 1);
  __shared__ double red[kJacThreads];
  const int tid = threadIdx.x;

  double tr = 0.0;
  for (int i = tid; i < c; i += kJacThreads) tr += G[i * c + i];
  tr = block_sum(tr, red);
  const double scale = tr > 0.0 ? 1.0 / tr : 1.0;
  for (int e = tid; e < c * c; e += kJacThreads) {
    const int i = e / c, j = e % c;
    Ab0[i * ld + j] = (float)(0.5 * (G[i * c + j] + G[j * c + i]) * scale);
    V[i * ld + j] = (i == j) ? 1.0f : 0.0f;
  }
  __syncthreads();
  float *A = Ab0, *An = Ab1;
  const int N = c + (c & 1);       // players of the round-robin (a dummy if c is odd)
  const int P = N / 2;
  // 16 x 16 thread grid: items are walked without integer division
  const int tx = tid % 16, ty = tid / 16;
  __shared__ float wsum[2][kJacThreads / 32];
  for (int sweep = 0; sweep < kMaxSweeps && N > 1; ++sweep) {
    float offf = 0.0f, totf = 0.0f;
    for (int i = ty; i < c; i += 16)
      for (int j = tx; j < c; j += 16) {
        const float v = A[i * ld + j];
        totf = fmaf(v, v, totf);
        if (i != j) offf = fmaf(v, v, offf);
      }
    for (int o = 16; o > 0; o >>= 1) {
      offf += __shfl_xor_sync(0xffffffffu, offf, o);
      totf += __shfl_xor_sync(0xffffffffu, totf, o);
    }
    if ((tid & 31) == 0) { wsum[0][tid >> 5] = offf; wsum[1][tid >> 5] = totf; }
    __syncthreads();
    float off = 0.0f, tot = 0.0f;
    for (int w = 0; w < kJacThreads / 32; ++w) { off += wsum[0][w]; tot += wsum[1][w]; }
    __syncthreads();
    // squared off-diagonal mass <= 1e-11 of the total: a relative residual of
    // ~3e-6, from which three FP64 refinement steps reach working accuracy even
    // for closely spaced eigenvalues (FP32 reaches it in ~6 sweeps at c = 50)
    if (off <= 1e-11f * tot || tot == 0.0f) break;
    for (int round = 0; round < N - 1; ++round) {
      if (tid < P) {
        const int j = tid;
        int p, q;
        if (j == 0) { p = round % (N - 1); q = N - 1; }
        else { p = (round + j) % (N - 1); q = (round - j + (N - 1)) % (N - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        float cs = 1.0f, sn = 0.0f;
        if (q < c) {
          const float apq = A[p * ld + q];
          const float app = A[p * ld + p], aqq = A[q * ld + q];
          if (fabsf(apq) > 1e-30f && fabsf(apq) > 1e-9f * sqrtf(fabsf(app * aqq))) {
            // correctly rounded divide / sqrt: c^2 + s^2 = 1 to FP32 rounding,
            // so rotations stay orthogonal and the stop test is reachable
            const float tau = (aqq - app) / (2.0f * apq);
            const float t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
            cs = 1.0f / sqrtf(fmaf(t, t, 1.0f));
            sn = t * cs;
          }
        }
        rc[j] = cs; rs[j] = sn; pp[j] = p; pq[j] = q;
      }
      __syncthreads();
      // A' = J^T A J block by block: rows of pair j, columns of pair jj
      for (int j = ty; j < P; j += 16) {
        const int p = pp[j], q = pq[j];
        const float cs = rc[j], sn = rs[j];
        const bool hq = q < c;
        for (int jj = tx; jj < P; jj += 16) {
          const int p2 = pp[jj], q2 = pq[jj];
          const float cs2 = rc[jj], sn2 = rs[jj];
          const bool hq2 = q2 < c;
          const float a = A[p * ld + p2];
          const float b = hq2 ? A[p * ld + q2] : 0.0f;
          const float cc = hq ? A[q * ld + p2] : 0.0f;
          const float dd = (hq && hq2) ? A[q * ld + q2] : 0.0f;
          const float a1 = cs2 * a - sn2 * b, b1 = sn2 * a + cs2 * b;
          const float c1 = cs2 * cc - sn2 * dd, d1 = sn2 * cc + cs2 * dd;
          An[p * ld + p2] = cs * a1 - sn * c1;
          if (hq2) An[p * ld + q2] = cs * b1 - sn * d1;
          if (hq) An[q * ld + p2] = sn * a1 + cs * c1;
          if (hq && hq2) An[q * ld + q2] = sn * b1 + cs * d1;
        }
      }
      // V <- V J (columns of each pair, in place; pairs are disjoint)
      for (int j = ty; j < P; j += 16) {
        const int p = pp[j], q = pq[j];
        const float sn = rs[j];
        if (q >= c || sn == 0.0f) continue;
        const float cs = rc[j];
        for (int i = tx; i < c; i += 16) {
          const float va = V[i * ld + p], vb = V[i * ld + q];
          V[i * ld + p] = cs * va - sn * vb;
          V[i * ld + q] = sn * va + cs * vb;
        }
      }
      __syncthreads();
      float *tmp = A; A = An; An = tmp;
    }
  }
  // sort eigenvalues (diagonal) in decreasing order; ties by index
  for (int i = tid; i < c; i += kJacThreads) {
    const float li = A[i * ld + i];
    int pos = 0;
    for (int j = 0; j < c; ++j) {
      const float lj = A[j * ld + j];
      pos += (lj > li) || (lj == li && j < i);
    }
    for (int r = 0; r < c; ++r) U[r * c + pos] = (double)V[r * ld + i];
  }
}

// One Ogita-Aishima step: given UtU (= U^T U), S (= U^T G U) and G, write
// Eout = I + E (so that the next U is U * Eout). The cluster threshold is
// floored at the rounding level of ||G||: eigenvalues that agree to working
// accuracy (exact degeneracies, e.g. the equal singular values of
// sin(2x+2y) = sin 2x cos 2y + cos 2x sin 2y) are only orthogonalized, never
// rotated by a quotient of two rounding errors.
// With orth_only set, every pair is treated as clustered: E = (I - U^T U)/2,
// one Newton-Schulz orthonormalization step (S and G are not read).
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
                 double *Eout) {
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
      s_delta = fmax(2.0 * (sqrt(s) + gn * sqrt(b)), 64.0 * c * u * gn);
      s_inv = gn > 0.0 ? rcp_newton(gn) : 1.0;
    }
    __syncthreads();
  }
  const double delta = orth_only ? 0.0 : s_delta;
  const double inv = orth_only ? 1.0 : s_inv;
  for (int i = tid / 32; i < c; i += kOaThreads / 32)
    for (int j = tid % 32; j < c; j += 32) {
      const int e = i * c + j;
      const double r = (i == j ? 1.0 : 0.0) - UtU[e];
      double E;
      if (!orth_only && i != j && fabs(lam[i] - lam[j]) > delta) {
        const float num = (float)(fma(lam[j], r, S[e]) * inv);
        const float den = (float)((lam[j] - lam[i]) * inv);
        E = (double)__fdividef(num, den);
      } else {
        E = 0.5 * r;
      }
      Eout[e] = E + (i == j ? 1.0 : 0.0);
    }
}

__global__ void __launch_bounds__(kThreads)
rownorm_kernel(const double *B1, long long N, double *e) {
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
  __shared__ double sorted[kMaxSmall];
  const int tid = threadIdx.x;
  for (int i = tid; i < c; i += kThreads) {
    const double ei = e[i];
    int pos = 0;
    for (int j = 0; j < c; ++j) {
      const double ej = e[j];
      pos += (ej > ei) || (ej == ei && j < i);
    }
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
    double tails[kMaxSmall + 1];
    tails[c] = 0.0;
    for (int p = c - 1; p >= 0; --p) {
      tail += fmax(sorted[p], 0.0);
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
  const int rho = (int)ranks[k];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < c * c; t += gridDim.x * blockDim.x) {
    const int l = t / c, j = t % c;
    K[t] = (j < rho) ? U[l * c + perm[j]] * sigma[j] : 0.0;
  }
}

__global__ void __launch_bounds__(kThreads)
delta2_kernel(const double *x, long long count, double tol, int d, double *out, double *partials,
              unsigned int *ticket) {
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
  for (int i = threadIdx.x; i < t.count; i += blockDim.x) ranks[i] = t.r[i];
}

size_t jac_smem(int c) {
  const int P = c / 2 + 1;
  return (size_t)3 * c * (c + 1) * sizeof(float) + 2 * P * sizeof(float) + 2 * P * sizeof(int);
}

struct Layout {
  double *G, *U0, *U1, *UtU, *T, *S, *E, *B1, *e, *sigma, *K, *tmp, *gs;
  int *perm;
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
  L.e = p; p += la;
  L.sigma = p; p += la;
  L.perm = (int *)p; p += la;
  L.B1 = p; p += (size_t)la * N;
  L.tmp = p; p += (size_t)mrows * la;
  L.gs = p;
  return L;
}

size_t carve_doubles(int la, long long N, long long mrows) {
  return (size_t)8 * la * la + 3 * (size_t)la + (size_t)la * N + (size_t)mrows * la;
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

cudaError_t trunc_step(double *Xk, int la, int n, int lb, double *Xkm1, int lm, int nm, int cap,
                       const double *delta2_dev, long long *ranks_dev, int k, double *scratch,
                       cudaStream_t st) {
  if (la > kMaxSmall) return cudaErrorInvalidValue;
  const long long N = (long long)n * lb;
  const long long mrows = (long long)lm * nm;
  Layout L = carve(scratch, la, N, mrows);
  cudaError_t e;
#define HATT_TRY(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
  HATT_TRY(gemm_f64(g_gram(Xk, la, N, L.G), L.gs, st));
  HATT_TRY(cudaFuncSetAttribute(jacobi_eig32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)jac_smem(kMaxSmall)));
  jacobi_eig32_kernel<<<1, kJacThreads, jac_smem(la), st>>>(L.G, la, L.U0);
  note_launch();
  HATT_TRY(cudaGetLastError());
  double *U = L.U0, *Un = L.U1;
  for (int it = 0; it <= kRefineSteps; ++it) {
    const int orth_only = (it == kRefineSteps);   // last step: orthonormalize only
    HATT_TRY(gemm_f64(g_tn(U, U, la, la, la, L.UtU, la), L.gs, st));
    if (!orth_only) {
      HATT_TRY(gemm_f64(g_nn(L.G, U, la, la, la, L.T), L.gs, st));
      HATT_TRY(gemm_f64(g_tn(U, L.T, la, la, la, L.S, la), L.gs, st));
    }
    oa_update_kernel<<<1, kOaThreads, 0, st>>>(L.UtU, L.S, L.G, la, orth_only, L.E);
    note_launch();
    HATT_TRY(cudaGetLastError());
    HATT_TRY(gemm_f64(g_nn(U, L.E, la, la, la, Un), L.gs, st));
    std::swap(U, Un);
  }
  HATT_TRY(gemm_f64(g_tn(U, Xk, la, N, N, L.B1, N), L.gs, st));
  rownorm_kernel<<<la, kThreads, 0, st>>>(L.B1, N, L.e);
  note_launch();
  HATT_TRY(cudaGetLastError());
  rank_kernel<<<1, kThreads, 0, st>>>(L.e, la, cap, delta2_dev, ranks_dev, k, L.perm, L.sigma);
  note_launch();
  HATT_TRY(cudaGetLastError());
  const long long tot = (long long)la * N;
  const int blocks = (int)std::min<long long>((tot + kThreads - 1) / kThreads, 8 * 152);
  newcore_kernel<<<blocks, kThreads, 0, st>>>(L.B1, la, N, L.perm, L.sigma, ranks_dev, k, Xk);
  note_launch();
  HATT_TRY(cudaGetLastError());
  kmat_kernel<<<(la * la + kThreads - 1) / kThreads, kThreads, 0, st>>>(U, la, L.perm, L.sigma,
                                                                         ranks_dev, k, L.K);
  note_launch();
  HATT_TRY(cudaGetLastError());
  HATT_TRY(gemm_f64(g_nn(Xkm1, L.K, mrows, la, la, L.tmp), L.gs, st));
  HATT_TRY(copy_f64(L.tmp, Xkm1, mrows * la, st));
#undef HATT_TRY
  return cudaSuccess;
}

cudaError_t trunc_delta2(const double *x, long long count, double tol, int d, double *delta2_dev,
                         double *partials, unsigned int *ticket, cudaStream_t st) {
  const int blocks = (int)std::max<long long>(1, std::min<long long>((count + kThreads - 1) / kThreads, 2 * 152));
  delta2_kernel<<<blocks, kThreads, 0, st>>>(x, count, tol, d, delta2_dev, partials, ticket);
  note_launch();
  return cudaGetLastError();
}

cudaError_t set_ranks(long long *ranks_dev, const long long *ranks_host, int count,
                      cudaStream_t st) {
  if (count > kMaxOrder + 1) return cudaErrorInvalidValue;
  RankTable t;
  t.count = count;
  for (int i = 0; i < count; ++i) t.r[i] = ranks_host[i];
  set_ranks_kernel<<<1, 256, 0, st>>>(t, ranks_dev);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hatt
