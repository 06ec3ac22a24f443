// TT operations of the Allen-Cahn application (Section 5, Example 4):
// the periodic second-difference Laplacian applied to a TT, and linear
// combinations of TTs. Both only assemble block cores (elementwise work).
// Also the selection of the leading singular directions of HPCRL-2 (Eq. (3.7)).
#include <algorithm>
#include "hatt_internal.cuh"

namespace hatt {
namespace {

constexpr int kOpThreads = 256;

int op_grid(long long count) {
  return (int)std::max<long long>(1, std::min<long long>((count + kOpThreads - 1) / kOpThreads, 8 * 152));
}

// (D u)(alpha, i, beta) = (u(alpha, i+1, beta) - 2 u(alpha, i, beta) + u(alpha, i-1, beta)) / h^2,
// indices modulo n (periodic).
__device__ __forceinline__ double stencil(const double *u, int n, int b, int alpha, int i,
                                          int beta, double inv_h2) {
  const int ip = (i + 1 == n) ? 0 : i + 1, im = (i == 0) ? n - 1 : i - 1;
  const long long row = (long long)alpha * n;
  return (u[(row + ip) * b + beta] - 2.0 * u[(row + i) * b + beta] + u[(row + im) * b + beta]) * inv_h2;
}

// Core k of Lap u. pos: 0 = only core (D u), 1 = first [u | D u],
// 2 = middle [[u, D u], [0, u]], 3 = last [[D u], [u]]. u is a x n x b.
__global__ void laplacian_core_kernel(const double *u, int a, int n, int b, int pos,
                                      double inv_h2, double *out) {
  pdl_enter();
  const int oa = (pos == 2 || pos == 3) ? 2 * a : a;
  const int ob = (pos == 1 || pos == 2) ? 2 * b : b;
  const long long total = (long long)oa * n * ob;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int beta = (int)(t % ob);
    const long long r = t / ob;
    const int i = (int)(r % n), alpha = (int)(r / n);
    double v = 0.0;
    if (pos == 0) {
      v = stencil(u, n, b, alpha, i, beta, inv_h2);
    } else if (pos == 1) {
      v = beta < b ? u[((long long)alpha * n + i) * b + beta] : stencil(u, n, b, alpha, i, beta - b, inv_h2);
    } else if (pos == 3) {
      v = alpha < a ? stencil(u, n, b, alpha, i, beta, inv_h2) : u[((long long)(alpha - a) * n + i) * b + beta];
    } else {
      const bool top = alpha < a, left = beta < b;
      if (top && left) v = u[((long long)alpha * n + i) * b + beta];
      else if (top) v = stencil(u, n, b, alpha, i, beta - b, inv_h2);
      else if (!left) v = u[((long long)(alpha - a) * n + i) * b + (beta - b)];
    }
    out[t] = v;
  }
}

// Writes coef * src (a x n x b) into the block of dst (A x n x B) whose top
// left corner is (ra, rb), or adds it there when accumulate is set.
__global__ void put_block_kernel(const double *src, int a, int n, int b, double coef, double *dst,
                                 int A, int B, int ra, int rb, int accumulate) {
  pdl_enter();
  const long long total = (long long)a * n * b;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int beta = (int)(t % b);
    const long long r = t / b;
    const int i = (int)(r % n), alpha = (int)(r / n);
    double *d = dst + ((long long)(ra + alpha) * n + i) * B + rb + beta;
    *d = accumulate ? fma(coef, src[t], *d) : coef * src[t];
  }
}

// HPCRL-2 selection. Uf = W V (x rows, c columns) holds W's right singular
// directions scaled by their singular values: column j has squared norm
// e_j = sigma_j^2. Keeps the columns with sigma_j > ep * sigma_max (at least
// one), in descending order of e_j (ties by index), and writes them into the
// first R columns of UR (x x c) = U_R S_R and VR (c x c) = V_R, leading
// dimension c; R goes to device memory, where the contractions that follow
// read it (their extents in R are device-side), so nothing waits on the host.
// Columns R .. c - 1 are left as they are: nothing reads them.
// One block: warp w sums the columns w, w + 32, ... in a fixed order, so the
// decision is the same on every run.
constexpr int kSelThreads = 1024;

__global__ void __launch_bounds__(kSelThreads)
select_directions_kernel(const double *Uf, const double *V, long long x, int c, double ep,
                         double *UR, double *VR, int *Rout) {
  pdl_enter();
  __shared__ double e[kMaxSmall];
  __shared__ int pos[kMaxSmall];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = warp; j < c; j += kSelThreads / 32) {
    double acc = 0.0;
    for (long long r = lane; r < x; r += 32) {
      const double v = Uf[r * c + j];
      acc = fma(v, v, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) e[j] = acc;
  }
  __syncthreads();
  double emax = 0.0;
  for (int j = 0; j < c; ++j) emax = fmax(emax, e[j]);
  const double thr = ep * ep * emax;
  int top = 0;   // index of the largest column (kept when nothing passes)
  for (int j = 1; j < c; ++j)
    if (e[j] > e[top]) top = j;
  for (int j = tid; j < c; j += kSelThreads) {
    const bool keep = e[j] > thr || j == top;
    int p = -1;
    if (keep) {
      p = 0;
      for (int i = 0; i < c; ++i) {
        const bool ki = e[i] > thr || i == top;
        if (ki && (e[i] > e[j] || (e[i] == e[j] && i < j))) ++p;
      }
    }
    pos[j] = p;
  }
  __syncthreads();
  if (tid == 0) {
    int R = 0;
    for (int j = 0; j < c; ++j) R += pos[j] >= 0;
    *Rout = R;
  }
  for (long long t = tid; t < x * c; t += kSelThreads) {
    const int j = (int)(t % c);
    if (pos[j] >= 0) UR[(t / c) * c + pos[j]] = Uf[t];
  }
  for (int t = tid; t < c * c; t += kSelThreads) {
    const int j = t % c;
    if (pos[j] >= 0) VR[(t / c) * c + pos[j]] = V[t];
  }
}

}  // namespace

cudaError_t laplacian_core(const double *u, int a, int n, int b, int pos, double inv_h2,
                           double *out, cudaStream_t st) {
  const int oa = (pos == 2 || pos == 3) ? 2 * a : a;
  const int ob = (pos == 1 || pos == 2) ? 2 * b : b;
  launch_k(laplacian_core_kernel, op_grid((long long)oa * n * ob), kOpThreads, 0, st, u, a, n, b, pos,
                                                                               inv_h2, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t put_block(const double *src, int a, int n, int b, double coef, double *dst, int A,
                      int B, int ra, int rb, bool accumulate, cudaStream_t st) {
  launch_k(put_block_kernel, op_grid((long long)a * n * b), kOpThreads, 0, st, src, a, n, b, coef, dst,
                                                                        A, B, ra, rb, accumulate);
  note_launch();
  return cudaGetLastError();
}

cudaError_t select_directions(const double *Uf, const double *V, long long x, int c, double ep,
                              double *UR, double *VR, int *R, cudaStream_t st) {
  if (c < 1 || c > kMaxSmall) return cudaErrorInvalidValue;
  launch_k(select_directions_kernel, 1, kSelThreads, 0, st, Uf, V, x, c, ep, UR, VR, R);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hatt
