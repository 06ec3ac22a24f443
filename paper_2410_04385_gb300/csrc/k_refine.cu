// FP64 refinement of symmetric eigenvectors in one launch on a thread-block
// cluster (the eigen solves of the truncation sweep and of HPCRL-2's
// selection, for matrices up to kEigFusedMax): the Ogita-Aishima steps
// (Ogita & Aishima, JJIAM 2018) R = I - U^T U, S = U^T G U,
// l_i = s_ii / (1 - r_ii), E_ij = (s_ij + l_j r_ij) / (l_j - l_i) for
// separated pairs (rotations above 0.1 left out) and r_ij / 2 otherwise,
// U <- U (I + E), then Newton-Schulz steps E = R / 2, stopping after the
// first step whose correction is below 1e-9 -- the same steps and test as
// the launch-per-step path (four GEMM launches and one update launch per
// step, the later steps turned into no-ops by a device flag). Here one launch
// runs them all: CTA r of the cluster owns a slice of the columns of R, S and
// the new U, every CTA holds G and U whole in shared memory, slices and
// per-CTA norms travel through distributed shared memory (three cluster
// barriers per step), and the steps after convergence are not run at all.
// The FP32 start comes from the tridiagonal solver (k_trunc.cu) in U.
//
// FP64 arithmetic on GB300 runs on two lanes per SM: scalar FP64 work is done
// by one thread and broadcast through shared memory, never repeated by every
// thread. No spin-waits: hardware block and cluster barriers only, reached
// the same number of times by every CTA (the step count comes from values
// every CTA reads from the same shared words).
#include <cooperative_groups.h>
#include <algorithm>
#include <mutex>
#include "hatt_internal.cuh"

namespace cg = cooperative_groups;

namespace hatt {
namespace {

constexpr int kThreadsE = 512;
constexpr int kRefine = 3;          // Ogita-Aishima steps
constexpr int kOrth = 3;            // closing Newton-Schulz steps
constexpr double kStepConverged = 1e-9;
constexpr int kMaxCluster = 16;

// Block-wide sum / max of one double per thread. Only the warp shuffles run
// in every thread; the final combination of the per-warp values runs in
// thread 0 and is broadcast through shared memory: on GB300 every FP64
// instruction that all 512 threads execute costs the SM ~256 clocks.
__device__ __forceinline__ double blk_reduce(double v, double *red, bool is_max) {
  for (int o = 16; o > 0; o >>= 1) {
    const double x = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, x) : v + x;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = is_max ? fmax(t, red[i]) : t + red[i];
    red[32] = t;
  }
  __syncthreads();
  return red[32];
}


// U (c x c, row-major, device) holds the start on entry and the refined
// eigenvectors on return; *skip != 0 leaves it untouched.
__global__ void __launch_bounds__(kThreadsE, 1)
oa_cluster_kernel(const double *G, int c, double *Uout, double floor_norm, const int *skip) {
  pdl_enter();
  if (skip && *skip) return;           // every CTA reads the same word
  cg::cluster_group cl = cg::this_cluster();
  const int P = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x;
  const int w = (c + P - 1) / P;
  const int j0 = min(c, rank * w), j1 = min(c, j0 + w), wl = j1 - j0;
  extern __shared__ __align__(16) double sm[];
  double *Gs = sm;                     // c x c
  double *Us = Gs + c * c;             // c x c
  double *lam = Us + c * c;            // c
  double *part = lam + c;              // 3 x kMaxCluster
  double *work = part + 3 * kMaxCluster;
  double *Rs = work, *Ts = Rs + c * w, *Ss = Ts + c * w, *Ns = Ss + c * w;
  __shared__ double red[33];
  __shared__ double s_gn, s_delta, s_inv, s_stop;

  double g2 = 0.0;
  for (int e = tid; e < c * c; e += nt) {
    const double v = G[e];
    Gs[e] = v;
    Us[e] = Uout[e];
    g2 = fma(v, v, g2);
  }
  g2 = blk_reduce(g2, red, false);
  if (tid == 0) s_gn = sqrt(g2);
  cl.sync();                           // every CTA has started and loaded U
  const double u = 1.1102230246251565e-16;
  for (int it = 0; it < kRefine + kOrth; ++it) {
    const bool orth = it >= kRefine;
    // R = I - U^T U and T = G U on the own columns, then S = U^T T
    for (int e = tid; e < c * wl; e += nt) {
      const int i = e / wl, jj = e - i * wl, j = j0 + jj;
      double r = 0.0, t = 0.0;
      if (orth) {
        for (int k = 0; k < c; ++k) r = fma(Us[k * c + i], Us[k * c + j], r);
      } else {
        for (int k = 0; k < c; ++k) {
          const double ukj = Us[k * c + j];
          r = fma(Us[k * c + i], ukj, r);
          t = fma(Gs[i * c + k], ukj, t);
        }
      }
      Rs[i * w + jj] = ((i == j) ? 1.0 : 0.0) - r;
      Ts[i * w + jj] = t;
    }
    __syncthreads();
    if (!orth) {
      for (int e = tid; e < c * wl; e += nt) {
        const int i = e / wl, jj = e - i * wl;
        double s = 0.0;
        for (int k = 0; k < c; ++k) s = fma(Us[k * c + i], Ts[k * w + jj], s);
        Ss[i * w + jj] = s;
      }
      __syncthreads();
      for (int jj = tid; jj < wl; jj += nt) {      // l_j to every CTA
        const int j = j0 + jj;
        const double l = Ss[j * w + jj] / (1.0 - Rs[j * w + jj]);
        for (int q = 0; q < P; ++q) cl.map_shared_rank(lam, q)[j] = l;
      }
      double r2 = 0.0, s2 = 0.0;
      for (int e = tid; e < c * wl; e += nt) {
        const int i = e / wl, jj = e - i * wl, j = j0 + jj;
        const double r = Rs[i * w + jj];
        double sd = Ss[i * w + jj];
        if (i == j) sd -= Ss[j * w + jj] / (1.0 - Rs[j * w + jj]);
        r2 = fma(r, r, r2);
        s2 = fma(sd, sd, s2);
      }
      r2 = blk_reduce(r2, red, false);
      s2 = blk_reduce(s2, red, false);
      if (tid == 0)
        for (int q = 0; q < P; ++q) {
          double *pr = cl.map_shared_rank(part, q);
          pr[2 * rank] = r2;
          pr[2 * rank + 1] = s2;
        }
      cl.sync();
      if (tid == 0) {
        double R2 = 0.0, S2 = 0.0;
        for (int q = 0; q < P; ++q) {
          R2 += part[2 * q];
          S2 += part[2 * q + 1];
        }
        const double gn = s_gn;
        s_delta = fmax(2.0 * (sqrt(S2) + gn * sqrt(R2)),
                       64.0 * c * u * (floor_norm > 0.0 ? floor_norm : gn));
        s_inv = gn > 0.0 ? 1.0 / gn : 1.0;
      }
      __syncthreads();
    }
    const double delta = s_delta, inv = s_inv;
    // E (over R, in place), then the new columns U (I + E)
    double emax = 0.0;
    for (int e = tid; e < c * wl; e += nt) {
      const int i = e / wl, jj = e - i * wl, j = j0 + jj;
      const double r = Rs[i * w + jj];
      double E = 0.5 * r;
      if (!orth && i != j && fabs(lam[i] - lam[j]) > delta) {
        const float num = (float)(fma(lam[j], r, Ss[i * w + jj]) * inv);
        const float den = (float)((lam[j] - lam[i]) * inv);
        const float qv = __fdividef(num, den);
        if (fabsf(qv) <= 0.1f) E = (double)qv;
      }
      emax = fmax(emax, fabs(E));
      Rs[i * w + jj] = E;
    }
    __syncthreads();
    for (int e = tid; e < c * wl; e += nt) {
      const int i = e / wl, jj = e - i * wl, j = j0 + jj;
      double v = Us[i * c + j];
      for (int k = 0; k < c; ++k) v = fma(Us[i * c + k], Rs[k * w + jj], v);
      Ns[i * w + jj] = v;
    }
    emax = blk_reduce(emax, red, true);
    if (tid == 0)
      for (int q = 0; q < P; ++q) cl.map_shared_rank(part, q)[2 * kMaxCluster + rank] = emax;
    cl.sync();                         // every CTA has finished reading U
    for (int q = 0; q < P; ++q) {
      double *dst = cl.map_shared_rank(Us, q);
      for (int e = tid; e < c * wl; e += nt) {
        const int i = e / wl, jj = e - i * wl;
        dst[i * c + j0 + jj] = Ns[i * w + jj];
      }
    }
    cl.sync();
    if (tid == 0) {
      double mx = 0.0;
      for (int q = 0; q < P; ++q) mx = fmax(mx, part[2 * kMaxCluster + q]);
      s_stop = (mx <= kStepConverged) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (s_stop != 0.0) break;          // the same decision in every CTA
  }
  for (int e = tid; e < c * wl; e += nt) {
    const int i = e / wl, jj = e - i * wl;
    Uout[i * c + j0 + jj] = Us[i * c + j0 + jj];
  }
}

int cluster_size_for(int c) { return c >= 32 ? 16 : (c >= 8 ? 8 : 1); }

size_t refine_smem(int c, int P) {
  const int w = (c + P - 1) / P;
  return ((size_t)2 * c * c + c + 3 * kMaxCluster + (size_t)4 * c * w) * sizeof(double);
}

}  // namespace

namespace {
// Largest cluster (16, else 8) the device can place with the kernel's shared
// memory, found once per device; 0 when not even 8 fit (then the caller keeps
// the launch-per-step path).
int g_max_cluster[kMaxDevices];
bool g_max_cluster_known[kMaxDevices];

std::mutex g_cluster_mu;

cudaError_t max_cluster(int *out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_cluster_mu);
  if (g_max_cluster_known[dev]) {
    *out = g_max_cluster[dev];
    return cudaSuccess;
  }
  e = cudaFuncSetAttribute(oa_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)refine_smem(kEigFusedMax, kMaxCluster));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(oa_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  int best = 0;
  for (int P : {kMaxCluster, 8}) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P);
    cfg.blockDim = dim3(kThreadsE);
    cfg.dynamicSmemBytes = refine_smem(kEigFusedMax, P);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, oa_cluster_kernel, &cfg) == cudaSuccess &&
        clusters > 0) {
      best = P;
      break;
    }
    cudaGetLastError();
  }
  g_max_cluster[dev] = best;
  g_max_cluster_known[dev] = true;
  *out = best;
  return cudaSuccess;
}
}  // namespace

cudaError_t refine_cluster_available(bool *ok) {
  int P = 0;
  const cudaError_t e = max_cluster(&P);
  *ok = (e == cudaSuccess && P > 0);
  return e;
}

cudaError_t refine_cluster(const double *G, int c, double *U, double floor_norm, const int *skip,
                           cudaStream_t st) {
  if (c < 1 || c > kEigFusedMax) return cudaErrorInvalidValue;
  int Pmax = 0;
  cudaError_t e = max_cluster(&Pmax);
  if (e != cudaSuccess) return e;
  if (Pmax == 0) return cudaErrorNotSupported;
  const int P = std::min(cluster_size_for(c), Pmax);
  const size_t smem = refine_smem(c, P);
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(kThreadsE);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = programmatic_launch() ? 2 : 1;
  e = cudaLaunchKernelEx(&cfg, oa_cluster_kernel, G, c, U, floor_norm, skip);
  note_launch();
  return e;
}

}  // namespace hatt
