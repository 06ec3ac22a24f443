// Sketch generation (Definition 2.1), the first PKP core of Algorithm 4 and
// small utility kernels (norm scaling, copies, rank compaction).
#include <algorithm>
#include "hatt_internal.cuh"

namespace hatt {
namespace {

__device__ int g_misc_health = 0;   // kHealthNonfinite: a non-finite ||W^{(k)}||

constexpr int kThreads = 256;

// Philox4x32-10 (Salmon et al., SC'11): multipliers and Weyl key increments.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ void philox4x32_10(uint32_t x[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint32_t lo0 = kPhiloxM0 * x[0], hi0 = __umulhi(kPhiloxM0, x[0]);
    const uint32_t lo1 = kPhiloxM1 * x[2], hi1 = __umulhi(kPhiloxM1, x[2]);
    const uint32_t y0 = hi1 ^ x[1] ^ k0;
    const uint32_t y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
  }
}

// (k + 1/2) * 2^-52 with k the top 26 bits of two words: exact, in (0, 1).
__device__ __forceinline__ double uniform52(uint32_t hi, uint32_t lo) {
  return ((double)(hi >> 6) * 67108864.0 + (double)(lo >> 6) + 0.5) * 0x1p-52;
}

__device__ __forceinline__ double sketch_gaussian(uint32_t flat, uint32_t core, uint32_t pair,
                                                  uint32_t k0, uint32_t k1) {
  uint32_t x[4] = {flat, core, pair, 0u};
  philox4x32_10(x, k0, k1);
  const double u1 = uniform52(x[0], x[1]);
  const double u2 = uniform52(x[2], x[3]);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

__global__ void __launch_bounds__(kThreads) sketch_kernel(SketchTable t, double *base) {
  pdl_enter();
  const long long total = t.offset[t.d];
  const uint64_t key = t.seed + (t.seed_offset ? *t.seed_offset : 0ull);
  const uint32_t k0 = (uint32_t)(key & 0xFFFFFFFFull);
  const uint32_t k1 = (uint32_t)(key >> 32);
  for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < total;
       e += (long long)gridDim.x * kThreads) {
    int lo = 0, hi = t.d - 1;            // core k with offset[k] <= e < offset[k+1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (t.offset[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const long long flat = e - t.offset[lo];
    const double cnt = (double)t.a[lo] * (double)t.n[lo] * (double)t.b[lo];
    base[e] = sketch_gaussian((uint32_t)flat, (uint32_t)lo, t.pair, k0, k1) / sqrt(cnt);
  }
}

__global__ void __launch_bounds__(kThreads)
sketch_core_kernel(double *out, int a, int n, int b, uint32_t core, uint32_t pair,
                   uint64_t seed) {
  pdl_enter();
  const long long total = (long long)a * n * b;
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull);
  const uint32_t k1 = (uint32_t)(seed >> 32);
  const double cnt = (double)a * (double)n * (double)b;
  for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < total;
       e += (long long)gridDim.x * kThreads)
    out[e] = sketch_gaussian((uint32_t)e, core, pair, k0, k1) / sqrt(cnt);
}

__global__ void philox_raw_kernel(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                  long long count) {
  pdl_enter();
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < count;
       j += (long long)gridDim.x * blockDim.x) {
    uint32_t x[4] = {ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3]};
    philox4x32_10(x, k0, k1);
    out[4 * j] = x[0];
    out[4 * j + 1] = x[1];
    out[4 * j + 2] = x[2];
    out[4 * j + 3] = x[3];
  }
}

__global__ void __launch_bounds__(kThreads)
inv_norm_kernel(const double *x, long long count, double *out, double *partials,
                unsigned int *ticket) {
  pdl_enter();
  __shared__ double red[kThreads];
  __shared__ bool last;
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < count;
       e += (long long)gridDim.x * kThreads)
    s = fma(x[e], x[e], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = red[0];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) t += ((volatile double *)partials)[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double ss = red[0];
    if (!isfinite(ss)) atomicOr(&g_misc_health, kHealthNonfinite);
    out[0] = ss > 0.0 ? 1.0 / sqrt(ss) : 1.0;
    *ticket = 0u;
  }
}

__global__ void pkp_first_kernel(const double *Y, const double *Z, int n, int r1, int s1,
                                 double *C) {
  pdl_enter();
  const long long total = (long long)n * r1 * s1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % s1);
    const int a = (int)((e / s1) % r1);
    const int i = (int)(e / ((long long)r1 * s1));
    C[e] = Y[(long long)i * r1 + a] * Z[(long long)i * s1 + b];
  }
}

__global__ void set_kernel(double *x, long long count, double v) {
  pdl_enter();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    x[e] = v;
}

__global__ void eye_kernel(double *X, int m) {
  pdl_enter();
  const long long total = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    X[e] = (e / m == e % m) ? 1.0 : 0.0;
}

// x[i] /= *divisor (a device scalar, e.g. a norm just computed on the stream).
__global__ void div_kernel(double *x, long long count, const double *divisor) {
  pdl_enter();
  const double q = *divisor;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = x[i] / q;
}

__global__ void copy_kernel(const double *src, double *dst, long long count) {
  pdl_enter();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

__global__ void compact_kernel(const double *src, double *dst, int la, int n, int lb,
                               const long long *ranks, int k) {
  pdl_enter();
  const int ra = (int)ranks[k], rb = (int)ranks[k + 1];
  const long long total = (long long)ra * n * rb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % rb);
    const long long ai = e / rb;             // a * n + i
    dst[e] = src[ai * lb + b];
  }
}

__global__ void sqrt_kernel(const double *x, double *out) {
  pdl_enter();
  out[0] = sqrt(fmax(x[0], 0.0));
}

int grid_for(long long count) {
  return (int)std::max<long long>(1, std::min<long long>((count + kThreads - 1) / kThreads, 8 * 152));
}

}  // namespace

cudaError_t sketch_fill(const SketchTable &t, double *base, cudaStream_t st) {
  const long long total = t.offset[t.d];
  if (total <= 0) return cudaSuccess;
  launch_k(sketch_kernel, grid_for(total), kThreads, 0, st, t, base);
  note_launch();
  return cudaGetLastError();
}

cudaError_t sketch_fill_ptrs(int d, const int64_t *n, const int64_t *ell, uint64_t seed,
                             uint32_t pair, double *const *cores, cudaStream_t st) {
  for (int k = 0; k < d; ++k) {
    const long long total = (long long)ell[k] * n[k] * ell[k + 1];
    if (total <= 0) continue;
    launch_k(sketch_core_kernel, grid_for(total), kThreads, 0, st, 
        cores[k], (int)ell[k], (int)n[k], (int)ell[k + 1], (uint32_t)k, pair, seed);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t philox_raw(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                       long long count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  launch_k(philox_raw_kernel, grid_for(count), kThreads, 0, st, ctr, k0, k1, out, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t inv_norm(const double *x, long long count, double *out, double *partials,
                     unsigned int *ticket, cudaStream_t st) {
  const int blocks = (int)std::max<long long>(1, std::min<long long>((count + kThreads - 1) / kThreads, 2 * 152));
  launch_k(inv_norm_kernel, blocks, kThreads, 0, st, x, count, out, partials, ticket);
  note_launch();
  return cudaGetLastError();
}

cudaError_t pkp_first(const double *Y, const double *Z, int n, int r1, int s1, double *C,
                      cudaStream_t st) {
  const long long total = (long long)n * r1 * s1;
  launch_k(pkp_first_kernel, grid_for(total), kThreads, 0, st, Y, Z, n, r1, s1, C);
  note_launch();
  return cudaGetLastError();
}

cudaError_t set_value(double *x, long long count, double v, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  launch_k(set_kernel, grid_for(count), kThreads, 0, st, x, count, v);
  note_launch();
  return cudaGetLastError();
}

cudaError_t set_identity(double *X, int m, cudaStream_t st) {
  const long long total = (long long)m * m;
  if (total <= 0) return cudaSuccess;
  launch_k(eye_kernel, grid_for(total), kThreads, 0, st, X, m);
  note_launch();
  return cudaGetLastError();
}

cudaError_t div_by_scalar(double *x, long long count, const double *divisor, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  launch_k(div_kernel, grid_for(count), kThreads, 0, st, x, count, divisor);
  note_launch();
  return cudaGetLastError();
}

cudaError_t copy_f64(const double *src, double *dst, long long count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  launch_k(copy_kernel, grid_for(count), kThreads, 0, st, src, dst, count);
  note_launch();
  return cudaGetLastError();
}

cudaError_t compact_core(const double *src, double *dst, int la, int n, int lb,
                         const long long *ranks_dev, int k, cudaStream_t st) {
  const long long total = (long long)la * n * lb;
  launch_k(compact_kernel, grid_for(total), kThreads, 0, st, src, dst, la, n, lb, ranks_dev, k);
  note_launch();
  return cudaGetLastError();
}

cudaError_t sqrt_scalar(const double *x, double *out, cudaStream_t st) {
  launch_k(sqrt_kernel, 1, 1, 0, st, x, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t misc_health_word(int *value, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_misc_health, sizeof(int));
  if (e == cudaSuccess && clear && *value != 0) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_misc_health, &zero, sizeof(int));
  }
  return e;
}

}  // namespace hatt
