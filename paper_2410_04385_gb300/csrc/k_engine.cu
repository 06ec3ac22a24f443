// Device side of the batched task engine (engine.cuh): the persistent kernel
// and the task bodies. Data produced inside the launch (by other CTAs) is read
// with __ldcg, through L2 only: the L1 caches of the SMs are not coherent and
// may hold lines of a buffer from before its last rewrite.
#include <algorithm>
#include "engine.cuh"

namespace hatt {
namespace {

constexpr int kT = kEngineThreads;
constexpr int kBK = 16;
constexpr int kMaxTile = 128;
constexpr int kMaxOut = 16;             // bm * bn <= kT * kMaxOut

// ---------------------------------------------------------------- sketch ---
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ void philox10(uint32_t x[4], uint32_t k0, uint32_t k1) {
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

// N(0,1) from two 52-bit uniforms (k + 1/2) 2^-52 (Box-Muller), the same
// counter layout as the single-pair sketch: (flat index, core, pair id, 0).
__device__ __forceinline__ double gaussian(uint32_t flat, uint32_t core, uint32_t pair,
                                           uint64_t seed) {
  uint32_t x[4] = {flat, core, pair, 0u};
  philox10(x, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const double u1 = ((double)(x[0] >> 6) * 67108864.0 + (double)(x[1] >> 6) + 0.5) * 0x1p-52;
  const double u2 = ((double)(x[2] >> 6) * 67108864.0 + (double)(x[3] >> 6) + 0.5) * 0x1p-52;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

__device__ void task_sketch(const EngineStage &s, int tile) {
  const long long total = (long long)s.a * s.n * s.b;
  const long long e0 = (long long)tile * s.chunk, e1 = min(total, e0 + s.chunk);
  const double scale = 1.0 / sqrt((double)s.a * (double)s.n * (double)s.b);
  for (long long e = e0 + threadIdx.x; e < e1; e += kT)
    s.out[e] = gaussian((uint32_t)e, (uint32_t)s.core, 0u, s.seed) * scale;
}

// ------------------------------------------------------------------ GEMM ---
// One bm x bn output tile of C[b] = alpha * A[b] B[b] (no split K): operands
// staged through shared memory in 16-deep k slices, outputs dealt linearly
// to the threads (at most kMaxOut each). prec == kPrecFP32 rounds the operands
// to FP32 and accumulates in FP32 (the low-precision sketch products).
template <typename T>
__device__ void gemm_tile_one(const EngineStage &s, int tm_i, int tn_i, int b, T *As, T *Bs);

template <typename T>
__device__ void gemm_tile_t(const EngineStage &s, int tile, double *smem) {
  if (s.skip_dev && __ldcg(s.skip_dev)) return;
  T *As = reinterpret_cast<T *>(smem);                     // kBK x (kMaxTile + 1)
  T *Bs = As + kBK * (kMaxTile + 1);
  const int tn_i = tile % s.tiles_n;
  const int rest = tile / s.tiles_n;
  const int tm_i = rest % s.tiles_m;
  const int bg = rest / s.tiles_m;
  for (int b = bg * s.bgroup; b < min(s.batch, (bg + 1) * s.bgroup); ++b)
    gemm_tile_one<T>(s, tm_i, tn_i, b, As, Bs);
}

// acc[q] += sum over a k slice of As[k][row q] Bs[k][column q] for the first
// NQ output slots; nqw is warp-uniform (the slots of the warp's lane 0), so no
// warp issues a DFMA for a slot none of its lanes owns -- a predicated-off
// DFMA holds the FP64 unit as long as a full one. Lanes with fewer slots
// multiply valid entries (index 0) into accumulators that are never stored.
template <int NQ, typename T>
__device__ __forceinline__ void mac_slots(int nqw, int kdepth, const T *As, const T *Bs,
                                          const int (&mn)[kMaxOut], T (&acc)[kMaxOut]) {
  if (nqw <= 0) return;
  if (nqw == NQ) {
    for (int kk = 0; kk < kdepth; ++kk) {
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        acc[q] = fma(As[kk * (kMaxTile + 1) + (mn[q] >> 8)], Bs[kk * (kMaxTile + 1) + (mn[q] & 255)],
                     acc[q]);
    }
    return;
  }
  if constexpr (NQ < kMaxOut) mac_slots<NQ + 1, T>(nqw, kdepth, As, Bs, mn, acc);
}

// The tile (tm_i, tn_i) of batch entry b.
template <typename T>
__device__ void gemm_tile_one(const EngineStage &s, int tm_i, int tn_i, int b, T *As, T *Bs) {
  const int tid = threadIdx.x;
  const int bm = s.bm, bn = s.bn;
  const int b1 = b / s.bdiv, b2 = b % s.bdiv;
  const double *A = s.A + b1 * s.sA1 + b2 * s.sA2;
  const double *B = s.B + b1 * s.sB1 + b2 * s.sB2;
  const int m0 = tm_i * bm, n0 = tn_i * bn;
  const int outs = bm * bn;
  int mn[kMaxOut];                      // output q of this thread: row << 8 | column in the tile
  T acc[kMaxOut];
#pragma unroll
  for (int q = 0; q < kMaxOut; ++q) {
    const int o = tid + kT * q;
    mn[q] = (o < outs) ? ((o / bn) << 8) | (o % bn) : 0;
    acc[q] = 0;
  }
  const int nq = (outs - tid + kT - 1) / kT;
  const int nqw = __shfl_sync(0xffffffffu, nq, 0);   // lane 0 owns the most outputs of its warp
  const bool a_kfast = (s.sAk == 1), b_nfast = (s.sBn == 1);
  for (int kt = 0; kt < s.K; kt += kBK) {
    for (int e = tid; e < bm * kBK; e += kT) {
      int mm, kk;
      if (a_kfast) { mm = e / kBK; kk = e % kBK; } else { kk = e / bm; mm = e % bm; }
      const int gm = m0 + mm, gk = kt + kk;
      const double v = (gm < s.M && gk < s.K) ? __ldcg(A + gm * s.sAm + gk * s.sAk) : 0.0;
      As[kk * (kMaxTile + 1) + mm] = (T)v;
    }
    for (int e = tid; e < bn * kBK; e += kT) {
      int nn, kk;
      if (b_nfast) { kk = e / bn; nn = e % bn; } else { nn = e / kBK; kk = e % kBK; }
      const int gn = n0 + nn, gk = kt + kk;
      const double v = (gn < s.N && gk < s.K) ? __ldcg(B + gk * s.sBk + gn * s.sBn) : 0.0;
      Bs[kk * (kMaxTile + 1) + nn] = (T)v;
    }
    __syncthreads();
    mac_slots<1>(nqw, min(kBK, s.K - kt), As, Bs, mn, acc);
    __syncthreads();
  }
  const double alpha = s.alpha_dev ? __ldcg(s.alpha_dev) : 1.0;
  double *C = s.C + b1 * s.sC1 + b2 * s.sC2;
#pragma unroll
  for (int q = 0; q < kMaxOut; ++q) {
    if (q >= nq) break;
    const int gm = m0 + (mn[q] >> 8), gn = n0 + (mn[q] & 255);
    if (gm < s.M && gn < s.N) C[gm * s.sCm + gn * s.sCn] = alpha * (double)acc[q];
  }
}

__device__ void task_gemm(const EngineStage &s, int tile, double *smem) {
  if (s.prec == kPrecFP32) gemm_tile_t<float>(s, tile, smem);
  else gemm_tile_t<double>(s, tile, smem);
}

// ----------------------------------------------------------------- norms ---
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kT / 32; ++i) t += red[i];
  return t;                             // valid in thread 0
}

__device__ void task_norm_part(const EngineStage &s, int tile, double *red) {
  const long long e0 = (long long)tile * s.chunk, e1 = min(s.count, e0 + s.chunk);
  double acc = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += kT) {
    const double v = __ldcg(s.x + e);
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) s.part[tile] = acc;
}

__device__ void task_norm_fin(const EngineStage &s, double *red, int *status) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)s.count; i += kT) acc += __ldcg(s.part + i);
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    if (!isfinite(acc)) atomicOr(status, kEngineNonfinite);
    s.out[0] = acc > 0.0 ? 1.0 / sqrt(acc) : 1.0;
  }
}

// C[0, i, a s1 + b] = Y[0, i, a] Z[0, i, b]
__device__ void task_pkp_first(const EngineStage &s, int tile) {
  const long long total = (long long)s.n * s.r1 * s.s1;
  const long long e0 = (long long)tile * s.chunk, e1 = min(total, e0 + s.chunk);
  for (long long e = e0 + threadIdx.x; e < e1; e += kT) {
    const int b = (int)(e % s.s1);
    const int a = (int)((e / s.s1) % s.r1);
    const int i = (int)(e / ((long long)s.r1 * s.s1));
    s.out[e] = __ldcg(s.Y + (long long)i * s.r1 + a) * __ldcg(s.Z + (long long)i * s.s1 + b);
  }
}

// ------------------------------------------------------------ Cholesky QR ---
// One pass of the Cholesky QR of hatt::qr_inplace (k_qr.cu), as two task
// kinds. Flags per QR (cleared before the launch): [0] done (later passes
// are no-ops), [1] skip this pass's apply, [2] passes applied, [3] shifted.

// 1/sqrt(x) for finite x > 0: FP32 seed and two Newton-Raphson steps in FP64.
__device__ __forceinline__ double rsqrt_nr(double x) {
  int e;
  double m = frexp(x, &e);
  if (e & 1) { m *= 2.0; e -= 1; }
  double y = (double)rsqrtf((float)m);
  y = y * fma(-0.5 * m, y * y, 1.5);
  y = y * fma(-0.5 * m, y * y, 1.5);
  return ldexp(y, -e / 2);
}

__device__ void task_chol(const EngineStage &s, double *smem, int *status) {
  int *flags = s.flags;
  __shared__ double s_dev, s_dmax, s_tr, s_rinv[kEngineMaxC];
  __shared__ int s_fail, s_done;
  const int c = s.c, m = s.m, ld = c + 1;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  if (tid == 0) s_done = *(volatile int *)flags;
  __syncthreads();
  if (s_done) {
    if (tid == 0) flags[1] = 1;
    return;
  }
  double *G = smem;                                 // c x ld
  double *red = smem + c * ld;                      // kT / 32
  double dev = 0.0, dmax = 0.0, tr = 0.0;
  int bad = 0;
  for (int e = tid; e < c * c; e += kT) {
    const int i = e / c, j = e % c;
    const double v = __ldcg(s.G + e);
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
  if (__syncthreads_or(bad)) {                       // a non-finite Gram matrix
    if (tid == 0) {
      atomicOr(status, kEngineNonfinite);
      flags[0] = 1;
      flags[1] = 1;
    }
    return;
  }
  for (int o = 16; o > 0; o >>= 1) {
    dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
  }
  __shared__ double w3[3][kT / 32];
  if ((tid & 31) == 0) { w3[0][tid >> 5] = dev; w3[1][tid >> 5] = dmax; w3[2][tid >> 5] = tr; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0, t = 0.0;
    for (int w = 0; w < kT / 32; ++w) { a = fmax(a, w3[0][w]); b = fmax(b, w3[1][w]); t += w3[2][w]; }
    s_dev = a; s_dmax = b; s_tr = t;
  }
  __syncthreads();
  (void)red;
  const double u = 1.1102230246251565e-16;
  if (s_dev <= 8.0 * c * u) {                       // orthonormal already
    if (tid == 0) { flags[0] = 1; flags[1] = 1; }
    return;
  }
  if (tid == 0) {
    flags[1] = 0;
    flags[2] += 1;
    if (s_dev <= 0.1 / c) flags[0] = 1;             // Gerschgorin: this pass is the last
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    double shift = 0.0;
    if (attempt == 1) {
      shift = 11.0 * ((double)m * c + (double)c * (c + 1)) * u * s_tr;
      if (!(shift > 0.0)) shift = 1e-300;
      for (int e = tid; e < c * c; e += kT) {
        const int i = e / c, j = e % c;
        G[i * ld + j] = __ldcg(s.G + e) + (i == j ? shift : 0.0);
      }
      if (tid == 0) flags[3] += 1;
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    const double floor_piv = (attempt == 0) ? (double)c * u * s_dmax : 0.0;
    for (int j = 0; j < c; ++j) {
      if (tid == 0) {
        double piv = G[j * ld + j];
        if (__ldcg(s.G + j * c + j) == 0.0) {
          piv = 1.0;                                // zero column: R_jj = 1, Q_j = 0
        } else if (!(piv > floor_piv)) {
          if (attempt == 0) s_fail = 1;
          else atomicOr(status, kEngineBreakdown);
          piv = fmax(shift, 1e-300);
        }
        const double y = rsqrt_nr(piv);
        G[j * ld + j] = piv * y;
        s_rinv[j] = y;
      }
      __syncthreads();
      if (s_fail) break;
      const double yj = s_rinv[j];
      for (int l = j + 1 + tid; l < c; l += kT) G[j * ld + l] *= yj;
      __syncthreads();
      for (int i = j + 1 + ty; i < c; i += 16) {
        const double rji = G[j * ld + i];
        for (int l = i + tx; l < c; l += 16) G[i * ld + l] = fma(-rji, G[j * ld + l], G[i * ld + l]);
      }
      __syncthreads();
    }
    __syncthreads();
    if (!s_fail) break;
  }
  for (int i = ty; i < c; i += 16)
    for (int l = tx; l < c; l += 16)
      s.Ut[i * c + l] = (l > i) ? G[i * ld + l] * s_rinv[i] : (l == i ? 1.0 : 0.0);
  for (int i = tid; i < c; i += kT) s.y[i] = s_rinv[i];
}

// Q = S R^{-1} on kEngineTrsmRows rows, one warp per row (k_qr.cu's apply).
__device__ void task_trsm(const EngineStage &s, int tile, double *smem) {
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = *(volatile int *)(s.flags + 1);
  __syncthreads();
  if (s_skip) return;
  const int c = s.c;
  double *Us = smem, *ys = smem + c * c;
  for (int e = threadIdx.x; e < c * c; e += kT) Us[e] = __ldcg(s.Ut + e);
  for (int e = threadIdx.x; e < c; e += kT) ys[e] = __ldcg(s.y + e);
  __syncthreads();
  const int lane = threadIdx.x & 31, warps = kT / 32;
  const int r0 = tile * kEngineTrsmRows, r1 = min(s.m, r0 + kEngineTrsmRows);
  const int ns = (c + 31) / 32;          // column slots in use (c <= kEngineMaxC)
  for (int r = r0 + (threadIdx.x >> 5); r < r1; r += warps) {
    double *row = s.S + (long long)r * c;
    double x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = (q < ns && lane + 32 * q < c) ? __ldcg(row + lane + 32 * q) : 0.0;
    switch (ns) {                        // warp-uniform slot loops (see trsm_row)
      case 1: trsm_row<1>(x, Us, c, lane); break;
      case 2: trsm_row<2>(x, Us, c, lane); break;
      case 3: trsm_row<3>(x, Us, c, lane); break;
      default: trsm_row<4>(x, Us, c, lane); break;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = lane + 32 * q;
      if (q < ns && col < c) row[col] = x[q] * ys[col];
    }
  }
}

__device__ void run_task(const EngineStage &s, int tile, double *smem, double *red, int *status) {
  switch (s.type) {
    case kStSketch: task_sketch(s, tile); break;
    case kStGemm: task_gemm(s, tile, smem); break;
    case kStNormPart: task_norm_part(s, tile, red); break;
    case kStNormFin: task_norm_fin(s, red, status); break;
    case kStPkpFirst: task_pkp_first(s, tile); break;
    case kStChol: task_chol(s, smem, status); break;
    case kStTrsm: task_trsm(s, tile, smem); break;
    case kStSet:
      if (threadIdx.x == 0) s.out[0] = s.value;
      break;
    default: break;
  }
}

// The persistent kernel: take the next task, wait for its pair's prerequisite
// count (bounded: spin_cap polls, or at once once any wait has run out), run
// it, publish it.
__global__ void __launch_bounds__(kT, 3)
engine_kernel(const EngineStage *stages, const EngineTask *tasks, int ntasks, int *head,
              int *done, int *status, long long spin_cap, long long *prof) {
  extern __shared__ __align__(16) double smem[];
  __shared__ double red[kT / 32];
  __shared__ int s_task;
  __shared__ long long pw[kProfWords];  // profile words, thread 0 only (see engine.cuh)
  if (threadIdx.x == 0)
    for (int i = 0; i < kProfWords; ++i) pw[i] = 0;
  const long long t_start = clock64();
  long long t0 = t_start;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_task = atomicAdd(head, 1);
    __syncthreads();
    const int t = s_task;
    if (threadIdx.x == 0) {
      const long long now = clock64();
      pw[2] += now - t0;
      t0 = now;
    }
    if (t >= ntasks) break;
    const EngineTask task = tasks[t];
    const int type = stages[task.stage].type & 7;
    if (threadIdx.x == 0) {
      volatile int *dp = done + task.pair;
      volatile int *sp = status;
      long long polls = 0;
      while (*dp < task.need) {
        if ((*sp & kEngineTimeout) != 0 || ++polls > spin_cap) {
          atomicOr(status, kEngineTimeout);
          break;
        }
        __nanosleep(256);
      }
      __threadfence();
      const long long now = clock64();
      pw[1] += now - t0;
      t0 = now;
    }
    __syncthreads();
    run_task(stages[task.stage], task.tile, smem, red, status);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicAdd(done + task.pair, 1);
      const long long now = clock64();
      pw[8 + type] += now - t0;
      pw[16 + type] += 1;
      t0 = now;
    }
  }
  if (threadIdx.x == 0 && prof && blockIdx.x < kMaxProfBlocks) {
    pw[0] = clock64() - t_start;
    for (int i = 0; i < kProfWords; ++i) prof[blockIdx.x * kProfWords + i] = pw[i];
  }
}

// All tiles of one GEMM stage as an ordinary grid (one CTA per tile): what the
// autotuner times for each candidate tile shape.
__global__ void __launch_bounds__(kT) engine_gemm_probe(EngineStage s) {
  extern __shared__ __align__(16) double smem[];
  task_gemm(s, blockIdx.x, smem);
}

}  // namespace

size_t engine_gemm_smem() { return (size_t)2 * kBK * (kMaxTile + 1) * sizeof(double); }

size_t engine_smem(int max_c) {
  const size_t chol = ((size_t)max_c * (max_c + 1) + kT / 32) * sizeof(double);
  const size_t trsm = ((size_t)max_c * max_c + max_c) * sizeof(double);
  return std::max(engine_gemm_smem(), std::max(chol, trsm));
}

cudaError_t engine_launch(const EngineStage *stages, const EngineTask *tasks, int ntasks,
                          int *head, int *done, int *status, long long spin_cap, int max_c,
                          int blocks, long long *prof, cudaStream_t st) {
  const size_t smem = engine_smem(max_c);
  cudaError_t e = cudaFuncSetAttribute(engine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  engine_kernel<<<blocks, kT, smem, st>>>(stages, tasks, ntasks, head, done, status, spin_cap,
                                          prof);
  note_launch();
  return cudaGetLastError();
}

cudaError_t engine_blocks(int max_c, int *blocks) {
  const size_t smem = engine_smem(max_c);
  cudaError_t e = cudaFuncSetAttribute(engine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel, kT, smem);
  if (e != cudaSuccess) return e;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *blocks = std::max(1, per_sm) * sms;
  return cudaSuccess;
}

cudaError_t engine_gemm_time(const EngineStage &s, cudaStream_t st, float *ms) {
  const int tiles = s.ntasks;
  cudaError_t e = cudaFuncSetAttribute(engine_gemm_probe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)engine_gemm_smem());
  if (e != cudaSuccess) return e;
  cudaEvent_t a, b;
  e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) { cudaEventDestroy(a); return e; }
  cudaEventRecord(a, st);
  engine_gemm_probe<<<tiles, kT, engine_gemm_smem(), st>>>(s);
  cudaEventRecord(b, st);
  e = cudaEventSynchronize(b);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t;
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace hatt
