// Batched, arbitrarily strided FP64 GEMM for the small contractions of HaTT.
//
// On GB300 the FP64 pipe delivers ~1.2 TFLOP/s (about two DFMA lanes per SM
// per clock) against ~73 TFLOP/s of FP32, so an FP64 contraction is bound by
// DFMA issue, not by memory: a 256-thread block with a 4x4 (or smaller)
// register tile and 16-deep shared-memory staging keeps the FP64 pipe fed.
// What matters is that every launch covers all 152 SMs: the planner picks the
// tile that wastes the fewest lanes and splits K until the grid has at least
// two blocks per SM. Split-K partial sums are reduced in a fixed order by a
// second kernel (no atomics), so results are bitwise reproducible.
#include <algorithm>
#include "hatt_internal.cuh"

namespace hatt {
namespace {

constexpr int kBK = 16;
constexpr int kThreads = 256;
constexpr int kTargetBlocks = 2 * 152;

struct Launch {
  int bm, bn, tiles_m, tiles_n, ksplit, kchunk;
};

template <int BM, int BN>
__global__ void __launch_bounds__(kThreads)
gemm_f64_kernel(Gemm g, int tiles_n, int tiles_m, int ksplit, int kchunk, double *partial) {
  constexpr int TM = BM / 16, TN = BN / 16;
  if (g.skip_dev && *g.skip_dev) return;
  __shared__ double As[kBK][BM + 1];
  __shared__ double Bs[kBK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  // 1-D grid: block -> (n tile, m tile, split, batch), n tile fastest
  long long blk = blockIdx.x;
  const int tn_i = (int)(blk % tiles_n); blk /= tiles_n;
  const int tm_i = (int)(blk % tiles_m); blk /= tiles_m;
  const int ks = (int)(blk % ksplit);
  const int b = (int)(blk / ksplit);
  const int b1 = b / g.bdiv, b2 = b % g.bdiv;
  const double *A = g.A + b1 * g.sA1 + b2 * g.sA2;
  const double *B = g.B + b1 * g.sB1 + b2 * g.sB2;
  const int m0 = tm_i * BM, n0 = tn_i * BN;
  const int kbeg = ks * kchunk;
  const int kend = min(g.K, kbeg + kchunk);

  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  const bool a_kfast = (g.sAk == 1);
  const bool b_nfast = (g.sBn == 1);
  for (int kt = kbeg; kt < kend; kt += kBK) {
    for (int e = tid; e < BM * kBK; e += kThreads) {
      int mm, kk;
      if (a_kfast) { mm = e / kBK; kk = e % kBK; } else { kk = e / BM; mm = e % BM; }
      const int gm = m0 + mm, gk = kt + kk;
      As[kk][mm] = (gm < g.M && gk < kend) ? A[gm * g.sAm + gk * g.sAk] : 0.0;
    }
    for (int e = tid; e < BN * kBK; e += kThreads) {
      int nn, kk;
      if (b_nfast) { kk = e / BN; nn = e % BN; } else { nn = e / kBK; kk = e % kBK; }
      const int gn = n0 + nn, gk = kt + kk;
      Bs[kk][nn] = (gn < g.N && gk < kend) ? B[gk * g.sBk + gn * g.sBn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      double av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }

  if (ksplit > 1) {
    double *P = partial + ((long long)b * ksplit + ks) * g.M * (long long)g.N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int gm = m0 + ty + 16 * i;
      if (gm >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gn = n0 + tx + 16 * j;
        if (gn < g.N) P[(long long)gm * g.N + gn] = acc[i][j];
      }
    }
    return;
  }
  const double alpha = g.alpha * (g.alpha_dev ? *g.alpha_dev : 1.0);
  double *C = g.C + b1 * g.sC1 + b2 * g.sC2;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= g.N) continue;
      double *c = C + gm * g.sCm + gn * g.sCn;
      const double v = alpha * acc[i][j];
      *c = (g.beta != 0.0) ? fma(g.beta, *c, v) : v;
    }
  }
}

__global__ void __launch_bounds__(kThreads)
gemm_reduce_kernel(Gemm g, int ksplit, const double *partial) {
  if (g.skip_dev && *g.skip_dev) return;
  const long long mn = (long long)g.M * g.N;
  const long long total = mn * g.batch;
  const double alpha = g.alpha * (g.alpha_dev ? *g.alpha_dev : 1.0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / mn);
    const long long e = t % mn;
    const int gm = (int)(e / g.N), gn = (int)(e % g.N);
    const double *P = partial + (long long)b * ksplit * mn + e;
    double s = 0.0;
    for (int k = 0; k < ksplit; ++k) s += P[k * mn];
    const int b1 = b / g.bdiv, b2 = b % g.bdiv;
    double *c = g.C + b1 * g.sC1 + b2 * g.sC2 + gm * g.sCm + gn * g.sCn;
    const double v = alpha * s;
    *c = (g.beta != 0.0) ? fma(g.beta, *c, v) : v;
  }
}

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

Launch plan(const Gemm &g) {
  static const int sizes[3] = {16, 32, 64};
  Launch best{64, 64, 0, 0, 1, 0};
  double best_cost = 1e300;
  for (int bm : sizes) {
    for (int bn : sizes) {
      const int tm = ceil_div(g.M, bm), tn = ceil_div(g.N, bn);
      // padded lanes issue DFMAs too: cost = padded outputs; prefer bigger tiles on ties
      const double cost = (double)tm * bm * tn * bn * (1.0 + 0.02 * (64.0 / bm + 64.0 / bn));
      if (cost < best_cost) {
        best_cost = cost;
        best.bm = bm;
        best.bn = bn;
        best.tiles_m = tm;
        best.tiles_n = tn;
      }
    }
  }
  const long long blocks = (long long)best.tiles_m * best.tiles_n * g.batch;
  int ksplit = 1;
  if (blocks < kTargetBlocks && g.K > 4 * kBK) {
    ksplit = ceil_div(kTargetBlocks, blocks);
    ksplit = std::min(ksplit, ceil_div(g.K, 4 * kBK));   // at least 64 of K per split
    ksplit = std::max(ksplit, 1);
  }
  int kchunk = ceil_div(g.K, ksplit);
  kchunk = ceil_div(kchunk, kBK) * kBK;
  ksplit = ceil_div(g.K, kchunk);
  best.ksplit = std::max(ksplit, 1);
  best.kchunk = std::max(kchunk, kBK);
  return best;
}

template <int BM, int BN>
void launch_tile(const Gemm &g, const Launch &L, double *scratch, cudaStream_t st) {
  const long long blocks = (long long)L.tiles_n * L.tiles_m * L.ksplit * g.batch;
  gemm_f64_kernel<BM, BN><<<(unsigned)blocks, kThreads, 0, st>>>(g, L.tiles_n, L.tiles_m,
                                                                 L.ksplit, L.kchunk, scratch);
}

}  // namespace

size_t gemm_scratch_doubles(const Gemm &g) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return 0;
  const Launch L = plan(g);
  return L.ksplit > 1 ? (size_t)L.ksplit * g.batch * (size_t)g.M * g.N : 0;
}

cudaError_t gemm_f64(const Gemm &g, double *scratch, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.K <= 0) {
    return cudaErrorInvalidValue;   // callers never issue empty contractions
  }
  const Launch L = plan(g);
  if (L.ksplit > 1 && scratch == nullptr) return cudaErrorInvalidValue;
  if ((long long)L.tiles_n * L.tiles_m * L.ksplit * g.batch >= (1LL << 31))
    return cudaErrorInvalidConfiguration;
  switch (L.bm * 100 + L.bn) {
    case 1616: launch_tile<16, 16>(g, L, scratch, st); break;
    case 1632: launch_tile<16, 32>(g, L, scratch, st); break;
    case 1664: launch_tile<16, 64>(g, L, scratch, st); break;
    case 3216: launch_tile<32, 16>(g, L, scratch, st); break;
    case 3232: launch_tile<32, 32>(g, L, scratch, st); break;
    case 3264: launch_tile<32, 64>(g, L, scratch, st); break;
    case 6416: launch_tile<64, 16>(g, L, scratch, st); break;
    case 6432: launch_tile<64, 32>(g, L, scratch, st); break;
    default:   launch_tile<64, 64>(g, L, scratch, st); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || L.ksplit == 1) return e;
  const long long total = (long long)g.M * g.N * g.batch;
  const int blocks = (int)std::min<long long>((total + kThreads - 1) / kThreads, 4 * 152);
  gemm_reduce_kernel<<<blocks, kThreads, 0, st>>>(g, L.ksplit, scratch);
  return cudaGetLastError();
}

}  // namespace hatt
