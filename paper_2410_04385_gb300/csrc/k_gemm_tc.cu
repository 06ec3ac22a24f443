// Tensor-core (tcgen05) GEMM for the low-precision HPCRL-1 products: TF32 or
// BF16 operands, FP32 accumulation in tensor memory, FP64 result.
//
// C[b](m, n) = alpha * sum_k A[b](m, k) B[b](k, n) with the strides of the
// FP64 Gemm descriptor. One CTA (4 warps) owns a 128 x bn tile of C, or of C^T
// when M < N so that the 128-row side of the tensor-core instruction covers
// the larger dimension. For each 128-byte slice of K (64 BF16 or 32 TF32
// elements) the 128 threads stage both operands from FP64, rounded exactly as
// the SIMT path rounds them (FP64 -> FP32 to nearest even, then TF32 to
// nearest / ties away or BF16 to nearest even), into shared memory in the
// K-major "core matrix" layout (8 rows x 16 bytes per core matrix, no
// swizzle); one thread issues the tcgen05.mma instructions of the slice
// (K = 16 BF16 or 8 TF32 each, M = 128, N = bn) and commits them to an
// mbarrier that all threads wait on before the next slice overwrites the
// operands. The accumulator lives in tensor memory (row i = TMEM lane i,
// column j = TMEM column j) and is read back with tcgen05.ld by the warp that
// owns the lane quarter. Split-K uses the same per-tile counters as the FP64
// GEMM: the last block of a tile sums the partials in split order.
//
// Waits are bounded: a wait that runs out sets a device error word, the
// block skips the rest of its work, writes NaN to its outputs, and still
// frees its tensor memory. About 100 KB of shared memory per block caps the
// residency at two blocks per SM, so two allocations of at most 256 columns
// always fit in the 512 columns of an SM and tcgen05.alloc never waits.
#include <algorithm>
#include <cstdint>
#include "hatt_internal.cuh"

namespace hatt {

__device__ int g_device_error = 0;

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;
constexpr int kTcMaxN = 256;
constexpr int kSliceBytes = 128;                 // K bytes per staged slice and row
constexpr int kTcSmem = 100 * 1024;              // caps residency at 2 blocks per SM
constexpr long long kWaitLimit = 2000000;        // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major, no swizzle: start address, the
// byte offset between core matrices adjacent in K (LBO) and in M/N (SBO),
// descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12: 1 = BF16 for kind::f16, 2 = TF32 for kind::tf32),
// K-major A and B, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t instr_desc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t round_bits(double x, bool tf32) {
  unsigned u = __float_as_uint((float)x);
  if (tf32) return (u + 0x1000u) & 0xFFFFE000u;
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;           // BF16 bits
}

// Operand element (row, k) of the tile in the logical orientation.
struct Operand {
  const double *p;
  long long s_row, s_k;
  int rows, kdim;
};

// Stage rows [r0, r0 + nrows) x k [k0, k0 + slice) of op into `dst` (core
// matrix layout, chunks = 8 per row); out-of-range entries are zero.
template <bool TF32>
__device__ __forceinline__ void stage(const Operand &op, int r0, int nrows, int k0, int kend,
                                      unsigned char *dst) {
  constexpr int eb = TF32 ? 4 : 2;
  constexpr int per_row = kSliceBytes / eb;                // elements per row and slice
  for (int e = threadIdx.x; e < nrows * per_row; e += kTcThreads) {
    const int row = e / per_row, kk = e % per_row;
    const int gr = r0 + row, gk = k0 + kk;
    const double v = (gr < op.rows && gk < kend) ? op.p[gr * op.s_row + gk * op.s_k] : 0.0;
    const int byte = kk * eb;
    const int off = ((row >> 3) * (kSliceBytes / 16) + (byte >> 4)) * 128 + (row & 7) * 16 + (byte & 15);
    if (TF32) *(uint32_t *)(dst + off) = round_bits(v, true);
    else *(uint16_t *)(dst + off) = (uint16_t)round_bits(v, false);
  }
}

template <bool TF32>
__global__ void __launch_bounds__(kTcThreads)
gemm_tc_kernel(Gemm g, int swap, int bn, int tiles_n, int tiles_m, int ksplit, int kchunk,
               int tmem_cols, double *partial, int *counters) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_last, s_fail;
  if (g.skip_dev && *g.skip_dev) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  long long blk = blockIdx.x;
  const int tn_i = (int)(blk % tiles_n); blk /= tiles_n;
  const int tm_i = (int)(blk % tiles_m); blk /= tiles_m;
  const int ks = (int)(blk % ksplit);
  const int b = (int)(blk / ksplit);
  const int b1 = b / g.bdiv, b2 = b % g.bdiv;
  const double *A = g.A + b1 * g.sA1 + b2 * g.sA2;
  const double *B = g.B + b1 * g.sB1 + b2 * g.sB2;
  // logical tile operands: rows of the tile come from "P" (128 per tile),
  // columns from "Q" (bn per tile); both indexed (row, k)
  Operand P, Q;
  if (!swap) {
    P = Operand{A, g.sAm, g.sAk, g.M, g.K};
    Q = Operand{B, g.sBn, g.sBk, g.N, g.K};
  } else {
    P = Operand{B, g.sBn, g.sBk, g.N, g.K};
    Q = Operand{A, g.sAm, g.sAk, g.M, g.K};
  }
  const int p0 = tm_i * kTcM, q0 = tn_i * bn;
  const int kbeg = ks * kchunk, kend = min(g.K, kbeg + kchunk);
  constexpr int eb = TF32 ? 4 : 2;
  constexpr int kslice = kSliceBytes / eb;
  unsigned char *Ps = sm;
  unsigned char *Qs = sm + kTcM * kSliceBytes;
  const uint32_t sbo = (kSliceBytes / 16) * 128;           // next 8-row group

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&s_taddr)), "r"(tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&s_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr;
  const uint32_t idesc = instr_desc(TF32 ? 2 : 1, kTcM, bn);

  uint32_t phase = 0;
  bool any = false;
  for (int k0 = kbeg; k0 < kend; k0 += kslice) {
    stage<TF32>(P, p0, kTcM, k0, kend, Ps);
    stage<TF32>(Q, q0, bn, k0, kend, Qs);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      for (int kk = 0; kk < kslice; kk += 32 / eb) {         // one instruction = 32 bytes of K
        const uint32_t off = (uint32_t)(kk * eb / 16) * 128;
        const uint64_t ad = smem_desc(smem_u32(Ps) + off, 128, sbo);
        const uint64_t bd = smem_desc(smem_u32(Qs) + off, 128, sbo);
        const uint32_t acc = any ? 1u : 0u;
        if (TF32)
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                       :: "r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
        else
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                       :: "r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
        any = true;
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&s_bar)) : "memory");
    }
    any = true;
    uint32_t done = 0;
    for (long long it = 0; it < kWaitLimit && !done; ++it)
      asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                   "selp.u32 %0, 1, 0, p;\n}\n"
                   : "=r"(done) : "r"(smem_u32(&s_bar)), "r"(phase) : "memory");
    phase ^= 1u;
    if (!done) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool fail = s_fail != 0;
  if (fail && tid == 0) atomicExch(&g_device_error, 1);

  // epilogue: thread = tile row (lane quarter of its warp), columns in 8s
  const double alpha = g.alpha * (g.alpha_dev ? *g.alpha_dev : 1.0);
  double *C = g.C + b1 * g.sC1 + b2 * g.sC2;
  const long long mn = (long long)g.M * g.N;
  const int prow = p0 + tid;                               // tile row -> P index
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  for (int c0 = 0; c0 < bn; c0 += 8) {
    uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (!fail && any) {
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                     "=r"(r[6]), "=r"(r[7])
                   : "r"(taddr + lane_base + (uint32_t)c0) : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    }
    for (int j = 0; j < 8; ++j) {
      const int qcol = q0 + c0 + j;
      const int gm = swap ? qcol : prow, gn = swap ? prow : qcol;
      if (gm >= g.M || gn >= g.N || c0 + j >= bn) continue;
      const double acc = fail ? __longlong_as_double(0x7FF8000000000000LL) : (double)__uint_as_float(r[j]);
      if (ksplit > 1) partial[((long long)b * ksplit + ks) * mn + (long long)gm * g.N + gn] = acc;
      else {
        double *c = C + gm * g.sCm + gn * g.sCn;
        const double v = alpha * acc;
        *c = (g.beta != 0.0) ? fma(g.beta, *c, v) : v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(tmem_cols) : "memory");
  if (ksplit == 1) return;
  // split-K: the last block of the tile sums the partials in split order
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const int t = (b * tiles_m + tm_i) * tiles_n + tn_i;
    const int prev = atomicAdd(&counters[t], 1);
    s_last = (prev == ksplit - 1);
    if (s_last) counters[t] = 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double *P0 = partial + (long long)b * ksplit * mn;
  for (int e = tid; e < kTcM * bn; e += kTcThreads) {
    const int tr = e / bn, tc = e % bn;
    const int pr = p0 + tr, qc = q0 + tc;
    const int gm = swap ? qc : pr, gn = swap ? pr : qc;
    if (gm >= g.M || gn >= g.N) continue;
    const long long off = (long long)gm * g.N + gn;
    double sum = 0.0;
    for (int k = 0; k < ksplit; ++k) sum += __ldcg(P0 + k * mn + off);
    double *c = C + gm * g.sCm + gn * g.sCn;
    const double v = alpha * sum;
    *c = (g.beta != 0.0) ? fma(g.beta, *c, v) : v;
  }
}

long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

struct TcLaunch {
  int swap, bn, tiles_m, tiles_n, ksplit, kchunk, tmem_cols;
};

TcLaunch tc_plan(const Gemm &g) {
  TcLaunch L{};
  L.swap = g.M < g.N;
  const long long rows = L.swap ? g.N : g.M, cols = L.swap ? g.M : g.N;
  const long long nt = cdiv(cols, kTcMaxN);
  L.bn = (int)(cdiv(cdiv(cols, nt), 16) * 16);
  L.tiles_m = (int)cdiv(rows, kTcM);
  L.tiles_n = (int)cdiv(cols, L.bn);
  const int kslice = kSliceBytes / (g.prec == kPrecTF32 ? 4 : 2);
  const long long tiles = (long long)L.tiles_m * L.tiles_n * g.batch;
  const long long slices = cdiv(g.K, kslice);
  long long ks = 1;
  if (tiles <= kTileCounters) ks = std::min<long long>(slices, std::max<long long>(1, cdiv(2 * 152, tiles)));
  L.kchunk = (int)(cdiv(slices, ks) * kslice);
  L.ksplit = (int)cdiv(g.K, L.kchunk);
  int tc = 32;
  while (tc < L.bn) tc <<= 1;
  L.tmem_cols = tc;
  return L;
}

}  // namespace

cudaError_t read_device_error(int *value) {
  int oz = 0, qr = 0, misc = 0;
  cudaError_t e = cudaMemcpyFromSymbol(value, g_device_error, sizeof(int));
  if (e == cudaSuccess) e = oz_error_word(&oz, false);
  if (e == cudaSuccess) e = qr_health_word(&qr, false);
  if (e == cudaSuccess) e = misc_health_word(&misc, false);
  if (e == cudaSuccess) *value = (*value != 0 || oz != 0 ? kHealthTimeout : 0) | qr | misc;
  return e;
}

cudaError_t clear_device_error() {
  const int zero = 0;
  int oz = 0;
  cudaError_t e = cudaMemcpyToSymbol(g_device_error, &zero, sizeof(int));
  if (e == cudaSuccess) e = oz_error_word(&oz, true);
  if (e == cudaSuccess) e = qr_health_word(&oz, true);
  if (e == cudaSuccess) e = misc_health_word(&oz, true);
  return e;
}

bool gemm_tc_supported(const Gemm &g) {
  // device-side extents (Gemm::dyn_dev) run on the emulated-format SIMT kernel
  return (g.prec == kPrecTF32 || g.prec == kPrecBF16) && g.dyn_dev == nullptr;
}

size_t gemm_tc_scratch_doubles(const Gemm &g) {
  const TcLaunch L = tc_plan(g);
  return L.ksplit > 1 ? (size_t)L.ksplit * g.batch * (size_t)g.M * g.N : 0;
}

cudaError_t gemm_tc(const Gemm &g, double *scratch, int *counters, cudaStream_t st) {
  const TcLaunch L = tc_plan(g);
  if (L.ksplit > 1 && (scratch == nullptr || counters == nullptr)) return cudaErrorInvalidValue;
  const long long blocks = (long long)L.tiles_n * L.tiles_m * L.ksplit * g.batch;
  if (blocks >= (1LL << 31)) return cudaErrorInvalidConfiguration;
  cudaError_t e;
  if (g.prec == kPrecTF32) {
    e = cudaFuncSetAttribute(gemm_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    launch_k(gemm_tc_kernel<true>, (unsigned)blocks, kTcThreads, kTcSmem, st, 
        g, L.swap, L.bn, L.tiles_n, L.tiles_m, L.ksplit, L.kchunk, L.tmem_cols, scratch, counters);
  } else {
    e = cudaFuncSetAttribute(gemm_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    launch_k(gemm_tc_kernel<false>, (unsigned)blocks, kTcThreads, kTcSmem, st, 
        g, L.swap, L.bn, L.tiles_n, L.tiles_m, L.ksplit, L.kchunk, L.tmem_cols, scratch, counters);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace hatt
