// FP64-accurate GEMM on the BF16 tensor cores (splitting in the manner of
// Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 2012).
//
// Every row of the left operand and every column of the right one is scaled
// by a power of two 2^-e so that its entries lie in (-1, 1); the scaled value
// is rounded to 54 fraction bits, V = rint(x 2^(54-e)), and |V| < 2^54 is cut
// into kS = 9 slices of kB = 6 bits, x = 2^e sum_p s_p 2^(-6(p+1)) with
// integer s_p in (-64, 64), exactly representable in BF16. Then
//   A B = diag(2^e) [ sum_{p,q} 2^(-6(p+q+2)) A_p B_q ] diag(2^f),
// and each slice product A_p B_q has integer entries that a tensor core
// accumulates exactly in FP32 as long as the sum stays below 2^24. Pairs with
// the same level L = p + q share the scale 2^(-6(L+2)) and go to one
// accumulator; with at most 9 pairs per level and 448 values of K per
// accumulation, 9 * 448 * 63^2 < 2^24, so every level sum is exact. Levels
// L <= 8 (45 of the 81 pairs) are kept: the dropped ones weigh less than
// 2^-54 of the leading term. After each 448-long piece of K the 9 level
// accumulators are read from tensor memory and added, scaled, into FP64
// registers. The result has the accuracy of an FP64 product (the splitting
// loses at most half a unit of 2^-54 of each row's / column's largest entry,
// FP64 GEMM error bounds are of the same kind), from BF16 tensor-core work.
//
// Kernels: oz_split_kernel writes the slices (BF16, rows padded to the tile,
// K padded to 64) and the exponents of one operand, a warp per row;
// oz_mma_kernel owns a 128 x 32 output tile (of C, or of C^T when M < N),
// stages all 9 slices of both operands for each 64-wide step of K into
// shared memory in the K-major core-matrix layout, and issues the 45 x 4
// tcgen05.mma instructions of the step into the 9 level accumulators (9 x 32
// tensor-memory columns). Waits are bounded as in the TF32 / BF16 kernel.
#include <algorithm>
#include <cstdint>
#include "hatt_internal.cuh"

namespace hatt {

__device__ int g_oz_error = 0;

namespace {

constexpr int kS = 9;                    // slices
constexpr int kB = 6;                    // bits per slice
constexpr int kLevels = kS;              // L = p + q in [0, kS - 1]
constexpr int kOzBn = 32;                // output columns per tile
constexpr int kOzRows = 128;             // output rows per tile (tensor-core M)
constexpr int kKStep = 64;               // K staged per step (128 bytes of BF16)
constexpr int kKPiece = 448;             // K per exact level accumulation
constexpr int kOzThreads = 128;
constexpr int kOzSmem = kS * (kOzRows + kOzBn) * kKStep * 2 + 1024;
constexpr int kTmemCols = 512;           // 9 x 32 used; the whole SM (one CTA per SM)
constexpr long long kOzWaitLimit = 2000000;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

struct OzOperand {                       // logical (row, k) view of an FP64 operand
  const double *p;
  long long s_row, s_k, s_b1, s_b2;
  int rows, K;
};

// One warp per (batch, row): exponent of the row maximum, then the slices.
// out[((b * kS + p) * rows_pad + r) * k_pad + k], exps[b * rows_pad + r].
__global__ void __launch_bounds__(256)
oz_split_kernel(OzOperand op, int nbatch, int bdiv, int rows_pad, int k_pad, uint16_t *out,
                int *exps, const int *skip) {
  pdl_enter();
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const long long w = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= (long long)nbatch * rows_pad) return;
  const int b = (int)(w / rows_pad), r = (int)(w % rows_pad);
  const double *row = op.p + (b / bdiv) * op.s_b1 + (b % bdiv) * op.s_b2 + r * op.s_row;
  const bool live = r < op.rows;
  double mx = 0.0;
  if (live)
    for (int k = lane; k < op.K; k += 32) mx = fmax(mx, fabs(row[k * op.s_k]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int e = 0;
  if (mx > 0.0) (void)frexp(mx, &e);     // mx = m 2^e, m in [0.5, 1): |x| 2^-e < 1
  if (lane == 0) exps[(long long)b * rows_pad + r] = e;
  for (int k = lane; k < k_pad; k += 32) {
    const double x = (live && k < op.K) ? row[k * op.s_k] : 0.0;
    const long long V = llrint(ldexp(x, 54 - e));          // |V| < 2^54 (<= 2^54 after rounding)
    const unsigned long long u = (unsigned long long)(V < 0 ? -V : V);
    const bool neg = V < 0;
    for (int p = 0; p < kS; ++p) {
      const unsigned sl = (unsigned)((u >> (48 - kB * p)) & 63u);
      const float f = neg ? -(float)sl : (float)sl;
      out[(((long long)b * kS + p) * rows_pad + r) * k_pad + k] = (uint16_t)(__float_as_uint(f) >> 16);
    }
  }
}

// Stage rows [r0, r0 + nrows) x k [k0, k0 + 64) of the kS slices: slice p goes
// to dst + p * nrows * 128 bytes, core-matrix layout (8 chunks of 16 bytes
// per row); a 16-byte chunk holds 8 consecutive BF16 values of one row. The
// copies are asynchronous (cp.async, 16 bytes each, all in flight at once);
// the caller waits for them with cp.async.wait_group.
__device__ __forceinline__ void oz_stage(const uint16_t *slices, int rows_pad, int k_pad, int r0,
                                         int nrows, int k0, unsigned char *dst) {
  const int chunks = nrows * (kKStep / 8);
  for (int t = threadIdx.x; t < kS * chunks; t += kOzThreads) {
    const int p = t / chunks, c = t % chunks;
    const int row = c / (kKStep / 8), ch = c % (kKStep / 8);
    const uint16_t *src = slices + ((long long)p * rows_pad + r0 + row) * k_pad + k0 + ch * 8;
    unsigned char *base = dst + (size_t)p * nrows * (kKStep * 2);
    const uint32_t d = smem_u32(base + ((row >> 3) * (kKStep / 8) + ch) * 128 + (row & 7) * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(d), "l"(src) : "memory");
  }
}

__global__ void __launch_bounds__(kOzThreads)
oz_mma_kernel(Gemm g, int swap, int tiles_n, int tiles_m, const uint16_t *Psl, const int *Pexp,
              int P_pad, int P_batched, const uint16_t *Qsl, const int *Qexp, int Q_pad,
              int Q_batched, int k_pad) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t s_taddr;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_fail;
  if (g.skip_dev && *g.skip_dev) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  long long blk = blockIdx.x;
  const int tn_i = (int)(blk % tiles_n); blk /= tiles_n;
  const int tm_i = (int)(blk % tiles_m);
  const int b = (int)(blk / tiles_m);
  const int p0 = tm_i * kOzRows, q0 = tn_i * kOzBn;
  const uint16_t *Pb = Psl + (P_batched ? (long long)b * kS * P_pad * k_pad : 0);
  const uint16_t *Qb = Qsl + (Q_batched ? (long long)b * kS * Q_pad * k_pad : 0);
  const int *Pe = Pexp + (P_batched ? (long long)b * P_pad : 0);
  const int *Qe = Qexp + (Q_batched ? (long long)b * Q_pad : 0);
  unsigned char *Ps = sm;
  unsigned char *Qs = sm + (size_t)kS * kOzRows * kKStep * 2;
  const uint32_t sbo = (kKStep / 8) * 128;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&s_taddr)), "r"(kTmemCols) : "memory");
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
  // kind::f16, BF16 x BF16 -> F32, K-major, M = 128, N = 32
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kOzBn >> 3) << 17) |
                         ((uint32_t)(kOzRows >> 4) << 24);
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

  double acc[kOzBn];
#pragma unroll
  for (int c = 0; c < kOzBn; ++c) acc[c] = 0.0;
  uint32_t phase = 0;
  bool fail = false;
  for (int kp = 0; kp < g.K && !fail; kp += kKPiece) {
    const int kpend = min(g.K, kp + kKPiece);
    for (int k0 = kp; k0 < kpend; k0 += kKStep) {
      oz_stage(Pb, P_pad, k_pad, p0, kOzRows, k0, Ps);
      oz_stage(Qb, Q_pad, k_pad, q0, kOzBn, k0, Qs);
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
        for (int p = 0; p < kS; ++p)
          for (int q = 0; p + q < kLevels; ++q) {
            const uint32_t d = taddr + (uint32_t)((p + q) * kOzBn);
            for (int kk = 0; kk < kKStep; kk += 16) {
              const uint32_t off = (uint32_t)(kk * 2 / 16) * 128;
              const uint64_t ad = smem_desc(smem_u32(Ps) + p * kOzRows * kKStep * 2 + off, 128, sbo);
              const uint64_t bd = smem_desc(smem_u32(Qs) + q * kOzBn * kKStep * 2 + off, 128, sbo);
              // the first instruction into level L of a piece is pair (0, L), kk = 0
              // of the piece's first step: it overwrites the accumulator
              const uint32_t en = (k0 == kp && kk == 0 && p == 0) ? 0u : 1u;
              asm volatile("{\n.reg .pred pr;\nsetp.ne.b32 pr, %4, 0;\n"
                           "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pr;\n}\n"
                           :: "r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(en) : "memory");
            }
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&s_bar)) : "memory");
      }
      uint32_t done = 0;
      for (long long it = 0; it < kOzWaitLimit && !done; ++it)
        asm volatile("{\n.reg .pred pr;\nmbarrier.try_wait.parity.shared::cta.b64 pr, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, pr;\n}\n"
                     : "=r"(done) : "r"(smem_u32(&s_bar)), "r"(phase) : "memory");
      phase ^= 1u;
      if (!done) s_fail = 1;
      __syncthreads();
      if (s_fail) { fail = true; break; }
    }
    if (fail) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // add the 9 level sums of this piece, scaled, to the FP64 accumulators
#pragma unroll 1
    for (int L = 0; L < kLevels; ++L) {
      const double scale = ldexp(1.0, -kB * (L + 2));
#pragma unroll
      for (int c0 = 0; c0 < kOzBn; c0 += 8) {
        uint32_t r[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                       "=r"(r[6]), "=r"(r[7])
                     : "r"(taddr + lane_base + (uint32_t)(L * kOzBn + c0)) : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[c0 + j] = fma((double)__uint_as_float(r[j]), scale, acc[c0 + j]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();                     // every lane read before the next piece overwrites
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (fail && tid == 0) atomicExch(&g_oz_error, 1);

  const double alpha = g.alpha * (g.alpha_dev ? *g.alpha_dev : 1.0);
  const int b1 = b / g.bdiv, b2 = b % g.bdiv;
  double *C = g.C + b1 * g.sC1 + b2 * g.sC2;
  const int prow = p0 + tid;
  const int eP = Pe[prow];
#pragma unroll
  for (int c = 0; c < kOzBn; ++c) {
    const int qcol = q0 + c;
    const int gm = swap ? qcol : prow, gn = swap ? prow : qcol;
    if (gm >= g.M || gn >= g.N) continue;
    const double v = fail ? __longlong_as_double(0x7FF8000000000000LL)
                          : alpha * ldexp(acc[c], eP + Qe[qcol]);
    double *cp = C + gm * g.sCm + gn * g.sCn;
    *cp = (g.beta != 0.0) ? fma(g.beta, *cp, v) : v;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(kTmemCols) : "memory");
}

long long ozdiv(long long a, long long b) { return (a + b - 1) / b; }

struct OzPlan {
  int swap, tiles_m, tiles_n, P_pad, Q_pad, k_pad, P_batched, Q_batched;
  OzOperand P, Q;
  int Pb, Qb;                            // batch elements split (1 when shared)
  size_t P_sl, Q_sl, P_ex, Q_ex;         // element counts of slices / exponents
};

OzPlan oz_plan(const Gemm &g) {
  OzPlan L{};
  L.swap = g.M < g.N;
  if (!L.swap) {
    L.P = OzOperand{g.A, g.sAm, g.sAk, g.sA1, g.sA2, g.M, g.K};
    L.Q = OzOperand{g.B, g.sBn, g.sBk, g.sB1, g.sB2, g.N, g.K};
  } else {
    L.P = OzOperand{g.B, g.sBn, g.sBk, g.sB1, g.sB2, g.N, g.K};
    L.Q = OzOperand{g.A, g.sAm, g.sAk, g.sA1, g.sA2, g.M, g.K};
  }
  L.P_batched = g.batch > 1 && (L.P.s_b1 != 0 || L.P.s_b2 != 0);
  L.Q_batched = g.batch > 1 && (L.Q.s_b1 != 0 || L.Q.s_b2 != 0);
  L.Pb = L.P_batched ? g.batch : 1;
  L.Qb = L.Q_batched ? g.batch : 1;
  L.tiles_m = (int)ozdiv(L.P.rows, kOzRows);
  L.tiles_n = (int)ozdiv(L.Q.rows, kOzBn);
  L.P_pad = L.tiles_m * kOzRows;
  L.Q_pad = L.tiles_n * kOzBn;
  L.k_pad = (int)(ozdiv(g.K, kKStep) * kKStep);
  L.P_sl = (size_t)L.Pb * kS * L.P_pad * L.k_pad;
  L.Q_sl = (size_t)L.Qb * kS * L.Q_pad * L.k_pad;
  L.P_ex = (size_t)L.Pb * L.P_pad;
  L.Q_ex = (size_t)L.Qb * L.Q_pad;
  return L;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t oz_bytes(const OzPlan &L) {
  return align256(L.P_sl * 2) + align256(L.Q_sl * 2) + align256(L.P_ex * 4) + align256(L.Q_ex * 4);
}

thread_local bool t_fp64_tc = false;

}  // namespace

void set_fp64_tensor_cores(bool on) { t_fp64_tc = on; }

bool gemm_oz_applicable(const Gemm &g) {
  if (!t_fp64_tc || g.prec != kPrecFP64 || g.dyn_dev != nullptr) return false;
  const double flops = 2.0 * g.M * g.N * (double)g.K * g.batch;
  return std::max(g.M, g.N) >= 128 && g.K >= 128 && flops >= 2e7;
}

size_t gemm_oz_scratch_doubles(const Gemm &g) {
  return (oz_bytes(oz_plan(g)) + 7) / 8;
}

cudaError_t gemm_oz(const Gemm &g, double *scratch, cudaStream_t st) {
  const OzPlan L = oz_plan(g);
  if (scratch == nullptr) return cudaErrorInvalidValue;
  char *p = (char *)scratch;
  uint16_t *Psl = (uint16_t *)p; p += align256(L.P_sl * 2);
  uint16_t *Qsl = (uint16_t *)p; p += align256(L.Q_sl * 2);
  int *Pex = (int *)p; p += align256(L.P_ex * 4);
  int *Qex = (int *)p;
  const long long prow = (long long)L.Pb * L.P_pad, qrow = (long long)L.Qb * L.Q_pad;
  launch_k(oz_split_kernel, (unsigned)ozdiv(prow, 8), 256, 0, st, L.P, L.Pb, g.bdiv, L.P_pad, L.k_pad,
                                                            Psl, Pex, g.skip_dev);
  note_launch();
  launch_k(oz_split_kernel, (unsigned)ozdiv(qrow, 8), 256, 0, st, L.Q, L.Qb, g.bdiv, L.Q_pad, L.k_pad,
                                                            Qsl, Qex, g.skip_dev);
  note_launch();
  cudaError_t e = cudaFuncSetAttribute(oz_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kOzSmem);
  if (e != cudaSuccess) return e;
  const long long blocks = (long long)L.tiles_m * L.tiles_n * g.batch;
  if (blocks >= (1LL << 31)) return cudaErrorInvalidConfiguration;
  launch_k(oz_mma_kernel, (unsigned)blocks, kOzThreads, kOzSmem, st, 
      g, L.swap, L.tiles_n, L.tiles_m, Psl, Pex, L.P_pad, L.P_batched, Qsl, Qex, L.Q_pad,
      L.Q_batched, L.k_pad);
  note_launch();
  return cudaGetLastError();
}

cudaError_t oz_error_word(int *value, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(value, g_oz_error, sizeof(int));
  if (e == cudaSuccess && clear && *value != 0) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_oz_error, &zero, sizeof(int));
  }
  return e;
}

}  // namespace hatt
