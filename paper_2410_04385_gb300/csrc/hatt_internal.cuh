// Internal declarations shared by the libhatt CUDA sources.
// Each kernel lives with its launch helper in one .cu file; the helpers below
// are the only cross-file interface (plain host functions, no relocatable
// device code).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <utility>

namespace hatt {

constexpr int kMaxSmall = 128;   // TT_MAX_SMALL_RANK

// Programmatic dependent launch. The path is a chain of ~1000 dependent small
// kernels, so the gap between one kernel's end and the next one's start is a
// large part of a step. Every kernel is launched with programmatic stream
// serialization (launch_k) and begins with pdl_enter: griddepcontrol.wait
// holds the grid until the grids it depends on have completed and their
// memory is visible, and launch_dependents then lets the following kernel be
// scheduled while this one runs (its blocks wait at their own pdl_enter).
// Since the wait comes before any load or store, every read-after-write and
// write-after-read order of the stream is kept. The batched entry point turns
// it off for the calling thread: with many streams in flight, the blocks that
// wait early hold SM slots that the other streams' kernels could use.
void set_programmatic_launch(bool on);
bool programmatic_launch();
template <typename... P, typename... A>
inline cudaError_t launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, A &&...args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = programmatic_launch() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Forward substitution of one row x (lane t holds columns t, t+32, t+64,
// t+96) against the unit upper triangle U~ in shared memory: step l
// broadcasts the finished x_l and the lanes update their later columns. The
// slots a step touches are chosen by warp-uniform loop bounds, never by
// per-lane predicates alone: a predicated-off DFMA holds the FP64 unit like a
// full one, and guarding all four slots at every step cost 2.4x (c = 50) to
// 4x (c = 32) the DFMAs the solve needs.
template <int NS>
__device__ __forceinline__ void trsm_row(double (&x)[4], const double *Us, int c, int lane) {
#pragma unroll
  for (int s0 = 0; s0 < NS; ++s0) {
    const int lend = min(c, 32 * (s0 + 1));
    for (int l = 32 * s0; l < lend; ++l) {
      const double xl = __shfl_sync(0xffffffffu, x[s0], l & 31);
      const double *u = Us + l * c;
#pragma unroll
      for (int s = s0; s < NS; ++s) {
        const int col = lane + 32 * s;
        if (col > l && col < c) x[s] = fma(-xl, u[col], x[s]);
      }
    }
  }
}

// Process-wide count of kernels enqueued by this library (each launch site
// calls note_launch once).
void note_launch();
long long launch_count();
// Split-K GEMMs count finished blocks per output tile in an int array of
// kTileCounters entries that is zero before every GEMM (each GEMM leaves it
// zero). The entry points carve one per call, clear it once, and make it the
// calling thread's current array for the duration of the call.
constexpr int kTileCounters = 4096;
void set_tile_counters(int *counters);
int *tile_counters();
// Kernel timer (see tt_kernel_timer_start): timer_begin returns a slot and
// records its start event on st, or -1 when the timer is off, full, or st is
// capturing; timer_end records the stop event, the launch's flops and its
// role (kRoleAux or kRoleMethod, the values of tt_kernel_timer_stop_ex).
int timer_begin(cudaStream_t st);
void timer_end(int slot, cudaStream_t st, double flops, int role);
constexpr int kRoleAux = 0;      // QR, truncation, refinement and inner-product products
constexpr int kRoleMethod = 1;   // the HaTT contractions: HPCRL (Alg. 3), C_k W, Q^T C_k, eq. (3.10)
constexpr int kMaxOrder = 512;   // largest d handled by the parameter tables

// ------------------------------------------------------------------ GEMM ---
// C[b](m, n) = alpha * (alpha_dev ? *alpha_dev : 1) * sum_k A[b](m, k) B[b](k, n)
//              + beta * C[b](m, n)
// with element offsets
//   A[b](m, k) = A[b1*sA1 + b2*sA2 + m*sAm + k*sAk],   b1 = b / bdiv, b2 = b % bdiv
//   B[b](k, n) = B[b1*sB1 + b2*sB2 + k*sBk + n*sBn]
//   C[b](m, n) = C[b1*sC1 + b2*sC2 + m*sCm + n*sCn]
// beta == 0 never reads C. When the planner splits K, partial sums go to a
// workspace buffer and a second kernel reduces them in a fixed order, so the
// result is bitwise reproducible.
// Arithmetic of a GEMM: FP64 throughout, or operands rounded to FP32 / TF32 /
// BF16 with FP32 accumulation (the values match tt_precision).
constexpr int kPrecFP64 = 0, kPrecFP32 = 1, kPrecTF32 = 2, kPrecBF16 = 3;

struct Gemm {
  int M = 0, N = 0, K = 0;
  int batch = 1, bdiv = 1;
  long long sA1 = 0, sA2 = 0, sAm = 0, sAk = 0;
  long long sB1 = 0, sB2 = 0, sBk = 0, sBn = 0;
  long long sC1 = 0, sC2 = 0, sCm = 0, sCn = 0;
  const double *A = nullptr, *B = nullptr;
  double *C = nullptr;
  double alpha = 1.0, beta = 0.0;
  const double *alpha_dev = nullptr;
  const int *skip_dev = nullptr;   // if set and *skip_dev != 0 the launch does nothing
  // Live extents from device memory (a rank the device chose): with dyn_dev
  // set and R = max(*dyn_dev, 0), the product runs over min(N, dyn_n R)
  // columns if dyn_n > 0 and min(K, dyn_k R) terms if dyn_k > 0; outputs in
  // the columns beyond are not written. Plans and scratch are sized for
  // (M, N, K); such products run on the FP64 / emulated-format SIMT kernels.
  const int *dyn_dev = nullptr;
  int dyn_n = 0, dyn_k = 0;
  int prec = 0;                    // kPrecFP64, or the operand type of a low-precision product
  int role = kRoleAux;             // kernel-timer tag: kRoleMethod for the HaTT contractions
};

// Doubles of split-K scratch this GEMM needs (0 if it runs unsplit).
size_t gemm_scratch_doubles(const Gemm &g);
// First-use timing of candidate GEMM plans (on by default; see k_gemm.cu).
void set_gemm_autotune(bool on);
// TF32 / BF16 products on the tensor cores (tcgen05, FP32 accumulator in
// tensor memory); gemm_f64 dispatches to them by g.prec.
bool gemm_tc_supported(const Gemm &g);
size_t gemm_tc_scratch_doubles(const Gemm &g);
cudaError_t gemm_tc(const Gemm &g, double *scratch, int *counters, cudaStream_t st);
// FP64-accurate products on the BF16 tensor cores (slices of 6 bits, exact
// FP32 accumulation per level): gemm_f64 uses them for large FP64 products
// while the calling thread has switched them on.
void set_fp64_tensor_cores(bool on);
bool gemm_oz_applicable(const Gemm &g);
size_t gemm_oz_scratch_doubles(const Gemm &g);
cudaError_t gemm_oz(const Gemm &g, double *scratch, cudaStream_t st);
cudaError_t oz_error_word(int *value, bool clear);
// Error word set by a device wait that ran out (the kernel wrote NaN to its
// outputs, freed its tensor memory and returned): read (synchronizing the
// device) and clear it.
cudaError_t read_device_error(int *value);
cudaError_t clear_device_error();
// Health bits of the device error word (tt_device_error): a bounded wait ran
// out, a non-finite value reached a norm or a Gram matrix, a shifted Cholesky
// factorization still met a non-positive pivot. Each source file that sets a
// bit owns its word; read_device_error ORs them.
constexpr int kHealthTimeout = 1, kHealthNonfinite = 2, kHealthBreakdown = 4;
cudaError_t qr_health_word(int *value, bool clear);
cudaError_t misc_health_word(int *value, bool clear);
// Enqueue; `scratch` must hold gemm_scratch_doubles(g) doubles.
cudaError_t gemm_f64(const Gemm &g, double *scratch, cudaStream_t st);

// ------------------------------------------------------------ sketch RNG ---
struct SketchTable {
  int d;
  uint64_t seed;
  const uint64_t *seed_offset = nullptr;   // device: key = seed + *seed_offset
  uint32_t pair;
  long long offset[kMaxOrder + 1];   // element offset of core k inside `base`
  int a[kMaxOrder], n[kMaxOrder], b[kMaxOrder];
};
// Fill the sketch cores (contiguous at `base`, core k at base + offset[k]).
cudaError_t sketch_fill(const SketchTable &t, double *base, cudaStream_t st);
// Fill per-core pointers (used by the public tt_sketch_tt).
cudaError_t sketch_fill_ptrs(int d, const int64_t *n, const int64_t *ell, uint64_t seed,
                             uint32_t pair, double *const *cores, cudaStream_t st);
cudaError_t philox_raw(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                       long long count, cudaStream_t st);

// ----------------------------------------------------------------- misc ---
// out[0] = 1 / ||x||_F (1 if the norm is 0); `partials` holds >= 1024 doubles,
// `ticket` one unsigned int that must be 0 on entry (the kernel resets it).
cudaError_t inv_norm(const double *x, long long count, double *out, double *partials,
                     unsigned int *ticket, cudaStream_t st);
// First core of the Hadamard product: C[0, i, a*s + b] = Y[0, i, a] * Z[0, i, b].
cudaError_t pkp_first(const double *Y, const double *Z, int n, int r1, int s1, double *C,
                      cudaStream_t st);
cudaError_t set_value(double *x, long long count, double v, cudaStream_t st);
// X = I (m x m, row-major).
cudaError_t set_identity(double *X, int m, cudaStream_t st);
cudaError_t copy_f64(const double *src, double *dst, long long count, cudaStream_t st);
cudaError_t div_by_scalar(double *x, long long count, const double *divisor, cudaStream_t st);
// TT operations of the Allen-Cahn application (k_ops.cu).
cudaError_t laplacian_core(const double *u, int a, int n, int b, int pos, double inv_h2,
                           double *out, cudaStream_t st);
cudaError_t put_block(const double *src, int a, int n, int b, double coef, double *dst, int A,
                      int B, int ra, int rb, bool accumulate, cudaStream_t st);
// dst[(a*n + i)*rb + b] = src[(a*n + i)*lb + b] for a < ra, b < rb, with ra, rb
// read from ranks_dev[k], ranks_dev[k+1] (device int64) and bounds la x n x lb.
cudaError_t compact_core(const double *src, double *dst, int la, int n, int lb,
                         const long long *ranks_dev, int k, cudaStream_t st);
// out = sqrt(max(x, 0)) for a device scalar.
cudaError_t sqrt_scalar(const double *x, double *out, cudaStream_t st);

// --------------------------------------------------------------- QR ---
// In-place orthonormalization of the m x c row-major matrix S (leading
// dimension ldS >= c) by repeated Cholesky QR passes. Needs qr_scratch_doubles.
size_t qr_scratch_doubles(int m, int c);
cudaError_t qr_inplace(double *S, int m, int c, long long ldS, double *scratch, int *flags,
                       cudaStream_t st);

// ------------------------------------------------------------ truncation ---
size_t trunc_scratch_doubles(int la, int n, int lb, int lm, int nm);
// One right-to-left truncation step on core k of a padded left-orthogonal TT.
//   Xk   : la x n x lb padded core (columns >= ranks_dev[k+1] are zero)
//   Xkm1 : lm x nm x la padded core k-1
// Chooses rho = ranks_dev[k] <= min(la, cap) by the tolerance rule with
// delta2_dev[0] = delta^2, replaces Xk by its rho orthonormal right factor and
// multiplies the left factor into Xkm1; rows/cols beyond rho are zeroed.
// deep (tolerance mode) adds the second eigen level and the cross step, which
// resolve energies far below u ||B||^2; without it (rank cap only) the
// low-energy directions may stay mixed, which does not change a rank cut.
cudaError_t trunc_step(double *Xk, int la, int n, int lb, double *Xkm1, int lm, int nm,
                       int cap, const double *delta2_dev, long long *ranks_dev, int k, bool deep,
                       double *scratch, cudaStream_t st);
// Whether the truncation sweep may synchronize the stream (outside capture) to
// stop its cluster levels early; the batched entry point switches it off for
// the calling thread while it issues its lanes.
void set_host_sync(bool allowed);
// FP64 refinement of a start U (c x c, in place) of the eigenvectors of the
// symmetric c x c matrix G in one launch on a thread-block cluster
// (k_refine.cu), for c <= kEigFusedMax; *skip != 0 leaves U untouched.
// refine_cluster_available says whether the device can place the cluster.
constexpr int kEigFusedMax = 96;
constexpr int kMaxDevices = 64;
cudaError_t refine_cluster_available(bool *ok);
cudaError_t refine_cluster(const double *G, int c, double *U, double floor_norm, const int *skip,
                           cudaStream_t st);
// Eigenvectors (columns of U, c x c row-major) of the symmetric c x c matrix G.
size_t sym_eig_scratch_doubles(int c);
cudaError_t sym_eig(const double *G, int c, double *U, double *scratch, cudaStream_t st);
// HPCRL-2: keeps the columns of Uf = W V (x x c) whose norms exceed ep times the
// largest, packed (leading dimension R) into UR and, with the same columns of
// V, into VR; writes R (>= 1) to device memory.
cudaError_t select_directions(const double *Uf, const double *V, long long x, int c, double ep,
                              double *UR, double *VR, int *R, cudaStream_t st);
// delta2_dev = (tol * ||x|| )^2 / (d-1) for a device vector x.
cudaError_t trunc_delta2(const double *x, long long count, double tol, int d, double *delta2_dev,
                         double *partials, unsigned int *ticket, cudaStream_t st);
cudaError_t set_ranks(long long *ranks_dev, const long long *ranks_host, int count,
                      cudaStream_t st);

}  // namespace hatt
