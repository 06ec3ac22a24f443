// Task engine of the batched entry point: one persistent launch recompresses
// many independent Hadamard products (Algorithms 3 and 4 per pair).
//
// The host turns every pair's launch sequence into stages (a GEMM, a norm, a
// Cholesky factorization, ...) and every stage into tasks (its output tiles,
// element chunks or row blocks). Tasks sit in one global queue; resident CTAs
// take the next index with an atomic ticket, wait until the pair's completion
// counter reaches the task's prerequisite count (the tasks of all earlier
// stages of that pair), run it and count it done. A task only waits on tasks
// earlier in the queue, which CTAs already hold and are running, so the
// launch cannot deadlock whatever the number of resident CTAs; every wait is
// also bounded and records a timeout status instead of spinning forever.
#pragma once

#include <stdint.h>
#include "hatt_internal.cuh"

namespace hatt {

enum EngineStageType : int {
  kStSketch = 0,     // Gaussian sketch core (Definition 2.1), chunks of elements
  kStGemm = 1,       // strided batched GEMM, output tiles
  kStNormPart = 2,   // partial sums of squares of W^{(k)}, chunks
  kStNormFin = 3,    // 1 / ||W^{(k)}|| from the partial sums (one task)
  kStPkpFirst = 4,   // first core of the Hadamard product, chunks
  kStChol = 5,       // Cholesky QR pass: convergence test + factorization (one task)
  kStTrsm = 6,       // Cholesky QR pass: S <- S R^{-1}, row blocks
  kStSet = 7,        // out[0] = value (W^{(d)} = [1], its inverse norm)
};

// One stage of one pair (plain data, copied to the device as an array).
struct EngineStage {
  int type = 0;
  int pair = 0;
  int ntasks = 0;
  // GEMM: the same operand layout as hatt::Gemm, tile bm x bn (no split K)
  int M = 0, N = 0, K = 0, batch = 1, bdiv = 1;
  long long sA1 = 0, sA2 = 0, sAm = 0, sAk = 0;
  long long sB1 = 0, sB2 = 0, sBk = 0, sBn = 0;
  long long sC1 = 0, sC2 = 0, sCm = 0, sCn = 0;
  const double *A = nullptr, *B = nullptr;
  double *C = nullptr;
  const double *alpha_dev = nullptr;
  const int *skip_dev = nullptr;
  int prec = 0;                         // kPrecFP64 or kPrecFP32 operands
  int bm = 0, bn = 0, tiles_m = 0, tiles_n = 0;
  int bgroup = 1;                       // consecutive batch entries per task
  // element stages: x / out / count, chunked by `chunk`
  const double *x = nullptr;
  double *out = nullptr;
  double *part = nullptr;               // norm partial sums (ntasks of them)
  long long count = 0, chunk = 0;
  double value = 0.0;
  // sketch core: a x n x b entries, counter = (flat, core, pair id, 0), key = seed
  int a = 0, n = 0, b = 0, core = 0;
  uint64_t seed = 0;
  // first core: Y (n x r1), Z (n x s1)
  const double *Y = nullptr, *Z = nullptr;
  int r1 = 0, s1 = 0;
  // Cholesky QR pass on the m x c matrix S (ld c): Gram G, unit triangle Ut,
  // inverse diagonal y, flags (done, skip apply, passes, shifted passes)
  double *S = nullptr, *G = nullptr, *Ut = nullptr, *y = nullptr;
  int *flags = nullptr;
  int m = 0, c = 0;
};

struct EngineTask {
  int stage;       // index into the stage array
  int tile;        // tile / chunk / row block within the stage
  int pair;
  int need;        // completed tasks of this pair required before it runs
};

// Status word of a launch (device int), bits: kEngineTimeout when a wait ran
// out (the task then ran anyway on whatever its inputs held), kEngineNonfinite
// when a norm of W^{(k)} or a QR Gram matrix was not finite, kEngineBreakdown
// when a shifted Cholesky factorization still met a non-positive pivot.
constexpr int kEngineTimeout = 1, kEngineNonfinite = 2, kEngineBreakdown = 4;

constexpr int kEngineThreads = 256;
constexpr int kEngineMaxC = 128;        // largest Cholesky / TRSM width
constexpr int kEngineTrsmRows = 64;     // rows per TRSM task

// Per-CTA profile of a launch (long long words, kProfWords per CTA): [0] cycles
// from the CTA's start to its end, [1] cycles polling for prerequisites,
// [2] cycles taking tickets, [8 + t] cycles running tasks of stage type t,
// [16 + t] tasks of type t. Thread 0 reads clock64 around each phase.
constexpr int kProfWords = 24;
constexpr int kMaxProfBlocks = 2048;

// Dynamic shared memory of the persistent kernel for Cholesky / TRSM width max_c.
size_t engine_smem(int max_c);
// Resident CTAs of the persistent kernel on the current device (SMs x per SM).
cudaError_t engine_blocks(int max_c, int *blocks);
// The persistent launch over ntasks queued tasks; head, done and status must be
// zero on entry (done: one counter per pair).
cudaError_t engine_launch(const EngineStage *stages, const EngineTask *tasks, int ntasks,
                          int *head, int *done, int *status, long long spin_cap, int max_c,
                          int blocks, long long *prof, cudaStream_t st);
// Average time of the GEMM stage s run alone (all its tiles as one grid), for
// the autotuner; synchronizes the stream.
cudaError_t engine_gemm_time(const EngineStage &s, cudaStream_t st, float *ms);

}  // namespace hatt
