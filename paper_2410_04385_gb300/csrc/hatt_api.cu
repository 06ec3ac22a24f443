// C-ABI entry points of libhatt: argument checks, rank plans, workspace
// layout and the launch sequences of HaTT-1 (Algorithms 3 and 4), TT rounding
// (Algorithm 1) and the TT inner product.
//
// Every sequence is written once and run twice: a planning pass that only
// measures buffers and scratch (no launches) and an execution pass that carves
// the caller's workspace identically and enqueues the kernels on the caller's
// stream. No device memory is allocated and the stream is never synchronized.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "hatt.h"
#include "hatt_internal.cuh"
#include "engine.cuh"

using hatt::Gemm;
typedef long long ll;

namespace hatt {
namespace {
std::atomic<long long> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

thread_local bool t_programmatic = true;
void set_programmatic_launch(bool on) { t_programmatic = on; }
bool programmatic_launch() { return t_programmatic; }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// Kernel timer state (tt_kernel_timer_start / _stop). Guarded by a mutex;
// `active` is read without it on the launch path so that the timer costs one
// relaxed load when it is off.
namespace {
struct KernelTimer {
  std::mutex mu;
  std::atomic<bool> active{false};
  std::vector<cudaEvent_t> ev;     // 2 per slot
  std::vector<double> flops;
  std::vector<int> role;
  int used = 0;
};
KernelTimer g_timer;
}  // namespace

int timer_begin(cudaStream_t st) {
  if (!g_timer.active.load(std::memory_order_relaxed)) return -1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return -1;
  }
  std::lock_guard<std::mutex> lk(g_timer.mu);
  const int cap = (int)g_timer.flops.size();
  if (!g_timer.active.load() || g_timer.used >= cap) return -1;
  const int slot = g_timer.used++;
  if (cudaEventRecord(g_timer.ev[2 * slot], st) != cudaSuccess) {
    cudaGetLastError();
    g_timer.flops[slot] = -1.0;     // marks a slot without a valid start
  }
  return slot;
}

void timer_end(int slot, cudaStream_t st, double flops, int role) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_timer.mu);
  if (slot >= (int)g_timer.flops.size()) return;
  if (g_timer.flops[slot] < 0.0) return;
  if (cudaEventRecord(g_timer.ev[2 * slot + 1], st) != cudaSuccess) {
    cudaGetLastError();
    g_timer.flops[slot] = -1.0;
    return;
  }
  g_timer.flops[slot] = flops;
  g_timer.role[slot] = role;
}

namespace {
void timer_release() {   // caller holds g_timer.mu
  g_timer.active.store(false);
  for (cudaEvent_t e : g_timer.ev) cudaEventDestroy(e);
  g_timer.ev.clear();
  g_timer.flops.clear();
  g_timer.role.clear();
  g_timer.used = 0;
}
}  // namespace
}  // namespace hatt

namespace {

// ---------------------------------------------------------------- helpers ---

struct Ws {
  bool exec = false;
  char *base = nullptr;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T *p = exec ? reinterpret_cast<T *>(base + off) : nullptr;
    off += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
};

// One step of a launch sequence as recorded for the batched task engine.
struct RecOp {
  enum Kind { kGemm, kQr, kSketch, kSet, kNorm, kPkpFirst } kind;
  Gemm g;                                   // kGemm
  double *S = nullptr;                      // kQr: m x c, leading dimension c
  int m = 0, c = 0;
  double *out = nullptr;                    // kSketch core / kSet / kNorm target / kPkpFirst C
  const double *x = nullptr;                // kNorm input
  long long count = 0;
  double value = 0.0;
  int a = 0, n = 0, b = 0, core = 0;        // kSketch
  uint64_t seed = 0;
  const double *Y = nullptr, *Z = nullptr;  // kPkpFirst
  int r1 = 0, s1 = 0;
};

// Runs a launch sequence in planning, execution or recording mode.
struct Runner {
  bool exec = false;
  cudaStream_t st = nullptr;
  size_t scratch_need = 0;       // doubles
  double *scratch = nullptr;
  cudaError_t err = cudaSuccess;
  std::vector<RecOp> *rec = nullptr;   // recording: collect the steps, launch nothing

  bool live() const { return exec && err == cudaSuccess; }
  void check(cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
  }
  void gemm(const Gemm &g) {
    if (rec) {
      if (g.dyn_dev) err = cudaErrorInvalidValue;   // the engine takes host extents only
      RecOp o{RecOp::kGemm};
      o.g = g;
      rec->push_back(o);
      return;
    }
    if (!exec) {
      scratch_need = std::max(scratch_need, hatt::gemm_scratch_doubles(g));
      return;
    }
    if (err == cudaSuccess) check(hatt::gemm_f64(g, scratch, st));
  }
  void qr(double *S, int m, int c, ll ld, int *flags) {
    if (rec) {
      RecOp o{RecOp::kQr};
      o.S = S;
      o.m = m;
      o.c = c;
      if (ld != c) err = cudaErrorInvalidValue;   // the recorded QR keeps ld = c
      rec->push_back(o);
      return;
    }
    if (!exec) {
      scratch_need = std::max(scratch_need, hatt::qr_scratch_doubles(m, c));
      return;
    }
    if (err == cudaSuccess) check(hatt::qr_inplace(S, m, c, ld, scratch, flags, st));
  }
  // Direct launches of the HaTT sequence (no scratch): launched when live,
  // recorded when recording.
  void sketch(const hatt::SketchTable &t, double *base) {
    if (rec) {
      for (int k = 0; k < t.d; ++k) {
        RecOp o{RecOp::kSketch};
        o.out = base + t.offset[k];
        o.a = t.a[k]; o.n = t.n[k]; o.b = t.b[k]; o.core = k; o.seed = t.seed;
        rec->push_back(o);
      }
      return;
    }
    if (live()) check(hatt::sketch_fill(t, base, st));
  }
  void set(double *x, double v) {
    if (rec) {
      RecOp o{RecOp::kSet};
      o.out = x;
      o.value = v;
      rec->push_back(o);
      return;
    }
    if (live()) check(hatt::set_value(x, 1, v, st));
  }
  void zero_ticket(unsigned int *ticket) {
    if (rec) return;
    if (live()) check(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st));
  }
  void inv_norm(const double *x, ll count, double *out, double *partials, unsigned int *ticket) {
    if (rec) {
      RecOp o{RecOp::kNorm};
      o.x = x;
      o.count = count;
      o.out = out;
      rec->push_back(o);
      return;
    }
    if (live()) check(hatt::inv_norm(x, count, out, partials, ticket, st));
  }
  void pkp_first(const double *Y, const double *Z, int n, int r1, int s1, double *C) {
    if (rec) {
      RecOp o{RecOp::kPkpFirst};
      o.Y = Y; o.Z = Z; o.n = n; o.r1 = r1; o.s1 = s1; o.out = C;
      rec->push_back(o);
      return;
    }
    if (live()) check(hatt::pkp_first(Y, Z, n, r1, s1, C, st));
  }
  void eig(const double *G, int c, double *U) {
    if (!exec) {
      scratch_need = std::max(scratch_need, hatt::sym_eig_scratch_doubles(c));
      return;
    }
    if (err == cudaSuccess) check(hatt::sym_eig(G, c, U, scratch, st));
  }
  void trunc(double *Xk, int la, int n, int lb, double *Xkm1, int lm, int nm, int cap,
             const double *delta2, ll *ranks, int k, bool deep) {
    if (!exec) {
      scratch_need = std::max(scratch_need, hatt::trunc_scratch_doubles(la, n, lb, lm, nm));
      return;
    }
    if (err == cudaSuccess)
      check(hatt::trunc_step(Xk, la, n, lb, Xkm1, lm, nm, cap, delta2, ranks, k, deep, scratch, st));
  }
};

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TT_OK;
  cudaGetLastError();   // clear a sticky launch error of this thread
  return TT_ERR_CUDA;
}

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
  const char *pa = (const char *)a, *pb = (const char *)b;
  return pa < pb + nb && pb < pa + na;
}

const ll kIntMax = (1LL << 31) - 1;

// Basic structural checks of one TT descriptor (host arrays only).
int check_tt(const tt_t *A, bool need_cores) {
  if (!A || !A->n || !A->r) return TT_ERR_ARG;
  if (A->d < 1) return TT_ERR_SHAPE;
  if (A->d > hatt::kMaxOrder) return TT_ERR_RANK;
  if (need_cores && !A->cores) return TT_ERR_ARG;
  if (A->r[0] != 1 || A->r[A->d] != 1) return TT_ERR_SHAPE;
  for (int k = 0; k < A->d; ++k) {
    if (A->n[k] < 1 || A->r[k + 1] < 1) return TT_ERR_SHAPE;
    if (A->n[k] > kIntMax || A->r[k + 1] > kIntMax) return TT_ERR_RANK;
    if (need_cores && !A->cores[k]) return TT_ERR_ARG;
    if ((double)A->r[k] * A->n[k] * A->r[k + 1] > 1e15) return TT_ERR_RANK;
  }
  return TT_OK;
}

// Rank clamps shared by HaTT and rounding: l_k = min(l_req, cap_k, products of
// mode sizes on either side), then l_k <= l_{k-1} n_{k-1} and l_k <= n_k l_{k+1}.
std::vector<ll> clamp_ranks(int d, const int64_t *n, const std::vector<ll> &cap, ll lreq) {
  std::vector<ll> l(d + 1, 1);
  const ll big = 1LL << 40;   // saturating products: any rank bound is far below this
  auto smul = [big](ll a, ll b) { return (a > big / b) ? big : std::min(big, a * b); };
  for (int k = 1; k < d; ++k) {
    ll left = 1, right = 1;
    for (int j = 0; j < k; ++j) left = smul(left, (ll)n[j]);
    for (int j = k; j < d; ++j) right = smul(right, (ll)n[j]);
    l[k] = std::min(std::min(lreq, cap[k]), std::min(left, right));
  }
  for (int k = 1; k < d; ++k) l[k] = std::min(l[k], smul(l[k - 1], (ll)n[k - 1]));
  for (int k = d - 1; k >= 1; --k) l[k] = std::min(l[k], smul((ll)n[k], l[k + 1]));
  return l;
}

// ------------------------------------------------------------ HaTT-1 run ---

struct HattArgs {
  int d;
  const int64_t *n, *r, *s;
  std::vector<ll> ell;
  double *const *Y;
  double *const *Z;
  double *const *Xout;
  bool trunc;
  int cap;
  double tol;
  uint64_t seed;
  const uint64_t *seed_offset = nullptr;   // device word added to the key (graph replays)
  int prec = hatt::kPrecFP64;   // arithmetic of the HPCRL-1 products (A2/A3)
  int variant = 1;              // 1 = HPCRL-1 (Eq. (3.6)), 2 = HPCRL-2 (Eq. (3.7))
  double ep = 0.0;              // HPCRL-2: keep sigma > ep * ||W^{(k)}||_2
  bool fixed = false;           // output in the bound layout, zero past the kept ranks
  std::vector<ll> outb;         // output rank bound reported by the plan
};

struct HattBufs {
  double *R, *W, *winv, *T1, *T2, *Ca, *Cb, *Mb, *U1, *Xpad, *partials, *delta2;
  ll *ranks;
  ll *oranks;                   // fixed-rank output: the bound ranks on the device
  int *flags;
  unsigned int *ticket;
  std::vector<ll> Roff, Woff, Xoff;
  // HPCRL-2 only: Gram and eigenvectors of W^{(k+1)}, W V, its kept columns
  // U_R S_R, V_R, R_k V_R, and the two partial contractions (sized for R = l)
  double *G2 = nullptr, *V2 = nullptr, *Uf = nullptr, *UR = nullptr, *VR = nullptr,
         *Rv = nullptr, *P2 = nullptr, *P3 = nullptr;
  int *Rdev = nullptr;
};

HattBufs carve_hatt(Ws &ws, const HattArgs &a) {
  HattBufs b;
  const int d = a.d;
  const auto &n = a.n;
  const auto &r = a.r;
  const auto &s = a.s;
  const auto &l = a.ell;
  b.Roff.assign(d + 1, 0);
  b.Xoff.assign(d + 1, 0);
  for (int k = 0; k < d; ++k) {
    b.Roff[k + 1] = b.Roff[k] + l[k] * n[k] * l[k + 1];
    b.Xoff[k + 1] = b.Xoff[k] + l[k] * n[k] * l[k + 1];
  }
  b.Woff.assign(d + 2, 0);   // W[k] for k = 1..d at Woff[k]
  for (int k = 1; k <= d; ++k) b.Woff[k + 1] = b.Woff[k] + (ll)r[k] * s[k] * l[k];
  ll t1 = 1, t2 = 1, cmax = 1, mmax = 1, umax = 1;
  for (int k = 1; k < d; ++k) {
    t1 = std::max(t1, (ll)n[k] * r[k + 1] * s[k + 1] * l[k]);
    t2 = std::max(t2, (ll)n[k] * r[k + 1] * s[k] * l[k]);
  }
  for (int k = 0; k < d; ++k) cmax = std::max(cmax, l[k] * n[k] * (ll)r[k + 1] * s[k + 1]);
  for (int k = 0; k + 1 < d; ++k) {
    mmax = std::max(mmax, l[k + 1] * (ll)r[k + 1] * s[k + 1]);
    umax = std::max(umax, l[k + 1] * (ll)r[k + 1] * n[k + 1] * s[k + 2]);
  }
  b.R = ws.take<double>(b.Roff[d]);
  b.W = ws.take<double>(b.Woff[d + 1]);
  b.winv = ws.take<double>(d + 2);
  b.T1 = ws.take<double>(t1);
  b.T2 = ws.take<double>(t2);
  b.Ca = ws.take<double>(cmax);
  b.Cb = ws.take<double>(cmax);
  b.Mb = ws.take<double>(mmax);
  b.U1 = ws.take<double>(umax);
  b.Xpad = a.trunc ? ws.take<double>(b.Xoff[d]) : nullptr;
  b.partials = ws.take<double>(1024);
  b.delta2 = ws.take<double>(1);
  b.ranks = ws.take<ll>(d + 1);
  b.oranks = ws.take<ll>(d + 1);
  b.flags = ws.take<int>(8);
  b.ticket = ws.take<unsigned int>(1);
  if (a.variant == 2) {
    ll c2 = 1, xc = 1, rv = 1, p2 = 1, p3 = 1;
    for (int k = 1; k < d; ++k) {
      const ll x = (ll)r[k + 1] * s[k + 1], c = l[k + 1];
      c2 = std::max(c2, c * c);
      xc = std::max(xc, x * c);
      rv = std::max(rv, l[k] * n[k] * c);
      p2 = std::max(p2, (ll)n[k] * r[k + 1] * s[k] * c);
      p3 = std::max(p3, (ll)r[k] * s[k] * n[k] * c);
    }
    b.G2 = ws.take<double>(c2);
    b.V2 = ws.take<double>(c2);
    b.Uf = ws.take<double>(xc);
    b.UR = ws.take<double>(xc);
    b.VR = ws.take<double>(c2);
    b.Rv = ws.take<double>(rv);
    b.P2 = ws.take<double>(p2);
    b.P3 = ws.take<double>(p3);
    b.Rdev = ws.take<int>(1);
  }
  return b;
}

// HPCRL-2 step (Eq. (3.7)): W^{(k)} from the leading singular directions of
// W^{(k+1)} = U S V^T (x = r_{k+1} s_{k+1} rows, c = l_{k+1} columns).
//   G = W^T W, V = eig(G), U S = W V / ||W||  (right singular vectors from the
//   Gram matrix; column norms of W V are the singular values),
//   keep the R columns with sigma > ep * sigma_max, then with R terms
//   Rv[l][g][i]       = sum_c R_k[l][i][c] V_R[c][g]
//   P2[i][a'][b][g]   = sum_b' Z_k[b][i][b'] (U S)_R[a' s1 + b'][g]
//   P3[a][b][g][i]    = sum_a' Y_k[a][i][a'] P2[i][a'][b][g]
//   W^{(k)}[a s0 + b][l] = sum_{g,i} P3[a][b][g][i] Rv[l][g][i]
// (the W_L W_R^T form: W_L = P3, W_R = Rv). R stays in device memory: the
// buffers are laid out for R = c (leading dimension c for g), the products
// run over the first R columns (Rv, P2, P3) and the first n_k R terms of the
// last one (g outer, i inner, so the live terms are a prefix), all read R
// on the device. No host synchronization: the step can be captured.
void hpcrl2_step(Runner &run, const HattArgs &a, const HattBufs &b, int k, double *Wnext,
                 double *Wout) {
  const auto &n = a.n;
  const auto &r = a.r;
  const auto &s = a.s;
  const auto &l = a.ell;
  const int r0 = (int)r[k], r1 = (int)r[k + 1], s0 = (int)s[k], s1 = (int)s[k + 1];
  const int l0 = (int)l[k], c = (int)l[k + 1], nk = (int)n[k];
  const int x = r1 * s1;
  const double *Rk = run.exec ? b.R + b.Roff[k] : nullptr;
  const int *Rdev = run.exec ? b.Rdev : nullptr;
  {   // G = W^T W
    Gemm g;
    g.M = c; g.N = c; g.K = x;
    g.A = Wnext; g.sAm = 1; g.sAk = c;
    g.B = Wnext; g.sBk = c; g.sBn = 1;
    g.C = b.G2; g.sCm = c; g.sCn = 1;
    if (c > 1) run.gemm(g);
  }
  if (c > 1) {
    run.eig(b.G2, c, b.V2);
  } else if (run.live()) {
    run.check(hatt::set_value(b.V2, 1, 1.0, run.st));
  }
  {   // Uf = W V / ||W||
    Gemm g;
    g.M = x; g.N = c; g.K = c;
    g.A = Wnext; g.sAm = c; g.sAk = 1;
    g.B = b.V2; g.sBk = c; g.sBn = 1;
    g.C = b.Uf; g.sCm = c; g.sCn = 1;
    g.alpha_dev = run.exec ? b.winv + (k + 1) : nullptr;
    run.gemm(g);
  }
  if (run.live()) run.check(hatt::select_directions(b.Uf, b.V2, x, c, a.ep, b.UR, b.VR, b.Rdev, run.st));
  {   // Rv = R_k V_R, batched over l
    Gemm g;
    g.role = hatt::kRoleMethod;
    g.M = nk; g.N = c; g.K = c;
    g.batch = l0; g.bdiv = 1;
    g.A = Rk; g.sA1 = (ll)nk * c; g.sAm = c; g.sAk = 1;
    g.B = b.VR; g.sBk = c; g.sBn = 1;
    g.C = b.Rv; g.sC1 = (ll)c * nk; g.sCm = 1; g.sCn = nk;
    g.dyn_dev = Rdev; g.dyn_n = 1;
    g.prec = a.prec;
    run.gemm(g);
  }
  {   // P2, batched over (i, a')
    Gemm g;
    g.role = hatt::kRoleMethod;
    g.M = s0; g.N = c; g.K = s1;
    g.batch = nk * r1; g.bdiv = r1;
    g.A = a.Z ? a.Z[k] : nullptr; g.sA1 = s1; g.sA2 = 0; g.sAm = (ll)nk * s1; g.sAk = 1;
    g.B = b.UR; g.sB1 = 0; g.sB2 = (ll)s1 * c; g.sBk = c; g.sBn = 1;
    g.C = b.P2; g.sC1 = (ll)r1 * s0 * c; g.sC2 = (ll)s0 * c; g.sCm = c; g.sCn = 1;
    g.dyn_dev = Rdev; g.dyn_n = 1;
    g.prec = a.prec;
    run.gemm(g);
  }
  {   // P3, batched over (i, b)
    Gemm g;
    g.role = hatt::kRoleMethod;
    g.M = r0; g.N = c; g.K = r1;
    g.batch = nk * s0; g.bdiv = s0;
    g.A = a.Y ? a.Y[k] : nullptr; g.sA1 = r1; g.sA2 = 0; g.sAm = (ll)nk * r1; g.sAk = 1;
    g.B = b.P2; g.sB1 = (ll)r1 * s0 * c; g.sB2 = c; g.sBk = (ll)s0 * c; g.sBn = 1;
    g.C = b.P3; g.sC1 = 1; g.sC2 = (ll)c * nk; g.sCm = (ll)s0 * c * nk; g.sCn = nk;
    g.dyn_dev = Rdev; g.dyn_n = 1;
    g.prec = a.prec;
    run.gemm(g);
  }
  {   // W^{(k)} = W_L W_R^T over the n_k R live terms
    Gemm g;
    g.role = hatt::kRoleMethod;
    g.M = r0 * s0; g.N = l0; g.K = nk * c;
    g.A = b.P3; g.sAm = (ll)c * nk; g.sAk = 1;
    g.B = b.Rv; g.sBk = 1; g.sBn = (ll)c * nk;
    g.C = Wout; g.sCm = l0; g.sCn = 1;
    g.dyn_dev = Rdev; g.dyn_k = nk;
    g.prec = a.prec;
    run.gemm(g);
  }
}

void run_hatt(Runner &run, const HattArgs &a, const HattBufs &b) {
  const int d = a.d;
  const auto &n = a.n;
  const auto &r = a.r;
  const auto &s = a.s;
  const auto &l = a.ell;
  auto Wk = [&](int k) { return run.exec ? b.W + b.Woff[k] : nullptr; };
  auto Xk = [&](int k) -> double * {
    if (!run.exec) return nullptr;
    return a.trunc ? b.Xpad + b.Xoff[k] : a.Xout[k];
  };

  if (d == 1) {   // the single core Y_1(i) Z_1(i)
    if (run.exec) run.pkp_first(a.Y[0], a.Z[0], (int)n[0], 1, 1, a.Xout[0]);
    return;
  }

  // A1: sketch cores R_k (Definition 2.1)
  if (run.live()) {
    hatt::SketchTable t;
    t.d = d;
    t.seed = a.seed;
    t.seed_offset = a.seed_offset;
    t.pair = 0;
    for (int k = 0; k <= d; ++k) t.offset[k] = b.Roff[k];
    for (int k = 0; k < d; ++k) {
      t.a[k] = (int)l[k];
      t.n[k] = (int)n[k];
      t.b[k] = (int)l[k + 1];
    }
    run.sketch(t, b.R);
    run.set(Wk(d), 1.0);                                          // W^{(d)} = [1]
    run.set(b.winv + d, 1.0);
    run.zero_ticket(b.ticket);
  }

  // A2/A3: HPCRL-1, W^{(k)} from W^{(k+1)} and cores k of Y, Z, R (Eq. (3.6))
  for (int k = d - 1; k >= 1; --k) {
    const int r0 = (int)r[k], r1 = (int)r[k + 1], s0 = (int)s[k], s1 = (int)s[k + 1];
    const int l0 = (int)l[k], l1 = (int)l[k + 1], nk = (int)n[k];
    const double *Rk = b.R + b.Roff[k];
    if (a.variant == 2) {
      hpcrl2_step(run, a, b, k, Wk(k + 1), Wk(k));
      if (run.live()) run.inv_norm(Wk(k), (ll)r0 * s0 * l0, b.winv + k, b.partials, b.ticket);
      continue;
    }
    {   // S1: T1[i][x][lam] = sum_g W[x][g] R_k[lam][i][g] / ||W||
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = r1 * s1; g.N = l0; g.K = l1;
      g.batch = nk; g.bdiv = 1;
      g.A = Wk(k + 1); g.sA1 = 0; g.sAm = l1; g.sAk = 1;
      g.B = Rk; g.sB1 = l1; g.sBk = 1; g.sBn = (ll)nk * l1;
      g.C = b.T1; g.sC1 = (ll)r1 * s1 * l0; g.sCm = l0; g.sCn = 1;
      g.alpha_dev = b.winv ? b.winv + (k + 1) : nullptr;
      g.prec = a.prec;
      run.gemm(g);
    }
    {   // S2: T2[i][a'][b][lam] = sum_b' Z_k[b][i][b'] T1[i][a'][b'][lam]
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = s0; g.N = l0; g.K = s1;
      g.batch = nk * r1; g.bdiv = r1;
      g.A = a.Y ? a.Z[k] : nullptr; g.sA1 = s1; g.sA2 = 0; g.sAm = (ll)nk * s1; g.sAk = 1;
      g.B = b.T1; g.sB1 = (ll)r1 * s1 * l0; g.sB2 = (ll)s1 * l0; g.sBk = l0; g.sBn = 1;
      g.C = b.T2; g.sC1 = (ll)r1 * s0 * l0; g.sC2 = (ll)s0 * l0; g.sCm = l0; g.sCn = 1;
      g.prec = a.prec;
      run.gemm(g);
    }
    {   // S3: W[a][b][lam] = sum_{i,a'} Y_k[a][i][a'] T2[i][a'][b][lam]
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = r0; g.N = s0 * l0; g.K = nk * r1;
      g.A = a.Y ? a.Y[k] : nullptr; g.sAm = (ll)nk * r1; g.sAk = 1;
      g.B = b.T2; g.sBk = (ll)s0 * l0; g.sBn = 1;
      g.C = Wk(k); g.sCm = (ll)s0 * l0; g.sCn = 1;
      g.prec = a.prec;
      run.gemm(g);
    }
    if (run.live()) run.inv_norm(Wk(k), (ll)r0 * s0 * l0, b.winv + k, b.partials, b.ticket);
  }

  // A4-A8: left-to-right pass (Algorithm 4)
  double *C = b.Ca, *Cn = b.Cb;
  if (run.live()) run.pkp_first(a.Y[0], a.Z[0], (int)n[0], (int)r[1], (int)s[1], C);
  for (int k = 0; k + 1 < d; ++k) {
    const ll m = l[k] * n[k];
    const int L = (int)l[k + 1];
    const int r1 = (int)r[k + 1], s1 = (int)s[k + 1], r2 = (int)r[k + 2], s2 = (int)s[k + 2];
    const int n1 = (int)n[k + 1];
    const int rs = r1 * s1;
    double *Q = Xk(k);
    {   // A5: S = C_k W^{(k+1)} / ||W||
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = (int)m; g.N = L; g.K = rs;
      g.A = C; g.sAm = rs; g.sAk = 1;
      g.B = Wk(k + 1); g.sBk = L; g.sBn = 1;
      g.C = Q; g.sCm = L; g.sCn = 1;
      g.alpha_dev = b.winv ? b.winv + (k + 1) : nullptr;
      run.gemm(g);
    }
    run.qr(Q, (int)m, L, L, b.flags);                // A6
    {   // A7: M = Q^T C_k
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = L; g.N = rs; g.K = (int)m;
      g.A = Q; g.sAm = 1; g.sAk = L;
      g.B = C; g.sBk = rs; g.sBn = 1;
      g.C = b.Mb; g.sCm = rs; g.sCn = 1;
      run.gemm(g);
    }
    {   // A8 stage 1: U1[(g,a)][(i,b')] = sum_b M[g][a][b] Z_{k+1}[b][i][b']
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = L * r1; g.N = n1 * s2; g.K = s1;
      g.A = b.Mb; g.sAm = s1; g.sAk = 1;
      g.B = a.Z ? a.Z[k + 1] : nullptr; g.sBk = (ll)n1 * s2; g.sBn = 1;
      g.C = b.U1; g.sCm = (ll)n1 * s2; g.sCn = 1;
      run.gemm(g);
    }
    double *dst = (k + 2 == d) ? Xk(d - 1) : Cn;
    {   // A8 stage 2: C_{k+1}[g][i][a'][b'] = sum_a Y_{k+1}[a][i][a'] U1[g][a][i][b']
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = r2; g.N = s2; g.K = r1;
      g.batch = L * n1; g.bdiv = n1;
      g.A = a.Y ? a.Y[k + 1] : nullptr; g.sA1 = 0; g.sA2 = r2; g.sAm = 1; g.sAk = (ll)n1 * r2;
      g.B = b.U1; g.sB1 = (ll)r1 * n1 * s2; g.sB2 = s2; g.sBk = (ll)n1 * s2; g.sBn = 1;
      g.C = dst; g.sC1 = (ll)n1 * r2 * s2; g.sC2 = (ll)r2 * s2; g.sCm = s2; g.sCn = 1;
      run.gemm(g);
    }
    std::swap(C, Cn);
  }

  if (!a.trunc) return;
  // A9: right-to-left truncation of the left-orthogonal result (padded)
  if (run.live()) {
    run.check(hatt::set_ranks(b.ranks, l.data(), d + 1, run.st));
    run.check(hatt::trunc_delta2(Xk(d - 1), l[d - 1] * n[d - 1], a.tol, d, b.delta2, b.partials,
                                 b.ticket, run.st));
  }
  for (int k = d - 1; k >= 1; --k)
    run.trunc(Xk(k), (int)l[k], (int)n[k], (int)l[k + 1], Xk(k - 1), (int)l[k - 1], (int)n[k - 1],
              a.cap, b.delta2, b.ranks, k, a.tol > 0.0);
  // compact to the kept ranks, or (fixed ranks) to the bound layout, where the
  // rows and columns past the kept ranks are already zero
  if (run.live() && a.fixed)
    run.check(hatt::set_ranks(b.oranks, a.outb.data(), d + 1, run.st));
  if (run.live())
    for (int k = 0; k < d; ++k)
      run.check(hatt::compact_core(Xk(k), a.Xout[k], (int)l[k], (int)n[k], (int)l[k + 1],
                                   a.fixed ? b.oranks : b.ranks, k, run.st));
}

// Planning + argument checks shared by plan and execute.
int prepare_hatt(const tt_t *Y, const tt_t *Z, const tt_opts *o, bool need_cores, HattArgs &a) {
  int st = check_tt(Y, need_cores);
  if (st != TT_OK) return st;
  st = check_tt(Z, need_cores);
  if (st != TT_OK) return st;
  if (!o) return TT_ERR_ARG;
  if (Y->d != Z->d) return TT_ERR_SHAPE;
  for (int k = 0; k < Y->d; ++k)
    if (Y->n[k] != Z->n[k]) return TT_ERR_SHAPE;
  if (o->max_rank < 0 || o->sketch_rank < 0 || o->oversample < 0 || !(o->tol >= 0.0) ||
      !std::isfinite(o->tol))
    return TT_ERR_ARG;
  if (o->precision < TT_FP64 || o->precision > TT_FP64_TC) return TT_ERR_ARG;
  if (o->variant != 1 && o->variant != 2) return TT_ERR_ARG;
  if (o->variant == 2 && (!(o->ep >= 0.0) || !(o->ep < 1.0))) return TT_ERR_ARG;
  if (o->fixed_ranks != 0 && o->fixed_ranks != 1) return TT_ERR_ARG;
  a.variant = o->variant;
  a.ep = o->ep;
  a.fixed = o->fixed_ranks == 1;
  a.prec = o->precision == TT_FP64_TC ? hatt::kPrecFP64 : o->precision;
  const int d = Y->d;
  a.d = d;
  a.n = Y->n;
  a.r = Y->r;
  a.s = Z->r;
  std::vector<ll> rs(d + 1);
  ll pkp = 1;
  for (int k = 0; k <= d; ++k) {
    rs[k] = (ll)Y->r[k] * Z->r[k];
    pkp = std::max(pkp, rs[k]);
  }
  ll lreq = o->sketch_rank > 0 ? o->sketch_rank
                               : (o->max_rank > 0 ? o->max_rank + o->oversample : pkp);
  a.ell = clamp_ranks(d, Y->n, rs, std::max<ll>(lreq, 1));
  for (int k = 0; k <= d; ++k)
    if (a.ell[k] > hatt::kMaxSmall) return TT_ERR_RANK;
  // every GEMM dimension must fit in int
  for (int k = 0; k < d; ++k) {
    if (a.ell[k] * Y->n[k] > kIntMax) return TT_ERR_RANK;
    if ((ll)Y->r[k + 1] * Z->r[k + 1] * Y->n[k] * std::max<ll>(a.ell[k], 1) > 4e9) return TT_ERR_RANK;
  }
  a.cap = (int)std::min<ll>(o->max_rank, hatt::kMaxSmall);
  a.tol = o->tol;
  a.seed = o->seed;
  a.seed_offset = o->seed_offset;
  bool below = false;
  for (int k = 1; k < d; ++k) below = below || (o->max_rank > 0 && a.ell[k] > o->max_rank);
  a.trunc = d > 1 && (o->tol > 0.0 || below);
  a.outb = a.ell;
  if (a.fixed && a.trunc && a.cap > 0)
    for (int k = 0; k <= d; ++k) a.outb[k] = std::min<ll>(a.ell[k], a.cap);
  return TT_OK;
}

// ------------------------------------------------------------- rounding ---

struct RoundArgs {
  int d;
  const int64_t *n, *r;
  std::vector<ll> b;      // bound ranks after the left-to-right QR sweep
  double *const *A;
  double *const *Bout;
  int cap;
  double tol;
  bool fixed = false;     // output in the bound layout outb, zero past the kept ranks
  std::vector<ll> outb;   // output rank bound reported by the plan
};

struct RoundBufs {
  double *Xpad, *Ca, *Cb, *Mb, *partials, *delta2;
  ll *ranks, *oranks;
  int *flags;
  unsigned int *ticket;
  std::vector<ll> Xoff;
};

RoundBufs carve_round(Ws &ws, const RoundArgs &a) {
  RoundBufs u;
  const int d = a.d;
  u.Xoff.assign(d + 1, 0);
  ll cmax = 1, mmax = 1;
  for (int k = 0; k < d; ++k) {
    u.Xoff[k + 1] = u.Xoff[k] + a.b[k] * a.n[k] * a.b[k + 1];
    cmax = std::max(cmax, a.b[k] * a.n[k] * (ll)a.r[k + 1]);
    mmax = std::max(mmax, a.b[k + 1] * (ll)a.r[k + 1]);
  }
  u.Xpad = ws.take<double>(u.Xoff[d]);
  u.Ca = ws.take<double>(cmax);
  u.Cb = ws.take<double>(cmax);
  u.Mb = ws.take<double>(mmax);
  u.partials = ws.take<double>(1024);
  u.delta2 = ws.take<double>(1);
  u.ranks = ws.take<ll>(d + 1);
  u.oranks = ws.take<ll>(d + 1);
  u.flags = ws.take<int>(8);
  u.ticket = ws.take<unsigned int>(1);
  return u;
}

void run_round(Runner &run, const RoundArgs &a, const RoundBufs &u) {
  const int d = a.d;
  const auto &n = a.n;
  const auto &r = a.r;
  const auto &bnd = a.b;
  auto Xk = [&](int k) { return run.exec ? u.Xpad + u.Xoff[k] : nullptr; };
  if (run.live()) {
    run.check(cudaMemsetAsync(u.ticket, 0, sizeof(unsigned int), run.st));
    run.check(hatt::copy_f64(a.A[0], u.Ca, n[0] * (ll)r[1], run.st));
  }
  double *C = u.Ca, *Cn = u.Cb;
  for (int k = 0; k + 1 < d; ++k) {
    const ll m = bnd[k] * n[k];
    const int cols = (int)r[k + 1];
    const int c = (int)bnd[k + 1];
    const int n1 = (int)n[k + 1], r2 = (int)r[k + 2];
    double *Q = Xk(k);
    const double *Msrc;
    if (c == cols) {
      if (run.live()) run.check(hatt::copy_f64(C, Q, m * cols, run.st));
      run.qr(Q, (int)m, c, c, u.flags);
      Gemm g;   // M = Q^T C
      g.M = c; g.N = cols; g.K = (int)m;
      g.A = Q; g.sAm = 1; g.sAk = c;
      g.B = C; g.sBk = cols; g.sBn = 1;
      g.C = u.Mb; g.sCm = cols; g.sCn = 1;
      run.gemm(g);
      Msrc = u.Mb;
    } else {   // wide unfolding: Q = I, the whole core moves right
      if (run.live()) run.check(hatt::set_identity(Q, (int)m, run.st));
      Msrc = C;
    }
    double *dst = (k + 2 == d) ? Xk(d - 1) : Cn;
    Gemm g;   // C_{k+1} = M H(A_{k+1})
    g.M = c; g.N = n1 * r2; g.K = cols;
    g.A = Msrc; g.sAm = cols; g.sAk = 1;
    g.B = a.A ? a.A[k + 1] : nullptr; g.sBk = (ll)n1 * r2; g.sBn = 1;
    g.C = dst; g.sCm = (ll)n1 * r2; g.sCn = 1;
    run.gemm(g);
    std::swap(C, Cn);
  }
  if (run.live()) {
    run.check(hatt::set_ranks(u.ranks, bnd.data(), d + 1, run.st));
    run.check(hatt::trunc_delta2(Xk(d - 1), bnd[d - 1] * n[d - 1], a.tol, d, u.delta2, u.partials,
                                 u.ticket, run.st));
  }
  for (int k = d - 1; k >= 1; --k)
    run.trunc(Xk(k), (int)bnd[k], (int)n[k], (int)bnd[k + 1], Xk(k - 1), (int)bnd[k - 1],
              (int)n[k - 1], a.cap, u.delta2, u.ranks, k, a.tol > 0.0);
  if (run.live() && a.fixed)
    run.check(hatt::set_ranks(u.oranks, a.outb.data(), d + 1, run.st));
  if (run.live())
    for (int k = 0; k < d; ++k)
      run.check(hatt::compact_core(Xk(k), a.Bout[k], (int)bnd[k], (int)n[k], (int)bnd[k + 1],
                                   a.fixed ? u.oranks : u.ranks, k, run.st));
}

int prepare_round(const tt_t *A, ll max_rank, double tol, int fixed, bool need_cores,
                  RoundArgs &a) {
  int st = check_tt(A, need_cores);
  if (st != TT_OK) return st;
  if (max_rank < 0 || !(tol >= 0.0) || !std::isfinite(tol)) return TT_ERR_ARG;
  if (fixed != 0 && fixed != 1) return TT_ERR_ARG;
  const int d = A->d;
  a.d = d;
  a.n = A->n;
  a.r = A->r;
  a.b.assign(d + 1, 1);
  for (int k = 0; k + 1 < d; ++k) a.b[k + 1] = std::min<ll>(A->r[k + 1], a.b[k] * A->n[k]);
  for (int k = 0; k <= d; ++k)
    if (a.b[k] > hatt::kMaxSmall || A->r[k] > hatt::kMaxSmall) return TT_ERR_RANK;
  for (int k = 0; k < d; ++k)
    if (a.b[k] * A->n[k] > kIntMax) return TT_ERR_RANK;
  a.cap = (int)std::min<ll>(max_rank, hatt::kMaxSmall);
  a.tol = tol;
  a.fixed = fixed == 1;
  a.outb = a.b;
  if (a.fixed && a.cap > 0)
    for (int k = 0; k <= d; ++k) a.outb[k] = std::min<ll>(a.b[k], a.cap);
  return TT_OK;
}

// ----------------------------------------------------------------- dot ---

struct DotBufs {
  double *Ga, *Gb, *T;
};

DotBufs carve_dot(Ws &ws, const tt_t *A, const tt_t *B) {
  DotBufs u;
  ll g = 1, t = 1;
  for (int k = 0; k <= A->d; ++k) g = std::max(g, (ll)A->r[k] * B->r[k]);
  for (int k = 0; k < A->d; ++k) t = std::max(t, (ll)A->r[k] * A->n[k] * B->r[k + 1]);
  u.Ga = ws.take<double>(g);
  u.Gb = ws.take<double>(g);
  u.T = ws.take<double>(t);
  return u;
}

void run_dot(Runner &run, const tt_t *A, const tt_t *B, const DotBufs &u, double *out) {
  double *G = u.Ga, *Gn = u.Gb;
  if (run.live()) run.check(hatt::set_value(G, 1, 1.0, run.st));
  for (int k = 0; k < A->d; ++k) {
    const int a0 = (int)A->r[k], a1 = (int)A->r[k + 1];
    const int b0 = (int)B->r[k], b1 = (int)B->r[k + 1], nk = (int)A->n[k];
    {   // T = G H(B_k)
      Gemm g;
      g.M = a0; g.N = nk * b1; g.K = b0;
      g.A = G; g.sAm = b0; g.sAk = 1;
      g.B = B->cores ? B->cores[k] : nullptr; g.sBk = (ll)nk * b1; g.sBn = 1;
      g.C = u.T; g.sCm = (ll)nk * b1; g.sCn = 1;
      run.gemm(g);
    }
    {   // G' = V(A_k)^T V(T)
      Gemm g;
      g.M = a1; g.N = b1; g.K = a0 * nk;
      g.A = A->cores ? A->cores[k] : nullptr; g.sAm = 1; g.sAk = a1;
      g.B = u.T; g.sBk = b1; g.sBn = 1;
      g.C = (k + 1 == A->d) ? out : Gn; g.sCm = b1; g.sCn = 1;
      run.gemm(g);
    }
    std::swap(G, Gn);
  }
}

int prepare_dot(const tt_t *A, const tt_t *B, bool need_cores) {
  int st = check_tt(A, need_cores);
  if (st != TT_OK) return st;
  st = check_tt(B, need_cores);
  if (st != TT_OK) return st;
  if (A->d != B->d) return TT_ERR_SHAPE;
  for (int k = 0; k < A->d; ++k) {
    if (A->n[k] != B->n[k]) return TT_ERR_SHAPE;
    if ((ll)A->r[k] * A->n[k] > kIntMax || (ll)B->r[k + 1] * B->n[k] > kIntMax) return TT_ERR_RANK;
  }
  return TT_OK;
}

template <class Carve, class Run>
size_t measure(Carve carve, Run runf) {
  Ws ws;
  Runner run;
  auto bufs = carve(ws);
  runf(run, bufs);
  ws.take<int>(hatt::kTileCounters);
  ws.take<double>(run.scratch_need);
  return ws.off + 256;
}

// Switches the FP64-accurate tensor-core products on for one call.
struct Fp64TcScope {
  explicit Fp64TcScope(bool on) { hatt::set_fp64_tensor_cores(on); }
  ~Fp64TcScope() { hatt::set_fp64_tensor_cores(false); }
};

// While a batch issues its lanes: the truncation sweep does not synchronize,
// and kernels are launched without programmatic serialization.
struct BatchScope {
  BatchScope() {
    hatt::set_host_sync(false);
    hatt::set_programmatic_launch(false);
  }
  ~BatchScope() {
    hatt::set_host_sync(true);
    hatt::set_programmatic_launch(true);
  }
};

// Makes a tile-counter array current for the calling thread during one call.
struct TileCounterScope {
  explicit TileCounterScope(int *p) { hatt::set_tile_counters(p); }
  ~TileCounterScope() { hatt::set_tile_counters(nullptr); }
};

template <class Carve, class Run>
int execute(void *workspace, size_t wsb, cudaStream_t st, Carve carve, Run runf) {
  // planning pass: scratch size
  Ws pws;
  Runner plan;
  auto pb = carve(pws);
  runf(plan, pb);
  // execution pass on the caller's workspace
  Ws ws;
  ws.exec = true;
  ws.base = (char *)workspace;
  auto bufs = carve(ws);
  Runner run;
  run.exec = true;
  run.st = st;
  int *counters = ws.take<int>(hatt::kTileCounters);
  run.scratch = ws.take<double>(plan.scratch_need);
  if (ws.off > wsb) return TT_ERR_WORKSPACE;
  run.check(cudaMemsetAsync(counters, 0, hatt::kTileCounters * sizeof(int), st));
  TileCounterScope scope(counters);
  runf(run, bufs);
  return from_cuda(run.err);
}

bool aligned(const void *p) { return ((uintptr_t)p & 255u) == 0; }

// ------------------------------------------------- batched task engine ---
// Host planner of tt_batched_*: every pair's launch sequence of run_hatt
// (HaTT-1 without the truncation sweep) becomes a chain of engine stages in
// the pair's own workspace; the stages of all pairs are interleaved into one
// task queue for the persistent kernel of k_engine.cu.

struct EnginePair {
  HattArgs a;
  size_t ws_off = 0, ws_bytes = 0;   // the pair's region of the workspace
  double cost = 0.0;                 // predicted flops (Section 4 model)
  std::vector<hatt::EngineStage> stages;
  std::vector<int> group;            // stages with the same group id share prerequisites
};

// Workspace of one pair: carve_hatt's buffers plus the QR's Gram, triangle,
// diagonal and per-core flags, and the norm partial sums.
struct EngineBufs {
  HattBufs h;
  double *G = nullptr, *Ut = nullptr, *y = nullptr, *part = nullptr;
  int *qflags = nullptr;
};

constexpr long long kEngineChunk = 32768;   // elements per element-wise task

EngineBufs carve_engine(Ws &ws, const HattArgs &a) {
  EngineBufs e;
  e.h = carve_hatt(ws, a);
  ll cmax = 1, wmax = 1;
  for (int k = 0; k <= a.d; ++k) cmax = std::max(cmax, a.ell[k]);
  for (int k = 1; k <= a.d; ++k) wmax = std::max(wmax, (ll)a.r[k] * a.s[k] * a.ell[k]);
  e.G = ws.take<double>(cmax * cmax);
  e.Ut = ws.take<double>(cmax * cmax);
  e.y = ws.take<double>(cmax);
  e.part = ws.take<double>((wmax + kEngineChunk - 1) / kEngineChunk + 1);
  e.qflags = ws.take<int>(4 * (size_t)a.d);
  return e;
}

// Tile edge for a dimension X: X itself if it fits under cap, else the edge in
// [cap/2, cap] with the least padding.
int eng_edge(int X, int cap) {
  if (X <= cap) return X;
  int best = cap;
  long long best_pad = ((X + cap - 1) / cap) * (long long)cap;
  for (int t = cap - 1; t >= std::max(1, cap / 2); --t) {
    const long long pad = ((X + t - 1) / (long long)t) * t;
    if (pad < best_pad) { best_pad = pad; best = t; }
  }
  return best;
}

// Tiles of bm x bn outputs; a task takes bgroup consecutive batch entries of
// one tile position, enough for ~kTaskFma multiply-adds (the per-task queue
// and wait overhead is a few microseconds).
constexpr double kTaskFma = 131072.0;

void eng_set_tiles(hatt::EngineStage &s, int bm, int bn) {
  s.bm = bm;
  s.bn = bn;
  s.tiles_m = (s.M + bm - 1) / bm;
  s.tiles_n = (s.N + bn - 1) / bn;
  const double work = (double)bm * bn * s.K;
  s.bgroup = (int)std::min<double>(s.batch, std::max(1.0, std::ceil(kTaskFma / work)));
  s.ntasks = s.tiles_m * s.tiles_n * ((s.batch + s.bgroup - 1) / s.bgroup);
}

// Candidate tile shapes (bm x bn <= 4096, each edge <= 128) for a GEMM.
std::vector<std::pair<int, int>> eng_tile_candidates(const hatt::EngineStage &s) {
  static const int caps[][2] = {{32, 32}, {64, 32}, {32, 64}, {64, 64}, {128, 32}, {32, 128}};
  std::vector<std::pair<int, int>> out;
  for (const auto &cp : caps) {
    const int bn = eng_edge(s.N, cp[1]);
    const int bm = eng_edge(s.M, std::min(cp[0], 4096 / bn));
    if (bm * bn > 4096) continue;
    std::pair<int, int> t(bm, bn);
    if (std::find(out.begin(), out.end(), t) == out.end()) out.push_back(t);
  }
  return out;
}

// Analytic default: the candidate with the least padded work per SM, preferring
// larger tiles (fewer tasks) on ties.
void eng_default_tiles(hatt::EngineStage &s) {
  double best = 1e300;
  int bm = 0, bn = 0;
  for (const auto &t : eng_tile_candidates(s)) {
    const double tiles = std::ceil((double)s.M / t.first) * std::ceil((double)s.N / t.second) * s.batch;
    const double work = tiles * t.first * t.second;       // padded outputs
    const double cost = work + tiles * 512.0;              // a per-task overhead in output units
    if (cost < best) { best = cost; bm = t.first; bn = t.second; }
  }
  eng_set_tiles(s, bm, bn);
}

hatt::EngineStage eng_gemm(const Gemm &g, int pair) {
  hatt::EngineStage s;
  s.type = hatt::kStGemm;
  s.pair = pair;
  s.M = g.M; s.N = g.N; s.K = g.K; s.batch = g.batch; s.bdiv = g.bdiv;
  s.sA1 = g.sA1; s.sA2 = g.sA2; s.sAm = g.sAm; s.sAk = g.sAk;
  s.sB1 = g.sB1; s.sB2 = g.sB2; s.sBk = g.sBk; s.sBn = g.sBn;
  s.sC1 = g.sC1; s.sC2 = g.sC2; s.sCm = g.sCm; s.sCn = g.sCn;
  s.A = g.A; s.B = g.B; s.C = g.C;
  s.alpha_dev = g.alpha_dev;
  s.skip_dev = g.skip_dev;
  s.prec = g.prec;
  eng_default_tiles(s);
  return s;
}

hatt::EngineStage eng_elem(int type, int pair, long long count) {
  hatt::EngineStage s;
  s.type = type;
  s.pair = pair;
  s.count = count;
  s.chunk = kEngineChunk;
  s.ntasks = (int)std::max<long long>(1, (count + kEngineChunk - 1) / kEngineChunk);
  return s;
}

// Expands one pair's recorded launch sequence into engine stages. QR k uses
// flag words qflags + 4 k (cleared before every run).
void eng_expand(const std::vector<RecOp> &ops, const EngineBufs &eb, int pair,
                std::vector<hatt::EngineStage> &out, std::vector<int> &group) {
  int qr_index = 0, gid = 0;
  for (size_t i = 0; i < ops.size(); ++i) {
    const RecOp &o = ops[i];
    switch (o.kind) {
      case RecOp::kGemm:
        out.push_back(eng_gemm(o.g, pair));
        group.push_back(++gid);
        break;
      case RecOp::kSketch: {   // the sketch cores depend on nothing: one group
        hatt::EngineStage s = eng_elem(hatt::kStSketch, pair, (long long)o.a * o.n * o.b);
        s.out = o.out; s.a = o.a; s.n = o.n; s.b = o.b; s.core = o.core; s.seed = o.seed;
        out.push_back(s);
        group.push_back((i > 0 && ops[i - 1].kind == RecOp::kSketch) ? gid : ++gid);
        break;
      }
      case RecOp::kSet: {
        hatt::EngineStage s = eng_elem(hatt::kStSet, pair, 1);
        s.out = o.out; s.value = o.value;
        out.push_back(s);
        group.push_back(++gid);
        break;
      }
      case RecOp::kNorm: {
        hatt::EngineStage p = eng_elem(hatt::kStNormPart, pair, o.count);
        p.x = o.x; p.part = eb.part;
        hatt::EngineStage f = eng_elem(hatt::kStNormFin, pair, p.ntasks);
        f.ntasks = 1; f.part = eb.part; f.out = o.out;
        out.push_back(p);
        group.push_back(++gid);
        out.push_back(f);
        group.push_back(++gid);
        break;
      }
      case RecOp::kPkpFirst: {
        hatt::EngineStage s = eng_elem(hatt::kStPkpFirst, pair, (long long)o.n * o.r1 * o.s1);
        s.Y = o.Y; s.Z = o.Z; s.n = o.n; s.r1 = o.r1; s.s1 = o.s1; s.out = o.out;
        out.push_back(s);
        group.push_back(++gid);
        break;
      }
      case RecOp::kQr: {
        int *flags = eb.qflags + 4 * qr_index++;
        for (int p = 0; p < 6; ++p) {
          Gemm g;                                  // G = S^T S, no-op once done
          g.M = o.c; g.N = o.c; g.K = o.m;
          g.A = o.S; g.sAm = 1; g.sAk = o.c;
          g.B = o.S; g.sBk = o.c; g.sBn = 1;
          g.C = eb.G; g.sCm = o.c; g.sCn = 1;
          g.skip_dev = flags;
          out.push_back(eng_gemm(g, pair));
          group.push_back(++gid);
          hatt::EngineStage ch;
          ch.type = hatt::kStChol; ch.pair = pair; ch.ntasks = 1;
          ch.S = o.S; ch.G = eb.G; ch.Ut = eb.Ut; ch.y = eb.y; ch.flags = flags;
          ch.m = o.m; ch.c = o.c;
          out.push_back(ch);
          group.push_back(++gid);
          hatt::EngineStage tr = ch;
          tr.type = hatt::kStTrsm;
          tr.ntasks = std::max(1, (o.m + hatt::kEngineTrsmRows - 1) / hatt::kEngineTrsmRows);
          out.push_back(tr);
          group.push_back(++gid);
        }
        break;
      }
    }
  }
}

double eng_stage_flops(const hatt::EngineStage &s) {
  switch (s.type) {
    case hatt::kStGemm: return 2.0 * s.M * (double)s.N * s.K * s.batch;
    case hatt::kStChol: return (double)s.c * s.c * s.c / 3.0;
    case hatt::kStTrsm: return (double)s.m * s.c * s.c;
    default: return (double)std::max<long long>(s.count, 1);
  }
}

}  // namespace

// The plan behind tt_batched_* (opaque to callers).
struct tt_batch_plan {
  int count = 0;
  std::vector<EnginePair> pairs;
  size_t ws_bytes = 0;
  size_t tables_off = 0;             // stage and task tables in the workspace
  int max_c = 1;
  std::vector<hatt::EngineStage> stages;
  std::vector<hatt::EngineTask> tasks;
  char *ws = nullptr;                // bound workspace
  int *head = nullptr, *done = nullptr, *status = nullptr, *qflags_all = nullptr;
  long long *prof = nullptr;         // per-CTA profile words (kProfWords each)
  size_t flags_bytes = 0;            // the per-pair QR flags, cleared every run
  int blocks = 0;
  double beta = 0.5;                 // wave shift of the shorter chains (LPT)
};

namespace {

// Interleaves the pairs' stages into one queue: stage j of a pair with S
// stages goes to wave j + beta (S_max - S), so the longest chains start
// first; within a wave the pairs run in decreasing predicted flops (LPT).
void eng_order(tt_batch_plan &P) {
  struct Item { double wave; double cost; int pair; int stage; };
  std::vector<Item> items;
  size_t smax = 0;
  for (const EnginePair &ep : P.pairs) smax = std::max(smax, ep.stages.size());
  std::vector<int> base(P.pairs.size() + 1, 0);
  for (size_t j = 0; j < P.pairs.size(); ++j) base[j + 1] = base[j] + (int)P.pairs[j].stages.size();
  for (size_t j = 0; j < P.pairs.size(); ++j) {
    const EnginePair &ep = P.pairs[j];
    const double shift = P.beta * (double)(smax - ep.stages.size());
    for (size_t i = 0; i < ep.stages.size(); ++i)
      items.push_back({std::floor(i + shift), ep.cost, (int)j, (int)i});
  }
  std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) {
    if (x.wave != y.wave) return x.wave < y.wave;
    if (x.cost != y.cost) return x.cost > y.cost;
    return x.pair < y.pair;
  });
  P.stages.clear();
  P.stages.reserve(items.size());
  for (size_t j = 0; j < P.pairs.size(); ++j)
    for (const hatt::EngineStage &s : P.pairs[j].stages) P.stages.push_back(s);
  // prerequisite counts: all tasks of the pair's earlier groups
  std::vector<std::vector<int>> need(P.pairs.size());
  for (size_t j = 0; j < P.pairs.size(); ++j) {
    const EnginePair &ep = P.pairs[j];
    need[j].assign(ep.stages.size(), 0);
    int done_before = 0, group_start = 0;
    for (size_t i = 0; i < ep.stages.size(); ++i) {
      if (i > 0 && ep.group[i] != ep.group[i - 1]) group_start = done_before;
      need[j][i] = group_start;
      done_before += ep.stages[i].ntasks;
    }
  }
  P.tasks.clear();
  for (const Item &it : items) {
    const hatt::EngineStage &s = P.pairs[it.pair].stages[it.stage];
    for (int t = 0; t < s.ntasks; ++t)
      P.tasks.push_back({base[it.pair] + it.stage, t, it.pair, need[it.pair][it.stage]});
  }
}

// Autotuner: the tile shape of every engine GEMM stage, chosen by timing the
// candidate shapes (engine_gemm_probe: all tiles of the stage as one grid) on
// the first stage of each shape bucket -- M, N, K and the batch rounded up to
// powers of two, and the operand precision -- and cached for the process.
// Only the buckets with the most flops are timed; the others, and GEMMs
// under 2e7 flops, keep the analytic choice. The cache can be saved and
// loaded as text lines (tt_batched_tune_cache).
struct TuneKey {
  int prec, M, N, K, B;
  bool operator<(const TuneKey &o) const {
    return std::tie(prec, M, N, K, B) < std::tie(o.prec, o.M, o.N, o.K, o.B);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;

TuneKey tune_key(const hatt::EngineStage &s) {
  auto p2 = [](int x) { int b = 1; while (b < x) b <<= 1; return b; };
  return {s.prec, p2(s.M), p2(s.N), p2(s.K), p2(s.batch)};
}

// Tunes the kEngineTuneBuckets buckets that carry the most flops in the whole
// batch (each timed once per candidate, on its first stage), then gives every
// GEMM stage its bucket's shape if tuned or cached, else keeps the analytic one.
constexpr int kEngineTuneBuckets = 48;

int eng_autotune(std::vector<EnginePair> &pairs, cudaStream_t st, int *tuned) {
  std::map<TuneKey, std::pair<double, hatt::EngineStage *>> buckets;   // flops, first stage
  for (EnginePair &ep : pairs)
    for (hatt::EngineStage &s : ep.stages) {
      if (s.type != hatt::kStGemm) continue;
      const double f = 2.0 * s.M * (double)s.N * s.K * s.batch;
      if (f < 2e7) continue;                                  // small: analytic tiles
      auto &b = buckets[tune_key(s)];
      if (!b.second) b.second = &s;
      b.first += f;
    }
  std::vector<std::pair<double, TuneKey>> order;
  for (const auto &kv : buckets) order.push_back({kv.second.first, kv.first});
  std::sort(order.begin(), order.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
  for (size_t i = 0; i < order.size() && (int)i < kEngineTuneBuckets; ++i) {
    const TuneKey key = order[i].second;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      if (g_tune.count(key)) continue;
    }
    const hatt::EngineStage &rep = *buckets[key].second;
    float best = 1e30f;
    std::pair<int, int> pick(rep.bm, rep.bn);
    for (const auto &t : eng_tile_candidates(rep)) {
      hatt::EngineStage probe = rep;
      probe.skip_dev = nullptr;
      eng_set_tiles(probe, t.first, t.second);
      float ms = 0.0f;
      const cudaError_t e = hatt::engine_gemm_time(probe, st, &ms);
      if (e != cudaSuccess) return from_cuda(e);
      if (ms < best) { best = ms; pick = t; }
    }
    ++*tuned;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = pick;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (EnginePair &ep : pairs)
    for (hatt::EngineStage &s : ep.stages) {
      if (s.type != hatt::kStGemm) continue;
      auto it = g_tune.find(tune_key(s));
      if (it == g_tune.end()) continue;
      const auto cands = eng_tile_candidates(s);
      if (std::find(cands.begin(), cands.end(), it->second) != cands.end())
        eng_set_tiles(s, it->second.first, it->second.second);
    }
  return TT_OK;
}

// Records one pair's sequence (run_hatt in recording mode) on the given base.
int eng_record_pair(EnginePair &ep, char *base, int *qflags, int pair, std::vector<RecOp> &ops) {
  Ws ws;
  ws.exec = true;
  ws.base = base;
  EngineBufs eb = carve_engine(ws, ep.a);
  eb.qflags = qflags;
  Runner run;
  run.exec = true;
  run.rec = &ops;
  ops.clear();
  run_hatt(run, ep.a, eb.h);
  if (run.err != cudaSuccess) return TT_ERR_ARG;
  ep.stages.clear();
  ep.group.clear();
  eng_expand(ops, eb, pair, ep.stages, ep.group);
  ep.cost = 0.0;
  for (const auto &s : ep.stages) ep.cost += eng_stage_flops(s);
  return TT_OK;
}

size_t eng_pair_bytes(const HattArgs &a) {
  Ws ws;
  carve_engine(ws, a);
  return (ws.off + 255) & ~(size_t)255;
}

}  // namespace

// ------------------------------------------------- allocation-free dot ---
// Scratch of tt_dot_noalloc: one fixed array in the device memory of every GPU
// that loads this library, held until the process exits. In host code the
// symbol is only a handle: its device address comes from cudaGetSymbolAddress,
// looked up once per device (with that device current) and cached.
constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};

cudaError_t noalloc_scratch_address(void **ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

// ===================================================================== ABI ===

extern "C" {

int tt_dot_noalloc(const tt_t *A, const tt_t *B, double *out, void *stream) {
  int st = prepare_dot(A, B, true);
  if (st != TT_OK) return st;
  if (!out) return TT_ERR_ARG;
  const size_t need = measure([&](Ws &ws) { return carve_dot(ws, A, B); },
                              [&](Runner &run, const DotBufs &u) { run_dot(run, A, B, u, nullptr); });
  if (need > kNoAllocScratchBytes) return TT_ERR_WORKSPACE;
  void *scratch = nullptr;
  cudaError_t e = noalloc_scratch_address(&scratch);
  if (e != cudaSuccess) return from_cuda(e);
  // every scratch buffer is written before it is read (the Gram seed G_0 = 1
  // is set by a kernel), so leftovers of an earlier call never matter
  return execute(scratch, kNoAllocScratchBytes, (cudaStream_t)stream,
                 [&](Ws &ws) { return carve_dot(ws, A, B); },
                 [&](Runner &run, const DotBufs &u) { run_dot(run, A, B, u, out); });
}

const char *tt_status_string(int status) {
  switch (status) {
    case TT_OK: return "ok";
    case TT_ERR_SHAPE: return "shape mismatch (orders, mode sizes, boundary ranks or aliasing)";
    case TT_ERR_RANK: return "rank or size above the supported bound";
    case TT_ERR_ARG: return "invalid argument (null pointer or option)";
    case TT_ERR_WORKSPACE: return "workspace too small or misaligned";
    case TT_ERR_CUDA: return "CUDA launch or copy failed";
    case TT_ERR_NONFINITE: return "non-finite value in an input or an intermediate";
    case TT_ERR_BREAKDOWN: return "QR breakdown: a shifted Cholesky pivot was not positive";
    case TT_ERR_TIMEOUT: return "a bounded device wait ran out";
    default: return "unknown status";
  }
}

int tt_hadamard_recompress_plan(const tt_t *Y, const tt_t *Z, const tt_opts *opts,
                                int64_t *out_rank_bound, size_t *workspace_bytes) {
  if (!out_rank_bound || !workspace_bytes) return TT_ERR_ARG;
  HattArgs a;
  int st = prepare_hatt(Y, Z, opts, false, a);
  if (st != TT_OK) return st;
  for (int k = 0; k <= a.d; ++k) out_rank_bound[k] = a.outb[k];
  a.Y = nullptr;
  a.Z = nullptr;
  a.Xout = nullptr;
  Fp64TcScope tc(opts->precision == TT_FP64_TC);
  *workspace_bytes = measure([&](Ws &ws) { return carve_hatt(ws, a); },
                             [&](Runner &run, const HattBufs &b) { run_hatt(run, a, b); });
  return TT_OK;
}

int tt_hadamard_recompress(const tt_t *Y, const tt_t *Z, const tt_opts *opts, tt_t *X,
                           void *workspace, size_t workspace_bytes, void *stream) {
  HattArgs a;
  int st = prepare_hatt(Y, Z, opts, true, a);
  if (st != TT_OK) return st;
  if (!X || !X->cores || !X->r || !X->n) return TT_ERR_ARG;
  if (X->d != Y->d) return TT_ERR_SHAPE;
  for (int k = 0; k < X->d; ++k) {
    if (X->n[k] != Y->n[k]) return TT_ERR_SHAPE;
    if (!X->cores[k]) return TT_ERR_ARG;
  }
  if (!workspace || !aligned(workspace)) return TT_ERR_WORKSPACE;
  // outputs must not overlap inputs
  for (int k = 0; k < a.d; ++k) {
    const size_t xb = (size_t)a.outb[k] * a.n[k] * a.outb[k + 1] * sizeof(double);
    for (int j = 0; j < a.d; ++j) {
      const size_t yb = (size_t)Y->r[j] * Y->n[j] * Y->r[j + 1] * sizeof(double);
      const size_t zb = (size_t)Z->r[j] * Z->n[j] * Z->r[j + 1] * sizeof(double);
      if (overlap(X->cores[k], xb, Y->cores[j], yb) || overlap(X->cores[k], xb, Z->cores[j], zb))
        return TT_ERR_SHAPE;
    }
  }
  a.Y = Y->cores;
  a.Z = Z->cores;
  a.Xout = X->cores;
  cudaStream_t strm = (cudaStream_t)stream;
  Fp64TcScope tc(opts->precision == TT_FP64_TC);
  HattBufs bufs_for_ranks;
  st = execute(workspace, workspace_bytes, strm,
               [&](Ws &ws) {
                 HattBufs b = carve_hatt(ws, a);
                 if (ws.exec) bufs_for_ranks = b;
                 return b;
               },
               [&](Runner &run, const HattBufs &b) { run_hatt(run, a, b); });
  if (st != TT_OK) return st;
  if (a.trunc && !a.fixed) {
    cudaError_t e = cudaMemcpyAsync(X->r, bufs_for_ranks.ranks, (a.d + 1) * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, strm);
    if (e != cudaSuccess) return from_cuda(e);
  } else {
    for (int k = 0; k <= a.d; ++k) X->r[k] = a.outb[k];
  }
  return TT_OK;
}

// ------------------------------------------------------------- batches ---
// Library-owned streams and events of the batched entry point, created once
// per device (cached until the process exits).
namespace {
constexpr int kMaxLanes = 32;
struct LaneSet {
  bool ready = false;
  cudaStream_t s[kMaxLanes] = {};
  cudaEvent_t join[kMaxLanes] = {};
  cudaEvent_t fork = nullptr;
};
std::mutex g_lanes_mu;
LaneSet g_lanes[kNoAllocMaxDevices];

cudaError_t lanes_for_device(LaneSet **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_lanes_mu);
  LaneSet &L = g_lanes[dev];
  if (!L.ready) {
    e = cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming);
    for (int i = 0; i < kMaxLanes && e == cudaSuccess; ++i) {
      e = cudaStreamCreateWithFlags(&L.s[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return e;
    L.ready = true;
  }
  *out = &L;
  return cudaSuccess;
}

// Per-lane workspace sizes (pair j runs on lane j % lanes) and the total.
int batch_layout(int count, const tt_t *Y, const tt_t *Z, const tt_opts *opts, int lanes,
                 std::vector<size_t> &lane_bytes, size_t &total) {
  if (count < 0 || lanes < 1 || lanes > kMaxLanes) return TT_ERR_ARG;
  if (count > 0 && (!Y || !Z || !opts)) return TT_ERR_ARG;
  lane_bytes.assign(lanes, 0);
  for (int j = 0; j < count; ++j) {
    std::vector<int64_t> bound((size_t)std::max(Y[j].d, 0) + 1);
    size_t b = 0;
    const int st = tt_hadamard_recompress_plan(&Y[j], &Z[j], &opts[j], bound.data(), &b);
    if (st != TT_OK) return st;
    size_t &lb = lane_bytes[j % lanes];
    lb = std::max(lb, (b + 255) & ~(size_t)255);
  }
  total = 0;
  for (size_t b : lane_bytes) total += b;
  total += 256;
  return TT_OK;
}
}  // namespace

int tt_hadamard_recompress_batch_plan(int32_t count, const tt_t *Y, const tt_t *Z,
                                      const tt_opts *opts, int32_t lanes,
                                      size_t *workspace_bytes) {
  if (!workspace_bytes) return TT_ERR_ARG;
  std::vector<size_t> lane_bytes;
  size_t total = 0;
  const int st = batch_layout(count, Y, Z, opts, lanes, lane_bytes, total);
  if (st != TT_OK) return st;
  *workspace_bytes = total;
  return TT_OK;
}

int tt_hadamard_recompress_batch(int32_t count, const tt_t *Y, const tt_t *Z,
                                 const tt_opts *opts, tt_t *X, int32_t lanes, void *workspace,
                                 size_t workspace_bytes, void *stream) {
  std::vector<size_t> lane_bytes;
  size_t total = 0;
  int st = batch_layout(count, Y, Z, opts, lanes, lane_bytes, total);
  if (st != TT_OK) return st;
  if (count == 0) return TT_OK;
  if (!X) return TT_ERR_ARG;
  if (!workspace || !aligned(workspace)) return TT_ERR_WORKSPACE;
  if (workspace_bytes < total) return TT_ERR_WORKSPACE;
  // validate every pair before anything is enqueued (shapes, outputs, aliasing)
  for (int j = 0; j < count; ++j) {
    HattArgs a;
    st = prepare_hatt(&Y[j], &Z[j], &opts[j], true, a);
    if (st != TT_OK) return st;
    if (!X[j].cores || !X[j].r || !X[j].n || X[j].d != Y[j].d) return TT_ERR_ARG;
  }
  LaneSet *L = nullptr;
  cudaError_t e = lanes_for_device(&L);
  if (e != cudaSuccess) return from_cuda(e);
  const cudaStream_t caller = (cudaStream_t)stream;
  const int used = std::min<int>(lanes, count);
  e = cudaEventRecord(L->fork, caller);
  for (int l = 0; l < used && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(L->s[l], L->fork, 0);
  if (e != cudaSuccess) return from_cuda(e);
  std::vector<char *> base(lanes);
  char *p = (char *)workspace;
  for (int l = 0; l < lanes; ++l) {
    base[l] = p;
    p += lane_bytes[l];
  }
  int first_error = TT_OK;
  BatchScope batch_scope;
  for (int j = 0; j < count && first_error == TT_OK; ++j) {
    const int l = j % lanes;
    first_error = tt_hadamard_recompress(&Y[j], &Z[j], &opts[j], &X[j], base[l], lane_bytes[l],
                                         L->s[l]);
  }
  // join every lane that was forked, also after an error, so the caller's
  // stream never runs ahead of work already enqueued on a lane
  for (int l = 0; l < used; ++l) {
    cudaError_t e2 = cudaEventRecord(L->join[l], L->s[l]);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(caller, L->join[l], 0);
    if (e2 != cudaSuccess && first_error == TT_OK) first_error = from_cuda(e2);
  }
  return first_error;
}

int tt_round_ex_plan(const tt_t *A, int64_t max_rank, double tol, int32_t fixed_ranks,
                     int64_t *out_rank_bound, size_t *workspace_bytes) {
  if (!out_rank_bound || !workspace_bytes) return TT_ERR_ARG;
  RoundArgs a;
  int st = prepare_round(A, max_rank, tol, fixed_ranks, false, a);
  if (st != TT_OK) return st;
  for (int k = 0; k <= a.d; ++k) out_rank_bound[k] = a.outb[k];
  a.A = nullptr;
  a.Bout = nullptr;
  *workspace_bytes = measure([&](Ws &ws) { return carve_round(ws, a); },
                             [&](Runner &run, const RoundBufs &u) { run_round(run, a, u); });
  return TT_OK;
}

int tt_round_plan(const tt_t *A, int64_t max_rank, double tol, int64_t *out_rank_bound,
                  size_t *workspace_bytes) {
  return tt_round_ex_plan(A, max_rank, tol, 0, out_rank_bound, workspace_bytes);
}

int tt_round_ex(const tt_t *A, int64_t max_rank, double tol, int32_t fixed_ranks, tt_t *B,
                void *workspace, size_t workspace_bytes, void *stream) {
  RoundArgs a;
  int st = prepare_round(A, max_rank, tol, fixed_ranks, true, a);
  if (st != TT_OK) return st;
  if (!B || !B->cores || !B->r || !B->n) return TT_ERR_ARG;
  if (B->d != A->d) return TT_ERR_SHAPE;
  for (int k = 0; k < A->d; ++k) {
    if (B->n[k] != A->n[k]) return TT_ERR_SHAPE;
    if (!B->cores[k]) return TT_ERR_ARG;
  }
  if (!workspace || !aligned(workspace)) return TT_ERR_WORKSPACE;
  for (int k = 0; k < a.d; ++k) {
    const size_t bb = (size_t)a.outb[k] * a.n[k] * a.outb[k + 1] * sizeof(double);
    for (int j = 0; j < a.d; ++j) {
      const size_t ab = (size_t)A->r[j] * A->n[j] * A->r[j + 1] * sizeof(double);
      if (overlap(B->cores[k], bb, A->cores[j], ab)) return TT_ERR_SHAPE;
    }
  }
  a.A = A->cores;
  a.Bout = B->cores;
  cudaStream_t strm = (cudaStream_t)stream;
  RoundBufs keep;
  st = execute(workspace, workspace_bytes, strm,
               [&](Ws &ws) {
                 RoundBufs u = carve_round(ws, a);
                 if (ws.exec) keep = u;
                 return u;
               },
               [&](Runner &run, const RoundBufs &u) { run_round(run, a, u); });
  if (st != TT_OK) return st;
  if (a.fixed) {
    for (int k = 0; k <= a.d; ++k) B->r[k] = a.outb[k];
    return TT_OK;
  }
  cudaError_t e = cudaMemcpyAsync(B->r, keep.ranks, (a.d + 1) * sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, strm);
  return from_cuda(e);
}

int tt_round(const tt_t *A, int64_t max_rank, double tol, tt_t *B, void *workspace,
             size_t workspace_bytes, void *stream) {
  return tt_round_ex(A, max_rank, tol, 0, B, workspace, workspace_bytes, stream);
}

int tt_dot_plan(const tt_t *A, const tt_t *B, size_t *workspace_bytes) {
  if (!workspace_bytes) return TT_ERR_ARG;
  int st = prepare_dot(A, B, false);
  if (st != TT_OK) return st;
  tt_t a0 = *A, b0 = *B;
  a0.cores = nullptr;
  b0.cores = nullptr;
  *workspace_bytes = measure([&](Ws &ws) { return carve_dot(ws, &a0, &b0); },
                             [&](Runner &run, const DotBufs &u) { run_dot(run, &a0, &b0, u, nullptr); });
  return TT_OK;
}

int tt_dot(const tt_t *A, const tt_t *B, double *out, void *workspace, size_t workspace_bytes,
           void *stream) {
  int st = prepare_dot(A, B, true);
  if (st != TT_OK) return st;
  if (!out) return TT_ERR_ARG;
  if (!workspace || !aligned(workspace)) return TT_ERR_WORKSPACE;
  return execute(workspace, workspace_bytes, (cudaStream_t)stream,
                 [&](Ws &ws) { return carve_dot(ws, A, B); },
                 [&](Runner &run, const DotBufs &u) { run_dot(run, A, B, u, out); });
}

int tt_norm(const tt_t *A, double *out, void *workspace, size_t workspace_bytes, void *stream) {
  int st = tt_dot(A, A, out, workspace, workspace_bytes, stream);
  if (st != TT_OK) return st;
  return from_cuda(hatt::sqrt_scalar(out, out, (cudaStream_t)stream));
}

int tt_sketch_tt(int32_t d, const int64_t *n, const int64_t *ell, uint64_t seed, uint32_t pair,
                 double **cores, void *stream) {
  if (!n || !ell || !cores) return TT_ERR_ARG;
  if (d < 1) return TT_ERR_SHAPE;
  if (d > hatt::kMaxOrder) return TT_ERR_RANK;
  if (ell[0] != 1 || ell[d] != 1) return TT_ERR_SHAPE;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1 || ell[k + 1] < 1) return TT_ERR_SHAPE;
    if ((double)ell[k] * n[k] * ell[k + 1] >= 4294967296.0) return TT_ERR_RANK;
    if (!cores[k]) return TT_ERR_ARG;
  }
  return from_cuda(hatt::sketch_fill_ptrs(d, n, ell, seed, pair, cores, (cudaStream_t)stream));
}

int64_t tt_launch_count(void) { return (int64_t)hatt::launch_count(); }

int tt_laplacian(const tt_t *A, double inv_h2, tt_t *L, void *stream) {
  int st = check_tt(A, true);
  if (st != TT_OK) return st;
  if (!L || !L->n || !L->r || !L->cores || !std::isfinite(inv_h2)) return TT_ERR_ARG;
  const int d = A->d;
  if (L->d != d) return TT_ERR_SHAPE;
  for (int k = 0; k < d; ++k) {
    if (L->n[k] != A->n[k] || !L->cores[k]) return TT_ERR_SHAPE;
    if (A->n[k] > kIntMax / 2 || 2 * A->r[k] > kIntMax) return TT_ERR_RANK;
  }
  for (int k = 0; k <= d; ++k) {
    const int64_t want = (k == 0 || k == d) ? 1 : 2 * A->r[k];
    if (L->r[k] != want) return TT_ERR_SHAPE;
  }
  cudaStream_t strm = (cudaStream_t)stream;
  for (int k = 0; k < d; ++k) {
    const int pos = d == 1 ? 0 : (k == 0 ? 1 : (k == d - 1 ? 3 : 2));
    cudaError_t e = hatt::laplacian_core(A->cores[k], (int)A->r[k], (int)A->n[k], (int)A->r[k + 1],
                                         pos, inv_h2, L->cores[k], strm);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return TT_OK;
}

int tt_lincomb(int32_t count, const tt_t *T, const double *coef, tt_t *S, void *stream) {
  if (count < 1 || !T || !coef || !S || !S->n || !S->r || !S->cores) return TT_ERR_ARG;
  for (int j = 0; j < count; ++j) {
    const int st = check_tt(&T[j], true);
    if (st != TT_OK) return st;
    if (!std::isfinite(coef[j])) return TT_ERR_ARG;
  }
  const int d = T[0].d;
  if (S->d != d) return TT_ERR_SHAPE;
  for (int j = 0; j < count; ++j) {
    if (T[j].d != d) return TT_ERR_SHAPE;
    for (int k = 0; k < d; ++k)
      if (T[j].n[k] != T[0].n[k]) return TT_ERR_SHAPE;
  }
  for (int k = 0; k < d; ++k)
    if (S->n[k] != T[0].n[k] || !S->cores[k]) return TT_ERR_SHAPE;
  for (int k = 0; k <= d; ++k) {
    ll want = 0;
    for (int j = 0; j < count; ++j) want += T[j].r[k];
    if (k == 0 || k == d) want = 1;
    if (S->r[k] != want) return TT_ERR_SHAPE;
    if (want > kIntMax) return TT_ERR_RANK;
  }
  cudaStream_t strm = (cudaStream_t)stream;
  for (int k = 0; k < d; ++k) {
    const int n = (int)T[0].n[k];
    const int A = (int)S->r[k], Bw = (int)S->r[k + 1];
    cudaError_t e = cudaSuccess;
    if (d > 1 && k > 0 && k < d - 1)
      e = cudaMemsetAsync(S->cores[k], 0, (size_t)A * n * Bw * sizeof(double), strm);
    int ra = 0, rb = 0;
    for (int j = 0; j < count && e == cudaSuccess; ++j) {
      const int a = (int)T[j].r[k], b = (int)T[j].r[k + 1];
      const double c = (k == 0) ? coef[j] : 1.0;          // coefficients on the first cores
      if (d == 1) {
        e = hatt::put_block(T[j].cores[0], 1, n, 1, coef[j], S->cores[0], 1, 1, 0, 0, j > 0, strm);
        continue;
      }
      e = hatt::put_block(T[j].cores[k], a, n, b, c, S->cores[k], A, Bw, ra, rb, false, strm);
      if (k > 0) ra += a;
      if (k < d - 1) rb += b;
    }
    if (e != cudaSuccess) return from_cuda(e);
  }
  return TT_OK;
}

int tt_scale(double *x, int64_t count, const double *divisor, void *stream) {
  if (count < 0) return TT_ERR_ARG;
  if (count == 0) return TT_OK;
  if (!x || !divisor) return TT_ERR_ARG;
  return from_cuda(hatt::div_by_scalar(x, count, divisor, (cudaStream_t)stream));
}

int tt_device_error(int32_t *value) {
  if (!value) return TT_ERR_ARG;
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = hatt::read_device_error(&v);
  if (e == cudaSuccess && v != 0) e = hatt::clear_device_error();
  if (e != cudaSuccess) return from_cuda(e);
  *value = v;
  return TT_OK;
}

int tt_device_status(int32_t *status) {
  if (!status) return TT_ERR_ARG;
  int32_t v = 0;
  const int st = tt_device_error(&v);
  if (st != TT_OK) return st;
  *status = (v & hatt::kHealthTimeout)     ? TT_ERR_TIMEOUT
            : (v & hatt::kHealthNonfinite) ? TT_ERR_NONFINITE
            : (v & hatt::kHealthBreakdown) ? TT_ERR_BREAKDOWN
                                           : TT_OK;
  return TT_OK;
}

// ------------------------------------------------------ one product ---
namespace {
struct NoBufs {};

int gemm_args(int32_t precision, int64_t M, int64_t N, int64_t K, int64_t batch, hatt::Gemm &g) {
  if (precision < TT_FP64 || precision > TT_FP64_TC) return TT_ERR_ARG;
  if (M < 0 || N < 0 || K < 1 || batch < 0) return TT_ERR_ARG;
  if (M > kIntMax || N > kIntMax || K > kIntMax || batch > kIntMax) return TT_ERR_SHAPE;
  if (M * K > kIntMax || K * N > kIntMax || M * N > kIntMax) return TT_ERR_SHAPE;
  g.M = (int)M;
  g.N = (int)N;
  g.K = (int)K;
  g.batch = (int)batch;
  g.bdiv = 1;
  g.sA1 = M * K; g.sAm = K; g.sAk = 1;
  g.sB1 = K * N; g.sBk = N; g.sBn = 1;
  g.sC1 = M * N; g.sCm = N; g.sCn = 1;
  g.prec = precision == TT_FP64_TC ? hatt::kPrecFP64 : precision;
  return TT_OK;
}
}  // namespace

int tt_gemm_plan(int32_t precision, int64_t M, int64_t N, int64_t K, int64_t batch,
                 size_t *workspace_bytes) {
  if (!workspace_bytes) return TT_ERR_ARG;
  hatt::Gemm g;
  const int st = gemm_args(precision, M, N, K, batch, g);
  if (st != TT_OK) return st;
  Fp64TcScope tc(precision == TT_FP64_TC);
  *workspace_bytes = measure([&](Ws &) { return NoBufs{}; },
                             [&](Runner &run, const NoBufs &) { run.gemm(g); });
  return TT_OK;
}

int tt_gemm(int32_t precision, int64_t M, int64_t N, int64_t K, int64_t batch, const double *A,
            const double *B, double *C, double alpha, void *workspace, size_t workspace_bytes,
            void *stream) {
  hatt::Gemm g;
  const int st = gemm_args(precision, M, N, K, batch, g);
  if (st != TT_OK) return st;
  if (M == 0 || N == 0 || batch == 0) return TT_OK;
  if (!A || !B || !C) return TT_ERR_ARG;
  if (!workspace || !aligned(workspace)) return TT_ERR_WORKSPACE;
  g.A = A;
  g.B = B;
  g.C = C;
  g.alpha = alpha;
  Fp64TcScope tc(precision == TT_FP64_TC);
  return execute(workspace, workspace_bytes, (cudaStream_t)stream, [&](Ws &) { return NoBufs{}; },
                 [&](Runner &run, const NoBufs &) { run.gemm(g); });
}

int tt_gemm_autotune(int32_t enable) {
  hatt::set_gemm_autotune(enable != 0);
  return TT_OK;
}

int tt_kernel_timer_start(int32_t capacity) {
  if (capacity < 1 || capacity > (1 << 20)) return TT_ERR_ARG;
  std::lock_guard<std::mutex> lk(hatt::g_timer.mu);
  hatt::timer_release();
  hatt::g_timer.ev.assign(2 * (size_t)capacity, nullptr);
  for (auto &e : hatt::g_timer.ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      e = nullptr;
      hatt::g_timer.ev.erase(std::remove(hatt::g_timer.ev.begin(), hatt::g_timer.ev.end(),
                                         (cudaEvent_t) nullptr),
                             hatt::g_timer.ev.end());
      hatt::timer_release();
      return TT_ERR_CUDA;
    }
  }
  hatt::g_timer.flops.assign((size_t)capacity, 0.0);
  hatt::g_timer.role.assign((size_t)capacity, hatt::kRoleAux);
  hatt::g_timer.used = 0;
  hatt::g_timer.active.store(true);
  return TT_OK;
}

int tt_kernel_timer_stop(double *ms, double *flops, int32_t capacity, int64_t *count) {
  return tt_kernel_timer_stop_ex(ms, flops, nullptr, capacity, count);
}

int tt_kernel_timer_stop_ex(double *ms, double *flops, int32_t *role, int32_t capacity,
                            int64_t *count) {
  if (capacity < 0 || (capacity > 0 && (ms == nullptr || flops == nullptr))) return TT_ERR_ARG;
  std::lock_guard<std::mutex> lk(hatt::g_timer.mu);
  if (!hatt::g_timer.active.load()) return TT_ERR_ARG;
  hatt::g_timer.active.store(false);
  const int used = hatt::g_timer.used;
  int status = TT_OK;
  for (int i = 0; i < used && i < capacity; ++i) {
    float t = 0.0f;
    const double f = hatt::g_timer.flops[i];
    if (f < 0.0) {
      ms[i] = -1.0;
      flops[i] = 0.0;
      if (role) role[i] = hatt::g_timer.role[i];
      continue;
    }
    if (cudaEventSynchronize(hatt::g_timer.ev[2 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, hatt::g_timer.ev[2 * i], hatt::g_timer.ev[2 * i + 1]) != cudaSuccess) {
      cudaGetLastError();
      status = TT_ERR_CUDA;
      t = -1.0f;
    }
    ms[i] = (double)t;
    flops[i] = f;
    if (role) role[i] = hatt::g_timer.role[i];
  }
  if (count) *count = used;
  hatt::timer_release();
  return status;
}

// ------------------------------------------------------------- batched ---

int tt_batched_plan_create(int32_t count, const tt_t *Y, const tt_t *Z, const tt_opts *opts,
                           tt_t *X, tt_batch_plan **plan, size_t *workspace_bytes) {
  if (!plan || !workspace_bytes || count < 1 || !Y || !Z || !opts || !X) return TT_ERR_ARG;
  *plan = nullptr;
  std::unique_ptr<tt_batch_plan> P(new tt_batch_plan());
  P->count = count;
  P->pairs.resize(count);
  size_t off = 0;
  long long flag_ints = 0;
  for (int j = 0; j < count; ++j) {
    EnginePair &ep = P->pairs[j];
    int st = prepare_hatt(&Y[j], &Z[j], &opts[j], true, ep.a);
    if (st != TT_OK) return st;
    // the engine runs HaTT-1 in FP64 or with FP32 sketch products, and
    // without the truncation sweep (sketch rank = output rank)
    if (ep.a.variant != 1 || ep.a.trunc || ep.a.seed_offset) return TT_ERR_ARG;
    if (opts[j].precision != TT_FP64 && opts[j].precision != TT_MIXED_FP32) return TT_ERR_ARG;
    if (!X[j].cores || !X[j].r || !X[j].n || X[j].d != Y[j].d) return TT_ERR_ARG;
    for (int k = 0; k < ep.a.d; ++k)
      if (X[j].n[k] != Y[j].n[k] || !X[j].cores[k]) return TT_ERR_SHAPE;
    ep.a.Y = Y[j].cores;
    ep.a.Z = Z[j].cores;
    ep.a.Xout = X[j].cores;
    for (int k = 0; k <= ep.a.d; ++k) X[j].r[k] = ep.a.outb[k];
    ep.ws_off = off;
    ep.ws_bytes = eng_pair_bytes(ep.a);
    off += ep.ws_bytes;
    flag_ints += 4LL * ep.a.d;
    for (int k = 0; k <= ep.a.d; ++k) P->max_c = std::max<int>(P->max_c, (int)ep.a.ell[k]);
  }
  // control words: head, status, per-pair completion counters, QR flags, then
  // the per-CTA profile words (all cleared every run)
  P->flags_bytes = ((2 + (size_t)count + (size_t)flag_ints) * sizeof(int) + 255) & ~(size_t)255;
  P->flags_bytes += (size_t)hatt::kMaxProfBlocks * hatt::kProfWords * sizeof(long long);
  const size_t ctl_off = off;
  off += P->flags_bytes;
  // count stages and the largest task count over the tile candidates with a
  // stand-in base address (pointers are formed, never dereferenced)
  std::vector<RecOp> ops;
  size_t nstages = 0, ntasks_max = 0;
  char *fake = reinterpret_cast<char *>((uintptr_t)1 << 40);
  int *fq = reinterpret_cast<int *>(fake + ctl_off) + 2 + count;
  for (int j = 0; j < count; ++j) {
    EnginePair &ep = P->pairs[j];
    int st = eng_record_pair(ep, fake + ep.ws_off, fq, j, ops);
    if (st != TT_OK) return st;
    fq += 4 * ep.a.d;
    nstages += ep.stages.size();
    for (const auto &s : ep.stages) {
      size_t most = (size_t)s.ntasks;
      if (s.type == hatt::kStGemm)
        for (const auto &t : eng_tile_candidates(s)) {
          hatt::EngineStage c = s;
          eng_set_tiles(c, t.first, t.second);
          most = std::max(most, (size_t)c.ntasks);
        }
      ntasks_max += most;
    }
    ep.stages.clear();
    ep.group.clear();
  }
  if (ntasks_max >= (size_t)INT32_MAX) return TT_ERR_RANK;
  P->tables_off = (off + 255) & ~(size_t)255;
  P->ws_bytes = P->tables_off + nstages * sizeof(hatt::EngineStage) +
                ntasks_max * sizeof(hatt::EngineTask) + 256;
  *workspace_bytes = P->ws_bytes;
  *plan = P.release();
  return TT_OK;
}

int tt_batched_plan_bind(tt_batch_plan *P, void *workspace, size_t workspace_bytes,
                         int32_t autotune, void *stream) {
  if (!P || (autotune != 0 && autotune != 1)) return TT_ERR_ARG;
  if (!workspace || !aligned(workspace) || workspace_bytes < P->ws_bytes) return TT_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return from_cuda(cudaGetLastError());
  if (cs != cudaStreamCaptureStatusNone) return TT_ERR_ARG;        // synchronizes: not capturable
  char *ws = (char *)workspace;
  const size_t ctl_off = P->pairs.back().ws_off + P->pairs.back().ws_bytes;
  int *ctl = reinterpret_cast<int *>(ws + ctl_off);
  P->ws = ws;
  P->head = ctl;
  P->status = ctl + 1;
  P->done = ctl + 2;
  P->qflags_all = ctl + 2 + P->count;
  P->prof = reinterpret_cast<long long *>(
      ws + ctl_off + P->flags_bytes - (size_t)hatt::kMaxProfBlocks * hatt::kProfWords * sizeof(long long));
  std::vector<RecOp> ops;
  int *fq = P->qflags_all;
  for (int j = 0; j < P->count; ++j) {
    EnginePair &ep = P->pairs[j];
    int s = eng_record_pair(ep, ws + ep.ws_off, fq, j, ops);
    if (s != TT_OK) return s;
    fq += 4 * ep.a.d;
  }
  cudaError_t e = cudaMemsetAsync(ctl, 0, P->flags_bytes, st);
  if (e != cudaSuccess) return from_cuda(e);
  if (autotune) {
    int tuned = 0;
    const int s = eng_autotune(P->pairs, st, &tuned);
    if (s != TT_OK) return s;
  }
  eng_order(*P);
  const size_t sb = P->stages.size() * sizeof(hatt::EngineStage);
  const size_t tb = P->tasks.size() * sizeof(hatt::EngineTask);
  if (P->tables_off + sb + tb > P->ws_bytes) return TT_ERR_WORKSPACE;
  e = cudaMemcpyAsync(ws + P->tables_off, P->stages.data(), sb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + P->tables_off + sb, P->tasks.data(), tb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = hatt::engine_blocks(P->max_c, &P->blocks);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);             // host tables may change later
  return from_cuda(e);
}

int tt_batched_run(tt_batch_plan *P, int64_t spin_cap, void *stream) {
  if (!P || !P->ws || spin_cap < 1) return TT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(P->head, 0, P->flags_bytes, st);
  if (e != cudaSuccess) return from_cuda(e);
  const auto *stages = reinterpret_cast<const hatt::EngineStage *>(P->ws + P->tables_off);
  const auto *tasks = reinterpret_cast<const hatt::EngineTask *>(
      P->ws + P->tables_off + P->stages.size() * sizeof(hatt::EngineStage));
  e = hatt::engine_launch(stages, tasks, (int)P->tasks.size(), P->head, P->done, P->status,
                          (long long)spin_cap, P->max_c, P->blocks, P->prof, st);
  return from_cuda(e);
}

int tt_batched_status(tt_batch_plan *P, void *stream, int32_t *status) {
  if (!P || !P->ws || !status) return TT_ERR_ARG;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, P->status, sizeof(int), cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return from_cuda(e);
  *status = (v & hatt::kEngineTimeout)     ? TT_ERR_TIMEOUT
            : (v & hatt::kEngineNonfinite) ? TT_ERR_NONFINITE
            : (v & hatt::kEngineBreakdown) ? TT_ERR_BREAKDOWN
                                           : TT_OK;
  return TT_OK;
}

int tt_batched_plan_info(const tt_batch_plan *P, int64_t *stages, int64_t *tasks, int32_t *blocks) {
  if (!P) return TT_ERR_ARG;
  if (stages) *stages = (int64_t)P->stages.size();
  if (tasks) *tasks = (int64_t)P->tasks.size();
  if (blocks) *blocks = P->blocks;
  return TT_OK;
}

int tt_batched_profile(tt_batch_plan *P, void *stream, int64_t *out) {
  if (!P || !P->ws || !out) return TT_ERR_ARG;
  const int n = std::min(P->blocks, hatt::kMaxProfBlocks);
  std::vector<long long> h((size_t)n * hatt::kProfWords);
  cudaError_t e = cudaMemcpyAsync(h.data(), P->prof, h.size() * sizeof(long long),
                                  cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return from_cuda(e);
  for (int i = 0; i < hatt::kProfWords; ++i) {
    long long sum = 0;
    for (int b = 0; b < n; ++b) sum += h[(size_t)b * hatt::kProfWords + i];
    out[i] = sum;
  }
  return TT_OK;
}

int tt_batched_plan_destroy(tt_batch_plan *P) {
  delete P;
  return TT_OK;
}

int tt_batched_tune_cache(const char *path, int32_t save) {
  if (!path || (save != 0 && save != 1)) return TT_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (save) {
    FILE *f = std::fopen(path, "w");
    if (!f) return TT_ERR_ARG;
    for (const auto &kv : g_tune)
      std::fprintf(f, "%d %d %d %d %d %d %d\n", kv.first.prec, kv.first.M, kv.first.N, kv.first.K,
                   kv.first.B, kv.second.first, kv.second.second);
    std::fclose(f);
    return TT_OK;
  }
  FILE *f = std::fopen(path, "r");
  if (!f) return TT_ERR_ARG;
  TuneKey k;
  int bm = 0, bn = 0;
  while (std::fscanf(f, "%d %d %d %d %d %d %d", &k.prec, &k.M, &k.N, &k.K, &k.B, &bm, &bn) == 7)
    if (bm > 0 && bn > 0 && bm <= 128 && bn <= 128 && bm * bn <= 4096) g_tune[k] = {bm, bn};
  std::fclose(f);
  return TT_OK;
}

int tt_philox4x32_10(const uint32_t *ctr, uint32_t key0, uint32_t key1, uint32_t *out,
                     int64_t count, void *stream) {
  if (count < 0) return TT_ERR_ARG;
  if (count == 0) return TT_OK;
  if (!ctr || !out) return TT_ERR_ARG;
  return from_cuda(hatt::philox_raw(ctr, key0, key1, out, count, (cudaStream_t)stream));
}

}  // extern "C"
