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
#include <mutex>
#include <vector>

#include "hatt.h"
#include "hatt_internal.cuh"

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

// Runs a launch sequence in planning or execution mode.
struct Runner {
  bool exec = false;
  cudaStream_t st = nullptr;
  size_t scratch_need = 0;       // doubles
  double *scratch = nullptr;
  cudaError_t err = cudaSuccess;

  bool live() const { return exec && err == cudaSuccess; }
  void check(cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
  }
  void gemm(const Gemm &g) {
    if (!exec) {
      scratch_need = std::max(scratch_need, hatt::gemm_scratch_doubles(g));
      return;
    }
    if (err == cudaSuccess) check(hatt::gemm_f64(g, scratch, st));
  }
  void qr(double *S, int m, int c, ll ld, int *flags) {
    if (!exec) {
      scratch_need = std::max(scratch_need, hatt::qr_scratch_doubles(m, c));
      return;
    }
    if (err == cudaSuccess) check(hatt::qr_inplace(S, m, c, ld, scratch, flags, st));
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
//   Rv[l][i][g]       = sum_c R_k[l][i][c] V_R[c][g]
//   P2[i][a'][b][g]   = sum_b' Z_k[b][i][b'] (U S)_R[a' s1 + b'][g]
//   P3[a][b][i][g]    = sum_a' Y_k[a][i][a'] P2[i][a'][b][g]
//   W^{(k)}[a s0 + b][l] = sum_{i,g} P3[a][b][i][g] Rv[l][i][g]
// (the W_L W_R^T form: W_L = P3, W_R = Rv). R is read on the host, so this
// variant synchronizes the stream once per core.
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
  auto contract = [&](int R) {
    {   // Rv = R_k V_R
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = l0 * nk; g.N = R; g.K = c;
      g.A = Rk; g.sAm = c; g.sAk = 1;
      g.B = b.VR; g.sBk = R; g.sBn = 1;
      g.C = b.Rv; g.sCm = R; g.sCn = 1;
      g.prec = a.prec;
      run.gemm(g);
    }
    {   // P2, batched over (i, a')
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = s0; g.N = R; g.K = s1;
      g.batch = nk * r1; g.bdiv = r1;
      g.A = a.Z ? a.Z[k] : nullptr; g.sA1 = s1; g.sA2 = 0; g.sAm = (ll)nk * s1; g.sAk = 1;
      g.B = b.UR; g.sB1 = 0; g.sB2 = (ll)s1 * R; g.sBk = R; g.sBn = 1;
      g.C = b.P2; g.sC1 = (ll)r1 * s0 * R; g.sC2 = (ll)s0 * R; g.sCm = R; g.sCn = 1;
      g.prec = a.prec;
      run.gemm(g);
    }
    {   // P3, batched over (i, b)
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = r0; g.N = R; g.K = r1;
      g.batch = nk * s0; g.bdiv = s0;
      g.A = a.Y ? a.Y[k] : nullptr; g.sA1 = r1; g.sA2 = 0; g.sAm = (ll)nk * r1; g.sAk = 1;
      g.B = b.P2; g.sB1 = (ll)r1 * s0 * R; g.sB2 = R; g.sBk = (ll)s0 * R; g.sBn = 1;
      g.C = b.P3; g.sC1 = R; g.sC2 = (ll)nk * R; g.sCm = (ll)s0 * nk * R; g.sCn = 1;
      g.prec = a.prec;
      run.gemm(g);
    }
    {   // W^{(k)} = W_L W_R^T
      Gemm g;
      g.role = hatt::kRoleMethod;
      g.M = r0 * s0; g.N = l0; g.K = nk * R;
      g.A = b.P3; g.sAm = (ll)nk * R; g.sAk = 1;
      g.B = b.Rv; g.sBk = 1; g.sBn = (ll)nk * R;
      g.C = Wout; g.sCm = l0; g.sCn = 1;
      g.prec = a.prec;
      run.gemm(g);
    }
  };
  if (!run.exec) {   // planning: every R the selection can return
    for (int R = 1; R <= c; ++R) contract(R);
    return;
  }
  if (!run.live()) return;
  run.check(hatt::select_directions(b.Uf, b.V2, x, c, a.ep, b.UR, b.VR, b.Rdev, run.st));
  int R = 0;
  run.check(cudaMemcpyAsync(&R, b.Rdev, sizeof(int), cudaMemcpyDeviceToHost, run.st));
  run.check(cudaStreamSynchronize(run.st));
  if (!run.live()) return;
  if (R < 1 || R > c) {
    run.check(cudaErrorUnknown);
    return;
  }
  contract(R);
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
    if (run.live()) run.check(hatt::pkp_first(a.Y[0], a.Z[0], (int)n[0], 1, 1, a.Xout[0], run.st));
    return;
  }

  // A1: sketch cores R_k (Definition 2.1)
  if (run.live()) {
    hatt::SketchTable t;
    t.d = d;
    t.seed = a.seed;
    t.pair = 0;
    for (int k = 0; k <= d; ++k) t.offset[k] = b.Roff[k];
    for (int k = 0; k < d; ++k) {
      t.a[k] = (int)l[k];
      t.n[k] = (int)n[k];
      t.b[k] = (int)l[k + 1];
    }
    run.check(hatt::sketch_fill(t, b.R, run.st));
    run.check(hatt::set_value(Wk(d), 1, 1.0, run.st));          // W^{(d)} = [1]
    run.check(hatt::set_value(b.winv + d, 1, 1.0, run.st));
    run.check(cudaMemsetAsync(b.ticket, 0, sizeof(unsigned int), run.st));
  }

  // A2/A3: HPCRL-1, W^{(k)} from W^{(k+1)} and cores k of Y, Z, R (Eq. (3.6))
  for (int k = d - 1; k >= 1; --k) {
    const int r0 = (int)r[k], r1 = (int)r[k + 1], s0 = (int)s[k], s1 = (int)s[k + 1];
    const int l0 = (int)l[k], l1 = (int)l[k + 1], nk = (int)n[k];
    const double *Rk = b.R + b.Roff[k];
    if (a.variant == 2) {
      hpcrl2_step(run, a, b, k, Wk(k + 1), Wk(k));
      if (run.live())
        run.check(hatt::inv_norm(Wk(k), (ll)r0 * s0 * l0, b.winv + k, b.partials, b.ticket, run.st));
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
    if (run.live())
      run.check(hatt::inv_norm(Wk(k), (ll)r0 * s0 * l0, b.winv + k, b.partials, b.ticket, run.st));
  }

  // A4-A8: left-to-right pass (Algorithm 4)
  double *C = b.Ca, *Cn = b.Cb;
  if (run.live())
    run.check(hatt::pkp_first(a.Y[0], a.Z[0], (int)n[0], (int)r[1], (int)s[1], C, run.st));
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
    case TT_ERR_NONFINITE: return "non-finite value";
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
  if (a.variant == 2) {   // the kept ranks are read on the host: no stream capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(strm, &cs) != cudaSuccess) return from_cuda(cudaGetLastError());
    if (cs != cudaStreamCaptureStatusNone) return TT_ERR_ARG;
  }
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
    if (opts[j].variant == 2) return TT_ERR_ARG;   // reads ranks on the host: one pair per call
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

int tt_philox4x32_10(const uint32_t *ctr, uint32_t key0, uint32_t key1, uint32_t *out,
                     int64_t count, void *stream) {
  if (count < 0) return TT_ERR_ARG;
  if (count == 0) return TT_OK;
  if (!ctr || !out) return TT_ERR_ARG;
  return from_cuda(hatt::philox_raw(ctr, key0, key1, out, count, (cudaStream_t)stream));
}

}  // extern "C"
