// C ABI of the approximate-deconvolution library: plans, workspaces, the
// solver drivers for Algorithms 1-4 and their capture into CUDA graphs.
//
// One application of G (Section 4, Eq. df / Eq. df2) is a chain of pass
// kernels (2D: 3 passes, 3D: 5 passes). A solve is
//   reset -> [reference pass if u0 given] -> initial residual r0 = u_bar - G u0
//   -> while (any field active) { one iteration of the chosen algorithm }
//   -> [CG: deferred u += alpha p] -> [true residual]
// The iteration body is captured once per (plan, method, tolerance, maxit,
// buffers) into the body graph of a conditional while node; the scalar
// recurrences and the loop condition are computed on the device by the last
// block of each dot-producing pass, so the host waits once per solve.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/gad.h"
#include "args.h"
#include "cnn.h"
#include "launch.h"
#include "plan.h"
#include "state.h"

using namespace gad;

namespace {

struct PassCfg {
  int E = 0, W = 0, T = 0, ld = 0;
  int chunk = 0;                     // stencil pass: march positions per block
  size_t smem = 0;
  FftPlan fft{};
  FftPlan fft_inv{};
  float rcp_a = 0.f, rcp_b = 0.f;
  dim3 grid;
};

struct Plan {
  int ndim = 2, nx = 0, ny = 0, nz = 1, kxn = 0, batch = 0;
  bool f64 = false;
  double gamma = 0.0;
  long long P = 0, SP = 0;
  PassCfg xf, xi, fl, yf, yi;
  PassCfg sn;                        // preconditioner stencil pass (W rows per block)
  const void* twx = nullptr;
  void *S1 = nullptr, *S2 = nullptr;
  void *R = nullptr, *Pv = nullptr, *Q = nullptr, *Sv = nullptr, *F0 = nullptr;
  void *Bh = nullptr, *Uh = nullptr, *Rh = nullptr, *Ph = nullptr, *F0h = nullptr;  // spectral-space vectors
  PassCfg sp;                        // spectral-space pass launch shape
  void* Uscratch = nullptr;          // stands in for u when a single pass is timed
  void *Bin = nullptr, *Bout = nullptr;   // batched solves: the group's fields gathered contiguously
  FieldState* st = nullptr;
  double* part = nullptr;
  unsigned* ticket = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  unsigned maxblk = 0;               // capacity of part (blocks per field)
  bool tuned = false;                // tile widths of the FFT passes tuned
  bool sp_tuned = false;             // spectral-pass launch width tuned
  std::vector<void*> owned;
};

struct GraphEntry {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  int n_init = 0, n_body = 0, n_fin = 0;
};

}  // namespace

struct LaunchRec {
  int kind = 0, E = 0, threads = 0;
  dim3 grid;
  size_t smem = 0;
  bool f64 = false;
  PassArgs<float> af{};
  PassArgs<double> ad{};
};

struct BatchedGroup {
  Plan* p = nullptr;
  std::vector<int> fields;          // indices into the caller's field arrays
  int n_init = 0, n_body = 0, n_fin = 0;
};

struct BatchedEntry {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<BatchedGroup> groups;
  // one launch per pass stage over all groups (k_multi): launches of the
  // initial residual, of one loop body and of the finish; owned device arrays
  bool multi = false;
  int m_init = 0, m_body = 0, m_fin = 0;
  std::vector<void*> owned;
};

struct CnnWork {
  gad::CnnBuffers w;
  std::vector<void*> owned;
  float* ub = nullptr;          // training minibatch gathers
  float* ut = nullptr;
  float* u0 = nullptr;
  double* losses = nullptr;     // per minibatch
  int nloss = 0;
};

struct ad_ctx {
  std::map<std::string, CnnWork*> cnn;        // learned-guess workspaces by (shape, batch)
  bool autotune = false;                      // tune the tiles of every new plan of a batched solve
  bool batched_multi = false;                 // batched solves: one launch per pass stage over all groups
  std::vector<LaunchRec>* record = nullptr;   // when set, pass launches are recorded, not issued
  std::map<std::string, BatchedEntry> bgraphs;
  std::vector<cudaStream_t> branches;         // capture streams of the batched graph's branches
  std::vector<cudaEvent_t> events;
  int device = 0;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  bool use_graph = true;
  std::map<std::pair<long long, int>, void*> tw;     // (length, is_f64) -> table
  std::map<std::string, Plan*> plans;
  std::map<std::string, GraphEntry> graphs;
  std::string err;
  int64_t launches = 0;
  void* stat_buf = nullptr;                   // device scratch of the statistics calls
  size_t stat_cap = 0;
  unsigned long long wait_ns = 1000000000ull; // limit of bounded device waits
  int rev_next = 0;                           // field order of the next pass launch
};

namespace {

ad_status fail(ad_ctx* c, ad_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

ad_status cuda_fail(ad_ctx* c, cudaError_t e, const char* where) {
  if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return AD_ERR_CUDA;
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);       \
  } while (0)

// exp(-2 pi i m / L), m in [0, L), evaluated in long double with exact
// values at the quarter points.
template <typename T>
std::vector<T> twiddle_host(long long L) {
  std::vector<T> t(2 * L);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (long long m = 0; m < L; ++m) {
    long double c, s;
    if (4 * m == L) { c = 0; s = -1; }
    else if (2 * m == L) { c = -1; s = 0; }
    else if (4 * m == 3 * L) { c = 0; s = 1; }
    else {
      const long double ang = two_pi * (long double)m / (long double)L;
      c = cosl(ang);
      s = -sinl(ang);
    }
    t[2 * m] = (T)c;
    t[2 * m + 1] = (T)s;
  }
  return t;
}

// The twiddle table of the FFT plan of length L for E elements per thread
// (plan.h): per-stage factors, cached per (plan, precision). Null (and AD_OK)
// when L has no plan; building the plan then fails.
ad_status get_plan_table(ad_ctx* ctx, int L, int E, bool reversed, bool f64, const void** out) {
  int rad[kMaxStages];
  const int n = plan_radices(L, E, reversed, rad);
  *out = nullptr;
  if (n == 0) return AD_OK;
  // keys of full tables are (L, 0 or 1); plan tables are (L | E | reversed, 2 or 3)
  const auto key = std::make_pair(((long long)L << 8) | ((long long)E << 1) | (reversed ? 1 : 0), f64 ? 3 : 2);
  auto it = ctx->tw.find(key);
  if (it != ctx->tw.end()) { *out = it->second; return AD_OK; }
  const size_t ents = (size_t)std::max(L - 1, 1);
  void* d = nullptr;
  const size_t bytes = ents * (f64 ? 16 : 8);
  if (cudaMalloc(&d, bytes) != cudaSuccess) { cudaGetLastError(); return fail(ctx, AD_ERR_NOMEM, "twiddle table"); }
  cudaError_t e;
  if (f64) {
    std::vector<double> h(2 * ents, 0.0);
    plan_twiddles<double>(rad, n, h.data());
    e = cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice);
  } else {
    std::vector<float> h(2 * ents, 0.f);
    plan_twiddles<float>(rad, n, h.data());
    e = cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) { cudaFree(d); return cuda_fail(ctx, e, "twiddle upload"); }
  ctx->tw[key] = d;
  *out = d;
  return AD_OK;
}

ad_status get_table(ad_ctx* ctx, long long L, bool f64, const void** out) {
  auto key = std::make_pair(L, f64 ? 1 : 0);
  auto it = ctx->tw.find(key);
  if (it != ctx->tw.end()) { *out = it->second; return AD_OK; }
  void* d = nullptr;
  size_t bytes = (size_t)L * (f64 ? 16 : 8);
  if (cudaMalloc(&d, bytes) != cudaSuccess) { cudaGetLastError(); return fail(ctx, AD_ERR_NOMEM, "twiddle table"); }
  cudaError_t e;
  if (f64) {
    auto h = twiddle_host<double>(L);
    e = cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice);
  } else {
    auto h = twiddle_host<float>(L);
    e = cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) { cudaFree(d); return cuda_fail(ctx, e, "twiddle upload"); }
  ctx->tw[key] = d;
  *out = d;
  return AD_OK;
}

// The tile shape of a pass (plan.h) copied into its launch configuration.
bool choose_tile(int L, int E, int slots, int div, size_t csize, PassCfg& pc) {
  TileShape ts;
  if (!gad::choose_tile(L, E, slots, div, csize, ts)) return false;
  pc.E = ts.E;
  pc.W = ts.W;
  pc.T = ts.T;
  pc.ld = ts.ld;
  pc.smem = ts.smem;
  return true;
}

// A method value: one of AD_VANCITTERT .. AD_SD, optionally OR-ed with AD_SPECTRAL.
bool method_ok(int m) {
  if (m < 0 || (m & ~(AD_SPECTRAL | AD_PRECOND | 3)) != 0) return false;
  // the preconditioner is defined for CG (in either space)
  if ((m & AD_PRECOND) && (m & 3) != AD_CG) return false;
  return true;
}
int method_base(int m) { return m & 3; }
bool method_spectral(int m) { return (m & AD_SPECTRAL) != 0; }
bool method_precond(int m) { return (m & AD_PRECOND) != 0; }

std::string plan_key(const ad_grid* g, int batch) {
  char buf[256];
  snprintf(buf, sizeof buf, "%d:%lld:%lld:%lld:%d:%a:%d", g->ndim, (long long)g->n[0], (long long)g->n[1],
           g->ndim == 3 ? (long long)g->n[2] : 1LL, (int)g->dtype, g->gamma, batch);
  return buf;
}

ad_status check_grid(ad_ctx* ctx, const ad_grid* g) {
  if (!g) return fail(ctx, AD_ERR_ARG, "grid is NULL");
  if (g->ndim != 2 && g->ndim != 3) return fail(ctx, AD_ERR_ARG, "ndim must be 2 or 3");
  if (g->dtype != AD_F32 && g->dtype != AD_F64) return fail(ctx, AD_ERR_ARG, "dtype must be AD_F32 or AD_F64");
  if (!(g->gamma > 0.0) || !std::isfinite(g->gamma)) return fail(ctx, AD_ERR_ARG, "gamma must be positive");
  for (int d = 0; d < g->ndim; ++d) {
    const long long n = g->n[d];
    if (n < 8 || n > 16384 || !smooth23(n) || (n % 2) != 0)
      return fail(ctx, AD_ERR_ARG, "each side must be an even 2^a 3^b in [8, 16384]");
  }
  if (g->n[0] % 4 != 0) return fail(ctx, AD_ERR_ARG, "Nx must be a multiple of 4");
  return AD_OK;
}

ad_status dmalloc(ad_ctx* ctx, Plan* p, void** out, size_t bytes) {
  if (cudaMalloc(out, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, AD_ERR_NOMEM, "workspace allocation of " + std::to_string(bytes) + " bytes");
  }
  p->owned.push_back(*out);
  return AD_OK;
}

void free_plan(Plan* p) {
  for (void* q : p->owned) cudaFree(q);
  delete p;
}

ad_status get_plan(ad_ctx* ctx, const ad_grid* g, int batch, Plan** out) {
  if (batch > AD_MAX_BATCH) return fail(ctx, AD_ERR_ARG, "batch > AD_MAX_BATCH");
  const std::string key = plan_key(g, batch);
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) { *out = it->second; return AD_OK; }
  Plan* p = new Plan;
  p->ndim = g->ndim;
  p->nx = (int)g->n[0];
  p->ny = (int)g->n[1];
  p->nz = g->ndim == 3 ? (int)g->n[2] : 1;
  p->kxn = p->nx / 2 + 1;
  p->batch = batch;
  p->f64 = g->dtype == AD_F64;
  p->gamma = g->gamma;
  p->P = (long long)p->nx * p->ny * p->nz;
  p->SP = (long long)p->kxn * p->ny * p->nz;
  const size_t cs = p->f64 ? 16 : 8, rs = p->f64 ? 8 : 4;
  ad_status s;
  const void* tx = nullptr;
  if ((s = get_table(ctx, p->nx, p->f64, &tx)) != AD_OK) { delete p; return s; }
  p->twx = tx;                                  // the real-to-complex split of the x passes
  const int M = p->nx / 2;
  const int Lf = p->ndim == 3 ? p->nz : p->ny;
  const void *px = nullptr, *pf = nullptr, *pfi = nullptr, *py = nullptr;
  if ((s = get_plan_table(ctx, M, pick_E(M), false, p->f64, &px)) != AD_OK ||
      (s = get_plan_table(ctx, Lf, pick_E(Lf), false, p->f64, &pf)) != AD_OK ||
      (s = get_plan_table(ctx, Lf, pick_E(Lf), true, p->f64, &pfi)) != AD_OK ||
      (p->ndim == 3 && (s = get_plan_table(ctx, p->ny, pick_E(p->ny), false, p->f64, &py)) != AD_OK)) {
    delete p;
    return s;
  }
  bool ok = true;
  // x passes: complex length M (packed real rows)
  ok = ok && choose_tile(M, pick_E(M), M + 1, pow2_part(p->ny), cs, p->xf);
  ok = ok && make_fft(M, p->xf.E, px, p->xf.fft);
  p->xf.rcp_a = 1.0f / (float)(p->nx / 4);
  p->xf.rcp_b = 1.0f / (float)(M / 2 + 1);
  p->xf.grid = dim3(p->ny * p->nz / std::max(p->xf.W, 1), batch);
  p->xi = p->xf;
  // filter pass along the last axis
  const int nseq = p->ndim == 3 ? p->kxn * p->ny : p->kxn;
  ok = ok && choose_tile(Lf, pick_E(Lf), Lf, 0, cs, p->fl);
  ok = ok && make_fft(Lf, p->fl.E, pf, p->fl.fft);
  ok = ok && make_fft(Lf, p->fl.E, pfi, p->fl.fft_inv, true);
  p->fl.rcp_a = 1.0f / (float)(Lf / 2);
  p->fl.rcp_b = 1.0f / (float)Lf;
  p->fl.grid = dim3((nseq + std::max(p->fl.W, 1) - 1) / std::max(p->fl.W, 1), batch);
  if (p->ndim == 3) {
    ok = ok && choose_tile(p->ny, pick_E(p->ny), p->ny, pow2_part(p->nz), cs, p->yf);
    ok = ok && make_fft(p->ny, p->yf.E, py, p->yf.fft);
    p->yf.rcp_a = 1.0f / (float)(p->ny / 2);
    p->yf.rcp_b = 1.0f / (float)p->ny;
    p->yf.grid = dim3(p->kxn * (p->nz / std::max(p->yf.W, 1)), batch);
    p->yi = p->yf;
  }
  if (!ok) { delete p; return fail(ctx, AD_ERR_ARG, "no tiling for this grid"); }
  {
    // stencil pass: the march runs along z (3D) or y (2D); a ring of four
    // slices in shared memory, a slice being W + 2 rows in 3D (W a power of
    // two dividing Ny, at most 16, four slices within 96 KB) and one row in
    // 2D; the march axis is cut into chunks (a divisor of its length) until
    // the launch has 4 blocks per SM or the chunks are down to 4 positions
    const size_t row = (size_t)p->nx * rs;
    int W = 1;
    if (p->ndim == 3)
      for (int w = 2; w <= 16 && p->ny % w == 0; w *= 2) {
        if (4 * (size_t)(w + 2) * row > 96 * 1024) break;
        W = w;
      }
    const int srows = p->ndim == 3 ? W + 2 : 1;
    const int nmarch = p->ndim == 3 ? p->nz : p->ny;
    const long long tiles = p->ndim == 3 ? p->ny / W : 1;
    int chunk = nmarch;
    for (int nch = 1; nch <= nmarch; ++nch) {
      if (nmarch % nch != 0) continue;
      chunk = nmarch / nch;
      if (tiles * nch * batch >= 4 * 152 || chunk <= 4) break;
    }
    p->sn = PassCfg{};
    p->sn.W = W;
    p->sn.chunk = chunk;
    p->sn.smem = 4 * (size_t)srows * row;
    const long long vec4 = (long long)W * p->nx / 4;
    p->sn.T = (int)std::min<long long>(256, (vec4 + 31) / 32 * 32);
    p->sn.rcp_a = 1.0f / (float)(p->nx / 4);
    p->sn.grid = dim3((unsigned)(tiles * (nmarch / chunk)), batch);
  }
  const size_t vb = (size_t)p->P * batch * rs, sb = (size_t)p->SP * batch * cs;
  if ((s = dmalloc(ctx, p, &p->S1, sb)) != AD_OK ||
      (p->ndim == 3 && (s = dmalloc(ctx, p, &p->S2, sb)) != AD_OK)) { free_plan(p); return s; }
  // partials sized for the narrowest tile the autotuner may pick (1/8 of the default width)
  const unsigned maxblk = 8 * std::max(p->xi.grid.x, p->fl.grid.x) + p->sn.grid.x + 8;
  p->maxblk = maxblk;
  if ((s = dmalloc(ctx, p, (void**)&p->st, sizeof(FieldState) * batch)) != AD_OK ||
      (s = dmalloc(ctx, p, (void**)&p->part, sizeof(double) * 4 * maxblk * batch)) != AD_OK ||
      (s = dmalloc(ctx, p, (void**)&p->ticket, sizeof(unsigned) * (4 + batch))) != AD_OK) { free_plan(p); return s; }
  if (cudaMemset(p->ticket, 0, sizeof(unsigned) * (4 + batch)) != cudaSuccess) {
    free_plan(p);
    return cuda_fail(ctx, cudaGetLastError(), "ticket");
  }
  (void)vb;
  ctx->plans[key] = p;
  *out = p;
  return AD_OK;
}

ad_status ensure_vectors(ad_ctx* ctx, Plan* p) {
  if (p->R) return AD_OK;
  const size_t vb = (size_t)p->P * p->batch * (p->f64 ? 8 : 4);
  ad_status s;
  if ((s = dmalloc(ctx, p, &p->R, vb)) != AD_OK || (s = dmalloc(ctx, p, &p->Pv, vb)) != AD_OK ||
      (s = dmalloc(ctx, p, &p->Q, vb)) != AD_OK || (s = dmalloc(ctx, p, &p->Sv, vb)) != AD_OK ||
      (s = dmalloc(ctx, p, &p->F0, vb)) != AD_OK)
    return s;
  return AD_OK;
}

// Spectral-space vectors (complex half spectra, SP per field) and the launch
// shape of the streaming spectral passes: each block streams a contiguous
// range of sequences, about 2048 element pairs at least, at most 1216 blocks
// (8 per SM) per field and never more than the partial-dot capacity. The
// shape depends on the grid only, so a field's result does not depend on
// the batch it is solved in.
ad_status ensure_spectral(ad_ctx* ctx, Plan* p) {
  if (p->Bh) return AD_OK;
  const size_t sb = (size_t)p->SP * p->batch * (p->f64 ? 16 : 8);
  ad_status s;
  if ((s = dmalloc(ctx, p, &p->Bh, sb)) != AD_OK || (s = dmalloc(ctx, p, &p->Uh, sb)) != AD_OK ||
      (s = dmalloc(ctx, p, &p->Rh, sb)) != AD_OK || (s = dmalloc(ctx, p, &p->Ph, sb)) != AD_OK ||
      (s = dmalloc(ctx, p, &p->F0h, sb)) != AD_OK)
    return s;
  const long long pairs = p->SP / 2;
  long long nb = (pairs + 2047) / 2048;
  nb = std::min<long long>(nb, 1216);
  nb = std::min<long long>(nb, (long long)p->maxblk);
  p->sp = PassCfg{};
  p->sp.T = 256;
  p->sp.grid = dim3((unsigned)std::max<long long>(nb, 1), p->batch);
  return AD_OK;
}

void drop_graphs(ad_ctx* ctx) {
  for (auto& kv : ctx->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.g) cudaGraphDestroy(kv.second.g);
  }
  ctx->graphs.clear();
  for (auto& kv : ctx->bgraphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.g) cudaGraphDestroy(kv.second.g);
    for (void* q : kv.second.owned) cudaFree(q);
  }
  ctx->bgraphs.clear();
}

ad_status ensure_hist(ad_ctx* ctx, Plan* p, int maxit) {
  if (maxit + 1 <= p->hist_cap) return AD_OK;
  drop_graphs(ctx);     // graphs hold the old history pointer
  if (p->hist) {
    cudaFree(p->hist);
    for (auto& q : p->owned) if (q == p->hist) q = nullptr;
  }
  p->hist = nullptr;
  int cap = std::max(maxit + 1, 64);
  ad_status s = dmalloc(ctx, p, (void**)&p->hist, sizeof(double) * (size_t)cap * p->batch);
  if (s != AD_OK) return s;
  p->hist_cap = cap;
  return AD_OK;
}

// ---------------------------------------------------------------------------
// Enqueueing one application of G with the given fused prologue/epilogue.
struct Fwd { int op = XF_COPY; const void* A = nullptr; const void* B = nullptr; void* O1 = nullptr; void* O2 = nullptr; void* O3 = nullptr;
             bool clear_cond = false; };
struct Flt { int op = FI_NONE; int stage = SS_NONE; };
struct Inv { int op = XI_STORE; const void* A = nullptr; const void* B = nullptr; const void* C = nullptr;
             void* O1 = nullptr; void* O2 = nullptr; int ndots = 0; int stage = SS_NONE; bool set_cond = false; };
struct Common { FieldState* st = nullptr; SolveConfig cfg{}; cudaGraphConditionalHandle cond = 0; bool in_graph = false; int force = 0;
                int ncomp = 0, npairs = 0, pair_code = 0; unsigned long long wait_ns = 1000000000ull; };

template <typename T>
PassArgs<T> base_args(const Plan* p, const Common& c) {
  PassArgs<T> a{};
  a.nx = p->nx; a.ny = p->ny; a.nz = p->nz; a.kxn = p->kxn;
  a.P = p->P; a.SP = p->SP;
  a.twx = p->twx;
  const double kc = p->gamma * (double)std::min(p->nx, std::min(p->ny, p->ndim == 3 ? p->nz : p->ny)) / 2.0;
  a.kc2 = (T)(kc * kc);
  a.inv_p = 1.0;                      // physical-space dots are plain sums
  a.gscale = (T)(1.0 / (double)p->P);
  // preconditioner weights (delta/h_d)^2 = (N_d / (2 pi k_c))^2
  const double tpk = 2.0 * 3.14159265358979323846 * kc;
  a.cx = (T)((p->nx / tpk) * (p->nx / tpk));
  a.cy = (T)((p->ny / tpk) * (p->ny / tpk));
  a.cz = (T)(p->ndim == 3 ? (p->nz / tpk) * (p->nz / tpk) : 0.0);
  a.S1 = p->S1; a.S2 = p->S2;
  a.st = c.st; a.cfg = c.cfg; a.part = p->part; a.ticket = p->ticket;
  a.cond = c.cond; a.batch = p->batch; a.force = c.force;
  a.ncomp = c.ncomp; a.npairs = c.npairs; a.pair_code = c.pair_code;
  a.wait_ns = c.wait_ns;
  return a;
}

template <typename T>
void set_pass(PassArgs<T>& a, const PassCfg& pc) {
  a.W = pc.W; a.ld = pc.ld; a.fft = pc.fft; a.fft_inv = pc.fft_inv; a.rcp_a = pc.rcp_a; a.rcp_b = pc.rcp_b;
  a.tfft = pc.T;
}

// Blocks always hold whole warps (the reductions shuffle over full warps).
int block_threads(const PassCfg& pc) { return (pc.T + 31) / 32 * 32; }

template <typename T> void store_args(LaunchRec& r, const PassArgs<T>& a);
template <> void store_args<float>(LaunchRec& r, const PassArgs<float>& a) { r.af = a; r.f64 = false; }
template <> void store_args<double>(LaunchRec& r, const PassArgs<double>& a) { r.ad = a; r.f64 = true; }

// Successive pass launches alternate the order of the fields (PassArgs::rev):
// a pass then starts on the fields the previous one finished with, whose
// vectors and spectra may still be in L2. A field's result does not depend on
// the order.
template <typename T>
cudaError_t issue(ad_ctx* ctx, int kind, const PassCfg& pc, cudaStream_t s, const PassArgs<T>& a0) {
  PassArgs<T> a = a0;
  a.rev = ctx->rev_next;
  ctx->rev_next ^= 1;
  if (ctx->record) {
    LaunchRec r;
    r.kind = kind; r.E = pc.E; r.grid = pc.grid; r.threads = block_threads(pc); r.smem = pc.smem;
    store_args<T>(r, a);
    ctx->record->push_back(r);
    return cudaSuccess;
  }
  return launch_pass<T>(kind, pc.E, pc.grid, block_threads(pc), pc.smem, s, a);
}

template <typename T>
ad_status enqueue_G(ad_ctx* ctx, Plan* p, cudaStream_t s, const Fwd& fw, const Flt& fl, const Inv& iv,
                    const Common& c, int* nl) {
  PassArgs<T> a = base_args<T>(p, c);
  // forward x pass
  set_pass(a, p->xf);
  a.op = fw.op; a.A = (const T*)fw.A; a.B = (const T*)fw.B;
  a.O1 = (T*)fw.O1; a.O2 = (T*)fw.O2; a.O3 = (T*)fw.O3;
  a.ndots = 0; a.stage = SS_NONE; a.set_cond = 0; a.clear_cond = (fw.clear_cond && c.in_graph) ? 1 : 0;
  CK(issue<T>(ctx, PK_XFWD, p->xf, s, a));
  ++*nl;
  if (p->ndim == 3) {
    set_pass(a, p->yf);
    CK(issue<T>(ctx, PK_YFWD, p->yf, s, a));
    ++*nl;
  }
  a.clear_cond = 0;
  set_pass(a, p->fl);
  a.op = fl.op;
  a.ndots = fl.op == FI_NONE ? 0 : (fl.op == FI_XGX ? 1 : 3);
  a.stage = fl.stage;
  a.inv_p = 1.0 / (double)p->P;       // Parseval: (a, b) = (1/P) sum_k a_hat conj(b_hat)
  CK(issue<T>(ctx, PK_FILT, p->fl, s, a));
  ++*nl;
  a.ndots = 0; a.stage = SS_NONE; a.inv_p = 1.0;
  if (p->ndim == 3) {
    set_pass(a, p->yi);
    CK(issue<T>(ctx, PK_YINV, p->yi, s, a));
    ++*nl;
  }
  set_pass(a, p->xi);
  a.op = iv.op; a.A = (const T*)iv.A; a.B = (const T*)iv.B; a.C = (const T*)iv.C;
  a.O1 = (T*)iv.O1; a.O2 = (T*)iv.O2; a.O3 = nullptr;
  a.ndots = iv.ndots; a.stage = iv.stage; a.set_cond = (iv.set_cond && c.in_graph) ? 1 : 0;
  CK(issue<T>(ctx, PK_XINV, p->xi, s, a));
  ++*nl;
  return AD_OK;
}

struct SolveIO {
  const void* ubar;
  void* u;
  const void* u0;
  int method;           // AD_VANCITTERT .. AD_SD (the AD_SPECTRAL flag goes to `spectral`)
  bool want_true;
  bool spectral = false;
  bool precond = false;   // AD_CG with the stencil preconditioner (AD_PRECOND)
};

// ---------------------------------------------------------------------------
// Spectral-space solve: transforms, streaming passes, init/body/finish.

// x = u_bar or u0 -> its half spectrum `out` (x pass, 3D y pass, last-axis pass).
template <typename T>
ad_status enqueue_fwd_transform(ad_ctx* ctx, Plan* p, cudaStream_t s, const void* x, void* out, int* nl) {
  Common c0;                            // no solver state: every field runs
  PassArgs<T> a = base_args<T>(p, c0);
  set_pass(a, p->xf);
  a.op = XF_COPY; a.A = (const T*)x;
  CK(issue<T>(ctx, PK_XFWD, p->xf, s, a));
  ++*nl;
  if (p->ndim == 3) {
    set_pass(a, p->yf);
    CK(issue<T>(ctx, PK_YFWD, p->yf, s, a));
    ++*nl;
  }
  set_pass(a, p->fl);
  a.O1 = (T*)out;
  CK(issue<T>(ctx, PK_LFWD, p->fl, s, a));
  ++*nl;
  return AD_OK;
}

// half spectrum `hat` -> physical field x (scaled by 1/P on the way).
template <typename T>
ad_status enqueue_inv_transform(ad_ctx* ctx, Plan* p, cudaStream_t s, const void* hat, void* x, int* nl) {
  Common c0;
  PassArgs<T> a = base_args<T>(p, c0);
  set_pass(a, p->fl);
  a.A = (const T*)hat;
  CK(issue<T>(ctx, PK_LINV, p->fl, s, a));
  ++*nl;
  a.A = nullptr;
  if (p->ndim == 3) {
    set_pass(a, p->yi);
    CK(issue<T>(ctx, PK_YINV, p->yi, s, a));
    ++*nl;
  }
  set_pass(a, p->xi);
  a.op = XI_STORE; a.O1 = (T*)x;
  CK(issue<T>(ctx, PK_XINV, p->xi, s, a));
  ++*nl;
  return AD_OK;
}

struct Spec {
  int op = SP_REF, stage = SS_NONE, ndots = 1;
  const void* A = nullptr; const void* B = nullptr;
  void* O1 = nullptr; void* O2 = nullptr; void* O3 = nullptr;
  bool clear_cond = false, set_cond = false;
};

template <typename T>
ad_status enqueue_spec(ad_ctx* ctx, Plan* p, cudaStream_t s, const Spec& sp, const Common& c, int* nl) {
  PassArgs<T> a = base_args<T>(p, c);
  a.op = sp.op; a.stage = sp.stage; a.ndots = sp.ndots;
  a.A = (const T*)sp.A; a.B = (const T*)sp.B;
  a.O1 = (T*)sp.O1; a.O2 = (T*)sp.O2; a.O3 = (T*)sp.O3;
  a.inv_p = 1.0 / (double)p->P;        // Parseval
  a.clear_cond = (sp.clear_cond && c.in_graph) ? 1 : 0;
  a.set_cond = (sp.set_cond && c.in_graph) ? 1 : 0;
  CK(issue<T>(ctx, PK_SPEC, p->sp, s, a));
  ++*nl;
  return AD_OK;
}

template <typename T>
ad_status enqueue_spec_init(ad_ctx* ctx, Plan* p, cudaStream_t s, const SolveIO& io, const Common& c, int* nl) {
  CK(launch_reset_state(p->st, p->batch, s));
  ++*nl;
  ad_status r;
  if ((r = enqueue_fwd_transform<T>(ctx, p, s, io.ubar, p->Bh, nl)) != AD_OK) return r;
  if (io.u0) {
    if ((r = enqueue_fwd_transform<T>(ctx, p, s, io.u0, p->Uh, nl)) != AD_OK) return r;
    Spec ref; ref.op = SP_REF; ref.stage = SS_REF; ref.A = p->Bh;
    if ((r = enqueue_spec<T>(ctx, p, s, ref, c, nl)) != AD_OK) return r;
  }
  Spec in; in.op = io.precond ? SP_PCG_INIT : SP_INIT; in.stage = io.precond ? SS_PCG_INIT : SS_INIT;
  in.ndots = io.precond ? 2 : 1; in.A = p->Bh;
  in.B = io.u0 ? p->Uh : nullptr;
  in.O1 = io.u0 ? nullptr : p->Uh;
  in.O2 = p->Rh;
  in.O3 = io.method == AD_BICGSTAB ? p->F0h : nullptr;
  return enqueue_spec<T>(ctx, p, s, in, c, nl);
}

template <typename T>
ad_status enqueue_spec_body(ad_ctx* ctx, Plan* p, cudaStream_t s, const SolveIO& io, const Common& c, int* nl) {
  ad_status r;
  switch (io.method) {
    case AD_VANCITTERT: {
      Spec k; k.op = SP_VC; k.stage = SS_VC; k.O1 = p->Uh; k.O2 = p->Rh; k.clear_cond = k.set_cond = true;
      return enqueue_spec<T>(ctx, p, s, k, c, nl);
    }
    case AD_SD: {
      Spec k1; k1.op = SP_SD_A; k1.stage = SS_SD_ALPHA; k1.A = p->Rh; k1.clear_cond = true;
      if ((r = enqueue_spec<T>(ctx, p, s, k1, c, nl)) != AD_OK) return r;
      Spec k2; k2.op = SP_SD; k2.stage = SS_VC; k2.O1 = p->Uh; k2.O2 = p->Rh; k2.set_cond = true;
      return enqueue_spec<T>(ctx, p, s, k2, c, nl);
    }
    case AD_CG: {
      if (io.precond) {            // preconditioned CG: z = M_hat r, p = z + beta p; u += alpha p, r -= alpha G p
        Spec k1; k1.op = SP_PCG_P; k1.stage = SS_CG_ALPHA; k1.A = p->Rh; k1.O1 = p->Ph; k1.clear_cond = true;
        if ((r = enqueue_spec<T>(ctx, p, s, k1, c, nl)) != AD_OK) return r;
        Spec k2; k2.op = SP_PCG; k2.stage = SS_PCG_END; k2.ndots = 2; k2.A = p->Ph; k2.O1 = p->Uh; k2.O2 = p->Rh;
        k2.set_cond = true;
        return enqueue_spec<T>(ctx, p, s, k2, c, nl);
      }
      Spec k1; k1.op = SP_CG_P; k1.stage = SS_CG_ALPHA; k1.A = p->Rh; k1.O1 = p->Ph; k1.clear_cond = true;
      if ((r = enqueue_spec<T>(ctx, p, s, k1, c, nl)) != AD_OK) return r;
      Spec k2; k2.op = SP_CG; k2.stage = SS_CG_BETA; k2.A = p->Ph; k2.O1 = p->Uh; k2.O2 = p->Rh; k2.set_cond = true;
      return enqueue_spec<T>(ctx, p, s, k2, c, nl);
    }
    case AD_BICGSTAB: {
      Spec k1; k1.op = SP_BI_P; k1.stage = SS_BI_ALPHA; k1.A = p->Rh; k1.B = p->F0h; k1.O1 = p->Ph;
      k1.clear_cond = true;
      if ((r = enqueue_spec<T>(ctx, p, s, k1, c, nl)) != AD_OK) return r;
      Spec k2; k2.op = SP_BI_S; k2.stage = SS_BI_OMEGA; k2.ndots = 3; k2.A = p->Rh; k2.B = p->Ph;
      if ((r = enqueue_spec<T>(ctx, p, s, k2, c, nl)) != AD_OK) return r;
      Spec k3; k3.op = SP_BI_END; k3.stage = SS_BI_END; k3.ndots = 2; k3.A = p->Ph; k3.B = p->F0h;
      k3.O1 = p->Uh; k3.O2 = p->Rh; k3.set_cond = true;
      return enqueue_spec<T>(ctx, p, s, k3, c, nl);
    }
    default:
      return fail(ctx, AD_ERR_ARG, "unknown method");
  }
}

// The initial residual r0 = u_bar - G u0 (and, with an explicit u0, the
// reference ||u_bar - G u_bar||): the passes of the physical-space init,
// after the state reset.
template <typename T>
ad_status enqueue_init_passes(ad_ctx* ctx, Plan* p, cudaStream_t s, const SolveIO& io, const Common& c, int* nl) {
  ad_status r;
  if (io.u0) {
    Fwd fw; fw.op = XF_COPY; fw.A = io.ubar;
    Inv iv; iv.op = XI_RES; iv.A = io.ubar; iv.ndots = 1; iv.stage = SS_REF;
    if ((r = enqueue_G<T>(ctx, p, s, fw, Flt{}, iv, c, nl)) != AD_OK) return r;
  }
  Fwd fw; fw.op = XF_COPY; fw.A = io.u0 ? io.u0 : io.ubar; fw.O1 = io.u;
  Inv iv; iv.op = XI_INIT; iv.A = io.ubar; iv.O1 = p->R; iv.O2 = io.method == AD_BICGSTAB ? p->F0 : nullptr;
  iv.ndots = 1; iv.stage = SS_INIT;
  return enqueue_G<T>(ctx, p, s, fw, Flt{}, iv, c, nl);
}

template <typename T>
ad_status enqueue_init(ad_ctx* ctx, Plan* p, cudaStream_t s, const SolveIO& io, const Common& c, int* nl) {
  if (io.spectral) return enqueue_spec_init<T>(ctx, p, s, io, c, nl);
  CK(launch_reset_state(p->st, p->batch, s));
  ++*nl;
  return enqueue_init_passes<T>(ctx, p, s, io, c, nl);
}

// z = M r (the preconditioner stencil) with the dot (r, z) -> rho, beta.
template <typename T>
ad_status enqueue_sten(ad_ctx* ctx, Plan* p, cudaStream_t s, const void* r, void* z, const Common& c,
                       bool clear_cond, int* nl) {
  PassArgs<T> a = base_args<T>(p, c);
  a.W = p->sn.W; a.chunk = p->sn.chunk; a.rcp_a = p->sn.rcp_a; a.tfft = p->sn.T;
  a.op = 0; a.A = (const T*)r; a.O1 = (T*)z;
  a.ndots = 1; a.stage = SS_PCG_RHO; a.set_cond = 0;
  a.clear_cond = (clear_cond && c.in_graph) ? 1 : 0;
  CK(issue<T>(ctx, PK_STEN, p->sn, s, a));
  ++*nl;
  return AD_OK;
}

template <typename T>
ad_status enqueue_body(ad_ctx* ctx, Plan* p, cudaStream_t s, const SolveIO& io, const Common& c, int* nl) {
  if (io.spectral) return enqueue_spec_body<T>(ctx, p, s, io, c, nl);
  ad_status r;
  if (io.precond) {                // preconditioned CG: z = M r; then Algorithm 3's pass with p = z + beta p
    if ((r = enqueue_sten<T>(ctx, p, s, p->R, p->Q, c, true, nl)) != AD_OK) return r;
    Fwd fw; fw.op = XF_CG; fw.A = p->Q; fw.O1 = io.u; fw.O2 = p->Pv;
    Flt fl; fl.op = FI_XGX; fl.stage = SS_CG_ALPHA;
    Inv iv; iv.op = XI_CG; iv.O1 = p->R; iv.ndots = 1; iv.stage = SS_PCG_STOP; iv.set_cond = true;
    return enqueue_G<T>(ctx, p, s, fw, fl, iv, c, nl);
  }
  switch (io.method) {
    case AD_VANCITTERT: {          // Algorithm 1: u += r; d = G r; r -= d
      Fwd fw; fw.clear_cond = true; fw.op = XF_VC; fw.A = p->R; fw.O1 = io.u;
      Inv iv; iv.op = XI_VC; iv.O1 = p->R; iv.ndots = 1; iv.stage = SS_VC; iv.set_cond = true;
      return enqueue_G<T>(ctx, p, s, fw, Flt{}, iv, c, nl);
    }
    case AD_SD: {                  // Algorithm 2: d = G r; alpha = (r,r)/(r,d); u += alpha r; r -= alpha d
      Fwd fw; fw.clear_cond = true; fw.op = XF_COPY; fw.A = p->R;
      Flt fl; fl.op = FI_XGX; fl.stage = SS_SD_ALPHA;
      Inv iv; iv.op = XI_SD; iv.O1 = p->R; iv.O2 = io.u; iv.ndots = 1; iv.stage = SS_VC; iv.set_cond = true;
      return enqueue_G<T>(ctx, p, s, fw, fl, iv, c, nl);
    }
    case AD_CG: {                  // Algorithm 3, u += alpha p deferred to the next forward pass
      Fwd fw; fw.clear_cond = true; fw.op = XF_CG; fw.A = p->R; fw.O1 = io.u; fw.O2 = p->Pv;
      Flt fl; fl.op = FI_XGX; fl.stage = SS_CG_ALPHA;
      Inv iv; iv.op = XI_CG; iv.O1 = p->R; iv.ndots = 1; iv.stage = SS_CG_BETA; iv.set_cond = true;
      return enqueue_G<T>(ctx, p, s, fw, fl, iv, c, nl);
    }
    case AD_BICGSTAB: {            // Algorithm 4: two applications of G per pass
      Fwd f1; f1.clear_cond = true; f1.op = XF_BI_P; f1.A = p->R; f1.B = p->Q; f1.O2 = p->Pv;
      Inv i1; i1.op = XI_BI_Q; i1.A = p->F0; i1.O1 = p->Q; i1.ndots = 1; i1.stage = SS_BI_ALPHA;
      if ((r = enqueue_G<T>(ctx, p, s, f1, Flt{}, i1, c, nl)) != AD_OK) return r;
      Fwd f2; f2.op = XF_BI_S; f2.A = p->R; f2.B = p->Q; f2.O3 = p->Sv;
      Flt fl; fl.op = FI_SST; fl.stage = SS_BI_OMEGA;
      Inv i2; i2.op = XI_BI_T; i2.A = p->F0; i2.B = p->Pv; i2.C = p->Sv; i2.O1 = io.u; i2.O2 = p->R;
      i2.ndots = 2; i2.stage = SS_BI_END; i2.set_cond = true;
      return enqueue_G<T>(ctx, p, s, f2, fl, i2, c, nl);
    }
    default:
      return fail(ctx, AD_ERR_ARG, "unknown method");
  }
}

template <typename T>
ad_status enqueue_finish(ad_ctx* ctx, Plan* p, cudaStream_t s, const SolveIO& io, const Common& c, int* nl) {
  if (io.spectral) {
    ad_status r = enqueue_inv_transform<T>(ctx, p, s, p->Uh, io.u, nl);
    if (r != AD_OK) return r;
  } else if (io.method == AD_CG) {
    CK(launch_cg_finish<T>((T*)io.u, (const T*)p->Pv, p->st, p->P, p->batch, s));
    ++*nl;
  }
  if (io.want_true) {
    Common cf = c;
    cf.force = 1;
    Fwd fw; fw.op = XF_COPY; fw.A = io.u;
    Inv iv; iv.op = XI_RES; iv.A = io.ubar; iv.ndots = 1; iv.stage = SS_TRUE;
    return enqueue_G<T>(ctx, p, s, fw, Flt{}, iv, cf, nl);
  }
  return AD_OK;
}

template <typename T>
ad_status build_graph(ad_ctx* ctx, Plan* p, const SolveIO& io, Common c, GraphEntry& ge) {
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ctx, e, "cudaGraphConditionalHandleCreate"); }
  c.cond = h;
  c.in_graph = true;
  e = cudaStreamBeginCaptureToGraph(ctx->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ctx, e, "cudaStreamBeginCaptureToGraph"); }
  int n_init = 0, n_body = 0, n_fin = 0;
  ad_status st = enqueue_init<T>(ctx, p, ctx->cap, io, c, &n_init);
  cudaGraph_t body = nullptr;
  if (st == AD_OK) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(ctx->cap, &cs, nullptr, &cg, &deps, nullptr, &nd);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "cudaStreamGetCaptureInfo");
    cudaGraphNode_t cn = nullptr;
    cudaGraphNodeParams np{};
    if (st == AD_OK) {
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      e = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &np);
      if (e != cudaSuccess) st = cuda_fail(ctx, e, "cudaGraphAddNode(while)");
    }
    if (st == AD_OK) {
      e = cudaStreamUpdateCaptureDependencies(ctx->cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
      if (e != cudaSuccess) st = cuda_fail(ctx, e, "cudaStreamUpdateCaptureDependencies");
    }
    if (st == AD_OK) {
      body = np.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(ctx->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) st = cuda_fail(ctx, e, "cudaStreamBeginCaptureToGraph(body)");
      else {
        st = enqueue_body<T>(ctx, p, ctx->cap2, io, c, &n_body);
        cudaGraph_t bg = nullptr;
        e = cudaStreamEndCapture(ctx->cap2, &bg);
        if (st == AD_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "cudaStreamEndCapture(body)");
      }
    }
    if (st == AD_OK) st = enqueue_finish<T>(ctx, p, ctx->cap, io, c, &n_fin);
  }
  cudaGraph_t gout = nullptr;
  e = cudaStreamEndCapture(ctx->cap, &gout);
  if (st == AD_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "cudaStreamEndCapture");
  if (st != AD_OK) { cudaGetLastError(); cudaGraphDestroy(g); return st; }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ctx, e, "cudaGraphInstantiate"); }
  ge.g = g;
  ge.exec = exec;
  ge.n_init = n_init;
  ge.n_body = n_body;
  ge.n_fin = n_fin;
  return AD_OK;
}

template <typename T>
ad_status run_solve(ad_ctx* ctx, Plan* p, const SolveIO& io, double tol, int maxit, cudaStream_t stream,
                    int* loops_out, int* n_body_out) {
  Common c;
  c.st = p->st;
  c.wait_ns = ctx->wait_ns;
  c.cfg.tol = tol;
  c.cfg.maxit = maxit;
  c.cfg.method = io.method;
  c.cfg.hist = p->hist;
  c.cfg.hist_ld = p->hist_cap;
  ad_status st;
  if (ctx->use_graph) {
    char buf[256];
    snprintf(buf, sizeof buf, "|%d|%d|%d|%a|%d|%p|%p|%p|%d", io.method, io.spectral ? 1 : 0, io.precond ? 1 : 0,
             tol, maxit, io.ubar, io.u, io.u0, io.want_true ? 1 : 0);
    char pk[128];
    snprintf(pk, sizeof pk, "%p", (void*)p);
    const std::string gkey = std::string(pk) + buf;
    auto it = ctx->graphs.find(gkey);
    if (it == ctx->graphs.end()) {
      GraphEntry ge;
      if ((st = build_graph<T>(ctx, p, io, c, ge)) != AD_OK) return st;
      it = ctx->graphs.emplace(gkey, ge).first;
    }
    CK(cudaGraphLaunch(it->second.exec, stream));
    *loops_out = -1;
    *n_body_out = it->second.n_body;
    ctx->launches = it->second.n_init + it->second.n_fin;   // body launches added after readback
    return AD_OK;
  }
  // host-driven loop: body chunks, poll the active flags in between
  int nl = 0;
  if ((st = enqueue_init<T>(ctx, p, stream, io, c, &nl)) != AD_OK) return st;
  std::vector<FieldState> hs(p->batch);
  int loops = 0;
  for (;;) {
    CK(cudaMemcpyAsync(hs.data(), p->st, sizeof(FieldState) * p->batch, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    bool any = false;
    for (auto& f : hs) any = any || f.active;
    if (!any) break;
    const int chunk = 4;
    for (int i = 0; i < chunk; ++i) {
      int nb = 0;
      if ((st = enqueue_body<T>(ctx, p, stream, io, c, &nb)) != AD_OK) return st;
      nl += nb;
      ++loops;
    }
  }
  if ((st = enqueue_finish<T>(ctx, p, stream, io, c, &nl)) != AD_OK) return st;
  ctx->launches = nl;
  *loops_out = loops;
  return AD_OK;
}

// ---------------------------------------------------------------------------
// Tile autotuner: for every pass of a plan, times each admissible tile width
// (block sizes 32..256 threads, shared memory <= 100 KB, the partial-dot
// capacity respected) in the launch configuration of one iteration of
// `method`, on the plan's own buffers, and keeps the fastest.

struct TileSlot {
  PassCfg* pc;
  int kind;
  int L;
  int slots;
  int div;      // W must divide this (0: ragged tiles allowed)
};

void set_tile(const Plan* p, PassCfg& pc, int kind, int L, int slots, int W) {
  const int ld = tile_ld(slots);
  pc.W = W;
  pc.T = (int)((long long)W * L / pc.E);
  pc.ld = ld;
  pc.smem = (size_t)W * ld * (p->f64 ? 16 : 8);
  const int nseq = p->ndim == 3 ? p->kxn * p->ny : p->kxn;
  switch (kind) {
    case PK_XFWD: case PK_XINV: pc.grid = dim3(p->ny * p->nz / W, p->batch); break;
    case PK_FILT: pc.grid = dim3((nseq + W - 1) / W, p->batch); break;
    default: pc.grid = dim3(p->kxn * (p->nz / W), p->batch); break;
  }
}

template <typename T>
double time_kind(ad_ctx* ctx, Plan* p, int method, int kind, int reps) {
  std::vector<LaunchRec> rec;
  ctx->record = &rec;
  Common c;
  c.st = p->st;
  c.cfg.tol = 0.0; c.cfg.maxit = 1; c.cfg.method = method; c.cfg.hist = p->hist; c.cfg.hist_ld = p->hist_cap;
  SolveIO io{p->F0, p->Uscratch, nullptr, method_base(method), false, method_spectral(method),
             method_precond(method)};
  int nl = 0;
  const ad_status s = enqueue_body<T>(ctx, p, nullptr, io, c, &nl);
  ctx->record = nullptr;
  if (s != AD_OK) return -1.0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.0; }
  double total = 0.0;
  bool ok = true;
  for (LaunchRec r : rec) {
    if (r.kind != kind) continue;
    r.af.force = r.ad.force = 1;
    r.af.stage = r.ad.stage = SS_NONE;
    r.af.set_cond = r.ad.set_cond = r.af.clear_cond = r.ad.clear_cond = 0;
    auto go = [&]() { return r.f64 ? launch_pass<double>(r.kind, r.E, r.grid, r.threads, r.smem, nullptr, r.ad)
                                    : launch_pass<float>(r.kind, r.E, r.grid, r.threads, r.smem, nullptr, r.af); };
    cudaError_t e = go();
    if (e == cudaSuccess) e = cudaEventRecord(e0, nullptr);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = go();
    if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { cudaGetLastError(); ok = false; break; }
    total += ms / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ok ? total : -1.0;
}

ad_status autotune_plan(ad_ctx* ctx, Plan* p, int method, int reps) {
  ad_status s;
  if ((s = ensure_vectors(ctx, p)) != AD_OK || (s = ensure_hist(ctx, p, 1)) != AD_OK) return s;
  if (!p->Uscratch && (s = dmalloc(ctx, p, &p->Uscratch, (size_t)p->P * p->batch * (p->f64 ? 8 : 4))) != AD_OK)
    return s;
  if (method_spectral(method)) {
    // spectral space: the passes stream; tune the blocks per field (element
    // pairs per block 512 .. 32768), timing the iteration's spectral passes
    if ((s = ensure_spectral(ctx, p)) != AD_OK) return s;
    const long long pairs = p->SP / 2;
    PassCfg best = p->sp;
    double best_ms = -1.0;
    for (long long per = 512; per <= 32768; per *= 2) {
      long long nb = std::min<long long>((pairs + per - 1) / per, std::min<long long>(4864, p->maxblk));
      nb = std::max<long long>(nb, 1);
      PassCfg trial = p->sp;
      trial.grid.x = (unsigned)nb;
      const PassCfg keep = p->sp;
      p->sp = trial;
      const double ms = p->f64 ? time_kind<double>(ctx, p, method, PK_SPEC, reps)
                               : time_kind<float>(ctx, p, method, PK_SPEC, reps);
      p->sp = keep;
      if (ms > 0.0 && (best_ms < 0.0 || ms < best_ms)) { best_ms = ms; best = trial; }
    }
    p->sp = best;
    CK(cudaDeviceSynchronize());
    drop_graphs(ctx);
    p->sp_tuned = true;
    return AD_OK;
  }
  const int M = p->nx / 2;
  const int Lf = p->ndim == 3 ? p->nz : p->ny;
  std::vector<TileSlot> slots = {{&p->xf, PK_XFWD, M, M + 1, pow2_part(p->ny)},
                                 {&p->xi, PK_XINV, M, M + 1, pow2_part(p->ny)},
                                 {&p->fl, PK_FILT, Lf, Lf, 0}};
  if (p->ndim == 3) {
    slots.push_back({&p->yf, PK_YFWD, p->ny, p->ny, pow2_part(p->nz)});
    slots.push_back({&p->yi, PK_YINV, p->ny, p->ny, pow2_part(p->nz)});
  }
  const size_t cs = p->f64 ? 16 : 8;
  for (TileSlot& sl : slots) {
    PassCfg best = *sl.pc;
    double best_ms = -1.0;
    for (int W = 1; W <= 4096; W *= 2) {
      if (sl.div > 0 && sl.div % W != 0) break;
      const long long tot = (long long)W * sl.L;
      if (tot % sl.pc->E != 0) continue;
      const long long T = tot / sl.pc->E;
      const int ld = tile_ld(sl.slots);
      if (T < 32 || T > 256 || (size_t)W * ld * cs > 100 * 1024) continue;
      PassCfg trial = *sl.pc;
      set_tile(p, trial, sl.kind, sl.L, sl.slots, W);
      if ((sl.kind == PK_XINV || sl.kind == PK_FILT) && trial.grid.x > p->maxblk) continue;
      const PassCfg keep = *sl.pc;
      *sl.pc = trial;
      const double ms = p->f64 ? time_kind<double>(ctx, p, method, sl.kind, reps)
                               : time_kind<float>(ctx, p, method, sl.kind, reps);
      *sl.pc = keep;
      if (ms > 0.0 && (best_ms < 0.0 || ms < best_ms)) { best_ms = ms; best = trial; }
    }
    *sl.pc = best;
  }
  CK(cudaDeviceSynchronize());
  drop_graphs(ctx);                 // cached graphs hold the old launch shapes
  p->tuned = true;
  return AD_OK;
}

// ---------------------------------------------------------------------------
// Learned initial guess (cnn.cu): workspaces and checks.

ad_status check_cnn_grid(ad_ctx* ctx, const ad_grid* g) {
  ad_status s = check_grid(ctx, g);
  if (s != AD_OK) return s;
  if (g->ndim != 3 || g->dtype != AD_F32) return fail(ctx, AD_ERR_ARG, "the learned guess takes 3D float32 fields");
  if (!cnn_shape_ok((int)g->n[0], (int)g->n[1], (int)g->n[2]))
    return fail(ctx, AD_ERR_ARG, "the learned guess needs Nx a multiple of 32");
  return AD_OK;
}

ad_status cnn_alloc(ad_ctx* ctx, CnnWork* cw, void** out, size_t bytes) {
  if (cudaMalloc(out, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, AD_ERR_NOMEM, "learned-guess workspace of " + std::to_string(bytes) + " bytes");
  }
  cw->owned.push_back(*out);
  return AD_OK;
}

// Workspace for (X, Y, Z, B); `training` adds gradients, moments and gathers.
ad_status get_cnn(ad_ctx* ctx, const ad_grid* g, int B, bool training, CnnWork** out) {
  if (B > AD_MAX_BATCH) return fail(ctx, AD_ERR_ARG, "batch > AD_MAX_BATCH");
  char key[128];
  snprintf(key, sizeof key, "%lld:%lld:%lld:%d", (long long)g->n[0], (long long)g->n[1], (long long)g->n[2], B);
  auto it = ctx->cnn.find(key);
  CnnWork* cw = it == ctx->cnn.end() ? nullptr : it->second;
  if (!cw) {
    cw = new CnnWork;
    ctx->cnn[key] = cw;
  }
  const size_t P = (size_t)g->n[0] * g->n[1] * g->n[2];
  const size_t act = sizeof(__nv_bfloat16) * P * 32 * B, frag = sizeof(uint2) * 27 * 2 * 4 * 32;
  ad_status s;
  gad::CnnBuffers& w = cw->w;
  if (!w.master) {
    if ((s = cnn_alloc(ctx, cw, (void**)&w.master, sizeof(float) * kCnnWeights)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.frag2, frag)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.frag3, frag)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.frag2t, frag)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.frag3t, frag)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.frag4, sizeof(uint2) * 27 * 2 * 32)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.H1, act)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.H2, act)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.H3, act)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.sumsq, sizeof(double) * (2 * B + 1))) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.flag, sizeof(int))) != AD_OK)
      return s;
    if (cudaMemset(w.flag, 0, sizeof(int)) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cnn flag");
    if (gad::conv_tc_shape_ok((int)g->n[0], (int)g->n[1], (int)g->n[2])) {
      const size_t ib = gad::conv_tc_image_bytes();
      if ((s = cnn_alloc(ctx, cw, (void**)&w.umma2, ib)) != AD_OK ||
          (s = cnn_alloc(ctx, cw, (void**)&w.umma3, ib)) != AD_OK ||
          (s = cnn_alloc(ctx, cw, (void**)&w.umma2t, ib)) != AD_OK ||
          (s = cnn_alloc(ctx, cw, (void**)&w.umma3t, ib)) != AD_OK)
        return s;
    }
  }
  w.wait_ns = ctx->wait_ns;
  if (training && !w.grad) {
    if ((s = cnn_alloc(ctx, cw, (void**)&w.grad, sizeof(float) * kCnnWeights)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.m, sizeof(float) * kCnnWeights)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.v, sizeof(float) * kCnnWeights)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.dA, act)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.dB, act)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.g, sizeof(float) * P * B)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&w.part, sizeof(float) * (size_t)kCnnPartFloats)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&cw->ub, sizeof(float) * P * B)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&cw->ut, sizeof(float) * P * B)) != AD_OK ||
        (s = cnn_alloc(ctx, cw, (void**)&cw->u0, sizeof(float) * P * B)) != AD_OK)
      return s;
  }
  *out = cw;
  return AD_OK;
}

// Reads back (and clears) the flag the tensor-core convolution sets when one
// of its bounded waits gave up; waits for the stream. AD_ERR_TIMEOUT if set.
ad_status cnn_flag_status(ad_ctx* ctx, CnnWork* cw, cudaStream_t st) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, cw->w.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h) {
    CK(cudaMemsetAsync(cw->w.flag, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    return fail(ctx, AD_ERR_TIMEOUT, "a bounded wait of the tensor-core convolution gave up");
  }
  return AD_OK;
}

// A = (delta/h)^2 = 1/(pi gamma)^2: delta = 1/k_c, k_c = gamma N/2, h = 2 pi/N
double cnn_ascale(double gamma) { return 1.0 / ((3.141592653589793 * gamma) * (3.141592653589793 * gamma)); }

// splitmix64 (Steele, Lea, Flood 2014) and a Box-Muller normal, host side
uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double normal01(uint64_t& st) {
  const double u1 = ((splitmix64(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((splitmix64(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// ---------------------------------------------------------------------------
// Batched solve of fields of uneven size: one CUDA graph whose concurrent
// branches each solve one group of same-shape fields (gathered into the
// group plan's contiguous buffers, solved with their own while node, then
// scattered back).

ad_status ensure_io(ad_ctx* ctx, Plan* p) {
  if (p->Bin) return AD_OK;
  const size_t vb = (size_t)p->P * p->batch * (p->f64 ? 8 : 4);
  ad_status s;
  if ((s = dmalloc(ctx, p, &p->Bin, vb)) != AD_OK || (s = dmalloc(ctx, p, &p->Bout, vb)) != AD_OK) return s;
  return AD_OK;
}

ad_status ensure_streams(ad_ctx* ctx, size_t n) {
  while (ctx->branches.size() < n) {
    cudaStream_t s;
    cudaEvent_t e1, e2;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ctx->branches.push_back(s);
    CK(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
    ctx->events.push_back(e1);
    ctx->events.push_back(e2);
  }
  return AD_OK;
}

template <typename T>
ad_status capture_group(ad_ctx* ctx, BatchedGroup& gr, cudaStream_t s, cudaGraphConditionalHandle h,
                        const void* const* ubar, void* const* u_out, int method, double tol, int maxit) {
  Plan* p = gr.p;
  Common c;
  c.st = p->st;
  c.wait_ns = ctx->wait_ns;
  c.cfg.tol = tol;
  c.cfg.maxit = maxit;
  c.cfg.method = method_base(method);
  c.cfg.hist = p->hist;
  c.cfg.hist_ld = p->hist_cap;
  c.cond = h;
  c.in_graph = true;
  const size_t bytes = (size_t)p->P * sizeof(T);
  for (size_t k = 0; k < gr.fields.size(); ++k)
    CK(cudaMemcpyAsync((char*)p->Bin + k * bytes, ubar[gr.fields[k]], bytes, cudaMemcpyDeviceToDevice, s));
  SolveIO io{p->Bin, p->Bout, nullptr, method_base(method), false, method_spectral(method),
             method_precond(method)};
  ad_status st = enqueue_init<T>(ctx, p, s, io, c, &gr.n_init);
  if (st != AD_OK) return st;
  cudaStreamCaptureStatus cs;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphNode_t cn = nullptr;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  CK(cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &np));
  CK(cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(ctx->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  st = enqueue_body<T>(ctx, p, ctx->cap2, io, c, &gr.n_body);
  cudaGraph_t bg = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->cap2, &bg);
  if (st != AD_OK) return st;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture(batched body)");
  if ((st = enqueue_finish<T>(ctx, p, s, io, c, &gr.n_fin)) != AD_OK) return st;
  for (size_t k = 0; k < gr.fields.size(); ++k)
    CK(cudaMemcpyAsync(u_out[gr.fields[k]], (char*)p->Bout + k * bytes, bytes, cudaMemcpyDeviceToDevice, s));
  return AD_OK;
}

// --- one launch per pass stage over all shape groups -----------------------
// The groups' own pass launches (recorded, not issued) are lined up by stage
// -- the k-th application of G in the sequence, and within it the x, y,
// filter, inverse y and inverse x passes -- and each stage becomes one k_multi
// launch per per-thread element count E over every group's blocks: a device
// work list of (group, field, tile) blocks; groups whose passes have other
// block sizes go to a launch of their own. 2D groups take no part in the y
// stages. The fields' dot reductions and scalar recurrences stay per group;
// the count of finished fields and the loop condition span all groups
// (MultiState).

int stage_slot(int kind) {
  switch (kind) {
    case PK_XFWD: return 0;
    case PK_YFWD: return 1;
    case PK_FILT: return 2;
    case PK_YINV: return 3;
    default: return 4;                 // PK_XINV
  }
}

struct MultiLaunch {
  int kind = 0, E = 0, blocks = 0, threads = 0, ngroups = 0;
  size_t smem = 0;
  const void* args = nullptr;          // device PassArgs<float>[ngroups]
  const int* start = nullptr;          // device int[ngroups + 1]
};

// Lines the groups' recorded launches up by stage and uploads one launch per
// (stage, E, block size). `first_clear`: only the first launch's first group keeps the
// loop-condition reset of the body's first pass.
ad_status merge_multi(ad_ctx* ctx, BatchedEntry& be, std::vector<std::vector<LaunchRec>>& recs, MultiState* ms,
                      bool first_clear, std::vector<MultiLaunch>& out) {
  // stage index of every record: 5 * (application of G) + slot of the pass
  // stage -> (E, block size) -> records: the groups of one launch share the
  // block size too, so every thread does the same work as in the group's own
  // launch and the reductions round identically
  std::map<int, std::map<std::pair<int, int>, std::vector<const LaunchRec*>>> stages;
  for (auto& rl : recs) {
    int app = -1;
    for (const LaunchRec& r : rl) {
      if (r.kind == PK_XFWD) ++app;
      if (r.f64 || r.kind > PK_YINV || app < 0) return fail(ctx, AD_ERR_ARG, "no multi-group launch for this pass");
      stages[5 * app + stage_slot(r.kind)][std::make_pair(r.E, r.threads)].push_back(&r);
    }
  }
  bool cleared = false;
  for (auto& st : stages) {
    for (auto& byE : st.second) {
      const auto& rs = byE.second;
      MultiLaunch m;
      m.kind = rs[0]->kind;
      m.E = byE.first.first;
      m.ngroups = (int)rs.size();
      std::vector<PassArgs<float>> args(rs.size());
      std::vector<int> start(rs.size() + 1, 0);
      for (size_t g = 0; g < rs.size(); ++g) {
        PassArgs<float> a = rs[g]->af;
        a.vgx = (int)rs[g]->grid.x;
        a.vgy = (int)rs[g]->grid.y;
        a.vbd = rs[g]->threads;
        a.ms = ms;
        if (a.clear_cond) {
          a.clear_cond = (first_clear && !cleared) ? 1 : 0;
          cleared = true;
        }
        args[g] = a;
        start[g + 1] = start[g] + (int)(rs[g]->grid.x * rs[g]->grid.y);
        m.threads = std::max(m.threads, rs[g]->threads);
        m.smem = std::max(m.smem, rs[g]->smem);
      }
      m.blocks = start.back();
      void *da = nullptr, *ds = nullptr;
      if (cudaMalloc(&da, sizeof(PassArgs<float>) * args.size()) != cudaSuccess ||
          cudaMalloc(&ds, sizeof(int) * start.size()) != cudaSuccess) {
        cudaGetLastError();
        if (da) cudaFree(da);
        return fail(ctx, AD_ERR_NOMEM, "multi-group launch arrays");
      }
      be.owned.push_back(da);
      be.owned.push_back(ds);
      CK(cudaMemcpy(da, args.data(), sizeof(PassArgs<float>) * args.size(), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(ds, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice));
      m.args = da;
      m.start = (const int*)ds;
      out.push_back(m);
    }
  }
  return AD_OK;
}

cudaError_t issue_multi(const std::vector<MultiLaunch>& ml, cudaStream_t s) {
  for (const MultiLaunch& m : ml) {
    const cudaError_t e = launch_multi<float>(m.kind, m.E, m.blocks, m.threads, m.smem, s,
                                              static_cast<const PassArgs<float>*>(m.args), m.start, m.ngroups);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Float32 physical-space Van Cittert, SD, CG and BiCGSTAB without a
// preconditioner (the other variants keep one graph branch per group).
bool multi_eligible(const BatchedEntry& be, int method) {
  if (method_spectral(method) || method_precond(method) || be.groups.size() < 2) return false;
  for (const BatchedGroup& gr : be.groups)
    if (gr.p->f64) return false;
  return true;
}

ad_status build_batched_multi(ad_ctx* ctx, BatchedEntry& be, const void* const* ubar, void* const* u_out, int method,
                              double tol, int maxit) {
  const size_t G = be.groups.size();
  // MultiState: counters, and every group's field states
  MultiState hms{};
  hms.ngroups = (int)G;
  std::vector<FieldState*> sts(G);
  std::vector<int> cnt(G);
  for (size_t j = 0; j < G; ++j) {
    sts[j] = be.groups[j].p->st;
    cnt[j] = (int)be.groups[j].fields.size();
    hms.nfields += cnt[j];
  }
  void *dms = nullptr, *dst = nullptr, *dcnt = nullptr;
  if (cudaMalloc(&dms, sizeof(MultiState)) != cudaSuccess || cudaMalloc(&dst, sizeof(FieldState*) * G) != cudaSuccess ||
      cudaMalloc(&dcnt, sizeof(int) * G) != cudaSuccess) {
    cudaGetLastError();
    if (dms) cudaFree(dms);
    if (dst) cudaFree(dst);
    return fail(ctx, AD_ERR_NOMEM, "multi-group state");
  }
  be.owned.push_back(dms);
  be.owned.push_back(dst);
  be.owned.push_back(dcnt);
  hms.st = (FieldState**)dst;
  hms.count = (int*)dcnt;
  CK(cudaMemcpy(dst, sts.data(), sizeof(FieldState*) * G, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dcnt, cnt.data(), sizeof(int) * G, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dms, &hms, sizeof(MultiState), cudaMemcpyHostToDevice));
  MultiState* ms = (MultiState*)dms;

  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ctx, e, "cudaGraphConditionalHandleCreate"); }
  // record every group's init and body launches
  std::vector<std::vector<LaunchRec>> rinit(G), rbody(G);
  ad_status st = AD_OK;
  for (size_t j = 0; j < G && st == AD_OK; ++j) {
    Plan* p = be.groups[j].p;
    Common c;
    c.st = p->st;
    c.wait_ns = ctx->wait_ns;
    c.cfg.tol = tol;
    c.cfg.maxit = maxit;
    c.cfg.method = method_base(method);
    c.cfg.hist = p->hist;
    c.cfg.hist_ld = p->hist_cap;
    c.cond = h;
    c.in_graph = true;
    SolveIO io{p->Bin, p->Bout, nullptr, method_base(method), false, false, false};
    int n = 0;
    ctx->record = &rinit[j];
    st = enqueue_init_passes<float>(ctx, p, nullptr, io, c, &n);
    if (st == AD_OK) {
      ctx->record = &rbody[j];
      st = enqueue_body<float>(ctx, p, nullptr, io, c, &n);
    }
    ctx->record = nullptr;
  }
  std::vector<MultiLaunch> minit, mbody;
  if (st == AD_OK) st = merge_multi(ctx, be, rinit, ms, false, minit);
  if (st == AD_OK) st = merge_multi(ctx, be, rbody, ms, true, mbody);
  if (st != AD_OK) { cudaGraphDestroy(g); return st; }
  e = cudaStreamBeginCaptureToGraph(ctx->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ctx, e, "cudaStreamBeginCaptureToGraph"); }
  // gather, reset the states, the initial residual of every field
  for (size_t j = 0; j < G && st == AD_OK; ++j) {
    const BatchedGroup& gr = be.groups[j];
    const size_t bytes = (size_t)gr.p->P * sizeof(float);
    for (size_t k = 0; k < gr.fields.size() && e == cudaSuccess; ++k)
      e = cudaMemcpyAsync((char*)gr.p->Bin + k * bytes, ubar[gr.fields[k]], bytes, cudaMemcpyDeviceToDevice, ctx->cap);
    if (e == cudaSuccess) e = launch_reset_state(gr.p->st, (int)gr.fields.size(), ctx->cap);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "multi-group gather");
  }
  if (st == AD_OK && (e = issue_multi(minit, ctx->cap)) != cudaSuccess) st = cuda_fail(ctx, e, "multi-group init");
  if (st == AD_OK) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphNode_t cn = nullptr;
    cudaGraphNodeParams np{};
    e = cudaStreamGetCaptureInfo(ctx->cap, &cs, nullptr, &cg, &deps, nullptr, &nd);
    if (e == cudaSuccess) {
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      e = cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &np);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(ctx->cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(ctx->cap2, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t eb = issue_multi(mbody, ctx->cap2);
      cudaGraph_t bg = nullptr;
      e = cudaStreamEndCapture(ctx->cap2, &bg);
      if (eb != cudaSuccess) e = eb;
    }
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "multi-group loop body");
  }
  // finish (CG's deferred update) and scatter, per group
  int nfin = 0;
  for (size_t j = 0; j < G && st == AD_OK; ++j) {
    const BatchedGroup& gr = be.groups[j];
    Common c;
    c.st = gr.p->st;
    c.wait_ns = ctx->wait_ns;
    SolveIO io{gr.p->Bin, gr.p->Bout, nullptr, method_base(method), false, false, false};
    st = enqueue_finish<float>(ctx, gr.p, ctx->cap, io, c, &nfin);
    const size_t bytes = (size_t)gr.p->P * sizeof(float);
    for (size_t k = 0; k < gr.fields.size() && st == AD_OK; ++k)
      if (cudaMemcpyAsync(u_out[gr.fields[k]], (char*)gr.p->Bout + k * bytes, bytes, cudaMemcpyDeviceToDevice,
                          ctx->cap) != cudaSuccess)
        st = cuda_fail(ctx, cudaGetLastError(), "multi-group scatter");
  }
  cudaGraph_t gout = nullptr;
  e = cudaStreamEndCapture(ctx->cap, &gout);
  if (st == AD_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "cudaStreamEndCapture(multi-group)");
  if (st != AD_OK) { cudaGetLastError(); cudaGraphDestroy(g); return st; }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ctx, e, "cudaGraphInstantiate(multi-group)"); }
  be.g = g;
  be.exec = exec;
  be.multi = true;
  be.m_init = (int)minit.size() + (int)G;
  be.m_body = (int)mbody.size();
  be.m_fin = nfin;
  return AD_OK;
}

ad_status build_batched(ad_ctx* ctx, BatchedEntry& be, const void* const* ubar, void* const* u_out, int method,
                        double tol, int maxit) {
  if (ctx->batched_multi && multi_eligible(be, method)) return build_batched_multi(ctx, be, ubar, u_out, method, tol, maxit);
  const size_t G = be.groups.size();
  ad_status st = ensure_streams(ctx, G);
  if (st != AD_OK) return st;
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  std::vector<cudaGraphConditionalHandle> hs(G);
  for (size_t i = 0; i < G; ++i) {
    cudaError_t e = cudaGraphConditionalHandleCreate(&hs[i], g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ctx, e, "cudaGraphConditionalHandleCreate"); }
  }
  cudaError_t e = cudaStreamBeginCaptureToGraph(ctx->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ctx, e, "cudaStreamBeginCaptureToGraph"); }
  e = cudaEventRecord(ctx->events[0], ctx->cap);
  if (e != cudaSuccess) st = cuda_fail(ctx, e, "fork event");
  for (size_t i = 0; i < G && st == AD_OK; ++i) {
    cudaStream_t bs = ctx->branches[i];
    e = cudaStreamWaitEvent(bs, ctx->events[0], 0);
    if (e != cudaSuccess) { st = cuda_fail(ctx, e, "branch fork"); break; }
    BatchedGroup& gr = be.groups[i];
    st = gr.p->f64 ? capture_group<double>(ctx, gr, bs, hs[i], ubar, u_out, method, tol, maxit)
                   : capture_group<float>(ctx, gr, bs, hs[i], ubar, u_out, method, tol, maxit);
    if (st != AD_OK) break;
    e = cudaEventRecord(ctx->events[2 * i + 1], bs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap, ctx->events[2 * i + 1], 0);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "branch join");
  }
  cudaGraph_t gout = nullptr;
  e = cudaStreamEndCapture(ctx->cap, &gout);
  if (st == AD_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "cudaStreamEndCapture(batched)");
  if (st != AD_OK) { cudaGetLastError(); cudaGraphDestroy(g); return st; }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ctx, e, "cudaGraphInstantiate(batched)"); }
  be.g = g;
  be.exec = exec;
  return AD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

ad_status ad_create(ad_ctx** out, int device) {
  if (!out) return AD_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return AD_ERR_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) return AD_ERR_CUDA;
  ad_ctx* c = new ad_ctx;
  c->device = device;
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return AD_ERR_CUDA;
  }
  *out = c;
  return AD_OK;
}

void ad_destroy(ad_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  drop_graphs(c);
  for (auto& kv : c->plans) free_plan(kv.second);
  for (auto& kv : c->cnn) {
    for (void* q : kv.second->owned) cudaFree(q);
    delete kv.second;
  }
  for (auto& kv : c->tw) cudaFree(kv.second);
  for (auto s : c->branches) cudaStreamDestroy(s);
  for (auto e : c->events) cudaEventDestroy(e);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->cap2) cudaStreamDestroy(c->cap2);
  if (c->stat_buf) cudaFree(c->stat_buf);
  delete c;
}

ad_status ad_time_pass(ad_ctx* ctx, const ad_grid* grid, int batch, ad_method method, int index, int reps,
                       void* stream, double* ms_per_launch, int* kind, int* op, int* count) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (batch < 1 || reps < 1 || !method_ok(method)) return fail(ctx, AD_ERR_ARG, "bad batch, reps or method");
  CK(cudaSetDevice(ctx->device));
  Plan* p = nullptr;
  if ((s = get_plan(ctx, grid, batch, &p)) != AD_OK) return s;
  if ((s = ensure_vectors(ctx, p)) != AD_OK) return s;
  if ((s = ensure_hist(ctx, p, 1)) != AD_OK) return s;
  if (!p->Uscratch && (s = dmalloc(ctx, p, &p->Uscratch, (size_t)p->P * p->batch * (p->f64 ? 8 : 4))) != AD_OK) return s;
  if (method_spectral(method) && (s = ensure_spectral(ctx, p)) != AD_OK) return s;
  // record one iteration body on internal buffers only
  std::vector<LaunchRec> rec;
  ctx->record = &rec;
  Common c;
  c.st = p->st;
  c.cfg.tol = 0.0; c.cfg.maxit = 1; c.cfg.method = method_base(method); c.cfg.hist = p->hist;
  c.cfg.hist_ld = p->hist_cap;
  SolveIO io{p->F0, p->Uscratch, nullptr, method_base(method), false, method_spectral(method),
             method_precond(method)};
  int nl = 0;
  s = p->f64 ? enqueue_body<double>(ctx, p, nullptr, io, c, &nl) : enqueue_body<float>(ctx, p, nullptr, io, c, &nl);
  ctx->record = nullptr;
  if (s != AD_OK) return s;
  if (count) *count = (int)rec.size();
  if (index == -1) return AD_OK;
  if (index < -2 || index >= (int)rec.size()) return fail(ctx, AD_ERR_ARG, "pass index out of range");
  // every field computes, no scalar update, no graph condition
  for (LaunchRec& q : rec) {
    q.af.force = q.ad.force = 1;
    q.af.stage = q.ad.stage = SS_NONE;
    q.af.set_cond = q.ad.set_cond = 0;
    q.af.clear_cond = q.ad.clear_cond = 0;
  }
  // index -2: the whole body, its launches in order
  const size_t first = index == -2 ? 0 : (size_t)index, last = index == -2 ? rec.size() : (size_t)index + 1;
  const LaunchRec& r = rec[first];
  if (kind) *kind = index == -2 ? -1 : r.kind;
  if (op) *op = index == -2 ? -1 : (r.f64 ? r.ad.op : r.af.op);
  cudaStream_t st = (cudaStream_t)stream;
  // a mid-solve state (pass 1, finite scalars), so that passes whose first
  // iteration skips work (p = r, no u update) are timed in their full form
  {
    std::vector<FieldState> hs(p->batch);
    for (auto& f : hs) {
      f = FieldState{};
      f.rho = 1.0; f.alpha = 0.5; f.beta = 0.25; f.omega = 0.5; f.ref = 1.0; f.h = 1.0;
      f.iter = 1; f.active = 1;
    }
    CK(cudaMemcpyAsync(p->st, hs.data(), sizeof(FieldState) * p->batch, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto go = [&]() {
    cudaError_t err = cudaSuccess;
    for (size_t i = first; i < last && err == cudaSuccess; ++i) {
      const LaunchRec& q = rec[i];
      err = q.f64 ? launch_pass<double>(q.kind, q.E, q.grid, q.threads, q.smem, st, q.ad)
                  : launch_pass<float>(q.kind, q.E, q.grid, q.threads, q.smem, st, q.af);
    }
    return err;
  };
  cudaError_t e = go();                              // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = go();
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ad_time_pass");
  if (ms_per_launch) *ms_per_launch = (double)ms / reps;
  ctx->launches = (long long)(reps + 1) * (long long)(last - first);
  return AD_OK;
}

ad_status ad_deconvolve_batched(ad_ctx* ctx, int nfields, const ad_grid* grids, const void* const* ubar,
                                void* const* u_out, ad_method method, double tol, int maxit, int* iterations,
                                ad_status* status, double* const* res_hist, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  if (nfields < 0) return fail(ctx, AD_ERR_ARG, "nfields < 0");
  if (nfields == 0) { ctx->launches = 0; return AD_OK; }
  if (!grids || !ubar || !u_out) return fail(ctx, AD_ERR_ARG, "NULL array argument");
  if (!method_ok(method)) return fail(ctx, AD_ERR_ARG, "unknown method");
  if (maxit < 0 || !(tol >= 0.0) || !std::isfinite(tol)) return fail(ctx, AD_ERR_ARG, "need maxit >= 0 and finite tol >= 0");
  ad_status s;
  for (int i = 0; i < nfields; ++i) {
    if ((s = check_grid(ctx, &grids[i])) != AD_OK) return s;
    if (!ubar[i] || !u_out[i]) return fail(ctx, AD_ERR_ARG, "NULL field pointer");
    if (ubar[i] == u_out[i]) return fail(ctx, AD_ERR_ARG, "u_out must not alias ubar");
    if (((uintptr_t)ubar[i] | (uintptr_t)u_out[i]) & 15) return fail(ctx, AD_ERR_ARG, "field pointers must be 16-byte aligned");
  }
  CK(cudaSetDevice(ctx->device));
  // group by shape (order of first appearance), one plan per group
  std::vector<std::string> keys;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < nfields; ++i) {
    const std::string k = plan_key(&grids[i], 0);
    size_t j = 0;
    while (j < keys.size() && keys[j] != k) ++j;
    if (j == keys.size()) { keys.push_back(k); members.emplace_back(); }
    members[j].push_back(i);
  }
  std::string bkey = "B|";
  char buf[128];
  snprintf(buf, sizeof buf, "%d|%a|%d|", (int)method, tol, maxit);
  bkey += buf;
  std::vector<BatchedGroup> groups(keys.size());
  for (size_t j = 0; j < keys.size(); ++j) {
    Plan* p = nullptr;
    if ((s = get_plan(ctx, &grids[members[j][0]], (int)members[j].size(), &p)) != AD_OK) return s;
    if ((s = ensure_vectors(ctx, p)) != AD_OK || (s = ensure_io(ctx, p)) != AD_OK) return s;
    if (method_spectral(method) && (s = ensure_spectral(ctx, p)) != AD_OK) return s;
    const bool tuned = method_spectral(method) ? p->sp_tuned : p->tuned;
    if (ctx->autotune && !tuned && (s = autotune_plan(ctx, p, (int)method, 10)) != AD_OK) return s;
    groups[j].p = p;
    groups[j].fields = members[j];
  }
  // history buffers (may drop cached graphs): size every group first
  for (auto& gr : groups)
    if ((s = ensure_hist(ctx, gr.p, maxit)) != AD_OK) return s;
  for (size_t j = 0; j < groups.size(); ++j) {
    snprintf(buf, sizeof buf, "%p:", (void*)groups[j].p);
    bkey += buf;
    for (int f : groups[j].fields) {
      snprintf(buf, sizeof buf, "%p>%p,", ubar[f], u_out[f]);
      bkey += buf;
    }
  }
  auto it = ctx->bgraphs.find(bkey);
  if (it == ctx->bgraphs.end()) {
    BatchedEntry be;
    be.groups = groups;
    if ((s = build_batched(ctx, be, ubar, u_out, (int)method, tol, maxit)) != AD_OK) return s;
    it = ctx->bgraphs.emplace(bkey, be).first;
  }
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaGraphLaunch(it->second.exec, st));
  std::vector<std::vector<FieldState>> hs(it->second.groups.size());
  for (size_t j = 0; j < it->second.groups.size(); ++j) {
    const BatchedGroup& gr = it->second.groups[j];
    hs[j].resize(gr.fields.size());
    CK(cudaMemcpyAsync(hs[j].data(), gr.p->st, sizeof(FieldState) * gr.fields.size(), cudaMemcpyDeviceToHost, st));
    if (res_hist)
      for (size_t k = 0; k < gr.fields.size(); ++k)
        if (res_hist[gr.fields[k]])
          CK(cudaMemcpyAsync(res_hist[gr.fields[k]], gr.p->hist + k * (size_t)gr.p->hist_cap,
                             sizeof(double) * (size_t)(maxit + 1), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  ad_status worst = AD_OK;
  int64_t launches = 0;
  int maxpass_all = 0;
  for (size_t j = 0; j < it->second.groups.size(); ++j) {
    const BatchedGroup& gr = it->second.groups[j];
    int maxpass = 0;
    for (size_t k = 0; k < gr.fields.size(); ++k) {
      const FieldState& f = hs[j][k];
      const int i = gr.fields[k];
      if (iterations) iterations[i] = f.iter;
      if (status) status[i] = (ad_status)f.status;
      if (worst == AD_OK && f.status != AD_OK) worst = (ad_status)f.status;
      maxpass = std::max(maxpass, f.iter + (f.status == AD_BREAKDOWN ? 1 : 0));
    }
    launches += gr.n_init + gr.n_fin + (int64_t)std::max(1, maxpass) * gr.n_body;
    maxpass_all = std::max(maxpass_all, maxpass);
  }
  if (it->second.multi)
    launches = it->second.m_init + it->second.m_fin + (int64_t)std::max(1, maxpass_all) * it->second.m_body;
  ctx->launches = launches;
  return worst;
}

ad_status ad_autotune(ad_ctx* ctx, const ad_grid* grid, int batch, ad_method method, int enable_for_batched) {
  if (!ctx) return AD_ERR_ARG;
  ctx->autotune = enable_for_batched != 0;
  if (!grid) return AD_OK;
  ad_status s = check_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (batch < 1 || !method_ok(method)) return fail(ctx, AD_ERR_ARG, "bad batch or method");
  CK(cudaSetDevice(ctx->device));
  Plan* p = nullptr;
  if ((s = get_plan(ctx, grid, batch, &p)) != AD_OK) return s;
  return autotune_plan(ctx, p, (int)method, 10);
}

int64_t ad_guess_weight_count(void) { return kCnnWeights; }

ad_status ad_guess_init(float* w, int64_t n, uint64_t seed, int stencil) {
  if (!w || n != kCnnWeights) return AD_ERR_ARG;
  uint64_t st = seed;
  const int fan_in[4] = {27, 27 * 32, 27 * 32, 27 * 32};
  const int off[5] = {kW1, kW2, kW3, kW4, kCnnWeights};
  for (int l = 0; l < 4; ++l) {
    double std_ = std::sqrt(2.0 / fan_in[l]);
    if (stencil) std_ *= 1e-3;
    else if (l == 3) std_ *= 0.1;
    for (int i = off[l]; i < off[l + 1]; ++i) w[i] = (float)(std_ * normal01(st));
  }
  if (stencil) {
    // the explicit inverse u0 = u_bar - (delta/h)^2 L_h u_bar with the 7-point
    // Laplacian L_h: layer 1 forms +L and -L (channels 0, 1), layers 2-3 pass
    // them on, layer 4 takes -(relu(L) - relu(-L)) = -L (the output scale is A)
    const int centre = 13;
    const int faces[6] = {4, 22, 10, 16, 12, 14};       // z-1, z+1, y-1, y+1, x-1, x+1
    for (int t = 0; t < 27; ++t) w[kW1 + t * 32 + 0] = w[kW1 + t * 32 + 1] = 0.f;
    w[kW1 + centre * 32 + 0] = -6.f;
    w[kW1 + centre * 32 + 1] = 6.f;
    for (int f : faces) {
      w[kW1 + f * 32 + 0] = 1.f;
      w[kW1 + f * 32 + 1] = -1.f;
    }
    for (int l : {kW2, kW3})             // channels 0, 1 receive only themselves (centre tap)
      for (int t = 0; t < 27; ++t)
        for (int ci = 0; ci < 32; ++ci)
          for (int co = 0; co < 2; ++co) w[l + (t * 32 + ci) * 32 + co] = (t == centre && ci == co) ? 1.f : 0.f;
    for (int t = 0; t < 27; ++t) w[kW4 + t * 32 + 0] = w[kW4 + t * 32 + 1] = 0.f;
    w[kW4 + centre * 32 + 0] = -1.f;
    w[kW4 + centre * 32 + 1] = 1.f;
  }
  return AD_OK;
}

ad_status ad_guess_infer(ad_ctx* ctx, const ad_grid* grid, const float* weights, const float* ubar, float* u0,
                         int batch, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_cnn_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (batch < 0) return fail(ctx, AD_ERR_ARG, "batch < 0");
  if (batch == 0) return AD_OK;
  if (!weights || !ubar || !u0) return fail(ctx, AD_ERR_ARG, "NULL pointer");
  CK(cudaSetDevice(ctx->device));
  CnnWork* cw = nullptr;
  if ((s = get_cnn(ctx, grid, batch, false, &cw)) != AD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(cw->w.master, weights, sizeof(float) * kCnnWeights, cudaMemcpyDeviceToDevice, st));
  CK(cnn_pack(cw->w, st));
  CK(cnn_forward(cw->w, ubar, u0, nullptr, (int)grid->n[0], (int)grid->n[1], (int)grid->n[2], batch,
                 cnn_ascale(grid->gamma), st));
  ctx->launches = 5 + 5 + 1 + (cw->w.umma2 ? 4 : 0);
  // the tensor-core path reports a bounded wait that gave up
  if (cw->w.umma2) return cnn_flag_status(ctx, cw, st);
  return AD_OK;
}

ad_status ad_guess_time_conv(ad_ctx* ctx, const ad_grid* grid, int batch, int reps, void* stream, double* ms,
                             int* tensor_cores) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_cnn_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (batch < 1 || reps < 1) return fail(ctx, AD_ERR_ARG, "need batch >= 1 and reps >= 1");
  CK(cudaSetDevice(ctx->device));
  CnnWork* cw = nullptr;
  if ((s = get_cnn(ctx, grid, batch, false, &cw)) != AD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int X = (int)grid->n[0], Y = (int)grid->n[1], Z = (int)grid->n[2];
  const size_t act = sizeof(__nv_bfloat16) * (size_t)X * Y * Z * 32 * batch;
  // defined inputs: zero weights and activations (the timing does not depend on the values)
  CK(cudaMemsetAsync(cw->w.master, 0, sizeof(float) * kCnnWeights, st));
  CK(cudaMemsetAsync(cw->w.H1, 0, act, st));
  CK(cnn_pack(cw->w, st));
  bool tc = false;
  CK(cnn_conv_layer(cw->w, X, Y, Z, batch, st, &tc));          // warm-up
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = cudaEventRecord(e0, st);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = cnn_conv_layer(cw->w, X, Y, Z, batch, st, nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ad_guess_time_conv");
  if (ms) *ms = (double)t / reps;
  if (tensor_cores) *tensor_cores = tc ? 1 : 0;
  ctx->launches = reps + 1;
  if (tc) return cnn_flag_status(ctx, cw, st);
  return AD_OK;
}

ad_status ad_guess_grad(ad_ctx* ctx, const ad_grid* grid, const float* weights, const float* ubar, const float* utrue,
                        int batch, float* grad, double* loss, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_cnn_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (batch < 1 || !weights || !ubar || !utrue || !grad) return fail(ctx, AD_ERR_ARG, "bad batch or NULL pointer");
  CK(cudaSetDevice(ctx->device));
  CnnWork* cw = nullptr;
  if ((s = get_cnn(ctx, grid, batch, true, &cw)) != AD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int X = (int)grid->n[0], Y = (int)grid->n[1], Z = (int)grid->n[2];
  CK(cudaMemcpyAsync(cw->w.master, weights, sizeof(float) * kCnnWeights, cudaMemcpyDeviceToDevice, st));
  CK(cnn_pack(cw->w, st));
  CK(cnn_forward(cw->w, ubar, cw->u0, utrue, X, Y, Z, batch, cnn_ascale(grid->gamma), st));
  CK(cnn_backward(cw->w, ubar, X, Y, Z, batch, st));
  CK(cudaMemcpyAsync(grad, cw->w.grad, sizeof(float) * kCnnWeights, cudaMemcpyDeviceToDevice, st));
  double l = 0.0;
  CK(cudaMemcpyAsync(&l, cw->w.sumsq + 2 * batch, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  return cnn_flag_status(ctx, cw, st);
}

ad_status ad_guess_train(ad_ctx* ctx, const ad_grid* grid, int npairs, const float* ubar, const float* utrue,
                         int epochs, int batch, double lr, uint64_t seed, float* weights, double* loss_hist,
                         void* stream) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_cnn_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (npairs < 1 || batch < 1 || batch > npairs || epochs < 0 || !(lr > 0.0) || !ubar || !utrue || !weights)
    return fail(ctx, AD_ERR_ARG, "bad training arguments");
  CK(cudaSetDevice(ctx->device));
  CnnWork* cw = nullptr;
  if ((s = get_cnn(ctx, grid, batch, true, &cw)) != AD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int X = (int)grid->n[0], Y = (int)grid->n[1], Z = (int)grid->n[2];
  const size_t P = (size_t)X * Y * Z;
  const int nmb = npairs / batch;
  if (cw->nloss < nmb) {
    if (cw->losses) cudaFree(cw->losses);
    for (auto& q : cw->owned) if (q == cw->losses) q = nullptr;
    cw->losses = nullptr;
    if ((s = cnn_alloc(ctx, cw, (void**)&cw->losses, sizeof(double) * nmb)) != AD_OK) return s;
    cw->nloss = nmb;
  }
  CK(cudaMemcpyAsync(cw->w.master, weights, sizeof(float) * kCnnWeights, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(cw->w.m, 0, sizeof(float) * kCnnWeights, st));
  CK(cudaMemsetAsync(cw->w.v, 0, sizeof(float) * kCnnWeights, st));
  std::vector<int> order(npairs);
  for (int i = 0; i < npairs; ++i) order[i] = i;
  uint64_t rs = seed;
  std::vector<double> lh(nmb);
  int step = 0;
  int64_t launches = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = npairs - 1; i > 0; --i) std::swap(order[i], order[(int)(splitmix64(rs) % (uint64_t)(i + 1))]);
    for (int mb = 0; mb < nmb; ++mb) {
      for (int k = 0; k < batch; ++k) {
        const size_t src = (size_t)order[mb * batch + k] * P;
        CK(cudaMemcpyAsync(cw->ub + k * P, ubar + src, sizeof(float) * P, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(cw->ut + k * P, utrue + src, sizeof(float) * P, cudaMemcpyDeviceToDevice, st));
      }
      CK(cnn_pack(cw->w, st));
      CK(cnn_forward(cw->w, cw->ub, cw->u0, cw->ut, X, Y, Z, batch, cnn_ascale(grid->gamma), st));
      CK(cnn_backward(cw->w, cw->ub, X, Y, Z, batch, st));
      CK(cnn_adam(cw->w, ++step, (float)lr, st));
      CK(cudaMemcpyAsync(cw->losses + mb, cw->w.sumsq + 2 * batch, sizeof(double), cudaMemcpyDeviceToDevice, st));
      launches += 4 + 6 + 11 + 1;
    }
    if (loss_hist) {
      CK(cudaMemcpyAsync(lh.data(), cw->losses, sizeof(double) * nmb, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      double m = 0.0;
      for (double v : lh) m += v;
      loss_hist[ep] = m / nmb;
    }
  }
  CK(cudaMemcpyAsync(weights, cw->w.master, sizeof(float) * kCnnWeights, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  ctx->launches = launches;
  return cnn_flag_status(ctx, cw, st);
}

ad_status ad_set_graph_mode(ad_ctx* c, int enable) {
  if (!c) return AD_ERR_ARG;
  c->use_graph = enable != 0;
  return AD_OK;
}

ad_status ad_set_batched_launch(ad_ctx* ctx, int one_launch_per_stage) {
  if (!ctx) return AD_ERR_ARG;
  const bool m = one_launch_per_stage != 0;
  if (m != ctx->batched_multi) {
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    drop_graphs(ctx);
  }
  ctx->batched_multi = m;
  return AD_OK;
}

int64_t ad_last_launch_count(const ad_ctx* c) { return c ? c->launches : 0; }

const char* ad_last_error(const ad_ctx* c) { return c ? c->err.c_str() : "no context"; }

const char* ad_status_str(ad_status s) {
  switch (s) {
    case AD_OK: return "converged";
    case AD_MAXIT: return "maximum number of passes reached";
    case AD_BREAKDOWN: return "Krylov breakdown (a scalar vanished or is not finite)";
    case AD_ERR_ARG: return "invalid argument";
    case AD_ERR_NONFINITE: return "initial residual is not finite";
    case AD_ERR_CUDA: return "CUDA runtime error";
    case AD_ERR_TIMEOUT: return "bounded device wait timed out";
    case AD_ERR_NOMEM: return "device allocation failed";
  }
  return "unknown status";
}

ad_status ad_filter(ad_ctx* ctx, const ad_grid* grid, const void* in, void* out, int batch, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (batch < 0) return fail(ctx, AD_ERR_ARG, "batch < 0");
  if (batch == 0) { ctx->launches = 0; return AD_OK; }
  if (!in || !out) return fail(ctx, AD_ERR_ARG, "NULL field pointer");
  if (((uintptr_t)in | (uintptr_t)out) & 15) return fail(ctx, AD_ERR_ARG, "field pointers must be 16-byte aligned");
  CK(cudaSetDevice(ctx->device));
  Plan* p = nullptr;
  if ((s = get_plan(ctx, grid, batch, &p)) != AD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  Common c;
  Fwd fw; fw.A = in;
  Inv iv; iv.op = XI_STORE; iv.O1 = out;
  int nl = 0;
  s = p->f64 ? enqueue_G<double>(ctx, p, st, fw, Flt{}, iv, c, &nl) : enqueue_G<float>(ctx, p, st, fw, Flt{}, iv, c, &nl);
  ctx->launches = nl;
  return s;
}

ad_status ad_deconvolve(ad_ctx* ctx, const ad_grid* grid, const void* ubar, void* u_out, int batch,
                        ad_method method, double tol, int maxit, const void* u0, int* iterations,
                        ad_status* status, double* res_hist, double* true_res, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (batch < 0) return fail(ctx, AD_ERR_ARG, "batch < 0");
  if (!method_ok(method)) return fail(ctx, AD_ERR_ARG, "unknown method");
  if (maxit < 0 || !(tol >= 0.0) || !std::isfinite(tol)) return fail(ctx, AD_ERR_ARG, "need maxit >= 0 and finite tol >= 0");
  if (batch == 0) { ctx->launches = 0; return AD_OK; }
  if (!ubar || !u_out) return fail(ctx, AD_ERR_ARG, "NULL field pointer");
  if (ubar == u_out) return fail(ctx, AD_ERR_ARG, "u_out must not alias ubar");
  if (((uintptr_t)ubar | (uintptr_t)u_out | (uintptr_t)u0) & 15)
    return fail(ctx, AD_ERR_ARG, "field pointers must be 16-byte aligned");
  CK(cudaSetDevice(ctx->device));
  Plan* p = nullptr;
  if ((s = get_plan(ctx, grid, batch, &p)) != AD_OK) return s;
  if ((s = ensure_vectors(ctx, p)) != AD_OK) return s;
  if ((s = ensure_hist(ctx, p, maxit)) != AD_OK) return s;
  if (method_spectral(method) && (s = ensure_spectral(ctx, p)) != AD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  SolveIO io{ubar, u_out, u0, method_base(method), true_res != nullptr, method_spectral(method),
             method_precond(method)};
  int loops = 0, n_body = 0;
  s = p->f64 ? run_solve<double>(ctx, p, io, tol, maxit, st, &loops, &n_body)
             : run_solve<float>(ctx, p, io, tol, maxit, st, &loops, &n_body);
  if (s != AD_OK) return s;
  std::vector<FieldState> hs(batch);
  CK(cudaMemcpyAsync(hs.data(), p->st, sizeof(FieldState) * batch, cudaMemcpyDeviceToHost, st));
  if (res_hist) {
    CK(cudaMemcpy2DAsync(res_hist, sizeof(double) * (size_t)(maxit + 1), p->hist, sizeof(double) * (size_t)p->hist_cap,
                         sizeof(double) * (size_t)(maxit + 1), batch, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  ad_status worst = AD_OK;
  int maxpass = 0;
  for (int b = 0; b < batch; ++b) {
    const FieldState& f = hs[b];
    if (iterations) iterations[b] = f.iter;
    if (status) status[b] = (ad_status)f.status;
    if (true_res) true_res[b] = f.true_res;
    if (worst == AD_OK && f.status != AD_OK) worst = (ad_status)f.status;
    maxpass = std::max(maxpass, f.iter + (f.status == AD_BREAKDOWN ? 1 : 0));
  }
  if (loops < 0) ctx->launches += (int64_t)std::max(1, maxpass) * n_body;   // graph: body ran max(1, passes) times
  return worst;
}

ad_status ad_deconvolve_host(ad_ctx* ctx, const ad_grid* grid, const void* ubar, void* u_out, int batch,
                             ad_method method, double tol, int maxit, int* iterations, ad_status* status,
                             double* res_hist, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (batch < 0) return fail(ctx, AD_ERR_ARG, "batch < 0");
  if (!method_ok(method)) return fail(ctx, AD_ERR_ARG, "unknown method");
  if (maxit < 0 || !(tol >= 0.0) || !std::isfinite(tol)) return fail(ctx, AD_ERR_ARG, "need maxit >= 0 and finite tol >= 0");
  if (batch == 0) { ctx->launches = 0; return AD_OK; }
  if (!ubar || !u_out) return fail(ctx, AD_ERR_ARG, "NULL field pointer");
  CK(cudaSetDevice(ctx->device));
  Plan* p = nullptr;
  if ((s = get_plan(ctx, grid, batch, &p)) != AD_OK || (s = ensure_io(ctx, p)) != AD_OK) return s;
  const size_t bytes = (size_t)p->P * batch * (p->f64 ? 8 : 4);
  cudaStream_t st = (cudaStream_t)stream;
  // staged through the plan's own device buffers, so the solve's graph is the same on every call
  CK(cudaMemcpyAsync(p->Bin, ubar, bytes, cudaMemcpyHostToDevice, st));
  s = ad_deconvolve(ctx, grid, p->Bin, p->Bout, batch, method, tol, maxit, nullptr, iterations, status, res_hist,
                    nullptr, stream);
  if (s == AD_ERR_ARG || s == AD_ERR_CUDA || s == AD_ERR_NOMEM) return s;   // the solve did not run
  CK(cudaMemcpyAsync(u_out, p->Bout, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return s;
}

// ---------------------------------------------------------------------------
// Closure and statistics of deconvolved fields.

namespace {

ad_status stat_scratch(ad_ctx* ctx, size_t bytes, void** out) {
  if (bytes > ctx->stat_cap) {
    if (ctx->stat_buf) cudaFree(ctx->stat_buf);
    ctx->stat_buf = nullptr;
    ctx->stat_cap = 0;
    if (cudaMalloc(&ctx->stat_buf, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, AD_ERR_NOMEM, "statistics scratch of " + std::to_string(bytes) + " bytes");
    }
    ctx->stat_cap = bytes;
  }
  *out = ctx->stat_buf;
  return AD_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

}  // namespace

ad_status ad_set_wait_limit(ad_ctx* ctx, uint64_t ns) {
  if (!ctx) return AD_ERR_ARG;
  if (ns == ctx->wait_ns) return AD_OK;
  CK(cudaSetDevice(ctx->device));
  CK(cudaDeviceSynchronize());
  drop_graphs(ctx);               // cached graphs hold the old limit
  ctx->wait_ns = ns;
  return AD_OK;
}

ad_status ad_closure(ad_ctx* ctx, const ad_grid* grid, int nvel, int ncomp, const void* ubar, const void* ustar,
                     void* tau, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (ncomp < 1 || ncomp > 3) return fail(ctx, AD_ERR_ARG, "ncomp must be 1, 2 or 3");
  if (nvel < 0) return fail(ctx, AD_ERR_ARG, "nvel < 0");
  const int npairs = ncomp * (ncomp + 1) / 2;
  if ((long long)nvel * npairs > AD_MAX_BATCH) return fail(ctx, AD_ERR_ARG, "nvel * pairs > AD_MAX_BATCH");
  if (nvel == 0) { ctx->launches = 0; return AD_OK; }
  if (!ubar || !ustar || !tau) return fail(ctx, AD_ERR_ARG, "NULL field pointer");
  if (((uintptr_t)ubar | (uintptr_t)ustar | (uintptr_t)tau) & 15)
    return fail(ctx, AD_ERR_ARG, "field pointers must be 16-byte aligned");
  const size_t es = grid->dtype == AD_F64 ? 8 : 4;
  const long long P = grid->n[0] * grid->n[1] * (grid->ndim == 3 ? grid->n[2] : 1);
  const size_t nin = (size_t)nvel * ncomp * P * es, nout = (size_t)nvel * npairs * P * es;
  if (overlaps(tau, nout, ubar, nin) || overlaps(tau, nout, ustar, nin))
    return fail(ctx, AD_ERR_ARG, "tau must not overlap ubar or ustar");
  CK(cudaSetDevice(ctx->device));
  Plan* p = nullptr;
  if ((s = get_plan(ctx, grid, nvel * npairs, &p)) != AD_OK) return s;
  Common c;
  c.ncomp = ncomp;
  c.npairs = npairs;
  int code = 0, q = 0;
  for (int i = 0; i < ncomp; ++i)
    for (int j = i; j < ncomp; ++j, ++q) code |= (i | (j << 2)) << (4 * q);
  c.pair_code = code;
  Fwd fw; fw.op = XF_MUL; fw.A = ustar;
  Inv iv; iv.op = XI_TAU; iv.B = ubar; iv.O1 = tau;
  int nl = 0;
  cudaStream_t st = (cudaStream_t)stream;
  s = p->f64 ? enqueue_G<double>(ctx, p, st, fw, Flt{}, iv, c, &nl) : enqueue_G<float>(ctx, p, st, fw, Flt{}, iv, c, &nl);
  ctx->launches = nl;
  return s;
}

ad_status ad_spectrum(ad_ctx* ctx, const ad_grid* grid, int nfields, int ncomp, const void* u, int nbins,
                      double* E, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_grid(ctx, grid);
  if (s != AD_OK) return s;
  if (ncomp < 1 || nfields < 0 || nfields % ncomp != 0) return fail(ctx, AD_ERR_ARG, "nfields must be a multiple of ncomp >= 1");
  if (nbins < 1 || nbins > AD_MAX_SHELLS) return fail(ctx, AD_ERR_ARG, "nbins must be in [1, AD_MAX_SHELLS]");
  if (nfields > AD_MAX_BATCH) return fail(ctx, AD_ERR_ARG, "nfields > AD_MAX_BATCH");
  if (nfields == 0) { ctx->launches = 0; return AD_OK; }
  if (!u || !E) return fail(ctx, AD_ERR_ARG, "NULL pointer");
  if ((uintptr_t)u & 15) return fail(ctx, AD_ERR_ARG, "field pointers must be 16-byte aligned");
  CK(cudaSetDevice(ctx->device));
  Plan* p = nullptr;
  if ((s = get_plan(ctx, grid, nfields, &p)) != AD_OK) return s;
  if ((s = ensure_spectral(ctx, p)) != AD_OK) return s;
  const int ngroups = nfields / ncomp;
  const size_t bytes = sizeof(double) * (size_t)ngroups * nbins;
  void* buf = nullptr;
  if ((s = stat_scratch(ctx, bytes, &buf)) != AD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int nl = 0;
  s = p->f64 ? enqueue_fwd_transform<double>(ctx, p, st, u, p->Bh, &nl)
             : enqueue_fwd_transform<float>(ctx, p, st, u, p->Bh, &nl);
  if (s != AD_OK) return s;
  CK(cudaMemsetAsync(buf, 0, bytes, st));
  const double scale = 1.0 / ((double)p->P * (double)p->P);
  CK(p->f64 ? launch_shell<double>(p->Bh, p->nx, p->ny, p->nz, p->SP, nfields, ncomp, nbins, scale, (double*)buf, st)
            : launch_shell<float>(p->Bh, p->nx, p->ny, p->nz, p->SP, nfields, ncomp, nbins, scale, (double*)buf, st));
  CK(cudaMemcpyAsync(E, buf, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ctx->launches = nl + 1;
  return AD_OK;
}

ad_status ad_histogram(ad_ctx* ctx, ad_dtype dtype, int64_t n, const void* x, double lo, double hi, int nbins,
                       int64_t* counts, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  if (dtype != AD_F32 && dtype != AD_F64) return fail(ctx, AD_ERR_ARG, "dtype must be AD_F32 or AD_F64");
  if (n < 0 || nbins < 1 || nbins > AD_MAX_HIST_BINS) return fail(ctx, AD_ERR_ARG, "need n >= 0 and 1 <= nbins <= AD_MAX_HIST_BINS");
  if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi)) return fail(ctx, AD_ERR_ARG, "need finite lo < hi");
  if (!counts) return fail(ctx, AD_ERR_ARG, "NULL counts");
  if (n > 0 && !x) return fail(ctx, AD_ERR_ARG, "NULL data");
  CK(cudaSetDevice(ctx->device));
  const size_t bytes = sizeof(unsigned long long) * (size_t)(nbins + 3);
  void* buf = nullptr;
  ad_status s;
  if ((s = stat_scratch(ctx, bytes, &buf)) != AD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(buf, 0, bytes, st));
  const double scale = (double)nbins / (hi - lo);
  if (n > 0) {
    CK(dtype == AD_F64 ? launch_hist<double>((const double*)x, n, lo, scale, nbins, (unsigned long long*)buf, st)
                       : launch_hist<float>((const float*)x, n, lo, scale, nbins, (unsigned long long*)buf, st));
  }
  std::vector<unsigned long long> h(nbins + 3);
  CK(cudaMemcpyAsync(h.data(), buf, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int b = 0; b < nbins + 3; ++b) counts[b] = (int64_t)h[b];
  ctx->launches = n > 0 ? 1 : 0;
  return AD_OK;
}

ad_status ad_curl(ad_ctx* ctx, const ad_grid* grid, int nvel, const void* u, void* omega, void* stream) {
  if (!ctx) return AD_ERR_ARG;
  ad_status s = check_grid(ctx, grid);
  if (s != AD_OK) return s;
  const int ncomp = grid->ndim, nout = grid->ndim == 2 ? 1 : 3;
  if (nvel < 0 || (long long)nvel * ncomp > AD_MAX_BATCH) return fail(ctx, AD_ERR_ARG, "bad nvel");
  if (nvel == 0) { ctx->launches = 0; return AD_OK; }
  if (!u || !omega) return fail(ctx, AD_ERR_ARG, "NULL field pointer");
  if (((uintptr_t)u | (uintptr_t)omega) & 15) return fail(ctx, AD_ERR_ARG, "field pointers must be 16-byte aligned");
  {
    const size_t es = grid->dtype == AD_F64 ? 8 : 4;
    const long long P = grid->n[0] * grid->n[1] * (grid->ndim == 3 ? grid->n[2] : 1);
    if (overlaps(omega, (size_t)nvel * nout * P * es, u, (size_t)nvel * ncomp * P * es))
      return fail(ctx, AD_ERR_ARG, "omega must not overlap u");
  }
  CK(cudaSetDevice(ctx->device));
  Plan *pin = nullptr, *pout = nullptr;
  if ((s = get_plan(ctx, grid, nvel * ncomp, &pin)) != AD_OK) return s;
  if ((s = ensure_spectral(ctx, pin)) != AD_OK) return s;
  if ((s = get_plan(ctx, grid, nvel * nout, &pout)) != AD_OK) return s;
  if ((s = ensure_spectral(ctx, pout)) != AD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int nl = 0;
  s = pin->f64 ? enqueue_fwd_transform<double>(ctx, pin, st, u, pin->Bh, &nl)
               : enqueue_fwd_transform<float>(ctx, pin, st, u, pin->Bh, &nl);
  if (s != AD_OK) return s;
  CK(pin->f64 ? launch_curl<double>(pin->Bh, pout->Uh, pin->nx, pin->ny, pin->nz, pin->SP, nvel, ncomp, st)
              : launch_curl<float>(pin->Bh, pout->Uh, pin->nx, pin->ny, pin->nz, pin->SP, nvel, ncomp, st));
  ++nl;
  s = pout->f64 ? enqueue_inv_transform<double>(ctx, pout, st, pout->Uh, omega, &nl)
                : enqueue_inv_transform<float>(ctx, pout, st, pout->Uh, omega, &nl);
  ctx->launches = nl;
  return s;
}

}  // extern "C"

