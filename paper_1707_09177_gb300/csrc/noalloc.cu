// ad_filter_static: the filter G (Eq. df2) without any device allocation.
//
// Some callers cannot let a library allocate device memory: real-time or
// embedded solvers that reserve all memory once at start-up and must never
// block later, applications whose device memory is owned by another
// allocator (a framework's caching pool) that a cudaMalloc behind its back
// would fragment or push over budget, and code that must not synchronize the
// device (cudaMalloc and cudaFree may). For them this entry point keeps its
// scratch -- the twiddle tables and the spectral buffers of the passes -- in
// one file-scope __device__ array of fixed size, reserved when the library is
// loaded and held by every GPU that loads it until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents. Nothing in it needs to start at zero: every call rewrites the
// twiddle tables and every spectral element before reading it. Calls whose
// work overlaps on a GPU (different streams, or different host threads) race
// on the array and give wrong results; serialize them.
//
// The array's name is only a host-side stand-in for the device object: its
// device address is looked up with cudaGetSymbolAddress the first time the
// entry point runs on a device (with that device current) and cached. That
// first call per device should therefore come before any stream capture.

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/gad.h"
#include "args.h"
#include "fft.cuh"
#include "launch.h"

using namespace gad;

static __device__ __align__(256) unsigned char g_static_scratch[AD_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mu;

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// exp(-2 pi i m / L), m in [0, L), written by the device into the scratch.
template <typename C, typename R>
__global__ void k_static_twiddles(C* tw, int L) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  double sn, cs;
  sincospi(2.0 * (double)m / (double)L, &sn, &cs);
  tw[m] = C{(R)cs, (R)(-sn)};
}

int phys_s(int i) { return i + (i >> 4); }

bool smooth23_s(long long n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

int pow2_part_s(long long n) {
  int p = 1;
  while (n % 2 == 0 && p < (1 << 20)) { n /= 2; p *= 2; }
  return p;
}

// Balanced radix list (at most 5 stages), fixed-size storage.
bool radices_s(int L, int E, int* rad, int* nrad) {
  int n = L, a = 0, b = 0, k = 0;
  while (n % 2 == 0) { n /= 2; ++a; }
  while (n % 3 == 0) { n /= 3; ++b; }
  if (n != 1 || (b > 0 && E % 3 != 0)) return false;
  const int maxlog = (E % 16 == 0) ? 4 : 3;
  const int ns = a > 0 ? (a + maxlog - 1) / maxlog : 0;
  if (b + ns > 5) return false;
  for (int i = 0; i < b; ++i) rad[k++] = 3;
  for (int i = 0; i < ns; ++i) rad[k++] = 1 << (a / ns + (i < a % ns ? 1 : 0));
  for (int i = 0; i < k; ++i)
    if (E % rad[i] != 0) return false;
  *nrad = k;
  return k > 0;
}

bool fft_s(int L, const int* rad, int nrad, const void* tab, long long Ltab, FftPlan& fp) {
  fp = FftPlan{};
  fp.L = L;
  fp.nst = nrad;
  fp.tw = tab;
  long long ns = 1;
  for (int q = 0; q < nrad; ++q) {
    FftStage& s = fp.st[q];
    s.radix = rad[q];
    s.ns = (int)ns;
    s.tw_step = (int)(Ltab / (ns * rad[q]));
    s.rcp_lr = 1.0f / (float)(L / rad[q]);
    s.rcp_ns = 1.0f / (float)ns;
    ns *= rad[q];
  }
  return ns == L;
}

struct StaticPass {
  int E = 0, W = 0, T = 0, ld = 0;
  size_t smem = 0;
  FftPlan fft{}, fft_inv{};
  float rcp_a = 0.f, rcp_b = 0.f;
  dim3 grid;
};

bool plan_s(int L, int slots, int div, size_t cs, const void* tab, long long Ltab, bool with_inverse,
            StaticPass& pc) {
  const int E = (L % 3 == 0) ? 24 : 16;
  int rad[8], nrad = 0;
  if (!radices_s(L, E, rad, &nrad) || !fft_s(L, rad, nrad, tab, Ltab, pc.fft)) return false;
  if (with_inverse) {
    int rev[8];
    for (int i = 0; i < nrad; ++i) rev[i] = rad[nrad - 1 - i];
    if (!fft_s(L, rev, nrad, tab, Ltab, pc.fft_inv)) return false;
  }
  int ld = phys_s(slots - 1) + 1;
  if ((ld & 1) == 0) ++ld;
  int bestW = 0, bestT = 0;
  double best = 1e30;
  for (int W = 1; W <= 4096; W *= 2) {
    if (div > 0 && div % W != 0) break;
    const long long tot = (long long)W * L;
    if (tot % E != 0) continue;
    const long long T = tot / E;
    if (T < 1 || T > 256 || (size_t)W * ld * cs > 100 * 1024) continue;
    const double score = std::fabs(std::log2((double)T / 256.0));
    if (score < best - 1e-9) { best = score; bestW = W; bestT = (int)T; }
  }
  if (!bestW) return false;
  pc.E = E;
  pc.W = bestW;
  pc.T = bestT;
  pc.ld = ld;
  pc.smem = (size_t)bestW * ld * cs;
  return true;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

template <typename T>
ad_status run_static(const ad_grid* g, const void* in, void* out, int batch, cudaStream_t st) {
  using C = typename cpx<T>::t;
  const int nx = (int)g->n[0], ny = (int)g->n[1], nz = g->ndim == 3 ? (int)g->n[2] : 1;
  const int kxn = nx / 2 + 1, M = nx / 2;
  const long long P = (long long)nx * ny * nz, SP = (long long)kxn * ny * nz;
  const size_t cs = sizeof(C);
  // scratch layout: twiddles for x, y, z | S1 | S2 (3D)
  const size_t tx = align256((size_t)nx * cs), ty = align256((size_t)ny * cs);
  const size_t tz = g->ndim == 3 ? align256((size_t)nz * cs) : 0;
  const size_t sb = align256((size_t)SP * batch * cs);
  const size_t need = tx + ty + tz + sb * (g->ndim == 3 ? 2 : 1);
  if (need > (size_t)AD_STATIC_SCRATCH_BYTES) return AD_ERR_ARG;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return AD_ERR_CUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  C* twx = reinterpret_cast<C*>(b);
  C* twy = reinterpret_cast<C*>(b + tx);
  C* twz = reinterpret_cast<C*>(b + tx + ty);
  void* S1 = b + tx + ty + tz;
  void* S2 = g->ndim == 3 ? (void*)(b + tx + ty + tz + sb) : nullptr;

  StaticPass xf, fl, yf;
  const int Lf = g->ndim == 3 ? nz : ny;
  const int nseq = g->ndim == 3 ? kxn * ny : kxn;
  bool ok = plan_s(M, M + 1, pow2_part_s(ny), cs, twx, nx, false, xf);
  ok = ok && plan_s(Lf, Lf, 0, cs, g->ndim == 3 ? (const void*)twz : (const void*)twy, Lf, true, fl);
  if (g->ndim == 3) ok = ok && plan_s(ny, ny, pow2_part_s(nz), cs, twy, ny, false, yf);
  if (!ok) return AD_ERR_ARG;
  xf.rcp_a = 1.0f / (float)(nx / 4);
  xf.rcp_b = 1.0f / (float)(M / 2 + 1);
  xf.grid = dim3(ny * nz / xf.W, batch);
  fl.grid = dim3((nseq + fl.W - 1) / fl.W, batch);
  if (g->ndim == 3) yf.grid = dim3(kxn * (nz / yf.W), batch);

  k_static_twiddles<C, T><<<(nx + 255) / 256, 256, 0, st>>>(twx, nx);
  k_static_twiddles<C, T><<<(ny + 255) / 256, 256, 0, st>>>(twy, ny);
  if (g->ndim == 3) k_static_twiddles<C, T><<<(nz + 255) / 256, 256, 0, st>>>(twz, nz);
  if (cudaGetLastError() != cudaSuccess) return AD_ERR_CUDA;

  PassArgs<T> a{};
  a.nx = nx; a.ny = ny; a.nz = nz; a.kxn = kxn;
  a.P = P; a.SP = SP;
  a.twx = twx;
  int nmin = nx < ny ? nx : ny;
  if (g->ndim == 3 && nz < nmin) nmin = nz;
  const double kc = g->gamma * (double)nmin / 2.0;       // k_c = gamma k_m, k_m = min(N)/2
  a.kc2 = (T)(kc * kc);
  a.inv_p = 1.0;
  a.gscale = (T)(1.0 / (double)P);
  a.S1 = S1; a.S2 = S2;
  a.batch = batch;
  auto launch = [&](int kind, const StaticPass& pc) {
    a.W = pc.W; a.ld = pc.ld; a.fft = pc.fft; a.fft_inv = pc.fft_inv; a.rcp_a = pc.rcp_a; a.rcp_b = pc.rcp_b;
    a.tfft = pc.T;
    return launch_pass<T>(kind, pc.E, pc.grid, (pc.T + 31) / 32 * 32, pc.smem, st, a);
  };
  a.op = XF_COPY; a.A = static_cast<const T*>(in);
  if (launch(PK_XFWD, xf) != cudaSuccess) return AD_ERR_CUDA;
  if (g->ndim == 3 && launch(PK_YFWD, yf) != cudaSuccess) return AD_ERR_CUDA;
  a.op = FI_NONE;
  if (launch(PK_FILT, fl) != cudaSuccess) return AD_ERR_CUDA;
  if (g->ndim == 3 && launch(PK_YINV, yf) != cudaSuccess) return AD_ERR_CUDA;
  a.op = XI_STORE; a.O1 = static_cast<T*>(out);
  if (launch(PK_XINV, xf) != cudaSuccess) return AD_ERR_CUDA;
  return AD_OK;
}

}  // namespace

extern "C" ad_status ad_filter_static(const ad_grid* grid, const void* in, void* out, int batch, void* stream) {
  if (!grid || (grid->ndim != 2 && grid->ndim != 3) || (grid->dtype != AD_F32 && grid->dtype != AD_F64) ||
      !(grid->gamma > 0.0) || !std::isfinite(grid->gamma) || batch < 0 || batch > AD_MAX_BATCH)
    return AD_ERR_ARG;
  for (int d = 0; d < grid->ndim; ++d) {
    const long long n = grid->n[d];
    if (n < 8 || n > 16384 || n % 2 != 0 || !smooth23_s(n)) return AD_ERR_ARG;
  }
  if (grid->n[0] % 4 != 0) return AD_ERR_ARG;
  if (batch == 0) return AD_OK;
  if (!in || !out || (((uintptr_t)in | (uintptr_t)out) & 15)) return AD_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return grid->dtype == AD_F64 ? run_static<double>(grid, in, out, batch, st)
                               : run_static<float>(grid, in, out, batch, st);
}
