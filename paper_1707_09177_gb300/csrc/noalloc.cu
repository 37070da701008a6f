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
// first call per device should therefore come before any stream capture. The
// cached address belongs to the device's context: after cudaDeviceReset on a
// device it is stale, so a process that resets a device must not call this
// entry point on that device again.

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/gad.h"
#include "args.h"
#include "fft.cuh"
#include "launch.h"
#include "plan.h"

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

// The twiddle table of an FFT plan (see FftPlan): entry e of stage q,
// e = tw_off(q) + (r - 1) ns(q) + k, is exp(-2 pi i r k / (rad[q] ns(q))).
struct RadixList {
  int r[kMaxStages];
  int n;
};

template <typename C, typename R>
__global__ void k_static_plan_twiddles(C* tw, RadixList rl, int L) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L - 1) return;
  int ns = 1, off = 0;
  for (int q = 0; q < rl.n; ++q) {
    const int cnt = (rl.r[q] - 1) * ns;
    if (e < off + cnt) {
      const int r = (e - off) / ns + 1, k = (e - off) - (r - 1) * ns;
      const int len = rl.r[q] * ns;
      const long long m = ((long long)r * k) % len;
      double sn, cs;
      sincospi(2.0 * (double)m / (double)len, &sn, &cs);
      tw[e] = C{(R)cs, (R)(-sn)};
      return;
    }
    off += cnt;
    ns *= rl.r[q];
  }
}

struct StaticPass {
  TileShape t;
  FftPlan fft{}, fft_inv{};
  float rcp_a = 0.f, rcp_b = 0.f;
  dim3 grid;
};

// The same plan and tile shape as the context-owning entry points build
// (plan.h), so the pass kernels take the same code paths.
bool plan_s(int L, int slots, int div, size_t cs, const void* tab, const void* tab_inv, StaticPass& pc) {
  const int E = pick_E(L);
  if (!make_fft(L, E, tab, pc.fft)) return false;
  if (tab_inv && !make_fft(L, E, tab_inv, pc.fft_inv, true)) return false;
  return choose_tile(L, E, slots, div, cs, pc.t);
}

// Fills a plan's twiddle table on the device (stream order).
template <typename C, typename R>
bool plan_table_s(int L, bool reversed, C* tw, cudaStream_t st) {
  RadixList rl{};
  rl.n = plan_radices(L, pick_E(L), reversed, rl.r);
  if (rl.n == 0) return false;
  if (L > 1) k_static_plan_twiddles<C, R><<<(L - 1 + 255) / 256, 256, 0, st>>>(tw, rl, L);
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
  // scratch layout: the x split's table (nx) | the plans' twiddle tables (x
  // plan: nx/2, filter plan and its reverse: L each, L the last axis; 3D: y
  // plan, ny) | S1 | S2 (3D)
  const int Lf = g->ndim == 3 ? nz : ny;
  const size_t tx = align256((size_t)nx * cs), tpx = align256((size_t)M * cs), tpf = align256((size_t)Lf * cs);
  const size_t tpy = g->ndim == 3 ? align256((size_t)ny * cs) : 0;
  const size_t sb = align256((size_t)SP * batch * cs);
  const size_t tabs = tx + tpx + 2 * tpf + tpy;
  const size_t need = tabs + sb * (g->ndim == 3 ? 2 : 1);
  if (need > (size_t)AD_STATIC_SCRATCH_BYTES) return AD_ERR_ARG;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return AD_ERR_CUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  C* twx = reinterpret_cast<C*>(b);
  C* tpx_d = reinterpret_cast<C*>(b + tx);
  C* tpf_d = reinterpret_cast<C*>(b + tx + tpx);
  C* tpfi_d = reinterpret_cast<C*>(b + tx + tpx + tpf);
  C* tpy_d = reinterpret_cast<C*>(b + tx + tpx + 2 * tpf);
  void* S1 = b + tabs;
  void* S2 = g->ndim == 3 ? (void*)(b + tabs + sb) : nullptr;

  StaticPass xf, fl, yf;
  const int nseq = g->ndim == 3 ? kxn * ny : kxn;
  bool ok = plan_s(M, M + 1, pow2_part(ny), cs, tpx_d, nullptr, xf);
  ok = ok && plan_s(Lf, Lf, 0, cs, tpf_d, tpfi_d, fl);
  if (g->ndim == 3) ok = ok && plan_s(ny, ny, pow2_part(nz), cs, tpy_d, nullptr, yf);
  if (!ok) return AD_ERR_ARG;
  xf.rcp_a = 1.0f / (float)(nx / 4);
  xf.rcp_b = 1.0f / (float)(M / 2 + 1);
  xf.grid = dim3(ny * nz / xf.t.W, batch);
  fl.grid = dim3((nseq + fl.t.W - 1) / fl.t.W, batch);
  if (g->ndim == 3) yf.grid = dim3(kxn * (nz / yf.t.W), batch);

  k_static_twiddles<C, T><<<(nx + 255) / 256, 256, 0, st>>>(twx, nx);
  ok = plan_table_s<C, T>(M, false, tpx_d, st) && plan_table_s<C, T>(Lf, false, tpf_d, st) &&
       plan_table_s<C, T>(Lf, true, tpfi_d, st) && (g->ndim != 3 || plan_table_s<C, T>(ny, false, tpy_d, st));
  if (!ok) return AD_ERR_ARG;
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
    a.W = pc.t.W; a.ld = pc.t.ld; a.fft = pc.fft; a.fft_inv = pc.fft_inv; a.rcp_a = pc.rcp_a; a.rcp_b = pc.rcp_b;
    a.tfft = pc.t.T;
    return launch_pass<T>(kind, pc.t.E, pc.grid, (pc.t.T + 31) / 32 * 32, pc.t.smem, st, a);
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
    if (n < 8 || n > 16384 || n % 2 != 0 || !smooth23(n)) return AD_ERR_ARG;
  }
  if (grid->n[0] % 4 != 0) return AD_ERR_ARG;
  if (batch == 0) return AD_OK;
  if (!in || !out || (((uintptr_t)in | (uintptr_t)out) & 15)) return AD_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return grid->dtype == AD_F64 ? run_static<double>(grid, in, out, batch, st)
                               : run_static<float>(grid, in, out, batch, st);
}
