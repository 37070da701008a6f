// Pass kernels of one application of the filter G (Section 4, Eq. df2:
// G_hat(k) = 1/(1 + |k|^2/k_c^2), applied spectrally) with the Krylov
// vector updates and inner products of Algorithms 1-4 fused into the first
// and last pass.
//
// Grids are C-ordered with x contiguous: field f, point (z, y, x) at
// f*P + (z*ny + y)*nx + x. One application of G runs
//   2D: xfwd -> filt(y) -> xinv
//   3D: xfwd -> yfwd -> filt(z) -> yinv -> xinv
// with two spectral buffers per field (complex, kxn = nx/2 + 1):
//   S1 [z][kx][y]  written by xfwd / yinv, read by yfwd / xinv (and by filt in 2D)
//   S2 [kx][ky][z] written by yfwd, filtered in place by filt (3D), read by yinv
// Every pass loads contiguous runs and, where the next pass needs another
// axis contiguous, stores its tile transposed (W consecutive sequences per
// wavenumber), so all global accesses are coalesced.
#pragma once

#include <cuda_runtime.h>

#include "args.h"
#include "fft.cuh"

namespace gad {

// ---------------------------------------------------------------------------
// Compensated accumulation for the inner products: exact float products
// (fma residual) summed with TwoSum, so each thread's partial carries about
// twice the working precision before it is widened to float64.
template <typename T>
struct Acc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {
    T t = s + x;
    T bp = t - s;
    T e = (s - (t - bp)) + (x - bp);
    s = t;
    c += e;
  }
  __device__ __forceinline__ void add_prod(T a, T b) {
    T p = a * b;
    T e = fma(a, b, -p);
    add(p);
    c += e;
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

template <typename T> struct V4 { T v[4]; };

__device__ __forceinline__ V4<float> ld4(const float* p) {
  float4 a = *reinterpret_cast<const float4*>(p);
  return {{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& x) {
  *reinterpret_cast<float4*>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  double2 a = reinterpret_cast<const double2*>(p)[0];
  double2 b = reinterpret_cast<const double2*>(p)[1];
  return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(double* p, const V4<double>& x) {
  reinterpret_cast<double2*>(p)[0] = make_double2(x.v[0], x.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(x.v[2], x.v[3]);
}

__device__ __forceinline__ float2 ldc2(const float2* p) { return *p; }
__device__ __forceinline__ double2 ldc2(const double2* p) { return *p; }

// ---------------------------------------------------------------------------
// Scalar recurrences, run once per field by the last block of a dot pass.
__device__ inline bool finite_d(double x) { return isfinite(x); }

__device__ inline void stop_or_continue(FieldState& s, const SolveConfig& cfg, int f, double rr) {
  s.iter += 1;
  const double h = s.ref > 0.0 ? sqrt(fmax(rr, 0.0)) / s.ref : 0.0;
  s.h = h;
  if (cfg.hist && s.iter <= cfg.maxit) cfg.hist[(long long)f * cfg.hist_ld + s.iter] = h;
  if (!finite_d(rr)) {
    s.status = 2; s.active = 0;                  // AD_BREAKDOWN
  } else if (s.early || h <= cfg.tol) {
    s.status = 0; s.active = 0;                  // AD_OK
  } else if (s.iter >= cfg.maxit) {
    s.status = 1; s.active = 0;                  // AD_MAXIT
  }
}

__device__ inline void scalar_update(int stage, FieldState& s, const double* d, const SolveConfig& cfg, int f) {
  switch (stage) {
    case SS_REF:
      s.ref = sqrt(fmax(d[0], 0.0));
      s.have_ref = 1;
      break;
    case SS_INIT: {
      const double rr = d[0];
      if (!s.have_ref) s.ref = sqrt(fmax(rr, 0.0));
      s.iter = 0;
      s.early = 0;
      s.fin_axpy = 0;
      const double h0 = s.ref > 0.0 ? sqrt(fmax(rr, 0.0)) / s.ref : 0.0;
      s.h = h0;
      if (cfg.hist) cfg.hist[(long long)f * cfg.hist_ld] = h0;
      s.rho = rr;                 // CG: rho_0; BiCGSTAB: rho_1 = (f0, r0) = (r0, r0)
      s.alpha = 1.0;
      s.omega = 1.0;
      s.beta = 0.0;
      if (!finite_d(rr) || !finite_d(s.ref)) { s.status = -2; s.active = 0; }
      else if (h0 <= cfg.tol) { s.status = 0; s.active = 0; }
      else if (cfg.maxit <= 0) { s.status = 1; s.active = 0; }
      else { s.status = 0; s.active = 1; }
      break;
    }
    case SS_VC:                  // Algorithms 1 and 2: end of a pass
      s.rho = d[0];
      stop_or_continue(s, cfg, f, d[0]);
      break;
    case SS_SD_ALPHA:
    case SS_CG_ALPHA: {
      const double a = s.rho / d[0];
      if (!(d[0] > 0.0) || !finite_d(a)) { s.status = 2; s.active = 0; }
      else s.alpha = a;
      break;
    }
    case SS_CG_BETA: {
      const double rr = d[0];
      s.beta = rr / s.rho;
      s.rho = rr;
      stop_or_continue(s, cfg, f, rr);
      if (!s.active) s.fin_axpy = 1;
      break;
    }
    case SS_BI_ALPHA: {
      const double fq = d[0];
      const double a = s.rho / fq;
      if (fq == 0.0 || !finite_d(fq) || !finite_d(a)) { s.status = 2; s.active = 0; }
      else s.alpha = a;
      break;
    }
    case SS_BI_OMEGA: {
      const double ss = d[0], st = d[1], tt = d[2];
      const double hs = s.ref > 0.0 ? sqrt(fmax(ss, 0.0)) / s.ref : 0.0;
      if (hs <= cfg.tol || tt == 0.0) { s.omega = 0.0; s.early = 1; }
      else {
        const double w = st / tt;
        if (!finite_d(w)) { s.status = 2; s.active = 0; }
        else s.omega = w;
      }
      break;
    }
    case SS_BI_END: {
      const double rr = d[0], fr = d[1];
      stop_or_continue(s, cfg, f, rr);
      if (s.active) {
        const double b = (fr / s.rho) * (s.alpha / s.omega);
        if (fr == 0.0 || !finite_d(fr) || !finite_d(b)) { s.status = 2; s.active = 0; }
        else { s.beta = b; s.rho = fr; }
      }
      break;
    }
    case SS_TRUE:
      s.true_res = s.ref > 0.0 ? sqrt(fmax(d[0], 0.0)) / s.ref : sqrt(fmax(d[0], 0.0));
      break;
    default:
      break;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of up to three dots into a per-block partial, then two
// arrival tickets. ticket[2 + f] counts the blocks of field f: the last one
// to arrive sums that field's partials in a fixed order (deterministic for a
// fixed launch shape) and runs the field's scalar update at once, while
// other fields' blocks are still running. ticket[0] counts finished fields:
// the last one sets the graph's loop condition. ticket[1] counts loop passes
// of the current solve (reset by the initial-residual pass).
template <typename T>
__device__ void block_finish(const PassArgs<T>& a, const Acc<T>* acc, int f, bool act) {
  __shared__ double red[32][3];
  __shared__ int last_field;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const int nblk = gridDim.x;
  if (act) {
    double v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = warp_sum(acc[d].value());
    if (lane == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) red[warp][d] = v[d];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double t = lane < nw ? red[lane][d] : 0.0;
        t = warp_sum(t);
        if (lane == 0) a.part[((long long)f * nblk + blockIdx.x) * 4 + d] = t * a.inv_p;
      }
    }
  }
  if (tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(a.ticket + 2 + f, 1u);
    last_field = (prev == (unsigned)nblk - 1u);
  }
  __syncthreads();
  if (!last_field) return;
  __threadfence();
  FieldState& s = a.st[f];
  if (act) {                    // act is the field's flag: every block of f saw the same value
    double t[3] = {0.0, 0.0, 0.0};
    const double* pf = a.part + (long long)f * nblk * 4;
    for (int b = tid; b < nblk; b += blockDim.x) {
#pragma unroll
      for (int d = 0; d < 3; ++d) t[d] += __ldcg(pf + (long long)b * 4 + d);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) t[d] = warp_sum(t[d]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) red[warp][d] = t[d];
    }
    __syncthreads();
    if (tid == 0) {
      double tot[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        tot[d] = 0.0;
        for (int q = 0; q < nw; ++q) tot[d] += red[q][d];
      }
      scalar_update(a.stage, s, tot, a.cfg, f);
    }
  }
  if (tid == 0) {
    a.ticket[2 + f] = 0u;
    __threadfence();
    const unsigned prevg = atomicAdd(a.ticket, 1u);
    if (prevg == gridDim.y - 1u) {                        // every field is reduced
      __threadfence();
      if (a.stage == SS_INIT) a.ticket[1] = 0u;
      if (a.set_cond) {
        unsigned any = 0;
        for (int g = 0; g < a.batch; ++g) any |= (*(volatile const int*)&a.st[g].active != 0);
        // every field stops by maxit passes; never iterate past that bound
        const unsigned loops = ++a.ticket[1];
        if (loops > (unsigned)a.cfg.maxit + 1u) any = 0;
        cudaGraphSetConditional(a.cond, any);
      }
      a.ticket[0] = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// Loads a W x n tile stored transposed in global memory (element (w, i) at
// g[i*gstride + w]) into the shared-memory rows, U independent loads per
// thread in flight.
template <typename C, int U>
__device__ __forceinline__ void load_transposed(C* s, int ld, const C* __restrict__ g, long long gstride, int W,
                                                int n, int tid, int nthr) {
  const int lw = __ffs(W) - 1;
  const int total = W * n;
  for (int base = tid; base < total; base += nthr * U) {
    C tmp[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * nthr;
      if (idx < total) tmp[u] = g[(long long)(idx >> lw) * gstride + (idx & (W - 1))];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * nthr;
      if (idx < total) s[(idx & (W - 1)) * ld + phys(idx >> lw)] = tmp[u];
    }
  }
}

// Stores the shared-memory rows transposed (element (w, i) to g[i*gstride + w]).
template <typename C>
__device__ __forceinline__ void store_transposed(const C* s, int ld, C* __restrict__ g, long long gstride, int W,
                                                 int n, int tid, int nthr) {
  const int lw = __ffs(W) - 1;
  for (int idx = tid; idx < W * n; idx += nthr)
    g[(long long)(idx >> lw) * gstride + (idx & (W - 1))] = s[(idx & (W - 1)) * ld + phys(idx >> lw)];
}

template <typename T> struct V2 { T x, y; };
template <typename T> __device__ __forceinline__ V2<T> ld2(const T* p) {
  using C = typename cpx<T>::t;
  const C c = *reinterpret_cast<const C*>(p);
  return {c.x, c.y};
}
template <typename T> __device__ __forceinline__ void st2(T* p, T a, T b) {
  using C = typename cpx<T>::t;
  *reinterpret_cast<C*>(p) = C{a, b};
}

// x and y passes fit 80 registers at E = 16 (3 blocks of 256 per SM); the filter
// pass keeps two FFT stages' worth of state live and gets 128.
#define GAD_BOUNDS(T, E) __launch_bounds__(256, (sizeof(T) == 4 && (E) == 16) ? 3 : 2)
#define GAD_BOUNDS_FILT __launch_bounds__(256, 2)

// Forward x pass: the Krylov prologue is fused into the first FFT stage,
// which reads the packed rows z[n] = x[2n] + i x[2n+1] straight from global
// memory; the real-to-complex split and the transposed store to S1 follow.
//   rcp_b = 1/(nx/4 + 1)
template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_xfwd(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  if (a.clear_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
  FieldState* st = a.st ? a.st + f : nullptr;
  if (st && !st->active && !a.force) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = a.nx, M = nx >> 1;
  const int row0 = blockIdx.x * a.W;
  const int z = row0 / a.ny, y0 = row0 - z * a.ny;
  const long long base = (long long)f * a.P + (long long)row0 * nx;
  const bool first = st ? (st->iter == 0) : true;
  const T al = st ? T(st->alpha) : T(0), be = st ? T(st->beta) : T(0), om = st ? T(st->omega) : T(0);
  const int op = a.op;
  const T* __restrict__ vA = a.A;
  const T* __restrict__ vB = a.B;
  T* vO1 = a.O1;
  T* vO2 = a.O2;
  T* vO3 = a.O3;

  auto load = [&](int w, int n) -> C {
    const long long g = base + (long long)w * nx + 2 * n;
    T x0, x1;
    switch (op) {
      case XF_VC: {                               // U += R; x = R
        const V2<T> r = ld2(vA + g), u = ld2(vO1 + g);
        st2(vO1 + g, u.x + r.x, u.y + r.y);
        x0 = r.x; x1 = r.y;
        break;
      }
      case XF_CG: {                               // U += alpha P; P = R + beta P
        const V2<T> r = ld2(vA + g);
        if (first) {
          x0 = r.x; x1 = r.y;
        } else {
          const V2<T> p = ld2(vO2 + g), u = ld2(vO1 + g);
          st2(vO1 + g, fma(al, p.x, u.x), fma(al, p.y, u.y));
          x0 = fma(be, p.x, r.x); x1 = fma(be, p.y, r.y);
        }
        st2(vO2 + g, x0, x1);
        break;
      }
      case XF_BI_P: {                             // P = R + beta (P - omega Q)
        const V2<T> r = ld2(vA + g);
        if (first) {
          x0 = r.x; x1 = r.y;
        } else {
          const V2<T> p = ld2(vO2 + g), q = ld2(vB + g);
          x0 = fma(be, fma(-om, q.x, p.x), r.x);
          x1 = fma(be, fma(-om, q.y, p.y), r.y);
        }
        st2(vO2 + g, x0, x1);
        break;
      }
      case XF_BI_S: {                             // S = R - alpha Q
        const V2<T> r = ld2(vA + g), q = ld2(vB + g);
        x0 = fma(-al, q.x, r.x); x1 = fma(-al, q.y, r.y);
        st2(vO3 + g, x0, x1);
        break;
      }
      default: {                                  // XF_COPY: x = A (and O1 = A)
        const V2<T> v = ld2(vA + g);
        if (vO1) st2(vO1 + g, v.x, v.y);
        x0 = v.x; x1 = v.y;
        break;
      }
    }
    return C{x0, x1};
  };
  SmemRows<C> rows{s, a.ld};
  fft_run<C, E, false>(s, a.ld, a.fft, tid, a.tfft, load, rows, false, true);
  // split the packed half-length transform into the real-input spectrum
  const C* twx = reinterpret_cast<const C*>(a.twx);
  const int h1 = (M >> 1) + 1;
  for (int idx = tid; idx < a.W * h1; idx += nthr) {
    const int w = fquot(idx, a.rcp_b);
    const int k = idx - w * h1;
    C* row = s + w * a.ld;
    if (k == 0) {
      const C z0 = row[0];
      row[0] = C{z0.x + z0.y, T(0)};
      row[phys(M)] = C{z0.x - z0.y, T(0)};
    } else {
      const C A = row[phys(k)], B = row[phys(M - k)];
      const C e = {T(0.5) * (A.x + B.x), T(0.5) * (A.y - B.y)};   // (A + conj B)/2
      const C o = {T(0.5) * (A.y + B.y), T(0.5) * (B.x - A.x)};   // -i (A - conj B)/2
      const C wo = cmul(twx[k], o);
      row[phys(k)] = cadd(e, wo);
      row[phys(M - k)] = cconj(csub(e, wo));
    }
  }
  __syncthreads();
  C* S1 = reinterpret_cast<C*>(a.S1) + (long long)f * a.SP + (long long)z * a.kxn * a.ny + y0;
  store_transposed(s, a.ld, S1, a.ny, a.W, M + 1, tid, nthr);
}

// Inverse x pass: transposed load from S1, complex-to-real preparation, FFT
// whose last stage writes the rows through the fused epilogue and dots.
template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_xinv(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  FieldState* st = a.st ? a.st + f : nullptr;
  const bool act = (st ? (st->active != 0) : true) || a.force;
  if (!act && a.ndots == 0) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = a.nx, M = nx >> 1;
  const int row0 = blockIdx.x * a.W;
  const int z = row0 / a.ny, y0 = row0 - z * a.ny;
  Acc<T> acc[3];
  if (act) {
    const C* S1 = reinterpret_cast<const C*>(a.S1) + (long long)f * a.SP + (long long)z * a.kxn * a.ny + y0;
    load_transposed<C, 8>(s, a.ld, S1, a.ny, a.W, M + 1, tid, nthr);
    __syncthreads();
    const C* twx = reinterpret_cast<const C*>(a.twx);
    const int h1 = (M >> 1) + 1;
    for (int idx = tid; idx < a.W * h1; idx += nthr) {
      const int w = fquot(idx, a.rcp_b);
      const int k = idx - w * h1;
      C* row = s + w * a.ld;
      if (k == 0) {
        const T x0 = row[0].x, xm = row[phys(M)].x;   // imaginary parts of DC/Nyquist dropped
        row[0] = C{x0 + xm, x0 - xm};
      } else {
        const C A = row[phys(k)], B = row[phys(M - k)];
        const C e = {A.x + B.x, A.y - B.y};            // A + conj B
        const C d = {A.x - B.x, A.y + B.y};            // A - conj B
        const C o = cmulc(d, twx[k]);                  // (A - conj B) conj(W^k)
        row[phys(k)] = C{e.x - o.y, e.y + o.x};        // e + i o
        row[phys(M - k)] = C{e.x + o.y, o.x - e.y};    // conj(e) + i conj(o)
      }
    }
    __syncthreads();
    const long long base = (long long)f * a.P + (long long)row0 * nx;
    const T al = st ? T(st->alpha) : T(0), om = st ? T(st->omega) : T(0);
    const int op = a.op;
    const T* __restrict__ vA = a.A;
    const T* __restrict__ vB = a.B;
    const T* __restrict__ vC = a.C;
    T* vO1 = a.O1;
    T* vO2 = a.O2;
    Acc<T> acc0, acc1;
    auto emit = [&](int w, int n, const C& y) {
      const long long g = base + (long long)w * nx + 2 * n;
      switch (op) {
        case XI_STORE:
          st2(vO1 + g, y.x, y.y);
          break;
        case XI_INIT: {
          const V2<T> u = ld2(vA + g);
          const T r0 = u.x - y.x, r1 = u.y - y.y;
          acc0.add_prod(r0, r0); acc0.add_prod(r1, r1);
          st2(vO1 + g, r0, r1);
          if (vO2) st2(vO2 + g, r0, r1);
          break;
        }
        case XI_RES: {
          const V2<T> u = ld2(vA + g);
          const T r0 = u.x - y.x, r1 = u.y - y.y;
          acc0.add_prod(r0, r0); acc0.add_prod(r1, r1);
          break;
        }
        case XI_VC: {
          const V2<T> r = ld2(vO1 + g);
          const T r0 = r.x - y.x, r1 = r.y - y.y;
          acc0.add_prod(r0, r0); acc0.add_prod(r1, r1);
          st2(vO1 + g, r0, r1);
          break;
        }
        case XI_CG: {
          const V2<T> r = ld2(vO1 + g);
          const T r0 = fma(-al, y.x, r.x), r1 = fma(-al, y.y, r.y);
          acc0.add_prod(r0, r0); acc0.add_prod(r1, r1);
          st2(vO1 + g, r0, r1);
          break;
        }
        case XI_SD: {
          const V2<T> r = ld2(vO1 + g), u = ld2(vO2 + g);
          st2(vO2 + g, fma(al, r.x, u.x), fma(al, r.y, u.y));
          const T r0 = fma(-al, y.x, r.x), r1 = fma(-al, y.y, r.y);
          acc0.add_prod(r0, r0); acc0.add_prod(r1, r1);
          st2(vO1 + g, r0, r1);
          break;
        }
        case XI_BI_Q: {
          const V2<T> f0 = ld2(vA + g);
          acc0.add_prod(f0.x, y.x); acc0.add_prod(f0.y, y.y);
          st2(vO1 + g, y.x, y.y);
          break;
        }
        case XI_BI_T: {
          const V2<T> f0 = ld2(vA + g), p = ld2(vB + g), sv = ld2(vC + g), u = ld2(vO1 + g);
          st2(vO1 + g, fma(om, sv.x, fma(al, p.x, u.x)), fma(om, sv.y, fma(al, p.y, u.y)));
          const T r0 = fma(-om, y.x, sv.x), r1 = fma(-om, y.y, sv.y);
          acc0.add_prod(r0, r0); acc0.add_prod(r1, r1);
          acc1.add_prod(f0.x, r0); acc1.add_prod(f0.y, r1);
          st2(vO2 + g, r0, r1);
          break;
        }
        default:
          break;
      }
    };
    SmemRows<C> rows{s, a.ld};
    fft_run<C, E, true>(s, a.ld, a.fft, tid, a.tfft, rows, emit, true, false);
    acc[0] = acc0;
    acc[1] = acc1;
  }
  if (a.ndots) block_finish(a, acc, f, act);
}

// Filter pass along the last axis (y in 2D, z in 3D): forward FFT of W
// contiguous sequences read straight from the spectral buffer, multiply by
// G_hat(k)/P with Parseval dots in registers, inverse FFT written straight
// back. fft holds the forward plan, fft_inv the reversed one. In 3D the
// sequence index is kx*ny + ky.
template <typename T, int E>
__global__ void GAD_BOUNDS_FILT k_filt(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  FieldState* st = a.st ? a.st + f : nullptr;
  const bool act = (st ? (st->active != 0) : true) || a.force;
  if (!act && a.ndots == 0) return;
  const int tid = threadIdx.x;
  const int L = a.fft.L, half = L >> 1;
  const bool three_d = a.nz > 1;
  const int nseq = three_d ? a.kxn * a.ny : a.kxn;
  const int seq0 = blockIdx.x * a.W;
  const int nvalid = min(a.W, nseq - seq0);
  C* S = reinterpret_cast<C*>(three_d ? a.S2 : a.S1) + (long long)f * a.SP + (long long)seq0 * L;
  Acc<T> acc[3];
  if (act) {
    const int nxh = a.nx >> 1, ny = a.ny;
    const T kc2 = a.kc2, gs = a.gscale;
    const int op = a.op;
    // Parseval sums have positive terms only: each thread sums its E terms
    // in plain T, and the partials are widened to float64 from there on
    T p0 = T(0), p1 = T(0), p2 = T(0);
    auto load = [&](int w, int i) -> C {
      return w < nvalid ? S[(long long)w * L + i] : C{T(0), T(0)};
    };
    auto mul = [&](int w, int i, C& X) {
      const int seq = seq0 + w;
      int kx, k2i;
      const int ki = i < half ? i : i - L;
      if (three_d) {
        kx = seq / ny;
        const int kyi = seq - kx * ny;
        const int ky = kyi < (ny >> 1) ? kyi : kyi - ny;
        k2i = kx * kx + ky * ky + ki * ki;
      } else {
        kx = seq;
        k2i = kx * kx + ki * ki;
      }
      const T g = kc2 / (kc2 + T(k2i));
      if (op != FI_NONE && w < nvalid) {
        const T wgt = (kx == 0 || kx == nxh) ? T(1) : T(2);
        const T m2 = X.x * X.x + X.y * X.y;
        const T wm = wgt * m2;
        if (op == FI_XGX) {
          p0 = fma(g, wm, p0);
        } else {
          p0 += wm;
          const T gw = g * wm;
          p1 += gw;
          p2 = fma(g, gw, p2);
        }
      }
      const T sc = g * gs;
      X = C{X.x * sc, X.y * sc};
    };
    auto emit = [&](int w, int i, const C& x) {
      if (w < nvalid) S[(long long)w * L + i] = x;
    };
    fft_filter_run<C, E>(s, a.ld, a.fft, a.fft_inv, tid, a.tfft, load, mul, emit);
    acc[0].s = p0;
    acc[1].s = p1;
    acc[2].s = p2;
  }
  if (a.ndots) block_finish(a, acc, f, act);
}

// 3D forward y pass: W consecutive z at one kx; the first stage reads the
// S1 rows [z][kx][:] directly, the tile is stored transposed into S2
// [kx][ky][z].  Grid x = kxn * (nz/W).
template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_yfwd(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  if (a.st && !a.st[f].active && !a.force) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = a.ny;
  const int zt = a.nz / a.W;
  const int kx = blockIdx.x / zt, z0 = (blockIdx.x - kx * zt) * a.W;
  const C* S1 = reinterpret_cast<const C*>(a.S1) + (long long)f * a.SP;
  const int kxn = a.kxn;
  auto load = [&](int w, int i) -> C { return S1[((long long)(z0 + w) * kxn + kx) * L + i]; };
  SmemRows<C> rows{s, a.ld};
  fft_run<C, E, false>(s, a.ld, a.fft, tid, a.tfft, load, rows, false, true);
  C* S2 = reinterpret_cast<C*>(a.S2) + (long long)f * a.SP + (long long)kx * L * a.nz + z0;
  store_transposed(s, a.ld, S2, a.nz, a.W, L, tid, nthr);
}

// 3D inverse y pass: transposed load from S2, inverse FFT whose last stage
// writes the S1 rows directly.
template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_yinv(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  if (a.st && !a.st[f].active && !a.force) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = a.ny;
  const int zt = a.nz / a.W;
  const int kx = blockIdx.x / zt, z0 = (blockIdx.x - kx * zt) * a.W;
  const C* S2 = reinterpret_cast<const C*>(a.S2) + (long long)f * a.SP + (long long)kx * L * a.nz + z0;
  load_transposed<C, 8>(s, a.ld, S2, a.nz, a.W, L, tid, nthr);
  __syncthreads();
  C* S1 = reinterpret_cast<C*>(a.S1) + (long long)f * a.SP;
  const int kxn = a.kxn;
  auto emit = [&](int w, int i, const C& x) { S1[((long long)(z0 + w) * kxn + kx) * L + i] = x; };
  SmemRows<C> rows{s, a.ld};
  fft_run<C, E, true>(s, a.ld, a.fft, tid, a.tfft, rows, emit, true, false);
}

// u += alpha p for fields whose last CG pass still owes it (Algorithm 3,
// deferred so that the forward pass of the next iteration can fuse it).
template <typename T>
__global__ void k_cg_finish(T* __restrict__ u, const T* __restrict__ p, const FieldState* st, long long P, int batch) {
  const int f = blockIdx.y;
  if (!st[f].fin_axpy) return;
  const T al = T(st[f].alpha);
  const long long n4 = P >> 2;
  T* uf = u + (long long)f * P;
  const T* pf = p + (long long)f * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    V4<T> uu = ld4(uf + 4 * i), pp = ld4(pf + 4 * i);
#pragma unroll
    for (int e = 0; e < 4; ++e) uu.v[e] = fma(al, pp.v[e], uu.v[e]);
    st4(uf + 4 * i, uu);
  }
}

// Resets the per-field solver state before a solve.
static __global__ void k_reset_state(FieldState* st, int batch) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= batch) return;
  FieldState z = {};
  z.active = 1;
  st[f] = z;
}

}  // namespace gad
