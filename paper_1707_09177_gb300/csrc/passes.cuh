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

// Block reduction of up to three dots, partial store, arrival ticket; the
// last block to arrive sums every field's partials in a fixed order and runs
// the scalar update (deterministic for a fixed launch shape).
template <typename T>
__device__ void block_finish(const PassArgs<T>& a, const Acc<T>* acc, int f, bool act) {
  __shared__ double red[32][3];
  __shared__ int am_last;
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
    const unsigned prev = atomicAdd(a.ticket, 1u);
    am_last = (prev == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  for (int g = warp; g < a.batch; g += nw) {
    FieldState& s = a.st[g];
    if (!s.active && !a.force) continue;
    double tot[3] = {0.0, 0.0, 0.0};
    for (int b = lane; b < nblk; b += 32) {
      const double* p = a.part + ((long long)g * nblk + b) * 4;
#pragma unroll
      for (int d = 0; d < 3; ++d) tot[d] += __ldcg(p + d);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) tot[d] = warp_sum(tot[d]);
    if (lane == 0) scalar_update(a.stage, s, tot, a.cfg, g);
  }
  __syncthreads();
  if (tid == 0) {
    if (a.stage == SS_INIT) a.ticket[1] = 0u;            // loop counter of this solve
    if (a.set_cond) {
      unsigned any = 0;
      for (int g = 0; g < a.batch; ++g) any |= (a.st[g].active != 0);
      // every field stops by maxit passes; never iterate past that bound
      const unsigned loops = ++a.ticket[1];
      if (loops > (unsigned)a.cfg.maxit + 1u) any = 0;
      cudaGraphSetConditional(a.cond, any);
    }
    a.ticket[0] = 0u;
  }
}

// ---------------------------------------------------------------------------
// Forward x pass: prologue, real-to-complex FFT of W rows, transposed store to S1.
//   rcp_a = 1/(nx/4), rcp_b = 1/(nx/4 + 1)
template <typename T, int E>
__global__ void __launch_bounds__(512) k_xfwd(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  if (a.clear_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
  FieldState* st = a.st ? a.st + f : nullptr;
  if (st && !st->active && !a.force) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = a.nx, M = nx >> 1, cpr = nx >> 2;
  const int row0 = blockIdx.x * a.W;
  const int z = row0 / a.ny, y0 = row0 - z * a.ny;
  const long long base = (long long)f * a.P + (long long)row0 * nx;
  const bool first = st ? (st->iter == 0) : true;
  const T al = st ? T(st->alpha) : T(0), be = st ? T(st->beta) : T(0), om = st ? T(st->omega) : T(0);

  for (int idx = tid; idx < a.W * cpr; idx += nthr) {
    const int w = fquot(idx, a.rcp_a);
    const int q = idx - w * cpr;
    const long long g = base + (long long)w * nx + 4 * q;
    V4<T> x;
    switch (a.op) {
      case XF_COPY: {
        x = ld4(a.A + g);
        if (a.O1) st4(a.O1 + g, x);
        break;
      }
      case XF_VC: {
        x = ld4(a.A + g);
        V4<T> u = ld4(a.O1 + g);
#pragma unroll
        for (int e = 0; e < 4; ++e) u.v[e] += x.v[e];
        st4(a.O1 + g, u);
        break;
      }
      case XF_CG: {
        V4<T> r = ld4(a.A + g);
        if (first) {
          x = r;
        } else {
          V4<T> p = ld4(a.O2 + g), u = ld4(a.O1 + g);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            u.v[e] = fma(al, p.v[e], u.v[e]);
            x.v[e] = fma(be, p.v[e], r.v[e]);
          }
          st4(a.O1 + g, u);
        }
        st4(a.O2 + g, x);
        break;
      }
      case XF_BI_P: {
        V4<T> r = ld4(a.A + g);
        if (first) {
          x = r;
        } else {
          V4<T> p = ld4(a.O2 + g), qv = ld4(a.B + g);
#pragma unroll
          for (int e = 0; e < 4; ++e) x.v[e] = fma(be, fma(-om, qv.v[e], p.v[e]), r.v[e]);
        }
        st4(a.O2 + g, x);
        break;
      }
      case XF_BI_S: {
        V4<T> r = ld4(a.A + g), qv = ld4(a.B + g);
#pragma unroll
        for (int e = 0; e < 4; ++e) x.v[e] = fma(-al, qv.v[e], r.v[e]);
        st4(a.O3 + g, x);
        break;
      }
      default:
        x = ld4(a.A + g);
        break;
    }
    C* row = s + w * a.ld;
    row[phys(2 * q)] = C{x.v[0], x.v[1]};
    row[phys(2 * q + 1)] = C{x.v[2], x.v[3]};
  }
  __syncthreads();
  fft_tile<C, E, false>(s, a.ld, a.fft, tid, a.tfft);
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
  const int lw = __ffs(a.W) - 1;
  for (int idx = tid; idx < a.W * (M + 1); idx += nthr) {
    const int w = idx & (a.W - 1), kx = idx >> lw;
    S1[(long long)kx * a.ny + w] = s[w * a.ld + phys(kx)];
  }
}

// Inverse x pass: transposed load from S1, complex-to-real FFT, epilogue and dots.
template <typename T, int E>
__global__ void __launch_bounds__(512) k_xinv(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  FieldState* st = a.st ? a.st + f : nullptr;
  const bool act = (st ? (st->active != 0) : true) || a.force;
  if (!act && a.ndots == 0) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = a.nx, M = nx >> 1, cpr = nx >> 2;
  const int row0 = blockIdx.x * a.W;
  const int z = row0 / a.ny, y0 = row0 - z * a.ny;
  Acc<T> acc[3];
  if (act) {
    const C* S1 = reinterpret_cast<const C*>(a.S1) + (long long)f * a.SP + (long long)z * a.kxn * a.ny + y0;
    const int lw = __ffs(a.W) - 1;
    for (int idx = tid; idx < a.W * (M + 1); idx += nthr) {
      const int w = idx & (a.W - 1), kx = idx >> lw;
      s[w * a.ld + phys(kx)] = S1[(long long)kx * a.ny + w];
    }
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
    fft_tile<C, E, true>(s, a.ld, a.fft, tid, a.tfft);
    const long long base = (long long)f * a.P + (long long)row0 * nx;
    const T al = st ? T(st->alpha) : T(0), om = st ? T(st->omega) : T(0);
    for (int idx = tid; idx < a.W * cpr; idx += nthr) {
      const int w = fquot(idx, a.rcp_a);
      const int q = idx - w * cpr;
      const long long g = base + (long long)w * nx + 4 * q;
      const C* row = s + w * a.ld;
      const C c0 = row[phys(2 * q)], c1 = row[phys(2 * q + 1)];
      V4<T> y = {{c0.x, c0.y, c1.x, c1.y}};
      switch (a.op) {
        case XI_STORE:
          st4(a.O1 + g, y);
          break;
        case XI_INIT: {
          V4<T> r = ld4(a.A + g);
#pragma unroll
          for (int e = 0; e < 4; ++e) { r.v[e] -= y.v[e]; acc[0].add_prod(r.v[e], r.v[e]); }
          st4(a.O1 + g, r);
          if (a.O2) st4(a.O2 + g, r);
          break;
        }
        case XI_RES: {
          V4<T> r = ld4(a.A + g);
#pragma unroll
          for (int e = 0; e < 4; ++e) { r.v[e] -= y.v[e]; acc[0].add_prod(r.v[e], r.v[e]); }
          break;
        }
        case XI_VC: {
          V4<T> r = ld4(a.O1 + g);
#pragma unroll
          for (int e = 0; e < 4; ++e) { r.v[e] -= y.v[e]; acc[0].add_prod(r.v[e], r.v[e]); }
          st4(a.O1 + g, r);
          break;
        }
        case XI_CG: {
          V4<T> r = ld4(a.O1 + g);
#pragma unroll
          for (int e = 0; e < 4; ++e) { r.v[e] = fma(-al, y.v[e], r.v[e]); acc[0].add_prod(r.v[e], r.v[e]); }
          st4(a.O1 + g, r);
          break;
        }
        case XI_SD: {
          V4<T> r = ld4(a.O1 + g), u = ld4(a.O2 + g);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            u.v[e] = fma(al, r.v[e], u.v[e]);
            r.v[e] = fma(-al, y.v[e], r.v[e]);
            acc[0].add_prod(r.v[e], r.v[e]);
          }
          st4(a.O1 + g, r);
          st4(a.O2 + g, u);
          break;
        }
        case XI_BI_Q: {
          V4<T> f0 = ld4(a.A + g);
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[0].add_prod(f0.v[e], y.v[e]);
          st4(a.O1 + g, y);
          break;
        }
        case XI_BI_T: {
          V4<T> f0 = ld4(a.A + g), p = ld4(a.B + g), sv = ld4(a.C + g), u = ld4(a.O1 + g);
          V4<T> r;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            u.v[e] = fma(om, sv.v[e], fma(al, p.v[e], u.v[e]));
            r.v[e] = fma(-om, y.v[e], sv.v[e]);
            acc[0].add_prod(r.v[e], r.v[e]);
            acc[1].add_prod(f0.v[e], r.v[e]);
          }
          st4(a.O1 + g, u);
          st4(a.O2 + g, r);
          break;
        }
        default:
          break;
      }
    }
  }
  if (a.ndots) block_finish(a, acc, f, act);
}

// Filter pass along the last axis (y in 2D, z in 3D): forward FFT of W
// contiguous sequences, multiply by G_hat(k)/P (with Parseval dots), inverse
// FFT, store back in place.  rcp_a = 1/(L/2), rcp_b = 1/L; in 3D the
// sequence index is kx*ny + ky.
template <typename T, int E>
__global__ void __launch_bounds__(512) k_filt(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  FieldState* st = a.st ? a.st + f : nullptr;
  const bool act = (st ? (st->active != 0) : true) || a.force;
  if (!act && a.ndots == 0) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = a.fft.L, half = L >> 1;
  const bool three_d = a.nz > 1;
  const int nseq = three_d ? a.kxn * a.ny : a.kxn;
  const int seq0 = blockIdx.x * a.W;
  C* S = reinterpret_cast<C*>(three_d ? a.S2 : a.S1) + (long long)f * a.SP + (long long)seq0 * L;
  Acc<T> acc[3];
  if (act) {
    for (int idx = tid; idx < a.W * half; idx += nthr) {
      const int w = fquot(idx, a.rcp_a);
      const int i2 = idx - w * half;
      C v0 = {T(0), T(0)}, v1 = {T(0), T(0)};
      if (seq0 + w < nseq) {
        const C* src = S + (long long)w * L + 2 * i2;
        v0 = src[0];
        v1 = src[1];
      }
      C* row = s + w * a.ld;
      row[phys(2 * i2)] = v0;
      row[phys(2 * i2 + 1)] = v1;
    }
    __syncthreads();
    fft_tile<C, E, false>(s, a.ld, a.fft, tid, a.tfft);
    const int nxh = a.nx >> 1;
    for (int idx = tid; idx < a.W * L; idx += nthr) {
      const int w = fquot(idx, a.rcp_b);
      const int i = idx - w * L;
      const int seq = seq0 + w;
      if (seq >= nseq) continue;
      int kx, k2i;
      const int ki = i < half ? i : i - L;
      if (three_d) {
        kx = seq / a.ny;
        const int kyi = seq - kx * a.ny;
        const int ky = kyi < (a.ny >> 1) ? kyi : kyi - a.ny;
        k2i = kx * kx + ky * ky + ki * ki;
      } else {
        kx = seq;
        k2i = kx * kx + ki * ki;
      }
      const T g = a.kc2 / (a.kc2 + T(k2i));
      C* pv = s + w * a.ld + phys(i);
      C X = *pv;
      if (a.op != FI_NONE) {
        const T wgt = (kx == 0 || kx == nxh) ? T(1) : T(2);
        const T m2 = X.x * X.x + X.y * X.y;
        if (a.op == FI_XGX) {
          acc[0].add(wgt * g * m2);
        } else {
          acc[0].add(wgt * m2);
          acc[1].add(wgt * g * m2);
          acc[2].add(wgt * g * g * m2);
        }
      }
      const T sc = g * a.gscale;
      *pv = C{X.x * sc, X.y * sc};
    }
    __syncthreads();
    fft_tile<C, E, true>(s, a.ld, a.fft, tid, a.tfft);
    for (int idx = tid; idx < a.W * half; idx += nthr) {
      const int w = fquot(idx, a.rcp_a);
      const int i2 = idx - w * half;
      if (seq0 + w >= nseq) continue;
      const C* row = s + w * a.ld;
      C* dst = S + (long long)w * L + 2 * i2;
      dst[0] = row[phys(2 * i2)];
      dst[1] = row[phys(2 * i2 + 1)];
    }
  }
  if (a.ndots) block_finish(a, acc, f, act);
}

// 3D forward y pass: W consecutive z at one kx; load S1 rows [z][kx][:],
// FFT along y, store transposed into S2 [kx][ky][z].  Grid x = kxn * (nz/W).
template <typename T, int E>
__global__ void __launch_bounds__(512) k_yfwd(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  if (a.st && !a.st[f].active && !a.force) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = a.ny, half = L >> 1;
  const int zt = a.nz / a.W;
  const int kx = blockIdx.x / zt, z0 = (blockIdx.x - kx * zt) * a.W;
  const C* S1 = reinterpret_cast<const C*>(a.S1) + (long long)f * a.SP;
  for (int idx = tid; idx < a.W * half; idx += nthr) {
    const int w = fquot(idx, a.rcp_a);
    const int i2 = idx - w * half;
    const C* src = S1 + ((long long)(z0 + w) * a.kxn + kx) * L + 2 * i2;
    C* row = s + w * a.ld;
    row[phys(2 * i2)] = src[0];
    row[phys(2 * i2 + 1)] = src[1];
  }
  __syncthreads();
  fft_tile<C, E, false>(s, a.ld, a.fft, tid, a.tfft);
  C* S2 = reinterpret_cast<C*>(a.S2) + (long long)f * a.SP + (long long)kx * L * a.nz + z0;
  const int lw = __ffs(a.W) - 1;
  for (int idx = tid; idx < a.W * L; idx += nthr) {
    const int w = idx & (a.W - 1), ky = idx >> lw;
    S2[(long long)ky * a.nz + w] = s[w * a.ld + phys(ky)];
  }
}

// 3D inverse y pass: transposed load from S2, inverse FFT along y, rows back to S1.
template <typename T, int E>
__global__ void __launch_bounds__(512) k_yinv(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = blockIdx.y;
  if (a.st && !a.st[f].active && !a.force) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = a.ny, half = L >> 1;
  const int zt = a.nz / a.W;
  const int kx = blockIdx.x / zt, z0 = (blockIdx.x - kx * zt) * a.W;
  const C* S2 = reinterpret_cast<const C*>(a.S2) + (long long)f * a.SP + (long long)kx * L * a.nz + z0;
  const int lw = __ffs(a.W) - 1;
  for (int idx = tid; idx < a.W * L; idx += nthr) {
    const int w = idx & (a.W - 1), ky = idx >> lw;
    s[w * a.ld + phys(ky)] = S2[(long long)ky * a.nz + w];
  }
  __syncthreads();
  fft_tile<C, E, true>(s, a.ld, a.fft, tid, a.tfft);
  C* S1 = reinterpret_cast<C*>(a.S1) + (long long)f * a.SP;
  for (int idx = tid; idx < a.W * half; idx += nthr) {
    const int w = fquot(idx, a.rcp_a);
    const int i2 = idx - w * half;
    C* dst = S1 + ((long long)(z0 + w) * a.kxn + kx) * L + 2 * i2;
    const C* row = s + w * a.ld;
    dst[0] = row[phys(2 * i2)];
    dst[1] = row[phys(2 * i2 + 1)];
  }
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
