// Spectral-space Krylov iteration. On the periodic grid G is diagonal in
// Fourier space (Section 4, Eq. df2: G_hat(k) = 1/(1 + |k|^2/k_c^2)), so
// Algorithms 1-4 can run on the half spectra of their vectors: G is a
// pointwise multiply, inner products are Parseval sums
//   (a, b) = (1/P) sum_{kx = 0..nx/2} w(kx) sum_{ky, kz} Re(a_hat conj(b_hat)),
//   w = 1 for kx = 0 and kx = nx/2, 2 otherwise,
// and the iterates equal the physical-space ones in exact arithmetic. u_bar
// is transformed once before the loop and u once after it (k_lfwd, k_linv
// finish the axis-by-axis transform of the x and y passes).
//
// Spectral vectors use the layout the last-axis transform produces: 2D
// [kx][ky] (sequence kx, length ny), 3D [kx][ky][kz] (sequence kx*ny + ky,
// length nz); element (seq, k) of field f at f*SP + seq*L + k.
#pragma once

#include "passes.cuh"

namespace gad {

// Forward FFT along the last axis: the tile's sequences are read from S1
// (2D) or S2 (3D) and written to the spectral vector O1, unscaled.
template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_lfwd(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = field_of(a), tid = threadIdx.x;
  const int L = a.fft.L;
  const bool three_d = a.nz > 1;
  const int nseq = three_d ? a.kxn * a.ny : a.kxn;
  const int seq0 = blockIdx.x * a.W;
  const int nvalid = min(a.W, nseq - seq0);
  const C* S = reinterpret_cast<const C*>(three_d ? a.S2 : a.S1) + (long long)f * a.SP + (long long)seq0 * L;
  C* O = reinterpret_cast<C*>(a.O1) + (long long)f * a.SP + (long long)seq0 * L;
  auto load = [&](int w, int i) -> C { return w < nvalid ? S[(long long)w * L + i] : C{T(0), T(0)}; };
  auto emit = [&](int w, int i, const C& x) {
    if (w < nvalid) O[(long long)w * L + i] = x;
  };
  fft_run<C, E, false>(s, a.ld, a.fft, tid, a.tfft, load, emit, false, false);
}

// Inverse FFT along the last axis: the spectral vector A, scaled by 1/P, is
// transformed into S1 (2D) or S2 (3D) for the inverse y and x passes.
template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_linv(PassArgs<T> a) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = field_of(a), tid = threadIdx.x;
  const int L = a.fft.L;
  const bool three_d = a.nz > 1;
  const int nseq = three_d ? a.kxn * a.ny : a.kxn;
  const int seq0 = blockIdx.x * a.W;
  const int nvalid = min(a.W, nseq - seq0);
  const C* X = reinterpret_cast<const C*>(a.A) + (long long)f * a.SP + (long long)seq0 * L;
  C* S = reinterpret_cast<C*>(three_d ? a.S2 : a.S1) + (long long)f * a.SP + (long long)seq0 * L;
  const T gs = a.gscale;
  auto load = [&](int w, int i) -> C {
    if (w >= nvalid) return C{T(0), T(0)};
    const C x = X[(long long)w * L + i];
    return C{x.x * gs, x.y * gs};
  };
  auto emit = [&](int w, int i, const C& x) {
    if (w < nvalid) S[(long long)w * L + i] = x;
  };
  fft_run<C, E, true>(s, a.ld, a.fft, tid, a.tfft, load, emit, false, false);
}

__device__ __forceinline__ float sinpi_t(float x) { return sinpif(x); }
__device__ __forceinline__ double sinpi_t(double x) { return sinpi(x); }

// Inputs of one element pair (two complex values = four reals) of a spectral pass.
template <typename T>
struct SpIn {
  V4<T> a, b, o1, o2;
};

template <typename T, int OP>
__device__ __forceinline__ void sp_load(SpIn<T>& x, const T* __restrict__ vA, const T* __restrict__ vB,
                                        const T* vO1, const T* vO2, long long o, bool first) {
  switch (OP) {
    case SP_REF: x.a = ld4(vA + o); break;
    case SP_INIT: case SP_PCG_INIT: x.a = ld4(vA + o); if (vB) x.b = ld4(vB + o); break;
    case SP_PCG_P: x.a = ld4(vA + o); if (!first) x.o1 = ld4(vO1 + o); break;
    case SP_PCG: x.a = ld4(vA + o); x.o1 = ld4(vO1 + o); x.o2 = ld4(vO2 + o); break;
    case SP_VC: case SP_SD: x.o1 = ld4(vO1 + o); x.o2 = ld4(vO2 + o); break;
    case SP_SD_A: x.a = ld4(vA + o); break;
    case SP_CG_P: x.a = ld4(vA + o); if (!first) x.o1 = ld4(vO1 + o); break;
    case SP_CG: x.a = ld4(vA + o); x.o1 = ld4(vO1 + o); x.o2 = ld4(vO2 + o); break;
    case SP_BI_P: x.a = ld4(vA + o); x.b = ld4(vB + o); if (!first) x.o1 = ld4(vO1 + o); break;
    case SP_BI_S: x.a = ld4(vA + o); x.b = ld4(vB + o); break;
    case SP_BI_END: x.a = ld4(vA + o); x.b = ld4(vB + o); x.o1 = ld4(vO1 + o); x.o2 = ld4(vO2 + o); break;
    default: break;
  }
}

// Updates of one element pair and its dot terms; d[k] receives the pair's
// sum of the k-th inner product (four FMA-formed products, weight applied).
template <typename T, int OP>
__device__ __forceinline__ void sp_compute(SpIn<T>& x, const T* g, const T* mh, T wgt, T al, T be, T om, bool first,
                                           bool has_b, T* d) {
  d[0] = d[1] = d[2] = T(0);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    switch (OP) {
      case SP_REF: {
        const T r = fma(-g[e], x.a.v[e], x.a.v[e]);
        d[0] = fma(r, r, d[0]);
        break;
      }
      case SP_INIT: {
        const T xv = has_b ? x.b.v[e] : x.a.v[e];
        const T r = fma(-g[e], xv, x.a.v[e]);
        x.o2.v[e] = r;
        d[0] = fma(r, r, d[0]);
        break;
      }
      case SP_PCG_INIT: {
        const T xv = has_b ? x.b.v[e] : x.a.v[e];
        const T r = fma(-g[e], xv, x.a.v[e]);
        x.o2.v[e] = r;
        d[0] = fma(r, r, d[0]);
        d[1] = fma(r, mh[e] * r, d[1]);
        break;
      }
      case SP_PCG_P: {                            // z = M r; p = z (first) or z + beta p
        const T z = mh[e] * x.a.v[e];
        const T p = first ? z : fma(be, x.o1.v[e], z);
        x.o1.v[e] = p;
        d[0] = fma(p, g[e] * p, d[0]);
        break;
      }
      case SP_PCG: {                              // u += alpha p; r -= alpha G p
        x.o1.v[e] = fma(al, x.a.v[e], x.o1.v[e]);
        const T r = fma(-al, g[e] * x.a.v[e], x.o2.v[e]);
        x.o2.v[e] = r;
        d[0] = fma(r, r, d[0]);
        d[1] = fma(r, mh[e] * r, d[1]);
        break;
      }
      case SP_VC: {
        x.o1.v[e] += x.o2.v[e];
        x.o2.v[e] = fma(-g[e], x.o2.v[e], x.o2.v[e]);
        d[0] = fma(x.o2.v[e], x.o2.v[e], d[0]);
        break;
      }
      case SP_SD_A:
        d[0] = fma(x.a.v[e], g[e] * x.a.v[e], d[0]);
        break;
      case SP_SD: {
        x.o1.v[e] = fma(al, x.o2.v[e], x.o1.v[e]);
        x.o2.v[e] = fma(-al, g[e] * x.o2.v[e], x.o2.v[e]);
        d[0] = fma(x.o2.v[e], x.o2.v[e], d[0]);
        break;
      }
      case SP_CG_P: {
        const T p = first ? x.a.v[e] : fma(be, x.o1.v[e], x.a.v[e]);
        x.o1.v[e] = p;
        d[0] = fma(p, g[e] * p, d[0]);
        break;
      }
      case SP_CG: {
        x.o1.v[e] = fma(al, x.a.v[e], x.o1.v[e]);
        x.o2.v[e] = fma(-al, g[e] * x.a.v[e], x.o2.v[e]);
        d[0] = fma(x.o2.v[e], x.o2.v[e], d[0]);
        break;
      }
      case SP_BI_P: {
        const T p = first ? x.a.v[e] : fma(be, fma(-om, g[e] * x.o1.v[e], x.o1.v[e]), x.a.v[e]);
        x.o1.v[e] = p;
        d[0] = fma(x.b.v[e], g[e] * p, d[0]);
        break;
      }
      case SP_BI_S: {
        const T s = fma(-al, g[e] * x.b.v[e], x.a.v[e]);
        const T t = g[e] * s;
        d[0] = fma(s, s, d[0]);
        d[1] = fma(s, t, d[1]);
        d[2] = fma(t, t, d[2]);
        break;
      }
      case SP_BI_END: {
        const T s = fma(-al, g[e] * x.a.v[e], x.o2.v[e]);
        const T t = g[e] * s;
        x.o1.v[e] = fma(om, s, fma(al, x.a.v[e], x.o1.v[e]));
        x.o2.v[e] = fma(-om, t, s);
        d[0] = fma(x.o2.v[e], x.o2.v[e], d[0]);
        d[1] = fma(x.b.v[e], x.o2.v[e], d[1]);
        break;
      }
      default:
        break;
    }
  }
  d[0] *= wgt;
  d[1] *= wgt;
  d[2] *= wgt;
}

template <typename T, int OP>
__device__ __forceinline__ void sp_store(const SpIn<T>& x, const T* vB, T* vO1, T* vO2, T* vO3, long long o) {
  switch (OP) {
    case SP_INIT: case SP_PCG_INIT:
      if (vO1) st4(vO1 + o, x.a);
      st4(vO2 + o, x.o2);
      if (vO3) st4(vO3 + o, x.o2);
      break;
    case SP_VC: case SP_SD: case SP_CG: case SP_BI_END: case SP_PCG: st4(vO1 + o, x.o1); st4(vO2 + o, x.o2); break;
    case SP_CG_P: case SP_BI_P: case SP_PCG_P: st4(vO1 + o, x.o1); break;
    default: break;
  }
}

// One spectral-space pass of a Krylov method (opcode OP), fused vector
// updates and up to three Parseval dots, then the per-field scalar
// recurrence in the last block of each field (block_finish). Each block
// streams a contiguous range of sequences; a thread takes two element pairs
// (two complex values each) per step, loading all their inputs before any
// arithmetic, with K = 256/(L/2) sequences per step when a sequence is
// shorter than the block. Dot terms: the four products of an element pair
// are summed with FMAs, and the pairs' sums are accumulated with TwoSum.
template <typename T, int OP>
__global__ void __launch_bounds__(256) k_spec(PassArgs<T> a) {
  const int f = field_of(a), tid = threadIdx.x;
  if (a.clear_cond && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) cudaGraphSetConditional(a.cond, 0u);
  FieldState* st = a.st + f;
  const bool act = st->active != 0 || a.force;
  Acc<T> acc[3];
  if (act) {
    const bool three_d = a.nz > 1;
    const int L = three_d ? a.nz : a.ny;
    const int H = L >> 1;                               // element pairs per sequence
    const long long nrows = a.SP / L;
    const long long r0 = nrows * blockIdx.x / gridDim.x, r1 = nrows * (blockIdx.x + 1) / gridDim.x;
    const int K = H >= 256 ? 1 : 256 / H;
    const int ro = H >= 256 ? 0 : tid / H;
    const int c0 = H >= 256 ? tid : tid - ro * H;
    const int cstep = H >= 256 ? 256 : H;
    if (ro < K) {
      const bool first = st->iter == 0;
      const T al = T(st->alpha), be = T(st->beta), om = T(st->omega);
      const T kc2 = a.kc2;
      const int nxh = a.nx >> 1, ny = a.ny, hl = L >> 1;
      const long long fo = (long long)f * a.SP * 2;
      const T* __restrict__ vA = a.A;
      const T* __restrict__ vB = a.B;
      T* __restrict__ vO1 = a.O1;
      T* __restrict__ vO2 = a.O2;
      T* __restrict__ vO3 = a.O3;
      const bool has_b = vB != nullptr;
      auto gpair = [&](int c, int k2r, T* g) {
        const int ka = 2 * c < hl ? 2 * c : 2 * c - L;
        const int kb = 2 * c + 1 < hl ? 2 * c + 1 : 2 * c + 1 - L;
        g[0] = g[1] = ghat(kc2, T(k2r + ka * ka));
        g[2] = g[3] = ghat(kc2, T(k2r + kb * kb));
      };
      // preconditioned CG: M_hat(k) = 1 + sum_d 4 c_d sin^2(pi k_d / N_d), the
      // symbol of the periodic finite-difference inverse of G
      constexpr bool pcg = OP == SP_PCG_INIT || OP == SP_PCG_P || OP == SP_PCG;
      const T cl = three_d ? a.cz : a.cy;
      auto mpair = [&](int c, T mrow, T* m) {
        const T sa = sinpi_t(T(2 * c) / T(L)), sb = sinpi_t(T(2 * c + 1) / T(L));
        m[0] = m[1] = T(1) + mrow + T(4) * cl * sa * sa;
        m[2] = m[3] = T(1) + mrow + T(4) * cl * sb * sb;
      };
      for (long long row = r0 + ro; row < r1; row += K) {
        int kx, k2r;
        if (three_d) {
          kx = (int)(row / ny);
          const int kyi = (int)(row - (long long)kx * ny);
          const int ky = kyi < (ny >> 1) ? kyi : kyi - ny;
          k2r = kx * kx + ky * ky;
        } else {
          kx = (int)row;
          k2r = kx * kx;
        }
        const T wgt = (kx == 0 || kx == nxh) ? T(1) : T(2);
        T mrow = T(0);
        if constexpr (pcg) {
          const T sx = sinpi_t(T(kx) / T(a.nx));
          mrow = T(4) * a.cx * sx * sx;
          if (three_d) {
            const T sy = sinpi_t(T(row - (long long)kx * ny) / T(ny));
            mrow += T(4) * a.cy * sy * sy;
          }
        }
        const long long rb = fo + row * L * 2;
        int c = c0;
        for (; c + cstep < H; c += 2 * cstep) {           // two element pairs per step
          SpIn<T> x0, x1;
          const long long o0 = rb + 4LL * c, o1 = rb + 4LL * (c + cstep);
          sp_load<T, OP>(x0, vA, vB, vO1, vO2, o0, first);
          sp_load<T, OP>(x1, vA, vB, vO1, vO2, o1, first);
          T g0[4], g1[4], m0[4], m1[4], d0[3], d1[3];
          gpair(c, k2r, g0);
          gpair(c + cstep, k2r, g1);
          if constexpr (pcg) {
            mpair(c, mrow, m0);
            mpair(c + cstep, mrow, m1);
          }
          sp_compute<T, OP>(x0, g0, m0, wgt, al, be, om, first, has_b, d0);
          sp_compute<T, OP>(x1, g1, m1, wgt, al, be, om, first, has_b, d1);
          sp_store<T, OP>(x0, vB, vO1, vO2, vO3, o0);
          sp_store<T, OP>(x1, vB, vO1, vO2, vO3, o1);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            acc[k].add(d0[k]);
            acc[k].add(d1[k]);
          }
        }
        if (c < H) {
          SpIn<T> x0;
          const long long o0 = rb + 4LL * c;
          sp_load<T, OP>(x0, vA, vB, vO1, vO2, o0, first);
          T g0[4], m0[4], d0[3];
          gpair(c, k2r, g0);
          if constexpr (pcg) mpair(c, mrow, m0);
          sp_compute<T, OP>(x0, g0, m0, wgt, al, be, om, first, has_b, d0);
          sp_store<T, OP>(x0, vB, vO1, vO2, vO3, o0);
#pragma unroll
          for (int k = 0; k < 3; ++k) acc[k].add(d0[k]);
        }
      }
    }
  }
  block_finish(a, acc, f, act);
}

template <typename T>
cudaError_t launch_spec(dim3 grid, cudaStream_t s, const PassArgs<T>& a) {
  switch (a.op) {
    case SP_REF: k_spec<T, SP_REF><<<grid, 256, 0, s>>>(a); break;
    case SP_INIT: k_spec<T, SP_INIT><<<grid, 256, 0, s>>>(a); break;
    case SP_VC: k_spec<T, SP_VC><<<grid, 256, 0, s>>>(a); break;
    case SP_SD_A: k_spec<T, SP_SD_A><<<grid, 256, 0, s>>>(a); break;
    case SP_SD: k_spec<T, SP_SD><<<grid, 256, 0, s>>>(a); break;
    case SP_CG_P: k_spec<T, SP_CG_P><<<grid, 256, 0, s>>>(a); break;
    case SP_CG: k_spec<T, SP_CG><<<grid, 256, 0, s>>>(a); break;
    case SP_BI_P: k_spec<T, SP_BI_P><<<grid, 256, 0, s>>>(a); break;
    case SP_BI_S: k_spec<T, SP_BI_S><<<grid, 256, 0, s>>>(a); break;
    case SP_BI_END: k_spec<T, SP_BI_END><<<grid, 256, 0, s>>>(a); break;
    case SP_PCG_INIT: k_spec<T, SP_PCG_INIT><<<grid, 256, 0, s>>>(a); break;
    case SP_PCG_P: k_spec<T, SP_PCG_P><<<grid, 256, 0, s>>>(a); break;
    case SP_PCG: k_spec<T, SP_PCG><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gad
