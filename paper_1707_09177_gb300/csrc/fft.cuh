// Shared-memory Stockham FFT building blocks for the filter passes.
//
// The filter G of the approximate-deconvolution problem is diagonal in
// Fourier space (Section 4, Eq. df2), so every application of G is a
// forward real FFT, a pointwise multiply and an inverse real FFT. These
// helpers run one axis of such a transform for a tile of W independent
// sequences held in shared memory.
//
// Shared-memory layout of a tile: sequence w occupies a row that starts at
// w*ld (ld odd, in complex units); element i of the row lives at
// phys(i) = i + i/16 (one pad slot every 16 elements). The pad makes the
// power-of-two strides of the Stockham write pattern bank-conflict free, the
// odd row stride makes column-wise (transposed) access conflict free.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "args.h"

namespace gad {

template <typename T> struct cpx;
template <> struct cpx<float> { using t = float2; };
template <> struct cpx<double> { using t = double2; };

__host__ __device__ __forceinline__ int phys(int i) { return i + (i >> 4); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return {a.x, -a.y}; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C cmi(C a) {
  return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { return {a.x * s, a.y * s}; }

// --- small DFTs in registers (forward: exp(-2 pi i nk/R), inverse: +) ---
template <bool INV, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = cmi<INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft3(C& a0, C& a1, C& a2) {
  using S = decltype(a0.x);
  const S h = S(0.86602540378443864676372317075294);  // sqrt(3)/2
  C t = cadd(a1, a2), d = csub(a1, a2);
  C m = {a0.x - S(0.5) * t.x, a0.y - S(0.5) * t.y};
  a0 = cadd(a0, t);
  C j = cscale(cmi<INV>(d), h);  // (-+ i) sqrt(3)/2 (a1 - a2)
  a1 = cadd(m, j);
  a2 = csub(m, j);
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C* a) {
  using S = decltype(a[0].x);
  const S r = S(0.70710678118654752440084436210485);
  dft4<INV>(a[0], a[2], a[4], a[6]);
  dft4<INV>(a[1], a[3], a[5], a[7]);
  // odd half times W8^k, k = 0..3
  C o1 = a[3], o2 = a[5], o3 = a[7];
  o1 = INV ? C{(o1.x - o1.y) * r, (o1.x + o1.y) * r} : C{(o1.x + o1.y) * r, (o1.y - o1.x) * r};
  o2 = cmi<INV>(o2);
  o3 = INV ? C{-(o3.x + o3.y) * r, (o3.x - o3.y) * r} : C{(o3.y - o3.x) * r, -(o3.x + o3.y) * r};
  C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  a[0] = cadd(e0, a[1]);
  a[4] = csub(e0, a[1]);
  a[1] = cadd(e1, o1);
  a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2);
  a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3);
  a[7] = csub(e3, o3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft16(C* a) {
  using S = decltype(a[0].x);
  // n = 4 n1 + n2, k = k1 + 4 k2: inner 4-point DFTs over n1, twiddle
  // W16^(n2 k1), outer 4-point DFTs over n2.
  C b[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C x0 = a[n2], x1 = a[4 + n2], x2 = a[8 + n2], x3 = a[12 + n2];
    dft4<INV>(x0, x1, x2, x3);
    b[n2 * 4 + 0] = x0;
    b[n2 * 4 + 1] = x1;
    b[n2 * 4 + 2] = x2;
    b[n2 * 4 + 3] = x3;
  }
  const S c1 = S(0.92387953251128675612818318939679);   // cos(pi/8)
  const S s1 = S(0.38268343236508977172845998403040);   // sin(pi/8)
  const S r2 = S(0.70710678118654752440084436210485);
  const S sg = INV ? S(1) : S(-1);
  // W16^m = cos(m pi/8) + sg i sin(m pi/8)
  const C w1 = {c1, sg * s1}, w2 = {r2, sg * r2}, w3 = {s1, sg * c1};
  const C w6 = {-r2, sg * r2}, w9 = {-c1, -sg * s1};
  b[1 * 4 + 1] = cmul(b[1 * 4 + 1], w1);
  b[1 * 4 + 2] = cmul(b[1 * 4 + 2], w2);
  b[1 * 4 + 3] = cmul(b[1 * 4 + 3], w3);
  b[2 * 4 + 1] = cmul(b[2 * 4 + 1], w2);
  b[2 * 4 + 2] = cmi<INV>(b[2 * 4 + 2]);   // W16^4
  b[2 * 4 + 3] = cmul(b[2 * 4 + 3], w6);
  b[3 * 4 + 1] = cmul(b[3 * 4 + 1], w3);
  b[3 * 4 + 2] = cmul(b[3 * 4 + 2], w6);
  b[3 * 4 + 3] = cmul(b[3 * 4 + 3], w9);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C x0 = b[0 * 4 + k1], x1 = b[1 * 4 + k1], x2 = b[2 * 4 + k1], x3 = b[3 * 4 + k1];
    dft4<INV>(x0, x1, x2, x3);
    a[k1 + 0] = x0;
    a[k1 + 4] = x1;
    a[k1 + 8] = x2;
    a[k1 + 12] = x3;
  }
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft(C* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
}

// exact small-integer quotient for q < 2^20: floor((x + 0.5) * rcp)
__device__ __forceinline__ int fquot(int x, float rcp) { return __float2int_rz((float(x) + 0.5f) * rcp); }

// Shared-memory row accessors for the inner stages.
template <typename C>
struct SmemRows {
  C* s;
  int ld;
  __device__ __forceinline__ C operator()(int w, int i) const { return s[w * ld + phys(i)]; }
  __device__ __forceinline__ void operator()(int w, int i, const C& x) const { s[w * ld + phys(i)] = x; }
};

template <class X> struct is_rows { static constexpr bool value = false; };
template <class C> struct is_rows<SmemRows<C>> { static constexpr bool value = true; };

// A run of R elements i0 + r*st (r < R) of one shared-memory row has a
// constant padded stride when st is a multiple of 16 (phys stride st + st/16)
// or when st = 1 and the run stays inside one 16-element block (R divides 16
// and i0 is a multiple of R): then phys(i0 + r*st) = phys(i0) + r*pst and the
// stage addresses its R elements with one add each instead of recomputing
// phys() per element. Returns pst, or 0 when the stride is not constant.
template <int R>
__device__ __forceinline__ int run_stride(int st) {
  if ((st & 15) == 0) return st + (st >> 4);
  if (st == 1 && (16 % R) == 0) return 1;
  return 0;
}

// One radix-R Stockham stage over the whole tile. Every thread owns E/R
// butterflies; all inputs are held in registers before any output is
// written, so a stage may overwrite its own input.
//   input  index of butterfly (j, r): j + r*L/R
//   output index:                     (j - k)*R + k + r*ns,  k = j mod ns
// `load(w, i)` returns input element i of sequence w and `emit(w, i, x)`
// consumes output element i: shared-memory rows for inner stages, global
// memory (with the fused Krylov prologue/epilogue) for the first and last
// stage. `mid_barrier` separates the loads from the writes when both touch
// the same shared-memory tile.
//
// LRC and NSC, when nonzero, are L/R and ns as compile-time constants (powers
// of two): the sequence and sub-transform indices become shifts and masks and
// the shared-memory runs get immediate offsets. They must equal the plan's
// values (fft_run_fixed checks the plan before taking that path).
template <typename C, int E, int R, bool INV, int LRC = 0, int NSC = 0, class Load, class Emit>
__device__ __forceinline__ void stage_io(int L, const FftStage& sg, const C* __restrict__ tw, int tid, int nthr,
                                         Load& load, Emit& emit, bool mid_barrier) {
  constexpr int NB = E / R;
  static_assert(NB * R == E, "radix must divide the per-thread element count");
  static_assert((LRC & (LRC - 1)) == 0 && (NSC & (NSC - 1)) == 0, "constant strides are powers of two");
  const int lr = LRC ? LRC : L / R;
  const int ns = NSC ? NSC : sg.ns;
  C v[NB][R];
  int wrow[NB], jj[NB];
  const bool on = tid < nthr;     // threads beyond the FFT's thread count only join barriers
  if (on) {
    const int lst = is_rows<Load>::value ? run_stride<R>(lr) : 0;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int bi = tid + b * nthr;
      int w, j;
      if constexpr (LRC > 0) {
        w = (int)((unsigned)bi / (unsigned)LRC);
        j = (int)((unsigned)bi % (unsigned)LRC);
      } else {
        w = fquot(bi, sg.rcp_lr);
        j = bi - w * lr;
      }
      wrow[b] = w;
      jj[b] = j;
      if constexpr (is_rows<Load>::value) {
        if (lst) {
          const C* p = load.s + w * load.ld + phys(j);
#pragma unroll
          for (int r = 0; r < R; ++r) v[b][r] = p[r * lst];
          continue;
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = load(w, j + r * lr);
    }
  }
  if (mid_barrier) __syncthreads();
  if (on) {
    const int est = is_rows<Emit>::value ? run_stride<R>(ns) : 0;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = jj[b];
      int k;
      if constexpr (NSC > 0) k = (int)((unsigned)j % (unsigned)NSC);
      else k = j - ns * fquot(j, sg.rcp_ns);
      if (ns > 1) {
        // factor r of butterfly k at tw_off + (r - 1) ns + k: consecutive
        // threads read consecutive entries
        const C* __restrict__ twk = tw + sg.tw_off + k;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C w = twk[(r - 1) * ns];
          v[b][r] = INV ? cmulc(v[b][r], w) : cmul(v[b][r], w);
        }
      }
      dft<R, INV>(v[b]);
      const int o = (j - k) * R + k;
      if constexpr (is_rows<Emit>::value) {
        if (est) {
          C* p = emit.s + wrow[b] * emit.ld + phys(o);
#pragma unroll
          for (int r = 0; r < R; ++r) p[r * est] = v[b][r];
          continue;
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) emit(wrow[b], o + r * ns, v[b][r]);
    }
  }
}

// Last forward stage, pointwise spectral multiply, and first inverse stage
// of the same radix, without leaving registers. The last forward stage
// (ns = L/R) leaves butterfly j holding X[j + r*L/R] in natural order; an
// inverse plan whose first radix is R reads exactly those elements for its
// butterfly j (ns = 1, no twiddles), so the multiply happens in between.
// `mul(w, i, x)` scales element i and may accumulate inner products;
// `emit(w, i, x)` consumes the inverse stage's outputs (index j*R + r).
// LRC as in stage_io.
template <typename C, int E, int R, int LRC = 0, class Load, class Mul, class Emit>
__device__ __forceinline__ void stage_filter(int L, const FftStage& sg, const C* __restrict__ tw, int tid, int nthr,
                                             Load& load, Mul& mul, Emit& emit, bool mid_barrier) {
  constexpr int NB = E / R;
  static_assert(NB * R == E, "radix must divide the per-thread element count");
  static_assert((LRC & (LRC - 1)) == 0, "constant strides are powers of two");
  const int lr = LRC ? LRC : L / R;
  C v[NB][R];
  int wrow[NB], jj[NB];
  const bool on = tid < nthr;
  if (on) {
    const int lst = is_rows<Load>::value ? run_stride<R>(lr) : 0;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int bi = tid + b * nthr;
      int w, j;
      if constexpr (LRC > 0) {
        w = (int)((unsigned)bi / (unsigned)LRC);
        j = (int)((unsigned)bi % (unsigned)LRC);
      } else {
        w = fquot(bi, sg.rcp_lr);
        j = bi - w * lr;
      }
      wrow[b] = w;
      jj[b] = j;
      if constexpr (is_rows<Load>::value) {
        if (lst) {
          const C* p = load.s + w * load.ld + phys(j);
#pragma unroll
          for (int r = 0; r < R; ++r) v[b][r] = p[r * lst];
          continue;
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = load(w, j + r * lr);
    }
  }
  if (mid_barrier) __syncthreads();
  if (on) {
    const int est = is_rows<Emit>::value ? run_stride<R>(1) : 0;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = jj[b];                  // k = j: ns = L/R exceeds every j
      if (lr > 1) {
        const C* __restrict__ twk = tw + sg.tw_off + j;     // ns = L/R = lr for the last stage
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], twk[(r - 1) * lr]);
      }
      dft<R, false>(v[b]);
#pragma unroll
      for (int r = 0; r < R; ++r) mul(wrow[b], j + r * lr, v[b][r]);
      dft<R, true>(v[b]);
      if constexpr (is_rows<Emit>::value) {
        if (est) {
          C* p = emit.s + wrow[b] * emit.ld + phys(j * R);
#pragma unroll
          for (int r = 0; r < R; ++r) p[r] = v[b][r];
          continue;
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) emit(wrow[b], j * R + r, v[b][r]);
    }
  }
}

// Stage q of a plan that lives in kernel-parameter space. Constant indices
// only: a runtime index into a parameter array would force a local-memory
// copy of the whole plan.
__device__ __forceinline__ FftStage stage_at(const FftPlan& p, int q) {
  switch (q) {
    case 0: return p.st[0];
    case 1: return p.st[1];
    case 2: return p.st[2];
    case 3: return p.st[3];
    case 4: return p.st[4];
    case 5: return p.st[5];
    case 6: return p.st[6];
    default: return p.st[7];
  }
}

// Runtime radix -> compile-time stage.
template <typename C, int E, bool INV, class Load, class Emit>
__device__ __forceinline__ void stage_dispatch(int L, const FftStage& sg, const C* __restrict__ tw, int tid, int nthr,
                                               Load& load, Emit& emit, bool mid_barrier) {
  switch (sg.radix) {
    case 2: if constexpr (E % 2 == 0) stage_io<C, E, 2, INV>(L, sg, tw, tid, nthr, load, emit, mid_barrier); break;
    case 3: if constexpr (E % 3 == 0) stage_io<C, E, 3, INV>(L, sg, tw, tid, nthr, load, emit, mid_barrier); break;
    case 4: if constexpr (E % 4 == 0) stage_io<C, E, 4, INV>(L, sg, tw, tid, nthr, load, emit, mid_barrier); break;
    case 8: if constexpr (E % 8 == 0) stage_io<C, E, 8, INV>(L, sg, tw, tid, nthr, load, emit, mid_barrier); break;
    case 16: if constexpr (E % 16 == 0) stage_io<C, E, 16, INV>(L, sg, tw, tid, nthr, load, emit, mid_barrier); break;
    default: break;
  }
}

template <typename C, int E, class Load, class Mul, class Emit>
__device__ __forceinline__ void filter_dispatch(int L, const FftStage& sg, const C* __restrict__ tw, int tid, int nthr,
                                                Load& load, Mul& mul, Emit& emit, bool mid_barrier) {
  switch (sg.radix) {
    case 2: if constexpr (E % 2 == 0) stage_filter<C, E, 2>(L, sg, tw, tid, nthr, load, mul, emit, mid_barrier); break;
    case 3: if constexpr (E % 3 == 0) stage_filter<C, E, 3>(L, sg, tw, tid, nthr, load, mul, emit, mid_barrier); break;
    case 4: if constexpr (E % 4 == 0) stage_filter<C, E, 4>(L, sg, tw, tid, nthr, load, mul, emit, mid_barrier); break;
    case 8: if constexpr (E % 8 == 0) stage_filter<C, E, 8>(L, sg, tw, tid, nthr, load, mul, emit, mid_barrier); break;
    case 16: if constexpr (E % 16 == 0) stage_filter<C, E, 16>(L, sg, tw, tid, nthr, load, mul, emit, mid_barrier); break;
    default: break;
  }
}

// Full transform of every sequence of the tile (natural order in and out),
// plans of at most 5 stages.
// The first stage reads through `load`, the last writes through `emit`; the
// stages in between go through the shared-memory tile. Ends without a
// trailing barrier when the last stage writes elsewhere than the tile.
// nthr is the FFT's logical thread count (W*L/E); the block may be larger.
template <typename C, int E, bool INV, class Load, class Emit>
__device__ __forceinline__ void fft_run(C* s, int ld, const FftPlan& p, int tid, int nthr, Load& load, Emit& emit,
                                        bool load_from_tile, bool emit_to_tile) {
  const C* tw = reinterpret_cast<const C*>(p.tw);
  SmemRows<C> rows{s, ld};
  const int n = p.nst;
  if (n == 1) {
    stage_dispatch<C, E, INV>(p.L, p.st[0], tw, tid, nthr, load, emit, load_from_tile && emit_to_tile);
    if (emit_to_tile) __syncthreads();
    return;
  }
  stage_dispatch<C, E, INV>(p.L, p.st[0], tw, tid, nthr, load, rows, load_from_tile);
  __syncthreads();
  // inner stages, unrolled with constant parameter indices (a loop over the
  // stage index spills the stage's registers to local memory)
  if (n > 2) { stage_dispatch<C, E, INV>(p.L, p.st[1], tw, tid, nthr, rows, rows, true); __syncthreads(); }
  if (n > 3) { stage_dispatch<C, E, INV>(p.L, p.st[2], tw, tid, nthr, rows, rows, true); __syncthreads(); }
  if (n > 4) { stage_dispatch<C, E, INV>(p.L, p.st[3], tw, tid, nthr, rows, rows, true); __syncthreads(); }
  const FftStage sl = stage_at(p, n - 1);
  stage_dispatch<C, E, INV>(p.L, sl, tw, tid, nthr, rows, emit, emit_to_tile);
  if (emit_to_tile) __syncthreads();
}

// Forward transform, multiply, inverse transform (the filter pass). `inv`
// must be the forward plan's radices in reverse order, so that the last
// forward and the first inverse stage meet in registers (stage_filter).
template <typename C, int E, class Load, class Mul, class Emit>
__device__ __forceinline__ void fft_filter_run(C* s, int ld, const FftPlan& fwd, const FftPlan& inv, int tid, int nthr,
                                               Load& load, Mul& mul, Emit& emit) {
  const C* tw = reinterpret_cast<const C*>(fwd.tw);
  const C* twi = reinterpret_cast<const C*>(inv.tw);
  SmemRows<C> rows{s, ld};
  const int n = fwd.nst;
  if (n == 1) {
    filter_dispatch<C, E>(fwd.L, fwd.st[0], tw, tid, nthr, load, mul, emit, false);
    return;
  }
  stage_dispatch<C, E, false>(fwd.L, fwd.st[0], tw, tid, nthr, load, rows, false);
  __syncthreads();
  if (n > 2) { stage_dispatch<C, E, false>(fwd.L, fwd.st[1], tw, tid, nthr, rows, rows, true); __syncthreads(); }
  if (n > 3) { stage_dispatch<C, E, false>(fwd.L, fwd.st[2], tw, tid, nthr, rows, rows, true); __syncthreads(); }
  if (n > 4) { stage_dispatch<C, E, false>(fwd.L, fwd.st[3], tw, tid, nthr, rows, rows, true); __syncthreads(); }
  const FftStage sf = stage_at(fwd, n - 1);
  filter_dispatch<C, E>(fwd.L, sf, tw, tid, nthr, rows, mul, rows, true);
  __syncthreads();
  if (n > 2) { stage_dispatch<C, E, true>(inv.L, inv.st[1], twi, tid, nthr, rows, rows, true); __syncthreads(); }
  if (n > 3) { stage_dispatch<C, E, true>(inv.L, inv.st[2], twi, tid, nthr, rows, rows, true); __syncthreads(); }
  if (n > 4) { stage_dispatch<C, E, true>(inv.L, inv.st[3], twi, tid, nthr, rows, rows, true); __syncthreads(); }
  const FftStage sl = stage_at(inv, n - 1);
  stage_dispatch<C, E, true>(inv.L, sl, twi, tid, nthr, rows, emit, false);
}

// --- fixed plans -----------------------------------------------------------
// The plan the host builds for a power-of-two length L and E elements per
// thread (balanced radices of at most 16 for E = 16, 8 otherwise), as
// compile-time constants: stage q has radix rad(q) and follows sub-transforms
// of size ns(q). REV lists the radices in reverse order (the filter pass's
// inverse plan).
__host__ __device__ constexpr int ct_log2(int L) { return L > 1 ? 1 + ct_log2(L >> 1) : 0; }

template <int L, int E, bool REV>
struct CtPlan {
  static_assert(L > 1 && (L & (L - 1)) == 0, "fixed plans are for powers of two");
  static constexpr int a = ct_log2(L);
  static constexpr int maxlog = (E % 16 == 0) ? 4 : 3;
  static constexpr int n = (a + maxlog - 1) / maxlog;
  __host__ __device__ static constexpr int fwd_rad(int q) { return 1 << (a / n + (q < a % n ? 1 : 0)); }
  __host__ __device__ static constexpr int rad(int q) { return REV ? fwd_rad(n - 1 - q) : fwd_rad(q); }
  __host__ __device__ static constexpr int ns(int q) { return q == 0 ? 1 : ns(q - 1) * rad(q - 1); }
};

// True when plan p is exactly CtPlan<L, E, REV> (length, stage count and
// every radix); the fixed path runs only then.
template <int L, int E, bool REV>
__device__ __forceinline__ bool ct_matches(const FftPlan& p) {
  using P = CtPlan<L, E, REV>;
  if (p.L != L || p.nst != P::n) return false;
  bool ok = true;
  if constexpr (P::n > 0) ok = ok && p.st[0].radix == P::rad(0);
  if constexpr (P::n > 1) ok = ok && p.st[1].radix == P::rad(1);
  if constexpr (P::n > 2) ok = ok && p.st[2].radix == P::rad(2);
  if constexpr (P::n > 3) ok = ok && p.st[3].radix == P::rad(3);
  if constexpr (P::n > 4) ok = ok && p.st[4].radix == P::rad(4);
  return ok && P::n <= 5;
}

template <typename C, int E, bool INV, int L, bool REV, int Q, class Load, class Emit>
__device__ __forceinline__ void ct_stage(const FftPlan& p, const C* __restrict__ tw, int tid, int nthr, Load& load,
                                         Emit& emit, bool mid_barrier) {
  using P = CtPlan<L, E, REV>;
  constexpr int R = P::rad(Q);
  if constexpr (E % R == 0)
    stage_io<C, E, R, INV, L / R, P::ns(Q)>(L, stage_at(p, Q), tw, tid, nthr, load, emit, mid_barrier);
}

// fft_run for a plan known to be CtPlan<L, E, false>.
template <typename C, int E, bool INV, int L, class Load, class Emit>
__device__ __forceinline__ void fft_run_ct(C* s, int ld, const FftPlan& p, int tid, int nthr, Load& load, Emit& emit,
                                           bool load_from_tile, bool emit_to_tile) {
  using P = CtPlan<L, E, false>;
  constexpr int n = P::n;
  const C* tw = reinterpret_cast<const C*>(p.tw);
  SmemRows<C> rows{s, ld};
  if constexpr (n == 1) {
    ct_stage<C, E, INV, L, false, 0>(p, tw, tid, nthr, load, emit, load_from_tile && emit_to_tile);
    if (emit_to_tile) __syncthreads();
  } else {
    ct_stage<C, E, INV, L, false, 0>(p, tw, tid, nthr, load, rows, load_from_tile);
    __syncthreads();
    if constexpr (n > 2) { ct_stage<C, E, INV, L, false, 1>(p, tw, tid, nthr, rows, rows, true); __syncthreads(); }
    if constexpr (n > 3) { ct_stage<C, E, INV, L, false, 2>(p, tw, tid, nthr, rows, rows, true); __syncthreads(); }
    if constexpr (n > 4) { ct_stage<C, E, INV, L, false, 3>(p, tw, tid, nthr, rows, rows, true); __syncthreads(); }
    ct_stage<C, E, INV, L, false, n - 1>(p, tw, tid, nthr, rows, emit, emit_to_tile);
    if (emit_to_tile) __syncthreads();
  }
}

// Runs fft_run's transform through the fixed plan of length L when p is that
// plan (float32 tiles, E = 16) and returns true; returns false, having done
// nothing, otherwise.
template <typename C, int E, bool INV, int L, class Load, class Emit>
__device__ __forceinline__ bool fft_run_fixed(C* s, int ld, const FftPlan& p, int tid, int nthr, Load& load,
                                              Emit& emit, bool load_from_tile, bool emit_to_tile) {
  if constexpr (E == 16 && sizeof(C) == 8) {
    if (ct_matches<L, E, false>(p)) {
      fft_run_ct<C, E, INV, L>(s, ld, p, tid, nthr, load, emit, load_from_tile, emit_to_tile);
      return true;
    }
  }
  return false;
}

// fft_filter_run for plans known to be CtPlan<L, E, false> (forward) and
// CtPlan<L, E, true> (inverse).
template <typename C, int E, int L, class Load, class Mul, class Emit>
__device__ __forceinline__ void fft_filter_run_ct(C* s, int ld, const FftPlan& fwd, const FftPlan& inv, int tid,
                                                  int nthr, Load& load, Mul& mul, Emit& emit) {
  using P = CtPlan<L, E, false>;
  constexpr int n = P::n;
  constexpr int RF = P::rad(n - 1);
  const C* tw = reinterpret_cast<const C*>(fwd.tw);
  const C* twi = reinterpret_cast<const C*>(inv.tw);
  SmemRows<C> rows{s, ld};
  if constexpr (n == 1) {
    stage_filter<C, E, RF, L / RF>(L, fwd.st[0], tw, tid, nthr, load, mul, emit, false);
  } else {
    ct_stage<C, E, false, L, false, 0>(fwd, tw, tid, nthr, load, rows, false);
    __syncthreads();
    if constexpr (n > 2) { ct_stage<C, E, false, L, false, 1>(fwd, tw, tid, nthr, rows, rows, true); __syncthreads(); }
    if constexpr (n > 3) { ct_stage<C, E, false, L, false, 2>(fwd, tw, tid, nthr, rows, rows, true); __syncthreads(); }
    if constexpr (n > 4) { ct_stage<C, E, false, L, false, 3>(fwd, tw, tid, nthr, rows, rows, true); __syncthreads(); }
    stage_filter<C, E, RF, L / RF>(L, stage_at(fwd, n - 1), tw, tid, nthr, rows, mul, rows, true);
    __syncthreads();
    if constexpr (n > 2) { ct_stage<C, E, true, L, true, 1>(inv, twi, tid, nthr, rows, rows, true); __syncthreads(); }
    if constexpr (n > 3) { ct_stage<C, E, true, L, true, 2>(inv, twi, tid, nthr, rows, rows, true); __syncthreads(); }
    if constexpr (n > 4) { ct_stage<C, E, true, L, true, 3>(inv, twi, tid, nthr, rows, rows, true); __syncthreads(); }
    ct_stage<C, E, true, L, true, n - 1>(inv, twi, tid, nthr, rows, emit, false);
  }
}

template <typename C, int E, int L, class Load, class Mul, class Emit>
__device__ __forceinline__ bool fft_filter_run_fixed(C* s, int ld, const FftPlan& fwd, const FftPlan& inv, int tid,
                                                     int nthr, Load& load, Mul& mul, Emit& emit) {
  if constexpr (E == 16 && sizeof(C) == 8) {
    if (ct_matches<L, E, false>(fwd) && ct_matches<L, E, true>(inv)) {
      fft_filter_run_ct<C, E, L>(s, ld, fwd, inv, tid, nthr, load, mul, emit);
      return true;
    }
  }
  return false;
}

}  // namespace gad
