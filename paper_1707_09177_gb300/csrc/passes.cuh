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

// Field of this block. Successive passes alternate the order in which the
// fields' blocks are launched (rev), so that each pass starts on the fields
// whose data the previous pass touched last and may still find in L2.
template <typename A>
__device__ __forceinline__ int field_of(const A& a) {
  return a.rev ? (int)gridDim.y - 1 - (int)blockIdx.y : (int)blockIdx.y;
}

// Block coordinates of a pass: the launch's own (blockIdx, gridDim) when the
// pass runs for one shape, or a block's place in its shape group's launch
// shape when one launch serves several groups (k_multi).
struct VBlock {
  int x, y, nx, ny;
};
__device__ __forceinline__ VBlock own_block() {
  return VBlock{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x, (int)gridDim.y};
}
template <typename A>
__device__ __forceinline__ int field_of(const A& a, const VBlock& vb) {
  return a.rev ? vb.ny - 1 - vb.y : vb.y;
}

// G_hat(k) = k_c^2/(k_c^2 + |k|^2). float32: reciprocal-based quotient
// (__fdividef, within 2 ulp; the spectra are stored in float32 anyway);
// float64: IEEE division.
__device__ __forceinline__ float ghat(float kc2, float k2) { return __fdividef(kc2, kc2 + k2); }
__device__ __forceinline__ double ghat(double kc2, double k2) { return kc2 / (kc2 + k2); }

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
  if (s.fault) {                 // a bounded wait of this field gave up: its dots are incomplete
    s.status = -4; s.active = 0; // AD_ERR_TIMEOUT
    return;
  }
  switch (stage) {
    case SS_REF:
      s.ref = sqrt(fmax(d[0], 0.0));
      s.have_ref = 1;
      break;
    case SS_INIT:
    case SS_PCG_INIT: {
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
      if (stage == SS_PCG_INIT && s.active) {
        s.rho = d[1];                             // rho_0 = (r_0, z_0)
        if (!(d[1] > 0.0) || !finite_d(d[1])) { s.status = 2; s.active = 0; }
      }
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
    case SS_PCG_RHO: {           // rho_{n+1} = (r_{n+1}, z_{n+1}); beta_n = rho_{n+1} / rho_n
      const double rz = d[0];
      if (!(rz > 0.0) || !finite_d(rz)) {
        s.status = 2; s.active = 0;                // AD_BREAKDOWN
        if (s.iter > 0) s.fin_axpy = 1;            // u += alpha p of the last pass is still owed
      } else if (s.iter == 0) {
        s.rho = rz;
      } else {
        s.beta = rz / s.rho;
        s.rho = rz;
      }
      break;
    }
    case SS_PCG_STOP:
      stop_or_continue(s, cfg, f, d[0]);
      if (!s.active) s.fin_axpy = 1;
      break;
    case SS_PCG_END: {           // stop test on (r, r); then rho_{n+1} = (r, z), beta_n
      stop_or_continue(s, cfg, f, d[0]);
      if (s.active) {
        const double rz = d[1];
        if (!(rz > 0.0) || !finite_d(rz)) { s.status = 2; s.active = 0; }
        else { s.beta = rz / s.rho; s.rho = rz; }
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

// A sum carried as an unevaluated pair of floats (hi + lo): TwoSum of the
// high parts, the low parts and the rounding error added and the pair
// renormalised. About twice float32 precision with float32 arithmetic: the
// block reductions of the float32 dots use it instead of float64, whose rate
// on this GPU is a small fraction of float32's.
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bp = s - a.x;
  const float e = (a.x - (s - bp)) + (b.x - bp);
  const float t = e + (a.y + b.y);
  const float hi = s + t;
  return make_float2(hi, t - (hi - s));
}

__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float2 w;
    w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    v = pair_add(v, w);
  }
  return v;
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
__device__ void block_finish(const PassArgs<T>& a, const Acc<T>* acc, int f, bool act, const VBlock& vb) {
  __shared__ double red[32][3];
  __shared__ int last_field;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the block size of the pass's own launch shape (a k_multi block may be
  // larger: its extra threads hold no terms), so that the reduction order,
  // and with it every rounding, is the same in both kinds of launch
  const int nthr = a.vbd ? a.vbd : (int)blockDim.x;
  const int nw = (nthr + 31) >> 5;
  const int nblk = vb.nx;
  if (act) {
    if constexpr (sizeof(T) == 4) {
      // float32 dots: the thread's compensated pair, reduced as float pairs
      __shared__ float2 redf[32][3];
      float2 v[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float hi = acc[d].s + acc[d].c;
        v[d] = warp_sum(make_float2(hi, acc[d].c - (hi - acc[d].s)));
      }
      if (lane == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) redf[warp][d] = v[d];
      }
      __syncthreads();
      if (warp == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          float2 t = lane < nw ? redf[lane][d] : make_float2(0.f, 0.f);
          t = warp_sum(t);
          if (lane == 0) a.part[((long long)f * nblk + vb.x) * 4 + d] = ((double)t.x + (double)t.y) * a.inv_p;
        }
      }
    } else {
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
          if (lane == 0) a.part[((long long)f * nblk + vb.x) * 4 + d] = t * a.inv_p;
        }
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
    for (int b = tid; b < nblk && tid < nthr; b += nthr) {
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
    // fields done: those of this launch, or, when one sequence of launches
    // serves several shape groups, those of every group (MultiState)
    unsigned* done = a.ms ? a.ms->ticket : a.ticket;
    const unsigned nfields = a.ms ? (unsigned)a.ms->nfields : (unsigned)vb.ny;
    const unsigned prevg = atomicAdd(done, 1u);
    if (prevg == nfields - 1u) {                          // every field is reduced
      __threadfence();
      if (a.stage == SS_INIT || a.stage == SS_PCG_INIT) done[1] = 0u;
      if (a.set_cond) {
        unsigned any = 0;
        if (a.ms) {
          for (int g = 0; g < a.ms->ngroups; ++g) {
            const FieldState* sg = a.ms->st[g];
            for (int k = 0; k < a.ms->count[g]; ++k) any |= (*(volatile const int*)&sg[k].active != 0);
          }
        } else {
          for (int g = 0; g < a.batch; ++g) any |= (*(volatile const int*)&a.st[g].active != 0);
        }
        // every field stops by maxit passes; never iterate past that bound
        const unsigned loops = ++done[1];
        if (loops > (unsigned)a.cfg.maxit + 1u) any = 0;
        cudaGraphSetConditional(a.cond, any);
      }
      done[0] = 0u;
    }
  }
}

template <typename T>
__device__ __forceinline__ void block_finish(const PassArgs<T>& a, const Acc<T>* acc, int f, bool act) {
  block_finish(a, acc, f, act, own_block());
}

// ---------------------------------------------------------------------------
// Loads a W x n tile stored transposed in global memory (element (w, i) at
// g[i*gstride + w]) into the shared-memory rows with asynchronous copies
// (cp.async, one per complex element): every copy of the tile is in flight
// at once without holding registers. Ends with the copies complete and a
// barrier.
template <typename C>
__device__ __forceinline__ void load_transposed(C* s, int ld, const C* __restrict__ g, long long gstride, int W,
                                                int n, int tid, int nthr) {
  const int lw = __ffs(W) - 1;
  const int total = W * n;
  for (int idx = tid; idx < total; idx += nthr) {
    const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(s + (idx & (W - 1)) * ld + phys(idx >> lw)));
    const C* src = g + (long long)(idx >> lw) * gstride + (idx & (W - 1));
    if constexpr (sizeof(C) == 8)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
    else
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
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

// Float32, E = 16: every pass runs at 64 registers (4 blocks of 256 per SM),
// the filter pass too although it keeps two FFT stages' worth of state live;
// a few spilled words cost less than the latency the extra warps hide
// (measured: the filter pass 28-31% faster than at 2 blocks and 128
// registers, the x/y passes 5-17% faster than at 3 blocks and 80). Float32,
// E = 24 (radix-3 lengths): 3 blocks per SM (14-15% faster per pass than 2 at
// 384^3 and 1536^2). Float64: 2 blocks.
#define GAD_BOUNDS(T, E) __launch_bounds__(256, sizeof(T) == 4 ? ((E) == 16 ? 4 : 3) : 2)
#define GAD_BOUNDS_FILT(T, E) __launch_bounds__(256, sizeof(T) == 4 ? ((E) == 16 ? 4 : 3) : 2)

// ---------------------------------------------------------------------------
// Row-tile streaming for the fused Krylov prologue/epilogue of the x passes.
//
// A block of an x pass owns W consecutive grid rows, i.e. one contiguous run
// of W*nx reals in every field vector. The vector updates are streamed over
// that run in chunks of four reals (one float4), U chunks per thread with all
// their loads issued before any store, so each thread keeps U x (vectors
// read) 16-byte loads in flight. Chunk c of row w holds the packed complex
// elements 2q, 2q+1 (q = c mod nx/4) of the tile's shared-memory row.

// L2 prefetch of a contiguous range (16-byte aligned, multiple of 16 bytes),
// split into 16 KiB bulk requests issued by the first threads of the block.
__device__ __forceinline__ void prefetch_l2(const void* p, long long bytes, int tid, int nthr) {
  const long long chunk = 16384;
  const long long n = (bytes + chunk - 1) / chunk;
  for (long long i = tid; i < n; i += nthr) {
    const long long off = i * chunk;
    const unsigned sz = (unsigned)min(chunk, bytes - off);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((const char*)p + off), "r"(sz) : "memory");
  }
}

template <int U, class Ld, class Fin>
__device__ __forceinline__ void stream_tile(int W, int nx, float rcp_q, long long base, int tid, int nthr, Ld& ld,
                                            Fin& fin) {
  const int qn = nx >> 2;
  const int total = W * qn;
  for (int c0 = tid; c0 < total; c0 += nthr * U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = c0 + u * nthr;
      if (c < total) {
        const int w = fquot(c, rcp_q);
        ld(u, base + (long long)w * nx + 4 * (c - w * qn));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = c0 + u * nthr;
      if (c < total) {
        const int w = fquot(c, rcp_q);
        const int q = c - w * qn;
        fin(u, w, q, base + (long long)w * nx + 4 * q);
      }
    }
  }
}

template <typename T> __device__ __forceinline__ void put_pair(typename cpx<T>::t* row, int q, const V4<T>& x) {
  using C = typename cpx<T>::t;
  row[phys(2 * q)] = C{x.v[0], x.v[1]};
  row[phys(2 * q + 1)] = C{x.v[2], x.v[3]};
}
template <typename T> __device__ __forceinline__ V4<T> get_pair(const typename cpx<T>::t* row, int q) {
  const auto a = row[phys(2 * q)], b = row[phys(2 * q + 1)];
  return {{a.x, a.y, b.x, b.y}};
}

// Component offsets of the closure pair that field f stands for: field f is
// pair p = f mod npairs of velocity v = f / npairs, whose components i and j
// start at (v ncomp + i) P and (v ncomp + j) P.
template <typename T>
__device__ __forceinline__ void pair_offsets(const PassArgs<T>& a, int f, long long& oi, long long& oj) {
  const int v = f / a.npairs, p = f - v * a.npairs;
  const int i = (a.pair_code >> (4 * p)) & 3, j = (a.pair_code >> (4 * p + 2)) & 3;
  oi = ((long long)v * a.ncomp + i) * a.P;
  oj = ((long long)v * a.ncomp + j) * a.P;
}

// x = prologue of the forward x pass for the block's row tile, written into
// the shared-memory rows as packed complex (z[n] = x[2n] + i x[2n+1]).
template <typename T, int U>
__device__ __forceinline__ void xfwd_prologue(const PassArgs<T>& a, typename cpx<T>::t* s, long long base, bool first,
                                              T al, T be, T om, int tid, int nthr, int f) {
  const T* __restrict__ vA = a.A;
  const T* __restrict__ vB = a.B;
  T* __restrict__ vO1 = a.O1;
  T* __restrict__ vO2 = a.O2;
  T* __restrict__ vO3 = a.O3;
  const int ld = a.ld, W = a.W, nx = a.nx;
  const float rq = a.rcp_a;
  V4<T> r_[U], x_[U], y_[U];
  switch (a.op) {
    case XF_VC: {                                 // U += R; x = R
      auto ldf = [&](int u, long long g) { r_[u] = ld4(vA + g); x_[u] = ld4(vO1 + g); };
      auto fin = [&](int u, int w, int q, long long g) {
        V4<T> o;
#pragma unroll
        for (int e = 0; e < 4; ++e) o.v[e] = x_[u].v[e] + r_[u].v[e];
        st4(vO1 + g, o);
        put_pair<T>(s + w * ld, q, r_[u]);
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    case XF_CG: {                                 // U += alpha P; P = R + beta P (first pass: P = R)
      if (first) {
        auto ldf = [&](int u, long long g) { r_[u] = ld4(vA + g); };
        auto fin = [&](int u, int w, int q, long long g) { st4(vO2 + g, r_[u]); put_pair<T>(s + w * ld, q, r_[u]); };
        stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      } else {
        auto ldf = [&](int u, long long g) { r_[u] = ld4(vA + g); x_[u] = ld4(vO2 + g); y_[u] = ld4(vO1 + g); };
        auto fin = [&](int u, int w, int q, long long g) {
          V4<T> uo, po;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            uo.v[e] = fma(al, x_[u].v[e], y_[u].v[e]);
            po.v[e] = fma(be, x_[u].v[e], r_[u].v[e]);
          }
          st4(vO1 + g, uo);
          st4(vO2 + g, po);
          put_pair<T>(s + w * ld, q, po);
        };
        stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      }
      break;
    }
    case XF_BI_P: {                               // P = R + beta (P - omega Q) (first pass: P = R)
      if (first) {
        auto ldf = [&](int u, long long g) { r_[u] = ld4(vA + g); };
        auto fin = [&](int u, int w, int q, long long g) { st4(vO2 + g, r_[u]); put_pair<T>(s + w * ld, q, r_[u]); };
        stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      } else {
        auto ldf = [&](int u, long long g) { r_[u] = ld4(vA + g); x_[u] = ld4(vO2 + g); y_[u] = ld4(vB + g); };
        auto fin = [&](int u, int w, int q, long long g) {
          V4<T> po;
#pragma unroll
          for (int e = 0; e < 4; ++e) po.v[e] = fma(be, fma(-om, y_[u].v[e], x_[u].v[e]), r_[u].v[e]);
          st4(vO2 + g, po);
          put_pair<T>(s + w * ld, q, po);
        };
        stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      }
      break;
    }
    case XF_BI_S: {                               // S = R - alpha Q
      auto ldf = [&](int u, long long g) { r_[u] = ld4(vA + g); y_[u] = ld4(vB + g); };
      auto fin = [&](int u, int w, int q, long long g) {
        V4<T> so;
#pragma unroll
        for (int e = 0; e < 4; ++e) so.v[e] = fma(-al, y_[u].v[e], r_[u].v[e]);
        st4(vO3 + g, so);
        put_pair<T>(s + w * ld, q, so);
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    case XF_MUL: {                                // closure: x = A_i A_j
      long long oi, oj;
      pair_offsets(a, f, oi, oj);
      const long long fb = (long long)f * a.P;
      auto ldf = [&](int u, long long g) { r_[u] = ld4(vA + (g - fb) + oi); y_[u] = ld4(vA + (g - fb) + oj); };
      auto fin = [&](int u, int w, int q, long long) {
        V4<T> xo;
#pragma unroll
        for (int e = 0; e < 4; ++e) xo.v[e] = r_[u].v[e] * y_[u].v[e];
        put_pair<T>(s + w * ld, q, xo);
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    default: {                                    // XF_COPY: x = A (and O1 = A)
      auto ldf = [&](int u, long long g) { r_[u] = ld4(vA + g); };
      auto fin = [&](int u, int w, int q, long long g) {
        if (vO1) st4(vO1 + g, r_[u]);
        put_pair<T>(s + w * ld, q, r_[u]);
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
  }
}

// Epilogue of the inverse x pass: y = G x sits in the shared-memory rows
// (packed, y[2n] + i y[2n+1]); the vector updates and dots of the algorithm
// are streamed over the block's row tile.
template <typename T, int U>
__device__ __forceinline__ void xinv_epilogue(const PassArgs<T>& a, const typename cpx<T>::t* s, long long base, T al,
                                              T om, Acc<T>& acc0, Acc<T>& acc1, int tid, int nthr, int f) {
  const T* __restrict__ vA = a.A;
  const T* __restrict__ vB = a.B;
  const T* __restrict__ vC = a.C;
  T* __restrict__ vO1 = a.O1;
  T* __restrict__ vO2 = a.O2;
  const int ld = a.ld, W = a.W, nx = a.nx;
  const float rq = a.rcp_a;
  V4<T> a_[U], b_[U], c_[U], d_[U];
  switch (a.op) {
    case XI_STORE: {
      auto ldf = [&](int, long long) {};
      auto fin = [&](int, int w, int q, long long g) { st4(vO1 + g, get_pair<T>(s + w * ld, q)); };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    case XI_INIT:                                 // r = A - y -> O1 (R), O2 (F0, optional); (r, r)
    case XI_RES: {                                // res = A - y; (res, res)
      const bool store = a.op == XI_INIT;
      auto ldf = [&](int u, long long g) { a_[u] = ld4(vA + g); };
      auto fin = [&](int u, int w, int q, long long g) {
        const V4<T> y = get_pair<T>(s + w * ld, q);
        V4<T> r;
#pragma unroll
        for (int e = 0; e < 4; ++e) { r.v[e] = a_[u].v[e] - y.v[e]; acc0.add_prod(r.v[e], r.v[e]); }
        if (store) {
          st4(vO1 + g, r);
          if (vO2) st4(vO2 + g, r);
        }
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    case XI_VC:                                   // R -= y; (R, R)
    case XI_CG: {                                 // R -= alpha y; (R, R)
      const bool vc = a.op == XI_VC;
      auto ldf = [&](int u, long long g) { a_[u] = ld4(vO1 + g); };
      auto fin = [&](int u, int w, int q, long long g) {
        const V4<T> y = get_pair<T>(s + w * ld, q);
        V4<T> r;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          r.v[e] = vc ? a_[u].v[e] - y.v[e] : fma(-al, y.v[e], a_[u].v[e]);
          acc0.add_prod(r.v[e], r.v[e]);
        }
        st4(vO1 + g, r);
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    case XI_SD: {                                 // U += alpha R; R -= alpha y; (R, R)
      auto ldf = [&](int u, long long g) { a_[u] = ld4(vO1 + g); b_[u] = ld4(vO2 + g); };
      auto fin = [&](int u, int w, int q, long long g) {
        const V4<T> y = get_pair<T>(s + w * ld, q);
        V4<T> r, uo;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uo.v[e] = fma(al, a_[u].v[e], b_[u].v[e]);
          r.v[e] = fma(-al, y.v[e], a_[u].v[e]);
          acc0.add_prod(r.v[e], r.v[e]);
        }
        st4(vO2 + g, uo);
        st4(vO1 + g, r);
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    case XI_BI_Q: {                               // Q = y; (F0, Q)
      auto ldf = [&](int u, long long g) { a_[u] = ld4(vA + g); };
      auto fin = [&](int u, int w, int q, long long g) {
        const V4<T> y = get_pair<T>(s + w * ld, q);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc0.add_prod(a_[u].v[e], y.v[e]);
        st4(vO1 + g, y);
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    case XI_BI_T: {          // t = y; U += alpha P + omega S; R = S - omega t; (R, R), (F0, R)
      auto ldf = [&](int u, long long g) {
        a_[u] = ld4(vA + g); b_[u] = ld4(vB + g); c_[u] = ld4(vC + g); d_[u] = ld4(vO1 + g);
      };
      auto fin = [&](int u, int w, int q, long long g) {
        const V4<T> y = get_pair<T>(s + w * ld, q);
        V4<T> r, uo;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uo.v[e] = fma(om, c_[u].v[e], fma(al, b_[u].v[e], d_[u].v[e]));
          r.v[e] = fma(-om, y.v[e], c_[u].v[e]);
          acc0.add_prod(r.v[e], r.v[e]);
          acc1.add_prod(a_[u].v[e], r.v[e]);
        }
        st4(vO1 + g, uo);
        st4(vO2 + g, r);
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    case XI_TAU: {                                // closure: O1 = B_i B_j - y
      long long oi, oj;
      pair_offsets(a, f, oi, oj);
      const long long fb = (long long)f * a.P;
      auto ldf = [&](int u, long long g) { b_[u] = ld4(vB + (g - fb) + oi); c_[u] = ld4(vB + (g - fb) + oj); };
      auto fin = [&](int u, int w, int q, long long g) {
        const V4<T> y = get_pair<T>(s + w * ld, q);
        V4<T> t;
#pragma unroll
        for (int e = 0; e < 4; ++e) t.v[e] = fma(b_[u].v[e], c_[u].v[e], -y.v[e]);
        st4(vO1 + g, t);
      };
      stream_tile<U>(W, nx, rq, base, tid, nthr, ldf, fin);
      break;
    }
    default:
      break;
  }
}

// Forward x pass: the Krylov prologue streams the block's row tile into the
// shared-memory rows as packed complex (z[n] = x[2n] + i x[2n+1]); the
// half-length FFT runs in shared memory, followed by the real-to-complex
// split and the transposed store to S1.
//   rcp_a = 1/(nx/4), rcp_b = 1/(nx/4 + 1)
template <typename T, int E>
__device__ __forceinline__ void xfwd_body(const PassArgs<T>& a, const VBlock& vb) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = field_of(a, vb);
  if (a.clear_cond && vb.x == 0 && vb.y == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
  FieldState* st = a.st ? a.st + f : nullptr;
  if (st && !st->active && !a.force) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = a.nx, M = nx >> 1;
  const int row0 = vb.x * a.W;
  const int z = row0 / a.ny, y0 = row0 - z * a.ny;
  const long long base = (long long)f * a.P + (long long)row0 * nx;
  const bool first = st ? (st->iter == 0) : true;
  const T al = st ? T(st->alpha) : T(0), be = st ? T(st->beta) : T(0), om = st ? T(st->omega) : T(0);
  {
    // the vectors the prologue reads, fetched into L2 as whole tiles so that
    // only the first of the streaming rounds waits on DRAM
    const long long tb = (long long)a.W * nx * sizeof(T);
    const int op = a.op;
    if (op == XF_MUL) {
      long long oi, oj;
      pair_offsets(a, f, oi, oj);
      const long long ro = (long long)row0 * nx;
      prefetch_l2(a.A + oi + ro, tb, tid, nthr);
      prefetch_l2(a.A + oj + ro, tb, tid, nthr);
    } else {
      prefetch_l2(a.A + base, tb, tid, nthr);
    }
    if (op == XF_VC || (op == XF_CG && !first)) prefetch_l2(a.O1 + base, tb, tid, nthr);
    if ((op == XF_CG || op == XF_BI_P) && !first) prefetch_l2(a.O2 + base, tb, tid, nthr);
    if ((op == XF_BI_P && !first) || op == XF_BI_S) prefetch_l2(a.B + base, tb, tid, nthr);
  }
  xfwd_prologue<T, 2>(a, s, base, first, al, be, om, tid, nthr, f);
  __syncthreads();
  SmemRows<C> rows{s, a.ld};
  if (!fft_run_fixed<C, E, false, 1024>(s, a.ld, a.fft, tid, a.tfft, rows, rows, true, true) &&
      !fft_run_fixed<C, E, false, 256>(s, a.ld, a.fft, tid, a.tfft, rows, rows, true, true) &&
      !fft_run_fixed<C, E, false, 128>(s, a.ld, a.fft, tid, a.tfft, rows, rows, true, true))
    fft_run<C, E, false>(s, a.ld, a.fft, tid, a.tfft, rows, rows, true, true);
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

template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_xfwd(const __grid_constant__ PassArgs<T> a) {
  xfwd_body<T, E>(a, own_block());
}

// Inverse x pass: transposed load from S1, complex-to-real preparation, FFT
// in shared memory, then the fused epilogue and dots streamed over the row
// tile.
template <typename T, int E>
__device__ __forceinline__ void xinv_body(const PassArgs<T>& a, const VBlock& vb) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = field_of(a, vb);
  FieldState* st = a.st ? a.st + f : nullptr;
  const bool act = (st ? (st->active != 0) : true) || a.force;
  if (!act && a.ndots == 0) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = a.nx, M = nx >> 1;
  const int row0 = vb.x * a.W;
  const int z = row0 / a.ny, y0 = row0 - z * a.ny;
  Acc<T> acc[3];
  if (act) {
    const long long base = (long long)f * a.P + (long long)row0 * nx;
    const C* S1 = reinterpret_cast<const C*>(a.S1) + (long long)f * a.SP + (long long)z * a.kxn * a.ny + y0;
    load_transposed(s, a.ld, S1, a.ny, a.W, M + 1, tid, nthr);
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
    SmemRows<C> rows{s, a.ld};
    if (!fft_run_fixed<C, E, true, 1024>(s, a.ld, a.fft, tid, a.tfft, rows, rows, true, true) &&
        !fft_run_fixed<C, E, true, 256>(s, a.ld, a.fft, tid, a.tfft, rows, rows, true, true) &&
        !fft_run_fixed<C, E, true, 128>(s, a.ld, a.fft, tid, a.tfft, rows, rows, true, true))
      fft_run<C, E, true>(s, a.ld, a.fft, tid, a.tfft, rows, rows, true, true);
    {
      // the epilogue's input vectors, fetched into L2 as whole tiles just
      // before the epilogue streams them: only its first round waits on DRAM.
      // (Fetched at block start instead, they stayed in L2 through the FFT and
      // were partly evicted before use: 1.29x the algorithmic DRAM traffic
      // for four input vectors, measured.)
      const long long tb = (long long)a.W * nx * sizeof(T);
      const int op = a.op;
      if (op == XI_INIT || op == XI_RES || op == XI_BI_Q || op == XI_BI_T) prefetch_l2(a.A + base, tb, tid, nthr);
      if (op == XI_VC || op == XI_CG || op == XI_SD || op == XI_BI_T) prefetch_l2(a.O1 + base, tb, tid, nthr);
      if (op == XI_SD) prefetch_l2(a.O2 + base, tb, tid, nthr);
      if (op == XI_TAU) {
        long long oi, oj;
        pair_offsets(a, f, oi, oj);
        const long long ro = (long long)row0 * nx;
        prefetch_l2(a.B + oi + ro, tb, tid, nthr);
        prefetch_l2(a.B + oj + ro, tb, tid, nthr);
      }
      if (op == XI_BI_T) {
        prefetch_l2(a.B + base, tb, tid, nthr);
        prefetch_l2(a.C + base, tb, tid, nthr);
      }
    }
    const T al = st ? T(st->alpha) : T(0), om = st ? T(st->omega) : T(0);
    Acc<T> acc0, acc1;
    xinv_epilogue<T, 2>(a, s, base, al, om, acc0, acc1, tid, nthr, f);
    acc[0] = acc0;
    acc[1] = acc1;
  }
  if (a.ndots) block_finish(a, acc, f, act, vb);
}

template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_xinv(const __grid_constant__ PassArgs<T> a) {
  xinv_body<T, E>(a, own_block());
}

// Filter pass along the last axis (y in 2D, z in 3D): forward FFT of W
// contiguous sequences read straight from the spectral buffer, multiply by
// G_hat(k)/P with Parseval dots in registers, inverse FFT written straight
// back. fft holds the forward plan, fft_inv the reversed one. In 3D the
// sequence index is kx*ny + ky.
template <typename T, int E>
__device__ __forceinline__ void filt_body(const PassArgs<T>& a, const VBlock& vb) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = field_of(a, vb);
  FieldState* st = a.st ? a.st + f : nullptr;
  const bool act = (st ? (st->active != 0) : true) || a.force;
  if (!act && a.ndots == 0) return;
  const int tid = threadIdx.x;
  const int L = a.fft.L, half = L >> 1;
  const bool three_d = a.nz > 1;
  const int nseq = three_d ? a.kxn * a.ny : a.kxn;
  const int seq0 = vb.x * a.W;
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
    // the sequence's part of |k|^2 and its Parseval weight, recomputed only
    // when the sequence changes (a butterfly's R elements share it)
    int cw = -1, ck2 = 0;
    T cwgt = T(0);
    auto mul = [&](int w, int i, C& X) {
      if (w != cw) {
        cw = w;
        const int seq = seq0 + w;
        int kx;
        if (three_d) {
          kx = seq / ny;
          const int kyi = seq - kx * ny;
          const int ky = kyi < (ny >> 1) ? kyi : kyi - ny;
          ck2 = kx * kx + ky * ky;
        } else {
          kx = seq;
          ck2 = kx * kx;
        }
        cwgt = (kx == 0 || kx == nxh) ? T(1) : T(2);
      }
      const int ki = i < half ? i : i - L;
      const T g = ghat(kc2, T(ck2 + ki * ki));
      if (op != FI_NONE && w < nvalid) {
        const T wgt = cwgt;
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
    if (!fft_filter_run_fixed<C, E, 2048>(s, a.ld, a.fft, a.fft_inv, tid, a.tfft, load, mul, emit) &&
        !fft_filter_run_fixed<C, E, 512>(s, a.ld, a.fft, a.fft_inv, tid, a.tfft, load, mul, emit) &&
        !fft_filter_run_fixed<C, E, 256>(s, a.ld, a.fft, a.fft_inv, tid, a.tfft, load, mul, emit))
      fft_filter_run<C, E>(s, a.ld, a.fft, a.fft_inv, tid, a.tfft, load, mul, emit);
    acc[0].s = p0;
    acc[1].s = p1;
    acc[2].s = p2;
  }
  if (a.ndots) block_finish(a, acc, f, act, vb);
}

template <typename T, int E>
__global__ void GAD_BOUNDS_FILT(T, E) k_filt(const __grid_constant__ PassArgs<T> a) {
  filt_body<T, E>(a, own_block());
}

// 3D forward y pass: W consecutive z at one kx; the first stage reads the
// S1 rows [z][kx][:] directly, the tile is stored transposed into S2
// [kx][ky][z].  Grid x = kxn * (nz/W).
template <typename T, int E>
__device__ __forceinline__ void yfwd_body(const PassArgs<T>& a, const VBlock& vb) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = field_of(a, vb);
  if (a.st && !a.st[f].active && !a.force) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = a.ny;
  const int zt = a.nz / a.W;
  const int kx = vb.x / zt, z0 = (vb.x - kx * zt) * a.W;
  const C* S1 = reinterpret_cast<const C*>(a.S1) + (long long)f * a.SP;
  const int kxn = a.kxn;
  auto load = [&](int w, int i) -> C { return S1[((long long)(z0 + w) * kxn + kx) * L + i]; };
  SmemRows<C> rows{s, a.ld};
  if (!fft_run_fixed<C, E, false, 512>(s, a.ld, a.fft, tid, a.tfft, load, rows, false, true) &&
      !fft_run_fixed<C, E, false, 256>(s, a.ld, a.fft, tid, a.tfft, load, rows, false, true))
    fft_run<C, E, false>(s, a.ld, a.fft, tid, a.tfft, load, rows, false, true);
  C* S2 = reinterpret_cast<C*>(a.S2) + (long long)f * a.SP + (long long)kx * L * a.nz + z0;
  store_transposed(s, a.ld, S2, a.nz, a.W, L, tid, nthr);
}

template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_yfwd(const __grid_constant__ PassArgs<T> a) {
  yfwd_body<T, E>(a, own_block());
}

// 3D inverse y pass: transposed load from S2, inverse FFT whose last stage
// writes the S1 rows directly.
template <typename T, int E>
__device__ __forceinline__ void yinv_body(const PassArgs<T>& a, const VBlock& vb) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int f = field_of(a, vb);
  if (a.st && !a.st[f].active && !a.force) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = a.ny;
  const int zt = a.nz / a.W;
  const int kx = vb.x / zt, z0 = (vb.x - kx * zt) * a.W;
  const C* S2 = reinterpret_cast<const C*>(a.S2) + (long long)f * a.SP + (long long)kx * L * a.nz + z0;
  load_transposed(s, a.ld, S2, a.nz, a.W, L, tid, nthr);
  C* S1 = reinterpret_cast<C*>(a.S1) + (long long)f * a.SP;
  const int kxn = a.kxn;
  auto emit = [&](int w, int i, const C& x) { S1[((long long)(z0 + w) * kxn + kx) * L + i] = x; };
  SmemRows<C> rows{s, a.ld};
  if (!fft_run_fixed<C, E, true, 512>(s, a.ld, a.fft, tid, a.tfft, rows, emit, true, false) &&
      !fft_run_fixed<C, E, true, 256>(s, a.ld, a.fft, tid, a.tfft, rows, emit, true, false))
    fft_run<C, E, true>(s, a.ld, a.fft, tid, a.tfft, rows, emit, true, false);
}

template <typename T, int E>
__global__ void GAD_BOUNDS(T, E) k_yinv(const __grid_constant__ PassArgs<T> a) {
  yinv_body<T, E>(a, own_block());
}

// One pass over several shape groups in a single launch: block b belongs to
// the group g with start[g] <= b < start[g + 1] and runs that group's pass
// (its PassArgs, copied to shared memory) at its place in the group's own
// launch shape (vgx x vgy blocks). Blocks of different groups differ in tile
// shape and FFT plan; the block size and shared memory are the maximum over
// the groups (threads beyond a group's FFT thread count only join barriers).
template <typename T, int E, int KIND>
__global__ void GAD_BOUNDS(T, E) k_multi(const PassArgs<T>* __restrict__ args, const int* __restrict__ start,
                                         int ngroups) {
  __shared__ PassArgs<T> sa;
  __shared__ int sg;
  if (threadIdx.x == 0) {
    int g = 0;
    while (g + 1 < ngroups && (int)blockIdx.x >= start[g + 1]) ++g;
    sg = g;
  }
  __syncthreads();
  {
    static_assert(sizeof(PassArgs<T>) % 4 == 0, "PassArgs copies as 32-bit words");
    const int* src = reinterpret_cast<const int*>(args + sg);
    int* dst = reinterpret_cast<int*>(&sa);
    for (int i = threadIdx.x; i < (int)(sizeof(PassArgs<T>) / 4); i += blockDim.x) dst[i] = src[i];
  }
  const int local = (int)blockIdx.x - start[sg];
  __syncthreads();
  const VBlock vb{local % sa.vgx, local / sa.vgx, sa.vgx, sa.vgy};
  if constexpr (KIND == 0) xfwd_body<T, E>(sa, vb);
  else if constexpr (KIND == 1) xinv_body<T, E>(sa, vb);
  else if constexpr (KIND == 2) filt_body<T, E>(sa, vb);
  else if constexpr (KIND == 3) yfwd_body<T, E>(sa, vb);
  else if constexpr (KIND == 4) yinv_body<T, E>(sa, vb);
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
