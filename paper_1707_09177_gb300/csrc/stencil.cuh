// Periodic finite-difference preconditioner of the preconditioned CG solve.
//
// G = (I - delta^2 Laplacian)^{-1} (Section 4, Eq. df) has a differential
// inverse; its second-order finite-difference version on the 2*pi-periodic
// grid,
//     z = M r = r + sum_d c_d (2 r_i - r_{i+e_d} - r_{i-e_d}),
//     c_d = (delta / h_d)^2 = (N_d / (2 pi k_c))^2,
// is symmetric positive definite, commutes with G, and bounds the spectrum of
// M G to [4/pi^2, 1]. The paper has no preconditioner; this is the textbook
// preconditioned CG with that M.
//
// Rows are staged in shared memory by bulk asynchronous copies (one per row:
// the rows are contiguous runs of nx values) that complete on mbarriers; the
// x neighbours wrap inside each staged row. Every wait on an mbarrier is
// bounded in time: a block that gives up flags its field (AD_ERR_TIMEOUT),
// waits (bounded) for its copies still in flight and takes no part in the
// result.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "args.h"
#include "passes.cuh"

namespace gad {

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `parity` of the mbarrier; false after `limit_ns` of waiting
// (limit_ns = 0: gives up at once, which is how the timeout path is tested).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (limit_ns == 0) return false;
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// z = M r with the inner product (r, z), marching along the outermost axis
// (z in 3D, y in 2D). A block owns `chunk` consecutive positions m0 ..
// m0+chunk-1 of that axis and, in 3D, a tile of W rows y0 .. y0+W-1. The rows
// one position needs -- a "slice": in 3D the tile's rows of plane m with its
// periodic y-halo rows (W + 2 rows), in 2D row m itself -- are staged by bulk
// copies (one per row, completing on the slot's mbarrier) into a ring of four
// slots. Output m reads slices m-1, m, m+1; slices m+2 and m+3 are in flight
// meanwhile, so every row is read from memory once per block (plus the two
// boundary slices of the chunk and, in 3D, the y halo).
//   A = r, O1 = z; W = tile rows (3D), chunk = positions per block;
//   grid: x = (ny / W) * (nz / chunk) in 3D, ny / chunk in 2D; y = fields;
//   shared memory: 4 slices.
template <typename T>
__global__ void __launch_bounds__(256) k_sten(PassArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[4];
  T* ring = reinterpret_cast<T*>(smem_raw);
  const int f = field_of(a);
  if (a.clear_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
  FieldState* st = a.st ? a.st + f : nullptr;
  const bool act = (st ? (st->active != 0) : true) || a.force;
  if (!act && a.ndots == 0) return;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const bool three_d = nz > 1;
  const int W = three_d ? a.W : 1;
  const int srows = three_d ? W + 2 : 1;
  const int nmarch = three_d ? nz : ny;
  const int chunk = a.chunk;
  const int tiles_y = three_d ? ny / W : 1;
  const int ct = blockIdx.x / tiles_y;
  const int y0 = (blockIdx.x - ct * tiles_y) * W;
  const int m0 = ct * chunk;
  const long long fbase = (long long)f * a.P;
  const long long slice_elems = (long long)srows * nx;
  const uint32_t row_bytes = (uint32_t)(nx * sizeof(T));
  const uint32_t slice_bytes = row_bytes * (uint32_t)srows;
  Acc<T> acc[3];
  auto slot = [&](int s) { return (s - (m0 - 1)) & 3; };
  // warp 0: stage slice s (march position, periodic) into its slot
  auto issue = [&](int s) {
    const int q = slot(s);
    int mm = s % nmarch;
    if (mm < 0) mm += nmarch;
    const uint32_t b = smem_u32(&bars[q]);
    if (lane == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(slice_bytes) : "memory");
    __syncwarp();
    for (int r = lane; r < srows; r += 32) {
      long long row;
      if (three_d) {
        int yy = y0 - 1 + r;
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        row = (long long)mm * ny + yy;
      } else {
        row = mm;
      }
      const T* src = a.A + fbase + row * nx;
      const uint32_t dst = smem_u32(ring + (long long)q * slice_elems + (long long)r * nx);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   ::"r"(dst), "l"(src), "r"(row_bytes), "r"(b) : "memory");
    }
  };
  if (act) {
    if (tid == 0) {
      for (int q = 0; q < 4; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[q])) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int last = m0 + chunk;                     // the last slice a block needs
    const int pre = min(m0 + 2, last);
    if (tid < 32)
      for (int s = m0 - 1; s <= pre; ++s) issue(s);
    unsigned ph = 0u, pending = 0u;                  // per slot: parity to wait for, issued and not waited
    for (int s = m0 - 1; s <= pre; ++s) pending |= 1u << slot(s);
    // waits for slice s; false (block-uniform) when the bounded wait gave up
    auto wait = [&](int s) -> bool {
      const int q = slot(s);
      const bool got = __syncthreads_and(mbar_wait_bounded(smem_u32(&bars[q]), (ph >> q) & 1u, a.wait_ns) ? 1 : 0) != 0;
      if (got) { ph ^= 1u << q; pending &= ~(1u << q); }
      return got;
    };
    bool ok = wait(m0 - 1) && wait(m0);
    const T cx = a.cx, cy = a.cy, cz = a.cz;
    const int qn = nx >> 2;
    T* __restrict__ out = a.O1;
    Acc<T> rz;
    for (int m = m0; ok && m < last; ++m) {
      if (!wait(m + 1)) { ok = false; break; }
      const T* sp = ring + (long long)slot(m - 1) * slice_elems;
      const T* sc = ring + (long long)slot(m) * slice_elems;
      const T* sn = ring + (long long)slot(m + 1) * slice_elems;
      const int mm = m >= nmarch ? m - nmarch : m;
      for (int c = tid; c < W * qn; c += nthr) {
        const int w = three_d ? fquot(c, a.rcp_a) : 0;
        const int x0 = 4 * (c - w * qn);
        // 3D: centre row w+1 of slice m, y neighbours rows w and w+2 of slice m,
        //     z neighbours row w+1 of slices m-1 and m+1
        // 2D: centre slice m, y neighbours slices m-1 and m+1
        const T* rc = sc + (long long)(three_d ? w + 1 : 0) * nx;
        const T* rn = three_d ? rc - nx : sp;
        const T* rs = three_d ? rc + nx : sn;
        const V4<T> cv = ld4(rc + x0), nv = ld4(rn + x0), sv = ld4(rs + x0);
        const T xl = rc[x0 == 0 ? nx - 1 : x0 - 1];
        const T xr = rc[x0 + 4 == nx ? 0 : x0 + 4];
        V4<T> bv{}, tv{};
        if (three_d) {
          bv = ld4(sp + (long long)(w + 1) * nx + x0);
          tv = ld4(sn + (long long)(w + 1) * nx + x0);
        }
        V4<T> zo;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          // every operation rounded separately, in this order (no contraction):
          // z = ((r + c_x d_x) + c_y d_y) + c_z d_z, d = (2 r - left) - right
          const T r = cv.v[e];
          const T two = r + r;
          const T dx = sub_rn(sub_rn(two, e == 0 ? xl : cv.v[e - 1]), e == 3 ? xr : cv.v[e + 1]);
          const T dy = sub_rn(sub_rn(two, nv.v[e]), sv.v[e]);
          T z = add_rn(r, mul_rn(cx, dx));
          z = add_rn(z, mul_rn(cy, dy));
          if (three_d) z = add_rn(z, mul_rn(cz, sub_rn(sub_rn(two, bv.v[e]), tv.v[e])));
          zo.v[e] = z;
          rz.add_prod(r, z);
        }
        const long long orow = three_d ? (long long)mm * ny + y0 + w : (long long)mm;
        st4(out + fbase + orow * nx + x0, zo);
      }
      __syncthreads();                               // slice m-1 is free
      if (m + 3 <= last) {
        if (tid < 32) issue(m + 3);
        pending |= 1u << slot(m + 3);
      }
    }
    if (!ok) {
      // flag the field; wait (bounded, 1 s) for every copy still in flight
      // before the block's shared memory is released
      if (tid == 0 && st) atomicExch(&st->fault, 1);
      for (int q = 0; q < 4; ++q)
        if ((pending >> q) & 1u) mbar_wait_bounded(smem_u32(&bars[q]), (ph >> q) & 1u, 1000000000ull);
      __syncthreads();
    } else {
      acc[0] = rz;
    }
  }
  if (a.ndots) block_finish(a, acc, f, act);
}

}  // namespace gad
