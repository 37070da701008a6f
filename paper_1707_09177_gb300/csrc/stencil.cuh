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
// One block owns a tile of W consecutive rows (y0 .. y0+W-1) of one z plane.
// Its halo -- rows y0-1 and y0+W of the plane (periodic in y) and, in 3D, the
// tile's rows in planes z-1 and z+1 (periodic in z) -- and the tile itself
// are staged in shared memory by bulk asynchronous copies (one per row, the
// rows are contiguous runs of nx values) that signal an mbarrier; the x
// neighbours wrap inside each staged row. The wait on the mbarrier is bounded
// in time: a block that gives up flags its field (AD_ERR_TIMEOUT) and takes
// no part in the result.
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
// (limit_ns = 0: one non-blocking test).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
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
    if (limit_ns == 0 || global_ns() - t0 > limit_ns) return false;
  }
}

// z = M r over the block's row tile, with the inner product (r, z).
//   A = r, O1 = z; W = rows per tile; cx, cy, cz = c_d of the x, y, z axes.
// Grid: x = (ny / W) * nz tiles, y = fields. Shared memory: (W + 2) rows in
// 2D, (3 W + 2) rows in 3D, nx values each.
template <typename T>
__global__ void __launch_bounds__(256) k_sten(PassArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* rows = reinterpret_cast<T*>(smem_raw);
  const int f = blockIdx.y;
  if (a.clear_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
  FieldState* st = a.st ? a.st + f : nullptr;
  const bool act = (st ? (st->active != 0) : true) || a.force;
  if (!act && a.ndots == 0) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = a.nx, ny = a.ny, nz = a.nz, W = a.W;
  const bool three_d = nz > 1;
  const int tiles_y = ny / W;
  const int zp = blockIdx.x / tiles_y;
  const int y0 = (blockIdx.x - zp * tiles_y) * W;
  const int nrows = three_d ? 3 * W + 2 : W + 2;
  const long long fbase = (long long)f * a.P;
  Acc<T> acc[3];
  bool ok = true;
  if (act) {
    const uint32_t b = smem_u32(&bar);
    const uint32_t row_bytes = (uint32_t)(nx * sizeof(T));
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid < 32) {
      if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     ::"r"(b), "r"(row_bytes * (uint32_t)nrows) : "memory");
      }
      __syncwarp();
      // row slot s: 0 .. W+1 -> plane zp, rows y0-1 .. y0+W;
      //             W+2+i    -> plane zp-1, row y0+i;  2W+2+i -> plane zp+1, row y0+i
      for (int s = tid; s < nrows; s += 32) {
        int zz = zp, yy;
        if (s < W + 2) {
          yy = y0 - 1 + s;
          yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        } else if (s < 2 * W + 2) {
          zz = zp == 0 ? nz - 1 : zp - 1;
          yy = y0 + (s - (W + 2));
        } else {
          zz = zp == nz - 1 ? 0 : zp + 1;
          yy = y0 + (s - (2 * W + 2));
        }
        const T* src = a.A + fbase + ((long long)zz * ny + yy) * nx;
        const uint32_t dst = smem_u32(rows + (long long)s * nx);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(dst), "l"(src), "r"(row_bytes), "r"(b) : "memory");
      }
    }
    // every thread waits; the block gives up as a whole if any thread did
    ok = __syncthreads_and(mbar_wait_bounded(b, 0u, a.wait_ns) ? 1 : 0) != 0;
    if (!ok) {
      // flag the field and wait (bounded, 1 s) for this block's copies to land
      // before its shared memory is released
      if (tid == 0 && st) atomicExch(&st->fault, 1);
      mbar_wait_bounded(b, 0u, 1000000000ull);
      __syncthreads();
    }
  }
  if (act && ok) {
    const T cx = a.cx, cy = a.cy, cz = a.cz;
    const int qn = nx >> 2;
    T* __restrict__ out = a.O1;
    Acc<T> rz;
    for (int c = tid; c < W * qn; c += nthr) {
      const int w = fquot(c, a.rcp_a);
      const int x0 = 4 * (c - w * qn);
      const T* rc = rows + (long long)(w + 1) * nx;
      const V4<T> cv = ld4(rc + x0), nv = ld4(rc - nx + x0), sv = ld4(rc + nx + x0);
      const T xl = rc[x0 == 0 ? nx - 1 : x0 - 1];
      const T xr = rc[x0 + 4 == nx ? 0 : x0 + 4];
      V4<T> bv{}, tv{};
      if (three_d) {
        bv = ld4(rows + (long long)(W + 2 + w) * nx + x0);
        tv = ld4(rows + (long long)(2 * W + 2 + w) * nx + x0);
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
      st4(out + fbase + ((long long)zp * ny + y0 + w) * nx + x0, zo);
    }
    acc[0] = rz;
  }
  if (a.ndots) block_finish(a, acc, f, act);
}

}  // namespace gad
