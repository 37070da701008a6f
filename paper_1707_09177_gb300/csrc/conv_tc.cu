// 32 -> 32 convolution layers of the learned initial guess on the Blackwell
// tensor cores (tcgen05): an implicit GEMM whose accumulator lives in tensor
// memory and whose activation rows are staged by TMA.
//
// One CTA owns an x-segment of 128 points of one (field, z) plane and marches
// along y. Output row y is the GEMM
//     D[128 points][32 out channels] = sum over 27 taps, 2 halves of 16 input channels
//         A_tap[128][16] * B_tap[16][32],
// 54 tcgen05.mma (M = 128, N = 32, K = 16, bf16 inputs, float32 accumulation in
// tensor memory). A_tap is not materialised: the staged rows hold every point
// of the segment plus one periodic neighbour on each side, 16 bytes (8
// channels) per point and channel group, in the no-swizzle K-major core-matrix
// layout with consecutive points 16 bytes apart; the x offset of a tap is a
// shift of the descriptor's start address by 16 bytes, the y and z offsets
// select the staged row. Rows are staged once per CTA in a ring of five y
// positions x three z planes (TMA for the 128 interior points of each channel
// group, plain loads for the two periodic neighbours), two y steps ahead of the
// tensor cores. The accumulator is double-buffered in tensor memory: the MMAs
// of row y run while the four warps read row y - 1 back (tcgen05.ld), apply
// the epilogue (ReLU, or the ReLU mask of the backward pass) and store bf16.
//
// Every mbarrier wait is bounded by %globaltimer; a CTA whose wait runs out
// sets the error flag, stops issuing work, waits (bounded) for what it has in
// flight, frees its tensor memory and returns.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "cnn.h"

namespace gad {

namespace {

constexpr int kTM = 128;                       // points per tile (GEMM M)
constexpr int kCh = 32;                        // channels
constexpr int kTaps = 27;
constexpr int kPlaneEntries = 144;             // 16-byte entries per channel-group plane
constexpr int kPlane = kPlaneEntries * 16;     // 2304 bytes
constexpr int kInterior = 8;                   // entry of the segment's first point (128-byte aligned)
constexpr int kRow = 4 * kPlane;               // one staged row: 4 channel groups
constexpr int kSlots = 5;                      // y positions in the ring
constexpr int kWBytes = kTaps * 2 * 1024;      // B operands: per tap and K half, 32 x 16 bf16
constexpr int kRowsOff = kWBytes;              // staged rows after the weights
constexpr int kBarOff = kRowsOff + kSlots * 3 * kRow;
constexpr int kSmemUsed = kBarOff + 128;
// the whole shared memory of an SM (one CTA per SM): every address a
// descriptor can reach under either reading of its two stride fields stays
// inside the allocation
constexpr int kSmemAlloc = 227 * 1024;
constexpr int kTxBytes = 3 * 4 * kTM * 16;     // bytes of one ring fill (3 rows x 4 groups x 128 points)
constexpr uint32_t kTmemCols = 64;             // two 32-column accumulators

static_assert(kSmemUsed <= kSmemAlloc, "shared-memory layout exceeds the allocation");
static_assert(kPlane % 128 == 0 && kRow % 1024 == 0 && kRowsOff % 1024 == 0, "TMA destinations 128-byte aligned");

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (limit_ns == 0) return false;
  const uint64_t t0 = gtime();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtime() - t0 > limit_ns) return false;
  }
}

// Shared-memory matrix descriptor, no swizzle: start address, leading (K
// direction) and stride (M/N direction) byte offsets between core matrices
// of 8 rows x 16 bytes, descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma kind::f16: D float32, A and B bf16,
// both K-major, N = 32, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(32 >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(dtmem), "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

struct ConvTcArgs {
  const __nv_bfloat16* Hin;      // [B][Z][Y][X][32]
  const uint4* Wimg;             // kWBytes: B operands in shared-memory order
  __nv_bfloat16* Hout;
  const __nv_bfloat16* Hmask;    // mode 1
  int X, Y, Z;
  int ychunk;                    // y rows per CTA
  int mode;                      // 0: ReLU; 1: zero where the mask is not positive
  unsigned long long wait_ns;
  int* flag;                     // set to 1 when a bounded wait runs out
};

// grid x = (X/128) * Z * (Y/ychunk), grid y = fields; 128 threads
__global__ void __launch_bounds__(128, 1) k_conv_tc(const __grid_constant__ CUtensorMap tmap, const ConvTcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nxs = a.X / kTM, nyc = a.Y / a.ychunk;
  int r = blockIdx.x;
  const int xs = r % nxs;
  r /= nxs;
  const int z = r % a.Z;
  const int yc = r / a.Z;
  const int b = blockIdx.y;
  const int x0 = xs * kTM, yb = yc * a.ychunk, ny = a.ychunk;
  (void)nyc;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kBarOff);        // [0..4] ring fills, [5..6] MMA done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kBarOff + 64);
  const uint32_t sbase = su32(sm);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kSlots + 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bars[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights: generic copy of the B-operand image
  {
    uint4* w = reinterpret_cast<uint4*>(sm);
    for (int i = tid; i < kWBytes / 16; i += 128) w[i] = __ldg(a.Wimg + i);
  }
  const long long plane_rows = (long long)a.Y * a.Z;     // rows per field
  // ring slot of y position yy (yy >= yb - 1) and the parity of its fill
  auto slot_of = [&](int yy) { return (yy - (yb - 1)) % kSlots; };
  auto fill_parity = [&](int yy) { return (uint32_t)(((yy - (yb - 1)) / kSlots) & 1); };
  auto row_smem = [&](int s, int zi) { return kRowsOff + (s * 3 + zi) * kRow; };
  // thread 0: TMA of the 3 rows (z - 1, z, z + 1) x 4 channel groups of y position yy
  auto issue_fill = [&](int yy) {
    const int s = slot_of(yy);
    const uint32_t bar = su32(&bars[s]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kTxBytes) : "memory");
    const int yw = wrapi(yy, a.Y);
    for (int zi = 0; zi < 3; ++zi) {
      const long long row = (long long)b * plane_rows + (long long)wrapi(z + zi - 1, a.Z) * a.Y + yw;
      for (int g = 0; g < 4; ++g)
        tma_load4(sbase + row_smem(s, zi) + g * kPlane + kInterior * 16, &tmap, 0, g, x0, (int)row, bar);
    }
  };
  // threads 0..23: the periodic neighbours (entries 7 and 136) of the rows of y position yy
  auto halo_fill = [&](int yy) {
    if (tid < 24) {
      const int s = slot_of(yy);
      const int zi = tid >> 3, g = (tid >> 1) & 3, side = tid & 1;
      const int yw = wrapi(yy, a.Y);
      const long long row = (long long)b * plane_rows + (long long)wrapi(z + zi - 1, a.Z) * a.Y + yw;
      const int x = side ? wrapi(x0 + kTM, a.X) : wrapi(x0 - 1, a.X);
      const uint4 v = *reinterpret_cast<const uint4*>(a.Hin + (row * a.X + x) * kCh + g * 8);
      *reinterpret_cast<uint4*>(sm + row_smem(s, zi) + g * kPlane + (side ? kInterior + kTM : kInterior - 1) * 16) = v;
    }
  };
  const int last_row = yb + ny;                    // the last y position any step reads
  __syncthreads();                                 // barriers initialised, TMEM address published
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // thread 0's bookkeeping: rows yb-1 .. issued are filled or in flight, rows yb-1 .. waited have landed
  int issued = yb - 2, waited = yb - 2, mma_steps = 0;
  if (tid == 0)
    for (int yy = yb - 1; yy <= yb + 3 && yy <= last_row; ++yy) {
      issue_fill(yy);
      issued = yy;
    }
  for (int yy = yb - 1; yy <= yb + 3 && yy <= last_row; ++yy) halo_fill(yy);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  // accumulator of step j: wait (warp-uniform) for its MMAs, read back this
  // warp's 32 points, apply the epilogue and store bf16
  auto epilogue = [&](int j) -> bool {
    const int buf = j & 1;
    bool got = bar_wait(su32(&bars[kSlots + buf]), (uint32_t)((j >> 1) & 1), a.wait_ns);
    got = __all_sync(0xffffffffu, got);
    if (!got) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t v[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * 32);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int y = yb + j;
    const long long p = (((long long)b * a.Z + z) * a.Y + y) * a.X + x0 + warp * 32 + lane;
    uint4* dst = reinterpret_cast<uint4*>(a.Hout + p * kCh);
    uint4 mk[4];
    if (a.mode == 1) {
      const uint4* m = reinterpret_cast<const uint4*>(a.Hmask + p * kCh);
#pragma unroll
      for (int q = 0; q < 4; ++q) mk[q] = m[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float f[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) f[e] = __uint_as_float(v[q * 8 + e]);
      if (a.mode == 0) {
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] = fmaxf(f[e], 0.f);
      } else {
        const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mk[q]);
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] = __bfloat162float(mb[e]) > 0.f ? f[e] : 0.f;
      }
      dst[q] = make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    return true;
  };

  bool aborted = false;
  for (int j = 0; j < ny; ++j) {
    const int y = yb + j;
    bool fail = false;
    if (tid == 0) {
      // rows y - 1, y, y + 1 must have landed
      while (!fail && waited < y + 1) {
        const int yy = waited + 1;
        if (bar_wait(su32(&bars[slot_of(yy)]), fill_parity(yy), a.wait_ns)) waited = yy;
        else fail = true;
      }
      if (!fail) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dt = tmem + (uint32_t)((j & 1) * 32);
#pragma unroll 1
        for (int tap = 0; tap < kTaps; ++tap) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          const uint32_t rb = sbase + row_smem(slot_of(y + dy - 1), dz);
#pragma unroll
          for (int kc = 0; kc < 2; ++kc) {
            const uint64_t ad = sdesc(rb + 2 * kc * kPlane + (kInterior - 1 + dx) * 16, kPlane, 128);
            const uint64_t bd = sdesc(sbase + (tap * 2 + kc) * 1024, 512, 128);
            mma_f16(dt, ad, bd, (tap | kc) != 0 ? 1u : 0u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&bars[kSlots + (j & 1)]))
                     : "memory");
        ++mma_steps;
      }
    }
    if (__syncthreads_or(fail)) { aborted = true; break; }
    if (j >= 1) fail = !epilogue(j - 1);
    if (__syncthreads_or(fail)) { aborted = true; break; }
    // the MMAs of row y - 1 were the last to read the ring slot of y - 2:
    // refill it with row y + 3, needed two steps on
    if (j >= 1 && y + 3 <= last_row) {
      if (tid == 0) {
        issue_fill(y + 3);
        issued = y + 3;
      }
      halo_fill(y + 3);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
  }
  if (!aborted && ny >= 1) aborted = __syncthreads_or(!epilogue(ny - 1));
  if (aborted) {
    // drain (bounded) what this CTA still has in flight before its shared and
    // tensor memory are released
    if (tid == 0) {
      *a.flag = 1;
      for (int yy = waited + 1; yy <= issued; ++yy)
        bar_wait(su32(&bars[slot_of(yy)]), fill_parity(yy), 1000000000ull);
      if (mma_steps > 0) {
        const int jl = mma_steps - 1;
        bar_wait(su32(&bars[kSlots + (jl & 1)]), (uint32_t)((jl >> 1) & 1), 1000000000ull);
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// B operands of the 54 MMAs in shared-memory order: (tap, K half kc) block of
// 1024 bytes = 2 K core-matrix columns (kg, 512 bytes apart) x 4 N core
// matrices (128 bytes apart) x 8 rows (16 bytes) of 8 K values. Element
// (n, k) of block (tap, kc), k = 16 kc + 8 kg + kk, is W[tap][k][n]
// (forward) or W[26 - tap][n][k] (backward data: flipped taps, swapped
// channels).
__global__ void k_pack_umma(const float* __restrict__ W, __nv_bfloat16* __restrict__ img, int transposed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kTaps * kCh * kCh) return;
  const int kk = i & 7, n = (i >> 3) & 31, kg = (i >> 8) & 1, kc = (i >> 9) & 1, tap = i >> 10;
  const int k = kc * 16 + kg * 8 + kk;
  const float w = transposed ? W[((kTaps - 1 - tap) * kCh + n) * kCh + k] : W[(tap * kCh + k) * kCh + n];
  const int off = (tap * 2 + kc) * 1024 + kg * 512 + (n >> 3) * 128 + (n & 7) * 16 + kk * 2;
  img[off / 2] = __float2bfloat16_rn(w);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

}  // namespace

bool conv_tc_shape_ok(int X, int Y, int Z) { return X % kTM == 0 && X >= kTM && Y >= 4 && Z >= 1; }

cudaError_t conv_tc_pack(const float* W, __nv_bfloat16* img, int transposed, cudaStream_t s) {
  k_pack_umma<<<(kTaps * kCh * kCh + 255) / 256, 256, 0, s>>>(W, img, transposed);
  return cudaGetLastError();
}

size_t conv_tc_image_bytes() { return (size_t)kWBytes; }

// y rows per CTA: the largest power-of-two divisor of Y (at most Y) that still
// gives at least two CTAs per SM over the launch, but no fewer than 4 rows.
static int pick_ychunk(int X, int Y, int Z, int B, int nsm) {
  const long long cols = (long long)(X / kTM) * Z * B;
  int yc = Y;
  while (yc % 2 == 0 && yc / 2 >= 4 && cols * (Y / yc) < 2LL * nsm) yc /= 2;
  return yc;
}

cudaError_t conv_tc_forward(const __nv_bfloat16* Hin, const __nv_bfloat16* Wimg, __nv_bfloat16* Hout,
                            const __nv_bfloat16* Hmask, int X, int Y, int Z, int B, int mode, int* flag,
                            unsigned long long wait_ns, cudaStream_t s) {
  if (!conv_tc_shape_ok(X, Y, Z) || B < 1 || ((uintptr_t)Hin & 15)) return cudaErrorInvalidValue;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // H as a 4D tensor (8 channels, 4 channel groups, X points, B*Z*Y rows) of bf16
  CUtensorMap map;
  std::memset(&map, 0, sizeof map);
  const cuuint64_t dims[4] = {8, 4, (cuuint64_t)X, (cuuint64_t)B * Z * Y};
  const cuuint64_t strides[3] = {16, 64, (cuuint64_t)X * 64};
  const cuuint32_t box[4] = {8, 1, (cuuint32_t)kTM, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(Hin), dims, strides,
                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAlloc);
  if (e != cudaSuccess) return e;
  ConvTcArgs a;
  a.Hin = Hin;
  a.Wimg = reinterpret_cast<const uint4*>(Wimg);
  a.Hout = Hout;
  a.Hmask = Hmask;
  a.X = X;
  a.Y = Y;
  a.Z = Z;
  a.ychunk = pick_ychunk(X, Y, Z, B, nsm);
  a.mode = mode;
  a.wait_ns = wait_ns;
  a.flag = flag;
  const dim3 grid((unsigned)((X / kTM) * Z * (Y / a.ychunk)), (unsigned)B);
  k_conv_tc<<<grid, 128, kSmemAlloc, s>>>(map, a);
  return cudaGetLastError();
}

}  // namespace gad
