// 32 -> 32 convolution layers of the learned initial guess on the Blackwell
// tensor cores (tcgen05): an implicit GEMM whose accumulator lives in tensor
// memory and whose activation rows are staged by TMA.
//
// One CTA owns an x-segment of 128 points of one (field, z) plane and a range
// of y. Output row y is
//     D_y[128 points][32 out channels] = sum over taps (dz, dy, dx) and 2 halves of
//         16 input channels of  A_{z+dz-1, y+dy-1, dx}[128][16] * W_{dz,dy,dx}[16][32].
// The CTA walks the INPUT rows y' instead: one input row (three z planes)
// contributes to the three output rows y'+1, y', y'-1 through the taps
// dy = 0, 1, 2, so for each (dz, dx, K half) one tcgen05.mma with N = 96
// (M = 128 points, K = 16 channels, bf16 inputs, float32 accumulation) adds
// A_{dz, y', dx} times the three tap blocks [W_{dz,0,dx} | W_{dz,1,dx} |
// W_{dz,2,dx}] into the accumulators of those three output rows at once: 18
// MMAs per input row instead of 54 with N = 32, and every staged row is used
// by one batch of MMAs. The accumulators of the output rows live in a ring of
// sixteen 32-column slots of tensor memory laid out so that rows y'+1, y',
// y'-1 occupy consecutive slots (slot(y) decreases with y); where the three
// wrap around the ring the MMA is split in two. Every slot starts at zero (the
// epilogue clears a slot after reading it) and every MMA accumulates.
// A_{dz, y', dx} is not materialised: the staged rows hold every point of the
// segment plus one periodic neighbour on each side, one 64-byte row (its 32
// channels) per point in the K-major layout with the 64-byte swizzle, so the
// x offset of a tap is a shift of the descriptor's start address by one row
// and the second half of K a shift by 32 bytes. The warps have one role each
// and hand work over through mbarriers:
//   warp 4 (producer): stages input rows (three z planes: one TMA load of the
//     128 interior points each, swizzled on the way in, and plain loads of the
//     two periodic neighbours, fetched one row ahead) into a ring of six slots,
//     refilling a slot as soon as the MMAs of the row it held have completed;
//   warp 5 (MMA): allocates the tensor memory, and for each input row waits
//     for its staging (and for the slot of the output row entering the ring to
//     be cleared), issues its MMAs, and commits them to the "empty" barrier of
//     the input slot and to the "full" barrier of the output row y'-1, which
//     no later input row touches;
//   warps 0-3 (epilogue): wait for an output row, read its accumulator back
//     (tcgen05.ld, warp w owning tensor-memory lanes 32w .. 32w+31), clear it
//     (tcgen05.st of zeros), release the slot, apply the epilogue (ReLU, or the
//     ReLU mask of the backward pass) and store bf16.
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
constexpr int kPt = 64;                        // bytes per staged point: its 32 channels, one swizzled row
constexpr int kInterior = 8;                   // row of the segment's first point (512-byte aligned)
constexpr int kRow = 144 * kPt;                // one staged z plane: 144 point rows (9216 bytes)
constexpr int kSlots = 6;                      // y positions in the ring
constexpr int kBBlock = 96 * 16 * 2;            // B operand of one (dz, dx, K half): 96 x 16 bf16
constexpr int kWBytes = 9 * 2 * kBBlock;          // all of them (55296 bytes)
constexpr int kRowsOff = kWBytes;              // staged rows after the weights
constexpr int kBarOff = kRowsOff + kSlots * 3 * kRow;
constexpr int kSmemUsed = kBarOff + 512;
// the whole shared memory of an SM (one CTA per SM): every address a
// descriptor can reach under either reading of its two stride fields stays
// inside the allocation
constexpr int kSmemAlloc = 227 * 1024;
constexpr int kTxBytes = 3 * kTM * kPt;       // bytes of one ring fill (3 planes x 128 points x 64 bytes)
constexpr int kAcc = 16;                       // output-row accumulators in tensor memory
constexpr uint32_t kTmemCols = 32 * kAcc;      // 32 float32 columns each: all 512 columns
constexpr int kThreads = 192;                  // 4 epilogue warps, producer warp, MMA warp

static_assert(kSmemUsed <= kSmemAlloc, "shared-memory layout exceeds the allocation");
static_assert(kRow % 1024 == 0 && kRowsOff % 1024 == 0 && (kInterior * kPt) % 512 == 0,
              "TMA destinations aligned to the 512-byte period of the 64-byte swizzle");

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

// Shared-memory matrix descriptor, K-major with the 64-byte swizzle: rows of
// 64 bytes (32 bf16 of K) whose four 16-byte chunks are permuted by
// chunk ^= bits 7-8 of the row's shared-memory address (the layout a TMA load
// with the 64-byte swizzle writes), 8-row groups 512 bytes apart (stride
// offset), the leading offset unused (encoded as 1), layout type 4. The
// tensor cores apply the permutation to the final addresses, so a start
// address shifted by whole 64-byte rows, or by 32 bytes for the second half
// of K, addresses the shifted matrix.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) |
         (4ull << 61);
}

// Instruction descriptor of tcgen05.mma kind::f16: D float32, A and B bf16,
// both K-major, M = 128, N given (a multiple of 16, at most 256).
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, 1, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc)
      : "memory");
}

__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
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

// grid x = (X/128) * Z * (Y/ychunk), grid y = fields; kThreads threads
__global__ void __launch_bounds__(kThreads, 1) k_conv_tc(const __grid_constant__ CUtensorMap tmap, const ConvTcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nxs = a.X / kTM;
  int r = blockIdx.x;
  const int xs = r % nxs;
  r /= nxs;
  const int z = r % a.Z;
  const int yc = r / a.Z;
  const int b = blockIdx.y;
  const int x0 = xs * kTM, yb = yc * a.ychunk, ny = a.ychunk;
  // barriers: full[kSlots] / empty[kSlots] (input ring slot staged / read by its MMAs),
  // accf[16] (output row's accumulator complete), acce[16] (read back and cleared)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kBarOff);
  const uint32_t full0 = su32(bars), empty0 = full0 + 8 * kSlots, accf0 = empty0 + 8 * kSlots,
                 acce0 = accf0 + 8 * kAcc;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kBarOff + 8 * (2 * kSlots + 2 * kAcc));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* rows_issued = reinterpret_cast<int*>(tmem_slot + 2);     // producer: input rows staged or in flight
  int* rows_done = reinterpret_cast<int*>(tmem_slot + 3);       // MMA warp: input rows whose MMAs it committed
  int* rows_ready = reinterpret_cast<int*>(tmem_slot + 4);      // MMA warp: input rows whose staging it waited for
  const uint32_t sbase = su32(sm);

  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kSlots; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * i) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * i) : "memory");
    }
    for (int i = 0; i < kAcc; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(accf0 + 8 * i) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(acce0 + 8 * i) : "memory");
    }
    *abort_flag = 0;
    *rows_issued = 0;
    *rows_done = 0;
    *rows_ready = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights: generic copy of the B-operand image, visible to the tensor cores
  {
    uint4* w = reinterpret_cast<uint4*>(sm);
    for (int i = tid; i < kWBytes / 16; i += kThreads) w[i] = __ldg(a.Wimg + i);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (warp < 4) {
    // every accumulator slot starts at zero (the MMAs always accumulate)
    uint32_t zr[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) zr[q] = 0u;
    for (int sl = 0; sl < kAcc; ++sl) {
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sl * 32);
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
          "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
          ::"r"(ta), "r"(zr[0]), "r"(zr[1]), "r"(zr[2]), "r"(zr[3]), "r"(zr[4]), "r"(zr[5]), "r"(zr[6]), "r"(zr[7]),
            "r"(zr[8]), "r"(zr[9]), "r"(zr[10]), "r"(zr[11]), "r"(zr[12]), "r"(zr[13]), "r"(zr[14]), "r"(zr[15]),
            "r"(zr[16]), "r"(zr[17]), "r"(zr[18]), "r"(zr[19]), "r"(zr[20]), "r"(zr[21]), "r"(zr[22]), "r"(zr[23]),
            "r"(zr[24]), "r"(zr[25]), "r"(zr[26]), "r"(zr[27]), "r"(zr[28]), "r"(zr[29]), "r"(zr[30]), "r"(zr[31])
          : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const long long plane_rows = (long long)a.Y * a.Z;     // rows per field
  const int nrows = ny + 2;                              // input rows: y positions yb - 1 .. yb + ny
  auto row_smem = [&](int s, int zi) { return kRowsOff + (s * 3 + zi) * kRow; };
  // accumulator slot of output row yb + m: consecutive output rows take
  // consecutive slots downwards, so rows y'+1, y', y'-1 are ascending slots
  auto acc_slot = [&](int m) { return (kAcc * 4096 - m) % kAcc; };
  // bounded wait that also gives up when another role has aborted
  auto wait = [&](uint32_t bar, uint32_t parity) -> bool {
    if (a.wait_ns == 0) return false;
    {
      // fast path: a phase that has completed costs no timer read
      uint32_t done;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(bar), "r"(parity)
          : "memory");
      if (done) return true;
    }
    // the abort flag and the timer are read every 64 polls only: polling
    // competes with the tensor cores for shared-memory bandwidth
    const uint64_t t0 = gtime();
    for (unsigned it = 1;; ++it) {
      uint32_t done;
      // suspend hint 20 us: the thread sleeps until the phase completes
      // instead of polling
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(bar), "r"(parity), "r"(20000u)
          : "memory");
      if (done) return true;
      if ((it & 63u) == 0u && (*abort_flag || gtime() - t0 > a.wait_ns)) return false;
    }
  };
  // the same wait for a whole warp: lane 0 polls, the others wait for its
  // answer at the shuffle (ordered after lane 0's observation of the phase)
  auto wait_warp = [&](uint32_t bar, uint32_t parity) -> bool {
    bool ok = false;
    if (lane == 0) ok = wait(bar, parity);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  };

  if (warp == 4) {
    // ---- producer: input rows i = 0 .. nrows-1 (y position yb - 1 + i) into
    // slot i % kSlots: per z plane one TMA load of the 128 interior points
    // (rows kInterior ..), and the two periodic neighbours (rows kInterior - 1
    // and kInterior + 128) by lanes 0-23, 16 bytes each (plane lane / 8, side
    // (lane / 4) & 1, chunk lane & 3), loaded one input row ahead so that
    // their latency overlaps the previous row's staging
    const int hzi = lane >> 3, hside = (lane >> 2) & 1, hc = lane & 3;
    const int hx = hside ? wrapi(x0 + kTM, a.X) : wrapi(x0 - 1, a.X);
    auto halo_load = [&](int i) -> uint4 {
      const long long row = (long long)b * plane_rows + (long long)wrapi(z + hzi - 1, a.Z) * a.Y + wrapi(yb - 1 + i, a.Y);
      return *reinterpret_cast<const uint4*>(a.Hin + (row * a.X + hx) * kCh + hc * 8);
    };
    uint4 hv = make_uint4(0u, 0u, 0u, 0u);
    if (lane < 24) hv = halo_load(0);
    for (int i = 0; i < nrows; ++i) {
      const int s = i % kSlots;
      bool ok = true;
      if (i >= kSlots) ok = wait_warp(empty0 + 8 * s, (uint32_t)(((i / kSlots) - 1) & 1));
      if (!ok) { *abort_flag = 1; break; }
      if (lane < 24) {
        const uint32_t ra = sbase + row_smem(s, hzi) + (hside ? kInterior + kTM : kInterior - 1) * kPt;
        const uint32_t dst = ra + ((uint32_t)(hc ^ ((ra >> 7) & 3)) << 4);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(hv.x), "r"(hv.y), "r"(hv.z), "r"(hv.w)
                     : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (i + 1 < nrows) hv = halo_load(i + 1);
      }
      __syncwarp();
      if (lane == 0) {
        const uint32_t bar = full0 + 8 * s;
        const int yw = wrapi(yb - 1 + i, a.Y);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kTxBytes) : "memory");
#pragma unroll
        for (int zi = 0; zi < 3; ++zi) {
          const int row = (int)((long long)b * plane_rows + (long long)wrapi(z + zi - 1, a.Z) * a.Y + yw);
          tma_load3(sbase + row_smem(s, zi) + kInterior * kPt, &tmap, 0, x0, row, bar);
        }
        *rows_issued = i + 1;
      }
      __syncwarp();
    }
  } else if (warp == 5) {
    // ---- MMA issue (lane 0): input row i = y' - (yb - 1) touches output rows
    // m = i, i - 1, i - 2 (relative to yb) through dy = 0, 1, 2
    if (lane == 0) {
      // descriptors of the first A tile (slot 0, dz = dx = kc = 0) and the
      // first B block (dz = dx = kc = 0, dy = 0)
      const uint64_t a0 = sdesc_sw64(sbase + kRowsOff + (kInterior - 1) * kPt);
      const uint64_t b0 = sdesc(sbase, kBBlock / 2, 128);
      for (int i = 0; i < nrows; ++i) {
        bool ok = wait(full0 + 8 * (i % kSlots), (uint32_t)((i / kSlots) & 1));
        if (ok) *rows_ready = i + 1;
        // output row m = i enters the ring: its slot's previous row (m - 16)
        // must have been read back and cleared
        if (ok && i < ny && i >= kAcc) ok = wait(acce0 + 8 * acc_slot(i), (uint32_t)(((i - kAcc) / kAcc) & 1));
        if (!ok) { *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int hi = min(i, ny - 1), lo = max(i - 2, 0);          // output rows in this CTA's range
        if (hi >= lo) {
          // runs of consecutive slots: rows hi, hi - 1, .., lo ascend through the slots
          int m0 = hi, cnt = hi - lo + 1;
          while (cnt > 0) {
            const int s0 = acc_slot(m0);
            const int run = min(cnt, kAcc - s0);
            const int g0 = i - m0;                                  // tap dy of output row m0
            const uint32_t dt = tmem + (uint32_t)(s0 * 32);
            const uint32_t idesc = idesc_n(32 * run);
            // the 18 MMAs of the run: their descriptors differ from the row's
            // first ones by compile-time offsets (in 16-byte units of the
            // start-address field, which stays below 2^14 inside shared
            // memory), so the issuing thread spends a few instructions per MMA
            const uint64_t arow = a0 + (uint64_t)((i % kSlots) * (3 * kRow / 16));
            const uint64_t brow = b0 + (uint64_t)(g0 * (512 / 16));
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
              for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                for (int kc = 0; kc < 2; ++kc)
                  mma_f16(dt, arow + (uint64_t)((dz * kRow + dx * kPt + kc * 32) / 16),
                          brow + (uint64_t)((((dz * 3 + dx) * 2 + kc) * kBBlock) / 16), idesc);
            m0 -= run;
            cnt -= run;
          }
        }
        // the staged row is read by no later MMA
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         empty0 + 8 * (i % kSlots))
                     : "memory");
        // output row i - 2 receives nothing more
        if (i >= 2 && i - 2 < ny)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           accf0 + 8 * acc_slot(i - 2))
                       : "memory");
        *rows_done = i + 1;
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue warps 0-3: output rows m = 0 .. ny-1
    uint32_t zr[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) zr[q] = 0u;
    for (int m = 0; m < ny; ++m) {
      const int sl = acc_slot(m);
      const bool ok = wait_warp(accf0 + 8 * sl, (uint32_t)((m / kAcc) & 1));
      if (!ok) { *abort_flag = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(sl * 32);
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
      // clear the slot for the output row that takes it next
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
          "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
          ::"r"(taddr), "r"(zr[0]), "r"(zr[1]), "r"(zr[2]), "r"(zr[3]), "r"(zr[4]), "r"(zr[5]), "r"(zr[6]),
            "r"(zr[7]), "r"(zr[8]), "r"(zr[9]), "r"(zr[10]), "r"(zr[11]), "r"(zr[12]), "r"(zr[13]), "r"(zr[14]),
            "r"(zr[15]), "r"(zr[16]), "r"(zr[17]), "r"(zr[18]), "r"(zr[19]), "r"(zr[20]), "r"(zr[21]), "r"(zr[22]),
            "r"(zr[23]), "r"(zr[24]), "r"(zr[25]), "r"(zr[26]), "r"(zr[27]), "r"(zr[28]), "r"(zr[29]), "r"(zr[30]),
            "r"(zr[31])
          : "memory");
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce0 + 8 * sl) : "memory");
      const int y = yb + m;
      const long long p = (((long long)b * a.Z + z) * a.Y + y) * a.X + x0 + warp * 32 + lane;
      uint4* dst = reinterpret_cast<uint4*>(a.Hout + p * kCh);
      uint4 mk[4];
      if (a.mode == 1) {
        const uint4* mp = reinterpret_cast<const uint4*>(a.Hmask + p * kCh);
#pragma unroll
        for (int q = 0; q < 4; ++q) mk[q] = mp[q];
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
    }
  }
  __syncthreads();
  if (*abort_flag && tid == 0) {
    // drain (bounded) what this CTA still has in flight before its shared and
    // tensor memory are released: the staged rows no MMA batch waited for, and
    // the MMAs of the last committed input row
    *a.flag = 1;
    const int ri = *rows_issued, rr = *rows_ready, rd = *rows_done;
    for (int i = rr; i < ri; ++i) bar_wait(full0 + 8 * (i % kSlots), (uint32_t)((i / kSlots) & 1), 1000000000ull);
    if (rd > 0) {
      const int i = rd - 1;
      bar_wait(empty0 + 8 * (i % kSlots), (uint32_t)((i / kSlots) & 1), 1000000000ull);
    }
  }
  __syncthreads();
  if (warp == 5) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// B operands in shared-memory order: block (dz, dx, K half kc) of kBBlock
// bytes = 2 K core-matrix columns (kg, kBBlock/2 bytes apart) x 12 N core
// matrices (128 bytes apart) x 8 rows (16 bytes) of 8 K values. Row n of the
// block is output channel n % 32 of tap dy = n / 32; element (n, k), k = 16 kc +
// 8 kg + kk, is W[tap][k][n % 32] (forward) or W[26 - tap][n % 32][k] (backward
// data: flipped taps, swapped channels), tap = (dz * 3 + dy) * 3 + dx.
__global__ void k_pack_umma(const float* __restrict__ W, __nv_bfloat16* __restrict__ img, int transposed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kTaps * kCh * kCh) return;
  const int kk = i & 7, n = (i >> 3) % 96, rest = (i >> 3) / 96;     // rest = ((dz * 3 + dx) * 2 + kc) * 2 + kg
  const int kg = rest & 1, kc = (rest >> 1) & 1, dzdx = rest >> 2;
  const int dz = dzdx / 3, dx = dzdx % 3, dy = n / 32, co = n % 32;
  const int tap = (dz * 3 + dy) * 3 + dx;
  const int k = kc * 16 + kg * 8 + kk;
  const float w = transposed ? W[((kTaps - 1 - tap) * kCh + co) * kCh + k] : W[(tap * kCh + k) * kCh + co];
  const int off = (dzdx * 2 + kc) * kBBlock + kg * (kBBlock / 2) + (n >> 3) * 128 + (n & 7) * 16 + kk * 2;
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
  if ((long long)B * Z * Y >= (1LL << 31)) return cudaErrorInvalidValue;     // TMA row coordinates are int32
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // H as a 3D tensor (32 channels, X points, B*Z*Y rows) of bf16; a box is
  // 128 points of one row, written to shared memory with the 64-byte swizzle
  CUtensorMap map;
  std::memset(&map, 0, sizeof map);
  const cuuint64_t dims[3] = {(cuuint64_t)kCh, (cuuint64_t)X, (cuuint64_t)B * Z * Y};
  const cuuint64_t strides[2] = {(cuuint64_t)kPt, (cuuint64_t)X * kPt};
  const cuuint32_t box[3] = {(cuuint32_t)kCh, (cuuint32_t)kTM, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(Hin), dims, strides,
                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
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
  k_conv_tc<<<grid, kThreads, kSmemAlloc, s>>>(map, a);
  return cudaGetLastError();
}

}  // namespace gad
