// Launch-argument structures shared by the host driver and the pass kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "state.h"

namespace gad {

// Per-stage description of a mixed-radix Stockham plan.
struct FftStage {
  int radix;        // 2, 3, 4, 8 or 16
  int ns;           // size of the sub-transforms already formed
  int tw_off;       // this stage's block in the plan's twiddle table
  float rcp_lr;     // 1 / (L / radix)
  float rcp_ns;     // 1 / ns
};

// The twiddle table of a plan holds, stage after stage, the factors
// exp(-2 pi i r k / (radix ns)) at tw_off + (r - 1) ns + k (r = 1 .. radix-1,
// k = 0 .. ns-1): the butterflies of consecutive threads (consecutive k) read
// consecutive entries. L - 1 entries in all.
struct FftPlan {
  int L;            // complex length
  int nst;          // number of stages
  FftStage st[8];
  const void* tw;   // the plan's twiddle table (complex, the field's precision)
};

// Prologue (forward x pass) opcodes: compute the field to transform and the
// vector updates that precede G in the algorithm.
enum XfOp : int {
  XF_COPY = 0,   // x = A; if O1: O1 = A
  XF_VC = 1,     // Algorithm 1: U += R (U = O1, R = A); x = R
  XF_CG = 2,     // Algorithm 3: U += alpha P; P = R + beta P (first pass: P = R); x = P
  XF_BI_P = 3,   // Algorithm 4: P = R + beta (P - omega Q) (first pass: P = R); x = P
  XF_BI_S = 4,   // Algorithm 4: S = R - alpha Q; x = S
  XF_MUL = 5,    // closure: x = A_i A_j, field f = pair p of velocity v, A = u* as [v][ncomp][P]
};

// Epilogue (inverse x pass) opcodes, y = G x.
enum XiOp : int {
  XI_STORE = 0,  // O1 = y
  XI_INIT = 1,   // r = A - y -> O1 (R), O2 (F0, optional); dot (r, r)
  XI_RES = 2,    // res = A - y; dot (res, res)
  XI_VC = 3,     // R -= y; dot (R, R)
  XI_CG = 4,     // R -= alpha y; dot (R, R)
  XI_SD = 5,     // U += alpha R; R -= alpha y; dot (R, R)
  XI_BI_Q = 6,   // Q = y; dot (F0, Q)
  XI_BI_T = 7,   // t = y; U += alpha P + omega S; R = S - omega t; dots (R, R), (F0, R)
  XI_TAU = 8,    // closure: O1 = B_i B_j - y (B = u_bar as [v][ncomp][P]; pair of field f as in XF_MUL)
};

// Filter-pass dot opcodes (Parseval sums over the half spectrum).
enum FiOp : int {
  FI_NONE = 0,
  FI_XGX = 1,    // (x, G x)
  FI_SST = 2,    // (s, s), (s, G s), (G s, G s)
};

// Spectral-space pass opcodes (the Krylov iteration on the half spectrum,
// G a pointwise multiply by G_hat(k)). Vectors are complex spectra in the
// layout of the last-axis transform: 2D [kx][ky], 3D [kx][ky][kz].
enum SpOp : int {
  SP_REF = 0,     // d = (b - G b, b - G b)                                  A = b
  SP_INIT = 1,    // r = b - G x, x = B (u0) or A (b); O1 = b (no u0), O2 = r, O3 = r (BiCGSTAB f0); d = (r, r)
  SP_VC = 2,      // Algorithm 1: O1 += O2; O2 -= G O2; d = (O2, O2)
  SP_SD_A = 3,    // Algorithm 2: d = (A, G A)
  SP_SD = 4,      // Algorithm 2: O1 += alpha O2; O2 -= alpha G O2; d = (O2, O2)
  SP_CG_P = 5,    // Algorithm 3: O1 = A (first pass) or A + beta O1; d = (O1, G O1)
  SP_CG = 6,      // Algorithm 3: O1 += alpha A; O2 -= alpha G A; d = (O2, O2)
  SP_BI_P = 7,    // Algorithm 4: O1 = A (first) or A + beta (O1 - omega G O1); d = (B, G O1)
  SP_BI_S = 8,    // Algorithm 4: s = A - alpha G B, t = G s; d = (s, s), (s, t), (t, t)
  SP_BI_END = 9,  // Algorithm 4: s, t from O2 and A; O1 += alpha A + omega s; O2 = s - omega t;
                  //              d = (O2, O2), (B, O2)
  SP_PCG_INIT = 10, // as SP_INIT, and d[1] = (r, M r) (preconditioned CG: rho_0)
  SP_PCG_P = 11,  // preconditioned CG: O1 = M A (first pass) or M A + beta O1; d = (O1, G O1)
  SP_PCG = 12,    // preconditioned CG: O1 += alpha A; O2 -= alpha G A; d = (O2, O2), (O2, M O2)
};

// A batched solve whose passes serve several shape groups per launch: the
// count of fields done in the current pass and the loop passes ([0], [1]),
// and every group's field states for the loop condition.
struct MultiState {
  unsigned ticket[4];
  int ngroups;
  int nfields;               // fields of all groups
  FieldState** st;           // [ngroups] the group's field states
  int* count;                // [ngroups] the group's field count
};

template <typename T>
struct PassArgs {
  int nx, ny, nz, kxn;       // real grid and kxn = nx/2 + 1
  long long P;               // real points per field
  long long SP;              // complex points per spectral buffer per field
  int W, ld;                 // tile width (sequences per block), smem row stride
  int tfft;                  // threads that run FFT butterflies (W*L/E); blockDim.x is
                             // this rounded up to a multiple of 32
  float rcp_a;               // reciprocal helpers for index splits (see kernels)
  float rcp_b;
  FftPlan fft;               // transform along this pass's axis
  FftPlan fft_inv;           // filter pass: the same radices in reverse order
  const void* twx;           // exp(-2 pi i m / nx) table for the real-FFT split
  T kc2;                     // k_c^2
  double inv_p;              // scale of the block dots: 1/P for Parseval sums, else 1
  T gscale;                  // 1/P folded into the filter multiply
  T cx, cy, cz;              // preconditioner stencil weights (delta/h_d)^2 of the x, y, z axes
  int ncomp, npairs;         // closure: components per velocity, pairs i <= j per velocity
  int pair_code;             // closure: pair p = (i, j) at bits 4p (i) and 4p + 2 (j)
  unsigned long long wait_ns;  // limit of a bounded device wait (0: give up at once)
  int chunk;                 // preconditioner stencil: positions of the march axis per block
  int rev;                   // fields in reverse launch order: field f = gridDim.y - 1 - blockIdx.y
  int vgx, vgy;              // launch shape of this group's pass (blocks per field, fields) in k_multi
  int vbd;                   // block size of that launch shape (0: blockDim.x)
  MultiState* ms;            // nullptr, or the batched solve this pass belongs to (k_multi)
  void* S1;
  void* S2;
  const T* A;
  const T* B;
  const T* C;
  T* O1;
  T* O2;
  T* O3;
  int op;
  int ndots;
  FieldState* st;            // nullptr for plain filtering
  SolveConfig cfg;
  double* part;              // [batch][gridDim.x][4] block partial dots
  unsigned* ticket;          // [0] fields done, [1] loop passes, [2 + f] blocks of field f
  int stage;                 // ScalarStage run by the last block
  int set_cond;              // last block sets the graph's while-condition
  cudaGraphConditionalHandle cond;
  int batch;
  int force;                 // run for every field regardless of its active flag
  int clear_cond;            // block (0,0) resets the while-condition to 0 first,
                             // so the loop ends unless the last pass re-arms it
};

}  // namespace gad
