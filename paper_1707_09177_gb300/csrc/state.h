// Device-side solver state shared by the pass kernels and the host driver.
#pragma once

#include <stdint.h>

namespace gad {

// Per-field scalars of one solve (float64 on the device). The recurrences
// follow Algorithms 1, 3 and 4; alpha/beta/omega/rho keep the paper's names.
struct FieldState {
  double rho;        // CG: (r_n, r_n); BiCGSTAB: rho_{n+1} = (f0, r_n)
  double alpha;
  double beta;
  double omega;
  double ref;        // ||u_bar - G u_bar||_2 (normaliser of the history)
  double h;          // last normalised residual
  double true_res;   // ||u_bar - G u|| / ref after the solve (optional)
  int iter;          // completed passes
  int status;        // ad_status value
  int active;        // 1 while the field still iterates
  int early;         // BiCGSTAB: this pass ends with omega = 0 (s small)
  int fin_axpy;      // CG: the final u += alpha p is still owed
  int have_ref;      // ref supplied by a separate pass (explicit u0)
  int fault;         // a bounded device wait of this field gave up (AD_ERR_TIMEOUT)
  int pad;
};

struct SolveConfig {
  double tol;
  int maxit;
  int method;
  double* hist;      // [batch][maxit + 1]
  int hist_ld;
};

// Which scalar update the last block of a dot-producing pass performs.
enum ScalarStage : int {
  SS_NONE = 0,
  SS_REF = 1,        // dots: (r,r) of u_bar - G u_bar       -> ref
  SS_INIT = 2,       // dots: (r0,r0)                        -> h_0, start
  SS_VC = 3,         // dots: (r,r)                          -> Algorithm 1 step end
  SS_CG_ALPHA = 4,   // dots: (p, G p)                       -> alpha_n
  SS_CG_BETA = 5,    // dots: (r,r)                          -> beta_n, stop test
  SS_BI_ALPHA = 6,   // dots: (f0, q)                        -> alpha_{n+1}
  SS_BI_OMEGA = 7,   // dots: (s,s), (s,t), (t,t)            -> omega_{n+1}
  SS_BI_END = 8,     // dots: (r,r), (f0, r)                 -> stop test, beta
  SS_TRUE = 9,       // dots: (res,res)                      -> true residual
  SS_SD_ALPHA = 10,  // dots: (r, G r)                       -> alpha_n (Algorithm 2)
  SS_PCG_RHO = 11,   // dots: (r, z), z = M r                -> rho, beta (preconditioned CG)
  SS_PCG_STOP = 12,  // dots: (r, r)                         -> stop test (preconditioned CG)
  SS_PCG_INIT = 13,  // dots: (r0, r0), (r0, z0)             -> h_0, start; rho = (r0, z0)
  SS_PCG_END = 14,   // dots: (r, r), (r, z)                 -> stop test, then rho, beta
};

}  // namespace gad
