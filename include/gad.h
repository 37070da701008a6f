/*
 * gad.h -- C ABI of the generalized approximate-deconvolution library.
 *
 * The library solves the approximate-deconvolution (AD) problem of San &
 * Vedula, "Generalized deconvolution procedure for structural modeling of
 * turbulence": given a filtered field u_bar on a periodic grid, recover u
 * with G u = u_bar (Section 3, Eq. tau3), where G is the Germano elliptic
 * differential filter G = (I - delta^2 Laplacian)^{-1}, delta = 1/k_c,
 * k_c = gamma k_m (Section 4, Eq. df), applied spectrally with transfer
 * function G_hat(k) = 1/(1 + (|k|/k_c)^2) (Eq. df2). The solve uses Van
 * Cittert (Algorithm 1), steepest descent (Algorithm 2), conjugate gradient
 * (Algorithm 3) or BiCGSTAB (Algorithm 4) iterations, all on one GPU.
 *
 * Conventions shared by every entry point
 *   - Fields are real, C-ordered with x contiguous, on a 2*pi-periodic grid:
 *     field b, point (z, y, x) is element b*P + (z*Ny + y)*Nx + x, with
 *     P = Nx*Ny*Nz (Nz = 1 in 2D). Wavenumbers are integers; k_m = min(N)/2.
 *   - Supported sides: every N_d of the form 2^a 3^b, N_d >= 8, with Nx a
 *     multiple of 4 and Ny, Nz even (powers of two and 2^a 3^b with a >= 2
 *     cover all workloads).
 *   - Field pointers are DEVICE pointers owned by the caller, 16-byte
 *     aligned, holding `batch` contiguous fields of the grid's dtype
 *     (float for AD_F32, double for AD_F64). The library owns its workspace
 *     (spectral buffers, Krylov vectors, scalars) inside the context and
 *     allocates it on the first call for a grid shape and batch size; later
 *     calls with that shape allocate nothing. A call takes at most
 *     AD_MAX_BATCH fields (each field owns one row of the launch grid).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is enqueued on it.
 *   - No entry point throws. Arguments are checked before any launch; an
 *     error returns a negative status and leaves outputs unspecified.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef GAD_H
#define GAD_H

#include <stdint.h>

#define AD_MAX_BATCH 65535

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AD_OK = 0,              /* converged: h_n <= tol                              */
  AD_MAXIT = 1,           /* maxit passes done without reaching tol (fixed-N)   */
  AD_BREAKDOWN = 2,       /* a Krylov scalar vanished or is not finite          */
  AD_ERR_ARG = -1,        /* bad argument (shape, pointer, method, batch ...)   */
  AD_ERR_NONFINITE = -2,  /* the initial residual is NaN or Inf                 */
  AD_ERR_CUDA = -3,       /* a CUDA runtime call failed                         */
  AD_ERR_TIMEOUT = -4,    /* a bounded device wait gave up                      */
  AD_ERR_NOMEM = -5       /* device allocation of the workspace failed          */
} ad_status;

typedef enum {
  AD_VANCITTERT = 0,      /* Algorithm 1 */
  AD_CG = 1,              /* Algorithm 3 */
  AD_BICGSTAB = 2,        /* Algorithm 4 */
  AD_SD = 3,              /* Algorithm 2 */
  /* Flag OR-ed into a method: iterate on the half spectra of the vectors.
   * G is diagonal in Fourier space (Eq. df2), so each pass is a pointwise
   * multiply by G_hat with the vector updates and Parseval inner products
   * fused into one streaming kernel (one for VC, two for SD and CG, three
   * for BiCGSTAB); u_bar is transformed once before the loop and u once
   * after it. Same iterates as the physical-space method in exact
   * arithmetic; in floating point the result differs by rounding. Accepted
   * by ad_deconvolve, ad_deconvolve_batched, ad_time_pass and ad_autotune. */
  AD_SPECTRAL = 4,
  /* Flag OR-ed into AD_CG, in physical space or with AD_SPECTRAL (with any
   * other method it is AD_ERR_ARG): preconditioned CG. The paper solves Eq. tau3 without a
   * preconditioner; this flag adds the textbook preconditioned CG with M,
   * the second-order periodic finite-difference version of the filter's
   * differential inverse G^{-1} = I - delta^2 Laplacian (Section 4, Eq. df):
   *   z = M r = r + sum_d c_d (2 r_i - r_{i+e_d} - r_{i-e_d}),
   *   c_d = (delta/h_d)^2 = (N_d / (2 pi k_c))^2,
   * evaluated in the field's precision as ((r + c_x d_x) + c_y d_y) + c_z d_z
   * with d = (2 r - left) - right, each operation rounded once. M is
   * symmetric positive definite and commutes with G; M G has its spectrum in
   * [4/pi^2, 1], so the pass count no longer grows with |k|^2/k_c^2. Per
   * pass: one stencil pass (z = M r, (r, z)) and one application of G with
   * Algorithm 3's updates (p = z + beta p); in spectral space M is the
   * pointwise multiply by its symbol M_hat(k) = 1 + sum_d 4 c_d sin^2(pi k_d /
   * N_d) inside two streaming passes. Same stopping rules and history
   * (unpreconditioned residual ||r_n|| / ||u_bar - G u_bar||); rho_n =
   * (r_n, z_n) <= 0 or not finite is AD_BREAKDOWN. Accepted by
   * ad_deconvolve, ad_deconvolve_batched and ad_time_pass. */
  AD_PRECOND = 8
} ad_method;

typedef enum { AD_F32 = 0, AD_F64 = 1 } ad_dtype;

typedef struct {
  int ndim;               /* 2 or 3                                              */
  int64_t n[3];           /* n[0] = Nx (contiguous), n[1] = Ny, n[2] = Nz (3D)   */
  ad_dtype dtype;         /* storage and FFT precision of the fields            */
  double gamma;           /* filter strength: k_c = gamma * min(N)/2, 0 < gamma  */
} ad_grid;

typedef struct ad_ctx ad_ctx;   /* opaque: plans, twiddle tables, workspaces, graphs */

/* Creates a context on CUDA device `device`. *ctx receives the handle, which
 * the caller releases with ad_destroy. Library housekeeping, no counterpart
 * in the paper. */
ad_status ad_create(ad_ctx** ctx, int device);

/* Frees every device buffer, graph and stream the context owns. NULL is
 * ignored. Library housekeeping, no counterpart in the paper. */
void ad_destroy(ad_ctx* ctx);

/* out = G in for `batch` fields (Section 4, Eq. df / Eq. df2, evaluated by
 * FFT). `in` and `out` may be the same buffer. batch = 0 is a no-op. */
ad_status ad_filter(ad_ctx* ctx, const ad_grid* grid, const void* in, void* out,
                    int batch, void* stream);

/* Solves G u = u_bar for `batch` independent fields (Section 3, Eq. tau3) with
 * `method`, each field with its own scalars and stopping decision.
 *   ubar        device, batch fields, input (not modified)
 *   u_out       device, batch fields, output u*; must not alias ubar
 *   tol, maxit  stop at the first pass n with h_n = ||r_n|| / ||u_bar - G u_bar||
 *               <= tol (AD_OK) or after maxit passes (AD_MAXIT); tol = 0,
 *               maxit = N runs exactly N passes. h_0 is tested first
 *               (h_0 <= tol -> 0 passes). maxit >= 0.
 *   u0          device initial guess (batch fields) or NULL for u0 = u_bar;
 *               the history stays normalised by ||u_bar - G u_bar||.
 *   iterations  host int[batch] (may be NULL): completed passes per field
 *   status      host ad_status[batch] (may be NULL): outcome per field
 *   res_hist    host double[batch][maxit+1] (may be NULL): h_0 .. h_iterations
 *               per field; entries after a field's last pass are unspecified
 *   true_res    host double[batch] (may be NULL): ||u_bar - G u*|| / ref,
 *               computed with one extra application of G when requested
 * Inner products and scalar recurrences run in float64 on the device; AD_F32
 * fields accumulate products in compensated float32 that is widened to
 * float64 per thread. The call returns when u_out and the host outputs are
 * ready. Return value: AD_OK if every field converged, otherwise the status of
 * the first field that did not (errors before launch are negative). */
ad_status ad_deconvolve(ad_ctx* ctx, const ad_grid* grid, const void* ubar, void* u_out,
                        int batch, ad_method method, double tol, int maxit,
                        const void* u0, int* iterations, ad_status* status,
                        double* res_hist, double* true_res, void* stream);

/* ad_deconvolve with the fields in HOST memory (Section 3, Eq. tau3; the same
 * Algorithms 1-4 and stopping rules): copies u_bar to device buffers that the
 * context owns for this grid and batch, solves from u0 = u_bar, and copies u*
 * back, all on `stream`.
 *   ubar        host, batch fields in the layout of ad_deconvolve (pinned
 *               memory copies fastest; pageable memory works)
 *   u_out       host, same size; may be ubar itself (u_bar is read in full
 *               before u_out is written)
 *   iterations, status, res_hist: as for ad_deconvolve
 * Returns when u_out and the host outputs are ready, with ad_deconvolve's
 * return value. Argument, allocation and CUDA errors (AD_ERR_ARG, AD_ERR_NOMEM,
 * AD_ERR_CUDA) leave u_out untouched; per-field outcomes, AD_ERR_NONFINITE
 * included, come with u_out written. */
ad_status ad_deconvolve_host(ad_ctx* ctx, const ad_grid* grid, const void* ubar, void* u_out,
                             int batch, ad_method method, double tol, int maxit,
                             int* iterations, ad_status* status, double* res_hist, void* stream);

/* Solves G u = u_bar for `nfields` fields of possibly different grids (2D and
 * 3D, any supported sizes, dtypes and gammas) in one call: one CUDA graph
 * whose concurrent branches each solve the fields of one grid shape (gathered
 * into a contiguous workspace, solved with their own device-side while loop,
 * scattered back). Same algorithms, stopping rules and precision as
 * ad_deconvolve, u0 = u_bar for every field.
 *   grids      host ad_grid[nfields]
 *   ubar       host array of nfields device pointers (inputs)
 *   u_out      host array of nfields device pointers (outputs, no aliasing)
 *   iterations host int[nfields] (may be NULL)
 *   status     host ad_status[nfields] (may be NULL)
 *   res_hist   host array of nfields host pointers to double[maxit+1] (the
 *              array or any entry may be NULL)
 * The graph is built on the first call for a given set of grids, pointers,
 * method, tol and maxit and reused afterwards. Returns AD_OK if every field
 * converged, else the status of the first field (in group order) that did not.
 * Batching of the paper's per-field solves; no counterpart in the paper. */
ad_status ad_deconvolve_batched(ad_ctx* ctx, int nfields, const ad_grid* grids, const void* const* ubar,
                                void* const* u_out, ad_method method, double tol, int maxit, int* iterations,
                                ad_status* status, double* const* res_hist, void* stream);

/* Learned initial guess for BiCGSTAB (no counterpart in the paper): a bias-free
 * 3x3x3 convolutional network with periodic padding, channels 1 -> 32 -> 32 ->
 * 32 -> 1, ReLU after the first three layers, applied to u_bar / sigma
 * (sigma = RMS of u_bar) with residual output u0 = u_bar + sigma * A * y,
 * A = 1/(pi gamma)^2 = (delta/h)^2 taken from the grid's gamma; pass u0 to
 * ad_deconvolve. bfloat16 activations, float32 accumulation (tensor cores
 * for the 32 -> 32 layers). Fields: 3D float32, Nx a multiple of 32.
 * Weights: float32 array of ad_guess_weight_count() values, layout
 *   W1[27][32], W2[27][32][32], W3[27][32][32], W4[27][32]  (tap, in, out),
 *   tap = (a*3 + b)*3 + c weighting the input at (z+a-1, y+b-1, x+c-1).
 * All field and weight pointers are device pointers unless stated. */
int64_t ad_guess_weight_count(void);

/* Initial weights (learned guess; the stencil start restates the inverse of
 * G, Eq. df) into a HOST array of n = ad_guess_weight_count() floats,
 * from a splitmix64 stream seeded by seed. stencil = 0: He-normal (last layer
 * scaled by 0.1). stencil != 0: the explicit local inverse of G,
 * u0 = u_bar - (delta/h)^2 L_h u_bar with the 7-point Laplacian L_h (channels
 * 0 and 1 carry +L and -L through the ReLUs), every other weight He-normal
 * scaled by 1e-3, so training starts from that approximation. */
ad_status ad_guess_init(float* weights_host, int64_t n, uint64_t seed, int stencil);

/* u0 = u_bar + sigma * A * CNN(u_bar / sigma) for `batch` fields (the learned
 * guess described above; no counterpart in the paper). */
ad_status ad_guess_infer(ad_ctx* ctx, const ad_grid* grid, const float* weights, const float* ubar, float* u0,
                         int batch, void* stream);

/* Loss (host double, batch mean of ||u0 - u_true||^2 / ||u_true||^2) and its
 * gradient with respect to the weights (device float array) for one batch
 * (learned guess; no counterpart in the paper). */
ad_status ad_guess_grad(ad_ctx* ctx, const ad_grid* grid, const float* weights, const float* ubar,
                        const float* utrue, int batch, float* grad, double* loss, void* stream);

/* Trains the weights in place with Adam (lr, beta1 0.9, beta2 0.999) for
 * `epochs` passes over `npairs` (u_bar, u_true) pairs ([npairs][P] device
 * arrays) in minibatches of `batch` drawn by a seeded shuffle; loss_hist
 * (host double[epochs], may be NULL) receives each epoch's mean loss.
 * Learned guess; no counterpart in the paper. */
ad_status ad_guess_train(ad_ctx* ctx, const ad_grid* grid, int npairs, const float* ubar, const float* utrue,
                         int epochs, int batch, double lr, uint64_t seed, float* weights, double* loss_hist,
                         void* stream);

/* Measures one forward 32 -> 32 layer of the learned guess's network
 * (ReLU(conv(H1, W2)) on the context's workspace for this grid and batch,
 * zero weights and activations) in the launch shape inference uses: warm-up,
 * then `reps` launches on `stream` between two CUDA events. Outputs (host,
 * may be NULL): ms per launch, tensor_cores = 1 when the layer ran on the
 * tcgen05 tensor-core kernel (x side a multiple of 128), 0 for the
 * warp-level mma kernel. Blocks the host until the timing completes. No
 * counterpart in the paper: it relates the convolution's time to the bf16
 * tensor-core roofline (55,296 flop per grid point per layer). */
ad_status ad_guess_time_conv(ad_ctx* ctx, const ad_grid* grid, int batch, int reps, void* stream, double* ms,
                             int* tensor_cores);

/* Tile autotuner. With `grid` non-NULL, tunes the plan for (grid, batch):
 * for every pass of one iteration of `method` it times each admissible tile
 * width (32-256 threads per block, <= 100 KB shared memory) with CUDA events
 * on the context's internal buffers and keeps the fastest; later solves on
 * that plan use the tuned tiles (cached graphs are rebuilt). Blocks the host
 * while timing. `enable_for_batched` != 0 makes ad_deconvolve_batched tune
 * every plan it creates (0 turns that off); `grid` may be NULL to set only
 * this flag. No counterpart in the paper. */
ad_status ad_autotune(ad_ctx* ctx, const ad_grid* grid, int batch, ad_method method, int enable_for_batched);

/* Measures one pass kernel of an iteration of `method` for this grid and
 * batch: the kernel is launched once to warm up, then `reps` times back to
 * back on `stream` between two CUDA events, in exactly the launch shape and
 * fused prologue/epilogue a solve uses, but on the context's internal
 * buffers (caller memory is never touched) and with every field forced
 * active and no scalar update. `index` selects the launch within the
 * iteration body (0 .. count-1, in launch order); index = -1 only reports
 * the count; index = -2 times the whole body (all its launches in order,
 * ms_per_launch is then per body, kind and op are -1). Outputs (host, may
 * be NULL): ms_per_launch, kind (0 forward x,
 * 1 inverse x, 2 filter, 3 forward y, 4 inverse y, 5 last-axis forward,
 * 6 last-axis inverse, 7 spectral-space pass, 8 preconditioner stencil), op (the fused
 * prologue/epilogue/dot code of that pass), count (launches per iteration).
 * Blocks the host until the timing completes. No counterpart in the paper:
 * it exists to relate measured kernel time to the HBM roofline. */
ad_status ad_time_pass(ad_ctx* ctx, const ad_grid* grid, int batch, ad_method method, int index, int reps,
                       void* stream, double* ms_per_launch, int* kind, int* op, int* count);

/* Size of the fixed device scratch array that ad_filter_static uses. */
#define AD_STATIC_SCRATCH_BYTES (32u << 20)

/* out = G in, like ad_filter, but allocating nothing: no context, no
 * cudaMalloc/cudaFree, no allocating library call. The paper has no
 * counterpart; this is for callers that cannot let a library allocate device
 * memory -- real-time or embedded codes that reserve all memory at start-up,
 * applications whose device memory belongs to another allocator, and code
 * that must not synchronize the device (allocation and freeing may).
 *   The scratch (twiddle tables and spectral buffers) lives in one
 * file-scope device array of AD_STATIC_SCRATCH_BYTES, held by every GPU that
 * loads the library until the process exits. A call needs, with cs = 8
 * (AD_F32) or 16 (AD_F64), L the last axis's length (Ny in 2D, Nz in 3D) and
 * each term rounded up to 256 bytes:
 *   cs*Nx + cs*Nx/2 + 2*cs*L [+ cs*Ny in 3D] + k * cs*batch*(Nx/2+1)*Ny*Nz,
 *   k = 1 (2D), 2 (3D)
 * bytes (twiddle tables and spectral buffers); larger requests return AD_ERR_ARG (e.g. 2D float32 up to one 2048^2
 * field, 3D float32 up to one 128^3 field). Grid rules, pointers and the
 * stream are as for ad_filter; `in` and `out` may be the same buffer.
 *   The device address of the array is looked up (cudaGetSymbolAddress) by
 * the first call on each device, with that device current; make that first
 * call before any stream capture. The cached address is the device
 * context's: after cudaDeviceReset on a device it is stale, and this entry
 * point must not be called on that device again. All calls on a device share the array and
 * leave their contents in it (nothing in it needs clearing: every call
 * rewrites what it reads); calls whose work overlaps on the GPU (other
 * streams or host threads) race on it and must be serialized.
 * Returns AD_OK, AD_ERR_ARG or AD_ERR_CUDA. */
ad_status ad_filter_static(const ad_grid* grid, const void* in, void* out, int batch, void* stream);

/* ---- Closure and statistics of deconvolved fields --------------------------
 * What the deconvolved field is for in the paper: the sub-filter stress of
 * the structural closure model (Section 3) and the energy spectra and
 * vorticity PDFs by which recovered fields are assessed (Sections 4.1, 4.2).
 * Velocities are stored component-major: velocity v, component c at field
 * index v*ncomp + c of a contiguous batch (components along x, y[, z]). */

/* Largest nbins of ad_spectrum and of ad_histogram. */
#define AD_MAX_SHELLS 8192
#define AD_MAX_HIST_BINS 16384

/* Sub-filter stress of the approximate-deconvolution closure, Eq. fge3 with
 * the unfiltered velocity replaced by its deconvolved estimate u*:
 *   tau_ij = u_bar_i u_bar_j - G(u*_i u*_j),   i <= j,
 * for nvel velocities of ncomp (1..3) components. With u* = u_bar this is the
 * Layton-Lewandowski model (Eq. tau2); with the Van Cittert estimate of N
 * passes it is the AD model of order N + 1 (Eq. tau3 and its second-order
 * form). One application of G over nvel * ncomp(ncomp+1)/2 fields; the
 * products are formed in the forward pass and the stress in the inverse one.
 *   ubar, ustar  device, [nvel][ncomp][P], inputs
 *   tau          device, [nvel][npairs][P] output, pairs ordered (0,0), (0,1),
 *                ..., (0,ncomp-1), (1,1), ..., (ncomp-1,ncomp-1); must not
 *                overlap the inputs
 * Enqueued on `stream` (asynchronous). */
ad_status ad_closure(ad_ctx* ctx, const ad_grid* grid, int nvel, int ncomp, const void* ubar, const void* ustar,
                     void* tau, void* stream);

/* Shell-summed energy spectrum of nfields fields taken in groups of ncomp
 * (the components of one velocity, or ncomp = 1 for scalar fields):
 *   E[g][k] = sum over the group's fields and over wavevectors k' with
 *             shell(|k'|^2) = k of |u_hat(k')|^2 / 2,   u_hat = FFT(u)/P,
 * for k = 0 .. nbins-1, where shell(m) is the nearest integer to sqrt(m),
 * halves rounded down (the smallest k >= 0 with k^2 + k >= m); wavevectors
 * of higher shells are not counted. sum_k E = mean(|u|^2)/2 (Parseval) when
 * every shell is counted. The paper shows such spectra (Sections 4.1, 4.2)
 * without stating a convention; this is the one used here.
 *   u   device, [nfields][P] input;  E host double[nfields/ncomp][nbins]
 * Accumulated in float64; the order of the per-shell additions is not fixed,
 * so repeated calls agree to rounding, not bit for bit. Blocks until E is
 * written. nbins <= AD_MAX_SHELLS. */
ad_status ad_spectrum(ad_ctx* ctx, const ad_grid* grid, int nfields, int ncomp, const void* u, int nbins,
                      double* E, void* stream);

/* Value histogram for a PDF (the vorticity PDFs of Sections 4.1, 4.2): with
 * scale = nbins/(hi - lo), value x falls in bin floor((x - lo) * scale),
 * computed in the data's precision with lo and scale rounded to it and each
 * operation rounded once.
 *   x       device, n values of dtype
 *   counts  host int64[nbins + 3]: the bins, then the number of values below
 *           (bin < 0), above (bin >= nbins) and NaN
 * The PDF is counts[b] / (n (hi - lo) / nbins). Exact integer counts.
 * Blocks until counts is written. nbins <= AD_MAX_HIST_BINS; lo < hi finite. */
ad_status ad_histogram(ad_ctx* ctx, ad_dtype dtype, int64_t n, const void* x, double lo, double hi, int nbins,
                       int64_t* counts, void* stream);

/* Vorticity (the field whose PDFs Sections 4.1 and 4.2 compare) by spectral
 * differentiation (d/dx_d multiplies the Fourier
 * coefficient by i k_d, zero at the Nyquist index), for nvel velocities:
 *   2D: u [nvel][2][Ny][Nx] -> omega [nvel][Ny][Nx], omega = dv/dx - du/dy
 *   3D: u [nvel][3][Nz][Ny][Nx] -> omega [nvel][3][...], omega = curl u
 * Device pointers; omega must not overlap u. Enqueued on `stream`. */
ad_status ad_curl(ad_ctx* ctx, const ad_grid* grid, int nvel, const void* u, void* omega, void* stream);

/* Time limit of the bounded device waits (the preconditioner's wait for its
 * staged rows, and the barrier waits of the learned guess's tensor-core
 * convolution; default 1e9 ns). A preconditioner block whose wait runs out
 * takes no part in the result, waits up to 1 s more for its own copies still
 * in flight, and its field ends with AD_ERR_TIMEOUT; a convolution CTA stops
 * issuing, drains (bounded) its loads and MMAs in flight and frees its tensor
 * memory, and the ad_guess_* call returns AD_ERR_TIMEOUT. The context stays
 * usable. ns = 0 makes
 * every such wait give up at once: that is how the timeout path is tested
 * without a fault. Cached solve graphs are dropped. No counterpart in the
 * paper. */
ad_status ad_set_wait_limit(ad_ctx* ctx, uint64_t ns);

/* Enables (1, default) or disables (0) capture of each solve into one CUDA
 * graph whose iteration loop is a device-side conditional while node. With 0
 * the host launches the iteration body in chunks and polls the device
 * between chunks (the same iterations of Algorithms 1-4 either way). Returns
 * AD_ERR_ARG for a NULL context. */
ad_status ad_set_graph_mode(ad_ctx* ctx, int enable);

/* How ad_deconvolve_batched runs a batch of several shapes. 0 (default): one
 * branch per shape group in the batch's graph, each with its own loop; the
 * branches run concurrently and each group stops when its fields converge.
 * 1: one launch per pass stage over the blocks of every shape group (a
 * device work list of (group, field, tile) blocks; groups whose pass has
 * another per-thread element count or block size get a launch of their
 * own), one loop for the whole batch; used for float32 Van Cittert, SD, CG
 * and BiCGSTAB in physical space, every other method or precision keeps the
 * branches. The results are bitwise the same either way (each group's passes
 * run in their own launch shape). Measured on the 48-field uneven batch the
 * branches are faster (the work list runs every stage until the slowest
 * field converges). Cached batched graphs are dropped. Returns AD_ERR_ARG for
 * a NULL context. No counterpart in the paper (Algorithms 1-4 solve one
 * field). */
ad_status ad_set_batched_launch(ad_ctx* ctx, int one_launch_per_stage);

/* Number of kernel launches the last ad_filter / ad_deconvolve call issued
 * (graph-internal launches counted per executed kernel node). Library
 * housekeeping, no counterpart in the paper. */
int64_t ad_last_launch_count(const ad_ctx* ctx);

/* Short English description of a status value (static storage). Library
 * housekeeping, no counterpart in the paper. */
const char* ad_status_str(ad_status s);

/* Detail of the last error seen by the context (static per-context storage).
 * Library housekeeping, no counterpart in the paper. */
const char* ad_last_error(const ad_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GAD_H */
