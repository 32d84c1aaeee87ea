/*
 * ar.h - C ABI of the GB300 (sm_103a) Anti-Reflective deblurring library.
 *
 * The library implements the hot path of the preconditioned Landweber
 * restoration of Dell'Acqua, Serra-Capizzano and Tablino-Possio, "Optimal
 * preconditioning for image deblurring with Anti-Reflective boundary
 * conditions": the AR blurring matrix A_n (Section 2.2 boundary rules and
 * eq. modello_discreto), its reblurred counterpart A' (Section 4), and the
 * optimal preconditioner D = T_n diag(d) T~_n (Theorems 1, 2 and 4, eq.
 * TikFilter) inside the D-Landweber iteration (eq. DLandweberMeth).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Images are n1 x n2, row-major (row index i1, column index i2), float32,
 *    contiguous, in DEVICE memory owned by the caller.  n1, n2 >= 1 for the
 *    blur, >= 3 wherever the preconditioner is involved.
 *  - A PSF of support q = (q1, q2) is a (2q1+1) x (2q2+1) row-major array with
 *    psf[(i1+q1)*(2q2+1) + (i2+q2)] = h_{i1,i2} (eq. coefficienti_psf).
 *    The blur is a true convolution, g_i = sum_s h_s f_{i-s}.
 *    0 <= q_j <= n_j - 1 for the blur (the anti-reflection must stay inside
 *    the image); the AR preconditioner additionally needs q_j <= n_j - 3 (the
 *    support condition of Section 2.2).  q_j <= 15 runs on the fast
 *    register-blocked kernels, larger supports on a generic kernel.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on `stream` unless stated otherwise.
 *  - Every call returns an ar_status; AR_OK is 0.  Nothing throws across
 *    the ABI.  ar_status_string() names a status; ar_last_error_detail()
 *    gives a human-readable detail of the last failure on the calling thread.
 *  - No call keeps a pointer to caller memory after it returns (asynchronous
 *    calls read/write it in stream order).
 */
#ifndef AR_H
#define AR_H

#if defined(__GNUC__)
#define AR_API __attribute__((visibility("default")))
#else
#define AR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ar_status {
    AR_OK = 0,
    AR_ERR_INVALID_ARG = 1,        /* null pointer, bad size or support, alpha <= 0, ... */
    AR_ERR_ALIAS = 2,              /* an output overlaps an input it must not overlap */
    AR_ERR_PSF_NOT_NORMALIZED = 3, /* |sum(h) - 1| > 1e-6 where the method needs sum(h) = 1 */
    AR_ERR_ALLOC = 4,              /* device or host allocation failed */
    AR_ERR_CUDA = 5,               /* a CUDA runtime/driver call failed */
    AR_ERR_NONFINITE = 6,          /* the restoration produced NaN or Inf */
    AR_ERR_TIMEOUT = 7,            /* a bounded device-side wait gave up */
    AR_ERR_UNSUPPORTED = 8         /* valid request this build cannot serve (e.g. no sm_103a GPU) */
} ar_status;

/* Boundary conditions.  AR_BC_ANTIREFLECTIVE is the paper's method (Section
 * 2.2, the default of every call without a bc argument); AR_BC_REFLECTIVE
 * (Section 2.1: reflection about the boundary, DCT-III algebra) and
 * AR_BC_PERIODIC (circulant) are the comparison BCs of Section 4's tables.
 * Every call with a bc argument supports all three: the Reflective
 * preconditioner works in the DCT-III basis, the Periodic one in the real
 * separable Hartley basis (see ar_symprec_setup_bc). */
typedef enum ar_bc { AR_BC_ANTIREFLECTIVE = 0, AR_BC_REFLECTIVE = 1, AR_BC_PERIODIC = 2 } ar_bc;

/* Arithmetic of the AR transform pair (Theorem 1) inside the preconditioner.
 *  AR_PRECISION_FP32:   dense contractions on the tensor cores, operands
 *                       split into three bfloat16 planes, the six products
 *                       with i + j <= 2 accumulated in float32: float32-grade
 *                       (the default).
 *  AR_PRECISION_BF16X2: two planes, the three products with i + j <= 1:
 *                       about 2^-16 relative per contraction, roughly half
 *                       the tensor work and two thirds of the operand bytes.
 *  AR_PRECISION_FFT:    FFT-style, float32 on the CUDA cores: every 1D
 *                       transform is its boundary terms plus a DST-I taken
 *                       from one real DFT of length n_j - 1, split by Good
 *                       and Thomas into two small dense DFTs of coprime
 *                       lengths (2047 = 23 x 89 at n = 2048).  AR BCs only,
 *                       and both n_j - 1 must split into coprime factors of
 *                       at most 256 (AR_ERR_UNSUPPORTED otherwise).
 *  AR_PRECISION_AUTO:   AR_PRECISION_FFT or AR_PRECISION_FP32, whichever the
 *                       library measures faster for the size (one timing of
 *                       each the first time a size is seen on a device, kept
 *                       for the process); AR_PRECISION_FP32 where the FFT-style
 *                       form does not apply. */
typedef enum ar_precision { AR_PRECISION_FP32 = 0, AR_PRECISION_BF16X2 = 1,
                            AR_PRECISION_FFT = 2, AR_PRECISION_AUTO = 3 } ar_precision;

/* Arithmetic of the blur and reblur stencils (the convolution of eq.
 * modello_discreto under the extension rules of Section 2.2 / 2.1).  OR
 * AR_STENCIL_F16X2 into the precision argument of ar_restore_ex,
 * ar_restore_bc and ar_restore_residuals, or pass it to ar_blur_apply_ex /
 * ar_reblur_apply_ex.
 *  AR_STENCIL_FP32:  float32 FMAs on the CUDA cores (the default).
 *  AR_STENCIL_F16X2: banded-Toeplitz products on the tensor cores.  Each
 *                    128 x 64 output tile scales its input box by a power of two
 *                    (largest magnitude to [2^14, 2^15)) and splits it into two
 *                    fp16 parts, as it does the PSF; three of the four products
 *                    accumulate in float32 (about 2^-21 relative per term, the
 *                    float32 stencil's order).  Serves q1, q2 <= 8 under AR and
 *                    Reflective BCs with n2 % 4 == 0 and a 16-byte aligned
 *                    input; other arguments take AR_STENCIL_FP32.
 *  AR_STENCIL_AUTO:  whichever of the two the library measures faster for the
 *                    shape (one timing of each, y = A x on a zero image of the
 *                    same size and PSF support, the first time a shape and
 *                    boundary condition are seen on a device; kept for the
 *                    process); AR_STENCIL_FP32 where the tensor-core path does
 *                    not apply.  The timing allocates two images and a plan
 *                    (stream-ordered) and synchronizes the stream. */
#define AR_STENCIL_FP32 0
#define AR_STENCIL_F16X2 16
#define AR_STENCIL_AUTO 32

/* Opaque preconditioner: the symmetrized-PSF eigenvalues and Tikhonov filter
 * for one (PSF, n1, n2, alpha), plus the AR transform operands and scratch
 * used by ar_symprec_solve.  Owned by the library; free with
 * ar_symprec_destroy. */
typedef struct ar_prec ar_prec;

/*
 * y = A_n x : anti-reflective blur (Section 2.2 extension rules applied
 * separably, which yields the double anti-reflection at the corners, then the
 * convolution of eq. modello_discreto).
 *   x, y    device float32, n1*n2 each; y must not overlap x (AR_ERR_ALIAS).
 *   psf     device float32, (2q1+1)*(2q2+1).  Not required to sum to one.
 * Errors: AR_ERR_INVALID_ARG (null pointer, n_j < 1, q_j < 0 or q_j > n_j - 1),
 *         AR_ERR_ALIAS, AR_ERR_CUDA (launch failure).
 */
AR_API ar_status ar_blur_apply(const float* x, float* y, int n1, int n2,
                        const float* psf, int q1, int q2, void* stream);

/*
 * y = A' x : the reblurred matrix of Section 4, i.e. the AR blur with the PSF
 * rotated by 180 degrees (h'_s = h_{-s}).  A' differs from A^T under AR BCs.
 * Arguments and errors as ar_blur_apply.
 */
AR_API ar_status ar_reblur_apply(const float* x, float* y, int n1, int n2,
                          const float* psf, int q1, int q2, void* stream);

/*
 * ar_blur_apply / ar_reblur_apply under the boundary condition bc (ar_bc).
 * Reflective extends by reflection about the boundary (Section 2.1:
 * x_{-1-i} = x_i, x_{n+i} = x_{n-1-i}, 0-based), Periodic by wrapping; the
 * reblur is the same blur with the PSF rotated by 180 degrees (for these two
 * BCs it equals the transpose of the blur matrix).  bc = AR_BC_ANTIREFLECTIVE
 * is ar_blur_apply / ar_reblur_apply.  Arguments and errors as ar_blur_apply,
 * plus AR_ERR_INVALID_ARG for an unknown bc.
 */
AR_API ar_status ar_blur_apply_bc(const float* x, float* y, int n1, int n2,
                                  const float* psf, int q1, int q2, int bc, void* stream);
AR_API ar_status ar_reblur_apply_bc(const float* x, float* y, int n1, int n2,
                                    const float* psf, int q1, int q2, int bc, void* stream);

/*
 * ar_blur_apply_bc / ar_reblur_apply_bc with the stencil arithmetic `stencil`
 * (AR_STENCIL_FP32, AR_STENCIL_F16X2 or AR_STENCIL_AUTO).  With AR_STENCIL_F16X2 the call
 * allocates (stream-ordered) and frees a plan of about 70 KB for the PSF.
 * Arguments and errors as ar_blur_apply_bc, plus AR_ERR_INVALID_ARG for an
 * unknown stencil and AR_ERR_ALLOC when the plan cannot be allocated.
 */
AR_API ar_status ar_blur_apply_ex(const float* x, float* y, int n1, int n2, const float* psf,
                                  int q1, int q2, int bc, int stencil, void* stream);
AR_API ar_status ar_reblur_apply_ex(const float* x, float* y, int n1, int n2, const float* psf,
                                    int q1, int q2, int bc, int stencil, void* stream);

/*
 * Build the optimal AR preconditioner (Theorem 4) for a PSF and image size:
 *   S0  s = symmetrized PSF, eq. simmetrizzata2d, in float64 on the GPU;
 *   S1  lambda[i1,i2] = f_s(x1_{i1}, x2_{i2}), the symbol of eq.
 *       funzione_generatrice on the AR grid of Theorem 2 (x = 0 for the first
 *       and last index, k*pi/(n-1) for k = 1..n-2), float64 on the GPU;
 *   S2  d = 1/(lambda^2 + alpha), eq. TikFilter, float64 on the GPU, kept in
 *       float64 and rounded once to float32 for the iteration;
 * and the AR transform operands of Theorem 1 (T_m, T~_m with the
 * normalisation alpha_m dropped, which cancels in T diag(d) T~).
 *   psf_host host float64 (2q1+1)*(2q2+1); must sum to 1 within 1e-6.
 *   alpha    Tikhonov parameter, > 0.
 *   out      receives the new object (left untouched on error).
 * Synchronizes `stream` before returning.
 * Errors: AR_ERR_INVALID_ARG (null, n_j < 3, q_j > n_j - 3, alpha <= 0 or not
 *         finite), AR_ERR_PSF_NOT_NORMALIZED, AR_ERR_ALLOC, AR_ERR_CUDA.
 */
AR_API ar_status ar_symprec_setup(const double* psf_host, int q1, int q2, int n1, int n2,
                           double alpha, void* stream, ar_prec** out);

/* ar_symprec_setup with an explicit ar_precision for the transform
 * contractions (ar_symprec_setup uses AR_PRECISION_FP32).  An unknown
 * precision returns AR_ERR_INVALID_ARG. */
AR_API ar_status ar_symprec_setup_ex(const double* psf_host, int q1, int q2, int n1, int n2,
                                     double alpha, int precision, void* stream, ar_prec** out);

/*
 * ar_symprec_setup_ex for the boundary condition bc (ar_bc), the optimal
 * preconditioner of each BC's algebra with the Tikhonov filter d of S2:
 *   AR_BC_ANTIREFLECTIVE  as ar_symprec_setup_ex;
 *   AR_BC_REFLECTIVE      D = R1 diag(d) R1^T (.) R2 diag(d) R2^T applied as
 *       R1 (d o (R1^T y R2)) R2^T, R the DCT-III matrix of eq. Rn, lambda the
 *       symbol of the symmetrized PSF at x_k = k pi / n (Section 2.1);
 *   AR_BC_PERIODIC        D = F* diag(d) F, the circulant solve, lambda =
 *       |sum_s h_s exp(-i s . w)| at w = 2 pi k / n (the PSF itself, not its
 *       symmetrization), applied in the real separable Hartley basis.
 * ar_symprec_eigenvalues returns these lambda and d (for Periodic in FFT
 * order).  Sizes: n_j >= 3; q_j <= n_j - 3 for AR, q_j <= n_j - 1 otherwise.
 * Errors as ar_symprec_setup_ex, plus AR_ERR_INVALID_ARG for an unknown bc.
 */
AR_API ar_status ar_symprec_setup_bc(const double* psf_host, int q1, int q2, int n1, int n2,
                                     double alpha, int bc, int precision, void* stream,
                                     ar_prec** out);

/*
 * z = D y = T_n diag(d) T~_n y (Theorem 1 with the filtered eigenvalues).
 *   y, z device float32, n1*n2 (the sizes given at setup).  z may equal y
 *   (in-place) but must not partially overlap it.
 * Uses scratch owned by P: concurrent solves with the same P on different
 * streams race; use one preconditioner per stream.
 * Errors: AR_ERR_INVALID_ARG, AR_ERR_ALIAS, AR_ERR_CUDA.
 */
AR_API ar_status ar_symprec_solve(const ar_prec* P, const float* y, float* z, void* stream);

/*
 * Copy the float64 eigenvalues lambda and filter d of P to host arrays of
 * n1*n2 doubles each (either may be NULL).  Synchronous.
 */
AR_API ar_status ar_symprec_eigenvalues(const ar_prec* P, double* lambda_host, double* d_host);

/* Sizes a preconditioner was built for (either pointer may be NULL). */
AR_API ar_status ar_symprec_shape(const ar_prec* P, int* n1, int* n2);

/* The transform arithmetic P runs with (an ar_precision other than
 * AR_PRECISION_AUTO: the choice AR_PRECISION_AUTO made). */
AR_API ar_status ar_symprec_precision(const ar_prec* P, int* precision);

/* Free a preconditioner (NULL is a no-op).  Waits for its pending work. */
AR_API void ar_symprec_destroy(ar_prec* P);

/*
 * (D-)Landweber restoration with reblurring, eqs. LandweberMeth and
 * DLandweberMeth with A' in place of A^H (Section 4):
 *     x_{k+1} = x_k + tau * D * A'(g - A x_k),  k = 0..iters-1,
 * D = I when precondition == 0, else the preconditioner of ar_symprec_setup
 * built inside the call from psf_host and alpha.
 *   g          device float32 n1*n2, the observed image.
 *   psf_host   host float64 PSF; must sum to 1 within 1e-6.
 *   alpha      Tikhonov parameter (> 0; ignored when precondition == 0).
 *   tau        step (> 0); the paper uses 1.
 *   iters      >= 0 iterations.
 *   x0         device float32 start image or NULL for x_0 = 0.  May equal x_out.
 *   f_true     device float32 true image or NULL.  When given, the relative
 *              restoration error ||x_{k+1} - f||_F / ||f||_F of every iterate
 *              is accumulated in float64 on the GPU.
 *   x_out      device float32 n1*n2, the final iterate; must not overlap g or f_true.
 *   rre_trace  host double[iters] or NULL (needs f_true): RRE of x_1..x_iters.
 *   best_iter  host int or NULL (needs f_true): first k in 1..iters with the
 *              minimum RRE (the tables' IT); 0 when iters == 0.
 * Synchronizes `stream` before returning.  Scratch is taken from the stream's
 * memory pool (cudaMallocAsync) and returned before the call ends.
 * Errors: AR_ERR_INVALID_ARG, AR_ERR_ALIAS, AR_ERR_PSF_NOT_NORMALIZED,
 *         AR_ERR_ALLOC, AR_ERR_CUDA, AR_ERR_NONFINITE (x_out holds NaN/Inf;
 *         the iterate is still written).
 */
AR_API ar_status ar_restore(const float* g, const double* psf_host,
                     int n1, int n2, int q1, int q2, double alpha, double tau,
                     int iters, int precondition,
                     const float* x0, const float* f_true, float* x_out,
                     double* rre_trace, int* best_iter, void* stream);

/*
 * Plain Landweber restoration (D = I) that allocates no memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot let a
 * library allocate device memory, e.g. a framework that has reserved the
 * whole GPU for its own pool, or a fixed-budget service that must never call
 * into the CUDA allocator while it runs.  It computes exactly what
 * ar_restore(..., precondition = 0, ...) computes, with the same kernels in
 * the same order, and takes the same arguments except alpha and precondition.
 *
 * Its scratch (the residual image, the float32 PSF copy and the float64 RRE
 * accumulators) lives in one file-scope static device array of about 4.1 MiB
 * that every GPU loading this library keeps until the process exits; the
 * stencils' bounded-wait flag is a static device int as well.  No
 * cudaMalloc, cudaFree or other allocating routine is called.  Limits:
 * n1*n2 <= AR_STATIC_MAX_PIXELS, (2q1+1)(2q2+1) <= AR_STATIC_MAX_PSF,
 * iters <= AR_STATIC_MAX_ITERS; larger requests return AR_ERR_INVALID_ARG
 * with a detail naming the limit.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current:
 * make that first call before any stream capture.  All calls on a device
 * share the array and the call clears what must start at zero; calls whose
 * GPU work overlaps (different streams or host threads) race.
 * Synchronizes `stream` before returning.
 * Errors: as ar_restore, plus AR_ERR_TIMEOUT when a stencil's bounded wait
 * for its halo tile gave up (x_out is then incomplete).
 */
#define AR_STATIC_MAX_PIXELS (1u << 20)
#define AR_STATIC_MAX_PSF 4096u
#define AR_STATIC_MAX_ITERS 4096u
AR_API ar_status ar_restore_plain_static(const float* g, const double* psf_host, int n1, int n2,
                                         int q1, int q2, double tau, int iters,
                                         const float* x0, const float* f_true, float* x_out,
                                         double* rre_trace, int* best_iter, void* stream);

/* ar_restore with an explicit ar_precision for the preconditioner's
 * contractions (ignored when precondition == 0), optionally OR-ed with
 * AR_STENCIL_F16X2 or AR_STENCIL_AUTO for the blur and reblur stencils
 * (honoured with and without the preconditioner; both together are
 * AR_ERR_INVALID_ARG).  ar_restore is
 * ar_restore_ex(..., AR_PRECISION_FP32, ...). */
AR_API ar_status ar_restore_ex(const float* g, const double* psf_host,
                               int n1, int n2, int q1, int q2, double alpha, double tau,
                               int iters, int precondition, int precision,
                               const float* x0, const float* f_true, float* x_out,
                               double* rre_trace, int* best_iter, void* stream);

/* ar_restore_ex under the boundary condition bc (ar_bc): the blur, the
 * reblur and, with precondition != 0, the preconditioner of
 * ar_symprec_setup_bc all use bc (the Landweber / D-Landweber comparison of
 * Section 4's tables).  ar_restore_ex is ar_restore_bc(..., AR_BC_ANTIREFLECTIVE,
 * ...).  Sizes as ar_symprec_setup_bc when preconditioned, else as
 * ar_blur_apply; other arguments and errors as ar_restore. */
AR_API ar_status ar_restore_bc(const float* g, const double* psf_host,
                               int n1, int n2, int q1, int q2, double alpha, double tau,
                               int iters, int bc, int precondition, int precision,
                               const float* x0, const float* f_true, float* x_out,
                               double* rre_trace, int* best_iter, void* stream);

/*
 * ar_restore_bc that also returns the residual norms of the iterates:
 * res_trace[k] = ||g - A x_k||_F for k = 0 .. iters (iters + 1 entries, x_0 the
 * start), A the blurring matrix of bc (the residual step of eq. DLandweberMeth).
 * The squares are summed in the blur's residual epilogue, float32 partials of a
 * thread's rows reduced in float64 (one atomic per CTA), and one more blur of the
 * final iterate gives k = iters.
 *   res_trace  host float64, iters + 1 entries, required (AR_ERR_INVALID_ARG if null).
 * Other arguments, ownership and errors as ar_restore_bc.
 */
AR_API ar_status ar_restore_residuals(const float* g, const double* psf_host,
                                      int n1, int n2, int q1, int q2, double alpha, double tau,
                                      int iters, int bc, int precondition, int precision,
                                      const float* x0, const float* f_true, float* x_out,
                                      double* rre_trace, int* best_iter, double* res_trace,
                                      void* stream);

/*
 * Batched restoration of many independent images (each with its own size,
 * PSF and alpha; AR BCs).  ar_batch_create builds every image's
 * preconditioner (as ar_symprec_setup) and scratch, then captures the whole
 * restoration of every image -- x_0 = 0, `iters` iterations of eq.
 * DLandweberMeth with the reblurred A' (plain Landweber when precondition ==
 * 0), the RRE of every iterate when f_true is given -- into one CUDA graph in
 * which every iteration of the whole batch is five launches: one persistent
 * stencil kernel (the blur and the reblur of every image, single tiles handed
 * out by a device-side queue, largest images first, each reblur tile waiting
 * with a bounded wait for its image's blur tiles) and four grouped
 * contractions (every image's tiles of one product of the AR transform pair).
 * `tuning` 0 lets an autotuner time the stencil launch's tile geometry (64- or
 * 54-row tiles) and persistent CTAs per SM (1..3) on the batch itself and keep
 * the fastest (ar_batch_tuning reports the candidates); 1..8 fixes the CTAs
 * per SM with 64-row tiles.  Needs q_j <= 15, n2 % 4 == 0 and 16-byte aligned
 * x_out (AR_ERR_UNSUPPORTED otherwise).  The images' device pointers are bound
 * at creation and must stay valid for the life of the plan.  Creation
 * synchronizes `stream`.  ar_batch_run launches the graph on `stream`
 * (asynchronous: every x_out is overwritten); ar_batch_results waits for the
 * last run and copies the RRE traces (count x iters doubles, may be NULL), the
 * best iterations (count ints, may be NULL) and the number of kernels one run
 * launches.  The stencils of a run equal those of ar_restore_ex bit for bit;
 * the contractions may pair their tiles differently from the single-image
 * loop (the batch always runs the last product in parity-paired clusters), so
 * the iterates agree with ar_restore_ex within the restoration's float32
 * tolerance.
 * Errors: AR_ERR_INVALID_ARG (item index in the detail), AR_ERR_ALIAS (an
 * output overlapping any input or output of the batch),
 * AR_ERR_PSF_NOT_NORMALIZED, AR_ERR_UNSUPPORTED, AR_ERR_ALLOC, AR_ERR_CUDA;
 * ar_batch_results: AR_ERR_NONFINITE, AR_ERR_TIMEOUT.
 */
typedef struct ar_batch_item {
    const float* g;            /* device n1*n2 observed image */
    const double* psf_host;    /* host (2q1+1)*(2q2+1) PSF summing to 1 */
    int n1, n2, q1, q2;
    double alpha;              /* Tikhonov parameter (> 0 when preconditioned) */
    const float* f_true;       /* device n1*n2 true image or NULL */
    float* x_out;              /* device n1*n2 result */
} ar_batch_item;
typedef struct ar_batch ar_batch;
AR_API ar_status ar_batch_create(const ar_batch_item* items, int count, double tau, int iters,
                                 int precondition, int precision, int tuning, void* stream,
                                 ar_batch** out);
AR_API ar_status ar_batch_run(ar_batch* B, void* stream);
AR_API ar_status ar_batch_results(ar_batch* B, double* rre_traces, int* best_iters,
                                  unsigned long long* kernels_per_run);
AR_API void ar_batch_destroy(ar_batch* B);
/* The stencil configuration the batch runs with (geometry 0: 64-row tiles, 1:
 * 54-row tiles; persistent CTAs per SM), the transform's form (bit 0: the
 * reblur writes the first product's input folded along the columns; bit 1:
 * the last product runs in parity-paired clusters) and, when autotuned, every
 * timed candidate (up to max_candidates of them: geometry, CTAs per SM, device
 * milliseconds of three batch iterations).  Any output may be NULL. */
AR_API ar_status ar_batch_tuning(const ar_batch* B, int* geometry, int* ctas_per_sm,
                                 int* transform, int* candidates, int* cand_geometry,
                                 int* cand_ctas, double* cand_ms, int max_candidates);

/*
 * Spectral correction of the symmetrized preconditioner (learned form).
 *
 * With s the symmetrized PSF (eq. simmetrizzata2d) and a = h - s, the
 * response of A'A at an AR frequency x of a large image is, averaged over the
 * sign flips of x, lambda_s(x)^2 + delta(x) with
 *     delta(x1, x2) = (|a^(x1, x2)|^2 + |a^(-x1, x2)|^2) / 2,
 *     a^(w) = sum_s a_s exp(-i s.w);
 * the corrected filter is d = 1/(lambda_s^2 + delta + alpha) (eq. TikFilter
 * with the refined eigenvalue).  The paper has no such correction; it is the
 * per-frequency refinement of the symmetrized eigenvalues that a small model
 * learns from the PSF's antisymmetric part: an MLP (ReLU, widths 225 -> 256
 * -> 256 -> 1089) mapping 16 (h - s) of a 15 x 15 PSF (row-major) to delta on
 * the 33 x 33 grid x_j = j pi / 32 of [0, pi]^2 (row-major), read on the AR
 * grid by bilinear interpolation.  A refined eigenvalue of A'A is a response
 * energy: every corrected filter is d = 1/(max(lambda_s^2 + delta, 0) + alpha),
 * so a table entry below -lambda_s^2 counts as -lambda_s^2.
 * Parameters are float32, row-major (inputs x outputs), in the order
 * W1 (225 x 256), b1, W2 (256 x 256), b2, W3 (256 x 1089), b3.
 *
 * Two kinds of training target exist: the closed form above
 * (ar_corr_targets, ar_corr_train), and tables read off restorations the
 * symmetrized method itself produces (ar_corr_restoration_targets,
 * ar_corr_train_tables).
 */
#define AR_CORR_Q 7
#define AR_CORR_IN 225
#define AR_CORR_HIDDEN 256
#define AR_CORR_GRID 33
#define AR_CORR_OUT 1089

typedef struct ar_corr ar_corr;

/* Number of float32 parameters of the model (403521). */
AR_API size_t ar_corr_param_count(void);

/* Create a model on the current device from ar_corr_param_count() host
 * floats (copied).  Errors: AR_ERR_INVALID_ARG (null, non-finite), AR_ERR_ALLOC. */
AR_API ar_status ar_corr_create(const float* params_host, ar_corr** out);

/* Copy the model's parameters to the host (waits for pending training). */
AR_API ar_status ar_corr_params(const ar_corr* M, float* params_host);

/* Free a model (NULL is a no-op). */
AR_API void ar_corr_destroy(ar_corr* M);

/* The training targets: delta on the 33 x 33 grid, float64, computed exactly
 * on the GPU, for `count` 15 x 15 PSFs (host float64, 225 each) into
 * delta_host (count x 1089).  Synchronous. */
AR_API ar_status ar_corr_targets(const double* psfs_host, int count, double* delta_host);

/* Train on `count` 15 x 15 PSFs (host float64): inputs 16 (h - s) and targets
 * delta computed on the GPU, then `epochs` passes over the PSFs in order, in
 * batches of `batch` (the last may be smaller), each one Adam step (beta1
 * 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the mean squared error
 * over the batch and the 1089 outputs.  loss_trace_host (may be NULL)
 * receives the mean batch loss of each epoch.  Synchronizes `stream`. */
AR_API ar_status ar_corr_train(ar_corr* M, const double* psfs_host, int count, int epochs,
                               int batch, double lr, float* loss_trace_host, void* stream);

/* Train as ar_corr_train on given target tables: tables_host holds count x
 * 1089 float64 values (row-major 33 x 33 per PSF, e.g. from
 * ar_corr_restoration_targets), used as float32 targets.  Errors as
 * ar_corr_train, plus AR_ERR_INVALID_ARG for a null or non-finite table. */
AR_API ar_status ar_corr_train_tables(ar_corr* M, const double* psfs_host,
                                      const double* tables_host, int count, int epochs,
                                      int batch, double lr, float* loss_trace_host, void* stream);

/*
 * Training targets from restorations the symmetrized method produces (Section
 * 4's D-Landweber, eq. DLandweberMeth with the reblurred A', x_0 = 0).  For
 * each of `count` 15 x 15 PSFs h (host float64, 225 each, unit sum):
 *   g = A f + nu ||A f||_F e / ||e||_F  (A the AR blur of h; f and e device
 *       float32 n1 x n2, the scene and a noise field, read only);
 *   `iters` iterations with the symmetrized preconditioner of parameter alpha
 *   and step tau, keeping each iteration's spectral operand W_k = d o (T~ z_k),
 *   z_k = A'(g - A x_k) (Theorem 1's basis);
 *   per interior AR frequency, the least-squares effective eigenvalue of A'A
 *   over consecutive iterates, mu = sum_k W_k (W_k - W_{k+1}) / (tau d sum_k W_k^2),
 *   which obeys z^_{k+1} = (1 - tau mu d) z^_k when T~ A'A T is diagonal there;
 *   the target delta = (mu - lambda_s^2) w / (w + 5 w_mean), w = sum_k W_k^2
 *   and w_mean its mean over the interior frequencies (frequencies where the
 *   image has no content, and the fit only rounding, stay near 0), pooled
 *   onto the 33 x 33 grid (each
 *   frequency adds to the four nodes around it with weight w times the node's
 *   bilinear weight; a node is the weighted mean, 0 if no weight falls).
 * tables_host receives count x 1089 float64.  The paper has no such
 * procedure: it generates the learned correction's training data from the
 * method's own iterations.  Requires n_j >= 17 (the support condition of the
 * preconditioner), iters >= 2, nu >= 0, alpha > 0, tau > 0.  Allocates stream-
 * ordered scratch; synchronizes `stream`.  Errors: AR_ERR_INVALID_ARG,
 * AR_ERR_PSF_NOT_NORMALIZED, AR_ERR_ALIAS (f partially overlaps e),
 * AR_ERR_ALLOC, AR_ERR_CUDA, AR_ERR_TIMEOUT, AR_ERR_NONFINITE (a table entry;
 * e.g. a diverging restoration).
 */
AR_API ar_status ar_corr_restoration_targets(const float* f, const float* e, int n1, int n2,
                                             const double* psfs_host, int count, double nu,
                                             double alpha, double tau, int iters,
                                             double* tables_host, void* stream);

/* The model's 33 x 33 delta table for one 15 x 15 PSF (host float64) into
 * table_host (1089 floats).  Synchronous. */
AR_API ar_status ar_corr_predict(const ar_corr* M, const double* psf_host, float* table_host);

/* ar_symprec_setup_ex (AR BCs) with the corrected filter
 * d = 1/(max(lambda_s^2 + delta, 0) + alpha): delta exact on the AR grid (float64)
 * when M is NULL, else read from M's prediction for the PSF (which must then
 * be 15 x 15).  Errors as ar_symprec_setup_ex. */
AR_API ar_status ar_symprec_setup_corrected(const double* psf_host, int q1, int q2, int n1, int n2,
                                            double alpha, const ar_corr* M, int precision,
                                            void* stream, ar_prec** out);

/* D-Landweber (eq. DLandweberMeth with the reblurred A' of Section 4) with a
 * preconditioner built beforehand (ar_symprec_setup*, any BC, symmetrized or
 * corrected): the blur and reblur take psf_host, which must have P's support
 * and sum to 1; g, x0, f_true, x_out are n1 x n2 as P.  Other arguments,
 * outputs and errors as ar_restore.  Calls that share P must not overlap in
 * time (P's transform buffers are reused). */
AR_API ar_status ar_restore_prec(const ar_prec* P, const float* g, const double* psf_host,
                                 double tau, int iters, const float* x0, const float* f_true,
                                 float* x_out, double* rre_trace, int* best_iter, void* stream);

/* Static name of a status code ("AR_OK", ...; "AR_UNKNOWN" otherwise). */
AR_API const char* ar_status_string(ar_status s);

/* Detail of the last failure on the calling thread ("" if none).  Valid
 * until the next failing call on the same thread. */
AR_API const char* ar_last_error_detail(void);

/*
 * Per-kernel-class device timing for benchmarks.  Between ar_profile_begin()
 * and ar_profile_end(), every kernel the library launches is bracketed by a
 * CUDA event pair on its launch stream; ar_profile_end() synchronizes those
 * events and returns, per class, the summed milliseconds and the number of
 * launches (arrays of nkinds entries, classes beyond nkinds are dropped).
 * Recording events between kernels serializes them: a profiled run measures
 * each kernel alone, without the overlap of dependent launches.
 */
enum { AR_PROF_STENCIL = 0, AR_PROF_CONTRACTION = 1, AR_PROF_SETUP = 2, AR_PROF_OTHER = 3,
       AR_PROF_KINDS = 4 };
AR_API ar_status ar_profile_begin(void);
AR_API ar_status ar_profile_end(double* ms, unsigned long long* launches, int nkinds);

/* Number of kernels this library has launched in this process (all devices,
 * all threads), for launch accounting by benchmarks. */
AR_API unsigned long long ar_kernel_launches(void);

/*
 * Failure-detection controls (no counterpart in the paper; they exist so that
 * the library's error paths can be tested without faulting a GPU).
 *
 * ar_set_stencil_wait_polls: the number of mbarrier polls a stencil kernel
 * spends waiting for a halo tile before it gives up, on the current device.
 * A kernel that gives up waits (with the default bound) for its copies still
 * in flight, records the failure in a device flag and returns; ar_restore*,
 * ar_restore_prec and ar_restore_plain_static then return AR_ERR_TIMEOUT.
 * polls = 0 makes every wait give up at once; AR_DEFAULT_WAIT_POLLS restores
 * the default.  Synchronous (a copy to a device variable); errors: AR_ERR_CUDA.
 *
 * ar_inject_alloc_failures: of the next device allocations of the
 * restoration scratch and of the preconditioner buffers (ar_restore*,
 * ar_restore_prec, ar_symprec_setup*), the first `skip` succeed and the
 * following `count` fail as if the allocator had returned
 * cudaErrorMemoryAllocation, without calling it; the failing call returns
 * AR_ERR_ALLOC and frees what it had allocated.  count <= 0 clears the
 * injection.  Process-wide, all threads.
 */
#define AR_DEFAULT_WAIT_POLLS (1u << 24)
AR_API ar_status ar_set_stencil_wait_polls(unsigned polls);
AR_API void ar_inject_alloc_failures(int skip, int count);

/* Library version string. */
AR_API const char* ar_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AR_H */
