// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/ar.h"

namespace ar {

// ------------------------------------------------ programmatic dependent launch
// Kernels of the iteration are launched with programmatic stream serialization:
// a kernel may begin (prologue, constant-operand loads) while its predecessor in
// the stream drains.  pdl_wait() blocks the calling thread until the
// predecessor grid has completed and its memory operations are visible;
// pdl_trigger() lets the successor be scheduled.  A kernel triggers only after
// its own pdl_wait(), so every grid before the predecessor is complete when a
// kernel starts.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------- errors ---
// Records a human-readable detail for ar_last_error_detail() and returns s.
ar_status fail(ar_status s, const char* fmt, ...);
ar_status cuda_fail(cudaError_t e, const char* what);

#define AR_CUDA(call)                                                         \
    do {                                                                      \
        cudaError_t _e = (call);                                              \
        if (_e != cudaSuccess) return ::ar::cuda_fail(_e, #call);             \
    } while (0)

#define AR_TRY(call)                                                          \
    do {                                                                      \
        ar_status _s = (call);                                                \
        if (_s != AR_OK) return _s;                                           \
    } while (0)

// ------------------------------------------------------------- stencils ---
// Epilogue of the fused AR pad + convolution kernel.
enum ConvMode : int {
    CONV_STORE = 0,      // out = A x
    CONV_RESIDUAL = 1,   // out = g - A x            (aux = g)
    CONV_AXPY = 2,       // out += tau * A x         (out read-modify-write)
    CONV_SPLIT3 = 3      // out planes = bf16x3 split of A x (transform operand)
};

struct ConvArgs {
    const float* x;      // input image n1 x n2
    float* out;          // output image (CONV_STORE/RESIDUAL/AXPY)
    const float* aux;    // g for CONV_RESIDUAL
    uint16_t* planes;    // CONV_SPLIT3: 3 bf16 planes, plane stride plane_stride, row pitch ld
    size_t plane_stride;
    int ld;
    const float* psf;    // device PSF (2q1+1) x (2q2+1)
    int n1, n2, q1, q2;
    int flip;            // 1: use h_{-s} (reblur A')
    int mode;
    float tau;
    const float* f;      // CONV_AXPY: true image or null
    double* sumsq;       // CONV_AXPY with f: += sum (x_new - f)^2; CONV_RESIDUAL:
                         // += sum r^2 (float64, float32 per-thread partials)
    int bc;              // AR_BC_ANTIREFLECTIVE / AR_BC_REFLECTIVE / AR_BC_PERIODIC
    int fold;            // CONV_SPLIT3: write the even/odd fold along the columns,
                         // y+_t = y_t + y_{n2-1-t} at column t and y-_t at column
                         // Kh + t (Kh = ceil(n2/2) rounded up to 64); needs the TMA path
    int early_trigger;   // the successor cannot crowd the SMs (a contraction, which
                         // needs a whole SM): let it launch when the last tile
                         // starts, not after it (TMA path; the TMA stencils launch
                         // as programmatic dependents)
    int spread;          // the launch owns the GPU (the single-image loop): a grid
                         // that fits one wave takes at most two CTAs per SM
    const uint8_t* tcplan;  // non-null: this PSF's plan for the tensor-core stencil
                            // (conv_tc_plan), used where that path applies
                            // (conv_tc_applies); the float32 stencil elsewhere
};

// Bytes of a tensor-core stencil plan (device memory, 16-byte aligned).
constexpr size_t kConvTcPlanBytes = 16 + 17 * 2 * 2048;

// Writes the plan of the device PSF (2q1+1) x (2q2+1) for y = A x (flip 0) or
// y = A' x (flip 1) on `stream`; q1, q2 <= 8.
ar_status conv_tc_plan(const float* psf, int q1, int q2, int flip, uint8_t* plan,
                       cudaStream_t stream);

// True when the tensor-core stencil serves these arguments: q1, q2 <= 8, AR or
// Reflective BC, n2 % 4 == 0 and a 16-byte aligned input image.
bool conv_tc_applies(const ConvArgs& a);

// Launches the AR stencil on `stream` (validated arguments).
ar_status conv_launch(const ConvArgs& a, cudaStream_t stream);

// Device int set to 1 by a stencil kernel whose bounded TMA wait gave up
// (cleared by the caller that reads it).
int* conv_error_flag();

// Sets the polls of the stencils' halo-tile waits on the current device.
ar_status conv_set_wait_polls(unsigned polls);

// Both stencils of a restoration iteration for many images in one persistent
// launch (ar_conv.cu): blurs[j] (CONV_RESIDUAL, x_j -> r_j) then reblurs[j]
// (CONV_SPLIT3 unfolded, or CONV_AXPY; input r_j; sumsq, if set, is the base of
// one float64 per iteration).  geometry 0: 64-row tiles, 1: 54-row tiles;
// ctas_per_sm: persistent CTAs per SM (capped by occupancy); iters: iterations
// per run (each uses its own queue counters, zeroed by conv_group_reset).
struct ConvGroup;
ar_status conv_group_create(const ConvArgs* blurs, const ConvArgs* reblurs, int count, int geometry,
                            int ctas_per_sm, int iters, ConvGroup** out);
ar_status conv_group_reset(ConvGroup* g, cudaStream_t s);
ar_status conv_group_apply(ConvGroup* g, int iter, cudaStream_t s);
int conv_group_ctas_per_sm(const ConvGroup* g);
void conv_group_destroy(ConvGroup* g);

// cuTensorMapEncodeTiled from the driver (null if unavailable), as void*.
void* tensor_map_encoder();

// ------------------------------------------------------------ transform ---
// Even/odd folds of one axis of length m (the AR transform's reflection
// symmetry): h = ceil(m/2) sums, ha = floor(m/2) differences; spectral halves
// padded to Hs (a multiple of 128), folded spatial halves to Kh (of 64).
struct FoldDims {
    int m, h, ha, Hs, Kh;
};

__host__ __device__ inline FoldDims fold_dims(int m) {
    FoldDims f;
    f.m = m;
    f.h = (m + 1) / 2;
    f.ha = m / 2;
    f.Hs = (f.h + 127) / 128 * 128;
    f.Kh = (f.h + 63) / 64 * 64;
    return f;
}

// Folded spectral index kf -> kind (0 u+, 1 odd interior, 2 u-, 3 even interior,
// -1 padding) and the natural spectral index s: the first half holds u+ (the
// sum of the two boundary coefficients) and s = 1, 3, 5, ..; the second u- and
// s = 2, 4, ...
__device__ __forceinline__ int spec_of(int kf, const FoldDims& f, int& s) {
    const bool anti = kf >= f.Hs;
    const int u = anti ? kf - f.Hs : kf;
    if (u == 0) {
        s = 0;
        return anti ? 2 : 0;
    }
    s = anti ? 2 * u : 2 * u - 1;
    if (s > f.m - 2) return -1;
    return anti ? 3 : 1;
}

// The transform pair of a boundary condition for one image size, applied as
// dense contractions (four for AR and Reflective, seven for Periodic).
// Implemented in ar_transform.cu.
struct TransformPlan;

// precision: AR_PRECISION_FP32 (three bf16 planes, six products) or
// AR_PRECISION_BF16X2 (two planes, three products); bc: an ar_bc value.
// fold_input: the stencil producing the DIN_SPLIT input can write it folded
// along the columns (AR plans then take it so when n2 is a multiple of 4).
// pair_out: AR plans run their last contraction in parity-paired clusters of
// four never (0), when all clusters fit at once or waves are unavoidable (1),
// or always (2, grouped launches, whose items come in many waves anyway).
ar_status transform_plan_create(int n1, int n2, int bc, int precision, cudaStream_t stream,
                                TransformPlan** out, bool fold_input = false, int pair_out = 1);
void transform_plan_destroy(TransformPlan* p);
// Frees the plan's buffers in the order of stream s (after its pending work).
void transform_plan_release(TransformPlan* p, cudaStream_t s);

// Where the input of D comes from.
enum DInput : int {
    DIN_FP32 = 0,        // y is a float32 image (ar_symprec_solve)
    DIN_SPLIT = 1        // the operand planes were already written by the stencil
};

// Final epilogue of D.
enum DOutput : int {
    DOUT_STORE = 0,      // z = D y
    DOUT_AXPY = 1        // x += tau * D y
};

// Hands the plan the filter d (float32, n1 x n2) the next transform_apply
// calls use: AR plans keep it in their folded spectral order (call after
// every change of d); other plans read d32 as given to transform_apply.
ar_status transform_set_filter(TransformPlan* p, const float* d32, cudaStream_t stream);

// Pointer to the operand planes the stencil must fill for DIN_SPLIT; *folded
// (may be null) tells whether they take the column-folded form (ConvArgs::fold).
uint16_t* transform_input_planes(TransformPlan* p, size_t* plane_stride, int* ld,
                                 int* folded = nullptr);

// d32 is the filter in the transform domain; for Periodic it is the part of d
// even in each frequency and d32_odd minus the part odd in both (null for the
// other BCs).  With dout == DOUT_AXPY and f non-null, sum (x_new - f)^2 is
// added to *sumsq (float64) in the same kernel that updates x.
ar_status transform_apply(TransformPlan* p, const float* d32, const float* d32_odd,
                          const float* y, DInput din,
                          float* out, DOutput dout, float tau, cudaStream_t stream,
                          const float* f = nullptr, double* sumsq = nullptr);

// Number of kernels one transform_apply launches (for launch accounting).
int transform_launches(const TransformPlan* p, DInput din);

// The four contractions of x_j += tau D_j z_j for many AR plans in four grouped
// launches (one per contraction, every plan's tiles as work items, largest K
// first).  The plans must agree on the last contraction's pairing
// (transform_plan_create's pair_out) and read their input as written by their
// reblur (DIN_SPLIT); fs[j] (may be
// null) and sumsq[j] give the RRE accumulation, sumsq[j] + iter per iteration.
struct TransformGroup;
ar_status transform_group_create(TransformPlan* const* plans, int count, float* const* outs,
                                 const float* const* fs, double* const* sumsq, float tau,
                                 TransformGroup** out);
ar_status transform_group_apply(TransformGroup* g, int iter, cudaStream_t s);
bool transform_group_paired(const TransformGroup* g);
void transform_group_destroy(TransformGroup* g);

// Device int set to 1 by a contraction kernel whose bounded wait gave up.
int* transform_error_flag(TransformPlan* p);

// The spectral operand W = d o (T~ y) of the last transform_apply of an AR
// plan in the folded order of both axes: bf16 planes [nplanes][N1][ld],
// N1 = 2 Hs(n1) rows, N2 = 2 Hs(n2) columns, and the folded filter (N1 x N2).
ar_status transform_spectral_view(const TransformPlan* p, const uint16_t** planes,
                                  size_t* pstride, int* ld, int* nplanes, const float** dfold);

// ------------------------------------------------- FFT-style transform ---
// D y = T diag(d) T~ y with each 1D AR transform as boundary terms plus a DST-I
// from a Good-Thomas factored real DFT (ar_fst.cu).  AR BCs, n_j - 1 split into
// coprime factors <= 256.
struct FstPlan;
bool fst_supported(int n1, int n2);
ar_status fst_plan_create(int n1, int n2, cudaStream_t s, FstPlan** out);
void fst_plan_destroy(FstPlan* p);
// The plan's float32 input buffer (n1 x n2): the reblur writes z there.
float* fst_input(FstPlan* p);
// out = D y (axpy false) or out += tau D y with sum (out_new - f)^2 added to
// *sumsq; y null reads fst_input(p).  d32: the filter, natural order.
ar_status fst_apply(FstPlan* p, const float* d32, const float* y, float* out, bool axpy, float tau,
                    cudaStream_t s, const float* f = nullptr, double* sumsq = nullptr);

// AR_PRECISION_AUTO resolved for an image size and BC (measured once per
// device and size); other precisions are returned as given.
ar_status resolve_precision(int precision, int bc, int n1, int n2, cudaStream_t s, int* out);
ar_status check_precision(int precision, int bc, int n1, int n2);

// ---------------------------------------------------------------- setup ---
// FP64 eigenvalue setup on the GPU.  AR and Reflective: symmetrize (eq.
// simmetrizzata2d), symbol (eq. funzione_generatrice) on the grid of the BC
// (Theorem 2 / Section 2.1).  Periodic: |lambda| of the circulant of the PSF
// itself, then the even/odd split of d that transform_apply takes (d32,
// d32_odd).  Tikhonov filter d = 1/(lambda^2 + alpha) (eq. TikFilter).
// delta_dev (AR / Reflective, may be null): a float64 correction added to
// lambda^2 in the filter, d = 1/(lambda^2 + delta + alpha).
ar_status setup_eigen(const double* psf_dev64, int q1, int q2, int n1, int n2, double alpha,
                      int bc, double* lam64, double* d64, float* d32, float* d32_odd,
                      double* scratch_dev, cudaStream_t stream, const double* delta_dev = nullptr);
size_t setup_scratch_doubles(int q1, int q2, int n1, int n2, int bc);

// ------------------------------------------------------------- reductions ---
// acc[0] += sum (x - f)^2, both n floats, float64 accumulation.
ar_status reduce_diff_sq(const float* x, const float* f, size_t n, double* acc, cudaStream_t s);
// acc[0] += sum f^2.
ar_status reduce_sq(const float* f, size_t n, double* acc, cudaStream_t s);
// cnt[0] += number of non-finite entries of x.
ar_status count_nonfinite(const float* x, size_t n, unsigned long long* cnt, cudaStream_t s);

int sm_count();

// cudaMallocAsync of the restoration's scratch and preconditioner buffers; fails
// with cudaErrorMemoryAllocation without calling the allocator while failures
// injected by ar_inject_alloc_failures() remain.
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s);

// ------------------------------------------------------ shared host helpers
bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes);
ar_status check_image_sizes(int n1, int n2, int nmin);
ar_status check_support(int n1, int n2, int q1, int q2, int margin);
ar_status check_psf_host(const double* h, int q1, int q2);
void set_pool_threshold_once();
// Builds a preconditioner on `s` without synchronizing (keep64: also keep the
// float64 eigenvalues and filter).
// Frees a preconditioner whose buffers came from the stream-ordered pool, in
// the order of stream s (no device-wide synchronization).
void prec_release(ar_prec* P, cudaStream_t s);

// correction: 0 none, 1 exact spectral correction, 2 the model's (AR only).
// grouped: the plan serves grouped launches (unfolded input, unpaired G4).
ar_status prec_build(const double* psf_host, int q1, int q2, int n1, int n2, double alpha,
                     int bc, int precision, cudaStream_t s, bool keep64, ar_prec** out,
                     int correction = 0, const ar_corr* model = nullptr, bool grouped = false);

// ----------------------------------------------------- spectral correction
// delta of the PSF (device float64) on the AR grid of an n1 x n2 image into
// `delta`: exact when model is null, else the model's bilinear reading
// (15 x 15 PSF).  `scratch` holds corr_scratch_doubles(q1, q2, n1, n2) doubles.
ar_status corr_delta(const double* psf_dev64, int q1, int q2, int n1, int n2, const ar_corr* model,
                     const double* psf_host, double* delta, double* scratch, cudaStream_t s);
size_t corr_scratch_doubles(int q1, int q2, int n1, int n2);
bool corr_on_current_device(const ar_corr* model);

// Launch accounting: every kernel launch site calls count_launch(k).
void count_launch(unsigned k = 1);

// Profiling (ar_profile_begin/end): bracket `launches` kernel launches of one
// class with prof_begin/prof_end; scopes opened inside a recording scope are
// not recorded (dependent launches are timed together, overlap included).
int prof_begin(int kind, cudaStream_t s, unsigned launches);
void prof_end(int idx, cudaStream_t s);

struct ProfScope {
    int idx;
    cudaStream_t s;
    ProfScope(int kind, cudaStream_t st, unsigned launches = 1)
        : idx(prof_begin(kind, st, launches)), s(st) {}
    ~ProfScope() { prof_end(idx, s); }
};

}  // namespace ar

struct ar_prec {
    int n1, n2, q1, q2;
    double alpha;
    int precision;
    int bc;
    int device;
    double* lam64;
    double* d64;
    float* d32;
    float* d32_odd;      // Periodic only: minus the part of d odd in both frequencies
    ar::TransformPlan* plan;   // dense contractions (null with the FFT-style form)
    ar::FstPlan* fst;          // AR_PRECISION_FFT: the FFT-style transform
};
