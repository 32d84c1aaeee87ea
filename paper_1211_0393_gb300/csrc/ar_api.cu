// C ABI of the library: argument validation, the preconditioner object and
// the (D-)Landweber restoration loop (eqs. LandweberMeth / DLandweberMeth with
// the reblurred A' of Section 4).  All arithmetic runs in the kernels of the
// other translation units; this file only validates, allocates and launches.

#include "ar_internal.cuh"

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

namespace ar {

static thread_local char g_detail[512] = "";

ar_status fail(ar_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
    va_end(ap);
    return s;
}

ar_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? AR_ERR_ALLOC : AR_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

static std::atomic<unsigned long long> g_launches{0};
// Injected allocation failures: `skip` more allocations succeed, then `fail` fail.
static std::mutex g_inject_mu;
static int g_inject_skip = 0, g_inject_fail = 0;

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s) {
    {
        std::lock_guard<std::mutex> lock(g_inject_mu);
        if (g_inject_fail > 0) {
            if (g_inject_skip > 0) {
                --g_inject_skip;
            } else {
                --g_inject_fail;
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
        }
    }
    return cudaMallocAsync(p, bytes, s);
}

void count_launch(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 148;
    }
    return cached[dev];
}

}  // namespace ar

using namespace ar;

namespace ar {

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return pa < pb + bbytes && pb < pa + abytes;
}

ar_status check_image_sizes(int n1, int n2, int nmin) {
    if (n1 < nmin || n2 < nmin)
        return fail(AR_ERR_INVALID_ARG, "image sizes n1=%d n2=%d must be >= %d", n1, n2, nmin);
    if ((long long)n1 * (long long)n2 > (1LL << 31))
        return fail(AR_ERR_INVALID_ARG, "image of %d x %d exceeds 2^31 pixels", n1, n2);
    return AR_OK;
}

ar_status check_support(int n1, int n2, int q1, int q2, int margin) {
    if (q1 < 0 || q2 < 0 || q1 > n1 - margin || q2 > n2 - margin)
        return fail(AR_ERR_INVALID_ARG,
                    "PSF support q=(%d,%d) must satisfy 0 <= q_j <= n_j - %d for n=(%d,%d)", q1, q2,
                    margin, n1, n2);
    return AR_OK;
}

ar_status check_psf_host(const double* h, int q1, int q2) {
    const size_t k = (size_t)(2 * q1 + 1) * (2 * q2 + 1);
    double s = 0.0;
    for (size_t i = 0; i < k; ++i) {
        if (!std::isfinite(h[i])) return fail(AR_ERR_INVALID_ARG, "PSF entry %zu is not finite", i);
        s += h[i];
    }
    if (std::fabs(s - 1.0) > 1e-6)
        return fail(AR_ERR_PSF_NOT_NORMALIZED, "PSF sums to %.17g, expected 1 within 1e-6", s);
    return AR_OK;
}

void set_pool_threshold_once() {
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long thr = ~0ULL;  // keep freed blocks in this process's pool
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

// Stream-ordered scratch released in the destructor (in stream order).
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    template <class T>
    ar_status get(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = dev_malloc_async(&q, count * sizeof(T) + 16, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (scratch)");
        ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return AR_OK;
    }
};

ar_status check_bc(int bc) {
    if (bc != AR_BC_ANTIREFLECTIVE && bc != AR_BC_REFLECTIVE && bc != AR_BC_PERIODIC)
        return fail(AR_ERR_INVALID_ARG, "unknown boundary condition %d", bc);
    return AR_OK;
}

namespace {
// AR_STENCIL_AUTO's measured choice per (device, n1, n2, q1, q2, bc).
std::mutex g_stencil_mu;
std::map<std::tuple<int, int, int, int, int, int>, int> g_stencil_choice;
}  // namespace

// The faster stencil arithmetic for a blur of this shape: one timing of each
// (y = A x on a zero image, median of three launches after a warm-up, CUDA
// events) the first time the shape is seen on a device, kept for the process;
// AR_STENCIL_FP32 where the tensor-core path does not apply.  psf is the
// caller's device PSF.
ar_status resolve_stencil(const float* psf, int n1, int n2, int q1, int q2, int bc, cudaStream_t s,
                          int* out) {
    *out = AR_STENCIL_FP32;
    ConvArgs a{};
    a.n1 = n1;
    a.n2 = n2;
    a.q1 = q1;
    a.q2 = q2;
    a.psf = psf;
    a.bc = bc;
    a.mode = CONV_STORE;
    if (!conv_tc_applies(a)) return AR_OK;          // aligned buffers below: q and bc decide
    int dev = 0;
    AR_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, n1, n2, q1, q2, bc);
    {
        std::lock_guard<std::mutex> lock(g_stencil_mu);
        auto it = g_stencil_choice.find(key);
        if (it != g_stencil_choice.end()) {
            *out = it->second;
            return AR_OK;
        }
    }
    set_pool_threshold_once();
    float t[2] = {0.f, 0.f};
    ar_status st = AR_OK;
    {
        Scratch ws(s);
        float *x = nullptr, *y = nullptr;
        uint8_t* plan = nullptr;
        const size_t n = (size_t)n1 * n2;
        st = ws.get(&x, n);
        if (st == AR_OK) st = ws.get(&y, n);
        if (st == AR_OK) st = ws.get(&plan, kConvTcPlanBytes);
        if (st == AR_OK && cudaMemsetAsync(x, 0, n * sizeof(float), s) != cudaSuccess)
            st = fail(AR_ERR_CUDA, "stencil timing input");
        if (st == AR_OK) st = conv_tc_plan(psf, q1, q2, 0, plan, s);
        a.x = x;
        a.out = y;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (st == AR_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
            st = fail(AR_ERR_CUDA, "stencil timing events");
        for (int v = 0; st == AR_OK && v < 2; ++v) {
            a.tcplan = v ? plan : nullptr;
            float r[3] = {0.f, 0.f, 0.f};
            st = conv_launch(a, s);                  // warm-up
            for (int k = 0; st == AR_OK && k < 3; ++k) {
                cudaEventRecord(e0, s);
                st = conv_launch(a, s);
                cudaEventRecord(e1, s);
                if (st == AR_OK && cudaEventSynchronize(e1) != cudaSuccess)
                    st = fail(AR_ERR_CUDA, "stencil timing");
                if (st == AR_OK) cudaEventElapsedTime(&r[k], e0, e1);
            }
            const float lo = r[0] < r[1] ? r[0] : r[1], hi = r[0] < r[1] ? r[1] : r[0];
            t[v] = r[2] < lo ? lo : (r[2] > hi ? hi : r[2]);
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
    if (st != AR_OK) return st;
    const int choice = t[1] < t[0] ? AR_STENCIL_F16X2 : AR_STENCIL_FP32;
    std::lock_guard<std::mutex> lock(g_stencil_mu);
    g_stencil_choice[key] = choice;
    *out = choice;
    return AR_OK;
}

ar_status apply_common(const float* x, float* y, int n1, int n2, const float* psf, int q1, int q2,
                       int bc, void* stream, int flip, int stencil = AR_STENCIL_FP32) {
    if (!x || !y || !psf) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    if (stencil != AR_STENCIL_FP32 && stencil != AR_STENCIL_F16X2 && stencil != AR_STENCIL_AUTO)
        return fail(AR_ERR_INVALID_ARG, "unknown stencil arithmetic %d", stencil);
    AR_TRY(check_bc(bc));
    AR_TRY(check_image_sizes(n1, n2, 1));
    AR_TRY(check_support(n1, n2, q1, q2, 1));
    const size_t nb = (size_t)n1 * n2 * sizeof(float);
    const size_t kb = (size_t)(2 * q1 + 1) * (2 * q2 + 1) * sizeof(float);
    if (overlaps(x, nb, y, nb)) return fail(AR_ERR_ALIAS, "output image overlaps the input image");
    if (overlaps(psf, kb, y, nb)) return fail(AR_ERR_ALIAS, "output image overlaps the PSF");
    ConvArgs a{};
    a.x = x;
    a.out = y;
    a.psf = psf;
    a.n1 = n1;
    a.n2 = n2;
    a.q1 = q1;
    a.q2 = q2;
    a.flip = flip;
    a.mode = CONV_STORE;
    a.bc = bc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (stencil == AR_STENCIL_AUTO) AR_TRY(resolve_stencil(psf, n1, n2, q1, q2, bc, s, &stencil));
    if (stencil == AR_STENCIL_F16X2 && conv_tc_applies(a)) {
        set_pool_threshold_once();       // the plan's stream-ordered allocation stays pooled
        Scratch ws(s);
        uint8_t* plan = nullptr;
        AR_TRY(ws.get(&plan, kConvTcPlanBytes));
        AR_TRY(conv_tc_plan(psf, q1, q2, flip, plan, s));
        a.tcplan = plan;
        return conv_launch(a, s);    // the plan is freed in stream order after the stencil
    }
    return conv_launch(a, s);
}

// Builds the preconditioner's device data on `s` without synchronizing.
void prec_release(ar_prec* P, cudaStream_t s) {
    if (!P) return;
    transform_plan_release(P->plan, s);
    if (P->fst) {
        cudaStreamSynchronize(s);
        fst_plan_destroy(P->fst);
    }
    for (void* q : {(void*)P->lam64, (void*)P->d64, (void*)P->d32, (void*)P->d32_odd})
        if (q) cudaFreeAsync(q, s);
    delete P;
}

ar_status prec_build(const double* psf_host, int q1, int q2, int n1, int n2, double alpha,
                     int bc, int precision, cudaStream_t s, bool keep64, ar_prec** out,
                     int correction, const ar_corr* model, bool grouped) {
    set_pool_threshold_once();
    ar_prec* P = new (std::nothrow) ar_prec();
    if (!P) return fail(AR_ERR_ALLOC, "host allocation of ar_prec");
    std::memset(P, 0, sizeof(*P));
    P->n1 = n1;
    P->n2 = n2;
    P->q1 = q1;
    P->q2 = q2;
    P->alpha = alpha;
    P->precision = precision;
    P->bc = bc;
    cudaGetDevice(&P->device);
    const size_t n = (size_t)n1 * n2;
    const size_t k = (size_t)(2 * q1 + 1) * (2 * q2 + 1);
    ar_status st = AR_OK;
    {
        Scratch tmp(s);
        double* h64 = nullptr;
        double* work = nullptr;
        st = tmp.get(&h64, k);
        if (st == AR_OK) st = tmp.get(&work, setup_scratch_doubles(q1, q2, n1, n2, bc));
        if (st == AR_OK) {
            cudaError_t e = cudaMemcpyAsync(h64, psf_host, k * sizeof(double),
                                            cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) st = cuda_fail(e, "PSF upload");
        }
        if (st == AR_OK && keep64) {
            if (dev_malloc_async((void**)&P->lam64, n * sizeof(double), s) != cudaSuccess ||
                dev_malloc_async((void**)&P->d64, n * sizeof(double), s) != cudaSuccess)
                st = fail(AR_ERR_ALLOC, "eigenvalue buffers");
        }
        if (st == AR_OK && dev_malloc_async((void**)&P->d32, n * sizeof(float), s) != cudaSuccess)
            st = fail(AR_ERR_ALLOC, "filter buffer");
        if (st == AR_OK && bc == AR_BC_PERIODIC &&
            dev_malloc_async((void**)&P->d32_odd, n * sizeof(float), s) != cudaSuccess)
            st = fail(AR_ERR_ALLOC, "odd filter buffer");
        double* delta = nullptr;
        if (st == AR_OK && correction) {
            double* cwork = nullptr;
            st = tmp.get(&delta, n);
            if (st == AR_OK) st = tmp.get(&cwork, corr_scratch_doubles(q1, q2, n1, n2));
            if (st == AR_OK)
                st = corr_delta(h64, q1, q2, n1, n2, correction == 2 ? model : nullptr, psf_host,
                                delta, cwork, s);
        }
        if (st == AR_OK)
            st = setup_eigen(h64, q1, q2, n1, n2, alpha, bc, P->lam64, P->d64, P->d32, P->d32_odd,
                             work, s, delta);
        if (precision == AR_PRECISION_FFT) {
            if (st == AR_OK) st = fst_plan_create(n1, n2, s, &P->fst);
        } else {
            // the reblur stencil writes the transform input folded (q <= 15, TMA path)
            if (st == AR_OK)
                st = transform_plan_create(n1, n2, bc, precision, s, &P->plan,
                                           (q1 > q2 ? q1 : q2) <= 15, grouped ? 2 : 1);
            if (st == AR_OK) st = transform_set_filter(P->plan, P->d32, s);
        }
    }
    if (st != AR_OK) {
        ar_symprec_destroy(P);
        return st;
    }
    *out = P;
    return AR_OK;
}

}  // namespace ar

namespace ar {

// The (D-)Landweber loop of ar_restore_bc on validated arguments; with Pext
// non-null its preconditioner is used instead of building one; with res_trace
// non-null the blur also accumulates ||g - A x_k||^2 (k = 0 .. iters, the last
// from one more blur of the final iterate).
static ar_status restore_run(const float* g, const double* psf_host, int n1, int n2, int q1, int q2,
                             double alpha, double tau, int iters, int bc, bool pc, int precision,
                             const float* x0, const float* f_true, float* x_out, double* rre_trace,
                             int* best_iter, void* stream, const ar_prec* Pext,
                             double* res_trace = nullptr) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    set_pool_threshold_once();
    bool tc_stencil = (precision & AR_STENCIL_F16X2) != 0;
    const bool auto_stencil = (precision & AR_STENCIL_AUTO) != 0;
    precision &= ~(AR_STENCIL_F16X2 | AR_STENCIL_AUTO);
    const size_t n = (size_t)n1 * n2;
    const size_t nb = n * sizeof(float);
    const size_t k = (size_t)(2 * q1 + 1) * (2 * q2 + 1);
    std::vector<float> h32(k);
    for (size_t i = 0; i < k; ++i) h32[i] = (float)psf_host[i];

    ar_prec* P = nullptr;            // built here (and destroyed) unless Pext is given
    const ar_prec* PP = Pext;
    unsigned long long bad = 0;
    int timeout = 0, conv_timeout = 0;
    int* conv_err = nullptr;
    std::vector<double> sums((size_t)iters + 1, 0.0);
    std::vector<double> rsums(res_trace ? (size_t)iters + 1 : 0, 0.0);
    ar_status st = AR_OK;
    {
        Scratch ws(s);
        float *psf = nullptr, *r = nullptr;
        double* dsum = nullptr;
        unsigned long long* dbad = nullptr;
        st = ws.get(&psf, k);
        if (st == AR_OK) st = ws.get(&r, n);
        if (st == AR_OK) st = ws.get(&dsum, (size_t)iters + 1);
        double* dres = nullptr;
        if (st == AR_OK && res_trace) st = ws.get(&dres, (size_t)iters + 1);
        if (st == AR_OK) st = ws.get(&dbad, 1);
        if (st == AR_OK && !(conv_err = conv_error_flag()))
            st = fail(AR_ERR_CUDA, "stencil error flag unavailable");
        if (st == AR_OK) {
            cudaError_t e = cudaMemcpyAsync(psf, h32.data(), k * sizeof(float),
                                            cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(dsum, 0, ((size_t)iters + 1) * sizeof(double), s);
            if (e == cudaSuccess && dres)
                e = cudaMemsetAsync(dres, 0, ((size_t)iters + 1) * sizeof(double), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(dbad, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(conv_err, 0, sizeof(int), s);
            if (e == cudaSuccess) {
                if (!x0) e = cudaMemsetAsync(x_out, 0, nb, s);
                else if (x0 != x_out) e = cudaMemcpyAsync(x_out, x0, nb, cudaMemcpyDeviceToDevice, s);
            }
            if (e != cudaSuccess) st = cuda_fail(e, "restore initialisation");
        }
        if (st == AR_OK && pc && !Pext) {
            int prec = precision;
            st = resolve_precision(precision, bc, n1, n2, s, &prec);
            if (st == AR_OK) st = prec_build(psf_host, q1, q2, n1, n2, alpha, bc, prec, s, false, &P);
            PP = P;
        }
        if (st == AR_OK && f_true) st = reduce_sq(f_true, n, dsum + iters, s);

        ConvArgs blur{};
        blur.x = x_out;
        blur.out = r;
        blur.aux = g;
        blur.psf = psf;
        blur.n1 = n1;
        blur.n2 = n2;
        blur.q1 = q1;
        blur.q2 = q2;
        blur.flip = 0;
        blur.mode = CONV_RESIDUAL;
        blur.bc = bc;
        ConvArgs reblur = blur;
        reblur.x = r;
        reblur.aux = nullptr;
        reblur.flip = 1;
        if (pc && st == AR_OK && PP->fst) {
            // A' r into the FFT-style transform's float32 input
            reblur.out = fst_input(PP->fst);
            reblur.mode = CONV_STORE;
        } else if (pc && st == AR_OK) {
            // A' r is written straight into the transform's bf16x3 operand planes
            reblur.out = nullptr;
            reblur.mode = CONV_SPLIT3;
            reblur.planes = transform_input_planes(PP->plan, &reblur.plane_stride, &reblur.ld,
                                                   &reblur.fold);
        } else {
            reblur.out = x_out;
            reblur.mode = CONV_AXPY;
            reblur.tau = (float)tau;
        }
        // successors: the reblur's is a contraction (no room beside the stencil) or
        // the blur; the blur's is a stencil (launched early beside the blur, the
        // folding reblur's CTAs ran slower: measured)
        reblur.early_trigger = reblur.mode == CONV_SPLIT3 || reblur.mode == CONV_STORE ? 1 : 0;
        blur.spread = reblur.spread = 1;
        reblur.f = f_true;
        if (st == AR_OK && auto_stencil) {            // the psf upload is ordered before
            int choice = AR_STENCIL_FP32;
            st = resolve_stencil(psf, n1, n2, q1, q2, bc, s, &choice);
            tc_stencil = choice == AR_STENCIL_F16X2;
        }
        if (st == AR_OK && tc_stencil && conv_tc_applies(blur)) {
            // the PSF's tensor-core plans for A and A' (the reblur's input r is
            // aligned like x_out when x_out is; conv_launch checks each call)
            uint8_t *pa = nullptr, *pr = nullptr;
            st = ws.get(&pa, kConvTcPlanBytes);
            if (st == AR_OK) st = ws.get(&pr, kConvTcPlanBytes);
            if (st == AR_OK) st = conv_tc_plan(psf, q1, q2, 0, pa, s);
            if (st == AR_OK) st = conv_tc_plan(psf, q1, q2, 1, pr, s);
            blur.tcplan = pa;
            reblur.tcplan = pr;
        }
        for (int it = 0; st == AR_OK && it < iters; ++it) {
            // the RRE numerator ||x_{k+1} - f||^2 is accumulated by the kernel that writes x_{k+1}
            blur.sumsq = dres ? dres + it : nullptr;             // ||r||^2 when requested
            st = conv_launch(blur, s);                           // r = g - A x_k
            if (!pc) reblur.sumsq = f_true ? dsum + it : nullptr;
            if (st == AR_OK) st = conv_launch(reblur, s);        // z = A' r  (or x += tau A' r)
            if (st == AR_OK && pc && PP->fst)                    // x += tau D z
                st = fst_apply(PP->fst, PP->d32, nullptr, x_out, true, (float)tau, s, f_true,
                               f_true ? dsum + it : nullptr);
            else if (st == AR_OK && pc)
                st = transform_apply(PP->plan, PP->d32, PP->d32_odd, nullptr, DIN_SPLIT, x_out,
                                     DOUT_AXPY, (float)tau, s, f_true,
                                     f_true ? dsum + it : nullptr);
        }
        if (st == AR_OK && dres) {                               // ||g - A x_iters||^2
            blur.sumsq = dres + iters;
            st = conv_launch(blur, s);
        }
        if (st == AR_OK) st = count_nonfinite(x_out, n, dbad, s);
        if (st == AR_OK) {
            cudaError_t e = cudaMemcpyAsync(sums.data(), dsum, sums.size() * sizeof(double),
                                            cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, dbad, sizeof(bad), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && dres)
                e = cudaMemcpyAsync(rsums.data(), dres, rsums.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && PP && PP->plan)
                e = cudaMemcpyAsync(&timeout, transform_error_flag(PP->plan), sizeof(int),
                                    cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&conv_timeout, conv_err, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) st = cuda_fail(e, "restore readback");
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (P) prec_release(P, s);       // after the synchronize above: no work pending
    if (st != AR_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "restore");
    if (res_trace)
        for (int k = 0; k <= iters; ++k) res_trace[k] = std::sqrt(rsums[(size_t)k]);
    if (f_true) {
        const double fn = sums[(size_t)iters];
        int best = 0;
        double bestv = 0.0;
        for (int it = 0; it < iters; ++it) {
            const double v = std::sqrt(sums[(size_t)it] / fn);
            if (rre_trace) rre_trace[it] = v;
            if (best == 0 || v < bestv) {
                best = it + 1;
                bestv = v;
            }
        }
        if (best_iter) *best_iter = best;
    }
    if (timeout) return fail(AR_ERR_TIMEOUT, "a tensor-core contraction gave up waiting");
    if (conv_timeout) return fail(AR_ERR_TIMEOUT, "a stencil gave up waiting for its halo tile");
    if (bad) return fail(AR_ERR_NONFINITE, "%llu non-finite entries in the final iterate", bad);
    return AR_OK;
}

ar_status check_precision(int precision, int bc, int n1, int n2) {
    if (precision < AR_PRECISION_FP32 || precision > AR_PRECISION_AUTO)
        return fail(AR_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (precision == AR_PRECISION_FFT && bc != AR_BC_ANTIREFLECTIVE)
        return fail(AR_ERR_UNSUPPORTED, "the FFT-style transform serves AR BCs only");
    if (precision == AR_PRECISION_FFT && !fst_supported(n1, n2))
        return fail(AR_ERR_UNSUPPORTED,
                    "FFT-style transform: n_j - 1 must split into coprime factors <= 256 "
                    "(n = %d x %d)", n1, n2);
    return AR_OK;
}

namespace {
// AR_PRECISION_AUTO's measured choice per (device, n1, n2).
std::mutex g_choice_mu;
std::map<std::tuple<int, int, int>, int> g_choice;

// Device milliseconds of one D application (median of three after a warm-up):
// the dense chain with its input already in operand form, or the FFT-style one.
ar_status time_transform(int precision, int n1, int n2, cudaStream_t s, float* ms) {
    const size_t n = (size_t)n1 * n2;
    float *d = nullptr, *y = nullptr, *z = nullptr;
    TransformPlan* tp = nullptr;
    FstPlan* fp = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ar_status st = AR_OK;
    cudaError_t ce = cudaMalloc((void**)&d, n * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&y, n * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&z, n * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMemsetAsync(d, 0, n * sizeof(float), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(y, 0, n * sizeof(float), s);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) st = cuda_fail(ce, "transform timing buffers");
    if (st == AR_OK) {
        if (precision == AR_PRECISION_FFT) st = fst_plan_create(n1, n2, s, &fp);
        else st = transform_plan_create(n1, n2, AR_BC_ANTIREFLECTIVE, precision, s, &tp, true);
    }
    if (st == AR_OK && tp) st = transform_set_filter(tp, d, s);
    auto once = [&](bool first) {
        if (fp) return fst_apply(fp, d, nullptr, z, false, 0.f, s);
        return transform_apply(tp, d, nullptr, first ? y : nullptr, first ? DIN_FP32 : DIN_SPLIT, z,
                               DOUT_STORE, 0.f, s);
    };
    if (st == AR_OK) st = once(true);
    float t[3] = {0.f, 0.f, 0.f};
    for (int r = 0; st == AR_OK && r < 3; ++r) {
        cudaEventRecord(e0, s);
        st = once(false);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(AR_ERR_CUDA, "transform timing");
        if (st == AR_OK) cudaEventElapsedTime(&t[r], e0, e1);
    }
    cudaStreamSynchronize(s);
    if (tp) transform_plan_destroy(tp);
    if (fp) fst_plan_destroy(fp);
    cudaFree(d);
    cudaFree(y);
    cudaFree(z);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const float lo = t[0] < t[1] ? t[0] : t[1], hi = t[0] < t[1] ? t[1] : t[0];
    *ms = t[2] < lo ? lo : (t[2] > hi ? hi : t[2]);
    return st;
}
}  // namespace

ar_status resolve_precision(int precision, int bc, int n1, int n2, cudaStream_t s, int* out) {
    *out = precision;
    if (precision != AR_PRECISION_AUTO) return AR_OK;
    *out = AR_PRECISION_FP32;
    if (bc != AR_BC_ANTIREFLECTIVE || !fst_supported(n1, n2)) return AR_OK;
    int dev = 0;
    AR_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, n1, n2);
    {
        std::lock_guard<std::mutex> lock(g_choice_mu);
        auto it = g_choice.find(key);
        if (it != g_choice.end()) {
            *out = it->second;
            return AR_OK;
        }
    }
    float t_dense = 0.f, t_fft = 0.f;
    AR_TRY(time_transform(AR_PRECISION_FP32, n1, n2, s, &t_dense));
    AR_TRY(time_transform(AR_PRECISION_FFT, n1, n2, s, &t_fft));
    const int choice = t_fft < t_dense ? AR_PRECISION_FFT : AR_PRECISION_FP32;
    std::lock_guard<std::mutex> lock(g_choice_mu);
    g_choice[key] = choice;
    *out = choice;
    return AR_OK;
}

// Argument checks shared by every entry point that takes ar_restore_bc's
// arguments, so that they accept exactly the same inputs.
static ar_status validate_restore_args(const float* g, const double* psf_host, int n1, int n2,
                                       int q1, int q2, double alpha, double tau, int iters, int bc,
                                       int precondition, int precision, const float* x0,
                                       const float* f_true, const float* x_out,
                                       const double* rre_trace, const int* best_iter) {
    if (!g || !psf_host || !x_out) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    AR_TRY(check_bc(bc));
    const bool pc = precondition != 0;
    if ((precision & AR_STENCIL_F16X2) && (precision & AR_STENCIL_AUTO))
        return fail(AR_ERR_INVALID_ARG, "AR_STENCIL_F16X2 and AR_STENCIL_AUTO together");
    precision &= ~(AR_STENCIL_F16X2 | AR_STENCIL_AUTO);   // the stencil flags combine with
                                                          // every precision
    if (pc) AR_TRY(check_precision(precision, bc, n1, n2));
    else if (precision < AR_PRECISION_FP32 || precision > AR_PRECISION_AUTO)
        return fail(AR_ERR_INVALID_ARG, "unknown precision %d", precision);
    AR_TRY(check_image_sizes(n1, n2, pc ? 3 : 1));
    AR_TRY(check_support(n1, n2, q1, q2, pc && bc == AR_BC_ANTIREFLECTIVE ? 3 : 1));
    if (iters < 0) return fail(AR_ERR_INVALID_ARG, "iters must be >= 0 (got %d)", iters);
    if (!(tau > 0.0) || !std::isfinite(tau))
        return fail(AR_ERR_INVALID_ARG, "tau must be finite and > 0 (got %g)", tau);
    if (pc && (!(alpha > 0.0) || !std::isfinite(alpha)))
        return fail(AR_ERR_INVALID_ARG, "alpha must be finite and > 0 (got %g)", alpha);
    if ((rre_trace || best_iter) && !f_true)
        return fail(AR_ERR_INVALID_ARG, "rre_trace/best_iter need f_true");
    AR_TRY(check_psf_host(psf_host, q1, q2));
    const size_t nb = (size_t)n1 * n2 * sizeof(float);
    if (overlaps(x_out, nb, g, nb)) return fail(AR_ERR_ALIAS, "x_out overlaps g");
    if (f_true && overlaps(x_out, nb, f_true, nb)) return fail(AR_ERR_ALIAS, "x_out overlaps f_true");
    if (x0 && x0 != x_out && overlaps(x0, nb, x_out, nb))
        return fail(AR_ERR_ALIAS, "x0 partially overlaps x_out");
    return AR_OK;
}

}  // namespace ar

extern "C" {

const char* ar_status_string(ar_status s) {
    switch (s) {
        case AR_OK: return "AR_OK";
        case AR_ERR_INVALID_ARG: return "AR_ERR_INVALID_ARG";
        case AR_ERR_ALIAS: return "AR_ERR_ALIAS";
        case AR_ERR_PSF_NOT_NORMALIZED: return "AR_ERR_PSF_NOT_NORMALIZED";
        case AR_ERR_ALLOC: return "AR_ERR_ALLOC";
        case AR_ERR_CUDA: return "AR_ERR_CUDA";
        case AR_ERR_NONFINITE: return "AR_ERR_NONFINITE";
        case AR_ERR_TIMEOUT: return "AR_ERR_TIMEOUT";
        case AR_ERR_UNSUPPORTED: return "AR_ERR_UNSUPPORTED";
    }
    return "AR_UNKNOWN";
}

const char* ar_last_error_detail(void) { return g_detail; }

const char* ar_version(void) { return "ar-gb300 0.1 (sm_103a)"; }

unsigned long long ar_kernel_launches(void) { return g_launches.load(); }

ar_status ar_set_stencil_wait_polls(unsigned polls) { return conv_set_wait_polls(polls); }

void ar_inject_alloc_failures(int skip, int count) {
    std::lock_guard<std::mutex> lock(g_inject_mu);
    g_inject_skip = skip > 0 ? skip : 0;
    g_inject_fail = count > 0 ? count : 0;
}

ar_status ar_blur_apply(const float* x, float* y, int n1, int n2, const float* psf, int q1, int q2,
                        void* stream) {
    return apply_common(x, y, n1, n2, psf, q1, q2, AR_BC_ANTIREFLECTIVE, stream, 0);
}

ar_status ar_reblur_apply(const float* x, float* y, int n1, int n2, const float* psf, int q1,
                          int q2, void* stream) {
    return apply_common(x, y, n1, n2, psf, q1, q2, AR_BC_ANTIREFLECTIVE, stream, 1);
}

ar_status ar_blur_apply_bc(const float* x, float* y, int n1, int n2, const float* psf, int q1,
                           int q2, int bc, void* stream) {
    return apply_common(x, y, n1, n2, psf, q1, q2, bc, stream, 0);
}

ar_status ar_reblur_apply_bc(const float* x, float* y, int n1, int n2, const float* psf, int q1,
                             int q2, int bc, void* stream) {
    return apply_common(x, y, n1, n2, psf, q1, q2, bc, stream, 1);
}

ar_status ar_blur_apply_ex(const float* x, float* y, int n1, int n2, const float* psf, int q1,
                           int q2, int bc, int stencil, void* stream) {
    return apply_common(x, y, n1, n2, psf, q1, q2, bc, stream, 0, stencil);
}

ar_status ar_reblur_apply_ex(const float* x, float* y, int n1, int n2, const float* psf, int q1,
                             int q2, int bc, int stencil, void* stream) {
    return apply_common(x, y, n1, n2, psf, q1, q2, bc, stream, 1, stencil);
}

ar_status ar_symprec_setup(const double* psf_host, int q1, int q2, int n1, int n2, double alpha,
                           void* stream, ar_prec** out) {
    return ar_symprec_setup_bc(psf_host, q1, q2, n1, n2, alpha, AR_BC_ANTIREFLECTIVE,
                               AR_PRECISION_FP32, stream, out);
}

ar_status ar_symprec_setup_ex(const double* psf_host, int q1, int q2, int n1, int n2, double alpha,
                              int precision, void* stream, ar_prec** out) {
    return ar_symprec_setup_bc(psf_host, q1, q2, n1, n2, alpha, AR_BC_ANTIREFLECTIVE, precision,
                               stream, out);
}

ar_status ar_symprec_setup_bc(const double* psf_host, int q1, int q2, int n1, int n2, double alpha,
                              int bc, int precision, void* stream, ar_prec** out) {
    if (!psf_host || !out) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    AR_TRY(check_bc(bc));
    AR_TRY(check_precision(precision, bc, n1, n2));
    AR_TRY(check_image_sizes(n1, n2, 3));
    // AR needs the interior grid of size n - 2 to hold the support
    AR_TRY(check_support(n1, n2, q1, q2, bc == AR_BC_ANTIREFLECTIVE ? 3 : 1));
    if (!(alpha > 0.0) || !std::isfinite(alpha))
        return fail(AR_ERR_INVALID_ARG, "alpha must be finite and > 0 (got %g)", alpha);
    AR_TRY(check_psf_host(psf_host, q1, q2));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ar_prec* P = nullptr;
    int prec = precision;
    AR_TRY(resolve_precision(precision, bc, n1, n2, s, &prec));
    AR_TRY(prec_build(psf_host, q1, q2, n1, n2, alpha, bc, prec, s, true, &P));
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ar_symprec_destroy(P);
        return cuda_fail(e, "setup");
    }
    *out = P;
    return AR_OK;
}

ar_status ar_symprec_setup_corrected(const double* psf_host, int q1, int q2, int n1, int n2,
                                     double alpha, const ar_corr* M, int precision, void* stream,
                                     ar_prec** out) {
    if (!psf_host || !out) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    if (precision != AR_PRECISION_FP32 && precision != AR_PRECISION_BF16X2)
        return fail(AR_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (M && (q1 != AR_CORR_Q || q2 != AR_CORR_Q))
        return fail(AR_ERR_INVALID_ARG, "the correction model takes %dx%d PSFs", 2 * AR_CORR_Q + 1,
                    2 * AR_CORR_Q + 1);
    if (M && !corr_on_current_device(M))
        return fail(AR_ERR_INVALID_ARG, "the correction model belongs to another device");
    AR_TRY(check_image_sizes(n1, n2, 3));
    AR_TRY(check_support(n1, n2, q1, q2, 3));
    if (!(alpha > 0.0) || !std::isfinite(alpha))
        return fail(AR_ERR_INVALID_ARG, "alpha must be finite and > 0 (got %g)", alpha);
    AR_TRY(check_psf_host(psf_host, q1, q2));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ar_prec* P = nullptr;
    AR_TRY(prec_build(psf_host, q1, q2, n1, n2, alpha, AR_BC_ANTIREFLECTIVE, precision, s, true, &P,
                      M ? 2 : 1, M));
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ar_symprec_destroy(P);
        return cuda_fail(e, "setup");
    }
    *out = P;
    return AR_OK;
}

ar_status ar_symprec_solve(const ar_prec* P, const float* y, float* z, void* stream) {
    if (!P || !y || !z) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    int dev = 0;
    AR_CUDA(cudaGetDevice(&dev));
    if (dev != P->device) return fail(AR_ERR_INVALID_ARG, "preconditioner belongs to device %d", P->device);
    const size_t nb = (size_t)P->n1 * P->n2 * sizeof(float);
    if (y != z && overlaps(y, nb, z, nb)) return fail(AR_ERR_ALIAS, "z partially overlaps y");
    if (P->fst)
        return fst_apply(P->fst, P->d32, y, z, false, 0.f, static_cast<cudaStream_t>(stream));
    return transform_apply(P->plan, P->d32, P->d32_odd, y, DIN_FP32, z, DOUT_STORE, 0.f,
                           static_cast<cudaStream_t>(stream));
}

ar_status ar_symprec_eigenvalues(const ar_prec* P, double* lambda_host, double* d_host) {
    if (!P) return fail(AR_ERR_INVALID_ARG, "null preconditioner");
    if (!P->lam64 || !P->d64) return fail(AR_ERR_INVALID_ARG, "float64 eigenvalues not kept");
    const size_t nb = (size_t)P->n1 * P->n2 * sizeof(double);
    if (lambda_host) AR_CUDA(cudaMemcpy(lambda_host, P->lam64, nb, cudaMemcpyDeviceToHost));
    if (d_host) AR_CUDA(cudaMemcpy(d_host, P->d64, nb, cudaMemcpyDeviceToHost));
    return AR_OK;
}

ar_status ar_symprec_precision(const ar_prec* P, int* precision) {
    if (!P || !precision) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    *precision = P->precision;
    return AR_OK;
}

ar_status ar_symprec_shape(const ar_prec* P, int* n1, int* n2) {
    if (!P) return fail(AR_ERR_INVALID_ARG, "null preconditioner");
    if (n1) *n1 = P->n1;
    if (n2) *n2 = P->n2;
    return AR_OK;
}

void ar_symprec_destroy(ar_prec* P) {
    if (!P) return;
    cudaDeviceSynchronize();
    transform_plan_destroy(P->plan);
    fst_plan_destroy(P->fst);
    cudaFree(P->lam64);
    cudaFree(P->d64);
    cudaFree(P->d32);
    cudaFree(P->d32_odd);
    delete P;
}

ar_status ar_restore(const float* g, const double* psf_host, int n1, int n2, int q1, int q2,
                     double alpha, double tau, int iters, int precondition, const float* x0,
                     const float* f_true, float* x_out, double* rre_trace, int* best_iter,
                     void* stream) {
    return ar_restore_bc(g, psf_host, n1, n2, q1, q2, alpha, tau, iters, AR_BC_ANTIREFLECTIVE,
                         precondition, AR_PRECISION_FP32, x0, f_true, x_out, rre_trace, best_iter,
                         stream);
}

ar_status ar_restore_ex(const float* g, const double* psf_host, int n1, int n2, int q1, int q2,
                        double alpha, double tau, int iters, int precondition, int precision,
                        const float* x0, const float* f_true, float* x_out, double* rre_trace,
                        int* best_iter, void* stream) {
    return ar_restore_bc(g, psf_host, n1, n2, q1, q2, alpha, tau, iters, AR_BC_ANTIREFLECTIVE,
                         precondition, precision, x0, f_true, x_out, rre_trace, best_iter, stream);
}

ar_status ar_restore_bc(const float* g, const double* psf_host, int n1, int n2, int q1, int q2,
                        double alpha, double tau, int iters, int bc, int precondition,
                        int precision, const float* x0, const float* f_true, float* x_out,
                        double* rre_trace, int* best_iter, void* stream) {
    AR_TRY(validate_restore_args(g, psf_host, n1, n2, q1, q2, alpha, tau, iters, bc, precondition,
                                 precision, x0, f_true, x_out, rre_trace, best_iter));
    return restore_run(g, psf_host, n1, n2, q1, q2, alpha, tau, iters, bc, precondition != 0,
                       precision, x0, f_true, x_out, rre_trace, best_iter, stream, nullptr);
}

ar_status ar_restore_residuals(const float* g, const double* psf_host, int n1, int n2, int q1,
                               int q2, double alpha, double tau, int iters, int bc,
                               int precondition, int precision, const float* x0,
                               const float* f_true, float* x_out, double* rre_trace,
                               int* best_iter, double* res_trace, void* stream) {
    if (!res_trace) return fail(AR_ERR_INVALID_ARG, "null pointer argument (res_trace)");
    AR_TRY(validate_restore_args(g, psf_host, n1, n2, q1, q2, alpha, tau, iters, bc, precondition,
                                 precision, x0, f_true, x_out, rre_trace, best_iter));
    return restore_run(g, psf_host, n1, n2, q1, q2, alpha, tau, iters, bc, precondition != 0,
                       precision, x0, f_true, x_out, rre_trace, best_iter, stream, nullptr,
                       res_trace);
}

ar_status ar_restore_prec(const ar_prec* P, const float* g, const double* psf_host, double tau,
                          int iters, const float* x0, const float* f_true, float* x_out,
                          double* rre_trace, int* best_iter, void* stream) {
    if (!P || !g || !psf_host || !x_out) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    const int n1 = P->n1, n2 = P->n2, q1 = P->q1, q2 = P->q2;
    int dev = 0;
    AR_CUDA(cudaGetDevice(&dev));
    if (dev != P->device) return fail(AR_ERR_INVALID_ARG, "preconditioner belongs to device %d", P->device);
    if (iters < 0) return fail(AR_ERR_INVALID_ARG, "iters must be >= 0 (got %d)", iters);
    if (!(tau > 0.0) || !std::isfinite(tau))
        return fail(AR_ERR_INVALID_ARG, "tau must be finite and > 0 (got %g)", tau);
    if ((rre_trace || best_iter) && !f_true)
        return fail(AR_ERR_INVALID_ARG, "rre_trace/best_iter need f_true");
    AR_TRY(check_psf_host(psf_host, q1, q2));
    const size_t nb = (size_t)n1 * n2 * sizeof(float);
    if (overlaps(x_out, nb, g, nb)) return fail(AR_ERR_ALIAS, "x_out overlaps g");
    if (f_true && overlaps(x_out, nb, f_true, nb)) return fail(AR_ERR_ALIAS, "x_out overlaps f_true");
    if (x0 && x0 != x_out && overlaps(x0, nb, x_out, nb))
        return fail(AR_ERR_ALIAS, "x0 partially overlaps x_out");
    return restore_run(g, psf_host, n1, n2, q1, q2, P->alpha, tau, iters, P->bc, true, P->precision,
                       x0, f_true, x_out, rre_trace, best_iter, stream, P);
}

}  // extern "C"
