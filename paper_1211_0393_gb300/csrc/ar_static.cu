// Plain Landweber restoration that allocates no memory.
//
// ar_restore() takes its scratch (the residual image r = g - A x_k, the
// device copy of the PSF, the float64 RRE accumulators) from the stream's
// memory pool.  Callers that have reserved the device memory themselves, for
// example a framework that pre-allocates the whole GPU into its own pool or a
// fixed-budget service that must never call into the CUDA allocator, cannot
// let a library allocate behind their back.  ar_restore_plain_static() runs
// the same kernels in the same order as ar_restore(..., precondition = 0, ...)
// but keeps that scratch in one file-scope static device array, so it calls no
// cudaMalloc, cudaFree or other allocating routine.
//
// The array is sized for images of up to AR_STATIC_MAX_PIXELS pixels, PSFs of
// up to AR_STATIC_MAX_PSF taps and AR_STATIC_MAX_ITERS iterations (about
// 4.1 MiB); every GPU that loads this library keeps it until the process
// exits.  All calls on a device share it: calls whose GPU work overlaps (on
// different streams, or from different host threads) race.

#include "ar_internal.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

namespace ar {
namespace {

constexpr size_t kMaxPixels = AR_STATIC_MAX_PIXELS;
constexpr size_t kMaxPsf = AR_STATIC_MAX_PSF;
constexpr size_t kMaxIters = AR_STATIC_MAX_ITERS;

constexpr size_t round256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffR = 0;                                             // float[kMaxPixels]
constexpr size_t kOffPsf = round256(kOffR + kMaxPixels * sizeof(float)); // float[kMaxPsf]
constexpr size_t kOffSums = round256(kOffPsf + kMaxPsf * sizeof(float)); // double[kMaxIters + 1]
constexpr size_t kOffBad = round256(kOffSums + (kMaxIters + 1) * sizeof(double));
constexpr size_t kScratchBytes = round256(kOffBad + sizeof(unsigned long long));

__device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Device address of g_static_scratch on the current device.  The host-side
// name of the array is not a device address; the address is looked up once
// per device with that device current.
ar_status scratch_base(unsigned char** out) {
    static std::mutex mu;
    static unsigned char* base[64] = {nullptr};
    int dev = 0;
    AR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(AR_ERR_UNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!base[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        base[dev] = static_cast<unsigned char*>(p);
    }
    *out = base[dev];
    return AR_OK;
}

}  // namespace
}  // namespace ar

using namespace ar;

extern "C" ar_status ar_restore_plain_static(const float* g, const double* psf_host, int n1, int n2,
                                             int q1, int q2, double tau, int iters,
                                             const float* x0, const float* f_true, float* x_out,
                                             double* rre_trace, int* best_iter, void* stream) {
    if (!g || !psf_host || !x_out) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    if (n1 < 1 || n2 < 1) return fail(AR_ERR_INVALID_ARG, "image sizes must be >= 1");
    if ((size_t)n1 * (size_t)n2 > kMaxPixels)
        return fail(AR_ERR_INVALID_ARG,
                    "image of %d x %d pixels exceeds the static scratch limit of %zu pixels", n1,
                    n2, kMaxPixels);
    if (q1 < 0 || q2 < 0 || q1 > n1 - 1 || q2 > n2 - 1)
        return fail(AR_ERR_INVALID_ARG, "PSF support q=(%d,%d) must satisfy 0 <= q_j <= n_j - 1",
                    q1, q2);
    const size_t k = (size_t)(2 * q1 + 1) * (2 * q2 + 1);
    if (k > kMaxPsf)
        return fail(AR_ERR_INVALID_ARG, "PSF of %zu taps exceeds the static scratch limit of %zu",
                    k, kMaxPsf);
    if (iters < 0 || (size_t)iters > kMaxIters)
        return fail(AR_ERR_INVALID_ARG, "iters=%d outside 0..%zu (static scratch limit)", iters,
                    kMaxIters);
    if (!(tau > 0.0) || !std::isfinite(tau))
        return fail(AR_ERR_INVALID_ARG, "tau must be finite and > 0 (got %g)", tau);
    if ((rre_trace || best_iter) && !f_true)
        return fail(AR_ERR_INVALID_ARG, "rre_trace/best_iter need f_true");
    double hs = 0.0;
    for (size_t i = 0; i < k; ++i) {
        if (!std::isfinite(psf_host[i]))
            return fail(AR_ERR_INVALID_ARG, "PSF entry %zu is not finite", i);
        hs += psf_host[i];
    }
    if (std::fabs(hs - 1.0) > 1e-6)
        return fail(AR_ERR_PSF_NOT_NORMALIZED, "PSF sums to %.17g, expected 1 within 1e-6", hs);
    const size_t n = (size_t)n1 * n2;
    const size_t nb = n * sizeof(float);
    if (overlaps(x_out, nb, g, nb)) return fail(AR_ERR_ALIAS, "x_out overlaps g");
    if (f_true && overlaps(x_out, nb, f_true, nb)) return fail(AR_ERR_ALIAS, "x_out overlaps f_true");
    if (x0 && x0 != x_out && overlaps(x0, nb, x_out, nb))
        return fail(AR_ERR_ALIAS, "x0 partially overlaps x_out");

    unsigned char* base = nullptr;
    AR_TRY(scratch_base(&base));
    // the stencils' bounded-wait flag is a static device int too (no allocation)
    int* conv_err = conv_error_flag();
    if (!conv_err) return fail(AR_ERR_CUDA, "stencil error flag unavailable");
    float* r = reinterpret_cast<float*>(base + kOffR);
    float* psf = reinterpret_cast<float*>(base + kOffPsf);
    double* dsum = reinterpret_cast<double*>(base + kOffSums);
    unsigned long long* dbad = reinterpret_cast<unsigned long long*>(base + kOffBad);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    float h32[kMaxPsf];
    for (size_t i = 0; i < k; ++i) h32[i] = (float)psf_host[i];
    // the accumulators keep the previous call's values: clear them first
    AR_CUDA(cudaMemcpyAsync(psf, h32, k * sizeof(float), cudaMemcpyHostToDevice, s));
    AR_CUDA(cudaMemsetAsync(dsum, 0, ((size_t)iters + 1) * sizeof(double), s));
    AR_CUDA(cudaMemsetAsync(dbad, 0, sizeof(unsigned long long), s));
    AR_CUDA(cudaMemsetAsync(conv_err, 0, sizeof(int), s));
    if (!x0) AR_CUDA(cudaMemsetAsync(x_out, 0, nb, s));
    else if (x0 != x_out) AR_CUDA(cudaMemcpyAsync(x_out, x0, nb, cudaMemcpyDeviceToDevice, s));
    if (f_true) AR_TRY(reduce_sq(f_true, n, dsum + iters, s));

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
    blur.spread = 1;
    ConvArgs reblur = blur;
    reblur.x = r;
    reblur.aux = nullptr;
    reblur.out = x_out;
    reblur.flip = 1;
    reblur.mode = CONV_AXPY;
    reblur.tau = (float)tau;
    reblur.f = f_true;
    for (int it = 0; it < iters; ++it) {
        AR_TRY(conv_launch(blur, s));                     // r = g - A x_k
        reblur.sumsq = f_true ? dsum + it : nullptr;
        AR_TRY(conv_launch(reblur, s));                   // x_{k+1} = x_k + tau A' r
    }
    AR_TRY(count_nonfinite(x_out, n, dbad, s));
    double sums[kMaxIters + 1];
    unsigned long long bad = 0;
    int conv_timeout = 0;
    AR_CUDA(cudaMemcpyAsync(sums, dsum, ((size_t)iters + 1) * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    AR_CUDA(cudaMemcpyAsync(&bad, dbad, sizeof(bad), cudaMemcpyDeviceToHost, s));
    AR_CUDA(cudaMemcpyAsync(&conv_timeout, conv_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AR_CUDA(cudaStreamSynchronize(s));
    if (f_true) {
        const double fn = sums[iters];
        int best = 0;
        double bestv = 0.0;
        for (int it = 0; it < iters; ++it) {
            const double v = std::sqrt(sums[it] / fn);
            if (rre_trace) rre_trace[it] = v;
            if (best == 0 || v < bestv) {
                best = it + 1;
                bestv = v;
            }
        }
        if (best_iter) *best_iter = best;
    }
    if (conv_timeout) return fail(AR_ERR_TIMEOUT, "a stencil gave up waiting for its halo tile");
    if (bad) return fail(AR_ERR_NONFINITE, "%llu non-finite entries in the final iterate", bad);
    return AR_OK;
}
