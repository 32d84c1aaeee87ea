// Batched (D-)Landweber restoration of many images of uneven sizes.
//
// A batch plan builds, once, every image's preconditioner (FP64 setup of
// eqs. simmetrizzata2d, funzione_generatrice and TikFilter) and scratch, and
// captures the whole restoration of every image (eq. DLandweberMeth with the
// reblurred A' of Section 4, x_0 = 0, RRE of every iterate) into one CUDA graph.
// Images are independent problems: their kernel chains are captured on
// `concurrency` parallel branches, so the kernels of different images overlap
// on the GPU and small images fill the SMs a single 1024^2 image leaves idle.
// Each ar_batch_run() is one graph launch.

#include "ar_internal.cuh"

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

struct ar_batch {
    int device = 0;
    int count = 0, iters = 0, precondition = 0;
    std::vector<ar_batch_item> items;
    std::vector<ar_prec*> precs;
    std::vector<float*> r, psf;
    std::vector<double*> sums;                 // [iters + 1] per image
    unsigned long long* bad = nullptr;         // [count]
    cudaStream_t cs = nullptr;                 // capture stream
    std::vector<cudaStream_t> branches;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    unsigned long long kernels_per_run = 0;
};

using namespace ar;

namespace {

ar_status validate_item(const ar_batch_item& it, int idx, int pc, int iters) {
    if (!it.g || !it.psf_host || !it.x_out)
        return fail(AR_ERR_INVALID_ARG, "item %d: null pointer", idx);
    AR_TRY(check_image_sizes(it.n1, it.n2, pc ? 3 : 1));
    AR_TRY(check_support(it.n1, it.n2, it.q1, it.q2, pc ? 3 : 1));
    if (pc && (!(it.alpha > 0.0) || !std::isfinite(it.alpha)))
        return fail(AR_ERR_INVALID_ARG, "item %d: alpha must be finite and > 0", idx);
    AR_TRY(check_psf_host(it.psf_host, it.q1, it.q2));
    const size_t nb = (size_t)it.n1 * it.n2 * sizeof(float);
    if (overlaps(it.x_out, nb, it.g, nb)) return fail(AR_ERR_ALIAS, "item %d: x_out overlaps g", idx);
    if (it.f_true && overlaps(it.x_out, nb, it.f_true, nb))
        return fail(AR_ERR_ALIAS, "item %d: x_out overlaps f_true", idx);
    (void)iters;
    return AR_OK;
}

// Enqueues image j's whole restoration on stream s (inside the capture).
ar_status enqueue_image(ar_batch* B, int j, cudaStream_t s, double tau) {
    const ar_batch_item& it = B->items[j];
    const size_t n = (size_t)it.n1 * it.n2;
    const bool pc = B->precondition != 0;
    AR_CUDA(cudaMemsetAsync(it.x_out, 0, n * sizeof(float), s));
    AR_CUDA(cudaMemsetAsync(B->sums[j], 0, ((size_t)B->iters + 1) * sizeof(double), s));
    if (it.f_true) AR_TRY(reduce_sq(it.f_true, n, B->sums[j] + B->iters, s));
    ConvArgs blur{};
    blur.x = it.x_out;
    blur.out = B->r[j];
    blur.aux = it.g;
    blur.psf = B->psf[j];
    blur.n1 = it.n1;
    blur.n2 = it.n2;
    blur.q1 = it.q1;
    blur.q2 = it.q2;
    blur.mode = CONV_RESIDUAL;
    ConvArgs reblur = blur;
    reblur.x = B->r[j];
    reblur.aux = nullptr;
    reblur.flip = 1;
    reblur.f = it.f_true;
    if (pc) {
        reblur.out = nullptr;
        reblur.mode = CONV_SPLIT3;
        reblur.planes = transform_input_planes(B->precs[j]->plan, &reblur.plane_stride, &reblur.ld,
                                               &reblur.fold);
    } else {
        reblur.out = it.x_out;
        reblur.mode = CONV_AXPY;
        reblur.tau = (float)tau;
    }
    // trigger placement as in the restoration loop of ar_restore
    reblur.early_trigger = pc ? 1 : 0;
    for (int k = 0; k < B->iters; ++k) {
        AR_TRY(conv_launch(blur, s));
        if (!pc) reblur.sumsq = it.f_true ? B->sums[j] + k : nullptr;
        AR_TRY(conv_launch(reblur, s));
        if (pc)
            AR_TRY(transform_apply(B->precs[j]->plan, B->precs[j]->d32, nullptr, nullptr,
                                   DIN_SPLIT, it.x_out, DOUT_AXPY, (float)tau, s, it.f_true,
                                   it.f_true ? B->sums[j] + k : nullptr));
    }
    AR_TRY(count_nonfinite(it.x_out, n, B->bad + j, s));
    return AR_OK;
}

}  // namespace

extern "C" {

void ar_batch_destroy(ar_batch* B) {
    if (!B) return;
    cudaDeviceSynchronize();
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (ar_prec* P : B->precs) ar_symprec_destroy(P);
    for (float* p : B->r) cudaFree(p);
    for (float* p : B->psf) cudaFree(p);
    for (double* p : B->sums) cudaFree(p);
    cudaFree(B->bad);
    for (cudaStream_t s : B->branches) cudaStreamDestroy(s);
    for (cudaEvent_t e : B->events) cudaEventDestroy(e);
    if (B->done) cudaEventDestroy(B->done);
    if (B->cs) cudaStreamDestroy(B->cs);
    delete B;
}

ar_status ar_batch_create(const ar_batch_item* items, int count, double tau, int iters,
                          int precondition, int precision, int concurrency, void* stream,
                          ar_batch** out) {
    if (!items || !out || count <= 0) return fail(AR_ERR_INVALID_ARG, "items/out null or count <= 0");
    if (iters < 0) return fail(AR_ERR_INVALID_ARG, "iters must be >= 0");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(AR_ERR_INVALID_ARG, "tau must be > 0");
    if (precision != AR_PRECISION_FP32 && precision != AR_PRECISION_BF16X2)
        return fail(AR_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (concurrency < 1 || concurrency > 64)
        return fail(AR_ERR_INVALID_ARG, "concurrency must be in 1..64 (got %d)", concurrency);
    const int pc = precondition != 0;
    for (int j = 0; j < count; ++j) AR_TRY(validate_item(items[j], j, pc, iters));
    for (int a = 0; a < count; ++a)
        for (int b = 0; b < count; ++b) {
            if (a == b) continue;
            const size_t na = (size_t)items[a].n1 * items[a].n2 * sizeof(float);
            const size_t nb = (size_t)items[b].n1 * items[b].n2 * sizeof(float);
            if (overlaps(items[a].x_out, na, items[b].x_out, nb) ||
                overlaps(items[a].x_out, na, items[b].g, nb) ||
                (items[b].f_true && overlaps(items[a].x_out, na, items[b].f_true, nb)))
                return fail(AR_ERR_ALIAS, "item %d's x_out overlaps an input or output of item %d", a, b);
        }
    set_pool_threshold_once();
    ar_batch* B = new (std::nothrow) ar_batch();
    if (!B) return fail(AR_ERR_ALLOC, "host allocation of the batch plan");
    B->count = count;
    cudaGetDevice(&B->device);
    B->iters = iters;
    B->precondition = pc;
    B->items.assign(items, items + count);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ar_status st = AR_OK;
    auto bail = [&](ar_status e) {
        ar_batch_destroy(B);
        return e;
    };
    B->precs.assign(count, nullptr);
    B->r.assign(count, nullptr);
    B->psf.assign(count, nullptr);
    B->sums.assign(count, nullptr);
    if (cudaMalloc((void**)&B->bad, count * sizeof(unsigned long long)) != cudaSuccess)
        return bail(fail(AR_ERR_ALLOC, "batch flags"));
    cudaMemset(B->bad, 0, count * sizeof(unsigned long long));
    for (int j = 0; j < count && st == AR_OK; ++j) {
        const ar_batch_item& it = items[j];
        const size_t n = (size_t)it.n1 * it.n2;
        const size_t k = (size_t)(2 * it.q1 + 1) * (2 * it.q2 + 1);
        if (cudaMalloc((void**)&B->r[j], n * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&B->psf[j], k * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&B->sums[j], ((size_t)iters + 1) * sizeof(double)) != cudaSuccess) {
            st = fail(AR_ERR_ALLOC, "batch scratch of item %d", j);
            break;
        }
        std::vector<float> h32(k);
        for (size_t i = 0; i < k; ++i) h32[i] = (float)it.psf_host[i];
        if (cudaMemcpy(B->psf[j], h32.data(), k * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(AR_ERR_CUDA, "PSF upload of item %d", j);
        if (st == AR_OK && pc)
            st = prec_build(it.psf_host, it.q1, it.q2, it.n1, it.n2, it.alpha,
                            AR_BC_ANTIREFLECTIVE, precision, s, false, &B->precs[j]);
    }
    if (st != AR_OK) return bail(st);
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(AR_ERR_CUDA, "batch setup"));

    // capture: fork `concurrency` branches off the capture stream, one image chain per turn
    const int nb = concurrency < count ? concurrency : count;
    if (cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(AR_ERR_CUDA, "capture stream"));
    B->branches.assign(nb, nullptr);
    B->events.assign(nb + 1, nullptr);
    for (int b = 0; b < nb; ++b)
        if (cudaStreamCreateWithFlags(&B->branches[b], cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(AR_ERR_CUDA, "branch stream"));
    for (auto& e : B->events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(AR_ERR_CUDA, "branch event"));
    if (cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(AR_ERR_CUDA, "done event"));
    const unsigned long long l0 = ar_kernel_launches();
    if (cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return bail(fail(AR_ERR_CUDA, "begin capture"));
    cudaEventRecord(B->events[nb], B->cs);
    for (int b = 0; b < nb; ++b) cudaStreamWaitEvent(B->branches[b], B->events[nb], 0);
    for (int j = 0; j < count && st == AR_OK; ++j) st = enqueue_image(B, j, B->branches[j % nb], tau);
    for (int b = 0; b < nb; ++b) {
        cudaEventRecord(B->events[b], B->branches[b]);
        cudaStreamWaitEvent(B->cs, B->events[b], 0);
    }
    cudaError_t ce = cudaStreamEndCapture(B->cs, &B->graph);
    if (st != AR_OK) return bail(st);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "end capture"));
    B->kernels_per_run = ar_kernel_launches() - l0;
    ce = cudaGraphInstantiate(&B->exec, B->graph, 0);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "graph instantiate"));
    *out = B;
    return AR_OK;
}

ar_status ar_batch_run(ar_batch* B, void* stream) {
    if (!B) return fail(AR_ERR_INVALID_ARG, "null batch");
    int dev = 0;
    AR_CUDA(cudaGetDevice(&dev));
    if (dev != B->device) return fail(AR_ERR_INVALID_ARG, "batch belongs to device %d", B->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    AR_CUDA(cudaMemsetAsync(B->bad, 0, B->count * sizeof(unsigned long long), s));
    AR_CUDA(cudaGraphLaunch(B->exec, s));
    AR_CUDA(cudaEventRecord(B->done, s));
    return AR_OK;
}

ar_status ar_batch_results(ar_batch* B, double* rre_traces, int* best_iters,
                           unsigned long long* kernels_per_run) {
    if (!B) return fail(AR_ERR_INVALID_ARG, "null batch");
    AR_CUDA(cudaEventSynchronize(B->done));
    if (kernels_per_run) *kernels_per_run = B->kernels_per_run;
    std::vector<double> sums((size_t)B->iters + 1);
    ar_status st = AR_OK;
    for (int j = 0; j < B->count; ++j) {
        if (!B->items[j].f_true) {
            if (best_iters) best_iters[j] = 0;
            continue;
        }
        AR_CUDA(cudaMemcpy(sums.data(), B->sums[j], sums.size() * sizeof(double),
                           cudaMemcpyDeviceToHost));
        const double fn = sums[B->iters];
        int best = 0;
        double bestv = 0.0;
        for (int k = 0; k < B->iters; ++k) {
            const double v = std::sqrt(sums[k] / fn);
            if (rre_traces) rre_traces[(size_t)j * B->iters + k] = v;
            if (best == 0 || v < bestv) {
                best = k + 1;
                bestv = v;
            }
        }
        if (best_iters) best_iters[j] = best;
    }
    std::vector<unsigned long long> bad(B->count);
    AR_CUDA(cudaMemcpy(bad.data(), B->bad, B->count * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost));
    for (int j = 0; j < B->count; ++j) {
        if (bad[j]) st = fail(AR_ERR_NONFINITE, "item %d: %llu non-finite entries", j, bad[j]);
        if (B->precs[j]) {
            int flag = 0;
            AR_CUDA(cudaMemcpy(&flag, transform_error_flag(B->precs[j]->plan), sizeof(int),
                               cudaMemcpyDeviceToHost));
            if (flag) st = fail(AR_ERR_TIMEOUT, "item %d: a contraction gave up waiting", j);
        }
    }
    return st;
}

}  // extern "C"
