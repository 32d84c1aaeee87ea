// Batched (D-)Landweber restoration of many images of uneven sizes.
//
// Images are independent problems (each with its own size, PSF and alpha).  A
// batch plan builds, once, every image's preconditioner (FP64 setup of eqs.
// simmetrizzata2d, funzione_generatrice and TikFilter; the constant transform
// matrices are cached per size) and scratch, then runs every iteration of
// eq. DLandweberMeth (reblurred A' of Section 4, x_0 = 0, RRE of every iterate)
// for all images at once:
//   * one persistent stencil launch (conv_group_*): the residual blur of every
//     image, then its reblur, as single tiles handed out by a device queue,
//     each reblur tile waiting (bounded) for its own image's blur tiles;
//   * four grouped contraction launches (transform_group_*), one per product of
//     the AR transform pair, every image's tiles as work items, largest K first.
// The whole restoration -- 5 launches per iteration instead of 6 per image per
// iteration -- is captured into one CUDA graph; ar_batch_run is one graph launch.
//
// A project autotuner picks the stencil launch's tile geometry (64- or 54-row
// tiles) and its persistent CTAs per SM by timing a few iterations of every
// candidate on the batch itself.

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
    std::vector<ar::ConvArgs> blurs, reblurs;
    ar::ConvGroup* conv = nullptr;
    ar::TransformGroup* tg = nullptr;
    cudaStream_t cs = nullptr;                 // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    unsigned long long kernels_per_run = 0;
    // autotuner: chosen geometry / CTAs per SM and every candidate's time
    int geometry = 0, ctas_per_sm = 0;
    std::vector<double> cand_ms;
    std::vector<int> cand_geo, cand_cta;
};

using namespace ar;

namespace {

ar_status validate_item(const ar_batch_item& it, int idx, int pc) {
    if (!it.g || !it.psf_host || !it.x_out)
        return fail(AR_ERR_INVALID_ARG, "item %d: null pointer", idx);
    AR_TRY(check_image_sizes(it.n1, it.n2, pc ? 3 : 1));
    AR_TRY(check_support(it.n1, it.n2, it.q1, it.q2, pc ? 3 : 1));
    if ((it.q1 > it.q2 ? it.q1 : it.q2) > 15)
        return fail(AR_ERR_UNSUPPORTED, "item %d: batched PSFs need q <= 15", idx);
    if ((it.n2 & 3) != 0 || (reinterpret_cast<uintptr_t>(it.x_out) & 15) != 0)
        return fail(AR_ERR_UNSUPPORTED, "item %d: batched images need n2 %% 4 == 0 and a "
                                        "16-byte aligned x_out", idx);
    if (pc && (!(it.alpha > 0.0) || !std::isfinite(it.alpha)))
        return fail(AR_ERR_INVALID_ARG, "item %d: alpha must be finite and > 0", idx);
    AR_TRY(check_psf_host(it.psf_host, it.q1, it.q2));
    const size_t nb = (size_t)it.n1 * it.n2 * sizeof(float);
    if (overlaps(it.x_out, nb, it.g, nb)) return fail(AR_ERR_ALIAS, "item %d: x_out overlaps g", idx);
    if (it.f_true && overlaps(it.x_out, nb, it.f_true, nb))
        return fail(AR_ERR_ALIAS, "item %d: x_out overlaps f_true", idx);
    return AR_OK;
}

// Enqueues `iters` iterations of the whole batch (from the current x_j) on s.
ar_status enqueue_iterations(ar_batch* B, int iters, cudaStream_t s) {
    AR_TRY(conv_group_reset(B->conv, s));
    for (int k = 0; k < iters; ++k) {
        AR_TRY(conv_group_apply(B->conv, k, s));
        if (B->tg) AR_TRY(transform_group_apply(B->tg, k, s));
    }
    return AR_OK;
}

// One restoration of the batch: x_j = 0, ||f_j||^2, `iters` iterations, the
// non-finite scan.
ar_status enqueue_run(ar_batch* B, cudaStream_t s) {
    for (int j = 0; j < B->count; ++j) {
        const ar_batch_item& it = B->items[(size_t)j];
        const size_t n = (size_t)it.n1 * it.n2;
        AR_CUDA(cudaMemsetAsync(it.x_out, 0, n * sizeof(float), s));
        AR_CUDA(cudaMemsetAsync(B->sums[(size_t)j], 0, ((size_t)B->iters + 1) * sizeof(double), s));
        if (it.f_true) AR_TRY(reduce_sq(it.f_true, n, B->sums[(size_t)j] + B->iters, s));
    }
    AR_TRY(enqueue_iterations(B, B->iters, s));
    for (int j = 0; j < B->count; ++j) {
        const ar_batch_item& it = B->items[(size_t)j];
        AR_TRY(count_nonfinite(it.x_out, (size_t)it.n1 * it.n2, B->bad + j, s));
    }
    return AR_OK;
}

ar_status make_conv_group(ar_batch* B, int geometry, int ctas, int iters, ConvGroup** out) {
    return conv_group_create(B->blurs.data(), B->reblurs.data(), B->count, geometry, ctas, iters, out);
}

// Device time of `iters` batch iterations with stencil geometry / CTAs per SM,
// captured and replayed (the second replay is timed).
ar_status time_candidate(ar_batch* B, int geometry, int ctas, int iters, double* ms, int* used) {
    ConvGroup* g = nullptr;
    AR_TRY(make_conv_group(B, geometry, ctas, iters, &g));
    *used = conv_group_ctas_per_sm(g);
    ConvGroup* keep = B->conv;
    B->conv = g;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ar_status st = AR_OK;
    cudaError_t ce = cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        st = enqueue_iterations(B, iters, B->cs);
        ce = cudaStreamEndCapture(B->cs, &graph);
    }
    if (st == AR_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (st == AR_OK && ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (st == AR_OK && ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (st == AR_OK && ce == cudaSuccess) ce = cudaGraphLaunch(exec, B->cs);
    if (st == AR_OK && ce == cudaSuccess) ce = cudaEventRecord(e0, B->cs);
    if (st == AR_OK && ce == cudaSuccess) ce = cudaGraphLaunch(exec, B->cs);
    if (st == AR_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, B->cs);
    if (st == AR_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float f = 0.f;
    if (st == AR_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&f, e0, e1);
    if (st == AR_OK && ce != cudaSuccess) st = cuda_fail(ce, "autotuner candidate");
    *ms = f;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    B->conv = keep;
    conv_group_destroy(g);
    return st;
}

}  // namespace

extern "C" {

void ar_batch_destroy(ar_batch* B) {
    if (!B) return;
    cudaDeviceSynchronize();
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    conv_group_destroy(B->conv);
    transform_group_destroy(B->tg);
    for (ar_prec* P : B->precs) ar_symprec_destroy(P);
    for (float* p : B->r) cudaFree(p);
    for (float* p : B->psf) cudaFree(p);
    for (double* p : B->sums) cudaFree(p);
    cudaFree(B->bad);
    if (B->done) cudaEventDestroy(B->done);
    if (B->cs) cudaStreamDestroy(B->cs);
    delete B;
}

ar_status ar_batch_create(const ar_batch_item* items, int count, double tau, int iters,
                          int precondition, int precision, int tuning, void* stream,
                          ar_batch** out) {
    if (!items || !out || count <= 0) return fail(AR_ERR_INVALID_ARG, "items/out null or count <= 0");
    if (iters < 0) return fail(AR_ERR_INVALID_ARG, "iters must be >= 0");
    if (!(tau > 0.0) || !std::isfinite(tau)) return fail(AR_ERR_INVALID_ARG, "tau must be > 0");
    if (precision != AR_PRECISION_FP32 && precision != AR_PRECISION_BF16X2)
        return fail(AR_ERR_INVALID_ARG, "unknown precision %d", precision);
    if (tuning < 0 || tuning > 8)
        return fail(AR_ERR_INVALID_ARG, "tuning must be 0 (autotune) or 1..8 CTAs per SM (got %d)",
                    tuning);
    const int pc = precondition != 0;
    for (int j = 0; j < count; ++j) AR_TRY(validate_item(items[j], j, pc));
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
    B->blurs.assign(count, ConvArgs{});
    B->reblurs.assign(count, ConvArgs{});
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
            st = prec_build(it.psf_host, it.q1, it.q2, it.n1, it.n2, it.alpha, AR_BC_ANTIREFLECTIVE,
                            precision, s, false, &B->precs[j], 0, nullptr, true);
        if (st != AR_OK) break;
        ConvArgs& blur = B->blurs[(size_t)j];
        blur.x = it.x_out;
        blur.out = B->r[j];
        blur.aux = it.g;
        blur.psf = B->psf[j];
        blur.n1 = it.n1;
        blur.n2 = it.n2;
        blur.q1 = it.q1;
        blur.q2 = it.q2;
        blur.mode = CONV_RESIDUAL;
        blur.bc = AR_BC_ANTIREFLECTIVE;
        ConvArgs& reblur = B->reblurs[(size_t)j];
        reblur = blur;
        reblur.x = B->r[j];
        reblur.aux = nullptr;
        reblur.flip = 1;
        if (pc) {
            reblur.out = nullptr;
            reblur.mode = CONV_SPLIT3;
            reblur.planes = transform_input_planes(B->precs[j]->plan, &reblur.plane_stride,
                                                   &reblur.ld, &reblur.fold);
        } else {
            reblur.out = it.x_out;
            reblur.mode = CONV_AXPY;
            reblur.tau = (float)tau;
            reblur.f = it.f_true;
            reblur.sumsq = it.f_true ? B->sums[j] : nullptr;      // + iteration in the kernel
        }
    }
    if (st != AR_OK) return bail(st);
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(AR_ERR_CUDA, "batch setup"));
    if (pc) {
        std::vector<TransformPlan*> plans((size_t)count);
        std::vector<float*> outs((size_t)count);
        std::vector<const float*> fs((size_t)count);
        std::vector<double*> sq((size_t)count);
        for (int j = 0; j < count; ++j) {
            plans[(size_t)j] = B->precs[(size_t)j]->plan;
            outs[(size_t)j] = items[j].x_out;
            fs[(size_t)j] = items[j].f_true;
            sq[(size_t)j] = B->sums[(size_t)j];
        }
        st = transform_group_create(plans.data(), count, outs.data(), fs.data(), sq.data(),
                                    (float)tau, &B->tg);
        if (st != AR_OK) return bail(st);
    }
    if (cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(AR_ERR_CUDA, "capture stream"));
    if (cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(AR_ERR_CUDA, "done event"));

    // autotuner: stencil geometry x persistent CTAs per SM, timed on the batch
    // (from x = 0, so that no candidate runs on stale data)
    for (int j = 0; j < count; ++j)
        if (cudaMemsetAsync(items[j].x_out, 0, (size_t)items[j].n1 * items[j].n2 * sizeof(float),
                            B->cs) != cudaSuccess)
            return bail(fail(AR_ERR_CUDA, "batch output initialisation"));
    B->geometry = 0;
    B->ctas_per_sm = tuning > 0 ? tuning : 2;
    if (tuning == 0 && iters > 0) {
        const int tune_iters = iters < 3 ? iters : 3;
        double best = 0.0;
        for (int geo = 0; geo < 2; ++geo)
            for (int ctas = 1; ctas <= 3; ++ctas) {
                double ms = 0.0;
                int used = 0;
                st = time_candidate(B, geo, ctas, tune_iters, &ms, &used);
                if (st != AR_OK) return bail(st);
                if (used != ctas) continue;            // occupancy caps it: same as a smaller one
                B->cand_geo.push_back(geo);
                B->cand_cta.push_back(ctas);
                B->cand_ms.push_back(ms);
                if (best == 0.0 || ms < best) {
                    best = ms;
                    B->geometry = geo;
                    B->ctas_per_sm = ctas;
                }
            }
    }
    st = make_conv_group(B, B->geometry, B->ctas_per_sm, iters > 0 ? iters : 1, &B->conv);
    if (st != AR_OK) return bail(st);
    B->ctas_per_sm = conv_group_ctas_per_sm(B->conv);

    const unsigned long long l0 = ar_kernel_launches();
    if (cudaStreamBeginCapture(B->cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bail(fail(AR_ERR_CUDA, "begin capture"));
    st = enqueue_run(B, B->cs);
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
    int* conv_err = conv_error_flag();
    if (!conv_err) return fail(AR_ERR_CUDA, "stencil error flag unavailable");
    AR_CUDA(cudaMemsetAsync(B->bad, 0, B->count * sizeof(unsigned long long), s));
    AR_CUDA(cudaMemsetAsync(conv_err, 0, sizeof(int), s));
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
    int conv_timeout = 0;
    int* conv_err = conv_error_flag();
    if (conv_err) AR_CUDA(cudaMemcpy(&conv_timeout, conv_err, sizeof(int), cudaMemcpyDeviceToHost));
    for (int j = 0; j < B->count; ++j) {
        if (bad[j]) st = fail(AR_ERR_NONFINITE, "item %d: %llu non-finite entries", j, bad[j]);
        if (B->precs[j]) {
            int flag = 0;
            AR_CUDA(cudaMemcpy(&flag, transform_error_flag(B->precs[j]->plan), sizeof(int),
                               cudaMemcpyDeviceToHost));
            if (flag) st = fail(AR_ERR_TIMEOUT, "item %d: a contraction gave up waiting", j);
        }
    }
    if (conv_timeout) st = fail(AR_ERR_TIMEOUT, "a batched stencil gave up waiting");
    return st;
}

ar_status ar_batch_tuning(const ar_batch* B, int* geometry, int* ctas_per_sm, int* transform,
                          int* candidates, int* cand_geometry, int* cand_ctas, double* cand_ms,
                          int max_candidates) {
    if (!B) return fail(AR_ERR_INVALID_ARG, "null batch");
    if (geometry) *geometry = B->geometry;
    if (transform) {
        *transform = 0;
        if (B->precondition && B->count > 0) {
            *transform |= B->reblurs[0].fold ? 1 : 0;
            *transform |= transform_group_paired(B->tg) ? 2 : 0;
        }
    }
    if (ctas_per_sm) *ctas_per_sm = B->ctas_per_sm;
    const int n = (int)B->cand_ms.size();
    if (candidates) *candidates = n;
    for (int i = 0; i < n && i < max_candidates; ++i) {
        if (cand_geometry) cand_geometry[i] = B->cand_geo[(size_t)i];
        if (cand_ctas) cand_ctas[i] = B->cand_cta[(size_t)i];
        if (cand_ms) cand_ms[i] = B->cand_ms[(size_t)i];
    }
    return AR_OK;
}

}  // extern "C"
