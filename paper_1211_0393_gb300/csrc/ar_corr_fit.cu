// Training targets of the learned spectral correction, read off restorations
// that the symmetrized D-Landweber itself produces.
//
// The iteration of Section 4 (eq. DLandweberMeth with the reblurred A'),
// x_{k+1} = x_k + tau D z_k with z_k = A'(g - A x_k), moves the reblurred
// residual by z_{k+1} = z_k - tau A'A D z_k.  In the AR basis of Theorem 1
// (z^ = T~ z, D = T diag(d) T~) that is z^_{k+1} = z^_k - tau M (d o z^_k) with
// M = T~ A'A T; were M diagonal, frequency by frequency
// z^_{k+1} = (1 - tau mu d) z^_k.  The restoration loop of this file keeps the
// spectral operand W_k = d o z^_k that the second contraction of every
// iteration produces, and accumulates per frequency, over consecutive iterates,
//     num = sum_k W_k (W_k - W_{k+1}),   wgt = sum_k W_k^2,
// whence the least-squares response mu^ = num / (tau d wgt) and the target
// delta^ = mu^ - lambda_s^2 (interior AR frequencies, shrunk towards 0 where
// the image has no content, see kPrior), pooled onto the model's 33 x 33 grid
// with weight wgt x the bilinear weight of each node.

#include "ar_internal.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace ar {
namespace {

constexpr int CG = AR_CORR_GRID;                  // model grid points per axis
constexpr int CQ = AR_CORR_Q;                     // the model's PSFs are (2 CQ + 1)^2
constexpr int CIN = (2 * CQ + 1) * (2 * CQ + 1);
constexpr int COUT = CG * CG;

unsigned blocks(size_t n) { return (unsigned)((n + 255) / 256); }

// g += nu ||g|| / ||e|| e, the norms' squares in sums[0], sums[1] (eq. of the
// noise model: a fixed relative noise level).
__global__ void noise_mix_kernel(float* __restrict__ g, const float* __restrict__ e, size_t n,
                                 const double* __restrict__ sums, double nu) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double sc = nu * sqrt(sums[0] / sums[1]);
    g[i] = (float)((double)g[i] + sc * (double)e[i]);
}

__device__ __forceinline__ float bf16_bits(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// W_k from its bf16 planes; with `first` unset, the pair (W_{k-1}, W_k) is added.
__global__ void spec_stats_kernel(const uint16_t* __restrict__ planes, size_t pstride, int ld,
                                  int np, int N1, int N2, float* __restrict__ wprev,
                                  double* __restrict__ num, double* __restrict__ wgt, int first) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N1 * N2) return;
    const size_t o = (size_t)(idx / N2) * ld + idx % N2;
    float tail = 0.f;
    for (int p = np - 1; p >= 1; --p) tail += bf16_bits(planes[p * pstride + o]);
    const float w = bf16_bits(planes[o]) + tail;
    if (!first) {
        const double wp = wprev[idx];
        num[idx] += wp * (wp - (double)w);
        wgt[idx] += wp * wp;
    }
    wprev[idx] = w;
}

// Prior weight of the fit, in units of the mean weight of the interior
// frequencies: delta^ = (mu^ - lambda_s^2) w / (w + kPrior w_mean), a Tikhonov
// fit of mu towards lambda_s^2.  Where the image has almost no content the fit
// divides two differences of tiny spectral values and is set by rounding; the
// prior keeps such frequencies near 0 (a perturbation e of the spectral values
// moves delta^ by at most about e sqrt(K) / (tau d sqrt(kPrior w_mean))).  The
// mean, not the largest weight, keeps the rule independent of the image size.
constexpr double kPrior = 5.0;

__device__ __forceinline__ bool interior(size_t idx, const FoldDims& f1, const FoldDims& f2,
                                         int& s1, int& s2) {
    const int N2 = 2 * f2.Hs;
    const int k1 = spec_of((int)(idx / N2), f1, s1), k2 = spec_of((int)(idx % N2), f2, s2);
    return (k1 == 1 || k1 == 3) && (k2 == 1 || k2 == 3);     // not a boundary line, not padding
}

// *wsum += the sum of wgt over the interior frequencies.
__global__ void weight_sum_kernel(const double* __restrict__ wgt, int n1, int n2,
                                  double* __restrict__ wsum) {
    const FoldDims f1 = fold_dims(n1), f2 = fold_dims(n2);
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    int s1, s2;
    if (idx < (size_t)(2 * f1.Hs) * (2 * f2.Hs) && interior(idx, f1, f2, s1, s2)) v = wgt[idx];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(wsum, v);
}

// mu^ - lambda_s^2 at every interior AR frequency, pooled onto the model grid:
// acc[node] += b wgt delta, acc[COUT + node] += b wgt.
__global__ void fit_pool_kernel(const double* __restrict__ num, const double* __restrict__ wgt,
                                const float* __restrict__ dfold, const double* __restrict__ lam,
                                int n1, int n2, double tau, const double* __restrict__ wsum,
                                double* __restrict__ acc) {
    const FoldDims f1 = fold_dims(n1), f2 = fold_dims(n2);
    const int N1 = 2 * f1.Hs, N2 = 2 * f2.Hs;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N1 * N2) return;
    int s1 = 0, s2 = 0;
    if (!interior(idx, f1, f2, s1, s2)) return;
    const double w8 = wgt[idx];
    if (!(w8 > 0.0)) return;
    const double mu = num[idx] / (tau * (double)dfold[idx] * w8);
    const double l = lam[(size_t)s1 * n2 + s2];
    const double rho = kPrior * *wsum / ((double)(n1 - 2) * (double)(n2 - 2));
    const double delta = (mu - l * l) * (w8 / (w8 + rho));
    // node coordinates u = x / pi * (G - 1), x = s pi / (m - 1)
    const double u1 = (double)s1 * (CG - 1) / (double)(n1 - 1);
    const double u2 = (double)s2 * (CG - 1) / (double)(n2 - 1);
    int i = (int)floor(u1), j = (int)floor(u2);
    i = i > CG - 2 ? CG - 2 : i;
    j = j > CG - 2 ? CG - 2 : j;
    const double t = u1 - i, v = u2 - j;
    const double b[4] = {(1 - t) * (1 - v), (1 - t) * v, t * (1 - v), t * v};
    const int node[4] = {i * CG + j, i * CG + j + 1, (i + 1) * CG + j, (i + 1) * CG + j + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        atomicAdd(acc + node[q], b[q] * w8 * delta);
        atomicAdd(acc + COUT + node[q], b[q] * w8);
    }
}

__global__ void pool_finish_kernel(const double* __restrict__ acc, double* __restrict__ table) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= COUT) return;
    const double w = acc[COUT + i];
    table[i] = w > 0.0 ? acc[i] / w : 0.0;
}

__global__ void or_flag_kernel(const int* __restrict__ src, int* __restrict__ dst) {
    if (*src) *dst = 1;
}

// Stream-ordered buffers released (in stream order) when the owner goes.
struct Buffers {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Buffers(cudaStream_t st) : s(st) {}
    ~Buffers() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    template <class T>
    ar_status get(T** p, size_t count) {
        void* q = nullptr;
        const cudaError_t e = dev_malloc_async(&q, count * sizeof(T) + 16, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (target scratch)");
        ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return AR_OK;
    }
};

}  // namespace
}  // namespace ar

using namespace ar;

extern "C" ar_status ar_corr_restoration_targets(const float* f, const float* e, int n1, int n2,
                                                 const double* psfs_host, int count, double nu,
                                                 double alpha, double tau, int iters,
                                                 double* tables_host, void* stream) {
    if (!f || !e || !psfs_host || !tables_host) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    if (count < 1) return fail(AR_ERR_INVALID_ARG, "count must be >= 1 (got %d)", count);
    if (iters < 2) return fail(AR_ERR_INVALID_ARG, "iters must be >= 2 (got %d)", iters);
    AR_TRY(check_image_sizes(n1, n2, 3));
    AR_TRY(check_support(n1, n2, CQ, CQ, 3));
    if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(AR_ERR_INVALID_ARG, "nu must be finite and >= 0");
    if (!(alpha > 0.0) || !std::isfinite(alpha))
        return fail(AR_ERR_INVALID_ARG, "alpha must be finite and > 0 (got %g)", alpha);
    if (!(tau > 0.0) || !std::isfinite(tau))
        return fail(AR_ERR_INVALID_ARG, "tau must be finite and > 0 (got %g)", tau);
    for (int j = 0; j < count; ++j) AR_TRY(check_psf_host(psfs_host + (size_t)j * CIN, CQ, CQ));
    const size_t nb = (size_t)n1 * n2 * sizeof(float);
    if (overlaps(f, nb, e, nb) && f != e) return fail(AR_ERR_ALIAS, "f partially overlaps e");
    set_pool_threshold_once();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* conv_err = conv_error_flag();
    if (!conv_err) return fail(AR_ERR_CUDA, "stencil error flag unavailable");
    const size_t n = (size_t)n1 * n2;
    const FoldDims f1 = fold_dims(n1), f2 = fold_dims(n2);
    const size_t nspec = (size_t)(2 * f1.Hs) * (2 * f2.Hs);
    std::vector<float> h32((size_t)count * CIN);
    for (size_t i = 0; i < h32.size(); ++i) h32[i] = (float)psfs_host[i];
    std::vector<double> tabs((size_t)count * COUT, 0.0);
    int anyerr = 0, conv_timeout = 0;
    ar_status st = AR_OK;
    {
        Buffers b(s);
        float *g = nullptr, *r = nullptr, *x = nullptr, *psf = nullptr, *wprev = nullptr;
        double *sums = nullptr, *num = nullptr, *wgt = nullptr, *acc = nullptr, *tab = nullptr;
        double* wsum = nullptr;
        int* derr = nullptr;
        if (st == AR_OK) st = b.get(&g, n);
        if (st == AR_OK) st = b.get(&r, n);
        if (st == AR_OK) st = b.get(&x, n);
        if (st == AR_OK) st = b.get(&psf, h32.size());
        if (st == AR_OK) st = b.get(&wprev, nspec);
        if (st == AR_OK) st = b.get(&sums, 2);
        if (st == AR_OK) st = b.get(&num, nspec);
        if (st == AR_OK) st = b.get(&wgt, nspec);
        if (st == AR_OK) st = b.get(&acc, 2 * COUT);
        if (st == AR_OK) st = b.get(&tab, tabs.size());
        if (st == AR_OK) st = b.get(&derr, 1);
        if (st == AR_OK) st = b.get(&wsum, 1);
        if (st == AR_OK) {
            cudaError_t ce = cudaMemcpyAsync(psf, h32.data(), h32.size() * sizeof(float),
                                             cudaMemcpyHostToDevice, s);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(derr, 0, sizeof(int), s);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(conv_err, 0, sizeof(int), s);
            if (ce != cudaSuccess) st = cuda_fail(ce, "target initialisation");
        }
        if (st == AR_OK) st = reduce_sq(e, n, sums + 1, s);          // ||e||^2, once
        for (int j = 0; st == AR_OK && j < count; ++j) {
            const double* hj = psfs_host + (size_t)j * CIN;
            const float* pj = psf + (size_t)j * CIN;
            // g = A f + nu ||A f|| e / ||e||
            ConvArgs gen{};
            gen.x = f;
            gen.out = g;
            gen.psf = pj;
            gen.n1 = n1;
            gen.n2 = n2;
            gen.q1 = gen.q2 = CQ;
            gen.mode = CONV_STORE;
            gen.bc = AR_BC_ANTIREFLECTIVE;
            st = conv_launch(gen, s);
            cudaError_t ce = cudaSuccess;
            if (st == AR_OK) ce = cudaMemsetAsync(sums, 0, sizeof(double), s);
            if (st == AR_OK && ce == cudaSuccess) st = reduce_sq(g, n, sums, s);
            if (st == AR_OK && ce == cudaSuccess) {
                noise_mix_kernel<<<blocks(n), 256, 0, s>>>(g, e, n, sums, nu);
                count_launch();
                ce = cudaGetLastError();
            }
            if (ce == cudaSuccess) ce = cudaMemsetAsync(x, 0, n * sizeof(float), s);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(num, 0, nspec * sizeof(double), s);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(wgt, 0, nspec * sizeof(double), s);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(acc, 0, 2 * COUT * sizeof(double), s);
            if (ce == cudaSuccess) ce = cudaMemsetAsync(wsum, 0, sizeof(double), s);
            if (ce != cudaSuccess) st = cuda_fail(ce, "target restoration setup");
            ar_prec* P = nullptr;
            if (st == AR_OK)
                st = prec_build(hj, CQ, CQ, n1, n2, alpha, AR_BC_ANTIREFLECTIVE, AR_PRECISION_FP32,
                                s, true, &P);
            const uint16_t* wpl = nullptr;
            size_t wps = 0;
            int wld = 0, wnp = 0;
            const float* dfold = nullptr;
            if (st == AR_OK) st = transform_spectral_view(P->plan, &wpl, &wps, &wld, &wnp, &dfold);
            ConvArgs blur{};
            blur.x = x;
            blur.out = r;
            blur.aux = g;
            blur.psf = pj;
            blur.n1 = n1;
            blur.n2 = n2;
            blur.q1 = blur.q2 = CQ;
            blur.mode = CONV_RESIDUAL;
            blur.bc = AR_BC_ANTIREFLECTIVE;
            blur.spread = 1;
            ConvArgs reblur = blur;
            reblur.x = r;
            reblur.aux = nullptr;
            reblur.out = nullptr;
            reblur.flip = 1;
            reblur.mode = CONV_SPLIT3;
            reblur.early_trigger = 1;
            if (st == AR_OK)
                reblur.planes = transform_input_planes(P->plan, &reblur.plane_stride, &reblur.ld,
                                                       &reblur.fold);
            for (int k = 0; st == AR_OK && k < iters; ++k) {
                st = conv_launch(blur, s);                               // r = g - A x_k
                if (st == AR_OK) st = conv_launch(reblur, s);            // z_k = A' r
                if (st == AR_OK)                                         // W_k, x_{k+1}
                    st = transform_apply(P->plan, P->d32, nullptr, nullptr, DIN_SPLIT, x,
                                         DOUT_AXPY, (float)tau, s);
                if (st == AR_OK) {
                    spec_stats_kernel<<<blocks(nspec), 256, 0, s>>>(
                        wpl, wps, wld, wnp, 2 * f1.Hs, 2 * f2.Hs, wprev, num, wgt, k == 0 ? 1 : 0);
                    count_launch();
                    if (cudaGetLastError() != cudaSuccess) st = fail(AR_ERR_CUDA, "spectral statistics");
                }
            }
            if (st == AR_OK) {
                weight_sum_kernel<<<blocks(nspec), 256, 0, s>>>(wgt, n1, n2, wsum);
                fit_pool_kernel<<<blocks(nspec), 256, 0, s>>>(num, wgt, dfold, P->lam64, n1, n2,
                                                              tau, wsum, acc);
                pool_finish_kernel<<<blocks(COUT), 256, 0, s>>>(acc, tab + (size_t)j * COUT);
                or_flag_kernel<<<1, 1, 0, s>>>(transform_error_flag(P->plan), derr);
                count_launch(4);
                if (cudaGetLastError() != cudaSuccess) st = fail(AR_ERR_CUDA, "target fit");
            }
            if (P) prec_release(P, s);
        }
        if (st == AR_OK) {
            cudaError_t ce = cudaMemcpyAsync(tabs.data(), tab, tabs.size() * sizeof(double),
                                             cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(&anyerr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(&conv_timeout, conv_err, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (ce != cudaSuccess) st = cuda_fail(ce, "target readback");
        }
    }
    const cudaError_t se = cudaStreamSynchronize(s);
    if (st != AR_OK) return st;
    if (se != cudaSuccess) return cuda_fail(se, "restoration targets");
    if (anyerr) return fail(AR_ERR_TIMEOUT, "a tensor-core contraction gave up waiting");
    if (conv_timeout) return fail(AR_ERR_TIMEOUT, "a stencil gave up waiting for its halo tile");
    for (size_t i = 0; i < tabs.size(); ++i)
        if (!std::isfinite(tabs[i]))
            return fail(AR_ERR_NONFINITE, "target table entry %zu is not finite", i);
    std::memcpy(tables_host, tabs.data(), tabs.size() * sizeof(double));
    return AR_OK;
}
