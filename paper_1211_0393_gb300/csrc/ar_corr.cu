// Spectral correction of the symmetrized preconditioner, and the small MLP
// that learns it (training and inference kernels).
//
// With s the symmetrized PSF (eq. simmetrizzata2d) and a = h - s the
// antisymmetric part, the response of A'A at an AR frequency x is, for large
// images, the flip average of |h^(x)|^2 = lambda_s(x)^2 + delta(x) with
//     delta(x1, x2) = (|a^(x1, x2)|^2 + |a^(-x1, x2)|^2) / 2,
//     a^(w) = sum_s a_s exp(-i s.w),
// so the corrected filter is d = 1/(lambda_s^2 + delta + alpha) (eq.
// TikFilter with the refined eigenvalue).  delta is computed exactly here in
// float64 (two separable passes over the support), either on the image's AR
// grid (the exact correction) or on the model's 33 x 33 grid of [0, pi]^2
// (its training targets).  The model maps 16 (h - s) of a 15 x 15 PSF
// through two ReLU layers of width 256 to the 33 x 33 table of delta, which
// the setup reads by bilinear interpolation on the AR grid.  Training is mean
// squared error with Adam, on float32 SIMT kernels (the model is small; its
// cost is negligible next to one restoration).

#include "ar_internal.cuh"

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace ar {
namespace {

constexpr int CQ = AR_CORR_Q;
constexpr int CK = 2 * CQ + 1;                 // 15
constexpr int CIN = AR_CORR_IN;                // 225
constexpr int CH = AR_CORR_HIDDEN;             // 256
constexpr int CG = AR_CORR_GRID;               // 33
constexpr int COUT = AR_CORR_OUT;              // 1089
constexpr float IN_SCALE = 16.f;

// parameter layout (row-major in x out): W1 b1 W2 b2 W3 b3
constexpr size_t OFF_W1 = 0;
constexpr size_t OFF_B1 = OFF_W1 + (size_t)CIN * CH;
constexpr size_t OFF_W2 = OFF_B1 + CH;
constexpr size_t OFF_B2 = OFF_W2 + (size_t)CH * CH;
constexpr size_t OFF_W3 = OFF_B2 + CH;
constexpr size_t OFF_B3 = OFF_W3 + (size_t)CH * COUT;
constexpr size_t NPARAM = OFF_B3 + COUT;

// ------------------------------------------------------------------ delta --

// a = h - s for a (2q1+1) x (2q2+1) PSF, in shared memory (float64).
__device__ void antisym_smem(const double* __restrict__ h, int q1, int q2, double* a) {
    const int kw = 2 * q2 + 1, n = (2 * q1 + 1) * kw;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int i1 = i / kw - q1, i2 = i % kw - q2;
        const double s = 0.25 * (h[(-i1 + q1) * kw + (-i2 + q2)] + h[(-i1 + q1) * kw + (i2 + q2)] +
                                 h[(i1 + q1) * kw + (-i2 + q2)] + h[(i1 + q1) * kw + (i2 + q2)]);
        a[i] = h[i] - s;
    }
}

// exp(-i s x) with x = k pi / den, reduced exactly: angle / pi = (s k mod 2 den) / den
__device__ __forceinline__ double2 phase(int s, long long k, long long den) {
    long long r = ((long long)s * k) % (2 * den);
    if (r < 0) r += 2 * den;
    double sv, cv;
    sincospi((double)r / (double)den, &sv, &cv);
    return make_double2(cv, -sv);
}

// Model targets: one CTA per PSF (15 x 15), delta on the 33 x 33 grid j pi / 32.
__global__ void corr_target_kernel(const double* __restrict__ psfs, double* __restrict__ out64,
                                   float* __restrict__ out32) {
    __shared__ double a[CIN];
    __shared__ double2 R[CK * CG];              // R[s1][j2] = sum_s2 a[s1][s2] e^{-i s2 x_j2}
    const double* h = psfs + (size_t)blockIdx.x * CIN;
    antisym_smem(h, CQ, CQ, a);
    __syncthreads();
    for (int i = threadIdx.x; i < CK * CG; i += blockDim.x) {
        const int s1 = i / CG, j2 = i % CG;
        double re = 0.0, im = 0.0;
        for (int s2 = -CQ; s2 <= CQ; ++s2) {
            const double2 e = phase(s2, j2, CG - 1);
            const double v = a[s1 * CK + s2 + CQ];
            re += v * e.x;
            im += v * e.y;
        }
        R[i] = make_double2(re, im);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < COUT; i += blockDim.x) {
        const int j1 = i / CG, j2 = i % CG;
        double pr = 0.0, pi = 0.0, mr = 0.0, mi = 0.0;
        for (int s1 = -CQ; s1 <= CQ; ++s1) {
            const double2 r = R[(s1 + CQ) * CG + j2];
            const double2 e = phase(s1, j1, CG - 1);      // e^{-i s1 x1}
            pr += r.x * e.x - r.y * e.y;                   // r e
            pi += r.x * e.y + r.y * e.x;
            mr += r.x * e.x + r.y * e.y;                   // r conj(e) = r e^{+i s1 x1}
            mi += r.y * e.x - r.x * e.y;
        }
        const double d = 0.5 * (pr * pr + pi * pi + mr * mr + mi * mi);
        if (out64) out64[(size_t)blockIdx.x * COUT + i] = d;
        if (out32) out32[(size_t)blockIdx.x * COUT + i] = (float)d;
    }
}

// Model inputs 16 (h - s), one CTA per PSF.
__global__ void corr_input_kernel(const double* __restrict__ psfs, float* __restrict__ X) {
    __shared__ double a[CIN];
    antisym_smem(psfs + (size_t)blockIdx.x * CIN, CQ, CQ, a);
    __syncthreads();
    for (int i = threadIdx.x; i < CIN; i += blockDim.x)
        X[(size_t)blockIdx.x * CIN + i] = (float)(IN_SCALE * a[i]);
}

// Exact delta on the image's AR grid (x = 0 at both ends, k pi / (m - 1)
// inside), any support: row pass R[s1][k2], then delta[k1][k2].
__device__ __forceinline__ long long ar_k(int k, int m) { return (k == 0 || k == m - 1) ? 0 : k; }

// E[k][s + q] = exp(-i s x_k) on the AR grid of size m, s = -q..q.
__global__ void phase_table_kernel(int m, int q, double2* __restrict__ E) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)m * (2 * q + 1)) return;
    const int k = (int)(idx / (2 * q + 1)), s = (int)(idx % (2 * q + 1)) - q;
    E[idx] = phase(s, ar_k(k, m), m - 1);
}

__global__ void delta_rows_kernel(const double* __restrict__ h, int q1, int q2, int n2,
                                  const double2* __restrict__ E2, double2* __restrict__ R) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)(2 * q1 + 1) * n2) return;
    const int s1 = (int)(idx / n2), k2 = (int)(idx % n2);
    const int kw = 2 * q2 + 1;
    double re = 0.0, im = 0.0;
    for (int s2 = -q2; s2 <= q2; ++s2) {
        const int i1 = s1 - q1, i2 = s2;
        const double s = 0.25 * (h[(-i1 + q1) * kw + (-i2 + q2)] + h[(-i1 + q1) * kw + (i2 + q2)] +
                                 h[(i1 + q1) * kw + (-i2 + q2)] + h[(i1 + q1) * kw + (i2 + q2)]);
        const double v = h[s1 * kw + s2 + q2] - s;
        const double2 e = E2[(size_t)k2 * kw + s2 + q2];
        re += v * e.x;
        im += v * e.y;
    }
    R[idx] = make_double2(re, im);
}

__global__ void delta_grid_kernel(const double2* __restrict__ R, int q1, int n1, int n2,
                                  const double2* __restrict__ E1, double* __restrict__ delta) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n1 * n2) return;
    const int k1 = (int)(idx / n2), k2 = (int)(idx % n2);
    double pr = 0.0, pi = 0.0, mr = 0.0, mi = 0.0;
    for (int s1 = -q1; s1 <= q1; ++s1) {
        const double2 r = R[(size_t)(s1 + q1) * n2 + k2];
        const double2 e = E1[(size_t)k1 * (2 * q1 + 1) + s1 + q1];
        pr += r.x * e.x - r.y * e.y;
        pi += r.x * e.y + r.y * e.x;
        mr += r.x * e.x + r.y * e.y;
        mi += r.y * e.x - r.x * e.y;
    }
    delta[idx] = 0.5 * (pr * pr + pi * pi + mr * mr + mi * mi);
}

// Bilinear reading of a 33 x 33 table on the AR grid (entries may be negative:
// the filter clamps lambda^2 + delta at 0).
__global__ void delta_table_kernel(const float* __restrict__ table, int n1, int n2,
                                   double* __restrict__ delta) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n1 * n2) return;
    const int k1 = (int)(idx / n2), k2 = (int)(idx % n2);
    // u = x / pi * (G - 1) with x = ar_k(k) pi / (m - 1)
    const double u1 = (double)ar_k(k1, n1) * (CG - 1) / (double)(n1 - 1);
    const double u2 = (double)ar_k(k2, n2) * (CG - 1) / (double)(n2 - 1);
    int i = (int)floor(u1), j = (int)floor(u2);
    i = i > CG - 2 ? CG - 2 : i;
    j = j > CG - 2 ? CG - 2 : j;
    const double t = u1 - i, w = u2 - j;
    auto T = [&](int r, int c) { return (double)table[r * CG + c]; };
    delta[idx] = (1 - t) * (1 - w) * T(i, j) + (1 - t) * w * T(i, j + 1) + t * (1 - w) * T(i + 1, j) +
                 t * w * T(i + 1, j + 1);
}

// --------------------------------------------------------------- the MLP --

// C[M x N] = op(A) op(B) (+ bias[n]) (ReLU), float32; op(A)[m][k] = TA ? A[k lda + m] : A[m lda + k],
// op(B)[k][n] = TB ? B[n ldb + k] : B[k ldb + n].  64 x 64 tiles, 4 x 4 outputs per thread.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B,
            int ldb, float* __restrict__ C, int ldc, const float* __restrict__ bias, int relu) {
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = threadIdx.x; i < 64 * 16; i += 256) {
            const int kk = i % 16, mm = i / 16;        // A tile element (mm, kk)
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.f;
            if (m < M && k < K) v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
            As[kk][mm] = v;
            const int nn = i % 64, kb = i / 64;         // B tile element (kb, nn)
            const int n = n0 + nn, k2 = k0 + kb;
            float w = 0.f;
            if (n < N && k2 < K) w = TB ? B[(size_t)n * ldb + k2] : B[(size_t)k2 * ldb + n];
            Bs[kb][nn] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int m = m0 + ty * 4 + r;
        if (m >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int n = n0 + tx * 4 + c;
            if (n >= N) continue;
            float v = acc[r][c] + (bias ? bias[n] : 0.f);
            if (relu) v = fmaxf(v, 0.f);
            C[(size_t)m * ldc + n] = v;
        }
    }
}

// dY = 2 (Y - T) / (B * O) in place of Y; *loss += mean (Y - T)^2 (float64).
__global__ void mse_grad_kernel(float* __restrict__ Y, const float* __restrict__ T, size_t n,
                                double* __restrict__ loss) {
    double acc = 0.0;
    const float sc = 2.f / (float)n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        acc += (double)d * d;
        Y[i] = sc * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(loss, acc / (double)n);
}

// dZ = dH * (H > 0) with H the ReLU output, in place of dH.
__global__ void relu_grad_kernel(float* __restrict__ dH, const float* __restrict__ H, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(H[i] > 0.f)) dH[i] = 0.f;
}

// g[n] = sum_m D[m][n] (bias gradients).
__global__ void colsum_kernel(const float* __restrict__ D, int M, int N, float* __restrict__ g) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += D[(size_t)m * N + n];
    g[n] = s;
}

// Adam (Kingma and Ba): c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float c1,
                            float c2, float eps) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

unsigned blocks_for(size_t n, unsigned t = 256) { return (unsigned)((n + t - 1) / t); }

template <bool TA, bool TB>
ar_status gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
               int ldc, const float* bias, bool relu, cudaStream_t s) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    gemm_kernel<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu ? 1 : 0);
    count_launch();
    AR_CUDA(cudaGetLastError());
    return AR_OK;
}

}  // namespace

// Forward pass for a batch of B inputs X (B x 225): H1, H2 (B x 256, after
// the ReLU; H > 0 exactly where the pre-activation is > 0, which is the mask
// of the backward pass) and Y (B x 1089).
struct MlpWork {
    float *H1 = nullptr, *H2 = nullptr, *Y = nullptr;
};

static ar_status mlp_forward(const float* P, const float* X, int B, MlpWork& w, cudaStream_t s) {
    AR_TRY((gemm<false, false>(B, CH, CIN, X, CIN, P + OFF_W1, CH, w.H1, CH, P + OFF_B1, true, s)));
    AR_TRY((gemm<false, false>(B, CH, CH, w.H1, CH, P + OFF_W2, CH, w.H2, CH, P + OFF_B2, true, s)));
    AR_TRY((gemm<false, false>(B, COUT, CH, w.H2, CH, P + OFF_W3, COUT, w.Y, COUT, P + OFF_B3, false,
                              s)));
    return AR_OK;
}

}  // namespace ar

struct ar_corr {
    int device;
    float* P;          // parameters (NPARAM)
    float* M;          // Adam first moments
    float* V;          // Adam second moments
    long long t;       // Adam step count
};

using namespace ar;

namespace ar {

// Exact or table-read delta on the AR grid of an n1 x n2 image, float64, into
// `delta` (n1 n2); `scratch` holds (2 q1 + 1) n2 double2 for the exact form.
ar_status corr_delta(const double* psf_dev64, int q1, int q2, int n1, int n2, const ar_corr* model,
                     const double* psf_host, double* delta, double* scratch, cudaStream_t s) {
    const size_t n = (size_t)n1 * n2;
    if (!model) {
        const size_t nr = (size_t)(2 * q1 + 1) * n2;
        const size_t ne1 = (size_t)n1 * (2 * q1 + 1), ne2 = (size_t)n2 * (2 * q2 + 1);
        double2* R = reinterpret_cast<double2*>(scratch);
        double2* E1 = R + nr;
        double2* E2 = E1 + ne1;
        phase_table_kernel<<<blocks_for(ne1), 256, 0, s>>>(n1, q1, E1);
        phase_table_kernel<<<blocks_for(ne2), 256, 0, s>>>(n2, q2, E2);
        delta_rows_kernel<<<blocks_for(nr), 256, 0, s>>>(psf_dev64, q1, q2, n2, E2, R);
        delta_grid_kernel<<<blocks_for(n), 256, 0, s>>>(R, q1, n1, n2, E1, delta);
        count_launch(4);
        AR_CUDA(cudaGetLastError());
        return AR_OK;
    }
    (void)psf_host;
    // the model's table for this PSF: input, forward pass, bilinear reading
    float* buf = reinterpret_cast<float*>(scratch);
    float* X = buf;                          // 225 (padded to 256)
    MlpWork w;
    w.H1 = X + 256;
    w.H2 = w.H1 + CH;
    w.Y = w.H2 + CH;
    corr_input_kernel<<<1, 256, 0, s>>>(psf_dev64, X);
    count_launch();
    AR_CUDA(cudaGetLastError());
    AR_TRY(mlp_forward(model->P, X, 1, w, s));
    delta_table_kernel<<<blocks_for(n), 256, 0, s>>>(w.Y, n1, n2, delta);
    count_launch();
    AR_CUDA(cudaGetLastError());
    return AR_OK;
}

bool corr_on_current_device(const ar_corr* model) {
    int dev = 0;
    return cudaGetDevice(&dev) == cudaSuccess && dev == model->device;
}

size_t corr_scratch_doubles(int q1, int q2, int n1, int n2) {
    const size_t exact = 2 * ((size_t)(2 * q1 + 1) * n2 + (size_t)n1 * (2 * q1 + 1) +
                              (size_t)n2 * (2 * q2 + 1));
    const size_t model = (256 + 2 * CH + COUT + 1) / 2 + 1;
    return exact > model ? exact : model;
}

}  // namespace ar

extern "C" {

size_t ar_corr_param_count(void) { return NPARAM; }

ar_status ar_corr_create(const float* params_host, ar_corr** out) {
    if (!params_host || !out) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    for (size_t i = 0; i < NPARAM; ++i)
        if (!std::isfinite(params_host[i]))
            return fail(AR_ERR_INVALID_ARG, "parameter %zu is not finite", i);
    ar_corr* M = new (std::nothrow) ar_corr();
    if (!M) return fail(AR_ERR_ALLOC, "host allocation of the model");
    std::memset(M, 0, sizeof(*M));
    cudaGetDevice(&M->device);
    const size_t nb = NPARAM * sizeof(float);
    cudaError_t e = cudaMalloc((void**)&M->P, nb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&M->M, nb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&M->V, nb);
    if (e == cudaSuccess) e = cudaMemcpy(M->P, params_host, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->M, 0, nb);
    if (e == cudaSuccess) e = cudaMemset(M->V, 0, nb);
    if (e != cudaSuccess) {
        ar_corr_destroy(M);
        return cuda_fail(e, "model allocation");
    }
    *out = M;
    return AR_OK;
}

void ar_corr_destroy(ar_corr* M) {
    if (!M) return;
    cudaDeviceSynchronize();
    cudaFree(M->P);
    cudaFree(M->M);
    cudaFree(M->V);
    delete M;
}

ar_status ar_corr_params(const ar_corr* M, float* params_host) {
    if (!M || !params_host) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    if (!corr_on_current_device(M)) return fail(AR_ERR_INVALID_ARG, "model belongs to another device");
    AR_CUDA(cudaDeviceSynchronize());
    AR_CUDA(cudaMemcpy(params_host, M->P, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return AR_OK;
}

static ar_status check_psfs15(const double* psfs, int count) {
    for (size_t i = 0; i < (size_t)count * CIN; ++i)
        if (!std::isfinite(psfs[i])) return fail(AR_ERR_INVALID_ARG, "PSF entry %zu is not finite", i);
    return AR_OK;
}

ar_status ar_corr_targets(const double* psfs_host, int count, double* delta_host) {
    if (!psfs_host || !delta_host || count < 1)
        return fail(AR_ERR_INVALID_ARG, "null pointer or count < 1");
    AR_TRY(check_psfs15(psfs_host, count));
    double *h = nullptr, *d = nullptr;
    cudaError_t e = cudaMalloc((void**)&h, (size_t)count * CIN * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d, (size_t)count * COUT * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpy(h, psfs_host, (size_t)count * CIN * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        corr_target_kernel<<<count, 256>>>(h, d, nullptr);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(delta_host, d, (size_t)count * COUT * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(h);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "correction targets");
    return AR_OK;
}

ar_status ar_corr_predict(const ar_corr* M, const double* psf_host, float* table_host) {
    if (!M || !psf_host || !table_host) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    if (!corr_on_current_device(M)) return fail(AR_ERR_INVALID_ARG, "model belongs to another device");
    AR_TRY(check_psfs15(psf_host, 1));
    double* h = nullptr;
    float* buf = nullptr;
    cudaError_t e = cudaMalloc((void**)&h, CIN * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&buf, (256 + 2 * CH + COUT) * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(h, psf_host, CIN * sizeof(double), cudaMemcpyHostToDevice);
    ar_status st = e == cudaSuccess ? AR_OK : cuda_fail(e, "predict buffers");
    if (st == AR_OK) {
        MlpWork w;
        w.H1 = buf + 256;
        w.H2 = w.H1 + CH;
        w.Y = w.H2 + CH;
        corr_input_kernel<<<1, 256>>>(h, buf);
        count_launch();
        st = cudaGetLastError() == cudaSuccess ? mlp_forward(M->P, buf, 1, w, 0)
                                               : fail(AR_ERR_CUDA, "input kernel");
        if (st == AR_OK) {
            e = cudaMemcpy(table_host, w.Y, COUT * sizeof(float), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = cuda_fail(e, "predict readback");
        }
    }
    cudaFree(h);
    cudaFree(buf);
    return st;
}

}  // extern "C"

// Adam on the model's mean squared error against the closed-form targets
// (tables_host null) or given target tables (count x 33 x 33 float64).
static ar_status corr_train(ar_corr* M, const double* psfs_host, const double* tables_host,
                            int count, int epochs, int batch, double lr, float* loss_trace_host,
                            void* stream) {
    if (!M || !psfs_host) return fail(AR_ERR_INVALID_ARG, "null pointer argument");
    if (!corr_on_current_device(M)) return fail(AR_ERR_INVALID_ARG, "model belongs to another device");
    if (count < 1 || epochs < 0 || batch < 1)
        return fail(AR_ERR_INVALID_ARG, "count %d, epochs %d, batch %d", count, epochs, batch);
    if (!(lr > 0.0) || !std::isfinite(lr))
        return fail(AR_ERR_INVALID_ARG, "learning rate must be finite and > 0");
    AR_TRY(check_psfs15(psfs_host, count));
    if (tables_host)
        for (size_t i = 0; i < (size_t)count * COUT; ++i)
            if (!std::isfinite(tables_host[i]))
                return fail(AR_ERR_INVALID_ARG, "target table entry %zu is not finite", i);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int B = batch < count ? batch : count;
    std::vector<void*> bufs;
    auto get = [&](void** p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) bufs.push_back(*p);
        return e;
    };
    double *h = nullptr, *loss = nullptr;
    float *X = nullptr, *T = nullptr, *G = nullptr, *dH = nullptr;
    MlpWork w;
    cudaError_t e = get((void**)&h, (size_t)count * CIN * sizeof(double));
    if (e == cudaSuccess) e = get((void**)&X, (size_t)count * CIN * sizeof(float));
    if (e == cudaSuccess) e = get((void**)&T, (size_t)count * COUT * sizeof(float));
    if (e == cudaSuccess) e = get((void**)&G, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = get((void**)&w.H1, (size_t)B * CH * sizeof(float));
    if (e == cudaSuccess) e = get((void**)&w.H2, (size_t)B * CH * sizeof(float));
    if (e == cudaSuccess) e = get((void**)&w.Y, (size_t)B * COUT * sizeof(float));
    if (e == cudaSuccess) e = get((void**)&dH, (size_t)B * CH * sizeof(float));
    if (e == cudaSuccess) e = get((void**)&loss, (size_t)(epochs > 0 ? epochs : 1) * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, psfs_host, (size_t)count * CIN * sizeof(double),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(loss, 0, (size_t)(epochs > 0 ? epochs : 1) * sizeof(double), s);
    ar_status st = e == cudaSuccess ? AR_OK : cuda_fail(e, "training buffers");
    std::vector<float> t32;
    if (st == AR_OK && tables_host) {
        t32.resize((size_t)count * COUT);
        for (size_t i = 0; i < t32.size(); ++i) t32[i] = (float)tables_host[i];
        e = cudaMemcpyAsync(T, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) st = cuda_fail(e, "target upload");
    }
    if (st == AR_OK) {
        corr_input_kernel<<<count, 256, 0, s>>>(h, X);
        count_launch();
        if (!tables_host) {
            corr_target_kernel<<<count, 256, 0, s>>>(h, nullptr, T);
            count_launch();
        }
        if (cudaGetLastError() != cudaSuccess) st = fail(AR_ERR_CUDA, "target kernels");
    }
    const int nb = (count + B - 1) / B;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; st == AR_OK && ep < epochs; ++ep) {
        for (int bi = 0; st == AR_OK && bi < nb; ++bi) {
            const int r0 = bi * B, rows = (count - r0) < B ? (count - r0) : B;
            const float* Xb = X + (size_t)r0 * CIN;
            const float* Tb = T + (size_t)r0 * COUT;
            st = mlp_forward(M->P, Xb, rows, w, s);
            if (st != AR_OK) break;
            const size_t ny = (size_t)rows * COUT;
            mse_grad_kernel<<<blocks_for(ny) < 1024 ? blocks_for(ny) : 1024, 256, 0, s>>>(
                w.Y, Tb, ny, loss + ep);                         // w.Y := dY
            count_launch();
            // layer 3: dW3 = H2^T dY, db3 = colsum dY, dH2 = dY W3^T
            st = gemm<true, false>(CH, COUT, rows, w.H2, CH, w.Y, COUT, G + OFF_W3, COUT, nullptr,
                                   false, s);
            if (st == AR_OK) {
                colsum_kernel<<<blocks_for(COUT), 256, 0, s>>>(w.Y, rows, COUT, G + OFF_B3);
                count_launch();
                st = gemm<false, true>(rows, CH, COUT, w.Y, COUT, M->P + OFF_W3, COUT, dH, CH,
                                       nullptr, false, s);
            }
            // layer 2
            if (st == AR_OK) {
                relu_grad_kernel<<<blocks_for((size_t)rows * CH), 256, 0, s>>>(dH, w.H2,
                                                                                 (size_t)rows * CH);
                count_launch();
                st = gemm<true, false>(CH, CH, rows, w.H1, CH, dH, CH, G + OFF_W2, CH, nullptr,
                                       false, s);
            }
            if (st == AR_OK) {
                colsum_kernel<<<blocks_for(CH), 256, 0, s>>>(dH, rows, CH, G + OFF_B2);
                count_launch();
                // dH1 = dZ2 W2^T (into H2, no longer needed)
                st = gemm<false, true>(rows, CH, CH, dH, CH, M->P + OFF_W2, CH, w.H2, CH, nullptr,
                                       false, s);
            }
            // layer 1
            if (st == AR_OK) {
                relu_grad_kernel<<<blocks_for((size_t)rows * CH), 256, 0, s>>>(w.H2, w.H1,
                                                                                 (size_t)rows * CH);
                count_launch();
                st = gemm<true, false>(CIN, CH, rows, Xb, CIN, w.H2, CH, G + OFF_W1, CH, nullptr,
                                       false, s);
            }
            if (st == AR_OK) {
                colsum_kernel<<<blocks_for(CH), 256, 0, s>>>(w.H2, rows, CH, G + OFF_B1);
                count_launch();
                M->t += 1;
                const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)M->t)));
                const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)M->t)));
                adam_kernel<<<blocks_for(NPARAM), 256, 0, s>>>(M->P, G, M->M, M->V, NPARAM,
                                                               (float)lr, b1, b2, c1, c2, 1e-8f);
                count_launch();
                if (cudaGetLastError() != cudaSuccess) st = fail(AR_ERR_CUDA, "training kernels");
            }
        }
    }
    std::vector<double> lh((size_t)(epochs > 0 ? epochs : 1), 0.0);
    if (st == AR_OK) {
        e = cudaMemcpyAsync(lh.data(), loss, lh.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "training");
    } else {
        cudaStreamSynchronize(s);
    }
    for (void* p : bufs) cudaFree(p);
    if (st != AR_OK) return st;
    if (loss_trace_host)
        for (int ep = 0; ep < epochs; ++ep) loss_trace_host[ep] = (float)(lh[ep] / nb);
    return AR_OK;
}

extern "C" {

ar_status ar_corr_train(ar_corr* M, const double* psfs_host, int count, int epochs, int batch,
                        double lr, float* loss_trace_host, void* stream) {
    return corr_train(M, psfs_host, nullptr, count, epochs, batch, lr, loss_trace_host, stream);
}

ar_status ar_corr_train_tables(ar_corr* M, const double* psfs_host, const double* tables_host,
                               int count, int epochs, int batch, double lr,
                               float* loss_trace_host, void* stream) {
    if (!tables_host) return fail(AR_ERR_INVALID_ARG, "null pointer argument (tables)");
    return corr_train(M, psfs_host, tables_host, count, epochs, batch, lr, loss_trace_host,
                      stream);
}

}  // extern "C"
