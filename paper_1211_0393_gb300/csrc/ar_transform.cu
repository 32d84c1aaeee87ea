// The AR transform pair of Theorem 1 applied as dense contractions.
//
// D y = T_n diag(d) T~_n y with T_n = T_{n1} (x) T_{n2} becomes, for an image Y,
//     D Y = T_{n1} ( d o (T~_{n1} Y T~_{n2}^T) ) T_{n2}^T,
// four dense products.  The transforms are used without the normalisation
// alpha_m of Theorem 1 (it cancels between T and T~):
//     T~'_m = [[1, 0, 0], [-Q p, Q, -Q J p], [0, 0, 1]]
//     T'_m  = [[1, 0, 0], [  p,  Q,    J p], [0, 0, 1]]
// with Q = Q_{m-2} of eq. Qn and p_j = 1 - j/(m-1).  Both are generated in
// float64 on the GPU.
//
// Every product is C = A B^T with both operands row-major ("K-major"), and is
// stored transposed, so the chain needs no explicit transposes:
//   G1: U^T  <- (Y  T~2^T)^T          A = Y   (n1 x n2),  B = T~2
//   G2: W    <- d o (U^T T~1^T)^T     A = U^T (n2 x n1),  B = T~1
//   G3: V^T  <- (W  T2^T)^T           A = W,              B = T2
//   G4: out  <- (V^T T1^T)^T (or out += tau * ...)
// This file holds the plan, the float64 matrix generator and a plain SIMT
// float32 contraction.

#include "ar_internal.cuh"

#include <cuda_bf16.h>
#include <cstdlib>
#include <new>

namespace ar {
namespace {

// ---------------------------------------------------------------- matrices --
__device__ __forceinline__ double q_entry(int s, int t, int m) {
    // Q_{m-2}[s, t] = sqrt(2/(m-1)) sin(s t pi/(m-1)), s, t = 1..m-2
    const long long per = 2LL * (m - 1);
    const long long r = ((long long)s * t) % per;
    return sqrt(2.0 / (double)(m - 1)) * sinpi((double)r / (double)(m - 1));
}

// qp[s] = (Q p)_s, qjp[s] = (Q J p)_s, s = 1..m-2 (index s-1), one block per row.
__global__ void boundary_columns_kernel(int m, double* qp, double* qjp) {
    const int s = blockIdx.x + 1;
    double a = 0.0, b = 0.0;
    for (int t = 1 + threadIdx.x; t <= m - 2; t += blockDim.x) {
        const double q = q_entry(s, t, m);
        const double pt = 1.0 - (double)t / (double)(m - 1);
        a += q * pt;
        b += q * (1.0 - pt);          // (J p)_t = p_{m-1-t} = t/(m-1)
    }
    __shared__ double ra[256], rb[256];
    ra[threadIdx.x] = a;
    rb[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            ra[threadIdx.x] += ra[threadIdx.x + w];
            rb[threadIdx.x] += rb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        qp[s - 1] = ra[0];
        qjp[s - 1] = rb[0];
    }
}

// Fills T~'_m (analysis) and T'_m (synthesis) as float32 row-major m x m.
__global__ void fill_transforms_f32_kernel(int m, const double* qp, const double* qjp,
                                           float* Tt, float* T) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)m * m) return;
    const int s = (int)(idx / m), t = (int)(idx % m);
    double vt, v;
    if (s == 0 || s == m - 1) {
        vt = v = (t == s) ? 1.0 : 0.0;
    } else if (t == 0) {
        vt = -qp[s - 1];
        v = 1.0 - (double)s / (double)(m - 1);
    } else if (t == m - 1) {
        vt = -qjp[s - 1];
        v = (double)s / (double)(m - 1);
    } else {
        vt = v = q_entry(s, t, m);
    }
    Tt[idx] = (float)vt;
    T[idx] = (float)v;
}

// ----------------------------------------------------- SIMT contraction --
enum Epi : int { EPI_T = 0, EPI_T_SCALE = 1, EPI_T_AXPY = 2 };

constexpr int BM = 64, BN = 64, BK = 16;

// C(i, j) = sum_k A[i, k] B[j, k]; stored transposed at out[j * ldc + i].
template <int EPI>
__global__ void __launch_bounds__(256)
gemm_nt_simt_kernel(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                    int M, int N, int K, float* __restrict__ out, int ldc,
                    const float* __restrict__ dscale, float tau) {
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tid = threadIdx.x;
    const int ti = tid % 16, tj = tid / 16;
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 256) {
            const int r = e / BK, k = e % BK;
            const int gi = i0 + r, gk = k0 + k;
            As[k][r] = (gi < M && gk < K) ? __ldg(A + (size_t)gi * lda + gk) : 0.f;
            const int gj = j0 + r;
            Bs[k][r] = (gj < N && gk < K) ? __ldg(B + (size_t)gj * ldb + gk) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[k][ti * 4 + u];
                b[u] = Bs[k][tj * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int j = j0 + tj * 4 + v;
        if (j >= N) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + ti * 4 + u;
            if (i >= M) continue;
            const size_t o = (size_t)j * ldc + i;
            if (EPI == EPI_T) out[o] = acc[u][v];
            else if (EPI == EPI_T_SCALE) out[o] = __ldg(dscale + o) * acc[u][v];
            else out[o] = fmaf(tau, acc[u][v], out[o]);
        }
    }
}

template <int EPI>
cudaError_t gemm_simt(const float* A, int lda, const float* B, int ldb, int M, int N, int K,
                      float* out, int ldc, const float* d, float tau, cudaStream_t s) {
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
    gemm_nt_simt_kernel<EPI><<<grid, 256, 0, s>>>(A, lda, B, ldb, M, N, K, out, ldc, d, tau);
    count_launch();
    return cudaGetLastError();
}

ar_status make_transforms(int m, float** Tt, float** T, cudaStream_t stream) {
    const size_t mm = (size_t)m * m;
    double* tmp = nullptr;
    AR_CUDA(cudaMallocAsync((void**)Tt, mm * sizeof(float), stream));
    AR_CUDA(cudaMallocAsync((void**)T, mm * sizeof(float), stream));
    AR_CUDA(cudaMallocAsync((void**)&tmp, 2 * (size_t)m * sizeof(double), stream));
    if (m > 2) {
        boundary_columns_kernel<<<m - 2, 256, 0, stream>>>(m, tmp, tmp + m);
        count_launch();
        AR_CUDA(cudaGetLastError());
    }
    fill_transforms_f32_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, stream>>>(m, tmp, tmp + m,
                                                                                *Tt, *T);
    count_launch();
    AR_CUDA(cudaGetLastError());
    AR_CUDA(cudaFreeAsync(tmp, stream));
    return AR_OK;
}

}  // namespace

struct TransformPlan {
    int n1, n2;
    float* Tt1 = nullptr;
    float* T1 = nullptr;
    float* Tt2 = nullptr;
    float* T2 = nullptr;
    float* bufA = nullptr;
    float* bufB = nullptr;
};

ar_status transform_plan_create(int n1, int n2, cudaStream_t stream, TransformPlan** out) {
    TransformPlan* p = new (std::nothrow) TransformPlan();
    if (!p) return fail(AR_ERR_ALLOC, "host allocation of the transform plan");
    p->n1 = n1;
    p->n2 = n2;
    ar_status st = make_transforms(n1, &p->Tt1, &p->T1, stream);
    if (st == AR_OK) {
        if (n2 == n1) {
            p->Tt2 = p->Tt1;
            p->T2 = p->T1;
        } else {
            st = make_transforms(n2, &p->Tt2, &p->T2, stream);
        }
    }
    const size_t n = (size_t)n1 * n2;
    if (st == AR_OK && cudaMallocAsync((void**)&p->bufA, n * sizeof(float), stream) != cudaSuccess)
        st = fail(AR_ERR_ALLOC, "transform scratch");
    if (st == AR_OK && cudaMallocAsync((void**)&p->bufB, n * sizeof(float), stream) != cudaSuccess)
        st = fail(AR_ERR_ALLOC, "transform scratch");
    if (st != AR_OK) {
        transform_plan_destroy(p);
        return st;
    }
    *out = p;
    return AR_OK;
}

void transform_plan_destroy(TransformPlan* p) {
    if (!p) return;
    if (p->Tt2 && p->Tt2 != p->Tt1) cudaFree(p->Tt2);
    if (p->T2 && p->T2 != p->T1) cudaFree(p->T2);
    cudaFree(p->Tt1);
    cudaFree(p->T1);
    cudaFree(p->bufA);
    cudaFree(p->bufB);
    delete p;
}

uint16_t* transform_input_planes(TransformPlan*, size_t* plane_stride, int* ld) {
    if (plane_stride) *plane_stride = 0;
    if (ld) *ld = 0;
    return nullptr;
}

int transform_launches(const TransformPlan*, DInput) { return 4; }

ar_status transform_apply(TransformPlan* p, const float* d32, const float* y, DInput din,
                          float* out, DOutput dout, float tau, cudaStream_t s) {
    if (din != DIN_FP32) return fail(AR_ERR_UNSUPPORTED, "split operand input not built");
    const int n1 = p->n1, n2 = p->n2;
    cudaError_t e;
    e = gemm_simt<EPI_T>(y, n2, p->Tt2, n2, n1, n2, n2, p->bufA, n1, nullptr, 0.f, s);
    if (e != cudaSuccess) return cuda_fail(e, "transform G1");
    e = gemm_simt<EPI_T_SCALE>(p->bufA, n1, p->Tt1, n1, n2, n1, n1, p->bufB, n2, d32, 0.f, s);
    if (e != cudaSuccess) return cuda_fail(e, "transform G2");
    e = gemm_simt<EPI_T>(p->bufB, n2, p->T2, n2, n1, n2, n2, p->bufA, n1, nullptr, 0.f, s);
    if (e != cudaSuccess) return cuda_fail(e, "transform G3");
    if (dout == DOUT_STORE)
        e = gemm_simt<EPI_T>(p->bufA, n1, p->T1, n1, n2, n1, n1, out, n2, nullptr, 0.f, s);
    else
        e = gemm_simt<EPI_T_AXPY>(p->bufA, n1, p->T1, n1, n2, n1, n1, out, n2, nullptr, tau, s);
    if (e != cudaSuccess) return cuda_fail(e, "transform G4");
    return AR_OK;
}

}  // namespace ar
