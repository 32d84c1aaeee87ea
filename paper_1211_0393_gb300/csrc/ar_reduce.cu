// Float64-accumulated reductions over float32 images: the relative
// restoration error ||x - f||_F / ||f||_F of Section 4 and a non-finite scan.
// Warp shuffles, one shared-memory stage per block, one atomic per block.

#include "ar_internal.cuh"

namespace ar {
namespace {

constexpr int RB = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_add(double v, double* acc) {
    __shared__ double part[RB / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < RB / 32 ? part[threadIdx.x] : 0.0;
        w = warp_sum(w);
        if (threadIdx.x == 0) atomicAdd(acc, w);
    }
}

__global__ void __launch_bounds__(RB) diff_sq_kernel(const float* __restrict__ x,
                                                     const float* __restrict__ f, size_t n,
                                                     double* acc) {
    double v = 0.0;
    for (size_t i = (size_t)blockIdx.x * RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB) {
        const double d = (double)x[i] - (double)(f ? __ldg(f + i) : 0.f);
        v = fma(d, d, v);
    }
    block_add(v, acc);
}

__global__ void __launch_bounds__(RB) nonfinite_kernel(const float* __restrict__ x, size_t n,
                                                       unsigned long long* cnt) {
    unsigned c = 0;
    for (size_t i = (size_t)blockIdx.x * RB + threadIdx.x; i < n; i += (size_t)gridDim.x * RB)
        c += isfinite(x[i]) ? 0u : 1u;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, (unsigned long long)c);
}

unsigned grid_for(size_t n) {
    size_t b = (n + RB - 1) / RB;
    const size_t cap = (size_t)sm_count() * 8;
    return (unsigned)(b < cap ? (b ? b : 1) : cap);
}

}  // namespace

ar_status reduce_diff_sq(const float* x, const float* f, size_t n, double* acc, cudaStream_t s) {
    ProfScope prof(AR_PROF_OTHER, s);
    diff_sq_kernel<<<grid_for(n), RB, 0, s>>>(x, f, n, acc);
    count_launch();
    AR_CUDA(cudaGetLastError());
    return AR_OK;
}

ar_status reduce_sq(const float* f, size_t n, double* acc, cudaStream_t s) {
    ProfScope prof(AR_PROF_OTHER, s);
    diff_sq_kernel<<<grid_for(n), RB, 0, s>>>(f, nullptr, n, acc);
    count_launch();
    AR_CUDA(cudaGetLastError());
    return AR_OK;
}

ar_status count_nonfinite(const float* x, size_t n, unsigned long long* cnt, cudaStream_t s) {
    ProfScope prof(AR_PROF_OTHER, s);
    nonfinite_kernel<<<grid_for(n), RB, 0, s>>>(x, n, cnt);
    count_launch();
    AR_CUDA(cudaGetLastError());
    return AR_OK;
}

}  // namespace ar
