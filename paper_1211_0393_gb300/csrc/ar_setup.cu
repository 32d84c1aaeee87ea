// FP64 eigenvalue setup of the optimal preconditioners, on the GPU.
//
// AR (the method) and Reflective (comparison BC):
//  S0  s = symmetrized PSF (eq. simmetrizzata2d, Theorem 4):
//        s_{+-i1,+-i2} = (h_{-i1,-i2} + h_{-i1,i2} + h_{i1,-i2} + h_{i1,i2}) / 4
//  S1  lambda[i1,i2] = f_s(x1_{i1}, x2_{i2}), the generating function of eq.
//      funzione_generatrice, on the grid of the BC.  AR (Theorem 2, in T_n's
//      column order): x_k = 0 for k = 0 and k = m-1 (the anti-reflection
//      centres) and x_k = k pi/(m-1) for k = 1..m-2 (the tau grid of
//      Q_{m-2}).  Reflective (Section 2.1, DCT-III): x_k = k pi/m, k = 0..m-1.
//      f is separable, f = sum_a cos(a x1) t_a(x2) with
//      t_a(x2) = w_a (s_{a,0} + 2 sum_{b>=1} s_{a,b} cos(b x2)), w_0 = 1, w_a = 2,
//      which regroups the four sums of the equation.
//  S2  d = 1/(lambda^2 + alpha), eq. TikFilter (with a spectral correction
//      delta when one is given: d = 1/(max(lambda^2 + delta, 0) + alpha)).
//
// Periodic (comparison BC): lambda = |sum_s h_s exp(-i s . w)| at
// w = 2 pi k / m, the eigenvalue magnitudes of the circulant of the PSF itself,
// summed as a row pass (b) then a column pass (a); d as in S2.  d is then
// split into the part even in each frequency, d_e = (d(k1,k2) + d(-k1,k2))/2,
// and the part odd in both, d_o = (d(k1,k2) - d(-k1,k2))/2 (d(-k) = d(k) for
// a real PSF), which the separable Hartley form of the circulant solve takes.
//
// All arithmetic is float64.  Trigonometric arguments are reduced exactly in
// integers first: cos(a k pi/(m-1)) = cospi(((a k) mod 2(m-1)) / (m-1)) and
// likewise for the other grids.

#include "ar_internal.cuh"

namespace ar {
namespace {

__device__ __forceinline__ double grid_cos(int a, int k, int m, int bc) {
    if (bc == AR_BC_REFLECTIVE) {     // cos(a k pi / m)
        const long long r = ((long long)a * k) % (2LL * m);
        return cospi((double)r / (double)m);
    }
    // cos(a * x_k) on the AR grid of size m
    if (k == 0 || k == m - 1) return 1.0;
    const long long per = 2LL * (m - 1);
    const long long r = ((long long)a * k) % per;
    return cospi((double)r / (double)(m - 1));
}

// exp(-i 2 pi j / m) for an integer j (any sign), reduced exactly.
__device__ __forceinline__ double2 unit_root(long long j, int m) {
    long long r = j % m;
    if (r < 0) r += m;
    double sv, cv;
    sincospi(2.0 * (double)r / (double)m, &sv, &cv);
    return make_double2(cv, -sv);
}

// scratch layout: s[(q1+1)*(q2+1)] | t[(q1+1) * n2] | c1[(q1+1) * n1]
__global__ void symmetrize_kernel(const double* __restrict__ h, int q1, int q2, double* s) {
    const int kw = 2 * q2 + 1;
    for (int i = threadIdx.x; i < (q1 + 1) * (q2 + 1); i += blockDim.x) {
        const int a = i / (q2 + 1), b = i % (q2 + 1);
        const double v = h[(q1 - a) * kw + (q2 - b)] + h[(q1 - a) * kw + (q2 + b)]
                       + h[(q1 + a) * kw + (q2 - b)] + h[(q1 + a) * kw + (q2 + b)];
        s[i] = 0.25 * v;
    }
}

// t[a][j] = w_a (s_{a,0} + 2 sum_{b>=1} s_{a,b} cos(b x2_j)),  c1[a][i] = cos(a x1_i)
__global__ void symbol_tables_kernel(const double* __restrict__ s, int q1, int q2, int n1, int n2,
                                     int bc, double* __restrict__ t, double* __restrict__ c1) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int nt = (q1 + 1) * n2;
    if (idx < nt) {
        const int a = idx / n2, j = idx % n2;
        double acc = 0.0;
        for (int b = q2; b >= 1; --b) acc += s[a * (q2 + 1) + b] * grid_cos(b, j, n2, bc);
        acc = s[a * (q2 + 1)] + 2.0 * acc;
        t[idx] = (a == 0 ? 1.0 : 2.0) * acc;
    } else if (idx < nt + (q1 + 1) * n1) {
        const int k = idx - nt;
        const int a = k / n1, i = k % n1;
        c1[k] = grid_cos(a, i, n1, bc);
    }
}

__global__ void eigen_kernel(const double* __restrict__ t, const double* __restrict__ c1,
                             int q1, int n1, int n2, double alpha,
                             double* __restrict__ lam64, double* __restrict__ d64,
                             float* __restrict__ d32, const double* __restrict__ delta) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n1 * n2) return;
    const int i = (int)(idx / n2), j = (int)(idx % n2);
    double lam = 0.0;
    for (int a = q1; a >= 0; --a) lam += c1[(size_t)a * n1 + i] * t[(size_t)a * n2 + j];
    const double d = 1.0 / (fmax(lam * lam + (delta ? delta[idx] : 0.0), 0.0) + alpha);
    if (lam64) lam64[idx] = lam;
    if (d64) d64[idx] = d;
    d32[idx] = (float)d;
}

// Periodic row pass: pr[a + q1][k2] = sum_b h_{a,b} exp(-i b 2 pi k2 / n2).
__global__ void periodic_rows_kernel(const double* __restrict__ h, int q1, int q2, int n2,
                                     double2* __restrict__ pr) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)(2 * q1 + 1) * n2) return;
    const int ai = (int)(idx / n2), k2 = (int)(idx % n2);
    const double* row = h + (size_t)ai * (2 * q2 + 1);
    double re = 0.0, im = 0.0;
    for (int b = -q2; b <= q2; ++b) {
        const double2 e = unit_root((long long)b * k2, n2);
        const double v = row[b + q2];
        re += v * e.x;
        im += v * e.y;
    }
    pr[idx] = make_double2(re, im);
}

// Periodic column pass: lambda(k1, k2) = |sum_a pr[a][k2] exp(-i a 2 pi k1 / n1)|
// and d = 1/(lambda^2 + alpha) (float64, into dfull).
__global__ void periodic_eigen_kernel(const double2* __restrict__ pr, int q1, int n1, int n2,
                                      double alpha, double* __restrict__ lam64,
                                      double* __restrict__ dfull) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n1 * n2) return;
    const int k1 = (int)(idx / n2), k2 = (int)(idx % n2);
    double re = 0.0, im = 0.0;
    for (int a = -q1; a <= q1; ++a) {
        const double2 p = pr[(size_t)(a + q1) * n2 + k2];
        const double2 e = unit_root((long long)a * k1, n1);
        re += p.x * e.x - p.y * e.y;
        im += p.x * e.y + p.y * e.x;
    }
    const double lam = hypot(re, im);
    if (lam64) lam64[idx] = lam;
    dfull[idx] = 1.0 / (lam * lam + alpha);
}

// d32 = (d(k1,k2) + d(-k1,k2)) / 2, d32_odd = -(d(k1,k2) - d(-k1,k2)) / 2.
__global__ void periodic_split_kernel(const double* __restrict__ dfull, int n1, int n2,
                                      float* __restrict__ d32, float* __restrict__ d32_odd) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n1 * n2) return;
    const int k1 = (int)(idx / n2), k2 = (int)(idx % n2);
    const double d = dfull[idx];
    const double dm = dfull[(size_t)((n1 - k1) % n1) * n2 + k2];
    d32[idx] = (float)(0.5 * (d + dm));
    d32_odd[idx] = (float)(-0.5 * (d - dm));
}

}  // namespace

size_t setup_scratch_doubles(int q1, int q2, int n1, int n2, int bc) {
    if (bc == AR_BC_PERIODIC) return 2 * (size_t)(2 * q1 + 1) * n2 + (size_t)n1 * n2;
    return (size_t)(q1 + 1) * (q2 + 1) + (size_t)(q1 + 1) * n2 + (size_t)(q1 + 1) * n1;
}

ar_status setup_eigen(const double* psf_dev64, int q1, int q2, int n1, int n2, double alpha,
                      int bc, double* lam64, double* d64, float* d32, float* d32_odd,
                      double* scratch, cudaStream_t stream, const double* delta_dev) {
    const size_t n = (size_t)n1 * n2;
    if (bc == AR_BC_PERIODIC) {
        double2* pr = reinterpret_cast<double2*>(scratch);
        double* dfull = d64 ? d64 : scratch + 2 * (size_t)(2 * q1 + 1) * n2;
        ProfScope prof(AR_PROF_SETUP, stream);
        const size_t nr = (size_t)(2 * q1 + 1) * n2;
        periodic_rows_kernel<<<(unsigned)((nr + 255) / 256), 256, 0, stream>>>(psf_dev64, q1, q2,
                                                                               n2, pr);
        count_launch();
        AR_CUDA(cudaGetLastError());
        periodic_eigen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(pr, q1, n1, n2,
                                                                               alpha, lam64, dfull);
        count_launch();
        AR_CUDA(cudaGetLastError());
        periodic_split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(dfull, n1, n2, d32,
                                                                               d32_odd);
        count_launch();
        AR_CUDA(cudaGetLastError());
        return AR_OK;
    }
    double* s = scratch;
    double* t = s + (size_t)(q1 + 1) * (q2 + 1);
    double* c1 = t + (size_t)(q1 + 1) * n2;
    ProfScope prof(AR_PROF_SETUP, stream);
    symmetrize_kernel<<<1, 256, 0, stream>>>(psf_dev64, q1, q2, s);
    count_launch();
    AR_CUDA(cudaGetLastError());
    const int ntab = (q1 + 1) * (n2 + n1);
    symbol_tables_kernel<<<(ntab + 255) / 256, 256, 0, stream>>>(s, q1, q2, n1, n2, bc, t, c1);
    count_launch();
    AR_CUDA(cudaGetLastError());
    eigen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(t, c1, q1, n1, n2, alpha,
                                                                  lam64, d64, d32, delta_dev);
    count_launch();
    AR_CUDA(cudaGetLastError());
    return AR_OK;
}

}  // namespace ar
