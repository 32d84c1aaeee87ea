// FFT-style AR transform pair: D y = T diag(d) T~ y with every one-dimensional
// transform of Theorem 1 applied through a fast sine transform instead of a
// dense product.
//
// Along an axis of length m (M = m - 2 interior samples, N = m - 1), without
// the normalisation alpha_m (it cancels between T and T~):
//   analysis  T~': y^_0 = y_0, y^_{m-1} = y_{m-1},
//                  y^_mid = Q_M (y_mid - p y_0 - J p y_{m-1}),
//   synthesis T' : y_0 = w_0, y_{m-1} = w_{m-1},
//                  y_mid = Q_M w_mid + p w_0 + J p w_{m-1},
// with p_t = 1 - t/(m-1), (J p)_t = t/(m-1) (t = 1..M), and Q_M the orthonormal
// DST-I, Q[s][t] = sqrt(2/N) sin(pi s t / N), symmetric (eq. Qn).
//
// S_s = sum_t v_t sin(pi s t / N) (s = 1..M) is computed from one real DFT of
// length N of
//   a_0 = 0,  a_j = sin(j pi / N) (v_j + v_{N-j}) + (v_j - v_{N-j}) / 2,
// whose coefficients A_k = sum_j a_j e^{-2 pi i j k / N} give
//   S_{2k} = -Im A_k,   S_1 = Re A_0 / 2,   S_{2k+1} = S_{2k-1} + Re A_k
// (N odd, so the even s reach M = N - 1 and the odd ones M - 1).  The DFT is
// split by Good and Thomas: with N = N1 N2, gcd(N1, N2) = 1, the input
// a_{(N2 n1 + N1 n2) mod N} on an N1 x N2 grid, an N2-point DFT along n2 and an
// N1-point DFT along n1 give A_k at (k mod N1, k mod N2), with no twiddle
// factors between the two passes.  Both passes are direct sums (small dense
// DFTs) in float32 from shared memory, taken of a_j less their mean (A_0 itself
// is summed in float64); the prefix sum of the odd coefficients runs in float64,
// and for odd N its end value, which S_N = 0 makes pure rounding, is removed as
// a linear bridge.  m = 2048 takes N = 2047 = 23 x 89.
//
// A 2D application is four row passes and two transposes: analysis along the
// rows (axis 2), transpose, analysis along axis 1 with the filter d fused,
// synthesis along axis 1, transpose, synthesis along the rows with the
// output (store, or x += tau * with the RRE sum) fused.

#include "ar_internal.cuh"

#include <cmath>
#include <new>

namespace ar {
namespace {

constexpr int FST_THREADS = 256;
constexpr int FST_MAXN = 256;          // largest factor (smem twiddle tables)

int gcd_int(int a, int b) {
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

int inv_mod(int a, int m) {            // a^-1 mod m (gcd(a, m) = 1, m >= 1)
    if (m == 1) return 0;
    for (int x = 1; x < m; ++x)
        if ((long long)a * x % m == 1) return x;
    return 0;
}

}  // namespace

struct FstFactor {
    int m, N, N1, N2;
    int r1, r2;                        // n1 = j r1 mod N1, n2 = j r2 mod N2 (input map)
};

// N = m - 1 as N1 N2, coprime, N1 <= N2 <= FST_MAXN, the most balanced such pair.
bool fst_factor(int m, FstFactor* out) {
    if (m < 4) return false;
    const int N = m - 1;
    int best = -1;
    for (int a = 1; a * a <= N; ++a) {
        if (N % a) continue;
        const int b = N / a;
        if (b > FST_MAXN || gcd_int(a, b) != 1) continue;
        best = a;
    }
    if (best < 0) return false;
    out->m = m;
    out->N = N;
    out->N1 = best;
    out->N2 = N / best;
    out->r1 = inv_mod(out->N2 % out->N1 == 0 ? 0 : out->N2 % out->N1, out->N1);
    out->r2 = inv_mod(out->N1 % out->N2, out->N2);
    return true;
}

namespace {

enum FstMode : int { FST_ANALYSIS = 0, FST_ANALYSIS_SCALE = 1, FST_SYNTHESIS = 2,
                     FST_SYNTHESIS_AXPY = 3 };

struct FstArgs {
    const float* in;       // rows x m, row-major
    float* out;            // rows x m (FST_SYNTHESIS_AXPY: x, updated in place)
    int rows;
    FstFactor f;
    int mode;
    const float* filt;     // FST_ANALYSIS_SCALE: d at filt[col * rows + row] (transposed layout)
    float tau;             // FST_SYNTHESIS_AXPY
    const float* ftrue;    // FST_SYNTHESIS_AXPY: true image (same layout) or null
    double* sumsq;         // += sum (x_new - f)^2
};

// Shared memory of one row, each part 16-byte aligned: the row (m floats), the
// N1 x N2 grid (N floats), the half spectrum of the first pass (N1 x K2h
// float2), A_k (H + 1 float2), the odd prefix (H + 1 doubles), the twiddle
// tables (N1 + N2 float2).
struct FstSmem {
    size_t row, X, Z, A, P, tw, total;
    __host__ __device__ FstSmem(const FstFactor& f) {
        const int K2h = (f.N2 + 1) / 2, H = (f.N - 1) / 2;
        auto a16 = [](size_t b) { return (b + 15) & ~size_t(15); };
        row = 0;
        X = a16(row + (size_t)f.m * 4);
        Z = a16(X + (size_t)f.N * 4);
        A = a16(Z + (size_t)f.N1 * K2h * 8);
        P = a16(A + (size_t)(H + 1) * 8);
        tw = a16(P + (size_t)(H + 1) * 8);
        total = a16(tw + (size_t)(f.N1 + f.N2) * 8);
    }
    static size_t bytes(const FstFactor& f) { return FstSmem(f).total; }
};

__global__ void __launch_bounds__(FST_THREADS)
fst_rows_kernel(const FstArgs a) {
    extern __shared__ __align__(16) unsigned char fst_smem[];
    const FstFactor f = a.f;
    const int m = f.m, N = f.N, N1 = f.N1, N2 = f.N2;
    const int K2h = (N2 + 1) / 2, H = (N - 1) / 2, M = m - 2;
    const FstSmem L(f);
    float* row = reinterpret_cast<float*>(fst_smem + L.row);          // m
    float* X = reinterpret_cast<float*>(fst_smem + L.X);              // N1 x N2
    float2* Z = reinterpret_cast<float2*>(fst_smem + L.Z);            // N1 x K2h
    float2* A = reinterpret_cast<float2*>(fst_smem + L.A);            // H + 1
    double* P = reinterpret_cast<double*>(fst_smem + L.P);            // H + 1 (odd prefix)
    float2* tw1 = reinterpret_cast<float2*>(fst_smem + L.tw);         // N1: (cos, sin)(2 pi r / N1)
    float2* tw2 = tw1 + N1;                                           // N2
    const int tid = threadIdx.x;
    __shared__ double red[FST_THREADS / 32];
    for (int r = tid; r < N1; r += FST_THREADS) {
        double sv, cv;
        sincospi(2.0 * r / N1, &sv, &cv);
        tw1[r] = make_float2((float)cv, (float)sv);
    }
    for (int r = tid; r < N2; r += FST_THREADS) {
        double sv, cv;
        sincospi(2.0 * r / N2, &sv, &cv);
        tw2[r] = make_float2((float)cv, (float)sv);
    }
    const float c = (float)sqrt(2.0 / N);
    const float inv = 1.0f / (float)(m - 1);
    double sq = 0.0;
    for (int rw = blockIdx.x; rw < a.rows; rw += gridDim.x) {
        __syncthreads();                                  // previous row done with smem
        const float* src = a.in + (size_t)rw * m;
        for (int t = tid; t < m; t += FST_THREADS) row[t] = __ldg(src + t);
        __syncthreads();
        const bool analysis = a.mode == FST_ANALYSIS || a.mode == FST_ANALYSIS_SCALE;
        const float y0 = row[0], ym = row[m - 1];
        // v_t (t = 1..M): the interior with, for the analysis, the linear part removed
        auto v = [&](int t) -> float {
            if (t < 1 || t > M) return 0.f;
            const float x = row[t];
            if (!analysis) return x;
            const float p = 1.0f - (float)t * inv;
            return x - p * y0 - ((float)t * inv) * ym;
        };
        // a_j on the Good-Thomas grid: j -> (j r1 mod N1, j r2 mod N2); their sum
        // A_0 in float64, and the DFT taken of a_j - A_0 / N (the same A_k, k > 0, with
        // partial sums free of the mean)
        double asum = 0.0;
        for (int j = tid; j < N; j += FST_THREADS) {
            float aj = 0.f;
            if (j > 0) {
                const float vj = v(j), vn = v(N - j);
                aj = sinpif((float)j / (float)N) * (vj + vn) + 0.5f * (vj - vn);
            }
            const int n1 = (int)(((long long)j * f.r1) % N1), n2 = (int)(((long long)j * f.r2) % N2);
            X[n1 * N2 + n2] = aj;
            asum += (double)aj;
        }
        for (int o = 16; o > 0; o >>= 1) asum += __shfl_down_sync(0xffffffffu, asum, o);
        if ((tid & 31) == 0) red[tid >> 5] = asum;
        __syncthreads();
        double A0 = 0.0;
        for (int w = 0; w < FST_THREADS / 32; ++w) A0 += red[w];
        const float mean = (float)(A0 / N);
        for (int j = tid; j < N; j += FST_THREADS) {
            const int n1 = (int)(((long long)j * f.r1) % N1), n2 = (int)(((long long)j * f.r2) % N2);
            X[n1 * N2 + n2] -= mean;
        }
        __syncthreads();
        // pass 1: Z[n1][k2] = sum_n2 X[n1][n2] e^{-2 pi i n2 k2 / N2}, k2 <= N2/2 (real input)
        for (int o = tid; o < N1 * K2h; o += FST_THREADS) {
            const int n1 = o / K2h, k2 = o % K2h;
            const float* xr = X + n1 * N2;
            float re = 0.f, im = 0.f;
            int r = 0;
            for (int n2 = 0; n2 < N2; ++n2) {
                const float x = xr[n2];
                const float2 w = tw2[r];
                re = fmaf(x, w.x, re);
                im = fmaf(-x, w.y, im);
                r += k2;
                if (r >= N2) r -= N2;
            }
            Z[o] = make_float2(re, im);
        }
        __syncthreads();
        // pass 2: A_k = sum_n1 Z[n1][k mod N2] e^{-2 pi i n1 (k mod N1) / N1}, k = 0..H
        for (int k = tid; k <= H; k += FST_THREADS) {
            const int k1 = k % N1, k2 = k % N2;
            const bool conj = k2 >= K2h;
            const int kk = conj ? N2 - k2 : k2;
            float re = 0.f, im = 0.f;
            int r = 0;
            for (int n1 = 0; n1 < N1; ++n1) {
                float2 z = Z[n1 * K2h + kk];
                if (conj) z.y = -z.y;
                const float2 w = tw1[r];                 // e^{-i th} = (cos, -sin)
                re = fmaf(z.x, w.x, fmaf(z.y, w.y, re));
                im = fmaf(z.y, w.x, fmaf(-z.x, w.y, im));
                r += k1;
                if (r >= N1) r -= N1;
            }
            A[k] = make_float2(re, im);
            P[k] = k == 0 ? 0.5 * A0 : (double)re;
        }
        __syncthreads();
        // inclusive prefix of P over k = 0..H (float64): S_{2k+1} = P_0 + .. + P_k
        if (tid < 32) {
            double carry = 0.0;
            for (int base = 0; base <= H; base += 32) {
                const int k = base + tid;
                double val = k <= H ? P[k] : 0.0;
                for (int d = 1; d < 32; d <<= 1) {
                    const double up = __shfl_up_sync(0xffffffffu, val, d);
                    if (tid >= d) val += up;
                }
                val += carry;
                if (k <= H) P[k] = val;
                carry = __shfl_sync(0xffffffffu, val, 31);
            }
        }
        __syncthreads();
        // N odd: S_N = sum_t v_t sin(pi t) = 0 ends the odd recurrence, so the prefix's
        // end value is its accumulated rounding: removed as a linear bridge
        const double PH = (N & 1) ? P[H] : 0.0;
        // outputs
        float* dst = a.out + (size_t)rw * m;
        float part = 0.f;
        for (int t = tid; t < m; t += FST_THREADS) {
            float val;
            if (t == 0 || t == m - 1) {
                val = row[t];
            } else {
                const int k = t >> 1;
                const float S = (t & 1) ? (float)(P[k] - (double)(k + 1) / (double)(H + 1) * PH)
                                        : -A[k].y;
                val = c * S;
                if (!analysis) {
                    const float p = 1.0f - (float)t * inv;
                    val += p * y0 + ((float)t * inv) * ym;
                }
            }
            if (a.mode == FST_ANALYSIS_SCALE) val *= __ldg(a.filt + (size_t)t * a.rows + rw);
            if (a.mode == FST_SYNTHESIS_AXPY) {
                const float xn = fmaf(a.tau, val, dst[t]);
                dst[t] = xn;
                if (a.ftrue) {
                    const float e = xn - __ldg(a.ftrue + (size_t)rw * m + t);
                    part = fmaf(e, e, part);
                }
            } else {
                dst[t] = val;
            }
        }
        sq += part;
    }
    if (a.sumsq) {
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < FST_THREADS / 32; ++w) t += red[w];
            if (t != 0.0) atomicAdd(a.sumsq, t);
        }
    }
}

// out (cols x rows) = in (rows x cols)^T, 32 x 32 tiles.
__global__ void transpose_kernel(const float* __restrict__ in, float* __restrict__ out, int rows,
                                 int cols) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = __ldg(in + (size_t)r * cols + c);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[threadIdx.x][i];
    }
}

}  // namespace

struct FstPlan {
    int n1, n2;
    FstFactor f1, f2;
    float* in = nullptr;       // n1 x n2: the transform input (the reblur writes it)
    float* u = nullptr;        // n1 x n2
    float* ut = nullptr;       // n2 x n1
    int grid1 = 0, grid2 = 0;  // persistent row grids of the two axes
};

bool fst_supported(int n1, int n2) {
    FstFactor a, b;
    return fst_factor(n1, &a) && fst_factor(n2, &b);
}

void fst_plan_destroy(FstPlan* p) {
    if (!p) return;
    cudaFree(p->in);
    cudaFree(p->u);
    cudaFree(p->ut);
    delete p;
}

static ar_status fst_attr(size_t smem) {
    static size_t set = 0;
    if (smem > set) {
        AR_CUDA(cudaFuncSetAttribute(fst_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        set = smem;
    }
    return AR_OK;
}

ar_status fst_plan_create(int n1, int n2, cudaStream_t s, FstPlan** out) {
    FstPlan* p = new (std::nothrow) FstPlan();
    if (!p) return fail(AR_ERR_ALLOC, "host allocation of the FFT-style plan");
    p->n1 = n1;
    p->n2 = n2;
    if (!fst_factor(n1, &p->f1) || !fst_factor(n2, &p->f2)) {
        delete p;
        return fail(AR_ERR_UNSUPPORTED,
                    "FFT-style transform: n_j - 1 must split into coprime factors <= %d (n = %d x %d)",
                    FST_MAXN, n1, n2);
    }
    const size_t nb = (size_t)n1 * n2 * sizeof(float);
    cudaError_t e = dev_malloc_async((void**)&p->in, nb, s);
    if (e == cudaSuccess) e = dev_malloc_async((void**)&p->u, nb, s);
    if (e == cudaSuccess) e = dev_malloc_async((void**)&p->ut, nb, s);
    if (e != cudaSuccess) {
        fst_plan_destroy(p);
        return cuda_fail(e, "FFT-style plan buffers");
    }
    const size_t smem = FstSmem::bytes(p->f1) > FstSmem::bytes(p->f2) ? FstSmem::bytes(p->f1)
                                                                      : FstSmem::bytes(p->f2);
    ar_status st = fst_attr(smem);
    if (st != AR_OK) {
        fst_plan_destroy(p);
        return st;
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fst_rows_kernel, FST_THREADS, smem);
    if (per_sm < 1) per_sm = 1;
    const int cap = per_sm * sm_count();
    p->grid1 = n1 < cap ? n1 : cap;        // rows of axis 2 (n1 rows of length n2)
    p->grid2 = n2 < cap ? n2 : cap;        // rows of axis 1 (n2 rows of length n1)
    *out = p;
    return AR_OK;
}

float* fst_input(FstPlan* p) { return p->in; }

static ar_status fst_rows(const FstArgs& a, int grid, cudaStream_t s) {
    count_launch();
    fst_rows_kernel<<<grid, FST_THREADS, FstSmem::bytes(a.f), s>>>(a);
    AR_CUDA(cudaGetLastError());
    return AR_OK;
}

static ar_status fst_transpose(const float* in, float* out, int rows, int cols, cudaStream_t s) {
    count_launch();
    transpose_kernel<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, s>>>(in, out, rows,
                                                                                     cols);
    AR_CUDA(cudaGetLastError());
    return AR_OK;
}

ar_status fst_apply(FstPlan* p, const float* d32, const float* y, float* out, bool axpy, float tau,
                    cudaStream_t s, const float* f, double* sumsq) {
    ProfScope prof(AR_PROF_CONTRACTION, s, 6);
    const int n1 = p->n1, n2 = p->n2;
    const float* src = y ? y : p->in;
    FstArgs a{};
    // analysis along the rows (axis 2): u = y T~2'^T
    a.in = src;
    a.out = p->u;
    a.rows = n1;
    a.f = p->f2;
    a.mode = FST_ANALYSIS;
    AR_TRY(fst_rows(a, p->grid1, s));
    AR_TRY(fst_transpose(p->u, p->ut, n1, n2, s));
    // analysis along axis 1 with the filter (ut is n2 x n1: d[s1][s2] at (row s2, col s1))
    a.in = p->ut;
    a.out = p->ut;
    a.rows = n2;
    a.f = p->f1;
    a.mode = FST_ANALYSIS_SCALE;
    a.filt = d32;
    AR_TRY(fst_rows(a, p->grid2, s));
    // synthesis along axis 1
    a.mode = FST_SYNTHESIS;
    a.filt = nullptr;
    AR_TRY(fst_rows(a, p->grid2, s));
    AR_TRY(fst_transpose(p->ut, p->u, n2, n1, s));
    // synthesis along the rows, into out (stored, or x += tau * with the RRE sum)
    a.in = p->u;
    a.out = out;
    a.rows = n1;
    a.f = p->f2;
    a.mode = axpy ? FST_SYNTHESIS_AXPY : FST_SYNTHESIS;
    a.tau = tau;
    a.ftrue = axpy ? f : nullptr;
    a.sumsq = axpy ? sumsq : nullptr;
    AR_TRY(fst_rows(a, p->grid1, s));
    return AR_OK;
}

}  // namespace ar
