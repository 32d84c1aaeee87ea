// Fused anti-reflective extension + 2D convolution (y = A_n x and y = A' x).
// The same kernels serve the comparison boundary conditions: reflective
// (Section 2.1) and periodic extensions are plain index maps.
//
// A_n x is the convolution g_i = sum_s h_s xt_{i-s} (eq. modello_discreto) of
// the image extended by the anti-reflective rules of Section 2.2: along each
// axis xt_{-i} = 2 x_0 - x_i and xt_{n-1+i} = 2 x_{n-1} - x_{n-1-i}; applying
// the row rule and then the column rule gives the double anti-reflection
// 4 x_c - 2 x - 2 x + x at the corners.  A' (Section 4, reblurring) is the same
// operator with the PSF rotated by 180 degrees.
//
// The extension is never materialised: every CTA brings its halo tile into
// shared memory (by TMA, double-buffered in a persistent loop over tiles,
// when the image rows are 16-byte aligned; otherwise by the threads,
// all loads of a thread in flight at once) and, on tiles that reach past the
// image, overwrites the out-of-image samples with their anti-reflections
// computed from in-tile samples.  Each thread then computes a vertical strip of
// R outputs of one column (R = 16 or 18, by the tile geometry), sliding a
// register window down the tile: per PSF column it loads R + 2Q values from
// shared memory (consecutive lanes read consecutive columns: conflict-free)
// and issues R (2Q+1) FMAs against broadcast PSF coefficients.  The kernel is
// FP32-FMA bound for Q >= 2.

#include "ar_internal.cuh"
#include "ar_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

namespace ar {
namespace {

constexpr int TX = 64;   // tile columns, one per thread
// Tile geometries: TY row strips of RS rows, a TH = TY RS row tile per CTA (per
// half-CTA in the folding reblur).  G64 (8 warps, 64-row tiles) serves every
// launch but the single-wave ones that G54 (6 warps, 54-row tiles) balances
// better (the choice depends on the image size only, so that a batch and a
// single restoration of the same image give identical results): a 1024-row image splits into 19 tiles of 54 rows, and the 304 tiles
// of a 1024^2 image give every SM two where 256 tiles of 64 rows give 104 SMs
// two and 48 SMs one (the folding reblur: 152 units instead of 128).
template <int TY_, int RS_>
struct Geo {
    static constexpr int TY = TY_, RS = RS_, TH = TY_ * RS_;
};
using G64 = Geo<4, 16>;
using G54 = Geo<3, 18>;
constexpr int QMAX_FAST = 15;

// Index of the sample that an out-of-image index j maps to under the
// reflective (f_{1-i} = f_i, f_{n+i} = f_{n+1-i}, Section 2.1) or periodic
// extension; in-image indices map to themselves.  Valid for -n <= j < 2n.
__device__ __forceinline__ int mirror_index(int j, int n, int bc) {
    if (j >= 0 && j < n) return j;
    if (bc == AR_BC_REFLECTIVE) return j < 0 ? -j - 1 : 2 * n - 1 - j;
    return j < 0 ? j + n : j - n;                           // periodic
}

// Sample of the anti-reflectively extended image at (j1, j2) (0-based; may
// lie outside the image by up to q).  Outside the extended domain the value
// only feeds outputs that are never stored, so 0 is returned without reading.
__device__ __forceinline__ float ext_value(const float* __restrict__ x, int n1, int n2,
                                           int q1, int q2, int j1, int j2, int bc) {
    if (j1 < -q1 || j1 >= n1 + q1 || j2 < -q2 || j2 >= n2 + q2) return 0.f;
    if (bc != AR_BC_ANTIREFLECTIVE)
        return __ldg(x + (size_t)mirror_index(j1, n1, bc) * n2 + mirror_index(j2, n2, bc));
    const bool r_in = (j1 >= 0 && j1 < n1);
    const bool c_in = (j2 >= 0 && j2 < n2);
    // row terms: edge row re (weight 2) and mirror row rm (weight -1)
    const int re = j1 < 0 ? 0 : n1 - 1;
    const int rm = j1 < 0 ? -j1 : 2 * (n1 - 1) - j1;
    const int ce = j2 < 0 ? 0 : n2 - 1;
    const int cm = j2 < 0 ? -j2 : 2 * (n2 - 1) - j2;
    if (r_in && c_in) return __ldg(x + (size_t)j1 * n2 + j2);
    if (c_in) {  // top/bottom border: rows are extended first
        return 2.f * __ldg(x + (size_t)re * n2 + j2) - __ldg(x + (size_t)rm * n2 + j2);
    }
    if (r_in) {  // left/right border
        const float* row = x + (size_t)j1 * n2;
        return 2.f * __ldg(row + ce) - __ldg(row + cm);
    }
    // corner: extend the two rows re, rm along the columns, then combine them
    const float* xe = x + (size_t)re * n2;
    const float* xm = x + (size_t)rm * n2;
    const float ve = 2.f * __ldg(xe + ce) - __ldg(xe + cm);
    const float vm = 2.f * __ldg(xm + ce) - __ldg(xm + cm);
    return 2.f * ve - vm;
}

__device__ __forceinline__ void split3_store(uint16_t* planes, size_t pstride, size_t off, float v) {
    const __nv_bfloat16 p0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(p0);
    const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(p1);
    const __nv_bfloat16 p2 = __float2bfloat16_rn(r2);
    planes[off] = __bfloat16_as_ushort(p0);
    planes[pstride + off] = __bfloat16_as_ushort(p1);
    planes[2 * pstride + off] = __bfloat16_as_ushort(p2);
}

// Writes one output; returns (x_new - f)^2 for CONV_AXPY with a true image, r^2
// for CONV_RESIDUAL when the residual norm is accumulated (sumsq set), else 0.
__device__ __forceinline__ float conv_epilogue(const ConvArgs& a, int row, int col, float v) {
    const size_t o = (size_t)row * a.n2 + col;
    switch (a.mode) {
        case CONV_STORE: a.out[o] = v; break;
        case CONV_RESIDUAL: {
            const float r = __ldg(a.aux + o) - v;
            a.out[o] = r;
            if (a.sumsq) return r * r;
            break;
        }
        case CONV_AXPY: {
            const float xn = fmaf(a.tau, v, a.out[o]);
            a.out[o] = xn;
            if (a.f) {
                const float e = xn - __ldg(a.f + o);
                return e * e;
            }
            break;
        }
        default: split3_store(a.planes, a.plane_stride, (size_t)row * a.ld + col, v); break;
    }
    return 0.f;
}

// *sumsq += the block's sum of v (one float64 atomic per block).  Each thread's
// v is a float32 sum of at most RS squares (relative error ~RS 2^-24, RS <= 18); the
// block reduction is float64.  Called by every thread of the block.
__device__ __forceinline__ void add_sumsq(double* sumsq, float vf) {
    __shared__ double part[32];
    double v = vf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0) part[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (nthreads + 31) / 32; ++w) t += part[w];
        if (t != 0.0) atomicAdd(sumsq, t);
    }
    __syncthreads();                     // part[] is reused by the next tile
}

// Coefficient rows are padded to a multiple of 4 so that a PSF column is
// read with 16-byte shared-memory loads.
template <int Q>
struct Coefs {
    static constexpr int K = 2 * Q + 1;
    static constexpr int KP = (K + 3) & ~3;
    static constexpr int COUNT = K * KP;
};

// Coefficients of the support padded to Q x Q: coef[b * KP + a] = h_{a-Q, b-Q}
// (h_{Q-a, Q-b} for A'), zero outside the true support and in the row padding.
template <int Q>
__device__ __forceinline__ void load_coefs(const ConvArgs& a, float* coef, int tid, int nthreads) {
    constexpr int KP = Coefs<Q>::KP;
    const int kw = 2 * a.q2 + 1;
    for (int i = tid; i < Coefs<Q>::COUNT; i += nthreads) {
        const int b = i / KP, aa = i % KP;
        const int s1 = aa - Q, s2 = b - Q;      // tap offsets in the padded support
        float v = 0.f;
        if (aa < 2 * Q + 1 && s1 >= -a.q1 && s1 <= a.q1 && s2 >= -a.q2 && s2 <= a.q2) {
            const int t1 = a.flip ? -s1 : s1, t2 = a.flip ? -s2 : s2;
            v = __ldg(a.psf + (t1 + a.q1) * kw + (t2 + a.q2));
        }
        coef[i] = v;
    }
}

// Out-of-image samples of a halo tile that reaches past the image, from the
// in-image samples of the same tile: tile(r, c) = tile[r * WP + c] holds the
// image sample (r0 - Q + r, c0 - Q + c).  Rows first (on in-image columns),
// then columns on every row of the extended domain, which gives the corner
// rules.  AR (Section 2.2): 2 x_edge - x_mirror; Reflective (Section 2.1):
// x_{-1-i} = x_i, x_{n+i} = x_{n-1-i}.  Edge and mirror samples lie in the
// tile.  Only the out-of-image strips (at most q rows or columns per side) are
// visited.
// Block barrier of a stencil: __syncthreads (BAR = 0) or named barrier BAR
// over `nthreads` threads (the tensor-core kernel's compute warps).
template <int BAR>
__device__ __forceinline__ void stencil_sync(int nthreads) {
    if (BAR == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"n"(BAR), "r"(nthreads) : "memory");
}

template <int Q, class G, int BAR = 0>
__device__ void fixup_tile(const ConvArgs& a, float* tile, int WP, int r0, int c0, int tid,
                           int nthreads) {
    constexpr int W = TX + 2 * Q, H = G::TH + 2 * Q;
    const bool ar = a.bc == AR_BC_ANTIREFLECTIVE;
    const int rb = r0 - Q, cb = c0 - Q;                 // image coordinates of tile (0, 0)
    // tile rows with j1 in [-q1, 0) and in [n1, n1 + q1), clipped to the tile
    const int t0 = max(0, -a.q1 - rb), t1 = min(H, -rb);
    const int b0 = max(0, a.n1 - rb), b1 = min(H, a.n1 + a.q1 - rb);
    const int nt = max(0, t1 - t0), nbot = max(0, b1 - b0);
    // in-image columns of the tile
    const int ci0 = max(0, -cb), ci1 = min(W, a.n2 - cb), nci = max(0, ci1 - ci0);
    for (int i = tid; i < (nt + nbot) * nci; i += nthreads) {
        const int k = i / nci, c = ci0 + i % nci;
        const int r = k < nt ? t0 + k : b0 + (k - nt);
        const int j1 = rb + r;
        int re, rm;
        if (j1 < 0) { re = 0; rm = ar ? -j1 : -j1 - 1; }
        else { re = a.n1 - 1; rm = ar ? 2 * (a.n1 - 1) - j1 : 2 * a.n1 - 1 - j1; }
        const float vm = tile[(rm - rb) * WP + c];
        tile[r * WP + c] = ar ? 2.f * tile[(re - rb) * WP + c] - vm : vm;
    }
    stencil_sync<BAR>(nthreads);
    // tile columns with j2 in [-q2, 0) and [n2, n2 + q2), on rows of the extended domain
    const int l0 = max(0, -a.q2 - cb), l1 = min(W, -cb);
    const int g0 = max(0, a.n2 - cb), g1 = min(W, a.n2 + a.q2 - cb);
    const int nl = max(0, l1 - l0), ng = max(0, g1 - g0);
    const int re0 = max(0, -a.q1 - rb), re1 = min(H, a.n1 + a.q1 - rb), nr = max(0, re1 - re0);
    for (int i = tid; i < (nl + ng) * nr; i += nthreads) {
        const int k = i / nr, r = re0 + i % nr;
        const int c = k < nl ? l0 + k : g0 + (k - nl);
        const int j2 = cb + c;
        int ce, cm;
        if (j2 < 0) { ce = 0; cm = ar ? -j2 : -j2 - 1; }
        else { ce = a.n2 - 1; cm = ar ? 2 * (a.n2 - 1) - j2 : 2 * a.n2 - 1 - j2; }
        const float vm = tile[r * WP + (cm - cb)];
        tile[r * WP + c] = ar ? 2.f * tile[r * WP + (ce - cb)] - vm : vm;
    }
    stencil_sync<BAR>(nthreads);
}

// Each thread computes a vertical strip of RS outputs of one column from the
// halo tile (row pitch WP) and applies the epilogue.
template <int Q, class G>
__device__ __forceinline__ void tile_acc(const float* tile, int WP, const float* coef, int tx,
                                         int ty, float (&acc)[G::RS]) {
    constexpr int K = 2 * Q + 1, RS = G::RS;
#pragma unroll
    for (int r = 0; r < RS; ++r) acc[r] = 0.f;

#pragma unroll 1
    for (int b = 0; b < K; ++b) {
        // output column tx reads tile column tx - s2 + Q = tx + 2Q - b
        const float* col = tile + (ty * RS) * WP + tx + 2 * Q - b;
        float win[RS + 2 * Q];
#pragma unroll
        for (int t = 0; t < RS + 2 * Q; ++t) win[t] = col[t * WP];
        float hc[Coefs<Q>::KP];
        const float4* cb = reinterpret_cast<const float4*>(coef + b * Coefs<Q>::KP);
#pragma unroll
        for (int j = 0; j < Coefs<Q>::KP / 4; ++j) {
            const float4 v = cb[j];
            hc[4 * j] = v.x;
            hc[4 * j + 1] = v.y;
            hc[4 * j + 2] = v.z;
            hc[4 * j + 3] = v.w;
        }
#pragma unroll
        for (int aa = 0; aa < K; ++aa) {
            const float hv = hc[aa];
            // output row r reads tile row r - s1 + Q = r + 2Q - aa (strip-relative)
#pragma unroll
            for (int r = 0; r < RS; ++r) acc[r] = fmaf(hv, win[r + 2 * Q - aa], acc[r]);
        }
    }
}

// RW: the mode reads global memory in its epilogue (residual, AXPY); the
// kernels are instantiated for both kinds, so that the store modes keep their
// own (smaller) register allocation.
template <int Q, bool RW, class G>
__device__ __forceinline__ void compute_tile(const ConvArgs& a, const float* tile, int WP,
                                             const float* coef, int r0, int c0) {
    constexpr int RS = G::RS;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int col = c0 + tx, row0 = r0 + ty * RS;
    const bool live = col < a.n2 && row0 < a.n1;
    if (RW) {
        // the epilogue's inputs (g for the residual; x and f for the update) are
        // read before the tap loop, so that their latency hides behind the FMAs
        const int nr = min(RS, a.n1 - row0);
        const bool res = a.mode == CONV_RESIDUAL;
        float pv[RS], fv[RS];
#pragma unroll
        for (int r = 0; r < RS; ++r) {
            const size_t o = (size_t)(row0 + r) * a.n2 + col;
            const bool in = live && r < nr;
            pv[r] = in ? (res ? __ldg(a.aux + o) : a.out[o]) : 0.f;
            fv[r] = in && !res && a.f ? __ldg(a.f + o) : 0.f;
        }
        float acc[RS];
        tile_acc<Q, G>(tile, WP, coef, tx, ty, acc);
        float sq = 0.f;
        if (live) {
#pragma unroll
            for (int r = 0; r < RS; ++r) {
                if (r >= nr) continue;
                const size_t o = (size_t)(row0 + r) * a.n2 + col;
                if (res) {
                    const float rv = pv[r] - acc[r];
                    a.out[o] = rv;
                    if (a.sumsq) sq += rv * rv;      // ||g - A x||^2 when requested
                } else {
                    const float xn = fmaf(a.tau, acc[r], pv[r]);
                    a.out[o] = xn;
                    if (a.f) {
                        const float e = xn - fv[r];
                        sq += e * e;
                    }
                }
            }
        }
        if (a.sumsq) add_sumsq(a.sumsq, sq);
        return;
    }
    float acc[RS];
    tile_acc<Q, G>(tile, WP, coef, tx, ty, acc);
    float sq = 0.f;
    if (live) {
#pragma unroll
        for (int r = 0; r < RS; ++r)
            if (row0 + r < a.n1) sq += conv_epilogue(a, row0 + r, col, acc[r]);
    }
    if (a.sumsq) add_sumsq(a.sumsq, sq);
}

// Fast path: support padded to Q x Q (Q = max(q1, q2) <= 15, zero taps outside
// the true support), 64 x 64 tiles (geometry G64), 16 rows per thread; the halo
// tile is loaded by the threads (any row pitch and alignment, every BC).
template <int Q, bool RW>
__global__ void __launch_bounds__(TX * G64::TY)
conv_fast_kernel(const ConvArgs a) {
    using G = G64;
    constexpr int TY = G::TY, TH = G::TH;
    constexpr int W = TX + 2 * Q;        // tile row length
    constexpr int H = TH + 2 * Q;        // tile rows
    __shared__ float tile[H * W];
    __shared__ __align__(16) float coef[Coefs<Q>::COUNT];   // see load_coefs

    const int tid = threadIdx.y * TX + threadIdx.x;
    const int r0 = blockIdx.y * TH;
    const int c0 = blockIdx.x * TX;

    pdl_wait();                          // the input image comes from the previous kernel
    load_coefs<Q>(a, coef, tid, TX * TY);
    // Phase 1: every tile sample at its coordinate clamped into the image
    // (reflective / periodic samples at their mapped coordinate).  All loads
    // of a thread are issued before the first shared-memory store.
    constexpr int NLD = (H * W + TX * TY - 1) / (TX * TY);
    {
        float v[NLD];
#pragma unroll
        for (int k = 0; k < NLD; ++k) {
            const int i = tid + k * TX * TY;
            v[k] = 0.f;
            if (i < H * W) {
                const int r = i / W, c = i % W;
                int j1 = r0 - Q + r, j2 = c0 - Q + c;
                if (a.bc != AR_BC_ANTIREFLECTIVE && j1 >= -a.q1 && j1 < a.n1 + a.q1 &&
                    j2 >= -a.q2 && j2 < a.n2 + a.q2) {
                    j1 = mirror_index(j1, a.n1, a.bc);      // reflective / periodic sample
                    j2 = mirror_index(j2, a.n2, a.bc);
                } else {
                    j1 = min(max(j1, 0), a.n1 - 1);
                    j2 = min(max(j2, 0), a.n2 - 1);
                }
                v[k] = __ldg(a.x + (size_t)j1 * a.n2 + j2);
            }
        }
#pragma unroll
        for (int k = 0; k < NLD; ++k) {
            const int i = tid + k * TX * TY;
            if (i < H * W) tile[i] = v[k];
        }
    }
    __syncthreads();
    // Phase 2 (AR tiles that reach past the image only): the anti-reflected samples.
    if (a.bc == AR_BC_ANTIREFLECTIVE &&
        (r0 - Q < 0 || r0 + TH + Q > a.n1 || c0 - Q < 0 || c0 + TX + Q > a.n2))
        fixup_tile<Q, G>(a, tile, W, r0, c0, tid, TX * TY);

    pdl_trigger();
    compute_tile<Q, RW, G>(a, tile, W, coef, r0, c0);
}

__device__ int g_conv_timeout;
// Polls of a stencil's wait for its halo tile before it gives up (settable
// from the host for failure-detection tests; the drain of copies still in
// flight after a give-up always waits the full tc::kMaxPolls).
__device__ uint32_t g_conv_wait_polls = tc::kMaxPolls;

// Halo tile of the TMA path: the box starts PADL >= Q columns left of the
// tile (a multiple of 4, so the box's x coordinate is 16-byte aligned) and
// is WB = TX + 2 PADL wide, HB = TH + 2Q high.  Two boxes per CTA: one in
// use, one in flight (a third was faster on 4096^2 images alone but cost
// resident CTAs and time inside the restoration loop).
template <int Q, class G>
struct TmaTile {
    static constexpr int PADL = (Q + 3) & ~3;
    static constexpr int WB = TX + 2 * PADL;
    static constexpr int HB = G::TH + 2 * Q;
    static constexpr uint32_t BYTES = (uint32_t)WB * HB * 4;
    static constexpr uint32_t BUF = (BYTES + 127u) & ~127u;   // buffers start 128-byte aligned
    static constexpr int NBUF = 2;
    static constexpr size_t SMEM = NBUF * (size_t)BUF + (size_t)Coefs<Q>::COUNT * 4 + 8 * NBUF + 128;
};

// Persistent TMA path (AR and Reflective, 16-byte aligned rows): each CTA
// walks the tiles t = blockIdx.x + i gridDim.x; thread 0 keeps the halo boxes
// of the next NBUF - 1 tiles requested by TMA (zeros outside the image) while
// the CTA works on the current one.  Out-of-image samples of the extended
// domain are then filled in shared memory.
template <int Q, bool RW, class G>
__global__ void __launch_bounds__(TX * G::TY)
conv_tma_kernel(const __grid_constant__ CUtensorMap tmx, const ConvArgs a, int ntx, int ntiles) {
    using namespace tc;
    using T = TmaTile<Q, G>;
    constexpr int TY = G::TY, TH = G::TH;
    constexpr int WB = T::WB, NBUF = T::NBUF;
    extern __shared__ __align__(128) uint8_t smem_raw_c[];
    // TMA destinations: 128-byte aligned (the allocation has 128 bytes of slack)
    uint8_t* sbase = smem_raw_c + ((128u - (smem_u32(smem_raw_c) & 127u)) & 127u);
    float* coef = reinterpret_cast<float*>(sbase + NBUF * T::BUF);
    const uint32_t bar0 = smem_u32(coef + Coefs<Q>::COUNT);   // NBUF mbarriers, 8 bytes apart
    const int tid = threadIdx.y * TX + threadIdx.x;
    auto buffer = [&](int i) { return reinterpret_cast<float*>(sbase + i * T::BUF); };

    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) mbar_init(bar0 + 8u * i, 1);
        fence_mbar_init();
        prefetch_tmap(&tmx);
    }
    load_coefs<Q>(a, coef, tid, TX * TY);
    __syncthreads();
    pdl_wait();                          // the input image comes from the previous kernel

    // local tile i of this CTA is t = blockIdx.x + i gridDim.x, in buffer i % NBUF
    auto request = [&](int i) {
        const int t = blockIdx.x + i * gridDim.x;
        const int r0 = (t / ntx) * TH, c0 = (t % ntx) * TX;
        const uint32_t bar = bar0 + 8u * (i % NBUF);
        fence_proxy_async_smem();        // generic writes to the buffer (fix-up) before the async copy
        mbar_arrive_expect_tx(bar, T::BYTES);
        tma_load_2d(smem_u32(buffer(i % NBUF)), &tmx, c0 - T::PADL, r0 - Q, bar);
    };
    const int nmine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t polls = g_conv_wait_polls;
    if (tid == 0)
        for (int i = 0; i < NBUF - 1 && i < nmine; ++i) request(i);
    int li = 0;
    bool failed = false;
    for (; li < nmine; ++li) {
        if (tid == 0 && li + NBUF - 1 < nmine) request(li + NBUF - 1);   // buffer of tile li-1
        const bool ok = mbar_wait(bar0 + 8u * (li % NBUF), (li / NBUF) & 1, polls);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const int t = blockIdx.x + li * gridDim.x;
        const int r0 = (t / ntx) * TH, c0 = (t % ntx) * TX;
        float* tile = buffer(li % NBUF) + (T::PADL - Q);
        if (r0 - Q < 0 || r0 + TH + Q > a.n1 || c0 - Q < 0 || c0 + TX + Q > a.n2)
            fixup_tile<Q, G>(a, tile, WB, r0, c0, tid, TX * TY);
        if (a.early_trigger && li == nmine - 1) pdl_trigger();
        compute_tile<Q, RW, G>(a, tile, WB, coef, r0, c0);
        __syncthreads();                 // the buffer is refilled for tile li + NBUF
    }
    if (!a.early_trigger) pdl_trigger();
    if (failed && tid == 0) {
        atomicExch(&g_conv_timeout, 1);
        // copies possibly still in flight (tiles li .. li + NBUF - 1): wait for
        // them (bounded) before the CTA's shared memory is released
        for (int i = li; i < li + NBUF && i < nmine; ++i)
            mbar_wait(bar0 + 8u * (i % NBUF), (i / NBUF) & 1);
    }
}

// Folding reblur (CONV_SPLIT3 with fold, AR and Reflective, TMA path): each
// work unit is a tile at columns [c0, c0 + 64) and its mirror at
// [n2 - c0 - 64, n2 - c0), computed side by side by the two 256-thread halves
// of the CTA.  Column c0 + j of the first pairs with column n2 - 1 - c0 - j,
// which is column 63 - j of the mirror tile; the halves swap their results
// through their (consumed) halo boxes and write the bf16x3 split of y+ (first
// half) and y- (second half) for t = c0 + j, zeros past ceil(n2/2) resp.
// floor(n2/2).
template <int Q, class G>
struct FoldTile {
    using T = TmaTile<Q, G>;
    static_assert(T::BYTES >= (uint32_t)G::TH * TX * 4, "a box holds a tile of results");
    static constexpr size_t SMEM = 2 * T::NBUF * (size_t)T::BUF + (size_t)Coefs<Q>::COUNT * 4 +
                                   8 * T::NBUF + 128;
};

template <int Q, class G>
__global__ void __launch_bounds__(2 * TX * G::TY)
conv_tma_fold_kernel(const __grid_constant__ CUtensorMap tmx, const ConvArgs a, int ncp,
                     int nunits) {
    using namespace tc;
    using T = TmaTile<Q, G>;
    constexpr int TY = G::TY, TH = G::TH, RS = G::RS;
    constexpr int WB = T::WB, NBUF = T::NBUF;
    extern __shared__ __align__(128) uint8_t smem_raw_c[];
    uint8_t* sbase = smem_raw_c + ((128u - (smem_u32(smem_raw_c) & 127u)) & 127u);
    float* coef = reinterpret_cast<float*>(sbase + 2 * NBUF * T::BUF);
    const uint32_t bar0 = smem_u32(coef + Coefs<Q>::COUNT);
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int grp = threadIdx.y / TY, gty = threadIdx.y % TY, gtid = tid % (TX * TY);
    const int h = (a.n2 + 1) / 2, ha = a.n2 / 2, kh = (h + 63) / 64 * 64;
    // box of buffer i, half g
    auto buffer = [&](int i, int g) {
        return reinterpret_cast<float*>(sbase + (2 * i + g) * T::BUF);
    };

    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) mbar_init(bar0 + 8u * i, 1);
        fence_mbar_init();
        prefetch_tmap(&tmx);
    }
    load_coefs<Q>(a, coef, tid, 2 * TX * TY);
    __syncthreads();
    pdl_wait();

    auto request = [&](int i) {
        const int u = blockIdx.x + i * gridDim.x;
        const int r0 = (u / ncp) * TH, c0 = (u % ncp) * TX, cm = a.n2 - c0 - TX;
        const uint32_t bar = bar0 + 8u * (i % NBUF);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, 2 * T::BYTES);
        tma_load_2d(smem_u32(buffer(i % NBUF, 0)), &tmx, c0 - T::PADL, r0 - Q, bar);
        tma_load_2d(smem_u32(buffer(i % NBUF, 1)), &tmx, cm - T::PADL, r0 - Q, bar);
    };
    const int nmine = blockIdx.x < nunits ? (nunits - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint32_t polls = g_conv_wait_polls;
    if (tid == 0)
        for (int i = 0; i < NBUF - 1 && i < nmine; ++i) request(i);
    int li = 0;
    bool failed = false;
    for (; li < nmine; ++li) {
        if (tid == 0 && li + NBUF - 1 < nmine) request(li + NBUF - 1);
        const bool ok = mbar_wait(bar0 + 8u * (li % NBUF), (li / NBUF) & 1, polls);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const int u = blockIdx.x + li * gridDim.x;
        const int r0 = (u / ncp) * TH, c0 = (u % ncp) * TX;
        const int cg = grp == 0 ? c0 : a.n2 - c0 - TX;
        float* tile = buffer(li % NBUF, grp) + (T::PADL - Q);
        // a tile and its mirror reach past the same image borders, so both
        // halves take the same barriers inside the fix-up
        if (r0 - Q < 0 || r0 + TH + Q > a.n1 || c0 - Q < 0 || c0 + TX + Q > a.n2)
            fixup_tile<Q, G>(a, tile, WB, r0, cg, gtid, TX * TY);
        if (li == nmine - 1) pdl_trigger();
        float acc[RS];
        tile_acc<Q, G>(tile, WB, coef, threadIdx.x, gty, acc);
        __syncthreads();                 // both boxes consumed: they take the results
        float* mine = buffer(li % NBUF, grp);
#pragma unroll
        for (int r = 0; r < RS; ++r) mine[(gty * RS + r) * TX + threadIdx.x] = acc[r];
        __syncthreads();
        const float* other = buffer(li % NBUF, 1 - grp);
        const int t = grp == 0 ? c0 + threadIdx.x : c0 + TX - 1 - threadIdx.x;
        const bool tv = grp == 0 ? t < h : t < ha;
        const int ocol = grp == 0 ? t : kh + t;
#pragma unroll
        for (int r = 0; r < RS; ++r) {
            const int rr = gty * RS + r, row = r0 + rr;
            if (row >= a.n1 || t >= kh) continue;
            const float partner = other[rr * TX + (TX - 1 - threadIdx.x)];
            const float v = tv ? (grp == 0 ? acc[r] + partner : partner - acc[r]) : 0.f;
            split3_store(a.planes, a.plane_stride, (size_t)row * a.ld + ocol, v);
        }
        __syncthreads();                 // the boxes are refilled for unit li + NBUF
    }
    if (failed && tid == 0) {
        atomicExch(&g_conv_timeout, 1);
        for (int i = li; i < li + NBUF && i < nmine; ++i)
            mbar_wait(bar0 + 8u * (i % NBUF), (i / NBUF) & 1);
    }
}

// ------------------------------------------------ tensor-core stencils ---
// The same convolution as banded-Toeplitz products on the tensor cores
// (tcgen05, kind::f16), for supports q1, q2 <= 8 under AR and Reflective BCs.
// An output tile is TCM = 128 rows (the MMA's M: one TMEM lane per row) by
// TCW = 64 columns.  Its halo box (rows r0 - 8 .. r0 + 135, columns c0 - 8 ..
// c0 + 71) arrives by TMA as float32, receives the boundary fix-up, is scaled
// by a power of two 2^ex that brings its largest magnitude into [2^14, 2^15),
// and is split into two fp16 planes, x 2^ex = x_hi + x_lo, x_lo the fp16
// rounding of the remainder.  A plane is K-major without swizzling: for each
// group of 8 box columns the box rows follow each other at 16-byte stride, so
// the operand "box rows u .. u + 127" is the plane's start address plus 16 u
// bytes: the input rows of PSF row s1 = 8 - u for every output row at once.
// The PSF, scaled by 2^eh the same way, is split into fp16 parts Th + Tl and
// laid out per PSF row as Toeplitz bands (conv_tc_plan_kernel).  Output chunk
// c (16 columns) reads box columns [16c, 16c + 32): the first half from the
// 16-column slice c of the box (band B0), the second from slice c + 1 (B1).
// Per PSF row and slice s two MMAs (K = 16, N = 64) accumulate into chunks s-1
// and s at once: x_hi against [Th B1 | Tl B1 | Th B0 | Tl B0] and x_lo against
// [0 | Th B1 | 0 | Th B0]; every chunk keeps P = sum x_hi Th and R = sum
// (x_hi Tl + x_lo Th) in TMEM, and y = (P + R) 2^-ex 2^-eh.  The split
// represents x and h to 2^-22 relative (11 + 11 bits); the dropped product
// x_lo Tl is below 2^-22 of each term; products are exact and accumulate in
// float32.  Elements far below the tile's largest (2^-28 of it) fall into
// fp16's subnormal range, an absolute error below 2^-39 of that largest.
constexpr int TCM = 128, TCW = 64, TCQ = 8;
constexpr int TCHB = TCM + 2 * TCQ;            // 144 box rows
constexpr int TCWB = TCW + 2 * TCQ;            // 80 box columns
constexpr int TCNG = TCWB / 8;                 // 10 groups of 8 columns
constexpr int TCNR = TCHB + 1;                 // plane rows per group (one spare: spreads
                                               // the split's 16-byte stores over the banks)
constexpr int TCU = 2 * TCQ + 1;               // PSF rows of the plan
constexpr int TCTHREADS = 256;
constexpr uint32_t TC_BOX_BYTES = (uint32_t)TCWB * TCHB * 4;
constexpr uint32_t TC_PLANE_BYTES = (uint32_t)TCNG * TCNR * 16;
constexpr uint32_t TC_BTILE = 64 * 16 * 2;    // N = 64 rows x K = 16 fp16
constexpr uint32_t TC_PLAN_HEAD = 16;          // int eh, padding
constexpr uint32_t TC_TMEM_COLS = 256;         // two accumulator sets of 4 chunks x 32
using GTC = Geo<8, 16>;                        // 128-row tiles for fixup_tile

// Shared-memory layout of the tile kernel (fold = 1: one plane set and a
// receive buffer for the partner's results instead of the second set).
template <int FOLD>
struct TcSmem {
    static constexpr uint32_t BOX = 0;
    static constexpr uint32_t PLANES = TC_BOX_BYTES;
    static constexpr uint32_t RECV = PLANES + 2 * TC_PLANE_BYTES;           // fold only
    static constexpr uint32_t BT =
        FOLD ? RECV + (uint32_t)TCM * (TCW + 1) * 4 : PLANES + 4 * TC_PLANE_BYTES;
    static constexpr uint32_t BARS = BT + (uint32_t)TCU * 2 * TC_BTILE;
    static constexpr uint32_t TOTAL = BARS + 192;
    static constexpr size_t SMEM = TOTAL + 1024;                            // alignment slack
    static_assert(BT % 16 == 0 && BARS % 8 == 0, "aligned regions");
};

// 2^e for e in [-126, 127] (exact).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Exponent that brings magnitude bits mb (|v| as uint32) into [2^14, 2^15):
// 0 for zero or non-finite maxima, clamped so that 2^e and 2^-e are normal.
__device__ __forceinline__ int tc_scale_exp(uint32_t mb) {
    if (mb == 0u || mb >= 0x7F800000u) return 0;
    int e;
    frexpf(__uint_as_float(mb), &e);                     // max = f 2^e, f in [0.5, 1)
    const int ex = 15 - e;
    return ex < -126 ? -126 : (ex > 126 ? 126 : ex);
}

// The plan of one PSF for the tensor-core stencils: int eh at byte 0, then for
// each PSF row u = 0 .. 16 (s1 = 8 - u) the B tiles of the hi and lo planes,
// N = 64 rows of K = 16 fp16, K-major without swizzle ([k / 8][n][k % 8]):
//   rows  0..15: Th B1,  16..31: Tl B1 (hi) / Th B1 (lo),
//   rows 32..47: Th B0,  48..63: Tl B0 (hi) / Th B0 (lo),
// the lo tile's rows 0..15 and 32..47 zero.  Row n of band Bb holds, for output
// column j = n % 16 of a chunk and k = 0..15, the tap h(s1, s2) with
// s2 = j + 8 - (16 b + k) (0 outside the support); A' (flip) takes h(-s1, -s2).
__global__ void __launch_bounds__(TCTHREADS)
conv_tc_plan_kernel(const float* __restrict__ psf, int q1, int q2, int flip, uint8_t* plan) {
    // block (u, p) writes the tile of PSF row u, plane p; every block finds the scale
    __shared__ uint32_t red[TCTHREADS / 32];
    const int tid = threadIdx.x, u = blockIdx.x, p = blockIdx.y;
    const int kw = 2 * q2 + 1, count = (2 * q1 + 1) * kw;
    uint32_t mb = 0;
    for (int i = tid; i < count; i += TCTHREADS) mb = max(mb, __float_as_uint(fabsf(psf[i])));
    mb = __reduce_max_sync(0xffffffffu, mb);
    if ((tid & 31) == 0) red[tid >> 5] = mb;
    __syncthreads();
    mb = 0;
    for (int w = 0; w < TCTHREADS / 32; ++w) mb = max(mb, red[w]);
    const int eh = tc_scale_exp(mb);
    const float sc = pow2f(eh);
    if (tid == 0 && u == 0 && p == 0) *reinterpret_cast<int*>(plan) = eh;
    uint16_t* tile =
        reinterpret_cast<uint16_t*>(plan + TC_PLAN_HEAD) + (size_t)(u * 2 + p) * (TC_BTILE / 2);
    for (int i = tid; i < 64 * 16; i += TCTHREADS) {
        const int n = i / 16, k = i % 16;
        const int band = n < 32 ? 1 : 0, part = (n / 16) & 1, j = n % 16;
        const int s1 = TCQ - u, s2 = j + TCQ - (16 * band + k);
        float hv = 0.f;
        if (s1 >= -q1 && s1 <= q1 && s2 >= -q2 && s2 <= q2) {
            const int t1 = flip ? -s1 : s1, t2 = flip ? -s2 : s2;
            hv = psf[(t1 + q1) * kw + (t2 + q2)];
        }
        const float hs = hv * sc;
        const __half th = __float2half_rn(hs);
        const __half tl = __float2half_rn(hs - __half2float(th));
        const __half v = p == 0 ? (part == 0 ? th : tl) : (part == 0 ? __float2half_rn(0.f) : th);
        tile[(k / 8) * 64 * 8 + n * 8 + k % 8] = __half_as_ushort(v);
    }
}

// Two fp16 halves of a pair of values (|x| < 2^15 after the tile's scaling):
// Veltkamp's splitting with sigma = 2^13 + 1 gives hi with at most 11
// significant bits (exact in fp16 in its normal range) and lo = x - hi
// exactly; lo is rounded to fp16 (11 of its at most 13 bits).  Plain
// round-to-nearest operations: nothing is contracted into FMAs.
__device__ __forceinline__ void tc_split2(float x0, float x1, uint32_t* hi, uint32_t* lo) {
    constexpr float SIGMA = 8193.f;
    const float g0 = __fmul_rn(SIGMA, x0), g1 = __fmul_rn(SIGMA, x1);
    const float h0 = __fsub_rn(g0, __fsub_rn(g0, x0)), h1 = __fsub_rn(g1, __fsub_rn(g1, x1));
    const __half2 hh = __floats2half2_rn(h0, h1);
    const __half2 ll = __floats2half2_rn(__fsub_rn(x0, h0), __fsub_rn(x1, h1));
    *hi = *reinterpret_cast<const uint32_t*>(&hh);
    *lo = *reinterpret_cast<const uint32_t*>(&ll);
}

// Box of tile i: fix-up, scale and split into the plane pair at `hi` (lo one
// plane further).  Returns the scale exponent; called by the NT threads that
// share barrier BAR (0: the whole block).
template <int BAR, int NT>
__device__ __forceinline__ int tc_split_box(const ConvArgs& a, float* box, uint8_t* hi, int r0,
                                            int c0, uint32_t* red, int tid) {
    if (r0 - TCQ < 0 || r0 + TCM + TCQ > a.n1 || c0 - TCQ < 0 || c0 + TCW + TCQ > a.n2)
        fixup_tile<TCQ, GTC, BAR>(a, box, TCWB, r0, c0, tid, NT);
    const float4* b4 = reinterpret_cast<const float4*>(box);
    uint32_t mb = 0;
#pragma unroll 4
    for (int it = tid; it < TCHB * TCNG; it += NT) {
        const int row = it / TCNG, g = it % TCNG;
        const float4 v0 = b4[row * (TCWB / 4) + 2 * g], v1 = b4[row * (TCWB / 4) + 2 * g + 1];
        mb = max(mb, max(max(__float_as_uint(fabsf(v0.x)), __float_as_uint(fabsf(v0.y))),
                         max(__float_as_uint(fabsf(v0.z)), __float_as_uint(fabsf(v0.w)))));
        mb = max(mb, max(max(__float_as_uint(fabsf(v1.x)), __float_as_uint(fabsf(v1.y))),
                         max(__float_as_uint(fabsf(v1.z)), __float_as_uint(fabsf(v1.w)))));
    }
    mb = __reduce_max_sync(0xffffffffu, mb);
    if ((tid & 31) == 0) red[tid >> 5] = mb;
    stencil_sync<BAR>(NT);
    mb = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) mb = max(mb, red[w]);
    const int ex = tc_scale_exp(mb);
    const float sc = pow2f(ex);
    uint8_t* lo = hi + TC_PLANE_BYTES;
#pragma unroll 2
    for (int it = tid; it < TCHB * TCNG; it += NT) {
        const int row = it / TCNG, g = it % TCNG;
        const float4 v0 = b4[row * (TCWB / 4) + 2 * g], v1 = b4[row * (TCWB / 4) + 2 * g + 1];
        uint32_t h[4], l[4];
        tc_split2(v0.x * sc, v0.y * sc, &h[0], &l[0]);
        tc_split2(v0.z * sc, v0.w * sc, &h[1], &l[1]);
        tc_split2(v1.x * sc, v1.y * sc, &h[2], &l[2]);
        tc_split2(v1.z * sc, v1.w * sc, &h[3], &l[3]);
        const size_t off = ((size_t)g * TCNR + row) * 16;
        *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    tc::fence_proxy_async_smem();        // the planes are read by the tensor cores
    return ex;
}

// The MMAs of one tile (one thread): planes at `hi` (lo one plane further),
// accumulators at TMEM column d, PSF rows u0 .. u1 of the B tiles at `bt`.
// Slice-major order: the MMAs of a slice accumulate into the same TMEM
// columns back to back, and the slices run 0, 2, 4, 1, 3 so that consecutive
// slices touch disjoint columns (an MMA into columns that the previous one
// only partly covered waits for it).  The first MMA of slices 0, 2 and 4
// initialises chunks 0 | 1, 2 | 3, which together cover the tile.
__device__ __forceinline__ void tc_issue(uint32_t hi, uint32_t bt, uint32_t d, int u0, int u1) {
    using namespace tc;
    constexpr uint32_t LBO = TCNR * 16;
    const uint64_t ah0 = desc_k_none(hi, LBO, 128), al0 = desc_k_none(hi + TC_PLANE_BYTES, LBO, 128);
    const uint64_t b0 = desc_k_none(bt, 64 * 16, 128);
    constexpr uint32_t id32 = idesc_f16_f32(TCM, 32), id64 = idesc_f16_f32(TCM, 64);
    constexpr uint64_t HALF0 = (32 * 16) >> 4;           // B rows 32..63: band B0
    constexpr int NS = TCW / 16;                          // chunks; slices 0 .. NS
    static_assert(NS == 4, "slice order below");
    constexpr int order[NS + 1] = {0, 2, 4, 1, 3};
#pragma unroll
    for (int oi = 0; oi <= NS; ++oi) {
        const int s = order[oi];
        // slice 0 feeds chunk 0 (band B0), slice NS chunk NS - 1 (band B1), the
        // others chunks s - 1 and s
        const uint32_t dd = s == 0 ? d : d + 32 * (s - 1);
        const uint32_t id = (s == 0 || s == NS) ? id32 : id64;
        const uint64_t boff = s == 0 ? HALF0 : 0;
        const uint64_t as = (uint64_t)(((2 * s) * LBO) >> 4);
        for (int u = u0; u <= u1; ++u) {
            const uint64_t bh = b0 + (uint64_t)((u * 2) * TC_BTILE >> 4) + boff;
            const uint64_t ao = as + (uint64_t)u;          // 16 u bytes: box rows u .. u + 127
            mma_bf16(dd, ah0 + ao, bh, id, (u == u0 && s % 2 == 0) ? 0u : 1u);
            mma_bf16(dd, al0 + ao, bh + (uint64_t)(TC_BTILE >> 4), id, 1u);
        }
    }
}

// bf16x3 split of 16 consecutive values into the three planes at element
// offset off (16-byte aligned rows: 8-element vector stores).
__device__ __forceinline__ void split3_store16(uint16_t* planes, size_t pstride, size_t off,
                                               const float (&y)[16], int nvalid) {
    if (nvalid < 16) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < nvalid) split3_store(planes, pstride, off + j, y[j]);
        return;
    }
    uint32_t w[3][8];
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
        uint32_t lo3[3], hi3[3];
        float v0 = y[j], v1 = y[j + 1];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const __nv_bfloat16 b0 = __float2bfloat16_rn(v0), b1 = __float2bfloat16_rn(v1);
            lo3[p] = __bfloat16_as_ushort(b0);
            hi3[p] = __bfloat16_as_ushort(b1);
            v0 -= __bfloat162float(b0);
            v1 -= __bfloat162float(b1);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) w[p][j / 2] = lo3[p] | (hi3[p] << 16);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        uint4* dst = reinterpret_cast<uint4*>(planes + p * pstride + off);
        dst[0] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
        dst[1] = make_uint4(w[p][4], w[p][5], w[p][6], w[p][7]);
    }
}

// Epilogue of 4 outputs y of row `row` at columns col .. col + 3 (n2 % 4 == 0,
// col % 4 == 0, all four inside the image); returns the squares the mode sums.
__device__ __forceinline__ float tc_store4(const ConvArgs& a, int row, int col, float4 yv,
                                           bool vec3) {
    const size_t o = (size_t)row * a.n2 + col;
    if (a.mode == CONV_SPLIT3) {
        const float y[4] = {yv.x, yv.y, yv.z, yv.w};
        const size_t po = (size_t)row * a.ld + col;
        if (vec3) {
            uint32_t w[3][2];
#pragma unroll
            for (int j = 0; j < 4; j += 2) {
                float v0 = y[j], v1 = y[j + 1];
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    const __nv_bfloat16 b0 = __float2bfloat16_rn(v0), b1 = __float2bfloat16_rn(v1);
                    w[p][j / 2] = (uint32_t)__bfloat16_as_ushort(b0) |
                                  ((uint32_t)__bfloat16_as_ushort(b1) << 16);
                    v0 -= __bfloat162float(b0);
                    v1 -= __bfloat162float(b1);
                }
            }
#pragma unroll
            for (int p = 0; p < 3; ++p)
                *reinterpret_cast<uint2*>(a.planes + p * a.plane_stride + po) = make_uint2(w[p][0], w[p][1]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) split3_store(a.planes, a.plane_stride, po + j, y[j]);
        }
        return 0.f;
    }
    float4* p4 = reinterpret_cast<float4*>(a.out + o);
    if (a.mode == CONV_STORE) {
        *p4 = yv;
        return 0.f;
    }
    if (a.mode == CONV_RESIDUAL) {
        const float4 g = __ldg(reinterpret_cast<const float4*>(a.aux + o));
        const float4 r = make_float4(g.x - yv.x, g.y - yv.y, g.z - yv.z, g.w - yv.w);
        *p4 = r;
        return a.sumsq ? r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w : 0.f;
    }
    const float4 xo = *p4;                                   // CONV_AXPY
    const float4 xn = make_float4(fmaf(a.tau, yv.x, xo.x), fmaf(a.tau, yv.y, xo.y),
                                  fmaf(a.tau, yv.z, xo.z), fmaf(a.tau, yv.w, xo.w));
    *p4 = xn;
    if (!a.f) return 0.f;
    const float4 f = __ldg(reinterpret_cast<const float4*>(a.f + o));
    const float e0 = xn.x - f.x, e1 = xn.y - f.y, e2 = xn.z - f.z, e3 = xn.w - f.w;
    return e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3;
}

// The results of this thread's chunk c of the tile in D (TMEM, lane base
// included): y = (P + R) scale.
__device__ __forceinline__ void tc_load_chunk(uint32_t d, int c, float scale, float (&y)[16]) {
    float P[16], R[16];
    tc::tmem_ld16x2(d + 32 * c, d + 32 * c + 16, P, R);
#pragma unroll
    for (int j = 0; j < 16; ++j) y[j] = (P[j] + R[j]) * scale;
}

// Sum of v over the NT compute threads of barrier BAR added to *sumsq (one
// float64 atomic per CTA; float32 per-thread partials).
template <int BAR, int NT>
__device__ __forceinline__ void tc_add_sumsq(double* sumsq, float vf, double* part, int tid) {
    double v = vf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) part[tid >> 5] = v;
    stencil_sync<BAR>(NT);
    if (tid == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) t += part[w];
        if (t != 0.0) atomicAdd(sumsq, t);
    }
    stencil_sync<BAR>(NT);
}

// OR of v over the NT threads of named barrier BAR.
template <int BAR, int NT>
__device__ __forceinline__ bool tc_bar_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(BAR), "n"(NT)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent tensor-core stencil (every mode but the folded one), warp
// specialised.  Warp 8 (one thread) is the producer: it requests the halo box
// of each tile by TMA as soon as the previous box has been split, and issues
// a tile's MMAs once its planes are written and its accumulator set (one of
// two) has been read out.  Warps 0-7 split box i into plane set i & 1, then
// read the accumulators of tile i - 1 and apply the epilogue, so that the
// split and the epilogue overlap the MMAs.  Each CTA walks the tiles
// t = blockIdx.x + i gridDim.x.  Every wait is bounded; a wait that gives up
// raises the CTA's flag, which ends both roles, and the producer waits
// (bounded) for its copies and MMAs in flight before the CTA exits.
constexpr int TC_NT = 256;                       // compute threads (named barrier 1)
constexpr int TC_TILE_THREADS = TC_NT + 32;      // plus the producer warp

__global__ void __launch_bounds__(TC_TILE_THREADS, 1)
conv_tc_kernel(const __grid_constant__ CUtensorMap tmx, const ConvArgs a, const uint8_t* plan,
               int ntx, int ntiles, int vec3) {
    using namespace tc;
    using L = TcSmem<0>;
    extern __shared__ __align__(1024) uint8_t smem_tc[];
    uint8_t* sb = smem_tc + ((1024u - (smem_u32(smem_tc) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(sb);
    float* box = reinterpret_cast<float*>(sb + L::BOX);
    // mbarriers: box full / empty, B tiles, and per accumulator set b: planes
    // full, MMAs done, accumulators free
    const uint32_t bars = sbase + L::BARS;
    const uint32_t box_full = bars, box_empty = bars + 8, b_bar = bars + 16;
    auto planes_full = [&](int b) { return bars + 24 + 8u * b; };
    auto mma_done = [&](int b) { return bars + 40 + 8u * b; };
    auto d_free = [&](int b) { return bars + 56 + 8u * b; };
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sb + L::BARS + 72);
    int* sflag = reinterpret_cast<int*>(sb + L::BARS + 76);
    int* sex = reinterpret_cast<int*>(sb + L::BARS + 80);
    uint32_t* red = reinterpret_cast<uint32_t*>(sb + L::BARS + 88);
    double* part = reinterpret_cast<double*>(sb + L::BARS + 120);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int u0 = TCQ - a.q1, u1 = TCQ + a.q1;
    const int nmine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid == 0) {
        mbar_init(box_full, 1);
        mbar_init(box_empty, 1);
        mbar_init(b_bar, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(planes_full(b), 1);
            mbar_init(mma_done(b), 1);
            mbar_init(d_free(b), 1);
        }
        *sflag = 0;
        fence_mbar_init();
        prefetch_tmap(&tmx);
    }
    if (warp == 8) {
        tmem_alloc(smem_u32(tslot), TC_TMEM_COLS);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    const float seh = pow2f(-__ldg(reinterpret_cast<const int*>(plan)));
    const uint32_t polls = g_conv_wait_polls;
    auto tile_origin = [&](int i, int* r0, int* c0) {
        const int t = blockIdx.x + i * gridDim.x;
        *r0 = (t / ntx) * TCM;
        *c0 = (t % ntx) * TCW;
    };
    auto plane_set = [&](int i) { return sb + L::PLANES + (uint32_t)(i & 1) * 2 * TC_PLANE_BYTES; };

    if (warp == 8) {
        // ---- producer
        if (lane == 0 && nmine > 0) {    // the plan does not depend on the previous kernel
            const uint32_t bytes = (uint32_t)(u1 - u0 + 1) * 2 * TC_BTILE;
            mbar_arrive_expect_tx(b_bar, bytes);
            bulk_load(sbase + L::BT + (uint32_t)u0 * 2 * TC_BTILE,
                      plan + TC_PLAN_HEAD + (size_t)u0 * 2 * TC_BTILE, bytes, b_bar);
        }
        pdl_wait();                      // the input image comes from the previous kernel
        if (lane == 0 && nmine > 0) {
            auto request = [&](int i) {
                int r0, c0;
                tile_origin(i, &r0, &c0);
                mbar_arrive_expect_tx(box_full, TC_BOX_BYTES);
                tma_load_2d(sbase + L::BOX, &tmx, c0 - TCQ, r0 - TCQ, box_full);
            };
            request(0);
            int requested = 1, issued = 0;
            bool ok = mbar_wait(b_bar, 0, polls);
            for (int i = 0; ok && i < nmine; ++i) {
                if (i + 1 < nmine) {     // box i is split: the buffer takes box i + 1
                    ok = mbar_wait(box_empty, (uint32_t)(i & 1), polls) && !*(volatile int*)sflag;
                    if (!ok) break;
                    request(i + 1);
                    requested = i + 2;
                }
                ok = mbar_wait(planes_full(i & 1), (uint32_t)((i >> 1) & 1), polls);
                if (ok && i >= 2) ok = mbar_wait(d_free(i & 1), (uint32_t)(((i - 2) >> 1) & 1), polls);
                if (!ok || *(volatile int*)sflag) break;
                fence_after_sync();
                tc_issue(smem_u32(plane_set(i)), sbase + L::BT, tmem + (uint32_t)(i & 1) * 128, u0,
                         u1);
                mma_commit(mma_done(i & 1));
                issued = i + 1;
            }
            if (!ok) {
                atomicExch(sflag, 1);
                atomicExch(&g_conv_timeout, 1);
            }
            // nothing in flight when the CTA exits (bounded waits; phases that
            // already completed return at once)
            mbar_wait(b_bar, 0);
            mbar_wait(box_full, (uint32_t)((requested - 1) & 1));
            if (issued > 0) mbar_wait(mma_done((issued - 1) & 1), (uint32_t)(((issued - 1) >> 1) & 1));
            if (issued > 1) mbar_wait(mma_done((issued - 2) & 1), (uint32_t)(((issued - 2) >> 1) & 1));
        }
    } else {
        // ---- compute warps
        pdl_wait();                      // before writing what the previous kernel may read
        const int quarter = warp & 3, hw = warp >> 2;
        const int m = quarter * 32 + lane;
        // Epilogue of tile j: each thread reads its row's accumulators (TMEM lane
        // m) and parks the results in plane set j & 1 (free: tile j's MMAs are done
        // and tile j + 2's split comes after this), then the warps walk the tile
        // row by row, so that the loads and stores of global memory are whole
        // 256-byte rows rather than 16-byte pieces of 32 rows.
        constexpr int STG = TCW + 4;                     // staging pitch (floats)
        static_assert(TCM * STG * 4 <= 2 * TC_PLANE_BYTES, "the staging fits a plane set");
        auto epilogue = [&](int j) -> bool {
            int r0, c0;
            tile_origin(j, &r0, &c0);
            bool ok = true;
            if (tid == 0) ok = mbar_wait(mma_done(j & 1), (uint32_t)((j >> 1) & 1), polls);
            if (tc_bar_or<1, TC_NT>(!ok)) return false;
            fence_after_sync();
            if (a.early_trigger && j == nmine - 1) pdl_trigger();
            const float scale = pow2f(-sex[j & 1]) * seh;
            const uint32_t d = tmem + (uint32_t)(j & 1) * 128 + ((uint32_t)(quarter * 32) << 16);
            float* stg = reinterpret_cast<float*>(plane_set(j));
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int c = 2 * hw + cc;
                float y[16];
                tc_load_chunk(d, c, scale, y);
                float4* dst = reinterpret_cast<float4*>(stg + m * STG + 16 * c);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    dst[q] = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
            }
            fence_before_sync();
            stencil_sync<1>(TC_NT);
            float sq = 0.f;
#pragma unroll 4
            for (int it = tid; it < TCM * (TCW / 4); it += TC_NT) {
                const int rl = it / (TCW / 4), q4 = it % (TCW / 4);
                const int row = r0 + rl, col = c0 + 4 * q4;
                if (row < a.n1 && col < a.n2)
                    sq += tc_store4(a, row, col,
                                    *reinterpret_cast<const float4*>(stg + rl * STG + 4 * q4), vec3 != 0);
            }
            if (a.sumsq) tc_add_sumsq<1, TC_NT>(a.sumsq, sq, part, tid);
            else stencil_sync<1>(TC_NT);
            if (tid == 0) mbar_arrive(d_free(j & 1));
            return true;
        };
        bool failed = false;
        for (int i = 0; i < nmine; ++i) {
            bool ok = true;
            if (tid == 0) ok = mbar_wait(box_full, (uint32_t)(i & 1), polls) && !*(volatile int*)sflag;
            if (tc_bar_or<1, TC_NT>(!ok)) {
                failed = true;
                break;
            }
            int r0, c0;
            tile_origin(i, &r0, &c0);
            const int ex = tc_split_box<1, TC_NT>(a, box, plane_set(i), r0, c0, red, tid);
            if (tid == 0) sex[i & 1] = ex;
            stencil_sync<1>(TC_NT);      // box read, planes written (each writer fenced)
            if (tid == 0) {
                mbar_arrive(box_empty);
                mbar_arrive(planes_full(i & 1));
            }
            if (i >= 1 && !epilogue(i - 1)) {
                failed = true;
                break;
            }
        }
        if (!failed && nmine > 0 && !epilogue(nmine - 1)) failed = true;
        if (failed && tid == 0) {
            atomicExch(sflag, 1);
            atomicExch(&g_conv_timeout, 1);
        }
    }
    if (!a.early_trigger) pdl_trigger();
    fence_before_sync();
    __syncthreads();
    if (warp == 8) {
        fence_after_sync();
        tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

// Folding variant (CONV_SPLIT3 with fold): a cluster of two CTAs per work
// unit, rank 0 on the tile at columns [c0, c0 + 64) and rank 1 on its mirror
// [n2 - c0 - 64, n2 - c0).  Column t = c0 + j pairs with n2 - 1 - t, column
// 63 - j of the mirror tile.  Each rank sends its results to the other's
// receive buffer (distributed shared memory); rank 0 writes the bf16x3 split
// of y+_t = y_t + y_{n2-1-t} at column t (zero from ceil(n2/2) on), rank 1 that
// of y-_t = y_t - y_{n2-1-t} at column Kh + t (zero from floor(n2/2) on).  One
// plane set: the split of the next unit waits for the current unit's MMAs.  A
// wait that gives up on either rank is exchanged with the peer, and both ranks
// leave the loop after the same cluster barrier.
constexpr int TC_RECV_PITCH = TCW + 1;          // conflict-free column reads of the buffer

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TCTHREADS, 1)
conv_tc_fold_kernel(const __grid_constant__ CUtensorMap tmx, const ConvArgs a, const uint8_t* plan,
                    int ncp, int nunits, int vec3) {
    using namespace tc;
    using L = TcSmem<1>;
    extern __shared__ __align__(1024) uint8_t smem_tc[];
    uint8_t* sb = smem_tc + ((1024u - (smem_u32(smem_tc) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(sb);
    float* box = reinterpret_cast<float*>(sb + L::BOX);
    const float* recv = reinterpret_cast<const float*>(sb + L::RECV);
    const uint32_t box_bar = sbase + L::BARS, b_bar = box_bar + 8, mma_bar = box_bar + 16;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sb + L::BARS + 32);
    int* sex = reinterpret_cast<int*>(sb + L::BARS + 40);
    uint32_t* red = reinterpret_cast<uint32_t*>(sb + L::BARS + 48);
    int* pbad_flag = reinterpret_cast<int*>(sb + L::BARS + 84);   // written by the peer
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = cluster_ctarank(), peer = rank ^ 1u;
    const int u0 = TCQ - a.q1, u1 = TCQ + a.q1;
    const int h = (a.n2 + 1) / 2, ha = a.n2 / 2, kh = (h + 63) / 64 * 64;
    const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
    const int nmine = cid < nunits ? (nunits - 1 - cid) / ncl + 1 : 0;   // the same on both ranks

    if (tid == 0) {
        mbar_init(box_bar, 1);
        mbar_init(b_bar, 1);
        mbar_init(mma_bar, 1);
        fence_mbar_init();
        prefetch_tmap(&tmx);
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), TC_TMEM_COLS);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;
    if (tid == 0 && nmine > 0) {
        const uint32_t bytes = (uint32_t)(u1 - u0 + 1) * 2 * TC_BTILE;
        mbar_arrive_expect_tx(b_bar, bytes);
        bulk_load(sbase + L::BT + (uint32_t)u0 * 2 * TC_BTILE,
                  plan + TC_PLAN_HEAD + (size_t)u0 * 2 * TC_BTILE, bytes, b_bar);
    }
    const float seh = pow2f(-__ldg(reinterpret_cast<const int*>(plan)));
    pdl_wait();

    auto unit_origin = [&](int i, int* r0, int* c0) {
        const int un = cid + i * ncl;
        *r0 = (un / ncp) * TCM;
        *c0 = (un % ncp) * TCW;                         // rank 0's tile; the mirror is n2 - c0 - 64
    };
    auto request = [&](int i) {
        int r0, c0;
        unit_origin(i, &r0, &c0);
        const int cg = rank == 0 ? c0 : a.n2 - c0 - TCW;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(box_bar, TC_BOX_BYTES);
        tma_load_2d(sbase + L::BOX, &tmx, cg - TCQ, r0 - TCQ, box_bar);
    };
    const uint32_t polls = g_conv_wait_polls;
    uint8_t* planes = sb + L::PLANES;
    const uint32_t rpeer = mapa(smem_u32(recv), peer);
    const uint32_t rflag = mapa(smem_u32(pbad_flag), peer);
    const int quarter = warp & 3, hw = warp >> 2;
    const int m = quarter * 32 + lane;
    bool failed = false;
    int li = 0, requested = 0, consumed = 0, issued = 0;
    if (nmine > 0 && tid == 0) request(0);
    requested = nmine > 0 ? 1 : 0;
    for (; li < nmine; ++li) {
        int r0, c0;
        unit_origin(li, &r0, &c0);
        const int cg = rank == 0 ? c0 : a.n2 - c0 - TCW;
        // 1. box -> planes -> MMAs (the previous unit's MMAs have completed)
        bool ok = true;
        if (tid == 0) {          // one thread polls; the others wait at the block barrier
            ok = mbar_wait(box_bar, (uint32_t)(li & 1), polls);
            if (li == 0) ok = ok && mbar_wait(b_bar, 0, polls);
        }
        bool bad = __syncthreads_or(!ok);
        if (!bad) {
            const int ex = tc_split_box<0, TCTHREADS>(a, box, planes, r0, cg, red, tid);
            consumed = li + 1;
            if (tid == 0) sex[0] = ex;
            fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                if (li + 1 < nmine) request(li + 1);
                fence_after_sync();
                tc_issue(smem_u32(planes), sbase + L::BT, tmem, u0, u1);
                mma_commit(mma_bar);
            }
            if (li + 1 < nmine) requested = li + 2;
            issued = li + 1;
            if (tid == 0) ok = mbar_wait(mma_bar, (uint32_t)(li & 1), polls);
            bad = __syncthreads_or(!ok);
            fence_after_sync();
        }
        if (li == nmine - 1) pdl_trigger();
        // 2. this tile's results -> the peer's receive buffer [row][TC_RECV_PITCH]
        const float scale = pow2f(-sex[0]) * seh;
        const uint32_t d = tmem + ((uint32_t)(quarter * 32) << 16);
        float y[2][16];
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = 2 * hw + cc;
            if (!bad) {
                tc_load_chunk(d, c, scale, y[cc]);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) y[cc][j] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j)
                st_cluster_f32(rpeer + 4u * (m * TC_RECV_PITCH + 16 * c + j), y[cc][j]);
        }
        if (tid == 0)
            asm volatile("st.shared::cluster.b32 [%0], %1;" ::"r"(rflag), "r"(bad ? 1 : 0) : "memory");
        fence_before_sync();
        cluster_sync();                  // the peer's results and status have arrived
        const bool pbad = *reinterpret_cast<volatile int*>(pbad_flag) != 0;
        // 3. the folded outputs of 16 columns per chunk
        const int row = r0 + m;
        if (!bad && !pbad && row < a.n1) {
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int c = 2 * hw + cc;
                float v[16];
                int ocol;
                if (rank == 0) {         // t = c0 + 16 c + j: y(16 c + j) + y_peer(63 - 16 c - j)
                    const int t0 = c0 + 16 * c;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        v[j] = t0 + j < h ? y[cc][j] + recv[m * TC_RECV_PITCH + (TCW - 1 - 16 * c - j)]
                                          : 0.f;
                    ocol = t0;
                } else {                 // t = c0 + 48 - 16 c + j: y_peer(t - c0) - y(15 + 16 c - j)
                    const int t0 = c0 + 48 - 16 * c;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        v[j] = t0 + j < ha ? recv[m * TC_RECV_PITCH + (48 - 16 * c + j)] - y[cc][15 - j]
                                           : 0.f;
                    ocol = kh + t0;
                }
                if (vec3) {
                    split3_store16(a.planes, a.plane_stride, (size_t)row * a.ld + ocol, v, 16);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        split3_store(a.planes, a.plane_stride, (size_t)row * a.ld + ocol + j, v[j]);
                }
            }
        }
        fence_before_sync();
        cluster_sync();                  // both buffers read before the next unit refills them
        if (bad || pbad) {
            failed = true;
            break;
        }
    }
    if (failed && tid == 0) {
        atomicExch(&g_conv_timeout, 1);
        mbar_wait(b_bar, 0);             // the B tiles' copy, if the first wait gave up
        for (int i = consumed; i < requested; ++i) mbar_wait(box_bar, (uint32_t)(i & 1));
        for (int i = li; i < issued; ++i) mbar_wait(mma_bar, (uint32_t)(i & 1));
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(tmem, TC_TMEM_COLS);
    }
}

// Generic path for large supports: one output per thread, taps read straight
// from the (L2-resident) input through the virtual extension.
__global__ void __launch_bounds__(256)
conv_generic_kernel(const ConvArgs a) {
    const int col = blockIdx.x * 32 + threadIdx.x;
    const int row = blockIdx.y * 8 + threadIdx.y;
    const bool in = row < a.n1 && col < a.n2;
    const int kw = 2 * a.q2 + 1;
    float acc = 0.f;
    float sq = 0.f;
    if (in) {
        for (int s2 = -a.q2; s2 <= a.q2; ++s2) {
            for (int s1 = -a.q1; s1 <= a.q1; ++s1) {
                const int t1 = a.flip ? -s1 : s1, t2 = a.flip ? -s2 : s2;
                const float hv = __ldg(a.psf + (t1 + a.q1) * kw + (t2 + a.q2));
                acc = fmaf(hv, ext_value(a.x, a.n1, a.n2, a.q1, a.q2, row - s1, col - s2, a.bc), acc);
            }
        }
        sq = conv_epilogue(a, row, col, acc);
    }
    if (a.sumsq) add_sumsq(a.sumsq, sq);
}

// TMA map of the float32 image x (n1 rows of n2) with the halo box of Q and G.
template <int Q, class G>
bool make_image_map(const ConvArgs& a, CUtensorMap* map) {
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)a.n2, (cuuint64_t)a.n1};
    cuuint64_t strides[1] = {(cuuint64_t)a.n2 * 4};
    cuuint32_t box[2] = {(cuuint32_t)TmaTile<Q, G>::WB, (cuuint32_t)TmaTile<Q, G>::HB};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.x), dims, strides, box,
               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Work units per SM of a launch of `units` that fits in one wave of `per` units per
// SM (0 when it does not fit): the most any SM gets, times the rows of a unit.
inline int wave_rows(int units, int per, int th) {
    const int nsm = sm_count();
    if (units > per * nsm) return 0;
    return (units + nsm - 1) / nsm * th;
}

// G54 where a single wave of it leaves the busiest SM at least 10% fewer rows.
inline bool prefer_g54(int units64, int units54, int per) {
    const int r64 = wave_rows(units64, per, G64::TH), r54 = wave_rows(units54, per, G54::TH);
    return r64 > 0 && r54 > 0 && 10 * r54 < 9 * r64;
}

template <int Q, class G>
cudaError_t launch_fold_g(const ConvArgs& a, cudaStream_t s) {
    using F = FoldTile<Q, G>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    static int per_sm = 1;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(conv_tma_fold_kernel<Q, G>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::SMEM);
        if (attr == cudaSuccess)
            attr = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, conv_tma_fold_kernel<Q, G>, 2 * TX * G::TY, F::SMEM);
        if (per_sm < 1) per_sm = 1;
    });
    if (attr != cudaSuccess) return attr;
    CUtensorMap map;
    if (!make_image_map<Q, G>(a, &map)) return cudaErrorInvalidValue;
    const int h = (a.n2 + 1) / 2;
    const int ncp = (h + TX - 1) / TX, nty = (a.n1 + G::TH - 1) / G::TH;
    const int nunits = ncp * nty;
    const int cap = sm_count() * per_sm;
    const int grid = nunits < cap ? nunits : cap;
    count_launch();
    return launch_pdl(conv_tma_fold_kernel<Q, G>, dim3(grid), dim3(TX, 2 * G::TY), F::SMEM, s, map,
                      a, ncp, nunits);
}

template <int Q>
cudaError_t launch_fold(const ConvArgs& a, cudaStream_t s) {
    const int ncp = ((a.n2 + 1) / 2 + TX - 1) / TX;
    const int u64 = ncp * ((a.n1 + G64::TH - 1) / G64::TH);
    const int u54 = ncp * ((a.n1 + G54::TH - 1) / G54::TH);
    return prefer_g54(u64, u54, 1) ? launch_fold_g<Q, G54>(a, s) : launch_fold_g<Q, G64>(a, s);
}

template <int Q, bool RW>
cudaError_t launch_tiles(const ConvArgs& a, cudaStream_t s);

template <int Q>
cudaError_t launch_fast(const ConvArgs& a, cudaStream_t s) {
    if (a.fold) {
        if (a.mode != CONV_SPLIT3 || a.bc == AR_BC_PERIODIC ||
            (reinterpret_cast<uintptr_t>(a.x) & 15) != 0 || (a.n2 & 3) != 0)
            return cudaErrorInvalidValue;            // callers request the fold only where it runs
        return launch_fold<Q>(a, s);
    }
    if (a.mode == CONV_RESIDUAL || a.mode == CONV_AXPY) return launch_tiles<Q, true>(a, s);
    return launch_tiles<Q, false>(a, s);
}

// The persistent TMA path with geometry G; false in *ok when the map cannot be made.
template <int Q, bool RW, class G>
cudaError_t launch_tma(const ConvArgs& a, cudaStream_t s, bool* ok) {
    using T = TmaTile<Q, G>;
    // a.spread: one wave of at most two CTAs per SM, by the shared-memory request,
    // so that CTAs placed while the predecessor drains cannot pile onto the SMs
    // that free up first
    constexpr size_t SMEM2 = T::SMEM > 80 * 1024 ? T::SMEM : 80 * 1024;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    static int per_sm = 1;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(conv_tma_kernel<Q, RW, G>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM2);
        if (attr == cudaSuccess)
            attr = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_tma_kernel<Q, RW, G>,
                                                                 TX * G::TY, T::SMEM);
        if (per_sm < 1) per_sm = 1;
    });
    CUtensorMap map;
    *ok = attr == cudaSuccess && make_image_map<Q, G>(a, &map);
    if (!*ok) return cudaSuccess;
    const int ntx = (a.n2 + TX - 1) / TX, nty = (a.n1 + G::TH - 1) / G::TH;
    const int ntiles = ntx * nty;
    const bool two = a.spread && ntiles <= 2 * sm_count();
    const int cap = sm_count() * per_sm;
    const int grid = ntiles < cap ? ntiles : cap;
    // a programmatic dependent: the CTAs are placed while the predecessor
    // drains; predecessors that could leave SMs idle for long (the last
    // contraction, stencils) let it launch only at their end, so that early
    // CTAs do not pile onto those SMs
    count_launch();
    return launch_pdl(conv_tma_kernel<Q, RW, G>, dim3(grid), dim3(TX, G::TY),
                      two ? SMEM2 : T::SMEM, s, map, a, ntx, ntiles);
}

template <int Q, bool RW>
cudaError_t launch_tiles(const ConvArgs& a, cudaStream_t s) {
    // TMA path: AR / Reflective, 16-byte aligned image and row pitch
    if (a.bc != AR_BC_PERIODIC && (reinterpret_cast<uintptr_t>(a.x) & 15) == 0 &&
        (a.n2 & 3) == 0) {
        const int ntx = (a.n2 + TX - 1) / TX;
        const int t64 = ntx * ((a.n1 + G64::TH - 1) / G64::TH);
        const int t54 = ntx * ((a.n1 + G54::TH - 1) / G54::TH);
        bool ok = false;
        const cudaError_t e = prefer_g54(t64, t54, 2) ? launch_tma<Q, RW, G54>(a, s, &ok)
                                                      : launch_tma<Q, RW, G64>(a, s, &ok);
        if (ok || e != cudaSuccess) return e;
    }
    dim3 grid((a.n2 + TX - 1) / TX, (a.n1 + G64::TH - 1) / G64::TH);
    count_launch();
    conv_fast_kernel<Q, RW><<<grid, dim3(TX, G64::TY), 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------ tensor-core stencils (host)
bool make_tc_map(const ConvArgs& a, CUtensorMap* map) {
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)a.n2, (cuuint64_t)a.n1};
    cuuint64_t strides[1] = {(cuuint64_t)a.n2 * 4};
    cuuint32_t box[2] = {(cuuint32_t)TCWB, (cuuint32_t)TCHB};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.x), dims, strides, box,
               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_tc(const ConvArgs& a, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    static int max_clusters = 0;         // co-resident clusters of the folding kernel
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)TcSmem<0>::SMEM);
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(conv_tc_fold_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)TcSmem<1>::SMEM);
        if (attr == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2 * (sm_count() / 2));
            cfg.blockDim = dim3(TCTHREADS);
            cfg.dynamicSmemBytes = TcSmem<1>::SMEM;
            attr = cudaOccupancyMaxActiveClusters(&max_clusters, conv_tc_fold_kernel, &cfg);
        }
        if (max_clusters < 1) max_clusters = 1;
    });
    if (attr != cudaSuccess) return attr;
    CUtensorMap map;
    if (!make_tc_map(a, &map)) return cudaErrorInvalidValue;
    const bool vec3 = a.mode == CONV_SPLIT3 && (reinterpret_cast<uintptr_t>(a.planes) & 15) == 0 &&
                      a.ld % 8 == 0 && a.plane_stride % 8 == 0;
    const int nty = (a.n1 + TCM - 1) / TCM;
    count_launch();
    if (a.fold) {
        const int h = (a.n2 + 1) / 2;
        const int ncp = (h + TCW - 1) / TCW, nunits = ncp * nty;
        const int ncl = nunits < max_clusters ? nunits : max_clusters;
        return launch_pdl(conv_tc_fold_kernel, dim3(2 * ncl), dim3(TCTHREADS), TcSmem<1>::SMEM, s,
                          map, a, a.tcplan, ncp, nunits, vec3 ? 1 : 0);
    }
    const int ntx = (a.n2 + TCW - 1) / TCW, ntiles = ntx * nty;
    const int grid = ntiles < sm_count() ? ntiles : sm_count();
    return launch_pdl(conv_tc_kernel, dim3(grid), dim3(TC_TILE_THREADS), TcSmem<0>::SMEM, s, map,
                      a, a.tcplan, ntx, ntiles, vec3 ? 1 : 0);
}

// ------------------------------------------------ batched stencils -------
// Both stencils of one restoration iteration for many images in one persistent
// launch: the residual blur r_j = g_j - A_j x_j of every image, then its
// reblur z_j = A'_j r_j (written as the transform operand, or x_j += tau z_j in
// plain mode).  Work items are single tiles, listed blur tiles first (largest
// images first), then the reblur tiles in the same order; a device counter
// hands them out.  A reblur tile of image j reads r_j around its tile, so it
// waits (bounded) until every blur tile of image j is done: each finished blur
// tile is published with a release increment of its image's counter, which the
// reblur's loader acquires before it issues the TMA copy.  Items are taken in
// list order, so every blur tile a waiting CTA depends on was taken earlier by
// a running CTA that needs nothing to finish it: the waits cannot deadlock.
// Each image has its own PSF support q (the tile code is instantiated for
// q = 0..15 and chosen per item) and its own TMA maps with a halo box for its q.
struct ConvJob {
    CUtensorMap mx;          // blur input x_j, halo box of (q, G)
    CUtensorMap mr;          // reblur input r_j
    ConvArgs blur, reblur;
    int q, ntx, ntiles;
    int ncp, nunits;         // folded reblur: column pairs per row band, work units
};

template <int Q, class G>
__device__ __forceinline__ void group_tile(const ConvArgs& a, float* box, float* coef, int r0,
                                           int c0, int tid) {
    constexpr int PADL = (Q + 3) & ~3;
    constexpr int WB = TX + 2 * PADL;
    load_coefs<Q>(a, coef, tid, TX * G::TY);
    __syncthreads();
    float* tile = box + (PADL - Q);
    if (r0 - Q < 0 || r0 + G::TH + Q > a.n1 || c0 - Q < 0 || c0 + TX + Q > a.n2)
        fixup_tile<Q, G>(a, tile, WB, r0, c0, tid, TX * G::TY);
    if (a.mode == CONV_RESIDUAL || a.mode == CONV_AXPY)
        compute_tile<Q, true, G>(a, tile, WB, coef, r0, c0);
    else
        compute_tile<Q, false, G>(a, tile, WB, coef, r0, c0);
}

// A folded reblur unit: the tile at columns [c0, c0 + 64) (box A) and its mirror
// at [cm, cm + 64), cm = n2 - c0 - 64 (box B), by the whole CTA one after the
// other; column c0 + j pairs with column 63 - j of the mirror.  Writes the
// bf16x3 split of y+_t = y_t + y_{n2-1-t} at column t and y-_t at Kh + t
// (t = c0 + j), zeros past ceil(n2/2) resp. floor(n2/2), as the single-image
// folding reblur.
template <int Q, class G>
__device__ __forceinline__ void group_fold_unit(const ConvArgs& a, float* boxA, float* boxB,
                                                float* coef, int r0, int c0, int tid) {
    constexpr int PADL = (Q + 3) & ~3;
    constexpr int WB = TX + 2 * PADL, RS = G::RS;
    const int cm = a.n2 - c0 - TX;
    load_coefs<Q>(a, coef, tid, TX * G::TY);
    __syncthreads();
    float* ta = boxA + (PADL - Q);
    float* tb = boxB + (PADL - Q);
    const bool rows_out = r0 - Q < 0 || r0 + G::TH + Q > a.n1;
    if (rows_out || c0 - Q < 0 || c0 + TX + Q > a.n2) fixup_tile<Q, G>(a, ta, WB, r0, c0, tid, TX * G::TY);
    if (rows_out || cm - Q < 0 || cm + TX + Q > a.n2) fixup_tile<Q, G>(a, tb, WB, r0, cm, tid, TX * G::TY);
    const int tx = threadIdx.x, ty = threadIdx.y;
    float acc[RS];
    tile_acc<Q, G>(ta, WB, coef, tx, ty, acc);
    __syncthreads();                     // box A consumed: it takes A's results
#pragma unroll
    for (int r = 0; r < RS; ++r) boxA[(ty * RS + r) * TX + tx] = acc[r];
    tile_acc<Q, G>(tb, WB, coef, tx, ty, acc);
    __syncthreads();                     // box B consumed: it takes B's results
#pragma unroll
    for (int r = 0; r < RS; ++r) boxB[(ty * RS + r) * TX + tx] = acc[r];
    __syncthreads();
    const int h = (a.n2 + 1) / 2, ha = a.n2 / 2, kh = (h + 63) / 64 * 64;
    const int t = c0 + tx;
#pragma unroll
    for (int r = 0; r < RS; ++r) {
        const int rr = ty * RS + r, row = r0 + rr;
        if (row >= a.n1 || t >= kh) continue;
        const float va = boxA[rr * TX + tx], vb = boxB[rr * TX + (TX - 1 - tx)];
        split3_store(a.planes, a.plane_stride, (size_t)row * a.ld + t, t < h ? va + vb : 0.f);
        split3_store(a.planes, a.plane_stride, (size_t)row * a.ld + kh + t, t < ha ? va - vb : 0.f);
    }
}

template <class G>
__device__ __forceinline__ void group_fold_dispatch(int q, const ConvArgs& a, float* boxA,
                                                    float* boxB, float* coef, int r0, int c0,
                                                    int tid) {
    switch (q) {
        case 0: group_fold_unit<0, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 1: group_fold_unit<1, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 2: group_fold_unit<2, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 3: group_fold_unit<3, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 4: group_fold_unit<4, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 5: group_fold_unit<5, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 6: group_fold_unit<6, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 7: group_fold_unit<7, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 8: group_fold_unit<8, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 9: group_fold_unit<9, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 10: group_fold_unit<10, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 11: group_fold_unit<11, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 12: group_fold_unit<12, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 13: group_fold_unit<13, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        case 14: group_fold_unit<14, G>(a, boxA, boxB, coef, r0, c0, tid); break;
        default: group_fold_unit<15, G>(a, boxA, boxB, coef, r0, c0, tid); break;
    }
}

template <class G>
__device__ __forceinline__ void group_dispatch(int q, const ConvArgs& a, float* box, float* coef,
                                               int r0, int c0, int tid) {
    switch (q) {
        case 0: group_tile<0, G>(a, box, coef, r0, c0, tid); break;
        case 1: group_tile<1, G>(a, box, coef, r0, c0, tid); break;
        case 2: group_tile<2, G>(a, box, coef, r0, c0, tid); break;
        case 3: group_tile<3, G>(a, box, coef, r0, c0, tid); break;
        case 4: group_tile<4, G>(a, box, coef, r0, c0, tid); break;
        case 5: group_tile<5, G>(a, box, coef, r0, c0, tid); break;
        case 6: group_tile<6, G>(a, box, coef, r0, c0, tid); break;
        case 7: group_tile<7, G>(a, box, coef, r0, c0, tid); break;
        case 8: group_tile<8, G>(a, box, coef, r0, c0, tid); break;
        case 9: group_tile<9, G>(a, box, coef, r0, c0, tid); break;
        case 10: group_tile<10, G>(a, box, coef, r0, c0, tid); break;
        case 11: group_tile<11, G>(a, box, coef, r0, c0, tid); break;
        case 12: group_tile<12, G>(a, box, coef, r0, c0, tid); break;
        case 13: group_tile<13, G>(a, box, coef, r0, c0, tid); break;
        case 14: group_tile<14, G>(a, box, coef, r0, c0, tid); break;
        default: group_tile<15, G>(a, box, coef, r0, c0, tid); break;
    }
}

// Polls of a reblur tile's wait for its image's blur tiles (each poll sleeps
// about 0.1 us: about 0.4 s in all).
constexpr uint32_t kDepPolls = 1u << 22;

// ctr[0]: the queue's next item; ctr[1 + j]: finished blur tiles of image j
// (zero at launch); buf: bytes of one halo buffer (the largest q's box).
template <class G>
__global__ void __launch_bounds__(TX * G::TY)
conv_group_kernel(const ConvJob* __restrict__ jobs, const int2* __restrict__ items, int nblur,
                  int nitems, int* __restrict__ ctr, int iter, uint32_t buf) {
    using namespace tc;
    extern __shared__ __align__(128) uint8_t smem_raw_c[];
    uint8_t* sbase = smem_raw_c + ((128u - (smem_u32(smem_raw_c) & 127u)) & 127u);
    float* coef = reinterpret_cast<float*>(sbase + 2 * buf);
    const uint32_t bar0 = smem_u32(coef + Coefs<QMAX_FAST>::COUNT);   // two mbarriers
    volatile int* slot = reinterpret_cast<volatile int*>(coef + Coefs<QMAX_FAST>::COUNT + 4);
    const int tid = threadIdx.y * TX + threadIdx.x;
    auto box = [&](int b) { return reinterpret_cast<float*>(sbase + b * buf); };
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8u, 1);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();                          // x_j and the planes come from the previous kernels
    const uint32_t polls = g_conv_wait_polls;
    bool req[2] = {false, false};        // thread 0: a copy on barrier b is in flight / landed
    // a folded reblur unit takes both buffers (its tile and the mirror tile), so
    // it is never prefetched and nothing is prefetched beside it
    auto is_fold = [&](int item) { return item >= nblur && jobs[items[item].x].reblur.fold; };
    auto request = [&](int item, int b) {
        const int2 w = items[item];
        const ConvJob& J = jobs[w.x];
        const int padl = (J.q + 3) & ~3;
        const uint32_t bytes = (uint32_t)(TX + 2 * padl) * (uint32_t)(G::TH + 2 * J.q) * 4u;
        fence_proxy_async_smem();        // generic writes to the buffers (fix-up) before the copy
        if (is_fold(item)) {
            const int r0 = (w.y / J.ncp) * G::TH, c0 = (w.y % J.ncp) * TX;
            const int cm = J.reblur.n2 - c0 - TX;
            mbar_arrive_expect_tx(bar0 + 8u * b, 2u * bytes);
            tma_load_2d(smem_u32(box(0)), &J.mr, c0 - padl, r0 - J.q, bar0 + 8u * b);
            tma_load_2d(smem_u32(box(1)), &J.mr, cm - padl, r0 - J.q, bar0 + 8u * b);
        } else {
            const int r0 = (w.y / J.ntx) * G::TH, c0 = (w.y % J.ntx) * TX;
            mbar_arrive_expect_tx(bar0 + 8u * b, bytes);
            tma_load_2d(smem_u32(box(b)), item >= nblur ? &J.mr : &J.mx, c0 - padl, r0 - J.q,
                        bar0 + 8u * b);
        }
        req[b] = true;
    };
    auto ready = [&](int item) {         // a reblur tile's image has all its blur tiles done
        if (item < nblur) return true;
        const int j = items[item].x;
        return ld_acquire_gpu(ctr + 1 + j) >= jobs[j].ntiles;
    };
    if (tid == 0) {
        const int it = atomicAdd(ctr, 1);
        slot[0] = it;
        if (it < nitems && ready(it)) {
            fence_proxy_async_global();
            request(it, 0);
        }
        slot[2] = 0;
    }
    int li = 0;
    bool failed = false;
    for (;; ++li) {
        const int b = li & 1;
        __syncthreads();                 // slot[b] is set; buffer b ^ 1 and coef are free
        const int item = slot[b];
        if (item >= nitems) break;
        if (tid == 0) {
            if (!req[b]) {               // the image's blur tiles were not done at dequeue
                uint32_t i = 0;
                for (; i < kDepPolls && !ready(item); ++i) __nanosleep(100);
                if (i == kDepPolls) {
                    slot[2] = 1;
                } else {
                    fence_proxy_async_global();
                    request(item, b);
                }
            }
            if (!slot[2]) {              // the next item, prefetched when it can start
                const int nx = atomicAdd(ctr, 1);
                slot[b ^ 1] = nx;
                if (nx < nitems && !is_fold(item) && !is_fold(nx) && ready(nx)) {
                    fence_proxy_async_global();
                    request(nx, b ^ 1);
                }
            }
        }
        __syncthreads();
        if (slot[2]) {
            failed = true;
            break;
        }
        const bool ok = mbar_wait(bar0 + 8u * b, (li >> 1) & 1, polls);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (tid == 0) req[b] = false;
        const int2 w = items[item];
        const ConvJob& J = jobs[w.x];
        const bool re = item >= nblur;
        ConvArgs a = re ? J.reblur : J.blur;
        if (a.sumsq) a.sumsq += iter;
        if (re && a.fold) {
            const int r0 = (w.y / J.ncp) * G::TH, c0 = (w.y % J.ncp) * TX;
            group_fold_dispatch<G>(J.q, a, box(0), box(1), coef, r0, c0, tid);
        } else {
            const int r0 = (w.y / J.ntx) * G::TH, c0 = (w.y % J.ntx) * TX;
            group_dispatch<G>(J.q, a, box(b), coef, r0, c0, tid);
        }
        if (!re) {
            __syncthreads();             // the tile's r is written
            if (tid == 0) {
                __threadfence();
                red_release_add_gpu(ctr + 1 + w.x, 1);
            }
        }
    }
    pdl_trigger();
    if (failed && tid == 0) {
        atomicExch(&g_conv_timeout, 1);
        for (int k = 0; k < 2; ++k)      // copies still in flight (bounded)
            if (req[k]) mbar_wait(bar0 + 8u * k, ((li + ((k - li) & 1)) >> 1) & 1);
    }
}

}  // namespace

int* conv_error_flag() {
    static int* p[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!p[dev]) {
        void* q = nullptr;
        if (cudaGetSymbolAddress(&q, g_conv_timeout) == cudaSuccess) p[dev] = static_cast<int*>(q);
    }
    return p[dev];
}

// ------------------------------------------------ batched stencils (host) --
namespace {

// TMA map of a float32 n1 x n2 image with the halo box of support q, geometry G.
bool make_box_map(const float* img, int n1, int n2, int q, int th, CUtensorMap* map) {
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!enc) return false;
    const int padl = (q + 3) & ~3;
    cuuint64_t dims[2] = {(cuuint64_t)n2, (cuuint64_t)n1};
    cuuint64_t strides[1] = {(cuuint64_t)n2 * 4};
    cuuint32_t box[2] = {(cuuint32_t)(TX + 2 * padl), (cuuint32_t)(th + 2 * q)};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(img), dims, strides, box,
               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

uint32_t box_bytes(int q, int th) {
    const int padl = (q + 3) & ~3;
    return ((uint32_t)(TX + 2 * padl) * (uint32_t)(th + 2 * q) * 4u + 127u) & ~127u;
}

template <class G>
cudaError_t group_attr(size_t smem, int* per_sm) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(conv_group_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    96 * 1024);
    });
    if (attr != cudaSuccess) return attr;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, conv_group_kernel<G>,
                                                         TX * G::TY, smem);
}

}  // namespace

struct ConvGroup {
    int geometry = 0, count = 0, nblur = 0, nitems = 0, grid = 0, iters = 0, stride = 0;
    int ctas_per_sm = 0;
    uint32_t buf = 0;
    size_t smem = 0;
    ConvJob* jobs = nullptr;
    int2* items = nullptr;
    int* ctr = nullptr;
};

void conv_group_destroy(ConvGroup* g) {
    if (!g) return;
    cudaFree(g->jobs);
    cudaFree(g->items);
    cudaFree(g->ctr);
    delete g;
}

int conv_group_ctas_per_sm(const ConvGroup* g) { return g->ctas_per_sm; }

ar_status conv_group_create(const ConvArgs* blurs, const ConvArgs* reblurs, int count, int geometry,
                            int ctas_per_sm, int iters, ConvGroup** out) {
    if (count < 1 || iters < 1 || (geometry != 0 && geometry != 1) || ctas_per_sm < 1)
        return fail(AR_ERR_INVALID_ARG, "batched stencil: count %d, iters %d, geometry %d", count,
                    iters, geometry);
    const int th = geometry == 0 ? G64::TH : G54::TH;
    std::vector<ConvJob> jobs((size_t)count);
    std::vector<double> cost((size_t)count);
    int qmax = 0;
    for (int j = 0; j < count; ++j) {
        const ConvArgs& b = blurs[j];
        const ConvArgs& r = reblurs[j];
        const int q = b.q1 > b.q2 ? b.q1 : b.q2;
        if (q > QMAX_FAST || b.bc == AR_BC_PERIODIC || (b.n2 & 3) != 0 ||
            (reinterpret_cast<uintptr_t>(b.x) & 15) != 0 || (reinterpret_cast<uintptr_t>(r.x) & 15) != 0 ||
            b.mode != CONV_RESIDUAL || (r.fold && r.mode != CONV_SPLIT3))
            return fail(AR_ERR_UNSUPPORTED,
                        "batched stencil: image %d needs q <= 15, n2 %% 4 == 0, aligned rows "
                        "and a non-periodic BC", j);
        ConvJob& J = jobs[(size_t)j];
        std::memset(&J, 0, sizeof(J));
        J.blur = b;
        J.reblur = r;
        J.q = q;
        J.ntx = (b.n2 + TX - 1) / TX;
        J.ntiles = J.ntx * ((b.n1 + th - 1) / th);
        J.ncp = ((b.n2 + 1) / 2 + TX - 1) / TX;
        J.nunits = J.ncp * ((b.n1 + th - 1) / th);
        if (!make_box_map(b.x, b.n1, b.n2, q, th, &J.mx) || !make_box_map(r.x, r.n1, r.n2, q, th, &J.mr))
            return fail(AR_ERR_CUDA, "batched stencil: tensor map of image %d", j);
        cost[(size_t)j] = (double)b.n1 * b.n2 * (2 * q + 1) * (2 * q + 1);
        qmax = q > qmax ? q : qmax;
    }
    // largest images first (the longest work first balances the tail), blur then reblur
    std::vector<int> order((size_t)count);
    for (int j = 0; j < count; ++j) order[(size_t)j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[(size_t)a] > cost[(size_t)b]; });
    std::vector<int2> items;
    for (int j : order)                                   // blur tiles
        for (int t = 0; t < jobs[(size_t)j].ntiles; ++t) items.push_back(make_int2(j, t));
    const int nblur = (int)items.size();
    for (int j : order) {                                 // reblur tiles, or folded units
        const ConvJob& J = jobs[(size_t)j];
        const int n = J.reblur.fold ? J.nunits : J.ntiles;
        for (int t = 0; t < n; ++t) items.push_back(make_int2(j, t));
    }
    ConvGroup* g = new (std::nothrow) ConvGroup();
    if (!g) return fail(AR_ERR_ALLOC, "host allocation of the batched stencil");
    g->geometry = geometry;
    g->count = count;
    g->nitems = (int)items.size();
    g->nblur = nblur;
    g->iters = iters;
    g->stride = 1 + count;
    g->buf = box_bytes(qmax, th);
    g->smem = 2 * (size_t)g->buf + (size_t)Coefs<QMAX_FAST>::COUNT * 4 + 64 + 128;
    int per_sm = 0;
    cudaError_t e = geometry == 0 ? group_attr<G64>(g->smem, &per_sm) : group_attr<G54>(g->smem, &per_sm);
    if (e != cudaSuccess || per_sm < 1) {
        conv_group_destroy(g);
        return e != cudaSuccess ? cuda_fail(e, "batched stencil occupancy")
                                : fail(AR_ERR_UNSUPPORTED, "batched stencil does not fit an SM");
    }
    g->ctas_per_sm = ctas_per_sm < per_sm ? ctas_per_sm : per_sm;
    const int cap = g->ctas_per_sm * sm_count();
    g->grid = g->nitems < cap ? g->nitems : cap;
    e = cudaMalloc((void**)&g->jobs, jobs.size() * sizeof(ConvJob));
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->items, items.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->ctr, (size_t)iters * g->stride * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(g->jobs, jobs.data(), jobs.size() * sizeof(ConvJob), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(g->ctr, 0, (size_t)iters * g->stride * sizeof(int));
    if (e != cudaSuccess) {
        conv_group_destroy(g);
        return cuda_fail(e, "batched stencil buffers");
    }
    *out = g;
    return AR_OK;
}

ar_status conv_group_reset(ConvGroup* g, cudaStream_t s) {
    AR_CUDA(cudaMemsetAsync(g->ctr, 0, (size_t)g->iters * g->stride * sizeof(int), s));
    return AR_OK;
}

ar_status conv_group_apply(ConvGroup* g, int iter, cudaStream_t s) {
    if (iter < 0 || iter >= g->iters) return fail(AR_ERR_INVALID_ARG, "iteration %d of %d", iter, g->iters);
    ProfScope prof(AR_PROF_STENCIL, s);
    count_launch();
    int* ctr = g->ctr + (size_t)iter * g->stride;
    cudaError_t e;
    if (g->geometry == 0)
        e = launch_pdl(conv_group_kernel<G64>, dim3(g->grid), dim3(TX, G64::TY), g->smem, s,
                       (const ConvJob*)g->jobs, (const int2*)g->items, g->nblur, g->nitems, ctr,
                       iter, g->buf);
    else
        e = launch_pdl(conv_group_kernel<G54>, dim3(g->grid), dim3(TX, G54::TY), g->smem, s,
                       (const ConvJob*)g->jobs, (const int2*)g->items, g->nblur, g->nitems, ctr,
                       iter, g->buf);
    if (e != cudaSuccess) return cuda_fail(e, "batched stencil launch");
    return AR_OK;
}

ar_status conv_set_wait_polls(unsigned polls) {
    AR_CUDA(cudaMemcpyToSymbol(g_conv_wait_polls, &polls, sizeof(polls)));
    return AR_OK;
}

ar_status conv_tc_plan(const float* psf, int q1, int q2, int flip, uint8_t* plan,
                       cudaStream_t s) {
    if (q1 > TCQ || q2 > TCQ || q1 < 0 || q2 < 0)
        return fail(AR_ERR_UNSUPPORTED, "tensor-core stencil plans take q <= %d", TCQ);
    count_launch();
    conv_tc_plan_kernel<<<dim3(TCU, 2), TCTHREADS, 0, s>>>(psf, q1, q2, flip, plan);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core stencil plan");
    return AR_OK;
}

bool conv_tc_applies(const ConvArgs& a) {
    // the epilogue moves 16-byte vectors of x, the output and the mode's inputs
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    return a.q1 <= TCQ && a.q2 <= TCQ && a.bc != AR_BC_PERIODIC && (a.n2 & 3) == 0 && al(a.x) &&
           al(a.out) && al(a.aux) && al(a.f);
}

ar_status conv_launch(const ConvArgs& a, cudaStream_t s) {
    if (a.n1 <= 0 || a.n2 <= 0) return AR_OK;
    ProfScope prof(AR_PROF_STENCIL, s);
    if (a.tcplan && conv_tc_applies(a)) {
        const cudaError_t e = launch_tc(a, s);
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core stencil launch");
        return AR_OK;
    }
    const int q = a.q1 > a.q2 ? a.q1 : a.q2;
    if (a.fold && q > QMAX_FAST) return fail(AR_ERR_UNSUPPORTED, "folded output needs q <= 15");
    cudaError_t e;
    switch (q) {
        case 0: e = launch_fast<0>(a, s); break;
        case 1: e = launch_fast<1>(a, s); break;
        case 2: e = launch_fast<2>(a, s); break;
        case 3: e = launch_fast<3>(a, s); break;
        case 4: e = launch_fast<4>(a, s); break;
        case 5: e = launch_fast<5>(a, s); break;
        case 6: e = launch_fast<6>(a, s); break;
        case 7: e = launch_fast<7>(a, s); break;
        case 8: e = launch_fast<8>(a, s); break;
        case 9: e = launch_fast<9>(a, s); break;
        case 10: e = launch_fast<10>(a, s); break;
        case 11: e = launch_fast<11>(a, s); break;
        case 12: e = launch_fast<12>(a, s); break;
        case 13: e = launch_fast<13>(a, s); break;
        case 14: e = launch_fast<14>(a, s); break;
        case 15: e = launch_fast<15>(a, s); break;
        default: {
            dim3 grid((a.n2 + 31) / 32, (a.n1 + 7) / 8);
            conv_generic_kernel<<<grid, dim3(32, 8), 0, s>>>(a);
            count_launch();
            e = cudaGetLastError();
        }
    }
    static_assert(QMAX_FAST == 15, "dispatch table covers 0..15");
    if (e != cudaSuccess) return cuda_fail(e, "conv kernel launch");
    return AR_OK;
}

}  // namespace ar
