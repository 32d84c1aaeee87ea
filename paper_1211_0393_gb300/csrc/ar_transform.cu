// The AR transform pair of Theorem 1 applied as dense tensor-core contractions.
//
// D y = T_n diag(d) T~_n y with T_n = T_{n1} (x) T_{n2} becomes, for an image Y,
//     D Y = T_{n1} ( d o (T~_{n1} Y T~_{n2}^T) ) T_{n2}^T,
// four dense products.  The transforms are used without the normalisation
// alpha_m of Theorem 1 (it cancels between T and T~):
//     T~'_m = [[1, 0, 0], [-Q p, Q, -Q J p], [0, 0, 1]]
//     T'_m  = [[1, 0, 0], [  p,  Q,    J p], [0, 0, 1]]
// with Q = Q_{m-2} of eq. Qn and p_j = 1 - j/(m-1); they are generated in
// float64 on the GPU.
//
// Every product is C = A B^T with both operands K-major, stored transposed,
// so the chain needs no explicit transposes:
//   G1: U^T <- (Y T~2^T)^T        A = Y   (n1 x n2)   B = T~2
//   G2: W   <- d o (U^T T~1^T)^T  A = U^T (n2 x n1)   B = T~1
//   G3: V^T <- (W T2^T)^T         A = W               B = T2
//   G4: out <- (V^T T1^T)^T       (or out += tau * ...)
//
// The comparison BCs use the same chain with other constant operands: the
// Reflective preconditioner (DCT-III, eq. Rn) takes T~ = R^T and T = R; the
// Periodic one (a circulant) is applied in the real separable Hartley basis
// with three more products (see transform_apply).
//
// Precision: each operand x is split into three bfloat16 planes
// x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1)),
// and the six products a_i b_j with i + j <= 2 are accumulated in float32 in
// tensor memory.  The dropped terms are below 2^-24 relative, so the
// contraction is as accurate as a float32 one.
//
// Kernel: one 128 x 128 output tile per pair of CTAs (a cluster of two that
// splits K in halves; tcgen05.mma M = 128, K = 16, with N = 256 over the
// back-to-back B planes b0 b1 where a product pair shares its A plane; four
// TMEM accumulators in two pairs taking the k-blocks in turn), operands staged
// by TMA (one 3D box loads the planes of a 64-byte-swizzled K-major tile of 32
// columns), a 4-stage (6 in the two-plane mode) mbarrier pipeline between a
// TMA producer thread and an MMA issuer thread, and an epilogue in which each
// CTA sends the peer's half of its partial tile through distributed shared
// memory, adds the half it receives, and writes its half transposed
// (coalesced along the tile's M index) with the next step fused: the bf16x3
// split of the next operand, the filter d, or x += tau * result.  Full-rate
// MMA at M = 128 needs N >= 128: with smaller N the six products' operand
// reads exceed the shared-memory bandwidth.
//
// For AR the chain runs on the even/odd folds of both axes (see transform_apply):
// every product is block diagonal in K, so a tile reads half of K.  G4 also folds
// its N index: tc_contract_pair_kernel runs clusters of four CTAs (the split-K
// pair times the two parities of N), whose parity tiles swap their sums and
// differences through distributed shared memory before the unfolding epilogue.

#include "ar_internal.cuh"
#include "ar_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <utility>

namespace ar {
namespace {

// K-blocks of 32 (64-byte rows, 64-byte swizzle): small stages let more of the
// shared memory be in flight while the tensor core reads one stage.
constexpr int BM = 128, BN = 128, BK = 32;
constexpr int MAX_PLANES = 3;                             // operand buffers hold three bf16 planes
constexpr uint32_t A_PLANE = BM * BK * 2;                 // 8 KiB
constexpr uint32_t B_PLANE = BN * BK * 2;                 // 8 KiB
// Split-K over the two CTAs of a cluster: CTA r accumulates its half of the
// k-blocks, then finishes columns [r*HALF, (r+1)*HALF) of the tile after
// receiving the peer's partial sums for them through distributed shared memory.
constexpr int SPLITK = 2;
constexpr int HALF = BN / SPLITK;
constexpr uint32_t RECV_BYTES = HALF * BM * 4;            // 32 KiB, column-major [HALF][BM]
// The products are spread over NACC accumulators of BN columns each (two
// pairs, alternating by k-block; within a pair the b0 and b1 products go to
// different halves), summed with round-to-nearest float32 adds in the
// epilogue: the tensor core's float32 accumulation loses up to an ulp per
// accumulate step, so fewer steps per accumulator keep a K = 1024 contraction
// at float32-grade accuracy.
constexpr int NACC = 4;
constexpr uint32_t TMEM_COLS = NACC * BN;                 // 512: the whole TMEM of the SM

// Precision modes.  NP = 3: three bf16 planes per operand, the six products
// a_i b_j with i + j <= 2 (float32-grade), four 48 KiB stages.  NP = 2: two
// planes, the three products with i + j <= 1 (about 2^-16 relative), six
// 32 KiB stages.
template <int NP>
struct TcMode {
    static constexpr int PLANES = NP;
    static constexpr int STAGES = NP == 3 ? 4 : 6;
    static constexpr uint32_t A_STAGE = PLANES * A_PLANE;
    static constexpr uint32_t B_STAGE = PLANES * B_PLANE;
    static constexpr uint32_t STAGE_BYTES = A_STAGE + B_STAGE;   // 48 KiB / 32 KiB
    static constexpr uint32_t CTRL_BYTES = 8 * (2 * STAGES + 2) + 16;
    static constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + RECV_BYTES + CTRL_BYTES + 1024;
};
static_assert(TcMode<3>::SMEM_BYTES <= 232448 && TcMode<2>::SMEM_BYTES <= 232448, "smem budget");

enum TcEpi : int { TE_SPLIT_T = 0, TE_SCALE_SPLIT_T = 1, TE_STORE_T = 2, TE_AXPY_T = 3 };

struct TcEpiArgs {
    int mode;
    uint16_t* planes;      // split output: planes[p * pstride + col * ld + row]
    size_t pstride;
    int ld;
    float* out;            // float32 output: out[col * ldo + row]
    int ldo;
    const float* d;        // filter: d[col * ldd + row]
    int ldd;
    float tau;
    const float* f;        // TE_AXPY_T: true image (same layout as out) or null
    double* sumsq;         // TE_AXPY_T with f: += sum (x_new - f)^2
    // Folded (even/odd) transforms.  kdiag: A and B are block diagonal in K, so
    // the output columns of the first half of N use the first half of K and
    // the others the second half.  pair: the 128 rows of an A tile are two
    // 64-row boxes, row r paired with row 64 + r of the tile:
    //   PAIR_MIRROR: boxes at rows m0 and mrows - m0 - 64 (row i with row
    //     mrows - 1 - i); the output is the even/odd fold of the M index, the
    //     sums (i < npair) and differences (i < nminus, at column kout + i);
    //   PAIR_HALVES: boxes at rows m0 and mhalf + m0 (row j of the first half
    //     with row j of the second); the output is the unfold, row j gets
    //     first + second (j < npair), row nout - 1 - j first - second (j < nminus).
    int kdiag;
    int pair;
    int mrows, mhalf, npair, nminus, kout, nout;
    // npar: the N index is folded too (B block diagonal, its first nhalf rows the
    // sums and the others the differences of the output columns s and noutn - 1 - s):
    // a cluster of four CTAs pairs the tiles at n and nhalf + n, which swap their
    // results through distributed shared memory; column s gets sum + difference
    // (s < npairn), column noutn - 1 - s sum - difference (s < nminusn)
    int npar;
    int nhalf, npairn, nminusn, noutn;
    // late_trigger: the successor may launch only once this grid's epilogues are
    // done (it is a stencil, whose CTAs would otherwise crowd the SMs that this
    // grid leaves idle); else it may launch as soon as the accumulators are ready
    int late_trigger;
};

enum TcPair : int { PAIR_NONE = 0, PAIR_MIRROR = 1, PAIR_HALVES = 2 };

__device__ __forceinline__ void split3(float v, uint16_t& h0, uint16_t& h1, uint16_t& h2) {
    const __nv_bfloat16 p0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(p0);
    const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
    h0 = __bfloat16_as_ushort(p0);
    h1 = __bfloat16_as_ushort(p1);
    h2 = __bfloat16_as_ushort(p2);
}

// Sum of the first `nacc` accumulators at 16 consecutive columns (zeros if none).
__device__ __forceinline__ void acc_sum16(uint32_t trow, int col0, int nacc, float (&v)[16]) {
    using namespace tc;
    float a[16], b[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = 0.f;
    if (nacc <= 0) return;
    tmem_ld16x2(trow + col0, trow + BN + col0, a, b);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = nacc > 1 ? a[j] + b[j] : a[j];
    if (nacc <= 2) return;
    tmem_ld16x2(trow + 2 * BN + col0, trow + 3 * BN + col0, a, b);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = nacc > 3 ? (v[j] + a[j]) + b[j] : v[j] + a[j];
}

constexpr int NTHREADS = 256;           // 8 warps: two per TMEM lane quarter in the epilogue
constexpr int WCOLS = HALF / 2;         // columns of the CTA's half handled by one warp

// The body of both contraction kernels: clusters of (1, 1, SPLITK) CTAs, or
// (1, 2, SPLITK) with the parity pairs of N (NPAR, ep.npar set).
// (bx, by) is the tile of the launch grid this cluster computes (blockIdx.x,
// blockIdx.y in a plain launch; a work item's tile in a grouped one).
template <int NP, bool NPAR>
__device__ __forceinline__ void tc_contract_body(const CUtensorMap& tmA, const CUtensorMap& tmA64,
                                                 const CUtensorMap& tmB, const CUtensorMap& tmO,
                                                 int M, int N, int K, const TcEpiArgs& ep, int* err,
                                                 int bx, int by) {
    using namespace tc;
    using Mode = TcMode<NP>;
    constexpr int STAGES = Mode::STAGES;
    constexpr uint32_t A_STAGE = Mode::A_STAGE;
    constexpr uint32_t STAGE_BYTES = Mode::STAGE_BYTES;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;         // swizzled tiles need 512 B alignment
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t recv = base + STAGES * STAGE_BYTES;
    const float* recv_ptr = reinterpret_cast<const float*>(gbase + STAGES * STAGE_BYTES);
    const uint32_t bars = recv + RECV_BYTES;
    const uint32_t done_bar = bars + 8u * (2 * STAGES);
    const uint32_t issued_bar = bars + 8u * (2 * STAGES + 1);   // the last MMA was issued
    uint32_t* tslot = reinterpret_cast<uint32_t*>(gbase + STAGES * STAGE_BYTES + RECV_BYTES +
                                                  8 * (2 * STAGES + 2));
    volatile int* sflag = reinterpret_cast<volatile int*>(tslot + 1);
    // after the main loop the stage area stages the split output tile [NP][HALF][BM]
    uint16_t* stage_out = reinterpret_cast<uint16_t*>(gbase);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, sub = warp >> 2;
    // cluster ranks run x fastest: (cy, cz) is rank cy + 2 cz with NPAR, cz without
    const uint32_t crank = cluster_ctarank();
    const uint32_t ks = NPAR ? crank >> 1 : crank;                // split-K half
    const uint32_t kpeer = NPAR ? crank ^ 2u : crank ^ 1u;        // the other split-K half
    const int parity = NPAR ? (int)(crank & 1u) : 0;
    const int m0 = bx * (ep.pair ? BM / 2 : BM);
    const int n0 = NPAR ? (by >> 1) * BN + parity * ep.nhalf : by * BN;
    // with NPAR the cluster is (1, 2, SPLITK): checked, not assumed
    const bool rank_ok = !NPAR || (cluster_ctaid_y() == (blockIdx.y & 1u) &&
                                   cluster_ctaid_z() == blockIdx.z &&
                                   crank == (blockIdx.y & 1u) + 2u * blockIdx.z);
    int nk_all = (K + BK - 1) / BK, kb0 = 0;
    if (ep.kdiag) {                      // block-diagonal operands: this tile's half of K
        nk_all /= 2;
        if (n0 >= N / 2) kb0 = nk_all;
    }
    const int nk_first = (nk_all + 1) / 2;
    const int kb_begin = kb0 + (ks == 0 ? 0 : nk_first);
    const int nk = ks == 0 ? nk_first : nk_all - nk_first;
    // A tile of k-block kb into dst: one 3D box, or two 64-row boxes per plane
    auto load_a = [&](uint32_t dst, int kb, uint32_t bar) {
        if (!ep.pair) {
            tma_load_3d(dst, &tmA, kb * BK, m0, 0, bar);
            return;
        }
        const int r2 = ep.pair == PAIR_MIRROR ? ep.mrows - m0 - BM / 2 : ep.mhalf + m0;
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) {
            tma_load_3d(dst + pl * A_PLANE, &tmA64, kb * BK, m0, pl, bar);
            tma_load_3d(dst + pl * A_PLANE + (BM / 2) * BK * 2, &tmA64, kb * BK, r2, pl, bar);
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bars + 8u * s, 1);                 // full[s]: TMA bytes landed
            mbar_init(bars + 8u * (STAGES + s), 1);      // empty[s]: MMAs reading it done
        }
        mbar_init(done_bar, 1);
        mbar_init(issued_bar, 1);
        *sflag = 0;
        fence_mbar_init();
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tslot), TMEM_COLS);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer.  The constant B operand of the first stages is
        // requested before waiting for the previous kernel, which writes A.
        const int npre = nk < STAGES ? nk : STAGES;
        for (int kb = 0; kb < npre; ++kb) {
            const uint32_t a = base + kb * STAGE_BYTES;
            mbar_arrive_expect_tx(bars + 8u * kb, STAGE_BYTES);
            tma_load_3d(a + A_STAGE, &tmB, (kb_begin + kb) * BK, n0, 0, bars + 8u * kb);
        }
        pdl_wait();
        for (int kb = 0; kb < npre; ++kb)
            load_a(base + kb * STAGE_BYTES, kb_begin + kb, bars + 8u * kb);
        int issued = npre;
        for (int kb = npre; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait(bars + 8u * (STAGES + s), ((kb / STAGES) & 1) ^ 1)) {
                *sflag = 1;
                break;
            }
            if (*sflag) break;
            const uint32_t a = base + s * STAGE_BYTES;
            mbar_arrive_expect_tx(bars + 8u * s, STAGE_BYTES);
            load_a(a, kb_begin + kb, bars + 8u * s);
            tma_load_3d(a + A_STAGE, &tmB, (kb_begin + kb) * BK, n0, 0, bars + 8u * s);
            ++issued;
        }
        // no load may still be in flight when the CTA exits
        for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
            if (!mbar_wait(bars + 8u * (kb % STAGES), (kb / STAGES) & 1)) *sflag = 1;
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer.  The B planes b0 and b1 lie back to back in shared
        // memory, so one N = 256 MMA forms a_i b0 and a_i b1 into the two
        // halves of an accumulator pair; k-blocks alternate between two pairs
        // (the four accumulators of the epilogue).  Per 16-wide k slice:
        //   NP = 3: a1 [b0 b1], a2 b0 (first half), a0 b2 (second half), a0 [b0 b1]
        //   NP = 2: a0 [b0 b1], a1 b0 (first half)
        // The first MMA into a pair covers both halves and initialises them.
        const uint32_t idesc128 = idesc_bf16_f32(BM, BN);
        const uint32_t idesc256 = idesc_bf16_f32(BM, 2 * BN);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait(bars + 8u * s, (kb / STAGES) & 1)) {
                *sflag = 1;
                break;
            }
            fence_after_sync();
            const uint32_t a = base + s * STAGE_BYTES;
            const uint32_t b = a + A_STAGE;
            const uint32_t d0 = tmem + (uint32_t)(kb & 1) * (2 * BN);
            const uint32_t d1 = d0 + BN;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint32_t acc = (kb >= 2 || kk != 0) ? 1u : 0u;
                const uint64_t b0 = desc_k_sw64(b + kk * 32);
                if (NP == 3) {
                    mma_bf16(d0, desc_k_sw64(a + A_PLANE + kk * 32), b0, idesc256, acc);
                    mma_bf16(d0, desc_k_sw64(a + 2 * A_PLANE + kk * 32), b0, idesc128, 1u);
                    mma_bf16(d1, desc_k_sw64(a + kk * 32), desc_k_sw64(b + 2 * B_PLANE + kk * 32),
                             idesc128, 1u);
                    mma_bf16(d0, desc_k_sw64(a + kk * 32), b0, idesc256, 1u);
                } else {
                    mma_bf16(d0, desc_k_sw64(a + kk * 32), b0, idesc256, acc);
                    mma_bf16(d0, desc_k_sw64(a + A_PLANE + kk * 32), b0, idesc128, 1u);
                }
            }
            mma_commit(bars + 8u * (STAGES + s));        // frees the stage when its MMAs finish
        }
        // every operand has landed: the epilogue's own loads no longer compete with TMA
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(issued_bar) : "memory");
        if (nk > 0) {
            mma_commit(done_bar);                        // accumulators complete
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(done_bar) : "memory");
        }
    }

    // ---- epilogue.  Warp w reads TMEM lanes 32(w%4).. (tile rows m0 + 32(w%4) + lane) and
    // handles WCOLS of the CTA's HALF columns; its inputs are fetched while the MMAs run.
    const int lrow = quarter * 32 + lane;
    // output row of this thread's values: the tile row, or for the unfold the
    // row j = m0 + lrow (first half of the tile) or nout - 1 - j (second half)
    int row = m0 + lrow;
    bool row_ok = row < M;
    if (ep.pair == PAIR_HALVES) {
        const int j = m0 + (lrow & (BM / 2 - 1));
        row = lrow < BM / 2 ? j : ep.nout - 1 - j;
        row_ok = lrow < BM / 2 ? j < ep.npair : j < ep.nminus;
    }
    const int ocol0 = (int)ks * HALF + sub * WCOLS;           // tile-relative own columns
    const int pcol0 = (int)(ks ^ 1u) * HALF + sub * WCOLS;    // tile-relative peer columns
    // output column of tile column c (N index n0 + c) and whether it is written
    auto out_col = [&](int c, bool& valid) {
        const int n = n0 + c;
        if constexpr (!NPAR) {
            valid = n < N;
            return n;
        } else {
            const int sidx = n - parity * ep.nhalf;
            valid = sidx < (parity ? ep.nminusn : ep.npairn);
            return parity ? ep.noutn - 1 - sidx : sidx;
        }
    };

    float pre[WCOLS];
    float pref[WCOLS];
    // the filter / iterate / true-image tiles are fetched once the main loop's
    // operands are in (while the last MMAs run): earlier they slowed its TMA loads
    if (ep.mode == TE_SCALE_SPLIT_T || ep.mode == TE_AXPY_T) mbar_wait(issued_bar, 0);
#pragma unroll
    for (int j = 0; j < WCOLS; ++j) {
        bool cin;
        const int col = out_col(ocol0 + j, cin);
        const bool in = row_ok && cin;
        pre[j] = 0.f;
        pref[j] = 0.f;
        if (ep.mode == TE_SCALE_SPLIT_T) {
            if (in) pre[j] = __ldg(ep.d + (size_t)col * ep.ldd + row);
        } else if (ep.mode == TE_AXPY_T) {
            if (in) {
                pre[j] = ep.out[(size_t)col * ep.ldo + row];
                if (ep.f) pref[j] = __ldg(ep.f + (size_t)col * ep.ldo + row);
            }
        }
    }

    pdl_wait();                          // before this kernel writes what the previous one read
    const bool ready = mbar_wait(done_bar, 0);
    __syncwarp();
    fence_after_sync();
    if (!ep.late_trigger) pdl_trigger();
    const bool ok = ready && *sflag == 0 && rank_ok;
    const int nacc = ok ? (2 * nk < NACC ? 2 * nk : NACC) : 0;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);

    // 1) the peer's columns -> the peer's receive buffer [HALF / 4][BM][4]: a
    //    thread's four consecutive columns are one 16-byte store, a warp's 512
    //    contiguous bytes
    const uint32_t rrecv = mapa(recv, kpeer);
#pragma unroll
    for (int c = 0; c < WCOLS / 16; ++c) {
        float v[16];
        acc_sum16(trow, pcol0 + c * 16, nacc, v);
#pragma unroll
        for (int j = 0; j < 16; j += 4)
            st_cluster_v4(rrecv + 16u * (((sub * WCOLS + c * 16 + j) >> 2) * BM + lrow), v[j],
                          v[j + 1], v[j + 2], v[j + 3]);
    }
    cluster_sync();

    // 2) own columns: own partial sums + the peer's, then the fused next step
    const bool split_out = ep.mode == TE_SPLIT_T || ep.mode == TE_SCALE_SPLIT_T;
    float xv[WCOLS];
#pragma unroll
    for (int c = 0; c < WCOLS / 16; ++c) {
        float v[16];
        acc_sum16(trow, ocol0 + c * 16, nacc, v);
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
            const int hc = sub * WCOLS + c * 16 + j;    // column within the CTA's half
            const float4 r = reinterpret_cast<const float4*>(recv_ptr)[(hc >> 2) * BM + lrow];
            xv[c * 16 + j] = v[j] + r.x;
            xv[c * 16 + j + 1] = v[j + 1] + r.y;
            xv[c * 16 + j + 2] = v[j + 2] + r.z;
            xv[c * 16 + j + 3] = v[j + 3] + r.w;
        }
    }
    // paired rows: exchange through shared memory ([HALF][BM] float32 in the
    // stage area, the split output staged after it)
    float* xbuf = reinterpret_cast<float*>(gbase);
    uint16_t* stage = ep.pair ? stage_out + 2 * HALF * BM : stage_out;
    if (ep.pair) {
#pragma unroll
        for (int jj = 0; jj < WCOLS; ++jj) xbuf[(sub * WCOLS + jj) * BM + lrow] = xv[jj];
        __syncthreads();
        const int partner = ep.pair == PAIR_MIRROR ? BM - 1 - lrow : lrow ^ (BM / 2);
        const bool first = lrow < BM / 2;
#pragma unroll
        for (int jj = 0; jj < WCOLS; ++jj) {
            const float xp = xbuf[(sub * WCOLS + jj) * BM + partner];
            xv[jj] = first ? xv[jj] + xp : xp - xv[jj];
        }
    }
    if constexpr (NPAR) {
        // the parity pair: sums (parity 0) and differences (parity 1) of the same
        // columns swap through the partner's pipeline area past the pair buffer
        // ([HALF][BM] float32 at byte 4 HALF BM); every CTA of the cluster left its
        // main loop before the split-K barrier above, so that area is free
        const uint32_t pbuf = base + 4u * HALF * BM;
        const uint32_t prx = mapa(pbuf, crank ^ 1u);
#pragma unroll
        for (int jj = 0; jj < WCOLS; jj += 4)       // [HALF / 4][BM][4], as the split-K buffer
            st_cluster_v4(prx + 16u * (((sub * WCOLS + jj) >> 2) * BM + lrow), xv[jj], xv[jj + 1],
                          xv[jj + 2], xv[jj + 3]);
        cluster_sync();
        const float4* pown = reinterpret_cast<const float4*>(gbase) + HALF * BM / 4;
#pragma unroll
        for (int jj = 0; jj < WCOLS; jj += 4) {
            const float4 o4 = pown[((sub * WCOLS + jj) >> 2) * BM + lrow];
            const float o[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                xv[jj + k] = parity == 0 ? xv[jj + k] + o[k] : o[k] - xv[jj + k];
        }
    }
    float sq = 0.f;                       // this thread's (x_new - f)^2, at most WCOLS terms
    if (ep.pair == PAIR_MIRROR) {
        // fold: lanes < 64 hold the sums of rows i = m0 + lrow, the others the
        // differences of rows i = m0 + 127 - lrow; beyond npair / nminus: 0
        const int box = lrow < BM / 2 ? 0 : 1;
        const int ir = box == 0 ? lrow : BM - 1 - lrow;
        const bool valid = m0 + ir < (box == 0 ? ep.npair : ep.nminus);
#pragma unroll
        for (int jj = 0; jj < WCOLS; ++jj) {
            const int hc = sub * WCOLS + jj;
            uint16_t h0, h1, h2;
            split3(valid ? xv[jj] : 0.f, h0, h1, h2);
            uint16_t* st = stage + (size_t)box * NP * HALF * (BM / 2);
            st[(0 * HALF + hc) * (BM / 2) + ir] = h0;
            st[(1 * HALF + hc) * (BM / 2) + ir] = h1;
            if (NP == 3) st[(2 * HALF + hc) * (BM / 2) + ir] = h2;
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < WCOLS; ++jj) {
            const int hc = sub * WCOLS + jj;
            float x = xv[jj];
            if (split_out) {
                if (ep.mode == TE_SCALE_SPLIT_T) x *= pre[jj];
                uint16_t h0, h1, h2;
                split3(x, h0, h1, h2);
                stage[(0 * HALF + hc) * BM + lrow] = h0;
                stage[(1 * HALF + hc) * BM + lrow] = h1;
                if (NP == 3) stage[(2 * HALF + hc) * BM + lrow] = h2;
            } else {
                bool cin;
                const int col = out_col(ocol0 + jj, cin);
                if (!(ok && row_ok && cin)) continue;
                const size_t o = (size_t)col * ep.ldo + row;
                if (ep.mode == TE_STORE_T) {
                    ep.out[o] = x;
                } else {
                    const float xn = fmaf(ep.tau, x, pre[jj]);
                    ep.out[o] = xn;
                    if (ep.f) {
                        const float e = xn - pref[jj];
                        sq = fmaf(e, e, sq);
                    }
                }
            }
        }
    }
    if (ep.sumsq) {                                      // fused ||x_{k+1} - f||^2, one float64 atomic per CTA
        __shared__ double part[NTHREADS / 32];
        double v = sq;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) part[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < NTHREADS / 32; ++w) t += part[w];
            if (t != 0.0) atomicAdd(ep.sumsq, t);
        }
    }
    if (split_out) {
        // the staged [NP][HALF][BM] tile leaves in one TMA store (rows past M and
        // columns past N are clipped by the tensor map); the fold's two
        // [NP][HALF][64] boxes go to columns m0 and kout + m0 of the output
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0 && ok) {
            const uint32_t sb = base + (ep.pair ? 2u * HALF * BM * 2u : 0u);
            if (ep.pair == PAIR_MIRROR) {
                tma_store_3d(&tmO, m0, n0 + (int)ks * HALF, 0, sb);
                tma_store_3d(&tmO, ep.kout + m0, n0 + (int)ks * HALF, 0,
                             sb + (uint32_t)(NP * HALF * (BM / 2) * 2));
            } else {
                tma_store_3d(&tmO, m0, n0 + (int)ks * HALF, 0, sb);
            }
            bulk_commit();
            bulk_wait_read();
        }
    }

    if (ep.late_trigger) pdl_trigger();
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    if (threadIdx.x == 0 && !ok) atomicExch(err, 1);
}

template <int NP>
__global__ void __cluster_dims__(1, 1, SPLITK) __launch_bounds__(NTHREADS, 1)
tc_contract_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA64,
                   const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmO,
                   int M, int N, int K, const TcEpiArgs ep, int* err) {
    tc_contract_body<NP, false>(tmA, tmA64, tmB, tmO, M, N, K, ep, err, blockIdx.x, blockIdx.y);
}

// npar: the parity pairs of N in the same cluster
template <int NP>
__global__ void __cluster_dims__(1, 2, SPLITK) __launch_bounds__(NTHREADS, 1)
tc_contract_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA64,
                        const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmO,
                        int M, int N, int K, const TcEpiArgs ep, int* err) {
    tc_contract_body<NP, true>(tmA, tmA64, tmB, tmO, M, N, K, ep, err, blockIdx.x, blockIdx.y);
}

// One contraction of many independent problems (the images of a batch) in one
// launch.  Every work item is one output tile of one problem; items are listed
// largest K first, and each cluster takes the item of its blockIdx.x, so the
// block scheduler hands the remaining items to clusters as SMs free up.  The
// problems' tensor maps and epilogues live in device memory (64-byte aligned
// maps, written before the launch).  `iter` offsets each problem's RRE
// accumulator (one float64 per iteration).
struct GroupJob {
    CUtensorMap tmA, tmA64, tmB, tmO;
    int M, N, K;
    TcEpiArgs ep;
    int* err;
};

template <int NP>
__global__ void __cluster_dims__(1, 1, SPLITK) __launch_bounds__(NTHREADS, 1)
tc_contract_group_kernel(const GroupJob* __restrict__ jobs, const int4* __restrict__ items, int iter) {
    const int4 it = items[blockIdx.x];                    // (job, m tile, n tile, -)
    const GroupJob& J = jobs[it.x];
    TcEpiArgs ep = J.ep;
    if (ep.sumsq) ep.sumsq += iter;
    tc_contract_body<NP, false>(J.tmA, J.tmA64, J.tmB, J.tmO, J.M, J.N, J.K, ep, J.err, it.y, it.z);
}

// The parity-paired last contraction of many problems: an item is a tile pair
// (n tile c of both parities), the cluster (1, 2, SPLITK) at grid y = parity.
template <int NP>
__global__ void __cluster_dims__(1, 2, SPLITK) __launch_bounds__(NTHREADS, 1)
tc_contract_group_pair_kernel(const GroupJob* __restrict__ jobs, const int4* __restrict__ items,
                              int iter) {
    const int4 it = items[blockIdx.x];                    // (job, m tile, n tile pair, -)
    const GroupJob& J = jobs[it.x];
    TcEpiArgs ep = J.ep;
    if (ep.sumsq) ep.sumsq += iter;
    tc_contract_body<NP, true>(J.tmA, J.tmA64, J.tmB, J.tmO, J.M, J.N, J.K, ep, J.err, it.y,
                               2 * it.z + (int)(blockIdx.y & 1u));
}

// ---------------------------------------------------------------- matrices --
// Q_{m-2}[s, t] = sqrt(2/(m-1)) sin(s t pi/(m-1)) depends only on
// r = (s t) mod 2(m-1): tab[r] holds the 2(m-1) distinct values, in float64.
__global__ void sine_table_kernel(int m, double* tab) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < 2 * (m - 1)) tab[r] = sqrt(2.0 / (double)(m - 1)) * sinpi((double)r / (double)(m - 1));
}

__device__ __forceinline__ double q_entry(const double* tab, int s, int t, int m) {
    return tab[((long long)s * t) % (2LL * (m - 1))];
}

// qp[s-1] = (Q p)_s, qjp[s-1] = (Q J p)_s, s = 1..m-2, one block per row.
__global__ void boundary_columns_kernel(int m, const double* tab, double* qp, double* qjp) {
    const int s = blockIdx.x + 1;
    double a = 0.0, b = 0.0;
    for (int t = 1 + threadIdx.x; t <= m - 2; t += blockDim.x) {
        const double q = q_entry(tab, s, t, m);
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

__device__ __forceinline__ void split3_f64(double v, uint16_t& h0, uint16_t& h1, uint16_t& h2) {
    const __nv_bfloat16 p0 = __double2bfloat16(v);
    const double r1 = v - (double)__bfloat162float(p0);
    const __nv_bfloat16 p1 = __double2bfloat16(r1);
    const __nv_bfloat16 p2 = __double2bfloat16(r1 - (double)__bfloat162float(p1));
    h0 = __bfloat16_as_ushort(p0);
    h1 = __bfloat16_as_ushort(p1);
    h2 = __bfloat16_as_ushort(p2);
}

// Comparison-BC transforms as bf16x3 planes, row pitch ld, entry (s, t):
//  Reflective (eq. Rn, DCT-III): Tt = R^T, T = R with
//    R[t][k] = sqrt((2 - delta_{k,0}) / m) cos(k (2t + 1) pi / (2m));
//  Periodic (separable Hartley, normalised): Tt = T = H with
//    H[s][t] = (cos + sin)(2 pi s t / m) / sqrt(m), and Tp = H' with
//    H'[s][t] = (cos - sin)(2 pi s t / m) / sqrt(m) (columns of H at -s).
// Arguments are reduced exactly in integers before cospi / sincospi.
__global__ void fill_bc_transforms_kernel(int m, int ld, int bc, uint16_t* Tt, uint16_t* T,
                                          uint16_t* Tp) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)m * m) return;
    const int s = (int)(idx / m), t = (int)(idx % m);
    const size_t ps = (size_t)m * ld, o = (size_t)s * ld + t;
    double vt, v, vp = 0.0;
    if (bc == AR_BC_REFLECTIVE) {
        // R^T[s][t] = R[t][s]
        const long long rt = ((long long)s * (2 * t + 1)) % (4LL * m);
        vt = sqrt((s == 0 ? 1.0 : 2.0) / (double)m) * cospi((double)rt / (2.0 * m));
        const long long r = ((long long)t * (2 * s + 1)) % (4LL * m);
        v = sqrt((t == 0 ? 1.0 : 2.0) / (double)m) * cospi((double)r / (2.0 * m));
    } else {
        const long long r = ((long long)s * t) % (long long)m;
        double sv, cv;
        sincospi(2.0 * (double)r / (double)m, &sv, &cv);
        const double sc = 1.0 / sqrt((double)m);
        vt = v = (cv + sv) * sc;
        vp = (cv - sv) * sc;
    }
    uint16_t a0, a1, a2;
    split3_f64(vt, a0, a1, a2);
    Tt[o] = a0;
    Tt[ps + o] = a1;
    Tt[2 * ps + o] = a2;
    split3_f64(v, a0, a1, a2);
    T[o] = a0;
    T[ps + o] = a1;
    T[2 * ps + o] = a2;
    if (Tp) {
        split3_f64(vp, a0, a1, a2);
        Tp[o] = a0;
        Tp[ps + o] = a1;
        Tp[2 * ps + o] = a2;
    }
}

// ----------------------------------------------------- folded AR transforms --
// The AR pair has the reflection symmetry of the sine transform: row s of
// T~'_m (s interior) satisfies T~'[s][m-1-t] = (-1)^(s+1) T~'[s][t], including
// the boundary columns (Q J p = (-1)^(s+1) Q p), and column k of T'_m
// satisfies T'[m-1-s][k] = (-1)^(k+1) T'[s][k].  With the spatial fold
// y+_t = y_t + y_{m-1-t}, y-_t = y_t - y_{m-1-t} (t < ceil(m/2), resp.
// floor(m/2)) and the spectral order [u+, s = 1, 3, 5, .. | u-, s = 2, 4, ..],
// where u+- = y+-_0 replace the unit rows 0 and m-1, the analysis and the
// synthesis become block diagonal (half the products).  Half blocks are
// padded: spectral and folded-output to a multiple of 128 rows (Hs), folded
// spatial K to a multiple of 64 (Kh).  The filter d is equal at spectral
// indices 0 and m-1, so it applies to u+ and u- alike.

// T~'_m[s][t] (normalisation dropped), T'_m[s][t] interior columns only
__device__ __forceinline__ double ar_tt(int s, int t, int m, const double* tab, const double* qp,
                                       const double* qjp) {
    if (s == 0) return t == 0 ? 1.0 : 0.0;
    if (s == m - 1) return t == m - 1 ? 1.0 : 0.0;
    if (t == 0) return -qp[s - 1];
    if (t == m - 1) return -qjp[s - 1];
    return q_entry(tab, s, t, m);
}

__device__ __forceinline__ double ar_t_interior(int s, int k, int m, const double* tab) {
    return (s == 0 || s == m - 1) ? 0.0 : q_entry(tab, s, k, m);
}

__device__ __forceinline__ void store3(uint16_t* T, size_t ps, size_t o, double v) {
    uint16_t a0, a1, a2;
    split3_f64(v, a0, a1, a2);
    T[o] = a0;
    T[ps + o] = a1;
    T[2 * ps + o] = a2;
}

// which: 0 Ttp (analysis, spectral rows folded, natural K), 1 Ttf (analysis,
// block diagonal over folded K), 2 Tsf (synthesis, folded outputs, block
// diagonal), 3 Tsp (synthesis, natural outputs, folded spectral K).
__global__ void fill_folded_kernel(int m, int which, int rows, int K, int ld, const double* tab,
                                   const double* qp, const double* qjp, uint16_t* T) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * K) return;
    const int r = (int)(idx / K), c = (int)(idx % K);
    const FoldDims f = fold_dims(m);
    double v = 0.0;
    int s = 0;
    if (which == 0) {                                   // row: spectral kf, col: t
        const int kind = spec_of(r, f, s);
        if (kind == 0) v = (c == 0 || c == m - 1) ? 1.0 : 0.0;
        else if (kind == 2) v = c == 0 ? 1.0 : (c == m - 1 ? -1.0 : 0.0);
        else if (kind > 0) v = ar_tt(s, c, m, tab, qp, qjp);
    } else if (which == 1) {                            // row: spectral kf, col: folded t
        const int kind = spec_of(r, f, s);
        const bool anti_row = r >= f.Hs, anti_col = c >= f.Kh;
        const int t = anti_col ? c - f.Kh : c;
        if (kind >= 0 && anti_row == anti_col && t < (anti_col ? f.ha : f.h)) {
            if (kind == 0 || kind == 2) v = t == 0 ? 1.0 : 0.0;
            else v = ar_tt(s, t, m, tab, qp, qjp) * (t == m - 1 - t ? 0.5 : 1.0);
        }
    } else if (which == 2) {                            // row: folded output s, col: spectral kf
        const bool anti_row = r >= f.Hs, anti_col = c >= f.Hs;
        const int so = anti_row ? r - f.Hs : r;
        int k = 0;
        const int kind = spec_of(c, f, k);
        if (kind >= 0 && anti_row == anti_col && so < (anti_row ? f.ha : f.h)) {
            if (kind == 0) v = 0.5;
            else if (kind == 2) v = 0.5 * (2.0 * (1.0 - (double)so / (double)(m - 1)) - 1.0);
            else v = ar_t_interior(so, k, m, tab);
        }
    } else {                                            // row: natural output s, col: spectral kf
        int k = 0;
        const int kind = spec_of(c, f, k);
        if (kind == 0) v = 0.5;
        else if (kind == 2) v = 0.5 * (2.0 * (1.0 - (double)r / (double)(m - 1)) - 1.0);
        else if (kind > 0) v = ar_t_interior(r, k, m, tab);
    }
    store3(T, (size_t)rows * ld, (size_t)r * ld + c, v);
}

// d in the folded spectral order of both axes (0 in the padding).
__global__ void fold_filter_kernel(const float* __restrict__ d, int n1, int n2,
                                   float* __restrict__ df) {
    const FoldDims f1 = fold_dims(n1), f2 = fold_dims(n2);
    const int N1 = 2 * f1.Hs, N2 = 2 * f2.Hs;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N1 * N2) return;
    const int a = (int)(idx / N2), b = (int)(idx % N2);
    int s1 = 0, s2 = 0;
    const bool ok = spec_of(a, f1, s1) >= 0 && spec_of(b, f2, s2) >= 0;
    df[idx] = ok ? d[(size_t)s1 * n2 + s2] : 0.f;
}

// float32 image -> bf16x3 planes of its fold along the columns: y+ at column
// t < ceil(n2/2), y- at Kh + t (t < floor(n2/2)), zeros in the padding.
__global__ void split_fold_kernel(const float* __restrict__ y, int n1, int n2, int ld,
                                  uint16_t* planes, size_t pstride) {
    const FoldDims f = fold_dims(n2);
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n1 * f.Kh) return;
    const int i = (int)(idx / f.Kh), t = (int)(idx % f.Kh);
    const float* row = y + (size_t)i * n2;
    const float a = t < n2 ? __ldg(row + t) : 0.f;
    const float b = t < n2 ? __ldg(row + n2 - 1 - t) : 0.f;
    uint16_t h0, h1, h2;
    const size_t o = (size_t)i * ld + t;
    split3(t < f.h ? a + b : 0.f, h0, h1, h2);
    planes[o] = h0;
    planes[pstride + o] = h1;
    planes[2 * pstride + o] = h2;
    split3(t < f.ha ? a - b : 0.f, h0, h1, h2);
    planes[o + f.Kh] = h0;
    planes[pstride + o + f.Kh] = h1;
    planes[2 * pstride + o + f.Kh] = h2;
}

// float32 image -> bf16x3 planes (row pitch ld).
__global__ void split_image_kernel(const float* __restrict__ y, int n1, int n2, int ld,
                                   uint16_t* planes, size_t pstride) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n1 * n2) return;
    const int i = (int)(idx / n2), j = (int)(idx % n2);
    uint16_t h0, h1, h2;
    split3(__ldg(y + idx), h0, h1, h2);
    const size_t o = (size_t)i * ld + j;
    planes[o] = h0;
    planes[pstride + o] = h1;
    planes[2 * pstride + o] = h2;
}

// ------------------------------------------------------------ host side --
}  // namespace

void* tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return reinterpret_cast<void*>(fn);
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
}

int round_up8(int v) { return (v + 7) & ~7; }

// 3D map over bf16x3 planes {K (inner), rows, 3 planes} with box
// {box_k, box_rows, 3}: 64-byte swizzle for operand loads, none for stores.
ar_status make_map(CUtensorMap* map, const uint16_t* planes, int K, int rows, int ld, int box_k,
                   int box_rows, int nplanes, bool swizzle, int box_planes = 0) {
    auto enc = encode_fn();
    if (!enc) return fail(AR_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)nplanes};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)rows * ld * 2};
    cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows,
                         (cuuint32_t)(box_planes ? box_planes : nplanes)};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(planes), dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     swizzle ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(AR_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return AR_OK;
}

struct Operand {               // bf16 planes of a rows x K matrix and its TMA maps
    uint16_t* planes = nullptr;
    int rows = 0, K = 0, ld = 0;
    size_t pstride = 0;
    CUtensorMap map[2];        // operand loads, [0]: 3 planes, [1]: 2 planes; box {BK, box_rows, np}, 64B swizzle
    CUtensorMap omap[2];       // epilogue stores (image operands): box {BM, HALF, np}
    CUtensorMap map64[2];      // paired A tiles: one plane of 64 rows, box {BK, 64, 1}
    CUtensorMap omapf[2];      // folded epilogue stores: box {64, HALF, np}
};

enum OperandMaps : int { OM_PAIR_A = 1, OM_FOLD_OUT = 2 };

inline int mode_index(int np) { return np == 3 ? 0 : 1; }

// only_np (0: both) restricts the maps of a per-plan image operand to the
// plan's precision mode.
ar_status alloc_operand(Operand& o, int rows, int K, int box_rows, cudaStream_t s,
                        bool permanent = false, int only_np = 0, int extra = 0) {
    o.rows = rows;
    o.K = K;
    o.ld = round_up8(K);
    o.pstride = (size_t)rows * o.ld;
    const size_t bytes = MAX_PLANES * o.pstride * sizeof(uint16_t);
    if (permanent) AR_CUDA(cudaMalloc((void**)&o.planes, bytes));
    else AR_CUDA(dev_malloc_async((void**)&o.planes, bytes, s));
    for (int np = 3; np >= 2; --np) {
        if (only_np && np != only_np) continue;
        AR_TRY(make_map(&o.map[mode_index(np)], o.planes, K, rows, o.ld, BK, box_rows, np, true));
        if (!permanent)
            AR_TRY(make_map(&o.omap[mode_index(np)], o.planes, K, rows, o.ld, BM, HALF, np, false));
        if (extra & OM_PAIR_A)
            AR_TRY(make_map(&o.map64[mode_index(np)], o.planes, K, rows, o.ld, BK, BM / 2, np, true,
                            1));
        if (extra & OM_FOLD_OUT)
            AR_TRY(make_map(&o.omapf[mode_index(np)], o.planes, K, rows, o.ld, BM / 2, HALF, np,
                            false));
    }
    return AR_OK;
}

// The constant operands of one BC and side length m: the analysis Tt and
// synthesis T matrices, and for Periodic the flipped synthesis Tp.
struct TransformSet {
    Operand Tt, T, Tp;
    Operand Ttp, Ttf, Tsf, Tsp;   // AR: the folded forms (the natural Tt, T are not built)
};

void free_set(TransformSet& ts) {
    for (Operand* o : {&ts.Tt, &ts.T, &ts.Tp, &ts.Ttp, &ts.Ttf, &ts.Tsf, &ts.Tsp}) cudaFree(o->planes);
}

// Builds the operands of (m, bc) on `s` and waits for them.  AR: the folded
// forms of T~'_m and T'_m of Theorem 1 (eq. Qn for the interior, the boundary
// columns Q p and Q J p as length-m reductions).
ar_status build_transforms(int m, int bc, TransformSet& ts, cudaStream_t s) {
    if (bc != AR_BC_ANTIREFLECTIVE) {
        AR_TRY(alloc_operand(ts.Tt, m, m, BN, s, true));
        AR_TRY(alloc_operand(ts.T, m, m, BN, s, true));
        const size_t mm = (size_t)m * m;
        if (bc == AR_BC_PERIODIC) AR_TRY(alloc_operand(ts.Tp, m, m, BN, s, true));
        fill_bc_transforms_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, s>>>(
            m, ts.Tt.ld, bc, ts.Tt.planes, ts.T.planes, ts.Tp.planes);
        count_launch();
        AR_CUDA(cudaGetLastError());
        AR_CUDA(cudaStreamSynchronize(s));
        return AR_OK;
    }
    const FoldDims f = fold_dims(m);
    const int Nf = 2 * f.Hs, Kf = 2 * f.Kh;
    AR_TRY(alloc_operand(ts.Ttp, Nf, m, BN, s, true));
    AR_TRY(alloc_operand(ts.Ttf, Nf, Kf, BN, s, true));
    AR_TRY(alloc_operand(ts.Tsf, Nf, Nf, BN, s, true));
    AR_TRY(alloc_operand(ts.Tsp, m, Nf, BN, s, true));
    double* tmp = nullptr;
    const int ntab = 2 * (m - 1);
    AR_CUDA(cudaMallocAsync((void**)&tmp, (2 * (size_t)m + ntab) * sizeof(double), s));
    double* tab = tmp + 2 * m;
    sine_table_kernel<<<(ntab + 255) / 256, 256, 0, s>>>(m, tab);
    count_launch();
    AR_CUDA(cudaGetLastError());
    if (m > 2) {
        boundary_columns_kernel<<<m - 2, 256, 0, s>>>(m, tab, tmp, tmp + m);
        count_launch();
        AR_CUDA(cudaGetLastError());
    }
    const Operand* mats[4] = {&ts.Ttp, &ts.Ttf, &ts.Tsf, &ts.Tsp};
    for (int w = 0; w < 4; ++w) {
        const Operand& o = *mats[w];
        const size_t n = (size_t)o.rows * o.K;
        fill_folded_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, w, o.rows, o.K, o.ld, tab,
                                                                      tmp, tmp + m, o.planes);
        count_launch();
        AR_CUDA(cudaGetLastError());
    }
    AR_CUDA(cudaFreeAsync(tmp, s));
    AR_CUDA(cudaStreamSynchronize(s));
    return AR_OK;
}

// The transform operands depend only on the side length and the BC: they are
// built once per (device, m, bc) and kept for the life of the process.
ar_status cached_transforms(int m, int bc, cudaStream_t s, TransformSet* out) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, TransformSet> cache;
    int dev = 0;
    AR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(dev, m, bc);
    auto it = cache.find(key);
    if (it == cache.end()) {
        TransformSet ts;
        ar_status st = build_transforms(m, bc, ts, s);
        if (st != AR_OK) {
            free_set(ts);
            return st;
        }
        it = cache.emplace(key, ts).first;
    }
    *out = it->second;
    return AR_OK;
}

template <int NP>
ar_status contract_np(const Operand& A, const Operand& B, const Operand* O, const TcEpiArgs& ep,
                      int* err, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(tc_contract_kernel<NP>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)TcMode<NP>::SMEM_BYTES);
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(tc_contract_pair_kernel<NP>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)TcMode<NP>::SMEM_BYTES);
    });
    if (attr != cudaSuccess) return cuda_fail(attr, "tc_contract_kernel smem attribute");
    const int mtiles = ep.pair ? (ep.npair + BM / 2 - 1) / (BM / 2) : (A.rows + BM - 1) / BM;
    const int ntiles = (B.rows + BN - 1) / BN;
    // npar: the two halves of N (nhalf rows of B each, a multiple of BN) pair
    // tile by tile, y = 2 c + parity
    if (ep.npar && (ep.nhalf % BN != 0 || B.rows != 2 * ep.nhalf))
        return fail(AR_ERR_UNSUPPORTED, "paired N halves need nhalf a multiple of %d", BN);
    dim3 grid(mtiles, ntiles, SPLITK);
    ProfScope prof(AR_PROF_CONTRACTION, s);
    const int mi = mode_index(NP);
    count_launch();
    const CUtensorMap& omap = !O ? A.map[mi] : (ep.pair == PAIR_MIRROR ? O->omapf[mi] : O->omap[mi]);
    AR_CUDA(launch_pdl(ep.npar ? tc_contract_pair_kernel<NP> : tc_contract_kernel<NP>, grid,
                       dim3(NTHREADS), (size_t)TcMode<NP>::SMEM_BYTES, s, A.map[mi],
                       ep.pair ? A.map64[mi] : A.map[mi], B.map[mi], omap, A.rows, B.rows, A.K, ep,
                       err));
    return AR_OK;
}

// C = A B^T with the epilogue `ep`; O receives the split output planes.
ar_status contract(int np, const Operand& A, const Operand& B, const Operand* O,
                   const TcEpiArgs& ep, int* err, cudaStream_t s) {
    return np == 2 ? contract_np<2>(A, B, O, ep, err, s) : contract_np<3>(A, B, O, ep, err, s);
}

// Clusters of four contraction CTAs that can be resident at once (0 on error).
template <int NP>
int max_quad_clusters() {
    static std::once_flag once;
    static int n = 0;
    std::call_once(once, [] {
        if (cudaFuncSetAttribute(tc_contract_pair_kernel<NP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TcMode<NP>::SMEM_BYTES) != cudaSuccess)
            return;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(1, 2, SPLITK);
        cfg.blockDim = dim3(NTHREADS);
        cfg.dynamicSmemBytes = TcMode<NP>::SMEM_BYTES;
        if (cudaOccupancyMaxActiveClusters(&n, tc_contract_pair_kernel<NP>, &cfg) != cudaSuccess) n = 0;
        cudaGetLastError();
    });
    return n;
}

}  // namespace

struct TransformPlan {
    int n1, n2;
    int bc;
    int np;                    // bf16 planes per operand: 3 (float32-grade) or 2 (fast)
    bool folded;               // AR: the even/odd folded chain
    bool fold_y;               // AR: Y arrives folded along the columns (G1 block diagonal)
    Operand Tt1, T1, Tt2, T2;  // constant operands (B side), owned by the process-wide cache
    Operand Tp1, Tp2;          // Periodic: flipped synthesis operands (cache-owned)
    Operand Ttp2, Ttf1, Tsf2, Tsp1;   // AR folded: G1 .. G4 constant operands (cache-owned)
    Operand Ttf2;              // AR folded, Y folded: G1's block-diagonal operand
    Operand Tsf1;              // AR folded, N folded: G4's block-diagonal operand
    bool fold_out;             // AR: G4 folds its N index too (clusters of four)
    Operand P;                 // n1 x n2 images: Y (all BCs), then W (Reflective, Periodic)
    Operand P2;                // Periodic: n1 x n2, the odd-part filtered spectrum
    Operand Qo;                // n2 x n1 images: U^T, then V^T (Reflective, Periodic)
    Operand U, W, V;           // AR folded intermediates (see transform_apply)
    float* dfold = nullptr;    // AR folded: the filter in folded spectral order
    int* err = nullptr;
};

ar_status transform_plan_create(int n1, int n2, int bc, int precision, cudaStream_t s,
                                TransformPlan** out, bool fold_input, int pair_out) {
    TransformPlan* p = new (std::nothrow) TransformPlan();
    if (!p) return fail(AR_ERR_ALLOC, "host allocation of the transform plan");
    p->n1 = n1;
    p->n2 = n2;
    p->bc = bc;
    p->np = precision == AR_PRECISION_BF16X2 ? 2 : 3;
    p->folded = bc == AR_BC_ANTIREFLECTIVE;
    p->fold_y = p->folded && fold_input && (n2 % 4) == 0;
    if (p->folded) {
        // G4 with its N index folded runs in clusters of four: taken when they all
        // fit at once, or when there are so many that waves are unavoidable anyway
        const FoldDims f1 = fold_dims(n1), f2 = fold_dims(n2);
        const int need = ((f2.h + BM / 2 - 1) / (BM / 2)) * (f1.Hs / BN);
        const int fit = p->np == 2 ? max_quad_clusters<2>() : max_quad_clusters<3>();
        p->fold_out = fit > 0 && (pair_out == 2 || (pair_out == 1 && (need <= fit || need > 2 * fit)));
    }
    TransformSet t1, t2;
    ar_status st = cached_transforms(n1, bc, s, &t1);
    if (st == AR_OK) st = cached_transforms(n2, bc, s, &t2);
    if (st == AR_OK) {
        p->Tt1 = t1.Tt;
        p->T1 = t1.T;
        p->Tp1 = t1.Tp;
        p->Tt2 = t2.Tt;
        p->T2 = t2.T;
        p->Tp2 = t2.Tp;
        p->Ttf1 = t1.Ttf;
        p->Tsp1 = t1.Tsp;
        p->Ttp2 = t2.Ttp;
        p->Ttf2 = t2.Ttf;
        p->Tsf2 = t2.Tsf;
        p->Tsf1 = t1.Tsf;
    }
    if (p->folded) {
        const FoldDims f1 = fold_dims(n1), f2 = fold_dims(n2);
        const int N1 = 2 * f1.Hs, N2 = 2 * f2.Hs, K1 = 2 * f1.Kh;
        // Y: n1 x n2, or n1 x 2 Kh2 folded along the columns (paired row loads in
        // G1); U: N2 x K1 (folded output of G1); W: N1 x N2; V: N2 x N1 (folded
        // output of G3, paired row loads in G4)
        if (st == AR_OK)
            st = alloc_operand(p->P, n1, p->fold_y ? 2 * f2.Kh : n2, BM, s, false, p->np, OM_PAIR_A);
        if (st == AR_OK) st = alloc_operand(p->U, N2, K1, BM, s, false, p->np, OM_FOLD_OUT);
        if (st == AR_OK) st = alloc_operand(p->W, N1, N2, BM, s, false, p->np);
        if (st == AR_OK) st = alloc_operand(p->V, N2, N1, BM, s, false, p->np, OM_PAIR_A);
        if (st == AR_OK &&
            dev_malloc_async((void**)&p->dfold, (size_t)N1 * N2 * sizeof(float), s) != cudaSuccess)
            st = fail(AR_ERR_ALLOC, "folded filter");
    } else {
        if (st == AR_OK) st = alloc_operand(p->P, n1, n2, BM, s, false, p->np);
        if (st == AR_OK && bc == AR_BC_PERIODIC)
            st = alloc_operand(p->P2, n1, n2, BM, s, false, p->np);
        if (st == AR_OK) st = alloc_operand(p->Qo, n2, n1, BM, s, false, p->np);
    }
    if (st == AR_OK && dev_malloc_async((void**)&p->err, sizeof(int), s) != cudaSuccess)
        st = fail(AR_ERR_ALLOC, "transform error flag");
    if (st == AR_OK && cudaMemsetAsync(p->err, 0, sizeof(int), s) != cudaSuccess)
        st = fail(AR_ERR_CUDA, "transform error flag init");
    if (st != AR_OK) {
        transform_plan_destroy(p);
        return st;
    }
    *out = p;
    return AR_OK;
}

ar_status transform_set_filter(TransformPlan* p, const float* d32, cudaStream_t s) {
    if (!p->folded) return AR_OK;
    const FoldDims f1 = fold_dims(p->n1), f2 = fold_dims(p->n2);
    const size_t n = (size_t)(2 * f1.Hs) * (2 * f2.Hs);
    fold_filter_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d32, p->n1, p->n2, p->dfold);
    count_launch();
    AR_CUDA(cudaGetLastError());
    return AR_OK;
}

static void plan_buffers(TransformPlan* p, void* (&q)[8]) {
    void* v[8] = {p->P.planes, p->P2.planes, p->Qo.planes, p->U.planes, p->W.planes,
                  p->V.planes, p->dfold, p->err};
    for (int i = 0; i < 8; ++i) q[i] = v[i];
}

void transform_plan_destroy(TransformPlan* p) {
    if (!p) return;
    void* q[8];
    plan_buffers(p, q);
    for (void* x : q) cudaFree(x);
    delete p;
}

void transform_plan_release(TransformPlan* p, cudaStream_t s) {
    if (!p) return;
    void* q[8];
    plan_buffers(p, q);
    for (void* x : q)
        if (x) cudaFreeAsync(x, s);
    delete p;
}

uint16_t* transform_input_planes(TransformPlan* p, size_t* plane_stride, int* ld, int* folded) {
    if (plane_stride) *plane_stride = p->P.pstride;
    if (ld) *ld = p->P.ld;
    if (folded) *folded = p->fold_y ? 1 : 0;
    return p->P.planes;
}

int* transform_error_flag(TransformPlan* p) { return p->err; }

ar_status transform_spectral_view(const TransformPlan* p, const uint16_t** planes,
                                  size_t* pstride, int* ld, int* nplanes, const float** dfold) {
    if (!p->folded) return fail(AR_ERR_UNSUPPORTED, "spectral view of a non-AR plan");
    *planes = p->W.planes;
    *pstride = p->W.pstride;
    *ld = p->W.ld;
    *nplanes = p->np;
    *dfold = p->dfold;
    return AR_OK;
}

// ------------------------------------------------------ grouped transforms --
// The four contractions of x += tau D z for many AR plans, one grouped launch
// per contraction (tc_contract_group_kernel): every plan's tiles of G1, then of
// G2, ... as work items, largest K first.  Each plan's input planes must have
// been written by its reblur (DIN_SPLIT); its G4 must be the unpaired one.
struct TransformGroup {
    int np = 3, count = 0;
    bool pair_g4 = false;
    GroupJob* jobs[4] = {nullptr, nullptr, nullptr, nullptr};
    int4* items[4] = {nullptr, nullptr, nullptr, nullptr};
    int nitems[4] = {0, 0, 0, 0};
};

void transform_group_destroy(TransformGroup* g) {
    if (!g) return;
    for (int k = 0; k < 4; ++k) {
        cudaFree(g->jobs[k]);
        cudaFree(g->items[k]);
    }
    delete g;
}

namespace {
template <int NP>
cudaError_t group_kernel_attr() {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(tc_contract_group_kernel<NP>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)TcMode<NP>::SMEM_BYTES);
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(tc_contract_group_pair_kernel<NP>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)TcMode<NP>::SMEM_BYTES);
    });
    return attr;
}
}  // namespace

ar_status transform_group_create(TransformPlan* const* plans, int count, float* const* outs,
                                 const float* const* fs, double* const* sumsq, float tau,
                                 TransformGroup** out) {
    if (count < 1) return fail(AR_ERR_INVALID_ARG, "empty transform group");
    const int np = plans[0]->np;
    const bool pair = plans[0]->fold_out;
    for (int j = 0; j < count; ++j) {
        const TransformPlan* p = plans[j];
        if (!p->folded || p->fold_out != pair || p->np != np)
            return fail(AR_ERR_UNSUPPORTED, "grouped transform: plan %d is not an AR plan of the "
                                            "group's precision and G4 pairing", j);
    }
    const int mi = mode_index(np);
    std::vector<GroupJob> jobs[4];
    std::vector<std::pair<int, int4>> items[4];          // (K of the tile, item)
    for (int j = 0; j < count; ++j) {
        TransformPlan* p = plans[j];
        const FoldDims f1 = fold_dims(p->n1), f2 = fold_dims(p->n2);
        TcEpiArgs e[4] = {};
        const Operand* A[4];
        const Operand* B[4];
        const Operand* O[4];
        // as transform_apply's folded chain (DIN_SPLIT, DOUT_AXPY)
        e[0].mode = TE_SPLIT_T;
        e[0].planes = p->U.planes;
        e[0].pstride = p->U.pstride;
        e[0].ld = p->U.ld;
        e[0].pair = PAIR_MIRROR;
        e[0].mrows = p->n1;
        e[0].npair = f1.h;
        e[0].nminus = f1.ha;
        e[0].kout = f1.Kh;
        e[0].kdiag = p->fold_y ? 1 : 0;
        A[0] = &p->P;
        B[0] = p->fold_y ? &p->Ttf2 : &p->Ttp2;
        O[0] = &p->U;
        e[1].mode = TE_SCALE_SPLIT_T;
        e[1].planes = p->W.planes;
        e[1].pstride = p->W.pstride;
        e[1].ld = p->W.ld;
        e[1].d = p->dfold;
        e[1].ldd = 2 * f2.Hs;
        e[1].kdiag = 1;
        A[1] = &p->U;
        B[1] = &p->Ttf1;
        O[1] = &p->W;
        e[2].mode = TE_SPLIT_T;
        e[2].planes = p->V.planes;
        e[2].pstride = p->V.pstride;
        e[2].ld = p->V.ld;
        e[2].kdiag = 1;
        A[2] = &p->W;
        B[2] = &p->Tsf2;
        O[2] = &p->V;
        e[3].mode = TE_AXPY_T;
        e[3].out = outs[j];
        e[3].ldo = p->n2;
        e[3].tau = tau;
        e[3].f = fs ? fs[j] : nullptr;
        e[3].sumsq = (fs && fs[j] && sumsq) ? sumsq[j] : nullptr;
        e[3].pair = PAIR_HALVES;
        e[3].mhalf = f2.Hs;
        e[3].npair = f2.h;
        e[3].nminus = f2.ha;
        e[3].nout = p->n2;
        e[3].late_trigger = 1;
        A[3] = &p->V;
        B[3] = &p->Tsp1;
        O[3] = nullptr;
        if (pair) {                       // N folded too: block diagonal, parity tiles paired
            e[3].kdiag = 1;
            e[3].npar = 1;
            e[3].nhalf = f1.Hs;
            e[3].npairn = f1.h;
            e[3].nminusn = f1.ha;
            e[3].noutn = p->n1;
            B[3] = &p->Tsf1;
        }
        for (int k = 0; k < 4; ++k) {
            GroupJob gj;
            std::memset(&gj, 0, sizeof(gj));
            gj.tmA = A[k]->map[mi];
            gj.tmA64 = e[k].pair ? A[k]->map64[mi] : A[k]->map[mi];
            gj.tmB = B[k]->map[mi];
            gj.tmO = !O[k] ? A[k]->map[mi]
                           : (e[k].pair == PAIR_MIRROR ? O[k]->omapf[mi] : O[k]->omap[mi]);
            gj.M = A[k]->rows;
            gj.N = B[k]->rows;
            gj.K = A[k]->K;
            gj.ep = e[k];
            gj.err = p->err;
            const int mt = e[k].pair ? (e[k].npair + BM / 2 - 1) / (BM / 2) : (A[k]->rows + BM - 1) / BM;
            // a paired item covers the n tile c of both parities (the N halves)
            const int nt = e[k].npar ? e[k].nhalf / BN : (B[k]->rows + BN - 1) / BN;
            const int keff = e[k].kdiag ? A[k]->K / 2 : A[k]->K;
            const int job = (int)jobs[k].size();
            jobs[k].push_back(gj);
            for (int a = 0; a < mt; ++a)
                for (int b = 0; b < nt; ++b) items[k].push_back({keff, make_int4(job, a, b, 0)});
        }
    }
    TransformGroup* g = new (std::nothrow) TransformGroup();
    if (!g) return fail(AR_ERR_ALLOC, "host allocation of the transform group");
    g->np = np;
    g->count = count;
    g->pair_g4 = pair;
    cudaError_t ce = np == 2 ? group_kernel_attr<2>() : group_kernel_attr<3>();
    for (int k = 0; ce == cudaSuccess && k < 4; ++k) {
        std::stable_sort(items[k].begin(), items[k].end(),
                         [](const std::pair<int, int4>& a, const std::pair<int, int4>& b) {
                             return a.first > b.first;
                         });
        std::vector<int4> it(items[k].size());
        for (size_t i = 0; i < it.size(); ++i) it[i] = items[k][i].second;
        g->nitems[k] = (int)it.size();
        ce = cudaMalloc((void**)&g->jobs[k], jobs[k].size() * sizeof(GroupJob));
        if (ce == cudaSuccess) ce = cudaMalloc((void**)&g->items[k], it.size() * sizeof(int4));
        if (ce == cudaSuccess)
            ce = cudaMemcpy(g->jobs[k], jobs[k].data(), jobs[k].size() * sizeof(GroupJob),
                            cudaMemcpyHostToDevice);
        if (ce == cudaSuccess)
            ce = cudaMemcpy(g->items[k], it.data(), it.size() * sizeof(int4), cudaMemcpyHostToDevice);
    }
    if (ce != cudaSuccess) {
        transform_group_destroy(g);
        return cuda_fail(ce, "transform group buffers");
    }
    *out = g;
    return AR_OK;
}

bool transform_group_paired(const TransformGroup* g) { return g && g->pair_g4; }

ar_status transform_group_apply(TransformGroup* g, int iter, cudaStream_t s) {
    for (int k = 0; k < 4; ++k) {
        ProfScope prof(AR_PROF_CONTRACTION, s);
        count_launch();
        const bool pk = k == 3 && g->pair_g4;
        const dim3 grid((unsigned)g->nitems[k], pk ? 2 : 1, SPLITK);
        auto kern = g->np == 2 ? (pk ? tc_contract_group_pair_kernel<2> : tc_contract_group_kernel<2>)
                               : (pk ? tc_contract_group_pair_kernel<3> : tc_contract_group_kernel<3>);
        const size_t smem = g->np == 2 ? (size_t)TcMode<2>::SMEM_BYTES : (size_t)TcMode<3>::SMEM_BYTES;
        cudaError_t e = launch_pdl(kern, grid, dim3(NTHREADS), smem, s, (const GroupJob*)g->jobs[k],
                                   (const int4*)g->items[k], iter);
        if (e != cudaSuccess) return cuda_fail(e, "grouped contraction launch");
    }
    return AR_OK;
}

int transform_launches(const TransformPlan* p, DInput din) {
    return (din == DIN_FP32 ? 1 : 0) + (p->bc == AR_BC_PERIODIC ? 7 : 4);
}

// AR / Reflective: D y = T1 (d o (Tt1 Y Tt2^T)) T2^T in four contractions
// G1..G4.  Periodic (circulant with the even filter d(-k) = d(k)): with the
// normalised separable Hartley matrix H (symmetric, H H = I) and Y^ = H Y H^T,
//   D y = H (d_e o Y^) H^T - H' (d_o o Y^) H'^T,
// where d_e is the part of d even in each frequency (diagonal in the
// separable Hartley basis) and d_o the part odd in both (which maps the
// Hartley basis vector of (k1, k2) to minus that of (-k1, -k2), whose matrix
// is H' = H with its columns at -k).  Seven contractions: G1, G2 (d_e) and
// G2' (-d_o, into P2) share Y^; G3, G4 and G3', G4' (added) synthesise.
ar_status transform_apply(TransformPlan* p, const float* d32, const float* d32_odd,
                          const float* y, DInput din, float* out, DOutput dout, float tau,
                          cudaStream_t s, const float* f, double* sumsq) {
    const int n1 = p->n1, n2 = p->n2;
    const bool periodic = p->bc == AR_BC_PERIODIC;
    if (periodic && !d32_odd) return fail(AR_ERR_INVALID_ARG, "periodic filter without odd part");
    if (din == DIN_FP32) {
        ProfScope prof(AR_PROF_OTHER, s);
        if (p->fold_y) {
            const size_t n = (size_t)n1 * fold_dims(n2).Kh;
            split_fold_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, n1, n2, p->P.ld,
                                                                          p->P.planes, p->P.pstride);
        } else {
            const size_t n = (size_t)n1 * n2;
            split_image_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, n1, n2, p->P.ld,
                                                                           p->P.planes, p->P.pstride);
        }
        count_launch();
        AR_CUDA(cudaGetLastError());
    }
    // the four contractions are dependent launches: timed as one interval
    ProfScope prof(AR_PROF_CONTRACTION, s, (unsigned)transform_launches(p, DIN_SPLIT));
    if (p->folded) {
        // G1: U = fold_1((Y Ttp2^T)^T)   A = Y rows paired (i, n1-1-i), output K-folded
        // G2: W = d o (U Ttf1^T)^T       block diagonal in K
        // G3: V = (W Tsf2^T)^T           block diagonal in K, output rows folded along axis 2
        // G4: out (+)= unfold_2((V Tsp1^T)^T)   A = V rows paired (j, h + j); with fold_out
        //     block diagonal against Tsf1, unfold_1 across the parity pair of CTAs
        const FoldDims f1 = fold_dims(n1), f2 = fold_dims(n2);
        TcEpiArgs e{};
        e.mode = TE_SPLIT_T;
        e.planes = p->U.planes;
        e.pstride = p->U.pstride;
        e.ld = p->U.ld;
        e.pair = PAIR_MIRROR;
        e.mrows = n1;
        e.npair = f1.h;
        e.nminus = f1.ha;
        e.kout = f1.Kh;
        e.kdiag = p->fold_y ? 1 : 0;     // Y folded along the columns: G1 block diagonal too
        AR_TRY(contract(p->np, p->P, p->fold_y ? p->Ttf2 : p->Ttp2, &p->U, e, p->err, s));
        TcEpiArgs e2{};
        e2.mode = TE_SCALE_SPLIT_T;
        e2.planes = p->W.planes;
        e2.pstride = p->W.pstride;
        e2.ld = p->W.ld;
        e2.d = p->dfold;
        e2.ldd = 2 * f2.Hs;
        e2.kdiag = 1;
        AR_TRY(contract(p->np, p->U, p->Ttf1, &p->W, e2, p->err, s));
        TcEpiArgs e3{};
        e3.mode = TE_SPLIT_T;
        e3.planes = p->V.planes;
        e3.pstride = p->V.pstride;
        e3.ld = p->V.ld;
        e3.kdiag = 1;
        AR_TRY(contract(p->np, p->W, p->Tsf2, &p->V, e3, p->err, s));
        TcEpiArgs e4{};
        e4.mode = dout == DOUT_STORE ? TE_STORE_T : TE_AXPY_T;
        e4.out = out;
        e4.ldo = n2;
        e4.tau = tau;
        if (dout == DOUT_AXPY) {
            e4.f = f;
            e4.sumsq = f ? sumsq : nullptr;
        }
        e4.pair = PAIR_HALVES;
        e4.mhalf = f2.Hs;
        e4.npair = f2.h;
        e4.nminus = f2.ha;
        e4.nout = n2;
        e4.late_trigger = 1;
        if (p->fold_out) {             // N folded too: block diagonal, parity tiles paired
            e4.kdiag = 1;
            e4.npar = 1;
            e4.nhalf = f1.Hs;
            e4.npairn = f1.h;
            e4.nminusn = f1.ha;
            e4.noutn = n1;
        }
        AR_TRY(contract(p->np, p->V, p->fold_out ? p->Tsf1 : p->Tsp1, nullptr, e4, p->err, s));
        return AR_OK;
    }
    TcEpiArgs e{};
    // G1: U^T = (Y T~2^T)^T  -> Q planes
    e.mode = TE_SPLIT_T;
    e.planes = p->Qo.planes;
    e.pstride = p->Qo.pstride;
    e.ld = p->Qo.ld;
    AR_TRY(contract(p->np, p->P, p->Tt2, &p->Qo, e, p->err, s));
    // G2: W = d o (U^T T~1^T)^T -> P planes
    e.mode = TE_SCALE_SPLIT_T;
    e.planes = p->P.planes;
    e.pstride = p->P.pstride;
    e.ld = p->P.ld;
    e.d = d32;
    e.ldd = n2;
    AR_TRY(contract(p->np, p->Qo, p->Tt1, &p->P, e, p->err, s));
    if (periodic) {    // G2': W' = (-d_o) o (U^T T~1^T)^T -> P2 planes
        e.planes = p->P2.planes;
        e.d = d32_odd;
        AR_TRY(contract(p->np, p->Qo, p->Tt1, &p->P2, e, p->err, s));
    }
    // G3: V^T = (W T2^T)^T -> Q planes
    e.mode = TE_SPLIT_T;
    e.planes = p->Qo.planes;
    e.pstride = p->Qo.pstride;
    e.ld = p->Qo.ld;
    e.d = nullptr;
    AR_TRY(contract(p->np, p->P, p->T2, &p->Qo, e, p->err, s));
    // G4: out (=|+= tau) (V^T T1^T)^T; the RRE sum rides on the last update of x
    TcEpiArgs e4{};
    e4.mode = dout == DOUT_STORE ? TE_STORE_T : TE_AXPY_T;
    e4.out = out;
    e4.ldo = n2;
    e4.tau = tau;
    if (dout == DOUT_AXPY && !periodic) {
        e4.f = f;
        e4.sumsq = f ? sumsq : nullptr;
    }
    e4.late_trigger = periodic ? 0 : 1;
    AR_TRY(contract(p->np, p->Qo, p->T1, nullptr, e4, p->err, s));
    if (periodic) {
        // G3': V'^T = (W' H'2^T)^T -> Q planes;  G4': out += tau (V'^T H'1^T)^T
        AR_TRY(contract(p->np, p->P2, p->Tp2, &p->Qo, e, p->err, s));
        e4.mode = TE_AXPY_T;
        e4.tau = dout == DOUT_STORE ? 1.f : tau;
        if (dout == DOUT_AXPY) {
            e4.f = f;
            e4.sumsq = f ? sumsq : nullptr;
        }
        e4.late_trigger = 1;
        AR_TRY(contract(p->np, p->Qo, p->Tp1, nullptr, e4, p->err, s));
    }
    return AR_OK;
}

}  // namespace ar
