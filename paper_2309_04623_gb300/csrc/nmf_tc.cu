// Tensor-core (tcgen05) forms of the weighted-NMF passes (arXiv:2309.04623,
// Sec. 2 Eq. 2-3; Sec. 4.1 target modelling), precisions NMF_BF16_SPLIT
// (weights streamed as scaled FP16) and NMF_BF16_SPLIT_W32 (FP32 weights).
//
// Both passes run one kernel template.  A CTA owns 128 rows of the MMA M
// dimension in TMEM lanes -- 128 pixels in the H pass, 128 reference frames
// (or science frames) in the W pass -- and streams the other dimension in
// chunks of 64 (or 32) through two TMA rings: data (V and the weights,
// released as soon as the elementwise step has read them) and operand
// images (released after the MMAs).  Per chunk, with BF16 hi + lo splits of
// the factors (x = hi + lo, lo the BF16 of the rounding remainder):
//   R    = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T      (3 BF16 MMAs, FP32 in TMEM)
//   D    = Wt o R,  X = Wt o (V - R),  X_lo = X - bf16(X)
//                                                    (threads, FP32; Eq. 2 term X (V - R))
//   den += D B_hi + D B_lo
//   G   += X B_hi + X B_lo + X_lo B_hi               (BF16 MMAs into TMEM; B read
//                                                    MN-major from its image)
// where (A, B) = (H tile, W chunk) in the H pass and (W tile, H chunk) in the
// W pass.  The numerator of Eq. 3, W^T (Wt o V), equals den + G, so the
// update is x <- x max(den + G, 0) / max(den, eps): the BF16 rounding acts on
// the weighted residual, which is small next to Wt o V.  H is carried inside
// the loop as three BF16 parts (hi + lo + lo2, ~FP32).  For k <= 32 the hi
// and lo parts of 32 components share one 64-component image block, so one
// MMA with N = 64 contracts with both.
//
// The reconstruction W H is never written to memory.  V stays FP32 (the
// residual needs it); per element and pass the kernels read 4 bytes of V and
// 2 (scaled FP16) or 4 (FP32) bytes of weights.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <mutex>
#include <set>
#include <utility>

#include "nmf_internal.cuh"
#include "nmf_tc.cuh"
#include "tc_ptx.cuh"

namespace nmfgb {

using namespace tc;

namespace {

constexpr int TILE = 128;            // MMA M
constexpr int NC_W = 64;             // pixels per unit of a W-pass split (a multiple of every layout's chunk)
constexpr int THREADS = 448;         // warp 0: TMA, 1: MMA, 2..9: chunk warps, 10..13: tile warps
constexpr int NEPI = 256;            // chunk-warp threads
constexpr int NTW = 128;             // tile-warp threads
constexpr int IMG_BLOCK = 8192;      // bytes of one 64 x 64 BF16 operand image block
#ifndef NMF_TC_RAHEAD
#define NMF_TC_RAHEAD 2              // W H may run this many chunks ahead of den/G
#endif
#ifndef NMF_TC_PF
#define NMF_TC_PF 0
#endif
constexpr int PF = NMF_TC_PF;        // chunks prefetched into L2 beyond the ring (0: none)
#ifndef NMF_TC_DG_FIRST
#define NMF_TC_DG_FIRST 1            // MMA issue order when both are ready: den/G, then W H
#endif
#ifndef NMF_TC_SLEEP_NS
#define NMF_TC_SLEEP_NS 20           // back-off of the MMA issue loop when nothing is ready
#endif
#ifndef NMF_TC_WREV
#define NMF_TC_WREV 0                // 1: W-pass CTAs take the pixel splits in reverse order
#endif
// Precision of the split form (each 1 = the more accurate choice)
#ifndef NMF_TC_WF16
#define NMF_TC_WF16 1                // weights stored FP16 with a power-of-two scale (else BF16)
#endif
#ifndef NMF_TC_GLO
#define NMF_TC_GLO 1                 // G also contracts with the lo part of the streamed factor
#endif
#ifndef NMF_TC_XLO
#define NMF_TC_XLO 1                 // the weighted residual X enters G as hi + lo BF16 parts
#endif
#ifndef NMF_TC_DLO
#define NMF_TC_DLO 1                 // den also contracts with the lo part of the streamed factor
#endif
#ifndef NMF_TC_DLO2
#define NMF_TC_DLO2 0                // D = Wt o R enters den as hi + lo BF16 parts
#endif

// Compile-time layout of one kernel variant: KP padded components (64 for
// K <= 64, 128 for K <= 128), NC streamed rows or pixels per chunk (64 or
// 32) and NDS data stages.  With 128 components the operand tiles are twice
// as wide, so chunks of 32 keep them in shared memory, and TMEM holds a
// single (den, G) accumulator pair (two would need 2 x 256 columns).  The
// den/G operands D and X live in TMEM, so shared memory holds only the two
// rings and the tile operand.
template <int KP_, int NC_, int NDS_, int NIS_ = 3, int RK_ = KP_, bool PK_ = false, int WB_ = 2>
struct Cfg {
    // bytes of a stored weight: 2 (scaled FP16) or 4 (FP32, the single-precision-weights form)
    static constexpr int WB = WB_;
    static constexpr int KP = KP_;                    // padded components (MMA N of den/G, image layout)
    static constexpr int RK = RK_;                    // components in W H and the update (<= KP)
    // packed images (k <= 32): one 64-component block per 64 rows holds the
    // hi parts in columns 0..31 and the lo parts in columns 32..63, so one
    // MMA with N = 64 contracts with both parts; otherwise hi and lo are
    // separate images
    static constexpr bool PK = PK_;
    static constexpr int NIMG = PK ? 1 : 2;           // images per operand
    static constexpr int KB = KP / 64;                // 64-component image blocks
    static constexpr int NC = NC_;                    // streamed chunk (MMA N of R, MMA K of den/G)
    static constexpr int CPT = NC / 2;                // streamed columns per chunk-warp thread
    // data stage: V tile (FP32) then weight tile (16-bit or FP32)
    static constexpr int ST_V = 0;
    static constexpr int ST_WT = TILE * NC * 4;
    static constexpr int DSTAGE = TILE * NC * (4 + WB);
    static constexpr int NDS = NDS_;                  // data stages
    static constexpr int IMG_BASE = NDS * DSTAGE;
    // image stage: NC rows of every 64-component block, hi then lo (packed:
    // the one image)
    static constexpr int SLICE = NC * 128;
    static constexpr int ST_BH = 0;
    static constexpr int ST_BL = KB * SLICE;
    static constexpr int ISTAGE = NIMG * KB * SLICE;
    static constexpr int NIS = NIS_;                  // image stages
    static constexpr int CHUNK_BYTES = KB * IMG_BLOCK;  // one 64-row chunk of an operand image
    // A operand of W H (hi, lo): KB blocks of 128 rows x 64 components
    static constexpr int A_BYTES = KB * 16384;
    static constexpr int OFF_AH = IMG_BASE + NIS * ISTAGE;
    static constexpr int OFF_AL = OFF_AH + A_BYTES;   // (separate images only)
    static constexpr int SMEM_BYTES = OFF_AH + NIMG * A_BYTES + 1024;  // + alignment slack
    // TMEM columns: NR R buffers, NACC (den, G) accumulator pairs, then two
    // operand buffers of the den/G MMAs, each holding D, X and the lo parts
    // of X (XLO) and of D (DLO2) as BF16 pairs (NC / 2 columns per matrix).
    // Two accumulator pairs let the H pass accumulate a tile while the
    // previous one is updated; two R buffers let W H run a chunk ahead of the
    // chunk warps.  The layout takes the first of (NR, NACC) = (2, 2),
    // (1, 2), (2, 1), (1, 1) that fits the 512 columns.
    static constexpr bool XLO = NMF_TC_XLO != 0;
    static constexpr bool DLO2 = NMF_TC_DLO2 != 0;
    static constexpr int DGN = PK ? 64 : (RK < 64 ? RK : 64);  // N of each den/G MMA
    static constexpr int ACCW = KB * DGN;             // TMEM columns of den (and of G; packed: hi | lo halves)
    static_assert(!PK || (KP == 64 && RK == 32), "packed images hold 32 components");
    static constexpr int DXW = (NC / 2) * (2 + (XLO ? 1 : 0) + (DLO2 ? 1 : 0));  // one operand buffer
    static constexpr int OFF_XL = NC, OFF_DL = NC + (XLO ? NC / 2 : 0);
    static constexpr bool fits(int nr, int nacc) { return nr * NC + 2 * ACCW * nacc + 2 * DXW <= 512; }
    static constexpr int NR = fits(2, 2) ? 2 : fits(1, 2) ? 1 : fits(2, 1) ? 2 : 1;
    static constexpr int NACC = fits(NR, 2) ? 2 : 1;
    static constexpr uint32_t TM_S0 = 0, TM_S1 = NR == 2 ? NC : 0, TM_ACC = NR * NC, TM_COLS = 512;
    static constexpr uint32_t TM_DX = TM_ACC + 2 * ACCW * NACC;
    static_assert(NC == 32 || NC == 64, "chunk");
    static_assert(TM_DX + 2 * DXW <= TM_COLS, "TMEM columns");
    static_assert(SMEM_BYTES <= 232448, "shared memory");
};

// Byte offset of element (row n, component j) in an operand image of
// 64-row chunks of KB 64 x 64 blocks.
__host__ __device__ __forceinline__ long long img_off(long long n, int j, int kb);

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Byte offset of BF16 element (r, c) in a 64 x 64 (or 128 x 64) K-major
// 128-byte-swizzled operand image.
__device__ __forceinline__ uint32_t sw_elem(uint32_t r, uint32_t c) {
    return (r >> 3) * 1024u + (r & 7u) * 128u + ((((c >> 3) ^ (r & 7u))) << 4) + (c & 7u) * 2u;
}

__host__ __device__ __forceinline__ long long img_off(long long n, int j, int kb) {
    return (n >> 6) * (long long)(kb * IMG_BLOCK) + (j >> 6) * IMG_BLOCK +
           (long long)((((uint32_t)n & 63u) >> 3) * 1024u + ((uint32_t)n & 7u) * 128u +
                       ((((uint32_t)(j & 63) >> 3) ^ ((uint32_t)n & 7u)) << 4) + ((uint32_t)j & 7u) * 2u);
}

// BF16 pairs of the rounding remainders of 8 values whose BF16 pairs are hpk
// (x - bf16(x): the lo parts of a hi + lo split).
__device__ __forceinline__ uint4 lo8(const float *x, const uint4 &hpk) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&hpk);
    float l[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        l[2 * i] = x[2 * i] - f.x;
        l[2 * i + 1] = x[2 * i + 1] - f.y;
    }
    return make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]), pack_bf16(l[4], l[5]), pack_bf16(l[6], l[7]));
}

// Elementwise body for 8 consecutive streamed elements of one row:
// r = R (TMEM), v = data, w = weight -> packed BF16 D and X and (XLO, DLO2)
// the BF16 of their rounding remainders, chi += X (V-R).
template <bool XLO, bool DLO2>
__device__ __forceinline__ void dx8(const float *r, const float *v, const float *w, uint4 &dpk, uint4 &xpk,
                                    uint4 &xlpk, uint4 &dlpk, float &chi) {
    float d[8], x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float e = v[i] - r[i];
        d[i] = w[i] * r[i];
        x[i] = w[i] * e;
        chi = fmaf(x[i], e, chi);
    }
    dpk = make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]), pack_bf16(d[6], d[7]));
    xpk = make_uint4(pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), pack_bf16(x[4], x[5]), pack_bf16(x[6], x[7]));
    if constexpr (XLO) xlpk = lo8(x, xpk);
    if constexpr (DLO2) dlpk = lo8(d, dpk);
}

__device__ __forceinline__ void bf16x8_to_f32(const uint4 &u, float *w) {
    const __nv_bfloat162 *b = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(b[i]);
        w[2 * i] = f.x;
        w[2 * i + 1] = f.y;
    }
}

// The stored 16-bit weights: BF16, or FP16 holding weight x 2^e (the scale
// is undone by the caller with an exact power-of-two product).
#if NMF_TC_WF16
typedef __half wt16_t;
__device__ __forceinline__ float wt16_to_f32(wt16_t x) { return __half2float(x); }
__device__ __forceinline__ void wt16x8_to_f32(const uint4 &u, float *w) {
    const __half2 *b = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __half22float2(b[i]);
        w[2 * i] = f.x;
        w[2 * i + 1] = f.y;
    }
}
#else
typedef __nv_bfloat16 wt16_t;
__device__ __forceinline__ float wt16_to_f32(wt16_t x) { return __bfloat162float(x); }
__device__ __forceinline__ void wt16x8_to_f32(const uint4 &u, float *w) { bf16x8_to_f32(u, w); }
#endif

__device__ double warp_sum_f64_tc(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Eq. 2 of the iterate the H pass of iteration t evaluated: the fixed-order
// FP64 sum of its per-block partials by `nthr` threads (tid < nthr, whole
// warps, synchronised by `sync`), then, by thread 0, the stopping rule and
// the record of the evaluated state.  A timed-out pass leaves the cost
// undefined (NaN) and the record untouched.
template <class Sync>
__device__ void record_cost_tc(const TcArgs &a, FitState *st, int t, int nparts, int tid, int nthr, double *red,
                               Sync sync) {
    double v = 0.0;
    for (int b = tid; b < nparts; b += nthr) v += __ldcg(a.chi2_part + b);
    v = warp_sum_f64_tc(v);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    sync();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < nthr / 32; ++w) tot += red[w];
        if (tot == tot) {
            if (a.tol > 0.0 && t >= 2 && (st->chi2_prev - tot) <= a.tol * st->chi2_prev) st->stop = 1;
            st->chi2_prev = tot;
            st->chi2_last = tot;
            st->iters_kept = t;
            st->final_buf = t & 1;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// the streaming pass
//
// Warp roles: warp 0 issues TMA and bulk copies, warp 1 issues the MMAs,
// warps 2..9 ("chunk warps") do the elementwise step of every chunk, warps
// 10..13 ("tile warps") handle tile transitions: in the H pass they build the
// H operand of the next pixel tile and apply the Eq. 3 update of the previous
// one from double-buffered TMEM accumulators, so a CTA streams the chunks of
// all its tiles back to back; in the W pass they write the split partials.

template <bool HPASS, class C>
__global__ void __launch_bounds__(THREADS, 1) pass_tc_kernel(const __grid_constant__ CUtensorMap mapV,
                                                            const __grid_constant__ CUtensorMap mapWt, TcArgs a,
                                                            int chi2_only) {
    constexpr int KP = C::KP;
    constexpr int NC = C::NC, KB = C::KB, CPT = C::CPT, NDS = C::NDS, NIS = C::NIS, NACC = C::NACC;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bar_dfull[NDS], bar_dempty[NDS], bar_ifull[NIS], bar_iempty[NIS];
    __shared__ uint64_t bar_sfull[C::NR], bar_sempty[C::NR];
    __shared__ uint64_t bar_dxfull[2], bar_dxempty[2], bar_afull, bar_aempty, bar_asaved, bar_accfull[NACC],
        bar_accempty[NACC], bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_flag, s_t, s_abort, s_last;
    __shared__ double s_red[THREADS / 32];

    FitState *st = a.st;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        int skip = st->stop | st->status;
        s_t = st->t;
        // past the loop's iteration count (a recorded body holding several
        // iterations): nothing to do; the W pass tells its update kernel
        if (!chi2_only && a.t_end > 0 && s_t >= a.t_end) skip = 1;
        if (!HPASS && a.t_end > 0 && blockIdx.x == 0) st->run = !skip;
        s_flag = skip;
        s_abort = 0;
    }
    __syncthreads();
    // the W pass may be launched (and take the SMs this grid leaves) now
    if (HPASS && a.h_flags) griddep_launch_dependents();
    if (s_flag) return;
    const int t = s_t;
    const unsigned seq = (unsigned)t + 1u;  // H passes of this stage once this one is done
    const bool do_update = !chi2_only;

    // work of this CTA: ntm tiles of the M dimension, nch chunks each
    const long long rows_total = a.rows;  // N (or M)
    const long long Pp = a.Pp;
    long long s0, s1;                     // streamed range [s0, s1) of every tile
    int ntm;
    int w_tile = 0, w_split = 0;          // W pass: row tile and pixel split of this block
    if (HPASS) {
        const int ntiles = (int)(Pp / TILE);
        ntm = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
        s0 = 0;
        s1 = rows_total;
    } else {
        // the explicit schedule (w_schedule), else blocks [0, full) take the
        // full row tiles, nsplit each, and the rest the last row tile
        // (row-tile-major measured faster than split-major)
        ntm = 1;
        if (a.w_nblk > 0) {
            const int b = (int)blockIdx.x;
            w_tile = a.w_tile[b];
            w_split = a.w_split[b];
            s0 = (long long)a.w_c0[b] * NC_W;
            s1 = (long long)a.w_c1[b] * NC_W < Pp ? (long long)a.w_c1[b] * NC_W : Pp;
        } else {
            const int ntr = (int)((rows_total + TILE - 1) / TILE);
            const int full = (ntr - 1) * a.nsplit;
            const bool last = (int)blockIdx.x >= full;
            w_tile = last ? ntr - 1 : (int)blockIdx.x / a.nsplit;
            w_split = last ? (int)blockIdx.x - full : (int)blockIdx.x % a.nsplit;
            const int len = last ? a.split_len_last : a.split_len;
            s0 = (long long)w_split * len;
            s1 = s0 + len < Pp ? s0 + len : Pp;
        }
    }
    const int nch = (int)((s1 - s0 + NC - 1) / NC);
    const int G = ntm * nch;
    auto tile_m0 = [&](int i) -> long long {
        return HPASS ? ((long long)blockIdx.x + (long long)i * gridDim.x) * TILE : (long long)w_tile * TILE;
    };
    // operand images: the tile operand A of W H and the streamed operand B
    // (the H image sets are picked by t's parity without indexing the
    // parameter arrays, which would copy them to local memory)
    const bool odd = (t & 1) != 0;
    uint8_t *const hk_in_h = odd ? a.hk_h[1] : a.hk_h[0], *const hk_in_l = odd ? a.hk_l[1] : a.hk_l[0];
    uint8_t *const hk_out_h = odd ? a.hk_h[0] : a.hk_h[1], *const hk_out_l = odd ? a.hk_l[0] : a.hk_l[1];
    uint8_t *const hk_in_l2 = odd ? a.hk_l2[1] : a.hk_l2[0], *const hk_out_l2 = odd ? a.hk_l2[0] : a.hk_l2[1];
    const uint8_t *srcAh = HPASS ? hk_in_h : a.wk_h;
    const uint8_t *srcAl = HPASS ? hk_in_l : a.wk_l;
    const uint8_t *srcBh = HPASS ? a.wk_h : hk_out_h;
    const uint8_t *srcBl = HPASS ? a.wk_l : hk_out_l;

    if (tid == 0) {
        for (int i = 0; i < NDS; ++i) {
            mbar_init(&bar_dfull[i], 1);
            mbar_init(&bar_dempty[i], NEPI);
        }
        for (int i = 0; i < NIS; ++i) {
            mbar_init(&bar_ifull[i], 1);
            mbar_init(&bar_iempty[i], 1);
        }
        for (int i = 0; i < C::NR; ++i) {
            mbar_init(&bar_sfull[i], 1);
            mbar_init(&bar_sempty[i], NEPI);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(&bar_accfull[i], 1);
            mbar_init(&bar_accempty[i], NTW);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_dxfull[i], NEPI);
            mbar_init(&bar_dxempty[i], 1);
        }
        mbar_init(&bar_afull, 1);
        mbar_init(&bar_aempty, 1);
        mbar_init(&bar_asaved, NTW);
        mbar_init(&bar_drain, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&s_tmem, C::TM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    int *err = &st->status;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            // copies issued so far: tile operands, and the last chunk whose
            // images / data tiles were issued (to drain them after an abort)
            int a_loads = 0, g_img = -1, g_data = -1;
            // tile operand of tile ti (its 128 rows: two consecutive 64-row
            // image chunks, every 64-component block to its own operand block)
            auto load_a = [&](int ti) {
                const long long ch = tile_m0(ti) / 64;
                ++a_loads;
                mbar_arrive_expect_tx(&bar_afull, C::NIMG * C::A_BYTES);
                for (int b = 0; b < KB; ++b)
                    for (int h = 0; h < 2; ++h) {
                        const long long src = (ch + h) * C::CHUNK_BYTES + b * IMG_BLOCK;
                        bulk_load(smem + C::OFF_AH + b * 16384 + h * IMG_BLOCK, srcAh + src, IMG_BLOCK, &bar_afull);
                        if (!C::PK)
                            bulk_load(smem + C::OFF_AL + b * 16384 + h * IMG_BLOCK, srcAl + src, IMG_BLOCK,
                                      &bar_afull);
                    }
            };
            auto prefetch_a = [&](int ti) {
                const long long ch = tile_m0(ti) / 64;
                bulk_prefetch_l2(srcAh + ch * C::CHUNK_BYTES, 2 * C::CHUNK_BYTES);
                if (!C::PK) bulk_prefetch_l2(srcAl + ch * C::CHUNK_BYTES, 2 * C::CHUNK_BYTES);
            };
            load_a(0);
            // byte offset of the streamed chunk starting at sc within an image
            auto img_src = [&](long long sc) -> long long {
                return (sc / 64) * C::CHUNK_BYTES + (sc % 64) / NC * C::SLICE;
            };
            // L2 prefetch runs PF chunks ahead of the shared-memory rings
            auto prefetch = [&](int g) {
                const long long m0 = tile_m0(g / nch);
                const long long sc = s0 + (long long)(g % nch) * NC;
                if (HPASS) {
                    tma_prefetch_2d(&mapV, (int)m0, (int)sc);
                    tma_prefetch_2d(&mapWt, (int)m0, (int)sc);
                } else {
                    for (int x = 0; x < NC; x += 32) tma_prefetch_2d(&mapV, (int)sc + x, (int)m0);
                    tma_prefetch_2d(&mapWt, (int)sc, (int)m0);
                }
                const long long src = img_src(sc);
                for (int b = 0; b < KB; ++b) {
                    bulk_prefetch_l2(srcBh + src + b * IMG_BLOCK, C::SLICE);
                    if (!C::PK) bulk_prefetch_l2(srcBl + src + b * IMG_BLOCK, C::SLICE);
                }
            };
            for (int g = 2; g < G && g < 2 + PF; ++g) prefetch(g);
            long long ready_tile = -1;  // W pass: the last H tile seen written
            for (int g = 0; g < G; ++g) {
                if (HPASS && g % nch == 0) {
                    // the next tile's operand replaces this one once the tile
                    // warps have saved it (they need it for the update)
                    const int ti = g / nch;
                    if (ti > 0) {
                        if (!mbar_wait(&bar_asaved, (ti - 1) & 1, &s_abort, err, NMF_ETIMEOUT)) break;
                        load_a(ti);
                    }
                    if (ti + 1 < ntm) prefetch_a(ti + 1);
                }
                if (PF > 0 && g >= 1 && g + PF + 1 < G) prefetch(g + PF + 1);
                const long long m0 = tile_m0(g / nch);
                const long long sc = s0 + (long long)(g % nch) * NC;  // streamed origin of this chunk
                // operand images of the chunk (released after the MMAs)
                const int is = g % NIS;
                if (g >= NIS && !mbar_wait(&bar_iempty[is], ((g / NIS) - 1) & 1, &s_abort, err, NMF_ETIMEOUT)) break;
                if (!HPASS && a.h_flags && sc / TILE != ready_tile) {
                    // this chunk's H images are written by the concurrent H pass.
                    // A planted missing arrival (failure-handling test) waits
                    // instead for a count the H pass never reaches.
                    const bool plant = a.fault_t >= 0 && t == a.fault_t && blockIdx.x == 0;
                    if (!flag_wait(a.h_flags + sc / TILE, plant ? 4u * seq + (1u << 30) : 4u * seq, &s_abort, err,
                                   NMF_ETIMEOUT, plant ? a.fault_ns : kWaitLimitNs))
                        break;
                    fence_proxy_async_global();
                    ready_tile = sc / TILE;
                }
                uint8_t *ist = smem + C::IMG_BASE + is * C::ISTAGE;
                const long long src = img_src(sc);
                mbar_arrive_expect_tx(&bar_ifull[is], C::ISTAGE);
                for (int b = 0; b < KB; ++b) {
                    bulk_load(ist + C::ST_BH + b * C::SLICE, srcBh + src + b * IMG_BLOCK, C::SLICE, &bar_ifull[is]);
                    if (!C::PK)
                        bulk_load(ist + C::ST_BL + b * C::SLICE, srcBl + src + b * IMG_BLOCK, C::SLICE,
                                  &bar_ifull[is]);
                }
                g_img = g;
                // data tiles (released once the elementwise step has read them)
                const int ds = g % NDS;
                if (g >= NDS && !mbar_wait(&bar_dempty[ds], ((g / NDS) - 1) & 1, &s_abort, err, NMF_ETIMEOUT)) break;
                uint8_t *dst = smem + ds * C::DSTAGE;
                mbar_arrive_expect_tx(&bar_dfull[ds], C::DSTAGE);
                if (HPASS) {
                    tma_load_2d(dst + C::ST_V, &mapV, (int)m0, (int)sc, &bar_dfull[ds]);
                    tma_load_2d(dst + C::ST_WT, &mapWt, (int)m0, (int)sc, &bar_dfull[ds]);
                } else {
                    for (int x = 0; x < NC; x += 32)
                        tma_load_2d(dst + C::ST_V + x * 512, &mapV, (int)sc + x, (int)m0, &bar_dfull[ds]);
                    if (C::WB == 4) {
                        // FP32 weights in 32-pixel boxes of 128-byte rows, like V
                        for (int x = 0; x < NC; x += 32)
                            tma_load_2d(dst + C::ST_WT + x * 512, &mapWt, (int)sc + x, (int)m0, &bar_dfull[ds]);
                    } else {
                        tma_load_2d(dst + C::ST_WT, &mapWt, (int)sc, (int)m0, &bar_dfull[ds]);
                    }
                }
                g_data = g;
            }
            // every copy issued lands before the block releases its shared
            // memory, also when the consumers wound down early (the last phase
            // issued on a barrier completes after all earlier ones; in a
            // normal run these phases are long complete)
            if (a_loads > 0) mbar_wait_drain(&bar_afull, (a_loads - 1) & 1);
            for (int i = 0; i < NIS; ++i) {
                const int gl = g_img - ((g_img - i) % NIS + NIS) % NIS;
                if (gl >= 0) mbar_wait_drain(&bar_ifull[i], (gl / NIS) & 1);
            }
            for (int i = 0; i < NDS; ++i) {
                const int gl = g_data - ((g_data - i) % NDS + NDS) % NDS;
                if (gl >= 0) mbar_wait_drain(&bar_dfull[i], (gl / NDS) & 1);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t aH = smem_u32(smem + C::OFF_AH), aL = smem_u32(smem + C::OFF_AL);
            constexpr uint32_t IDESC_R = idesc_bf16(TILE, NC);
            constexpr uint32_t IDESC_MN = idesc_bf16_bmn(TILE, C::DGN);
            // Event-driven issue: W H for chunk r as soon as its images have
            // landed, its TMEM buffer is free and its tile's A operand is in
            // place; den/G for chunk m as soon as the chunk warps have written
            // its operands and its accumulator pair is free.  Neither waits
            // behind the other.
            int r = 0, m = 0;
            bool ok = true;
            const unsigned long long t0 = global_ns();
            auto try_r = [&]() -> bool {
                if (r < G && r <= m + NMF_TC_RAHEAD) {
                    constexpr int NR = C::NR;
                    const int s = r % NR, is = r % NIS, ti = r / nch, c = r % nch;
                    if (mbar_test(&bar_ifull[is], (r / NIS) & 1) &&
                        (r < NR || mbar_test(&bar_sempty[s], ((r / NR) - 1) & 1)) &&
                        (c != 0 || mbar_test(&bar_afull, ti & 1))) {
                        tc_fence_after();
                        const uint32_t bH = smem_u32(smem + C::IMG_BASE + is * C::ISTAGE + C::ST_BH);
                        const uint32_t bL = smem_u32(smem + C::IMG_BASE + is * C::ISTAGE + C::ST_BL);
                        const uint32_t dS = tmem + (s ? C::TM_S1 : C::TM_S0);
#pragma unroll
                        for (int kk = 0; kk < C::RK / 16; ++kk) {
                            const uint32_t ao = (kk >> 2) * 16384 + (kk & 3) * 32;
                            const uint32_t bo = (kk >> 2) * C::SLICE + (kk & 3) * 32;
                            // packed: the lo parts sit 32 components (64 bytes) after the hi parts
                            const uint64_t ah = sdesc_kmajor_sw128(aH + ao);
                            const uint64_t al = sdesc_kmajor_sw128(C::PK ? aH + ao + 64 : aL + ao);
                            const uint64_t bh = sdesc_kmajor_sw128(bH + bo);
                            const uint64_t bl = sdesc_kmajor_sw128(C::PK ? bH + bo + 64 : bL + bo);
                            mma_bf16(dS, ah, bh, IDESC_R, kk > 0 ? 1u : 0u);
                            mma_bf16(dS, ah, bl, IDESC_R, 1u);
                            mma_bf16(dS, al, bh, IDESC_R, 1u);
                        }
                        mma_commit(&bar_sfull[s]);
                        if (c == nch - 1) mma_commit(&bar_aempty);  // the tile's A operand is no longer read
                        ++r;
                        return true;
                    }
                }
                return false;
            };
            auto try_dg = [&]() -> bool {
                if (m < r) {
                    const int ti = m / nch, c = m % nch, b = ti % NACC;
                    if (mbar_test(&bar_dxfull[m & 1], (m >> 1) & 1) &&
                        (c != 0 || ti < NACC || mbar_test(&bar_accempty[b], ((ti / NACC) - 1) & 1))) {
                        tc_fence_after();
                        if (do_update) {
                            // B_hi of the chunk read MN-major (K = streamed index),
                            // one MMA per 64-component block (N = 32 when only 32
                            // components are live)
                            const uint32_t cB = smem_u32(smem + C::IMG_BASE + (m % NIS) * C::ISTAGE + C::ST_BH);
                            const uint32_t cBl = cB + (C::ST_BL - C::ST_BH);
                            const uint32_t dDen = tmem + C::TM_ACC + 2 * C::ACCW * b, dG = dDen + C::ACCW;
                            const uint32_t tD = tmem + C::TM_DX + (m & 1) * C::DXW, tX = tD + NC / 2;
                            const uint32_t tXl = tD + C::OFF_XL, tDl = tD + C::OFF_DL;
                            // den += D B_hi + D B_lo, G += X B_hi + X B_lo + X_lo B_hi: the
                            // streamed factor in hi + lo parts in both, the weighted residual X
                            // in hi + lo parts (G decides where the iteration goes; measured on
                            // the 500-iteration STIS run, D's lo part changes nothing beyond
                            // 1e-4 and costs 10 % more time)
#pragma unroll
                            for (int kk = 0; kk < NC / 16; ++kk) {
                                const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
#pragma unroll
                                for (int bb = 0; bb < KB; ++bb) {
                                    const uint64_t bd = sdesc_mnmajor_sw128(cB + bb * C::SLICE + kk * 2048);
                                    const uint64_t bl = sdesc_mnmajor_sw128(cBl + bb * C::SLICE + kk * 2048);
                                    const uint32_t oD = C::DGN * bb;
                                    mma_bf16_ta(dDen + oD, tD + 8 * kk, bd, IDESC_MN, acc);
                                    mma_bf16_ta(dG + oD, tX + 8 * kk, bd, IDESC_MN, acc);
                                    // (packed images: bd already spans hi | lo)
                                    if (NMF_TC_DLO && !C::PK) mma_bf16_ta(dDen + oD, tD + 8 * kk, bl, IDESC_MN, 1u);
                                    if (C::DLO2) mma_bf16_ta(dDen + oD, tDl + 8 * kk, bd, IDESC_MN, 1u);
                                    if (NMF_TC_GLO && !C::PK) mma_bf16_ta(dG + oD, tX + 8 * kk, bl, IDESC_MN, 1u);
                                    if (C::XLO) mma_bf16_ta(dG + oD, tXl + 8 * kk, bd, IDESC_MN, 1u);
                                }
                            }
                        }
                        // with no new MMA (chi2-only) the commits still arrive after
                        // the earlier ones, so both modes follow one protocol
                        mma_commit(&bar_dxempty[m & 1]);
                        mma_commit(&bar_iempty[m % NIS]);
                        if (c == nch - 1) mma_commit(&bar_accfull[b]);
                        ++m;
                        return true;
                    }
                }
                return false;
            };
            while (ok && m < G) {
                // den/G first: its completion frees the D/X buffer the chunk
                // warps wait on, so it goes to the tensor core ahead of W H
                // for a later chunk
                const bool progressed = NMF_TC_DG_FIRST ? (try_dg() | try_r()) : (try_r() | try_dg());
                if (!progressed) {
                    if (NMF_TC_SLEEP_NS > 0) __nanosleep(NMF_TC_SLEEP_NS);
                    if (s_abort) {
                        ok = false;
                    } else if (global_ns() - t0 > kWaitLimitNs) {
                        atomicCAS(err, 0, NMF_ETIMEOUT);
                        s_abort = 1;
                        ok = false;
                    }
                }
            }
            // every MMA issued completes before the block releases its TMEM
            // and shared memory, also when the block wound down early
            mma_commit(&bar_drain);
            mbar_wait_drain(&bar_drain, 0);
        }
    } else if (warp < 2 + NEPI / 32) {
        // ------------------------------------------------------------ chunk warps
        const int e = warp - 2;               // 0..7
        const int q = warp & 3;               // TMEM lane quarter of this warp
        const int hf = e >> 2;                // which half of the streamed columns
        const int row = 32 * q + lane;        // TMEM lane = M row in the tile
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        const float wsi = NMF_TC_WF16 ? st->wscale_inv : 1.0f;  // undoes the weights' storage scale
        float chi = 0.0f;
        bool ok = true;
        for (int g = 0; g < G && ok; ++g) {
            const int s = g % C::NR;
            ok = mbar_wait(&bar_sfull[s], (g / C::NR) & 1, &s_abort, err, NMF_ETIMEOUT);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc_fence_after();
            float r[CPT];
#pragma unroll
            for (int x = 0; x < CPT; x += 16)
                tmem_ld16(tl + (s ? C::TM_S1 : C::TM_S0) + CPT * hf + x, *reinterpret_cast<float(*)[16]>(r + x));
            tmem_ld_wait();
            tc_fence_before();
            mbar_arrive(&bar_sempty[s]);
            ok = mbar_wait(&bar_dfull[g % NDS], (g / NDS) & 1, &s_abort, err, NMF_ETIMEOUT);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            const uint8_t *stg = smem + (g % NDS) * C::DSTAGE;
            uint4 dpk[CPT / 8], xpk[CPT / 8], xlpk[C::XLO ? CPT / 8 : 1], dlpk[C::DLO2 ? CPT / 8 : 1];
#pragma unroll
            for (int cb = 0; cb < CPT / 8; ++cb) {
                float v[8], w[8];
                const int c0 = CPT * hf + 8 * cb;  // first streamed column of this group
                if (HPASS) {
                    // column `row` (pixel) of streamed rows c0 .. c0 + 7
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int n = c0 + i;
                        v[i] = reinterpret_cast<const float *>(stg + C::ST_V)[n * TILE + row];
                        w[i] = C::WB == 4 ? reinterpret_cast<const float *>(stg + C::ST_WT)[n * TILE + row]
                                          : wsi * wt16_to_f32(reinterpret_cast<const wt16_t *>(stg + C::ST_WT)[n * TILE + row]);
                    }
                } else {
                    // row `row` (frame), streamed pixels c0 .. c0 + 7: V in 32-pixel
                    // boxes of 128-byte rows (128-byte swizzle); the weights in
                    // NC-wide rows (128- or 64-byte swizzle)
                    const uint8_t *vb = stg + C::ST_V + (c0 >> 5) * 16384 + row * 128;
                    const int q16 = (c0 & 31) >> 2;
                    const float4 v0 = *reinterpret_cast<const float4 *>(vb + ((q16 ^ (row & 7)) << 4));
                    const float4 v1 = *reinterpret_cast<const float4 *>(vb + (((q16 + 1) ^ (row & 7)) << 4));
                    v[0] = v0.x; v[1] = v0.y; v[2] = v0.z; v[3] = v0.w;
                    v[4] = v1.x; v[5] = v1.y; v[6] = v1.z; v[7] = v1.w;
                    if constexpr (C::WB == 4) {
                        const uint8_t *wbp = stg + C::ST_WT + (c0 >> 5) * 16384 + row * 128;
                        const float4 w0 = *reinterpret_cast<const float4 *>(wbp + ((q16 ^ (row & 7)) << 4));
                        const float4 w1 = *reinterpret_cast<const float4 *>(wbp + (((q16 + 1) ^ (row & 7)) << 4));
                        w[0] = w0.x; w[1] = w0.y; w[2] = w0.z; w[3] = w0.w;
                        w[4] = w1.x; w[5] = w1.y; w[6] = w1.z; w[7] = w1.w;
                    } else {
                        const int wc = c0 >> 3;
                        const uint32_t woff = NC == 64 ? row * 128 + ((wc ^ (row & 7)) << 4)
                                                       : row * 64 + ((wc ^ ((row >> 1) & 3)) << 4);
                        const uint4 wb = *reinterpret_cast<const uint4 *>(stg + C::ST_WT + woff);
                        wt16x8_to_f32(wb, w);
#pragma unroll
                        for (int i = 0; i < 8; ++i) w[i] *= wsi;
                    }
                }
                dx8<C::XLO, C::DLO2>(r + 8 * cb, v, w, dpk[cb], xpk[cb], xlpk[C::XLO ? cb : 0],
                                     dlpk[C::DLO2 ? cb : 0], chi);
            }
            mbar_arrive(&bar_dempty[g % NDS]);  // this thread has read its V and Wt
            // D/X buffer g & 1 is free once the den/G MMAs of chunk g - 2 are done
            if (g >= 2) ok = mbar_wait(&bar_dxempty[g & 1], ((g >> 1) - 1) & 1, &s_abort, err, NMF_ETIMEOUT);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            if (do_update) {
                // this thread's CPT streamed columns of its row, BF16 pairs
                const uint32_t tD = tl + C::TM_DX + (g & 1) * C::DXW + CPT / 2 * hf;
                if constexpr (CPT == 32) {
                    tmem_st16(tD, reinterpret_cast<const uint32_t *>(dpk));
                    tmem_st16(tD + NC / 2, reinterpret_cast<const uint32_t *>(xpk));
                    if constexpr (C::XLO) tmem_st16(tD + C::OFF_XL, reinterpret_cast<const uint32_t *>(xlpk));
                    if constexpr (C::DLO2) tmem_st16(tD + C::OFF_DL, reinterpret_cast<const uint32_t *>(dlpk));
                } else {
                    tmem_st8(tD, reinterpret_cast<const uint32_t *>(dpk));
                    tmem_st8(tD + NC / 2, reinterpret_cast<const uint32_t *>(xpk));
                    if constexpr (C::XLO) tmem_st8(tD + C::OFF_XL, reinterpret_cast<const uint32_t *>(xlpk));
                    if constexpr (C::DLO2) tmem_st8(tD + C::OFF_DL, reinterpret_cast<const uint32_t *>(dlpk));
                }
                tmem_st_wait();
            }
            tc_fence_before();
            mbar_arrive(&bar_dxfull[g & 1]);
        }
        if (HPASS) {
            // Eq. 2 of the incoming iterate: FP32 per thread, FP64 across threads
            const double cd = warp_sum_f64_tc((double)chi);
            if (lane == 0) s_red[e] = cd;
        }
    } else {
        // ------------------------------------------------------------ tile warps
        const int q = warp & 3;
        const int row = 32 * q + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        bool ok = true;
        if (HPASS) {
            // Per tile: save the tile's H (its A operand, hi + lo) once the
            // W H MMAs are done with it, release the buffer to the next
            // tile's operand, then apply Eq. 3 from the TMEM accumulators
            // and write the new H as operand images.
            constexpr bool SAVE = KP == 64;  // old H kept in registers (else re-read from the images in L2)
            constexpr int RK = C::RK;
            const uint8_t *hin_h = hk_in_h, *hin_l = hk_in_l, *hin_l2 = hk_in_l2;
            uint8_t *hout_h = hk_out_h, *hout_l = hk_out_l, *hout_l2 = hk_out_l2;
            for (int i = 0; i < ntm && ok; ++i) {
                const int b = i % NACC;
                const long long p = tile_m0(i) + row;
                ok = mbar_wait(&bar_afull, i & 1, &s_abort, err, NMF_ETIMEOUT);
                if (ok) ok = mbar_wait(&bar_aempty, i & 1, &s_abort, err, NMF_ETIMEOUT);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                uint4 sh[SAVE ? RK / 8 : 1], sl[SAVE ? RK / 8 : 1];
                if constexpr (SAVE) {
#pragma unroll
                    for (int cb = 0; cb < RK / 8; ++cb) {
                        sh[cb] = *reinterpret_cast<const uint4 *>(smem + C::OFF_AH + sw_elem(row, 8 * cb));
                        sl[cb] = *reinterpret_cast<const uint4 *>(C::PK ? smem + C::OFF_AH + sw_elem(row, 32 + 8 * cb)
                                                                        : smem + C::OFF_AL + sw_elem(row, 8 * cb));
                    }
                }
                fence_proxy_async_smem();
                mbar_arrive(&bar_asaved);
                ok = mbar_wait(&bar_accfull[b], (i / NACC) & 1, &s_abort, err, NMF_ETIMEOUT);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc_fence_after();
                if (do_update) {
                    // Eq. 3:  H <- H (den + G) / max(den, eps), 16 components at a time
#pragma unroll(KP == 64 ? 4 : 1)
                    for (int pc = 0; pc < RK / 16; ++pc) {
                        float den[16], g[16];
                        const uint32_t acc = tl + C::TM_ACC + 2 * C::ACCW * b + 16 * pc;
                        tmem_ld16(acc, den);
                        tmem_ld16(acc + C::ACCW, g);
                        if constexpr (C::PK) {
                            // packed: add the contractions with the lo parts (16 columns at a time)
                            float lo_part[16];
                            tmem_ld16(acc + 32, lo_part);
                            tmem_ld_wait();
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) den[jj] += lo_part[jj];
                            tmem_ld16(acc + C::ACCW + 32, lo_part);
                            tmem_ld_wait();
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) g[jj] += lo_part[jj];
                        }
                        uint4 oh[2], ol[2], ol2[2];
#pragma unroll
                        for (int x = 0; x < 2; ++x)
                            ol2[x] = __ldg(reinterpret_cast<const uint4 *>(hin_l2 + img_off(p, 16 * pc + 8 * x, KB)));
                        if constexpr (SAVE) {
                            oh[0] = sh[(2 * pc) % (RK / 8)];
                            oh[1] = sh[(2 * pc + 1) % (RK / 8)];
                            ol[0] = sl[(2 * pc) % (RK / 8)];
                            ol[1] = sl[(2 * pc + 1) % (RK / 8)];
                        } else {
#pragma unroll
                            for (int x = 0; x < 2; ++x) {
                                const long long off = img_off(p, 16 * pc + 8 * x, KB);
                                oh[x] = __ldg(reinterpret_cast<const uint4 *>(hin_h + off));
                                ol[x] = __ldg(reinterpret_cast<const uint4 *>(hin_l + off));
                            }
                        }
                        tmem_ld_wait();
#pragma unroll
                        for (int x = 0; x < 2; ++x) {
                            float hh[8], hl[8], hl2[8], hi[8], lo[8], lo2[8];
                            bf16x8_to_f32(oh[x], hh);
                            bf16x8_to_f32(ol[x], hl);
                            bf16x8_to_f32(ol2[x], hl2);
#pragma unroll
                            for (int ii = 0; ii < 8; ++ii) {
                                const int jj = 8 * x + ii;
                                const float h = (hh[ii] + hl[ii]) + hl2[ii];
                                // the numerator den + G is W^T (Wt o V) >= 0; the clamp
                                // only removes a negative rounding residue
                                const float nv = h == 0.0f ? 0.0f
                                                           : flush_tiny(__fdividef(h * fmaxf(den[jj] + g[jj], 0.0f),
                                                                                   fmaxf(den[jj], a.eps)));
                                hi[ii] = __bfloat162float(__float2bfloat16_rn(nv));
                                lo[ii] = __bfloat162float(__float2bfloat16_rn(nv - hi[ii]));
                                lo2[ii] = (nv - hi[ii]) - lo[ii];
                            }
                            const long long off = img_off(p, 16 * pc + 8 * x, KB);
                            *reinterpret_cast<uint4 *>(hout_h + off) =
                                make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]),
                                           pack_bf16(hi[6], hi[7]));
                            *reinterpret_cast<uint4 *>(C::PK ? hout_h + img_off(p, 32 + 16 * pc + 8 * x, KB)
                                                             : hout_l + off) =
                                make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]),
                                           pack_bf16(lo[6], lo[7]));
                            *reinterpret_cast<uint4 *>(hout_l2 + off) =
                                make_uint4(pack_bf16(lo2[0], lo2[1]), pack_bf16(lo2[2], lo2[3]),
                                           pack_bf16(lo2[4], lo2[5]), pack_bf16(lo2[6], lo2[7]));
                        }
                    }
                    if (a.h_flags) {
                        // publish this warp's quarter of the tile to the
                        // concurrent W pass: the tile is written once all four
                        // tile warps have counted it (4 per iteration)
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) atomicAdd(a.h_flags + tile_m0(i) / TILE, 1u);
                    }
                }
                tc_fence_before();
                mbar_arrive(&bar_accempty[b]);
            }
        } else {
            if (a.t_end > 0 && a.h_blocks > 0 && blockIdx.x == 0) {
                // Eq. 2 of this iteration's incoming iterate and the stopping
                // rule, from the H pass's per-block shares (the tile warps
                // are idle until the accumulators are full).  If the rule
                // fires, the update kernel leaves W as it is.  Every tile
                // thread reaches the barrier inside, timed out or not.
                if (a.h_flags) flag_wait(&st->h_done, seq * (unsigned)a.h_blocks, &s_abort, err, NMF_ETIMEOUT);
                record_cost_tc(a, st, t, a.h_blocks, tid - 32 * (2 + NEPI / 32), NTW, s_red,
                               [] { asm volatile("bar.sync 1, %0;" ::"n"(NTW)); });
            }
            // partial sums of this pixel split for the W (or C) update
            ok = __all_sync(0xffffffffu, mbar_wait(&bar_accfull[0], 0, &s_abort, err, NMF_ETIMEOUT));
            tc_fence_after();
            if (ok && do_update) {
                const long long n = tile_m0(0) + row;
                const int nq = (a.k + 31) / 32;  // partials of components >= k are never read
#pragma unroll 1
                for (int qq = 0; qq < nq; ++qq) {
                    float den[32], g[32];
                    const uint32_t acc = tl + C::TM_ACC + 32 * qq;
                    tmem_ld16(acc, *reinterpret_cast<float(*)[16]>(den));
                    tmem_ld16(acc + 16, *reinterpret_cast<float(*)[16]>(den + 16));
                    tmem_ld16(acc + C::ACCW, *reinterpret_cast<float(*)[16]>(g));
                    tmem_ld16(acc + C::ACCW + 16, *reinterpret_cast<float(*)[16]>(g + 16));
                    if constexpr (C::PK) {
                        // packed: add the contractions with the lo parts (columns 32..63)
                        float dl[32], gl[32];
                        tmem_ld16(acc + 32, *reinterpret_cast<float(*)[16]>(dl));
                        tmem_ld16(acc + 48, *reinterpret_cast<float(*)[16]>(dl + 16));
                        tmem_ld16(acc + C::ACCW + 32, *reinterpret_cast<float(*)[16]>(gl));
                        tmem_ld16(acc + C::ACCW + 48, *reinterpret_cast<float(*)[16]>(gl + 16));
                        tmem_ld_wait();
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            den[jj] += dl[jj];
                            g[jj] += gl[jj];
                        }
                    }
                    tmem_ld_wait();
                    if (n < rows_total) {
                        float *pp = a.part + ((long long)w_split * rows_total + n) * (2 * KP);
#pragma unroll
                        for (int jj = 0; jj < 32; jj += 4) {
                            *reinterpret_cast<float4 *>(pp + 32 * qq + jj) =
                                make_float4(den[jj], den[jj + 1], den[jj + 2], den[jj + 3]);
                            *reinterpret_cast<float4 *>(pp + KP + 32 * qq + jj) =
                                make_float4(g[jj], g[jj + 1], g[jj + 2], g[jj + 3]);
                        }
                    }
                }
            }
        }
    }

    // ------------------------------------------------------------ teardown
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, C::TM_COLS);
    if (HPASS) {
        // this block's share of Eq. 2; inside a tensor-core fit loop (t_end
        // set) the W pass of the same iteration sums and records the shares
        // (off this kernel's tail), else the last block does it here
        const bool here = chi2_only || a.t_end == 0;
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < NEPI / 32; ++w) tot += s_red[w];
            a.chi2_part[blockIdx.x] = tot;
            if (!here && a.h_flags) {
                // for the concurrent W pass, which sums the shares
                __threadfence();
                atomicAdd(&st->h_done, 1u);
            }
            if (here) {
                __threadfence();
                const unsigned tk = atomicAdd(&st->ticket_h, 1u);
                s_last = (tk == gridDim.x - 1);
            }
        }
        if (here) {
            __syncthreads();
            if (s_last) {
                __threadfence();
                record_cost_tc(a, st, t, (int)gridDim.x, tid, THREADS, s_red, [] { __syncthreads(); });
                if (tid == 0) st->ticket_h = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// W (or C) update: fixed-order sum over the pixel splits, Eq. 3, and the
// BF16 operand images of the new coefficients.

__global__ void __launch_bounds__(256) wupdate_tc_kernel(TcArgs a) {
    __shared__ float s_d[8][32], s_g[8][32];
    FitState *st = a.st;
    if (st->stop | st->status) return;
    if (a.t_end > 0 && !st->run) return;  // the W pass of this iteration did not run
    // block (row n, 32 components): warp w sums splits w, w + 8, ... with
    // lane j reading component j (coalesced), then warp 0 adds the eight
    // warp sums in order
    const int nq = (a.k + 31) / 32;
    const long long n = blockIdx.x / nq;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = 32 * (int)(blockIdx.x % nq) + lane;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t = st->t + 1;
    const int kp = a.kp;
    const long long stride = a.rows * (2LL * kp);
    // pixel splits of this row's tile: the W pass's schedule, or nsplit
    // (nsplit_last for the last, partial, row tile)
    const int nsp = a.w_nblk > 0 ? (int)a.w_nsplit[n / TILE]
                                 : (n >= (a.rows - 1) / TILE * TILE ? a.nsplit_last : a.nsplit);
    float sd = 0.f, sg = 0.f;
    if (j < a.k) {
        // all of this warp's partials are loaded before any is added (one L2
        // round trip instead of one per split), then added in split order
        constexpr int PER_WARP = (kMaxWSplits + 7) / 8;
        const float *pp = a.part + n * (2LL * kp) + j;
        float vd[PER_WARP], vg[PER_WARP];
#pragma unroll
        for (int i = 0; i < PER_WARP; ++i) {
            const int sp = warp + 8 * i;
            vd[i] = sp < nsp ? __ldcg(pp + sp * stride) : 0.0f;
            vg[i] = sp < nsp ? __ldcg(pp + sp * stride + kp) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < PER_WARP; ++i) {
            if (warp + 8 * i < nsp) {
                sd += vd[i];
                sg += vg[i];
            }
        }
    }
    s_d[warp][lane] = sd;
    s_g[warp][lane] = sg;
    __syncthreads();
    if (warp != 0 || j >= a.k) return;
    sd = s_d[0][lane];
    sg = s_g[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) {
        sd += s_d[w][lane];
        sg += s_g[w][lane];
    }
    float *wp = a.W + n * a.ldw + j;
    const float w = *wp;
    // the numerator sd + sg is (Wt o V) H^T >= 0; the clamp only removes a
    // negative rounding residue
    const float nw = w == 0.0f ? 0.0f : flush_tiny((w * fmaxf(sd + sg, 0.0f)) / fmaxf(sd, a.eps));
    *wp = nw;
    const __nv_bfloat16 hi = __float2bfloat16_rn(nw);
    const __nv_bfloat16 lo = __float2bfloat16_rn(nw - __bfloat162float(hi));
    const long long off = img_off(n, j, kp / 64);
    *reinterpret_cast<__nv_bfloat16 *>(a.wk_h + off) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(a.packed ? a.wk_h + img_off(n, 32 + j, 1) : a.wk_l + off) = lo;
}

// Operand images (hi, lo) of a coefficient matrix (rows x k, ld ldw) or of a
// basis (k x Pp): element (row, j).  Entries outside [0, k) x [0, rows) are
// left as they are (zero).
__global__ void images_kernel(const float *X, long long rows, int k, long long ld, int x_is_kxP, uint8_t *Kh,
                              uint8_t *Kl, uint8_t *Kl2, int kb, int packed) {
    const long long total = rows * k;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long n = i / k;
        const int j = (int)(i % k);
        const float v = x_is_kxP ? X[(long long)j * ld + n] : X[n * ld + j];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const float r = v - __bfloat162float(hi);
        const __nv_bfloat16 lo = __float2bfloat16_rn(r);
        const long long off = img_off(n, j, kb);
        *reinterpret_cast<__nv_bfloat16 *>(Kh + off) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(packed ? Kh + img_off(n, 32 + j, 1) : Kl + off) = lo;
        if (Kl2) *reinterpret_cast<__nv_bfloat16 *>(Kl2 + off) = __float2bfloat16_rn(r - __bfloat162float(lo));
    }
}

// The current iterate of H in FP32 from its operand images: set s = t & 1
// into buffer s (Hb0 or Hb1), (hi + lo) + lo2.
__global__ void h_from_images_kernel(const FitState *st, const uint8_t *h0, const uint8_t *l0, const uint8_t *m0,
                                     const uint8_t *h1, const uint8_t *l1, const uint8_t *m1, float *Hb0,
                                     float *Hb1, int k, long long Pp, int kb, int packed) {
    const int sset = st->t & 1;
    const uint8_t *ih = sset ? h1 : h0, *il = sset ? l1 : l0, *im = sset ? m1 : m0;
    float *H = sset ? Hb1 : Hb0;
    const long long total = (long long)k * Pp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / Pp);
        const long long p = i % Pp;
        const long long off = img_off(p, j, kb);
        H[i] = (__bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(ih + off)) +
                __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(packed ? ih + img_off(p, 32 + j, 1)
                                                                                  : il + off))) +
               __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(im + off));
    }
}

// Largest weight (for the FP16 storage scale): block maximum of the bit
// patterns (non-negative floats order as unsigned integers), one atomicMax
// per block.  Negative or non-finite weights are flagged by the conversion.
__global__ void __launch_bounds__(256) weights_max_kernel(const float *src, long long total, FitState *st) {
    __shared__ unsigned red[8];
    unsigned m = 0u;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const float x = src[i];
        if (x > 0.0f && x <= 3.402823466e38f) m = max(m, __float_as_uint(x));
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = max(m, red[w]);
        if (m) atomicMax(&st->wmax_bits, m);
    }
}

// Weights to 16 bits (row-padded copy, zero padding): BF16, or FP16 of the
// weight times 2^e with e chosen so that the largest weight lands in
// [2^14, 2^15) (FP16's largest finite value is 65504): every weight within
// 2^-29 of the largest keeps FP16's 11 significant bits, and the scale is
// exact to undo.  Validates the weights (negative or non-finite: NMF_EDATA).
__global__ void weights_16_kernel(const float *src, long long rows, long long cols, long long ld_src,
                                  wt16_t *dst, long long ld_dst, FitState *st) {
    const long long total = rows * ld_dst;
#if NMF_TC_WF16
    const unsigned mb = st->wmax_bits;
    int e = 0;
    if (mb != 0u) {
        const int ex = (int)((mb >> 23) & 0xFFu) - 127;  // floor(log2(max)) for a normal max
        e = 14 - (ex < -126 ? -126 : ex);
        if (e > 126) e = 126;
    }
    const float scale = ldexpf(1.0f, e);
    if (blockIdx.x == 0 && threadIdx.x == 0) st->wscale_inv = ldexpf(1.0f, -e);
#endif
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / ld_dst, c = i % ld_dst;
        float x = 0.0f;
        if (c < cols) {
            x = src[r * ld_src + c];
            if (!(x >= 0.0f && x <= 3.402823466e38f)) bad = true;
        }
#if NMF_TC_WF16
        dst[i] = __float2half_rn(x * scale);
#else
        dst[i] = __float2bfloat16_rn(x);
#endif
    }
    if (bad) atomicExch(&st->status, (int)NMF_EDATA);
}

// ---------------------------------------------------------------------------
// host side

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

bool make_map(CUtensorMap *m, CUtensorMapDataType dt, int esize, const void *base, long long cols, long long rows,
              long long ld, int box_x, int box_y, CUtensorMapSwizzle sw) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
    cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    cuuint32_t es[2] = {1, 1};
    return enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t set_smem(const void *kern, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, kern})) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert({dev, kern});
    return e;
}

int num_sms() {
    static int n[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (n[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        n[dev] = v;
    }
    return n[dev];
}

int grid_1d(long long work) {
    long long g = (work + 255) / 256;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int tc_max_k() { return 128; }
int tc_kp(int k) { return k <= 64 ? 64 : 128; }
bool tc_packed(int k) { return k <= 32; }
int tc_split_granule() { return NC_W; }
int tc_num_sms() { return num_sms(); }
int tc_hpass_blocks(long long Pp) {
    const int ntiles = (int)(Pp / TILE);
    return ntiles < num_sms() ? ntiles : num_sms();
}
int tc_tile() { return TILE; }
size_t tc_image_bytes(long long rows, int k) {
    return (size_t)((rows + 127) / 128 * 2) * (size_t)(tc_kp(k) / 64) * IMG_BLOCK;
}

cudaError_t tc_weights_bf16(const float *src, long long rows, long long cols, void *dst, long long ld_dst,
                            FitState *st, cudaStream_t s) {
#if NMF_TC_WF16
    count_launches(1);
    weights_max_kernel<<<grid_1d(rows * cols), 256, 0, s>>>(src, rows * cols, st);
#endif
    count_launches(1);
    weights_16_kernel<<<grid_1d(rows * ld_dst), 256, 0, s>>>(src, rows, cols, cols, reinterpret_cast<wt16_t *>(dst),
                                                             ld_dst, st);
    return cudaGetLastError();
}

cudaError_t tc_images(const float *X, long long rows, int k, long long ld, bool x_is_kxP, uint8_t *Kh, uint8_t *Kl,
                      int kp, bool packed, cudaStream_t s, uint8_t *Kl2) {
    if (rows * k == 0) return cudaSuccess;
    count_launches(1);
    images_kernel<<<grid_1d(rows * k), 256, 0, s>>>(X, rows, k, ld, x_is_kxP ? 1 : 0, Kh, Kl, Kl2, kp / 64,
                                                    packed ? 1 : 0);
    return cudaGetLastError();
}

// The variants run for each component width.
#ifndef NMF_TC_NC64
#define NMF_TC_NC64 64
#endif
#ifndef NMF_TC_NDS64
#define NMF_TC_NDS64 (NMF_TC_NC64 == 64 ? 2 : 4)
#endif
#ifndef NMF_TC_NIS64
#define NMF_TC_NIS64 4
#endif
using Cfg64 = Cfg<64, NMF_TC_NC64, NMF_TC_NDS64, NMF_TC_NIS64>;
#ifndef NMF_TC_NDS32
#define NMF_TC_NDS32 NMF_TC_NDS64
#endif
#ifndef NMF_TC_NIS32
#define NMF_TC_NIS32 NMF_TC_NIS64
#endif
using Cfg32 = Cfg<64, NMF_TC_NC64, NMF_TC_NDS32, NMF_TC_NIS32, 32, true>;  // k <= 32: packed images
// k <= 128: 64-row chunks with one R buffer and one (den, G) pair (the
// 512 TMEM columns hold no more at 128 components), two data and two image
// stages; 16-22 % faster per iteration than 32-row chunks with two R
// buffers at k = 100 and 128
#ifndef NMF_TC_NC128
#define NMF_TC_NC128 64
#endif
#ifndef NMF_TC_NDS128
#define NMF_TC_NDS128 (NMF_TC_NC128 == 64 ? 2 : 4)
#endif
#ifndef NMF_TC_NIS128
#define NMF_TC_NIS128 (NMF_TC_NC128 == 64 ? 2 : 3)
#endif
using Cfg128 = Cfg<128, NMF_TC_NC128, NMF_TC_NDS128, NMF_TC_NIS128>;

// The layouts with FP32 weights (8 bytes per element and pass): the same
// kernels with 64-KB data stages; at k <= 128, where 64-row chunks would not
// leave room for the image ring, 32-row chunks with two data stages of 32 KB
// and four image stages
#ifndef NMF_TC_NDS128W
#define NMF_TC_NDS128W 2
#endif
#ifndef NMF_TC_NIS128W
#define NMF_TC_NIS128W 4
#endif
using Cfg32w = Cfg<64, 64, 2, 4, 32, true, 4>;
using Cfg64w = Cfg<64, 64, 2, 4, 64, false, 4>;
using Cfg128w = Cfg<128, 32, NMF_TC_NDS128W, NMF_TC_NIS128W, 128, false, 4>;
static_assert(Cfg32w::NC == Cfg64w::NC && Cfg32::NC == Cfg64::NC, "one chunk width per component block");

cudaError_t tc_h_from_images(const TcArgs &a, float *Hb0, float *Hb1, cudaStream_t s) {
    count_launches(1);
    h_from_images_kernel<<<grid_1d((long long)a.k * a.Pp), 256, 0, s>>>(
        a.st, a.hk_h[0], a.hk_l[0], a.hk_l2[0], a.hk_h[1], a.hk_l[1], a.hk_l2[1], Hb0, Hb1, a.k, a.Pp, a.kp / 64,
        a.packed);
    return cudaGetLastError();
}

bool tc_make_maps(TcMaps *m, const float *V, const void *Wtb, long long rows, long long Pp, int kp, bool wt32) {
    const int nc = wt32 ? (kp == 64 ? Cfg64w::NC : Cfg128w::NC) : (kp == 64 ? Cfg64::NC : Cfg128::NC);
    bool ok = true;
    ok &= make_map(&m->hV, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, V, Pp, rows, Pp, TILE, nc, CU_TENSOR_MAP_SWIZZLE_NONE);
    ok &= make_map(&m->wV, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, V, Pp, rows, Pp, 32, TILE, CU_TENSOR_MAP_SWIZZLE_128B);
    if (wt32) {
        // FP32 weights (Wtb is the FP32 padded copy): laid out like V
        ok &= make_map(&m->hWt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Wtb, Pp, rows, Pp, TILE, nc,
                       CU_TENSOR_MAP_SWIZZLE_NONE);
        ok &= make_map(&m->wWt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Wtb, Pp, rows, Pp, 32, TILE,
                       CU_TENSOR_MAP_SWIZZLE_128B);
        return ok;
    }
    const CUtensorMapDataType wt = NMF_TC_WF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    ok &= make_map(&m->hWt, wt, 2, Wtb, Pp, rows, Pp, TILE, nc,
                   CU_TENSOR_MAP_SWIZZLE_NONE);
    ok &= make_map(&m->wWt, wt, 2, Wtb, Pp, rows, Pp, nc, TILE,
                   nc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B);
    return ok;
}

namespace {

template <class C>
cudaError_t hpass_cfg(const TcMaps &m, const TcArgs &a, bool chi2_only, cudaStream_t s) {
    auto kern = pass_tc_kernel<true, C>;
    cudaError_t e = set_smem(reinterpret_cast<const void *>(kern), C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = tc_hpass_blocks(a.Pp);
    count_launches(1);
    kern<<<(unsigned)grid, THREADS, C::SMEM_BYTES, s>>>(m.hV, m.hWt, a, chi2_only ? 1 : 0);
    return cudaGetLastError();
}

template <class C>
cudaError_t wpass_cfg(const TcMaps &m, const TcArgs &a, cudaStream_t s) {
    auto kern = pass_tc_kernel<false, C>;
    cudaError_t e = set_smem(reinterpret_cast<const void *>(kern), C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const long long ntr = (a.rows + TILE - 1) / TILE;
    const unsigned grid = a.w_nblk > 0 ? (unsigned)a.w_nblk : (unsigned)((ntr - 1) * a.nsplit + a.nsplit_last);
    count_launches(2);
    if (a.h_flags) {
        // may start while the H pass runs: its chunks wait for their tiles
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(THREADS);
        cfg.dynamicSmemBytes = C::SMEM_BYTES;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, m.wV, m.wWt, a, 0);
        if (e != cudaSuccess) return e;
    } else {
        kern<<<grid, THREADS, C::SMEM_BYTES, s>>>(m.wV, m.wWt, a, 0);
    }
    wupdate_tc_kernel<<<(unsigned)(a.rows * ((a.k + 31) / 32)), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t tc_hpass(const TcMaps &m, const TcArgs &a, bool chi2_only, cudaStream_t s) {
    if (a.wt32) {
        if (a.kp == 128) return hpass_cfg<Cfg128w>(m, a, chi2_only, s);
        return a.k <= 32 ? hpass_cfg<Cfg32w>(m, a, chi2_only, s) : hpass_cfg<Cfg64w>(m, a, chi2_only, s);
    }
    if (a.kp == 128) return hpass_cfg<Cfg128>(m, a, chi2_only, s);
    return a.k <= 32 ? hpass_cfg<Cfg32>(m, a, chi2_only, s) : hpass_cfg<Cfg64>(m, a, chi2_only, s);
}

cudaError_t tc_wpass(const TcMaps &m, const TcArgs &a, cudaStream_t s) {
    if (a.wt32) {
        if (a.kp == 128) return wpass_cfg<Cfg128w>(m, a, s);
        return a.k <= 32 ? wpass_cfg<Cfg32w>(m, a, s) : wpass_cfg<Cfg64w>(m, a, s);
    }
    if (a.kp == 128) return wpass_cfg<Cfg128>(m, a, s);
    return a.k <= 32 ? wpass_cfg<Cfg32>(m, a, s) : wpass_cfg<Cfg64>(m, a, s);
}

}  // namespace nmfgb
