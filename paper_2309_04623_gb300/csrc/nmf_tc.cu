// Tensor-core (tcgen05) form of the weighted-NMF passes (arXiv:2309.04623,
// Sec. 2 Eq. 2-3; Sec. 4.1 target modelling), precision NMF_BF16_SPLIT.
//
// Both passes run one kernel template.  A CTA owns 128 rows of the MMA M
// dimension in TMEM lanes -- 128 pixels in the H pass, 128 reference frames
// (or science frames) in the W pass -- and streams the other dimension in
// chunks of 64 through two TMA rings (data V, Wt: two stages, released as
// soon as the elementwise step has read them; operand images: three stages,
// released after the MMAs).  Per chunk:
//   R   = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T       (3 BF16 MMAs, FP32 in TMEM)
//   D   = Wt o R,  X = Wt o (V - R)                    (threads, FP32; Eq. 2 term X (V-R))
//   den += D B_hi, G += X B_hi                      (2 BF16 MMAs into TMEM; B_hi
//                                                   read MN-major, no transposed copy)
// where (A, B) = (H tile, W chunk) in the H pass and (W tile, H chunk) in the
// W pass.  The numerator of Eq. 3 is
// W^T (Wt o V) = den + G exactly, so the update is x <- x (den + G) / den:
// the BF16 rounding acts on the residual image E = V - R, which is small
// next to V, rather than on V itself.  R is formed from hi/lo split factors
// so that E is accurate to ~1e-6 of V.
//
// The reconstruction W H is never written to memory.  V stays FP32 (E needs
// it), the weights are stored once as BF16.  Per element and pass the kernel
// reads 6 bytes.
#include <cuda_bf16.h>
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
constexpr int NC = 64;               // streamed chunk (MMA N of R, MMA K of den/G)
constexpr int KP = 64;               // padded components (MMA K of R, MMA N of den/G)
constexpr int THREADS = 448;         // warp 0: TMA, 1: MMA, 2..9: chunk warps, 10..13: tile warps
constexpr int NEPI = 256;            // chunk-warp threads
constexpr int NTW = 128;             // tile-warp threads
constexpr int IMG_CHUNK = 8192;      // bytes of one 64 x 64 BF16 operand image
constexpr int PF = 2;                // chunks prefetched into L2 beyond the ring

// shared-memory layout (bytes from a 1024-aligned base)
constexpr int ST_V = 0;              // data stage: V tile, FP32, 32 KB
constexpr int ST_WT = 32768;         //             weight tile, BF16, 16 KB
constexpr int DSTAGE = 49152;
constexpr int NDS = 2;               // data stages
constexpr int IMG_BASE = NDS * DSTAGE;
constexpr int ST_BH = 0;             // image stage: B operand of R, hi, 8 KB (also the den/G operand)
constexpr int ST_BL = 8192;          //              B operand of R, lo, 8 KB
constexpr int ISTAGE = 16384;
constexpr int NIS = 3;               // image stages
constexpr int OFF_AH = IMG_BASE + NIS * ISTAGE;  // A operand of R, hi, 16 KB
constexpr int OFF_AL = OFF_AH + 16384;
constexpr int OFF_D = OFF_AL + 16384;
constexpr int OFF_X = OFF_D + 16384;
constexpr int SMEM_BYTES = OFF_X + 16384 + 1024;  // + alignment slack

// TMEM columns: two R buffers, then two (den, G) accumulator pairs
constexpr uint32_t TM_S0 = 0, TM_S1 = 64, TM_ACC = 128, TM_COLS = 512;

constexpr uint32_t IDESC = idesc_bf16(TILE, 64);
constexpr uint32_t IDESC_MN = idesc_bf16_bmn(TILE, 64);

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float bf16_lo_part(float x, float hi) { return x - hi; }

// Byte offset of BF16 element (r, c) in a 64 x 64 (or 128 x 64) K-major
// 128-byte-swizzled operand image.
__device__ __forceinline__ uint32_t sw_elem(uint32_t r, uint32_t c) {
    return (r >> 3) * 1024u + (r & 7u) * 128u + ((((c >> 3) ^ (r & 7u))) << 4) + (c & 7u) * 2u;
}

// Elementwise body for 8 consecutive streamed elements of one row:
// r = R (TMEM), v = data, w = weight -> packed BF16 D and X, chi += X (V-R).
__device__ __forceinline__ void dx8(const float *r, const float *v, const float *w, uint4 &dpk, uint4 &xpk,
                                    float &chi) {
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

__device__ double warp_sum_f64_tc(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
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

template <bool HPASS>
__global__ void __launch_bounds__(THREADS, 1) pass_tc_kernel(const __grid_constant__ CUtensorMap mapV,
                                                            const __grid_constant__ CUtensorMap mapWt, TcArgs a,
                                                            int chi2_only) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bar_dfull[NDS], bar_dempty[NDS], bar_ifull[NIS], bar_iempty[NIS];
    __shared__ uint64_t bar_sfull[2], bar_sempty[2];
    __shared__ uint64_t bar_dxfull, bar_dxempty, bar_afull, bar_aempty, bar_accfull[2], bar_accempty[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_flag, s_t, s_abort, s_last;
    __shared__ double s_red[THREADS / 32];

    FitState *st = a.st;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        s_flag = st->stop | st->status;
        s_t = st->t;
        s_abort = 0;
    }
    __syncthreads();
    if (s_flag) return;
    const int t = s_t;
    const bool do_update = !chi2_only;

    // work of this CTA: ntm tiles of the M dimension, nch chunks each
    const long long rows_total = a.rows;  // N (or M)
    const long long Pp = a.Pp;
    long long s0, s1;                     // streamed range [s0, s1) of every tile
    int ntm;
    if (HPASS) {
        const int ntiles = (int)(Pp / TILE);
        ntm = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
        s0 = 0;
        s1 = rows_total;
    } else {
        ntm = 1;
        s0 = (long long)blockIdx.x * a.split_len;
        s1 = s0 + a.split_len < Pp ? s0 + a.split_len : Pp;
    }
    const int nch = (int)((s1 - s0 + NC - 1) / NC);
    const int G = ntm * nch;
    auto tile_m0 = [&](int i) -> long long {
        return HPASS ? ((long long)blockIdx.x + (long long)i * gridDim.x) * TILE : (long long)blockIdx.y * TILE;
    };
    const float *Hin = (t & 1) ? a.Hb1 : a.Hb0;  // H pass input (fit); projection: Hb0 == Hb1
    float *Hout = (t & 1) ? a.Hb0 : a.Hb1;

    if (tid == 0) {
        for (int i = 0; i < NDS; ++i) {
            mbar_init(&bar_dfull[i], 1);
            mbar_init(&bar_dempty[i], NEPI);
        }
        for (int i = 0; i < NIS; ++i) {
            mbar_init(&bar_ifull[i], 1);
            mbar_init(&bar_iempty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_sfull[i], 1);
            mbar_init(&bar_sempty[i], NEPI);
            mbar_init(&bar_accfull[i], 1);
            mbar_init(&bar_accempty[i], NTW);
        }
        mbar_init(&bar_dxfull, NEPI);
        mbar_init(&bar_dxempty, 1);
        mbar_init(&bar_afull, HPASS ? NTW : 1);
        mbar_init(&bar_aempty, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&s_tmem, TM_COLS);
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
            if (!HPASS) {
                // W (or C) tile operands: two consecutive 64-row image chunks
                const long long ch = tile_m0(0) / 64;
                mbar_arrive_expect_tx(&bar_afull, 32768);
                bulk_load(smem + OFF_AH, a.imgAh + ch * IMG_CHUNK, 16384, &bar_afull);
                bulk_load(smem + OFF_AL, a.imgAl + ch * IMG_CHUNK, 16384, &bar_afull);
            }
            // L2 prefetch runs PF chunks ahead of the two-stage shared-memory ring
            auto prefetch = [&](int g) {
                const long long m0 = tile_m0(g / nch);
                const long long sc = s0 + (long long)(g % nch) * NC;
                if (HPASS) {
                    tma_prefetch_2d(&mapV, (int)m0, (int)sc);
                    tma_prefetch_2d(&mapWt, (int)m0, (int)sc);
                } else {
                    tma_prefetch_2d(&mapV, (int)sc, (int)m0);
                    tma_prefetch_2d(&mapV, (int)sc + 32, (int)m0);
                    tma_prefetch_2d(&mapWt, (int)sc, (int)m0);
                }
                const long long ic = sc / 64;
                bulk_prefetch_l2(a.imgBh + ic * IMG_CHUNK, IMG_CHUNK);
                bulk_prefetch_l2(a.imgBl + ic * IMG_CHUNK, IMG_CHUNK);
            };
            for (int g = 2; g < G && g < 2 + PF; ++g) prefetch(g);
            for (int g = 0; g < G; ++g) {
                if (g >= 1 && g + PF + 1 < G) prefetch(g + PF + 1);
                const long long m0 = tile_m0(g / nch);
                const long long sc = s0 + (long long)(g % nch) * NC;  // streamed origin of this chunk
                // operand images of the chunk (three-stage ring, released after the MMAs)
                const int is = g % NIS;
                if (g >= NIS && !mbar_wait(&bar_iempty[is], ((g / NIS) - 1) & 1, &s_abort, err, NMF_ETIMEOUT)) break;
                uint8_t *ist = smem + IMG_BASE + is * ISTAGE;
                const long long ic = sc / 64;  // image chunk of the streamed dimension
                mbar_arrive_expect_tx(&bar_ifull[is], ISTAGE);
                bulk_load(ist + ST_BH, a.imgBh + ic * IMG_CHUNK, IMG_CHUNK, &bar_ifull[is]);
                bulk_load(ist + ST_BL, a.imgBl + ic * IMG_CHUNK, IMG_CHUNK, &bar_ifull[is]);
                // data tiles (two-stage ring, released once the elementwise step has read them)
                const int ds = g % NDS;
                if (g >= NDS && !mbar_wait(&bar_dempty[ds], ((g / NDS) - 1) & 1, &s_abort, err, NMF_ETIMEOUT)) break;
                uint8_t *dst = smem + ds * DSTAGE;
                mbar_arrive_expect_tx(&bar_dfull[ds], DSTAGE);
                if (HPASS) {
                    tma_load_2d(dst + ST_V, &mapV, (int)m0, (int)sc, &bar_dfull[ds]);
                    tma_load_2d(dst + ST_WT, &mapWt, (int)m0, (int)sc, &bar_dfull[ds]);
                } else {
                    tma_load_2d(dst + ST_V, &mapV, (int)sc, (int)m0, &bar_dfull[ds]);
                    tma_load_2d(dst + ST_V + 16384, &mapV, (int)sc + 32, (int)m0, &bar_dfull[ds]);
                    tma_load_2d(dst + ST_WT, &mapWt, (int)sc, (int)m0, &bar_dfull[ds]);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t aH = smem_u32(smem + OFF_AH), aL = smem_u32(smem + OFF_AL);
            const uint32_t dA = smem_u32(smem + OFF_D), xA = smem_u32(smem + OFF_X);
            // Event-driven issue: W H for chunk r as soon as its data has
            // landed, its TMEM buffer is free and its tile's A operand is in
            // place; den/G for chunk m as soon as the chunk warps have written
            // its operands and its accumulator buffer is free.  Neither waits
            // behind the other.
            int r = 0, m = 0;
            bool ok = true;
            const unsigned long long t0 = global_ns();
            while (ok && m < G) {
                bool progressed = false;
                if (r < G && r <= m + 2) {
                    const int s = r & 1, is = r % NIS, ti = r / nch, c = r % nch;
                    if (mbar_test(&bar_ifull[is], (r / NIS) & 1) &&
                        (r < 2 || mbar_test(&bar_sempty[s], ((r >> 1) - 1) & 1)) &&
                        (c != 0 || mbar_test(&bar_afull, ti & 1))) {
                        tc_fence_after();
                        const uint32_t bH = smem_u32(smem + IMG_BASE + is * ISTAGE + ST_BH);
                        const uint32_t bL = smem_u32(smem + IMG_BASE + is * ISTAGE + ST_BL);
                        const uint32_t dS = tmem + (s ? TM_S1 : TM_S0);
#pragma unroll
                        for (int kk = 0; kk < KP / 16; ++kk) {
                            const uint64_t ah = sdesc_kmajor_sw128(aH + kk * 32);
                            const uint64_t al = sdesc_kmajor_sw128(aL + kk * 32);
                            const uint64_t bh = sdesc_kmajor_sw128(bH + kk * 32);
                            const uint64_t bl = sdesc_kmajor_sw128(bL + kk * 32);
                            mma_bf16(dS, ah, bh, IDESC, kk > 0 ? 1u : 0u);
                            mma_bf16(dS, ah, bl, IDESC, 1u);
                            mma_bf16(dS, al, bh, IDESC, 1u);
                        }
                        mma_commit(&bar_sfull[s]);
                        if (c == nch - 1) mma_commit(&bar_aempty);  // the tile's A operand is no longer read
                        ++r;
                        progressed = true;
                    }
                }
                if (m < r) {
                    const int ti = m / nch, c = m % nch;
                    if (mbar_test(&bar_dxfull, m & 1) &&
                        (c != 0 || ti < 2 || mbar_test(&bar_accempty[ti & 1], ((ti >> 1) - 1) & 1))) {
                        tc_fence_after();
                        if (do_update) {
                            // B_hi of the chunk read MN-major: K = streamed index (rows)
                            const uint32_t cB = smem_u32(smem + IMG_BASE + (m % NIS) * ISTAGE + ST_BH);
                            const uint32_t dDen = tmem + TM_ACC + 128 * (ti & 1);
#pragma unroll
                            for (int kk = 0; kk < NC / 16; ++kk) {
                                const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
                                mma_bf16(dDen, sdesc_kmajor_sw128(dA + kk * 32), sdesc_mnmajor_sw128(cB + kk * 2048),
                                         IDESC_MN, acc);
                                mma_bf16(dDen + 64, sdesc_kmajor_sw128(xA + kk * 32),
                                         sdesc_mnmajor_sw128(cB + kk * 2048), IDESC_MN, acc);
                            }
                        }
                        // with no new MMA (chi2-only) the commits still arrive after
                        // the earlier ones, so both modes follow one protocol
                        mma_commit(&bar_dxempty);
                        mma_commit(&bar_iempty[m % NIS]);
                        if (c == nch - 1) mma_commit(&bar_accfull[ti & 1]);
                        ++m;
                        progressed = true;
                    }
                }
                if (!progressed) {
                    __nanosleep(20);
                    if (s_abort) {
                        ok = false;
                    } else if (global_ns() - t0 > kWaitLimitNs) {
                        atomicCAS(err, 0, NMF_ETIMEOUT);
                        s_abort = 1;
                        ok = false;
                    }
                }
            }
        }
    } else if (warp < 2 + NEPI / 32) {
        // ------------------------------------------------------------ chunk warps
        const int e = warp - 2;               // 0..7
        const int q = warp & 3;               // TMEM lane quarter of this warp
        const int hf = e >> 2;                // which 32 of the 64 streamed columns
        const int row = 32 * q + lane;        // TMEM lane = M row in the tile
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        float chi = 0.0f;
        bool ok = true;
        for (int g = 0; g < G && ok; ++g) {
            const int s = g & 1;
            ok = mbar_wait(&bar_sfull[s], (g >> 1) & 1, &s_abort, err, NMF_ETIMEOUT);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc_fence_after();
            float r[32];
            tmem_ld16(tl + (s ? TM_S1 : TM_S0) + 32 * hf, *reinterpret_cast<float(*)[16]>(r));
            tmem_ld16(tl + (s ? TM_S1 : TM_S0) + 32 * hf + 16, *reinterpret_cast<float(*)[16]>(r + 16));
            tmem_ld_wait();
            tc_fence_before();
            mbar_arrive(&bar_sempty[s]);
            ok = mbar_wait(&bar_dfull[g % NDS], (g / NDS) & 1, &s_abort, err, NMF_ETIMEOUT);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            const uint8_t *stg = smem + (g % NDS) * DSTAGE;
            uint4 dpk[4], xpk[4];
#pragma unroll
            for (int cb = 0; cb < 4; ++cb) {
                float v[8], w[8];
                if (HPASS) {
                    // column `row` (pixel) of rows 32hf + 8cb + i (streamed refs)
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int n = 32 * hf + 8 * cb + i;
                        v[i] = reinterpret_cast<const float *>(stg + ST_V)[n * TILE + row];
                        w[i] = __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(stg + ST_WT)[n * TILE + row]);
                    }
                } else {
                    // row `row` (frame), streamed pixels 32hf + 8cb .. +8, 128-byte swizzled tiles
                    const uint8_t *vb = stg + ST_V + hf * 16384 + row * 128;
                    const float4 v0 = *reinterpret_cast<const float4 *>(vb + (((2 * cb) ^ (row & 7)) << 4));
                    const float4 v1 = *reinterpret_cast<const float4 *>(vb + (((2 * cb + 1) ^ (row & 7)) << 4));
                    v[0] = v0.x; v[1] = v0.y; v[2] = v0.z; v[3] = v0.w;
                    v[4] = v1.x; v[5] = v1.y; v[6] = v1.z; v[7] = v1.w;
                    const uint4 wb = *reinterpret_cast<const uint4 *>(stg + ST_WT + row * 128 +
                                                                     (((4 * hf + cb) ^ (row & 7)) << 4));
                    bf16x8_to_f32(wb, w);
                }
                dx8(r + 8 * cb, v, w, dpk[cb], xpk[cb], chi);
            }
            mbar_arrive(&bar_dempty[g % NDS]);  // this thread has read its V and Wt
            // the D/X buffers are free once the previous chunk's den/G MMAs are done
            if (g >= 1) ok = mbar_wait(&bar_dxempty, (g - 1) & 1, &s_abort, err, NMF_ETIMEOUT);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            if (do_update) {
#pragma unroll
                for (int cb = 0; cb < 4; ++cb) {
                    const uint32_t off = (uint32_t)sw_elem(row, 32 * hf + 8 * cb);
                    *reinterpret_cast<uint4 *>(smem + OFF_D + off) = dpk[cb];
                    *reinterpret_cast<uint4 *>(smem + OFF_X + off) = xpk[cb];
                }
                fence_proxy_async_smem();
            }
            mbar_arrive(&bar_dxfull);
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
            for (int i = 0; i <= ntm && ok; ++i) {
                if (i < ntm) {
                    // H operand (A of W H) of tile i: row = pixel, 64 components, hi/lo
                    const long long p = tile_m0(i) + row;
                    float hv[KP];
#pragma unroll
                    for (int j = 0; j < KP; ++j) hv[j] = (j < a.k) ? __ldg(Hin + (long long)j * Pp + p) : 0.0f;
                    if (i >= 1) ok = mbar_wait(&bar_aempty, (i - 1) & 1, &s_abort, err, NMF_ETIMEOUT);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
#pragma unroll
                    for (int cb = 0; cb < KP / 8; ++cb) {
                        float hi[8], lo[8];
#pragma unroll
                        for (int ii = 0; ii < 8; ++ii) {
                            hi[ii] = __bfloat162float(__float2bfloat16_rn(hv[8 * cb + ii]));
                            lo[ii] = bf16_lo_part(hv[8 * cb + ii], hi[ii]);
                        }
                        const uint32_t off = sw_elem(row, 8 * cb);
                        *reinterpret_cast<uint4 *>(smem + OFF_AH + off) =
                            make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]),
                                       pack_bf16(hi[6], hi[7]));
                        *reinterpret_cast<uint4 *>(smem + OFF_AL + off) =
                            make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]),
                                       pack_bf16(lo[6], lo[7]));
                    }
                    fence_proxy_async_smem();
                    mbar_arrive(&bar_afull);
                }
                if (i >= 1) {
                    // Eq. 3 update of tile i-1:  H <- H (den + G) / max(den, eps)
                    const int tp = i - 1, b = tp & 1;
                    ok = mbar_wait(&bar_accfull[b], (tp >> 1) & 1, &s_abort, err, NMF_ETIMEOUT);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    tc_fence_after();
                    const long long p = tile_m0(tp) + row;
                    uint8_t *hk_hi = a.outHKh + (p >> 6) * IMG_CHUNK;
                    uint8_t *hk_lo = a.outHKl + (p >> 6) * IMG_CHUNK;
                    const uint32_t pr = (uint32_t)(p & 63);
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        // all loads of the old H first (read-only path), then the stores
                        float hold[32];
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            const int j = 32 * half + jj;
                            hold[jj] = (j < a.k) ? __ldg(Hin + (long long)j * Pp + p) : 0.0f;
                        }
                        float den[32], g[32];
                        const uint32_t acc = tl + TM_ACC + 128 * b + 32 * half;
                        tmem_ld16(acc, *reinterpret_cast<float(*)[16]>(den));
                        tmem_ld16(acc + 16, *reinterpret_cast<float(*)[16]>(den + 16));
                        tmem_ld16(acc + 64, *reinterpret_cast<float(*)[16]>(g));
                        tmem_ld16(acc + 80, *reinterpret_cast<float(*)[16]>(g + 16));
                        tmem_ld_wait();
                        if (do_update) {
#pragma unroll
                            for (int cb = 0; cb < 4; ++cb) {
                                float hi[8], lo[8], hn[8];
#pragma unroll
                                for (int ii = 0; ii < 8; ++ii) {
                                    const int jj = 8 * cb + ii, j = 32 * half + jj;
                                    const float h = hold[jj];
                                    const float nv =
                                        h == 0.0f ? 0.0f : __fdividef(h * (den[jj] + g[jj]), fmaxf(den[jj], a.eps));
                                    hn[ii] = nv;
                                    if (j < a.k) Hout[(long long)j * Pp + p] = nv;
                                    hi[ii] = __bfloat162float(__float2bfloat16_rn(nv));
                                    lo[ii] = bf16_lo_part(nv, hi[ii]);
                                }
                                const uint32_t off = sw_elem(pr, 32 * half + 8 * cb);
                                *reinterpret_cast<uint4 *>(hk_hi + off) =
                                    make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]),
                                               pack_bf16(hi[4], hi[5]), pack_bf16(hi[6], hi[7]));
                                *reinterpret_cast<uint4 *>(hk_lo + off) =
                                    make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]),
                                               pack_bf16(lo[4], lo[5]), pack_bf16(lo[6], lo[7]));
                            }
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(&bar_accempty[b]);
                }
            }
        } else {
            // partial sums of this pixel split for the W (or C) update
            ok = __all_sync(0xffffffffu, mbar_wait(&bar_accfull[0], 0, &s_abort, err, NMF_ETIMEOUT));
            tc_fence_after();
            if (ok && do_update) {
                const long long n = tile_m0(0) + row;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    float den[32], g[32];
                    const uint32_t acc = tl + TM_ACC + 32 * half;
                    tmem_ld16(acc, *reinterpret_cast<float(*)[16]>(den));
                    tmem_ld16(acc + 16, *reinterpret_cast<float(*)[16]>(den + 16));
                    tmem_ld16(acc + 64, *reinterpret_cast<float(*)[16]>(g));
                    tmem_ld16(acc + 80, *reinterpret_cast<float(*)[16]>(g + 16));
                    tmem_ld_wait();
                    if (n < rows_total) {
                        float *pp = a.part + ((long long)blockIdx.x * rows_total + n) * (2 * KP);
#pragma unroll
                        for (int jj = 0; jj < 32; jj += 4) {
                            *reinterpret_cast<float4 *>(pp + 32 * half + jj) =
                                make_float4(den[jj], den[jj + 1], den[jj + 2], den[jj + 3]);
                            *reinterpret_cast<float4 *>(pp + KP + 32 * half + jj) =
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
    if (warp == 1) tmem_dealloc(tmem, TM_COLS);
    if (HPASS) {
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < NEPI / 32; ++w) tot += s_red[w];
            a.chi2_part[blockIdx.x] = tot;
            __threadfence();
            const unsigned tk = atomicAdd(&st->ticket_h, 1u);
            s_last = (tk == gridDim.x - 1);
        }
        __syncthreads();
        if (s_last) {
            // fixed-order FP64 sum of the per-block partials by all threads
            __threadfence();
            double v = 0.0;
            for (unsigned b = tid; b < gridDim.x; b += THREADS) v += __ldcg(a.chi2_part + b);
            v = warp_sum_f64_tc(v);
            if (lane == 0) s_red[warp] = v;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int w = 0; w < THREADS / 32; ++w) tot += s_red[w];
                st->ticket_h = 0;
                if (tot == tot) {  // a timed-out pass leaves the cost undefined; keep the record
                    if (a.tol > 0.0 && t >= 2 && (st->chi2_prev - tot) <= a.tol * st->chi2_prev) st->stop = 1;
                    st->chi2_prev = tot;
                    st->chi2_last = tot;
                    st->iters_kept = t;
                    st->final_buf = t & 1;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// W (or C) update: fixed-order sum over the pixel splits, Eq. 3, and the
// BF16 operand images of the new coefficients.  One warp per coefficient.

__global__ void __launch_bounds__(256) wupdate_tc_kernel(TcArgs a) {
    FitState *st = a.st;
    if (st->stop | st->status) return;
    const long long gw = ((long long)blockIdx.x * 256 + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t = st->t + 1;
    if (gw >= a.rows * a.k) return;
    const long long n = gw / a.k;
    const int j = (int)(gw % a.k);
    float sd = 0.f, sg = 0.f;
    for (int sp = lane; sp < a.nsplit; sp += 32) {
        const float *pp = a.part + ((long long)sp * a.rows + n) * (2 * KP);
        sd += __ldcg(pp + j);
        sg += __ldcg(pp + KP + j);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
        sg += __shfl_xor_sync(0xffffffffu, sg, o);
    }
    if (lane == 0) {
        float *wp = a.W + n * a.ldw + j;
        const float w = *wp;
        const float nw = w == 0.0f ? 0.0f : (w * (sd + sg)) / fmaxf(sd, a.eps);
        *wp = nw;
        const __nv_bfloat16 hi = __float2bfloat16_rn(nw);
        const __nv_bfloat16 lo = __float2bfloat16_rn(nw - __bfloat162float(hi));
        const long long ch = n >> 6;
        const uint32_t r = (uint32_t)(n & 63);
        *reinterpret_cast<__nv_bfloat16 *>(a.outWKh + ch * IMG_CHUNK + sw_elem(r, j)) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(a.outWKl + ch * IMG_CHUNK + sw_elem(r, j)) = lo;
    }
}

// Operand images (hi, lo) of a coefficient matrix (rows x k, ld ldw) or of a
// basis (k x Pp): element (row, j).  Entries outside [0, k) x [0, rows) are
// left as they are (zero).
__global__ void images_kernel(const float *X, long long rows, int k, long long ld, int x_is_kxP, uint8_t *Kh,
                              uint8_t *Kl) {
    const long long total = rows * k;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long n = i / k;
        const int j = (int)(i % k);
        const float v = x_is_kxP ? X[(long long)j * ld + n] : X[n * ld + j];
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        const long long ch = n >> 6;
        const uint32_t r = (uint32_t)(n & 63);
        *reinterpret_cast<__nv_bfloat16 *>(Kh + ch * IMG_CHUNK + sw_elem(r, j)) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(Kl + ch * IMG_CHUNK + sw_elem(r, j)) = lo;
    }
}

// Weights to BF16 (row-padded copy, zero padding).
__global__ void weights_bf16_kernel(const float *src, long long rows, long long cols, long long ld_src,
                                    __nv_bfloat16 *dst, long long ld_dst, FitState *st) {
    const long long total = rows * ld_dst;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / ld_dst, c = i % ld_dst;
        float x = 0.0f;
        if (c < cols) {
            x = src[r * ld_src + c];
            if (!(x >= 0.0f && x <= 3.402823466e38f)) bad = true;
        }
        dst[i] = __float2bfloat16_rn(x);
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

cudaError_t set_smem(const void *kern) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, kern})) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
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

int tc_max_k() { return KP; }
int tc_chunk() { return NC; }
int tc_tile() { return TILE; }
size_t tc_image_bytes(long long rows) { return (size_t)((rows + 127) / 128 * 2) * IMG_CHUNK; }

cudaError_t tc_weights_bf16(const float *src, long long rows, long long cols, void *dst, long long ld_dst,
                            FitState *st, cudaStream_t s) {
    count_launches(1);
    weights_bf16_kernel<<<grid_1d(rows * ld_dst), 256, 0, s>>>(src, rows, cols, cols,
                                                                 reinterpret_cast<__nv_bfloat16 *>(dst), ld_dst, st);
    return cudaGetLastError();
}

cudaError_t tc_images(const float *X, long long rows, int k, long long ld, bool x_is_kxP, uint8_t *Kh, uint8_t *Kl,
                      cudaStream_t s) {
    if (rows * k == 0) return cudaSuccess;
    count_launches(1);
    images_kernel<<<grid_1d(rows * k), 256, 0, s>>>(X, rows, k, ld, x_is_kxP ? 1 : 0, Kh, Kl);
    return cudaGetLastError();
}

bool tc_make_maps(TcMaps *m, const float *V, const void *Wtb, long long rows, long long Pp) {
    bool ok = true;
    ok &= make_map(&m->hV, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, V, Pp, rows, Pp, TILE, NC, CU_TENSOR_MAP_SWIZZLE_NONE);
    ok &= make_map(&m->hWt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Wtb, Pp, rows, Pp, TILE, NC,
                   CU_TENSOR_MAP_SWIZZLE_NONE);
    ok &= make_map(&m->wV, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, V, Pp, rows, Pp, 32, TILE, CU_TENSOR_MAP_SWIZZLE_128B);
    ok &= make_map(&m->wWt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Wtb, Pp, rows, Pp, 64, TILE,
                   CU_TENSOR_MAP_SWIZZLE_128B);
    return ok;
}

cudaError_t tc_hpass(const TcMaps &m, const TcArgs &a, bool chi2_only, cudaStream_t s) {
    auto kern = pass_tc_kernel<true>;
    cudaError_t e = set_smem(reinterpret_cast<const void *>(kern));
    if (e != cudaSuccess) return e;
    const int ntiles = (int)(a.Pp / TILE);
    const int grid = ntiles < num_sms() ? ntiles : num_sms();
    count_launches(1);
    kern<<<(unsigned)grid, THREADS, SMEM_BYTES, s>>>(m.hV, m.hWt, a, chi2_only ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t tc_wpass(const TcMaps &m, const TcArgs &a, cudaStream_t s) {
    auto kern = pass_tc_kernel<false>;
    cudaError_t e = set_smem(reinterpret_cast<const void *>(kern));
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)a.nsplit, (unsigned)((a.rows + TILE - 1) / TILE));
    count_launches(2);
    kern<<<grid, THREADS, SMEM_BYTES, s>>>(m.wV, m.wWt, a, 0);
    const long long warps = a.rows * a.k;
    wupdate_tc_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace nmfgb
