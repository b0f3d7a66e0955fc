// FP32 CUDA-core kernels of the weighted-NMF hot path (arXiv:2309.04623,
// Sec. 2 Eq. 2-3 and Sec. 4.1).  This is the plain FP32 form: every product
// and sum is a float FMA, so it follows the FP64 oracle to ~1e-6.
//
// Per iteration at rank k the hot path streams the N x P data twice:
//   H pass  (one block per pixel tile, loop over all N rows):
//           R = W H_tile, chi2 += Wt (V - R)^2, num += W^T (Wt o V),
//           den += W^T (Wt o R); epilogue H <- H num / max(den, eps).
//   W pass  (one block per row tile x pixel split, loop over the split):
//           R = W H_new, num += (Wt o V) H^T, den += (Wt o R) H^T into
//           per-split partials; a reduction kernel sums the splits in a fixed
//           order (one warp per coefficient) and applies
//           W <- W num / max(den, eps).
// The N x P reconstruction W H is never written to memory.  The cost Eq. 2
// of the incoming iterate is reduced in FP64 by the H pass, and its last
// block applies the stopping rule on the device.
#include <math.h>

#include <mutex>
#include <set>
#include <utility>

#include "nmf_internal.cuh"

namespace nmfgb {

// ---------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous global->shared copy; zero-fills when !pred (the
// source operand is then a valid dummy address and no byte is read).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(pred ? 16 : 0));
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool pred) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(pred ? 4 : 0));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ double warp_sum_f64(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// The multiplicative rule with the zero guard and the epsilon clamp (Eq. 3),
// then the tiny-entry rule (flush_tiny).
__device__ __forceinline__ float mu_update(float x, float num, float den, float eps) {
    return x == 0.0f ? 0.0f : flush_tiny((x * num) / fmaxf(den, eps));
}

// Fixed-order FP64 sum of `count` partials by one block (deterministic).
template <int THREADS>
__device__ double block_sum_partials(const double *part, int count, double *red) {
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += THREADS) v += __ldcg(part + i);
    v = warp_sum_f64(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < THREADS / 32; ++w) tot += red[w];
    return tot;  // valid in thread 0
}

// Stopping rule (Sec. 2), applied when the cost of the state after t
// iterations is known.  Called by one thread.
__device__ void record_cost(FitState *st, int t, double c, double tol) {
    if (tol > 0.0 && t >= 2 && (st->chi2_prev - c) <= tol * st->chi2_prev) st->stop = 1;
    st->chi2_prev = c;
    st->chi2_last = c;
    st->iters_kept = t;
    st->final_buf = t & 1;
}

// ---------------------------------------------------------------------------
// H pass

constexpr int HP_THREADS = 128;
#ifndef NMF_HP_NC
#define NMF_HP_NC 16
#endif
#ifndef NMF_HP_MINB
#define NMF_HP_MINB 4
#endif
// Lanes per pixel in the H pass for k <= 32 (1: one thread holds all 32
// components; 2: two lanes split them, halving the registers per thread).
#ifndef NMF_HP_SL32
#define NMF_HP_SL32 2
#endif
constexpr int HP_NC = NMF_HP_NC;  // rows per staged chunk

// W rows are staged with each lane's KS components padded to KS + 4 floats,
// so the SL lanes of a pixel read different shared-memory banks.
template <int KS, int SL>
__host__ __device__ constexpr int hp_row_floats() { return SL * (KS + 4); }

template <int KS, int SL>
__host__ __device__ constexpr int hp_smem_floats() {
    return 4 * HP_NC * (HP_THREADS / SL) + 2 * HP_NC * hp_row_floats<KS, SL>();
}

// Thread layout: SL adjacent lanes share one pixel; lane s of the group owns
// components [s*KS, (s+1)*KS).  The partial dot products of R are combined
// with xor shuffles inside the group.
template <int KS, int SL, bool CHI2_ONLY>
__global__ void __launch_bounds__(HP_THREADS, (KS >= 32 ? 3 : NMF_HP_MINB)) hpass_f32_kernel(PassArgs a) {
    constexpr int PX = HP_THREADS / SL;  // pixels per block
    constexpr int KP = KS * SL;
    extern __shared__ __align__(16) float smem[];
    float *Vs = smem;                  // [2][NC][PX]
    float *Ws = Vs + 2 * HP_NC * PX;   // [2][NC][PX]
    constexpr int KPP = hp_row_floats<KS, SL>();
    float *Wm = Ws + 2 * HP_NC * PX;   // [2][NC][SL][KS + 4]
    __shared__ double red[HP_THREADS / 32];
    __shared__ int s_flag, s_t, s_last;

    FitState *st = a.st;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_flag = st->stop | st->status;
        s_t = st->t;
    }
    __syncthreads();
    if (s_flag) return;
    const int t = s_t;
    const float *Hin = (t & 1) ? a.Hb1 : a.Hb0;
    float *Hout = (t & 1) ? a.Hb0 : a.Hb1;

    const int s = tid % SL, q = tid / SL;
    const long long Pp = a.Pp;
    const long long p0 = (long long)blockIdx.x * PX;
    const long long p = p0 + q;
    const bool pin = p < Pp;
    const int j0 = s * KS;

    float h[KS], num[KS], den[KS];
#pragma unroll
    for (int j = 0; j < KS; ++j) {
        const int jg = j0 + j;
        h[j] = (pin && jg < a.k) ? __ldg(Hin + (long long)jg * Pp + p) : 0.0f;
        num[j] = 0.0f;
        den[j] = 0.0f;
    }

    const long long N = a.rows;
    const int nch = (int)((N + HP_NC - 1) / HP_NC);
    auto stage = [&](int c, int b) {
        const long long n0 = (long long)c * HP_NC;
        for (int i = tid; i < HP_NC * PX / 4; i += HP_THREADS) {
            const int r = i / (PX / 4), c4 = i % (PX / 4);
            const long long n = n0 + r, pp = p0 + c4 * 4;
            const bool ok = n < N && pp < Pp;
            const long long off = ok ? n * Pp + pp : 0;
            cp_async16(Vs + (b * HP_NC + r) * PX + c4 * 4, a.V + off, ok);
            cp_async16(Ws + (b * HP_NC + r) * PX + c4 * 4, a.Wt + off, ok);
        }
        for (int i = tid; i < HP_NC * KP / 4; i += HP_THREADS) {
            const int r = i / (KP / 4), c4 = i % (KP / 4);
            const long long n = n0 + r;
            const bool ok = n < N;
            const int jj = c4 * 4;
            cp_async16(Wm + (b * HP_NC + r) * KPP + (jj / KS) * (KS + 4) + jj % KS,
                       a.W + (ok ? n * a.ldw + jj : 0), ok);
        }
        cp_async_commit();
    };

    float chi = 0.0f;
    stage(0, 0);
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        if (c + 1 < nch) {
            stage(c + 1, b ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *vs = Vs + b * HP_NC * PX;
        const float *ws = Ws + b * HP_NC * PX;
        const float *wm = Wm + b * HP_NC * KPP + s * (KS + 4);
#pragma unroll 1
        for (int r = 0; r < HP_NC; ++r) {
            // the W row is read from shared memory (a broadcast) once for R
            // and once for the updates, so only 4 values are live at a time
            const float4 *wr4 = reinterpret_cast<const float4 *>(wm + r * KPP);
            float racc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < KS; j += 4) {
                const float4 w4 = wr4[j / 4];
                racc[0] = fmaf(w4.x, h[j], racc[0]);
                racc[1] = fmaf(w4.y, h[j + 1], racc[1]);
                racc[2] = fmaf(w4.z, h[j + 2], racc[2]);
                racc[3] = fmaf(w4.w, h[j + 3], racc[3]);
            }
            float rr = (racc[0] + racc[1]) + (racc[2] + racc[3]);
#pragma unroll
            for (int o = 1; o < SL; o <<= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
            const float v = vs[r * PX + q], w = ws[r * PX + q];
            if (!CHI2_ONLY) {
                const float av = w * v, d = w * rr;
#pragma unroll
                for (int j = 0; j < KS; j += 4) {
                    const float4 w4 = wr4[j / 4];
                    num[j] = fmaf(w4.x, av, num[j]);
                    den[j] = fmaf(w4.x, d, den[j]);
                    num[j + 1] = fmaf(w4.y, av, num[j + 1]);
                    den[j + 1] = fmaf(w4.y, d, den[j + 1]);
                    num[j + 2] = fmaf(w4.z, av, num[j + 2]);
                    den[j + 2] = fmaf(w4.z, d, den[j + 2]);
                    num[j + 3] = fmaf(w4.w, av, num[j + 3]);
                    den[j + 3] = fmaf(w4.w, d, den[j + 3]);
                }
            }
            const float e = v - rr;
            chi = fmaf(w * e, e, chi);
        }
        __syncthreads();
    }

    if (!CHI2_ONLY && pin) {
#pragma unroll
        for (int j = 0; j < KS; ++j) {
            const int jg = j0 + j;
            if (jg < a.k) Hout[(long long)jg * Pp + p] = mu_update(h[j], num[j], den[j], a.eps);
        }
    }

    // Eq. 2 of the incoming iterate: FP32 per thread, FP64 across threads.
    double cd = (s == 0) ? (double)chi : 0.0;
    cd = warp_sum_f64(cd);
    if ((tid & 31) == 0) red[tid >> 5] = cd;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < HP_THREADS / 32; ++w) tot += red[w];
        a.chi2_part[blockIdx.x] = tot;
        __threadfence();
        const unsigned tk = atomicAdd(&st->ticket_h, 1u);
        s_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const double tot = block_sum_partials<HP_THREADS>(a.chi2_part, gridDim.x, red);
        if (tid == 0) {
            st->ticket_h = 0;
            record_cost(st, t, tot, a.tol);
        }
    }
}

// ---------------------------------------------------------------------------
// W pass (also the projection of science frames, with H fixed)

constexpr int WP_THREADS = 128;  // 4 warps, each takes every 4th pixel of a chunk

template <int KP>
__host__ __device__ constexpr int wp_chunk() {
    return KP <= 32 ? 128 : (KP == 64 ? 64 : 32);
}

template <int KS, int SL>
__host__ __device__ constexpr int wp_smem_floats() {
    constexpr int KP = KS * SL, RT = 32 / SL, PC = wp_chunk<KS * SL>();
    constexpr int main_ = 4 * RT * (PC + 1) + 2 * PC * (SL * (KS + 4) + 4);
    constexpr int red_ = 4 * 32 * 2 * KS;
    return main_ > red_ ? main_ : red_;
}

// Thread layout: a warp holds RT = 32/SL rows, SL adjacent lanes per row
// (lane s owns components [s*KS, (s+1)*KS)); the 4 warps of a block split the
// pixels of each chunk and are summed at the end.
template <int KS, int SL, int MODE>
__global__ void __launch_bounds__(WP_THREADS) wpass_f32_kernel(PassArgs a) {
    constexpr int KP = KS * SL, RT = 32 / SL, PC = wp_chunk<KP>();
    constexpr int VST = PC + 1;   // odd row stride: lanes of different rows hit different banks
    // H chunk stored transposed [pixel][lane group][KS + 4]: the SL lanes of a
    // row read different banks
    constexpr int HST = SL * (KS + 4) + 4;
    extern __shared__ __align__(16) float smem[];
    float *Vs = smem;                 // [2][RT][VST]
    float *Ws = Vs + 2 * RT * VST;    // [2][RT][VST]
    float *Hs = Ws + 2 * RT * VST;    // [2][PC][HST]
    __shared__ int s_flag, s_t;

    FitState *st = a.st;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_flag = st->stop | st->status;
        s_t = st->t;
    }
    __syncthreads();
    if (s_flag) return;
    // the H pass of this iteration wrote its result into buffer (t+1)&1
    const float *Hn = (s_t & 1) ? a.Hb0 : a.Hb1;

    const int lane = tid & 31, warp = tid >> 5;
    const int s = lane % SL, r = lane / SL;
    const long long rows = a.rows, Pp = a.Pp;
    const long long n0 = (long long)blockIdx.y * RT;
    const long long n = n0 + r;
    const bool nin = n < rows;
    const int j0 = s * KS;

    float wr[KS], num[KS], den[KS];
#pragma unroll
    for (int j = 0; j < KS; ++j) {
        wr[j] = (nin && j0 + j < a.k) ? a.W[n * a.ldw + j0 + j] : 0.0f;
        num[j] = 0.0f;
        den[j] = 0.0f;
    }

    const long long pa = (long long)blockIdx.x * a.split_len;
    const long long pb = (pa + a.split_len < Pp) ? pa + a.split_len : Pp;
    const int nch = (int)((pb - pa + PC - 1) / PC);
    auto stage = [&](int c, int b) {
        const long long pc0 = pa + (long long)c * PC;
        for (int i = tid; i < RT * PC; i += WP_THREADS) {
            const int rr = i / PC, col = i % PC;
            const long long nn = n0 + rr, pp = pc0 + col;
            const bool ok = nn < rows && pp < pb;
            const long long off = ok ? nn * Pp + pp : 0;
            cp_async4(Vs + (b * RT + rr) * VST + col, a.V + off, ok);
            cp_async4(Ws + (b * RT + rr) * VST + col, a.Wt + off, ok);
        }
        for (int i = tid; i < KP * PC; i += WP_THREADS) {
            const int j = i / PC, col = i % PC;
            const long long pp = pc0 + col;
            const bool ok = j < a.k && pp < pb;
            cp_async4(Hs + (b * PC + col) * HST + (j / KS) * (KS + 4) + j % KS, Hn + (ok ? (long long)j * Pp + pp : 0),
                      ok);
        }
        cp_async_commit();
    };

    stage(0, 0);
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        if (c + 1 < nch) {
            stage(c + 1, b ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *vs = Vs + (b * RT + r) * VST;
        const float *ws = Ws + (b * RT + r) * VST;
        const float *hs = Hs + b * PC * HST + s * (KS + 4);
#pragma unroll 2
        for (int pp = warp; pp < PC; pp += 4) {
            float hv[KS];
#pragma unroll
            for (int j = 0; j < KS; j += 4) {
                const float4 h4 = *reinterpret_cast<const float4 *>(hs + pp * HST + j);
                hv[j] = h4.x;
                hv[j + 1] = h4.y;
                hv[j + 2] = h4.z;
                hv[j + 3] = h4.w;
            }
            float racc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < KS; ++j) racc[j & 3] = fmaf(wr[j], hv[j], racc[j & 3]);
            float rr = (racc[0] + racc[1]) + (racc[2] + racc[3]);
#pragma unroll
            for (int o = 1; o < SL; o <<= 1) rr += __shfl_xor_sync(0xffffffffu, rr, o);
            const float v = vs[pp], w = ws[pp];
            const float d = w * rr;
            if (MODE != WP_PROJ_NEXT) {
                const float av = w * v;
#pragma unroll
                for (int j = 0; j < KS; ++j) num[j] = fmaf(av, hv[j], num[j]);
            }
#pragma unroll
            for (int j = 0; j < KS; ++j) den[j] = fmaf(d, hv[j], den[j]);
        }
        __syncthreads();
    }

    // sum the 4 warps (fixed order) and write this split's partials
    float *red = smem;  // [4][32][2*KS]
#pragma unroll
    for (int j = 0; j < KS; ++j) {
        red[(warp * 32 + lane) * 2 * KS + j] = num[j];
        red[(warp * 32 + lane) * 2 * KS + KS + j] = den[j];
    }
    __syncthreads();
    if (warp == 0 && nin) {
        float *pn = a.part + ((long long)blockIdx.x * rows + n) * 2 * a.ldw;
        for (int j = 0; j < KS; ++j) {
            if (j0 + j >= a.k) break;
            float sn = 0.f, sd = 0.f;
            for (int w = 0; w < 4; ++w) {
                sn += red[(w * 32 + lane) * 2 * KS + j];
                sd += red[(w * 32 + lane) * 2 * KS + KS + j];
            }
            pn[j0 + j] = sn;
            pn[a.ldw + j0 + j] = sd;
        }
    }
}

// Sum the W-pass partials over the pixel splits and apply Eq. 3 to W (or to
// the projection coefficients C).  One warp per (row, component): lane l sums
// splits l, l+32, ... and a fixed shuffle tree combines the lanes, so the
// result is deterministic.  Block 0 advances the iteration counter.
template <int MODE>
__global__ void __launch_bounds__(256) wreduce_kernel(PassArgs a) {
    FitState *st = a.st;
    if (st->stop | st->status) return;
    const long long gw = ((long long)blockIdx.x * 256 + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t = st->t + 1;
    if (gw >= a.rows * a.k) return;
    const long long n = gw / a.k;
    const int j = (int)(gw % a.k);
    float sn = 0.f, sd = 0.f;
    for (int sp = lane; sp < a.nsplit; sp += 32) {
        const float *pn = a.part + ((long long)sp * a.rows + n) * 2 * a.ldw;
        if (MODE != WP_PROJ_NEXT) sn += __ldcg(pn + j);
        sd += __ldcg(pn + a.ldw + j);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    if (lane == 0) {
        if (MODE == WP_PROJ_FIRST) a.num_const[n * a.ldw + j] = sn;
        if (MODE == WP_PROJ_NEXT) sn = a.num_const[n * a.ldw + j];
        float *wp = a.W + n * a.ldw + j;
        *wp = mu_update(*wp, sn, sd, a.eps);
    }
}

// ---------------------------------------------------------------------------
// per-stage bookkeeping

__global__ void stage_begin_kernel(FitState *st) {
    st->stop = 0;
    st->t = 0;
    st->h_done = 0;
    st->iters_kept = 0;
    st->final_buf = 0;
    st->ticket_h = 0;
    st->ticket_all = 0;
    st->chi2_prev = 0.0;
}

// Resume iterating after the stopping rule fired (the FP32 polish): clear
// the flag and allow extra_iters more iterations.
__global__ void clear_stop_kernel(FitState *st, int extra_iters) {
    st->stop = 0;
    st->t_limit = st->t + extra_iters;
}

// Loop control of a stage's iteration loop recorded as a graph WHILE node:
// keep iterating while iterations remain (t < n_iter, or t < t_limit when
// n_iter < 0), the stopping rule has not fired and no error is recorded.
__global__ void loop_ctl_kernel(const FitState *st, int n_iter, cudaGraphConditionalHandle h) {
    const int limit = n_iter < 0 ? st->t_limit : n_iter;
    const int go = !(st->stop | st->status) && st->t < limit;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Per-stage normalisation, first half: partial sums of squares of every H
// row of the kept state, NORM_SLICES slices per row (FP32 per thread, FP64
// across threads).
constexpr int NORM_SLICES = 16;

__global__ void __launch_bounds__(256) norm_partial_kernel(PassArgs a) {
    __shared__ double red[8];
    const FitState *st = a.st;
    const int i = blockIdx.x, sl = blockIdx.y;
    const float *row = (st->final_buf ? a.Hb1 : a.Hb0) + (long long)i * a.Pp;
    float v = 0.0f;
    for (long long p = (long long)sl * 256 + threadIdx.x; p < a.Pp; p += NORM_SLICES * 256) v = fmaf(row[p], row[p], v);
    double d = warp_sum_f64((double)v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += red[w];
        a.norm_part[i * NORM_SLICES + sl] = tot;
    }
}

// Second half: move the kept state into buffer 0 and, with normalisation,
// give every H row unit L2 norm (FP64 norm) and scale the matching W column
// by it, so W H is unchanged.  Block (x, i): pixels [256x, 256x+256) of row
// i; the extra block x = gridDim.x - 1 scales column i of W.
__global__ void __launch_bounds__(256) stage_end_kernel(PassArgs a, int normalize, double *chi2_hist,
                                                        int32_t *iters_done, int kidx) {
    __shared__ double s_scale;
    const FitState *st = a.st;
    const int i = blockIdx.y;
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int sl = 0; sl < NORM_SLICES; ++sl) tot += a.norm_part[i * NORM_SLICES + sl];
        s_scale = sqrt(tot);
    }
    __syncthreads();
    const double sc = s_scale;
    const bool scale = normalize && sc > 0.0;
    const float *src = (st->final_buf ? a.Hb1 : a.Hb0) + (long long)i * a.Pp;
    float *dst = a.Hb0 + (long long)i * a.Pp;
    if (blockIdx.x == gridDim.x - 1) {
        if (scale)
            for (long long n = threadIdx.x; n < a.rows; n += 256)
                a.W[n * a.ldw + i] = flush_tiny((float)((double)a.W[n * a.ldw + i] * sc));
    } else {
        const long long p = (long long)blockIdx.x * 256 + threadIdx.x;
        if (p < a.Pp) {
            if (scale)
                dst[p] = flush_tiny((float)((double)src[p] / sc));
            else if (src != dst)
                dst[p] = src[p];
        }
    }
    if (blockIdx.x == 0 && i == 0 && threadIdx.x == 0) {
        chi2_hist[kidx] = st->chi2_last;
        iters_done[kidx] = st->iters_kept;
    }
}

// Copy rows x cols from a strided source into a strided destination whose
// columns [cols, dst_cols) are zero-filled; optionally flag negative or
// non-finite values in the control block.
__global__ void prologue_copy_kernel(const float *src, long long rows, long long cols, long long ld_src, float *dst,
                                     long long ld_dst, long long dst_cols, FitState *st, int check) {
    const long long total = rows * dst_cols;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / dst_cols, c = i % dst_cols;
        float x = 0.0f;
        if (c < cols) {
            x = src[r * ld_src + c];
            if (check && !(x >= 0.0f && x <= 3.402823466e38f)) bad = true;
        }
        dst[r * ld_dst + c] = x;
    }
    if (bad) atomicExch(&st->status, (int)NMF_EDATA);
}

__global__ void copy_out_kernel(const float *src, long long rows, long long cols, long long ld_src, float *dst,
                                long long ld_dst) {
    const long long total = rows * cols;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / cols, c = i % cols;
        dst[r * ld_dst + c] = src[r * ld_src + c];
    }
}

// ---------------------------------------------------------------------------
// PSF subtraction (Sec. 4.1): R = T - f (C H), optional scatter to the image.

__global__ void __launch_bounds__(256) subtract_kernel(const float *T, const float *C, const float *H, long long M,
                                                       int K, long long P, const float *factor, float *R,
                                                       const int32_t *scatter_idx, float *img,
                                                       long long img_pixels) {
    __shared__ float cs[kMaxK];
    const long long m = blockIdx.y;
    for (int i = threadIdx.x; i < K; i += 256) cs[i] = C[m * K + i];
    __syncthreads();
    const float f = factor ? factor[m] : 1.0f;
    const long long p = (long long)blockIdx.x * 256 + threadIdx.x;
    if (p >= P) return;
    float model = 0.0f;
    for (int i = 0; i < K; ++i) model = fmaf(cs[i], H[(long long)i * P + p], model);
    const float res = T[m * P + p] - f * model;
    R[m * P + p] = res;
    if (img) img[m * img_pixels + scatter_idx[p]] = res;
}

// ---------------------------------------------------------------------------
// launchers

static inline int grid_for(long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_prologue_copy(const float *src, long long rows, long long cols, long long ld_src, float *dst,
                                 long long ld_dst, long long dst_cols, FitState *st, int check, cudaStream_t s) {
    if (rows * dst_cols == 0) return cudaSuccess;
    count_launches(1);
    prologue_copy_kernel<<<grid_for(rows * dst_cols, 256), 256, 0, s>>>(src, rows, cols, ld_src, dst, ld_dst,
                                                                          dst_cols, st, check);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(const float *src, long long rows, long long cols, long long ld_src, float *dst,
                            long long ld_dst, cudaStream_t s) {
    if (rows * cols == 0) return cudaSuccess;
    count_launches(1);
    copy_out_kernel<<<grid_for(rows * cols, 256), 256, 0, s>>>(src, rows, cols, ld_src, dst, ld_dst);
    return cudaGetLastError();
}

cudaError_t launch_loop_ctl(const FitState *st, int n_iter, cudaGraphConditionalHandle h, cudaStream_t s) {
    count_launches(1);
    loop_ctl_kernel<<<1, 1, 0, s>>>(st, n_iter, h);
    return cudaGetLastError();
}

cudaError_t launch_clear_stop(FitState *st, int extra_iters, cudaStream_t s) {
    count_launches(1);
    clear_stop_kernel<<<1, 1, 0, s>>>(st, extra_iters);
    return cudaGetLastError();
}

cudaError_t launch_stage_begin(FitState *st, cudaStream_t s) {
    count_launches(1);
    stage_begin_kernel<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

// Opt a kernel into more than 48 KB of dynamic shared memory, once per
// kernel and device (the attribute is per device context).
static cudaError_t set_smem_once(const void *kern, size_t smem) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, kern})) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done.insert({dev, kern});
    return e;
}

static int kp_of(int k) { return k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : k <= 64 ? 64 : 128; }

template <int KS, int SL, bool C2>
static cudaError_t hpass_launch(const PassArgs &a, cudaStream_t s) {
    constexpr int PX = HP_THREADS / SL;
    const size_t smem = sizeof(float) * hp_smem_floats<KS, SL>();
    auto kern = hpass_f32_kernel<KS, SL, C2>;
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)((a.Pp + PX - 1) / PX);
    count_launches(1);
    kern<<<grid, HP_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

int hpass_f32_blocks(const PassArgs &a) {
    const int kp = kp_of(a.k);
    const int sl = kp < 32 ? 1 : (kp == 32 ? NMF_HP_SL32 : kp / 32);
    const int px = HP_THREADS / sl;
    return (int)((a.Pp + px - 1) / px);
}

cudaError_t launch_hpass_f32(const PassArgs &a, bool chi2_only, cudaStream_t s) {
    constexpr int KS32 = 32 / NMF_HP_SL32;
    switch (kp_of(a.k)) {
        case 8: return chi2_only ? hpass_launch<8, 1, true>(a, s) : hpass_launch<8, 1, false>(a, s);
        case 16: return chi2_only ? hpass_launch<16, 1, true>(a, s) : hpass_launch<16, 1, false>(a, s);
        case 32:
            return chi2_only ? hpass_launch<KS32, NMF_HP_SL32, true>(a, s)
                             : hpass_launch<KS32, NMF_HP_SL32, false>(a, s);
        case 64: return chi2_only ? hpass_launch<32, 2, true>(a, s) : hpass_launch<32, 2, false>(a, s);
        default: return chi2_only ? hpass_launch<32, 4, true>(a, s) : hpass_launch<32, 4, false>(a, s);
    }
}

int wpass_row_tiles(int k, long long rows) {
    const int kp = kp_of(k);
    const int sl = kp <= 32 ? 1 : kp / 32;
    const int rt = 32 / sl;
    return (int)((rows + rt - 1) / rt);
}

int wpass_chunk_pixels() { return 128; }

template <int KS, int SL, int MODE>
static cudaError_t wpass_launch(const PassArgs &a, cudaStream_t s) {
    const size_t smem = sizeof(float) * wp_smem_floats<KS, SL>();
    auto kern = wpass_f32_kernel<KS, SL, MODE>;
    cudaError_t e = set_smem_once(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    dim3 grid(a.nsplit, wpass_row_tiles(a.k, a.rows));
    count_launches(2);
    kern<<<grid, WP_THREADS, smem, s>>>(a);
    const long long warps = a.rows * a.k;
    wreduce_kernel<MODE><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KS, int SL>
static cudaError_t wpass_mode(const PassArgs &a, int mode, cudaStream_t s) {
    switch (mode) {
        case WP_FIT: return wpass_launch<KS, SL, WP_FIT>(a, s);
        case WP_PROJ_FIRST: return wpass_launch<KS, SL, WP_PROJ_FIRST>(a, s);
        default: return wpass_launch<KS, SL, WP_PROJ_NEXT>(a, s);
    }
}

cudaError_t launch_wpass_f32(const PassArgs &a, int mode, cudaStream_t s) {
    switch (kp_of(a.k)) {
        case 8: return wpass_mode<8, 1>(a, mode, s);
        case 16: return wpass_mode<16, 1>(a, mode, s);
        case 32: return wpass_mode<32, 1>(a, mode, s);
        case 64: return wpass_mode<32, 2>(a, mode, s);
        default: return wpass_mode<32, 4>(a, mode, s);
    }
}

cudaError_t launch_stage_end(const PassArgs &a, int normalize, double *chi2_hist, int32_t *iters_done, int kidx,
                             cudaStream_t s) {
    count_launches(2);
    norm_partial_kernel<<<dim3(a.k, NORM_SLICES), 256, 0, s>>>(a);
    stage_end_kernel<<<dim3((unsigned)((a.Pp + 255) / 256 + 1), a.k), 256, 0, s>>>(a, normalize, chi2_hist,
                                                                                 iters_done, kidx);
    return cudaGetLastError();
}

cudaError_t launch_subtract(const float *T, const float *C, const float *H, long long M, int K, long long P,
                            const float *factor, float *R, const int32_t *scatter_idx, long long img_pixels,
                            float *img, cudaStream_t s) {
    if (M == 0 || P == 0) return cudaSuccess;
    if (img) {
        cudaError_t e = cudaMemsetAsync(img, 0, sizeof(float) * (size_t)M * (size_t)img_pixels, s);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)((P + 255) / 256), (unsigned)M);
    count_launches(1);
    subtract_kernel<<<grid, 256, 0, s>>>(T, C, H, M, K, P, factor, R, scatter_idx, img, img_pixels);
    return cudaGetLastError();
}

}  // namespace nmfgb
