// North-up rotation and stacking of the subtracted frames (arXiv:2309.04623,
// Sec. 4.1 and 4.2: every PSF-subtracted frame is rotated by its position
// angle, then the rotated frames are combined to raise the signal-to-noise
// ratio and the sky coverage).
//
// Frame f's content is rotated by angle_f about (cx, cy), x = column,
// y = row:
//     out_f(x, y) = in_f(xs, ys),  xs = cx + (c (x - cx) + s (y - cy)),
//                                  ys = cy + (c (y - cy) - s (x - cx)),
// with c, s the cosine and sine of the angle rounded to float, and in_f
// between pixel centres by bilinear interpolation of its four neighbours.
// A neighbour of zero weight is not used; a used neighbour outside the
// frame, NaN, or flagged invalid makes the output missing (NaN).  The
// stacked image is, per pixel, the mean or the median of the frames that
// cover it.
//
// One kernel does both steps.  A block owns an 8 x 4 patch of the output;
// its 32 x G threads split the frames (thread (i, g) takes frames
// g, g + G, ...), gather the (at most four) source pixels of each from L1/L2,
// optionally write the rotated value, and stage it in shared memory; after
// one barrier the block combines each pixel's F values: the mean by thread
// (i, 0) in frame order, the median by ranking the values over all G groups.
// The rotated frames need not round-trip through HBM, and G independent
// frame walks per pixel keep enough loads in flight to stream the frames.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>
#include <set>

#include "nmf_internal.cuh"

namespace nmfgb {
namespace {

constexpr int ROT_MAX_F = 1024;
constexpr int ROT_MAX_SIDE = 16384;  // coordinates stay exact in float
// |centre| <= 2^20 keeps every source coordinate within +-2^22 (floor_exact)
constexpr float ROT_MAX_CENTRE = 1048576.0f;
constexpr int ROT_TX = 32;           // output pixels per block: an 8 x 4 patch
constexpr int ROT_PW = 8, ROT_PH = 4; // patch width and height
static_assert(ROT_PW * ROT_PH == ROT_TX, "one warp covers the patch");
constexpr int ROT_G = 8;             // frame groups per block
constexpr double ROT_PI = 3.14159265358979323846;

// Cosine and sine of every frame's angle, passed by value (8 KB of kernel
// parameters; no device buffer, so the launch captures into a graph as is).
struct RotTrig {
    float c[ROT_MAX_F];
    float s[ROT_MAX_F];
};

enum { MODE_ROTATE = 0, MODE_MEAN = 1, MODE_MEDIAN = 2 };

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }

// floor(v) for |v| < 2^22 without a conversion instruction (conversions run
// on GB300's narrow FP64/conversion pipe): v + 1.5 * 2^23 rounded down is
// floor(v) + 1.5 * 2^23 exactly, and in [2^23, 2^24) consecutive floats are
// consecutive integers with consecutive bit patterns.  vf = floor(v) as float.
constexpr float kFloorBias = 12582912.0f;

__device__ __forceinline__ int floor_exact(float v, float &vf) {
    const float t = __fadd_rd(v, kFloorBias);
    vf = __fsub_rn(t, kFloorBias);
    return __float_as_int(t) - __float_as_int(kFloorBias);
}

// Bilinear value of frame `src` at the rotated position of pixel (x, y)
// (dx = x - cx, dy = y - cy), or NaN if a used neighbour is missing.
__device__ __forceinline__ float rotated_value(const float *__restrict__ src, const uint8_t *__restrict__ valid,
                                               int nx, int ny, float c, float s, float cx, float cy, float dx,
                                               float dy) {
    // Source position: float, rounded after every operation (no contraction),
    // so that the choice of neighbours is reproducible by any float code.
    const float xs = __fadd_rn(cx, __fadd_rn(__fmul_rn(c, dx), __fmul_rn(s, dy)));
    const float ys = __fadd_rn(cy, __fsub_rn(__fmul_rn(c, dy), __fmul_rn(s, dx)));
    float x0f, y0f;
    const int x0 = floor_exact(xs, x0f), y0 = floor_exact(ys, y0f);
    const float fx = __fsub_rn(xs, x0f), fy = __fsub_rn(ys, y0f);
    const int ux = fx > 0.0f, uy = fy > 0.0f;
    if (x0 < 0 || y0 < 0 || x0 + ux > nx - 1 || y0 + uy > ny - 1) return qnan();
    const int q = y0 * nx + x0;  // < ny * nx <= 2^28
    const float v00 = __ldg(src + q);
    const float v10 = ux ? __ldg(src + q + 1) : 0.0f;
    const float v01 = uy ? __ldg(src + q + nx) : 0.0f;
    const float v11 = (ux & uy) ? __ldg(src + q + nx + 1) : 0.0f;
    bool ok = !isnan(v00) && !isnan(v10) && !isnan(v01) && !isnan(v11);
    if (valid) {
        ok = ok && __ldg(valid + q) != 0;
        if (ux) ok = ok && __ldg(valid + q + 1) != 0;
        if (uy) ok = ok && __ldg(valid + q + nx) != 0;
        if (ux & uy) ok = ok && __ldg(valid + q + nx + 1) != 0;
    }
    if (!ok) return qnan();
    const float wx0 = 1.0f - fx, wy0 = 1.0f - fy;
    return wy0 * (wx0 * v00 + fx * v10) + fy * (wx0 * v01 + fx * v11);
}

// Block = one 8 x 4 output patch, threads (32, G): thread i owns pixel
// (i % 8, i / 8) of the patch, warp g the frames g, g + G, ...  A warp's
// gathers then come from a compact rotated patch (a few cache lines per
// load) rather than from a rotated 32-pixel line.
template <int MODE>
__global__ void __launch_bounds__(ROT_TX * ROT_G, 4) rotate_kernel(const float *__restrict__ img, int F, int ny,
                                                                   int nx, const uint8_t *__restrict__ valid,
                                                                   const RotTrig trig, float cx, float cy,
                                                                   float *__restrict__ rot, float *__restrict__ out,
                                                                   int32_t *__restrict__ count) {
    extern __shared__ float vals[];  // F x 32: frame f's value of the block's pixel i at vals[f * 32 + i]
    __shared__ float sel[2][ROT_TX];  // MODE_MEDIAN: the two middle values of every pixel
    const int i = threadIdx.x, g = threadIdx.y, G = blockDim.y;
    const int x = blockIdx.x * ROT_PW + (i & (ROT_PW - 1));
    const int y = blockIdx.y * ROT_PH + i / ROT_PW;
    const bool live = x < nx && y < ny;
    const long long npix = (long long)ny * nx;
    const long long p = (long long)y * nx + x;
    if (live) {
        const float dx = __fsub_rn((float)x, cx), dy = __fsub_rn((float)y, cy);
#pragma unroll 4
        for (int f = g; f < F; f += G) {
            const float val = rotated_value(img + (long long)f * npix, valid, nx, ny, trig.c[f], trig.s[f], cx, cy,
                                            dx, dy);
            if (rot) rot[(long long)f * npix + p] = val;
            if (MODE != MODE_ROTATE || count) vals[f * ROT_TX + i] = val;
        }
    }
    if (MODE == MODE_ROTATE && !count) return;  // uniform over the block
    __syncthreads();
    // frames covering this pixel (every group counts; the loop is the same for all)
    int n = 0;
    if (live)
        for (int f = 0; f < F; ++f) n += isnan(vals[f * ROT_TX + i]) ? 0 : 1;
    if (MODE == MODE_MEDIAN) {
        // Rank of each present value among the present values (ties broken
        // by frame index, so ranks are distinct): the values of rank
        // (n - 1) / 2 and n / 2 are the middle ones.  Group g ranks frames
        // g, g + G, ...; every rank is unique, so each slot has one writer.
        if (live && n) {
            const int k1 = (n - 1) / 2, k2 = n / 2;
            for (int f = g; f < F; f += G) {
                const float v = vals[f * ROT_TX + i];
                if (isnan(v)) continue;
                int r = 0;
                for (int j = 0; j < F; ++j) {
                    const float u = vals[j * ROT_TX + i];  // NaN compares false: not counted
                    r += (u < v || (u == v && j < f)) ? 1 : 0;
                }
                if (r == k1) sel[0][i] = v;
                if (r == k2) sel[1][i] = v;
            }
        }
        __syncthreads();
    }
    if (g != 0 || !live) return;
    if (MODE == MODE_MEAN) {
        float sum = 0.0f, comp = 0.0f;  // Neumaier-compensated sum in frame order
        for (int f = 0; f < F; ++f) {
            const float v = vals[f * ROT_TX + i];
            if (isnan(v)) continue;
            const float t = sum + v;
            comp += fabsf(sum) >= fabsf(v) ? (sum - t) + v : (v - t) + sum;
            sum = t;
        }
        out[p] = n ? (sum + comp) / (float)n : qnan();
    } else if (MODE == MODE_MEDIAN) {
        out[p] = n ? 0.5f * sel[0][i] + 0.5f * sel[1][i] : qnan();
    }
    if (count) count[p] = n;
}

template <int MODE>
cudaError_t smem_opt_in() {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(dev)) return cudaSuccess;
    e = cudaFuncSetAttribute(rotate_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float) * ROT_TX * ROT_MAX_F));
    if (e == cudaSuccess) done.insert(dev);
    return e;
}

template <int MODE>
cudaError_t launch_rotate(const float *img, int F, int ny, int nx, const uint8_t *valid, const RotTrig &trig,
                          float cx, float cy, float *rot, float *out, int32_t *count, cudaStream_t s) {
    cudaError_t e = smem_opt_in<MODE>();
    if (e != cudaSuccess) return e;
    const dim3 block(ROT_TX, F < ROT_G ? F : ROT_G);
    const dim3 grid((unsigned)((nx + ROT_PW - 1) / ROT_PW), (unsigned)((ny + ROT_PH - 1) / ROT_PH));
    const size_t smem = (MODE == MODE_ROTATE && !count) ? 0 : sizeof(float) * ROT_TX * (size_t)F;
    rotate_kernel<MODE><<<grid, block, smem, s>>>(img, F, ny, nx, valid, trig, cx, cy, rot, out, count);
    return cudaGetLastError();
}

}  // namespace
}  // namespace nmfgb

using namespace nmfgb;

extern "C" {

nmf_status nmf_derotate_combine(const float *img, int64_t F, int32_t ny, int32_t nx, const uint8_t *valid,
                                const double *angle_deg, float cx, float cy, int32_t method, float *rot,
                                float *out, int32_t *count, void *stream) {
    if (!img || !angle_deg || (!rot && !out && !count)) return NMF_EINVAL;
    if (F < 1 || F > ROT_MAX_F || ny < 1 || nx < 1 || ny > ROT_MAX_SIDE || nx > ROT_MAX_SIDE) return NMF_EINVAL;
    if (method != NMF_COMBINE_MEAN && method != NMF_COMBINE_MEDIAN) return NMF_EINVAL;
    if (!(fabsf(cx) <= ROT_MAX_CENTRE) || !(fabsf(cy) <= ROT_MAX_CENTRE)) return NMF_EINVAL;  // also NaN
    RotTrig trig = {};
    for (int64_t f = 0; f < F; ++f) {
        if (!isfinite(angle_deg[f])) return NMF_EINVAL;
        const double th = angle_deg[f] * (ROT_PI / 180.0);
        trig.c[f] = (float)cos(th);
        trig.s[f] = (float)sin(th);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    count_launches(1);
    cudaError_t e;
    if (!out)
        e = launch_rotate<MODE_ROTATE>(img, (int)F, ny, nx, valid, trig, cx, cy, rot, out, count, s);
    else if (method == NMF_COMBINE_MEAN)
        e = launch_rotate<MODE_MEAN>(img, (int)F, ny, nx, valid, trig, cx, cy, rot, out, count, s);
    else
        e = launch_rotate<MODE_MEDIAN>(img, (int)F, ny, nx, valid, trig, cx, cy, rot, out, count, s);
    return e == cudaSuccess ? NMF_OK : NMF_ECUDA;
}

}  // extern "C"
