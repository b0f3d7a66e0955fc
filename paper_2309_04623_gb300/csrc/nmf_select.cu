// Reference selection (arXiv:2309.04623, Sec. 4.1): the library frames
// closest to each target frame by the Euclidean norm of the difference,
// weighted as in the NMF cost (Eq. 2),
//     D[m, n] = sum_p WtT[m, p] (T[m, p] - V[n, p])^2,
// and the n_keep closest frames of every target, closest first, equal
// distances in library order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <set>
#include <utility>

#include "nmf_internal.cuh"

namespace nmfgb {
namespace {

constexpr int SEL_THREADS = 256;
constexpr int SEL_MB = 8;   // targets per block
constexpr int SEL_NB = 8;   // library frames per block
constexpr int SEL_MAX_N = 8192;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block (n tile, m tile): every thread sums its pixels (p = tid, tid + 256,
// ...) in FP32 for the 8 x 8 (target, frame) pairs, then the pairs are summed
// over the block in FP64 in a fixed order.
__global__ void __launch_bounds__(SEL_THREADS) distances_kernel(const float *T, const float *WtT, const float *V,
                                                                long long M, long long N, long long P, double *D) {
    __shared__ double red[SEL_THREADS / 32][SEL_MB * SEL_NB];
    const long long m0 = (long long)blockIdx.y * SEL_MB, n0 = (long long)blockIdx.x * SEL_NB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float acc[SEL_MB][SEL_NB];
#pragma unroll
    for (int i = 0; i < SEL_MB; ++i)
#pragma unroll
        for (int j = 0; j < SEL_NB; ++j) acc[i][j] = 0.0f;
    const float *tr[SEL_MB], *wr[SEL_MB], *vr[SEL_NB];
#pragma unroll
    for (int i = 0; i < SEL_MB; ++i) {
        const long long m = m0 + i < M ? m0 + i : M - 1;  // rows past the end repeat the last (not stored)
        tr[i] = T + m * P;
        wr[i] = WtT + m * P;
    }
#pragma unroll
    for (int j = 0; j < SEL_NB; ++j) vr[j] = V + (n0 + j < N ? n0 + j : N - 1) * P;
    for (long long p = tid; p < P; p += SEL_THREADS) {
        float v[SEL_NB];
#pragma unroll
        for (int j = 0; j < SEL_NB; ++j) v[j] = __ldg(vr[j] + p);
#pragma unroll
        for (int i = 0; i < SEL_MB; ++i) {
            const float t = __ldg(tr[i] + p), w = __ldg(wr[i] + p);
#pragma unroll
            for (int j = 0; j < SEL_NB; ++j) {
                const float d = t - v[j];
                acc[i][j] = fmaf(w * d, d, acc[i][j]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < SEL_MB; ++i)
#pragma unroll
        for (int j = 0; j < SEL_NB; ++j) {
            const double s = warp_sum_d((double)acc[i][j]);
            if (lane == 0) red[warp][i * SEL_NB + j] = s;
        }
    __syncthreads();
    if (tid < SEL_MB * SEL_NB) {
        const int i = tid / SEL_NB, j = tid % SEL_NB;
        if (m0 + i < M && n0 + j < N) {
            double s = 0.0;
            for (int w = 0; w < SEL_THREADS / 32; ++w) s += red[w][tid];
            D[(m0 + i) * N + n0 + j] = s;
        }
    }
}

// One block per target: the rank of frame n is the number of frames closer
// to the target, or as close and earlier in the library; ranks below n_keep
// are written out.
__global__ void __launch_bounds__(SEL_THREADS) select_kernel(const double *D, long long N, int n_keep, int32_t *idx) {
    extern __shared__ double drow[];
    const long long m = blockIdx.x;
    for (long long n = threadIdx.x; n < N; n += SEL_THREADS) drow[n] = D[m * N + n];
    __syncthreads();
    for (long long n = threadIdx.x; n < N; n += SEL_THREADS) {
        const double d = drow[n];
        long long rank = 0;
        for (long long q = 0; q < N; ++q) {
            const double e = drow[q];
            rank += (e < d || (e == d && q < n)) ? 1 : 0;
        }
        if (rank < n_keep) idx[m * n_keep + rank] = (int32_t)n;
    }
}

// Opt the selection kernel into up to SEL_MAX_N doubles of dynamic shared
// memory, once per device.
cudaError_t select_smem() {
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(dev)) return cudaSuccess;
    e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * SEL_MAX_N));
    if (e == cudaSuccess) done.insert(dev);
    return e;
}

}  // namespace
}  // namespace nmfgb

using namespace nmfgb;

extern "C" {

nmf_status nmf_select_references(const float *T, const float *WtT, int64_t M, const float *V, int64_t N, int64_t P,
                                 int32_t n_keep, double *dist, int32_t *idx, void *stream) {
    if (!T || !WtT || !V || !dist || !idx) return NMF_EINVAL;
    if (M < 1 || N < 1 || P < 1 || P >= (1LL << 31) || M >= (1LL << 31) || N > SEL_MAX_N) return NMF_EINVAL;
    if (n_keep < 1 || n_keep > N) return NMF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 grid((unsigned)((N + SEL_NB - 1) / SEL_NB), (unsigned)((M + SEL_MB - 1) / SEL_MB));
    count_launches(2);
    distances_kernel<<<grid, SEL_THREADS, 0, s>>>(T, WtT, V, M, N, P, dist);
    if (cudaGetLastError() != cudaSuccess) return NMF_ECUDA;
    const size_t smem = sizeof(double) * (size_t)N;
    if (select_smem() != cudaSuccess) return NMF_ECUDA;
    select_kernel<<<(unsigned)M, SEL_THREADS, smem, s>>>(dist, N, n_keep, idx);
    return cudaGetLastError() == cudaSuccess ? NMF_OK : NMF_ECUDA;
}

}  // extern "C"
