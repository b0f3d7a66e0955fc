// Reference selection (arXiv:2309.04623, Sec. 4.1): the library frames
// closest to each target frame by the Euclidean norm of the difference,
// weighted as in the NMF cost (Eq. 2),
//     D[m, n] = sum_p WtT[m, p] (T[m, p] - V[n, p])^2,
// and the n_keep closest frames of every target, closest first, equal
// distances in library order.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <set>
#include <utility>

#include "nmf_internal.cuh"

namespace nmfgb {
namespace {

namespace cg = cooperative_groups;

constexpr int SEL_THREADS = 256;
constexpr int SEL_MB = 4;      // targets per block
constexpr int SEL_NB = 8;      // library frames per block
constexpr int SEL_SPLIT = 8;   // CTAs of a cluster, each over 1/8 of the pixels
constexpr int SEL_MAX_N = 8192;

// Cluster (n tile, m tile) of SEL_SPLIT CTAs along z; CTA z sums the pixels
// of the z-th eighth of the frame.  Every thread sums its pixels (stride 256)
// in FP32 for the 4 x 8 (target, frame) pairs; the pairs are then summed over
// the CTA in a fixed order, and CTA 0 of the cluster adds the eight CTAs' sums
// in FP64 in rank order, reading them from their shared memory (DSMEM).
// Offsets inside a tile are 32-bit: 8 rows x P < 2^31.
__global__ void __cluster_dims__(1, 1, SEL_SPLIT) __launch_bounds__(SEL_THREADS, 2)
    distances_kernel(const float *__restrict__ T, const float *__restrict__ WtT, const float *__restrict__ V,
                     long long M, long long N, int P, double *__restrict__ D) {
    static_assert(SEL_MB * SEL_NB * 8 == SEL_THREADS, "8 threads per pair in the CTA sum");
    // row pitch 264 = 256 + 8: the transposed writes (a row, consecutive
    // threads) and the strided reads (thread (pair, seg) reads seg, seg + 8,
    // ...) both fall in 32 distinct banks
    __shared__ float red[SEL_MB * SEL_NB][SEL_THREADS + 8];
    __shared__ double part[SEL_MB * SEL_NB];
    cg::cluster_group cluster = cg::this_cluster();
    const long long m0 = (long long)blockIdx.y * SEL_MB, n0 = (long long)blockIdx.x * SEL_NB;
    const int mc = M - m0 < SEL_MB ? (int)(M - m0) : SEL_MB;
    const int nc = N - n0 < SEL_NB ? (int)(N - n0) : SEL_NB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunk = (P + SEL_SPLIT - 1) / SEL_SPLIT;
    const int pb = (int)cluster.block_rank() * chunk;
    const int pe = P - pb < chunk ? P : pb + chunk;
    const float *Tb = T + m0 * P, *Wb = WtT + m0 * P, *Vb = V + n0 * P;
    float acc[SEL_MB][SEL_NB];
#pragma unroll
    for (int i = 0; i < SEL_MB; ++i)
#pragma unroll
        for (int j = 0; j < SEL_NB; ++j) acc[i][j] = 0.0f;
    // Two pixels per pass (p and p + 256): all their loads are issued before
    // the arithmetic that consumes them.
    for (int p = pb + tid; p < pe; p += 2 * SEL_THREADS) {
        const bool two = p + SEL_THREADS < pe;
        const int p2 = two ? p + SEL_THREADS : p;
        float v[2][SEL_NB], t[2][SEL_MB], w[2][SEL_MB];
#pragma unroll
        for (int j = 0; j < SEL_NB; ++j) {  // rows past the end repeat the last (never stored)
            const int o = (j < nc ? j : nc - 1) * P;
            v[0][j] = __ldg(Vb + o + p);
            v[1][j] = __ldg(Vb + o + p2);
        }
#pragma unroll
        for (int i = 0; i < SEL_MB; ++i) {
            const int o = (i < mc ? i : mc - 1) * P;
            t[0][i] = __ldg(Tb + o + p);
            w[0][i] = __ldg(Wb + o + p);
            t[1][i] = __ldg(Tb + o + p2);
            w[1][i] = two ? __ldg(Wb + o + p2) : 0.0f;  // a repeated pixel adds nothing
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int i = 0; i < SEL_MB; ++i)
#pragma unroll
                for (int j = 0; j < SEL_NB; ++j) {
                    const float d = t[h][i] - v[h][j];
                    acc[i][j] = fmaf(w[h][i] * d, d, acc[i][j]);
                }
    }
    // CTA sum of every pair: the 256 partials of a pair are transposed
    // through shared memory, 8 threads add 32 each (every 8th), then a fixed xor-shuffle
    // tree over those 8 (FP32: GB300's FP64 rate is a small fraction of its
    // FP32 rate, and the per-thread partials are FP32 already).
#pragma unroll
    for (int i = 0; i < SEL_MB; ++i)
#pragma unroll
        for (int j = 0; j < SEL_NB; ++j) red[i * SEL_NB + j][tid] = acc[i][j];
    __syncthreads();
    {
        const int pair = tid >> 3, seg = tid & 7;  // 32 pairs x 8 interleaved sets of 32 partials
        const float *row = red[pair] + seg;
        float s = 0.0f;
#pragma unroll 8
        for (int q = 0; q < 32; ++q) s += row[q * 8];
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (seg == 0) part[pair] = (double)s;
    }
    cluster.sync();  // every CTA's part[] is complete
    if (cluster.block_rank() == 0 && tid < SEL_MB * SEL_NB) {
        const int i = tid / SEL_NB, j = tid % SEL_NB;
        double s = 0.0;
        for (int r = 0; r < SEL_SPLIT; ++r) s += cluster.map_shared_rank(part, r)[tid];
        if (i < mc && j < nc) D[(m0 + i) * N + n0 + j] = s;
    }
    cluster.sync();  // no CTA leaves while CTA 0 may still read its shared memory
}

// One block per target: the rank of frame n is the number of frames closer
// to the target, or as close and earlier in the library; ranks below n_keep
// are written out.  Distances are sums of non-negative terms (never -0, NaN
// or negative), so their IEEE bit patterns read as int64 order exactly as the
// values do: the comparisons run on the integer pipes (GB300's FP64 pipe is
// narrow).
__global__ void __launch_bounds__(SEL_THREADS) select_kernel(const double *D, long long N, int n_keep, int32_t *idx) {
    extern __shared__ long long key[];
    const long long m = blockIdx.x;
    for (long long n = threadIdx.x; n < N; n += SEL_THREADS) key[n] = __double_as_longlong(D[m * N + n]);
    __syncthreads();
    for (long long n = threadIdx.x; n < N; n += SEL_THREADS) {
        const long long d = key[n];
        int rank = 0;
        for (int q = 0; q < (int)N; ++q) {
            const long long e = key[q];
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
                             (int)(sizeof(long long) * SEL_MAX_N));
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
    if (M < 1 || N < 1 || P < 1 || P >= (1LL << 28) || M > 65535LL * SEL_MB || N > SEL_MAX_N) return NMF_EINVAL;
    if (n_keep < 1 || n_keep > N) return NMF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 grid((unsigned)((N + SEL_NB - 1) / SEL_NB), (unsigned)((M + SEL_MB - 1) / SEL_MB), SEL_SPLIT);
    count_launches(2);
    distances_kernel<<<grid, SEL_THREADS, 0, s>>>(T, WtT, V, M, N, (int)P, dist);
    if (cudaGetLastError() != cudaSuccess) return NMF_ECUDA;
    const size_t smem = sizeof(long long) * (size_t)N;
    if (select_smem() != cudaSuccess) return NMF_ECUDA;
    select_kernel<<<(unsigned)M, SEL_THREADS, smem, s>>>(dist, N, n_keep, idx);
    return cudaGetLastError() == cudaSuccess ? NMF_OK : NMF_ECUDA;
}

}  // extern "C"
