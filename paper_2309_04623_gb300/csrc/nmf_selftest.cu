// Measurement and failure-handling aids (no step of the paper's method).
//
// The FP32 FMA-rate kernel measures the CUDA cores' ceiling, against which
// the plain FP32 form is reported.
//
// Self-test of the bounded device waits (failure handling): the waits the
// tensor-core kernels use between their warps (mbarriers) and between the H
// and W passes (counters in global memory) give up after a time limit,
// record NMF_ETIMEOUT and return, so that a missing arrival ends a call with
// an error status instead of a hang.  This test makes each wait run out on
// purpose (a barrier nobody arrives at, a counter nobody raises) with a
// short limit; nothing faults, traps or spins without bound.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nmf_internal.cuh"
#include "tc_ptx.cuh"

namespace nmfgb {
namespace {

__device__ unsigned g_selftest_flag;  // never raised
__device__ int g_selftest_status[2];

__global__ void wait_selftest_kernel(unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    __shared__ int abort0, abort1;
    if (threadIdx.x != 0) return;
    abort0 = 0;
    abort1 = 0;
    g_selftest_status[0] = 0;
    g_selftest_status[1] = 0;
    tc::mbar_init(&bar, 1);  // expects one arrival that never comes
    tc::fence_mbar_init();
    const bool a = tc::mbar_wait(&bar, 0, &abort0, &g_selftest_status[0], NMF_ETIMEOUT, limit_ns);
    const bool b = tc::flag_wait(&g_selftest_flag, 1u, &abort1, &g_selftest_status[1], NMF_ETIMEOUT, limit_ns);
    if (a) g_selftest_status[0] = NMF_OK;  // (cannot happen) a wait that returned true records no error
    if (b) g_selftest_status[1] = NMF_OK;
}

// FP32 fused multiply-add rate of the CUDA cores: every thread runs eight
// independent FMA chains (enough to cover the pipeline latency at full
// occupancy).  The multiplier and addend are runtime values and the result
// is stored under a condition the compiler cannot decide, so no chain is
// folded or dropped.
__global__ void __launch_bounds__(512) fma_rate_kernel(float *out, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (float)threadIdx.x * 1e-3f + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    }
    float sum = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) sum += x[i];
    if (sum == -1.0f) out[blockIdx.x] = sum;
}

__device__ float g_fma_sink[4096];

}  // namespace
}  // namespace nmfgb

using namespace nmfgb;

extern "C" {

nmf_status nmf_wait_selftest(int64_t limit_ns, int32_t *status, void *stream) {
    if (!status || limit_ns < 1000 || limit_ns > 100000000) return NMF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    count_launches(1);
    wait_selftest_kernel<<<1, 32, 0, s>>>((unsigned long long)limit_ns);
    if (cudaGetLastError() != cudaSuccess) return NMF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return NMF_ECUDA;
    int h[2] = {-1, -1};
    if (cudaMemcpyFromSymbol(h, g_selftest_status, sizeof(h)) != cudaSuccess) return NMF_ECUDA;
    status[0] = h[0];
    status[1] = h[1];
    return NMF_OK;
}

nmf_status nmf_fp32_fma_rate(int32_t iters, double *tflops, void *stream) {
    if (!tflops || iters < 1 || iters > (1 << 24)) return NMF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    NMF_CUDA_TRY(cudaGetDevice(&dev));
    NMF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 4 * sms, threads = 512;
    if (blocks > 4096) return NMF_EINVAL;
    float *sink = nullptr;
    NMF_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&sink), g_fma_sink));
    cudaEvent_t e0, e1;
    NMF_CUDA_TRY(cudaEventCreate(&e0));
    NMF_CUDA_TRY(cudaEventCreate(&e1));
    count_launches(2);
    fma_rate_kernel<<<blocks, threads, 0, s>>>(sink, iters / 8 > 0 ? iters / 8 : 1, 0.9999f, 1e-4f);  // warm-up
    cudaEventRecord(e0, s);
    fma_rate_kernel<<<blocks, threads, 0, s>>>(sink, iters, 0.9999f, 1e-4f);
    cudaEventRecord(e1, s);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    NMF_CUDA_TRY(e);
    NMF_CUDA_TRY(cudaGetLastError());
    const double flops = 2.0 * 8.0 * (double)iters * (double)blocks * (double)threads;
    *tflops = ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return NMF_OK;
}

}  // extern "C"
