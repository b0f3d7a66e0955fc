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

}  // extern "C"
