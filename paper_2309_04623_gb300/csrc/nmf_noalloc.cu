// nmf_project_target_noalloc: target modelling without any device allocation
// by the library or the caller.
//
// Some callers cannot hand the library a workspace: a host program whose
// device memory budget is fixed at start-up and handed out by another
// framework, a real-time loop that must not call cudaMalloc (it can block and
// synchronise the device at unpredictable moments), or code running where an
// allocation is simply not permitted.  This entry point serves them: its only
// scratch memory is a fixed-size array compiled into the library.
//
// The scratch lives in the file-scope array below.  Every GPU that loads the
// library carries it (NOALLOC_SCRATCH_BYTES) until the process exits.  In host
// code the array's name is not a device address, so the first call on each
// device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it; that first call should therefore come before any
// stream capture.  The cached address belongs to the device's primary context:
// resetting the device (cudaDeviceReset) after the first call is not
// supported.  All calls share the one array: calls whose work can overlap on
// the GPU (different streams, or different host threads on one device) race
// on it and must be serialised by the caller.
#include <string.h>

#include <mutex>

#include "nmf_internal.cuh"

namespace nmfgb {

namespace {

// Limits of the no-allocation form (checked on every call).
constexpr int kNaMaxM = 64;       // science frames per call
constexpr int kNaMaxK = 64;       // components
constexpr int kNaMaxSplits = 64;  // pixel splits of the W pass

// layout of the scratch array: control block, per-split partial sums
// (kNaMaxSplits x kNaMaxM x kNaMaxK x 2 floats), constant numerator
constexpr size_t kNaStateBytes = 256;
constexpr size_t kNaPartBytes = sizeof(float) * 2ull * kNaMaxSplits * kNaMaxM * kNaMaxK;
constexpr size_t kNaNumBytes = sizeof(float) * (size_t)kNaMaxM * kNaMaxK;
constexpr size_t NOALLOC_SCRATCH_BYTES = kNaStateBytes + kNaPartBytes + kNaNumBytes;
static_assert(sizeof(FitState) <= kNaStateBytes, "the control block fits its share of the scratch");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_na_mu;
void *g_na_ptr[64] = {};

// Device address of the scratch array on the current device (looked up once
// per device).  Returns nullptr on failure.
void *scratch_address(cudaError_t *err) {
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess || p == nullptr) return nullptr;
        g_na_ptr[dev] = p;
    }
    return g_na_ptr[dev];
}

}  // namespace
}  // namespace nmfgb

using namespace nmfgb;

extern "C" {

nmf_status nmf_project_target_noalloc(const float *H, int32_t K, int64_t P, const float *T, const float *WtT,
                                      int64_t M, float *C, int32_t iters, double eps, void *stream) {
    if (!H || !T || !WtT || !C) return NMF_EINVAL;
    if (M < 1 || M > kNaMaxM || K < 1 || K > kNaMaxK || P < 1 || P >= (1LL << 31) || (long long)K > P)
        return NMF_EINVAL;
    if (iters < 0 || !(eps > 0.0) || !(eps <= 1.0)) return NMF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    char *base = static_cast<char *>(scratch_address(&e));
    if (!base) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress(scratch)");

    // The kernels read the caller's unpadded arrays in place (row stride P)
    // and update C in place (leading dimension K).
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.V = T;
    a.Wt = WtT;
    a.W = C;
    a.Hb0 = a.Hb1 = const_cast<float *>(H);
    a.st = reinterpret_cast<FitState *>(base);
    a.part = reinterpret_cast<float *>(base + kNaStateBytes);
    a.num_const = reinterpret_cast<float *>(base + kNaStateBytes + kNaPartBytes);
    a.rows = M;
    a.P = P;
    a.Pp = P;
    a.k = K;
    a.ldw = K;
    a.eps = (float)eps;
    // pixel splits as for nmf_project_target, at most kNaMaxSplits (the
    // partial sums' share of the scratch)
    choose_splits(M, K, P, kNaMaxSplits, &a.nsplit, &a.split_len);

    // the control block keeps the previous call's contents: start it at zero
    NMF_CUDA_TRY(cudaMemsetAsync(base, 0, kNaStateBytes, s));
    NMF_CUDA_TRY(launch_stage_begin(a.st, s));
    for (int it = 0; it < iters; ++it) NMF_CUDA_TRY(launch_wpass_f32(a, it == 0 ? WP_PROJ_FIRST : WP_PROJ_NEXT, s));
    return NMF_OK;
}

}  // extern "C"
