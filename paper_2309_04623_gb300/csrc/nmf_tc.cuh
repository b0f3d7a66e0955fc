// Declarations of the tensor-core (tcgen05) passes, nmf_tc.cu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nmf_internal.cuh"

namespace nmfgb {

// Arguments of the tcgen05 passes.  Operand "images" are BF16 tiles of 64
// rows x 64 components laid out exactly as the 128-byte-swizzled K-major
// shared-memory operand (8 KB each), so a 1-D bulk copy stages them.
struct TcArgs {
    float *Hb0, *Hb1;        // FP32 H ping-pong (K x Pp); equal for a projection
    float *W;                // FP32 coefficients (rows x ldw)
    float *part;             // W-pass partials: nsplit x rows x (den[64], G[64])
    double *chi2_part;       // one FP64 partial per H-pass block
    FitState *st;
    // images read by the passes
    const uint8_t *imgAh, *imgAl;          // W pass: coefficient rows (hi, lo)
    const uint8_t *imgBh, *imgBl;          // streamed operands: H pass -> W images, W pass -> H images
    // images written
    uint8_t *outHKh, *outHKl;              // H pass: new H (hi, lo)
    uint8_t *outWKh, *outWKl;              // W update: new W (hi, lo)
    long long rows;          // N (fit) or M (projection)
    long long Pp;            // padded pixels (multiple of 128)
    int k, ldw, nsplit, split_len;
    int kp;                  // padded components of the kernels: 64 (k <= 64) or 128
    float eps;
    double tol;
};

struct TcMaps {
    CUtensorMap hV, hWt;  // H pass: boxes {128 px, NC rows}, no swizzle
    CUtensorMap wV, wWt;  // W pass: boxes {32 px, 128 rows} (128-byte swizzle), {NC px, 128 rows}
};

int tc_max_k();                       // largest K of the form
int tc_kp(int k);                     // padded components for rank k (64 or 128)
int tc_split_granule();               // W-pass split lengths are multiples of this
int tc_tile();
size_t tc_image_bytes(long long rows, int k);  // one operand image (hi or lo) of `rows` rows at rank <= k
cudaError_t tc_weights_bf16(const float *src, long long rows, long long cols, void *dst, long long ld_dst,
                            FitState *st, cudaStream_t s);
cudaError_t tc_images(const float *X, long long rows, int k, long long ld, bool x_is_kxP, uint8_t *Kh, uint8_t *Kl,
                      int kp, cudaStream_t s);
bool tc_make_maps(TcMaps *m, const float *V, const void *Wtb, long long rows, long long Pp, int kp);
cudaError_t tc_hpass(const TcMaps &m, const TcArgs &a, bool chi2_only, cudaStream_t s);
cudaError_t tc_wpass(const TcMaps &m, const TcArgs &a, cudaStream_t s);

}  // namespace nmfgb
