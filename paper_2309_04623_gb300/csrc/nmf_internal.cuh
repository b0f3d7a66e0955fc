// Internal declarations shared by the CUDA translation units of libnmfgb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nmf.h"

namespace nmfgb {

// Every N x P array the kernels stream is kept in the workspace with its rows
// padded to a multiple of 128 pixels: 16-byte vector copies and TMA boxes
// need aligned row starts, and the zero padding (weight 0) contributes
// nothing to any sum.
constexpr int kPadP = 128;
inline int64_t pad_p(int64_t P) { return (P + kPadP - 1) / kPadP * kPadP; }
// Coefficient rows (W, C) are kept with a padded leading dimension too.
inline int pad_k(int k) { return (k + 31) / 32 * 32; }
constexpr int kMaxK = 128;

// Entries of W, H (and C) that a multiplicative update or the per-stage
// normalisation leaves below 2^-126, the smallest normal FP32 value, are set
// to exactly zero (and stay zero, like every zero entry).  The factors are
// stored in FP32, whose normal range ends there; flushing explicitly makes
// the cut-off an exact, reproducible rule that an FP64 computation can apply
// identically.
constexpr float kTinyFactor = 1.17549435082228750797e-38f;  // 2^-126
__host__ __device__ __forceinline__ float flush_tiny(float x) { return x < kTinyFactor ? 0.0f : x; }

// Device-resident control block of one fit or projection.  Written only by
// the library's own kernels (no host round trip inside a call).
struct FitState {
    int status;         // nmf_status of device-detected errors
    int stop;           // stopping rule fired in the current stage
    int t;              // iterations completed in the current stage
    int iters_kept;     // iteration count of the state that is kept
    int final_buf;      // which of the two H buffers holds the kept state
    unsigned ticket_h;  // last-block ticket of the H pass
    unsigned ticket_all;// last-block ticket over W row tiles
    int t_limit;        // iteration count at which a resumed (polish) loop ends
    int run;            // tensor-core W pass: this iteration runs (its update kernel reads this)
    unsigned h_done;    // tensor-core H-pass blocks that have left their share of Eq. 2 in this stage
    double chi2_prev;   // Eq. 2 after the previous iteration
    double chi2_last;   // Eq. 2 of the kept state
    unsigned wmax_bits; // tensor-core form: bit pattern of the largest weight (non-negative floats order as integers)
    float wscale_inv;   // FP16-weights form: the stored 16-bit weights times this are the weights (a power of two)
};

// Arguments of the streaming passes (fit and projection).
struct PassArgs {
    const float *V;     // rows x Pp, padded copy of the data (V, or T)
    const float *Wt;    // rows x Pp, padded weights
    float *W;           // rows x ldw coefficients (W, or C)
    float *Hb0, *Hb1;   // the two H buffers (K x Pp); equal for a projection
    float *part;        // W-pass partial sums: nsplit x rows x ldw x 2
    float *num_const;   // projection only: rows x ldw constant numerator
    double *chi2_part;  // one FP64 partial per H-pass block
    double *norm_part;  // per-stage normalisation: kMaxK x 16 partial sums of squares
    unsigned *tickets;  // one per W row tile
    FitState *st;
    long long rows;     // N (fit) or M (projection)
    long long P, Pp;
    int k;              // active components in this stage
    int ldw;            // leading dimension of W (>= pad_k(K))
    int nsplit;         // pixel splits of the W pass
    int split_len;      // pixels per split (multiple of the pass chunk)
    float eps;
    double tol;
};

// Process-wide count of kernels launched by the library (nmf_launch_count).
void count_launches(unsigned long long n);

// Records the failed CUDA call for nmf_last_cuda_error() and returns
// NMF_ECUDA (nmf_capi.cu).
nmf_status cuda_fail(cudaError_t e, const char *what);

#define NMF_CUDA_TRY(expr)                                     \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #expr);    \
    } while (0)

// Pixel splits of the FP32 W pass for `rows` rows at rank k over Pp
// pixels: about four blocks per SM, each split a multiple of the pass chunk,
// at most max_splits splits (nmf_capi.cu).
void choose_splits(long long rows, int k, long long Pp, int max_splits, int *nsplit, int *split_len);

// ---- kernel launchers (nmf_simt.cu) -------------------------------------
cudaError_t launch_prologue_copy(const float *src, long long rows, long long cols, long long ld_src,
                                 float *dst, long long ld_dst, long long dst_cols, FitState *st, int check,
                                 cudaStream_t s);
cudaError_t launch_copy_out(const float *src, long long rows, long long cols, long long ld_src, float *dst,
                            long long ld_dst, cudaStream_t s);
cudaError_t launch_stage_begin(FitState *st, cudaStream_t s);
cudaError_t launch_clear_stop(FitState *st, int extra_iters, cudaStream_t s);
cudaError_t launch_loop_ctl(const FitState *st, int n_iter, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_hpass_f32(const PassArgs &a, bool chi2_only, cudaStream_t s);
int hpass_f32_blocks(const PassArgs &a);
cudaError_t launch_wpass_f32(const PassArgs &a, int mode, cudaStream_t s);
int wpass_row_tiles(int k, long long rows);
int wpass_chunk_pixels();
cudaError_t launch_stage_end(const PassArgs &a, int normalize, double *chi2_hist, int32_t *iters_done, int kidx,
                             cudaStream_t s);
cudaError_t launch_subtract(const float *T, const float *C, const float *H, long long M, int K, long long P,
                            const float *factor, float *R, const int32_t *scatter_idx, long long img_pixels,
                            float *img, cudaStream_t s);

// W-pass modes
enum { WP_FIT = 0, WP_PROJ_FIRST = 1, WP_PROJ_NEXT = 2 };

}  // namespace nmfgb
