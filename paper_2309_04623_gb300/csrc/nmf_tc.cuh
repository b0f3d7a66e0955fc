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
constexpr int kMaxWBlocks = 256;      // blocks of an explicitly scheduled W pass
constexpr int kMaxWRowTiles = 16;     // row tiles of an explicitly scheduled W pass

struct TcArgs {
    float *W;                // FP32 coefficients (rows x ldw), updated by the W pass
    float *part;             // W-pass partials: split x rows x (den[KP], G[KP])
    double *chi2_part;       // one FP64 partial per H-pass block
    FitState *st;
    // operand images of the coefficients (W or C): read as the streamed
    // operand of the H pass and the tile operand of the W pass, rewritten
    // by the W update
    uint8_t *wk_h, *wk_l;
    // operand images of the basis H, two sets (hi, lo) used in turn: the H
    // pass of iteration t reads set t & 1 and writes set (t + 1) & 1, which
    // the W pass of the same iteration streams.  A projection points both
    // sets at the one fixed basis.  The images are the iterate of H inside
    // the tensor-core loop (hi + lo, 16 significant bits).
    uint8_t *hk_h[2], *hk_l[2];
    // third parts of the basis images (BF16 of H - hi - lo), two sets like
    // the others: hi + lo + lo2 carries H at single precision through the
    // tensor-core loop (the MMAs read only hi and lo); NULL in a projection
    uint8_t *hk_l2[2];
    long long rows;          // N (fit) or M (projection)
    long long Pp;            // padded pixels (multiple of 128)
    int k, ldw;
    // W-pass pixel splits: every full 128-row tile in nsplit splits of
    // split_len pixels, the last (partial) row tile in nsplit_last splits of
    // split_len_last, so that every block streams about the same bytes
    int nsplit, split_len, nsplit_last, split_len_last;
    // W pass overlapping the H pass: an explicit schedule of w_nblk blocks
    // (0: the splits above).  Block b streams chunks [w_c0[b], w_c1[b]) of
    // 64 pixels of row tile w_tile[b] into partial slot w_split[b]; the
    // blocks that start while the H pass finishes its last tiles take longer
    // ranges of pixels already written, the ones that start when it ends
    // shorter ones.  Row tile t has w_nsplit[t] slots.
    int w_nblk;
    uint16_t w_c0[kMaxWBlocks], w_c1[kMaxWBlocks];
    uint8_t w_tile[kMaxWBlocks], w_split[kMaxWBlocks];
    uint8_t w_nsplit[kMaxWRowTiles];
    int kp;                  // padded components of the kernels: 64 (k <= 64) or 128
    int packed;              // images packed (k <= 32): hi in columns 0..31, lo in 32..63 of one block
    int wt32;                // weights streamed as FP32 (the single-precision-weights form) instead of scaled FP16
    // iteration count of the loop (0: none): passes of an iteration t >= t_end
    // do nothing, so a recorded loop body may hold several iterations
    int t_end;
    int h_blocks;            // fit: blocks of the H pass, whose Eq. 2 shares the W pass records
    // fit, single reduction: per 128-pixel tile, 4 x the H passes of this
    // stage that have written the tile's new H images (one count per tile
    // warp; cleared at each stage start).  The W pass is then launched as a
    // programmatic dependent of the H pass and each of its chunks waits only
    // for the tile it reads (NULL: plain launch order)
    unsigned *h_flags;
    float eps;
    double tol;
    // failure-handling test aid (nmf_debug_plant_timeout): at iteration
    // fault_t of a fit loop (< 0: never), block 0 of the W pass waits for an
    // H tile count that is never reached, bounded by fault_ns
    int fault_t;
    unsigned long long fault_ns;
};

struct TcMaps {
    CUtensorMap hV, hWt;  // H pass: boxes {128 px, NC rows}, no swizzle
    CUtensorMap wV, wWt;  // W pass: boxes {32 px, 128 rows} (128-byte swizzle), {NC px, 128 rows}
};

int tc_max_k();                       // largest K of the form
int tc_kp(int k);                     // padded components for rank k (64 or 128)
bool tc_packed(int k);                // rank k uses packed images (hi and lo in one 64-component block)
constexpr int kMaxWSplits = 128;      // most pixel splits of a W pass (the partials' workspace holds this many)
int tc_split_granule();               // W-pass split lengths are multiples of this
int tc_num_sms();                     // streaming multiprocessors of the current device
int tc_hpass_blocks(long long Pp);    // blocks of an H pass over Pp pixels
int tc_tile();
size_t tc_image_bytes(long long rows, int k);  // one operand image (hi or lo) of `rows` rows at rank <= k
// The FP16-weights form's weight copy: FP16 of the weights times a power of
// two chosen from their maximum (recorded in st), padded to ld_dst.
cudaError_t tc_weights_bf16(const float *src, long long rows, long long cols, void *dst, long long ld_dst,
                            FitState *st, cudaStream_t s);
cudaError_t tc_images(const float *X, long long rows, int k, long long ld, bool x_is_kxP, uint8_t *Kh, uint8_t *Kl,
                      int kp, bool packed, cudaStream_t s, uint8_t *Kl2 = nullptr);
// FP32 H (K x Pp, buffer st->t & 1 of Hb0 / Hb1) from the image set st->t & 1
// (hi + lo + lo2): the current iterate after a tensor-core loop.
cudaError_t tc_h_from_images(const TcArgs &a, float *Hb0, float *Hb1, cudaStream_t s);
bool tc_make_maps(TcMaps *m, const float *V, const void *Wtb, long long rows, long long Pp, int kp, bool wt32);
cudaError_t tc_hpass(const TcMaps &m, const TcArgs &a, bool chi2_only, cudaStream_t s);
cudaError_t tc_wpass(const TcMaps &m, const TcArgs &a, cudaStream_t s);

}  // namespace nmfgb
