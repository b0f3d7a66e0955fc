/*
 * libnmfgb -- weighted non-negative matrix factorisation of a reference-PSF
 * library, target modelling and PSF subtraction on one GB300 (sm_103a).
 *
 * Method: arXiv:2309.04623 ("NMF-based GPU accelerated coronagraphy
 * pipeline").  Sec. 2, Eq. 2 (weighted Frobenius cost) and Eq. 3
 * (multiplicative updates) define the fit; Sec. 4.1 defines target modelling
 * (each science frame modelled on its own with the fitted components) and the
 * subtraction that follows it.
 *
 * Notation.  The paper factors X ~ W H with weights V; this library names the
 * data V and the weights Wt:
 *   V   N x P   reference library: N frames, P pixels kept by the mask,
 *               row-major, one frame per row, pixels contiguous
 *   Wt  N x P   weights 1/sigma^2 (0 marks missing data), same layout
 *   W   N x K   coefficients, row-major (ld = K)
 *   H   K x P   basis components, row-major (ld = P)
 *   T   M x P   science frames, WtT their weights, C M x K their coefficients
 *
 * Conventions for every entry point below.
 *   - Pointers named as device pointers must point to GPU memory of the
 *     current device, owned and allocated by the caller; the library never
 *     frees them.  Only nmf_reduce_host takes host pointers.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are asynchronous and stream-ordered unless stated otherwise.
 *   - Argument errors are returned synchronously and nothing is launched.
 *   - Errors found on the device (negative or non-finite data: NMF_EDATA; a
 *     bounded wait between the kernels' warps or passes that gave up:
 *     NMF_ETIMEOUT) are written to a status word inside the caller's
 *     workspace; read it with nmf_workspace_status() after the work has
 *     completed.  The library never aborts or traps.
 *   - Limits: 1 <= K <= 128 (both precisions), K <= min(N, P) (the
 *     number of components cannot exceed the library size, Sec. 5.2),
 *     P < 2^31, N, M < 2^31.
 */
#ifndef NMF_GB300_H
#define NMF_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NMF_API __attribute__((visibility("default")))
#else
#define NMF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NMF_OK = 0,
    NMF_EINVAL = 1,   /* bad argument (sizes, null pointers, limits, workspace too small) */
    NMF_ENOMEM = 2,   /* device allocation failed (nmf_reduce_host only) */
    NMF_ECUDA = 3,    /* a CUDA runtime call failed */
    NMF_ETIMEOUT = 4, /* device-detected: a bounded device-side wait gave up (1 s limit); the call's
                         remaining kernels return at once and the status word records it */
    NMF_ENOTCONV = 5, /* reserved */
    NMF_EDATA = 6     /* device-detected: negative or non-finite V, Wt, T, WtT, W0, H0 or C0 */
} nmf_status;

typedef enum {
    NMF_FP32 = 0,       /* plain FP32 arithmetic on CUDA cores (follows the FP64 oracle to ~1e-6) */
    NMF_TF32_SPLIT = 1, /* reserved (not implemented: returns NMF_EINVAL; the BF16 split below reaches
                           the same accuracy with half the operand bytes) */
    NMF_BF16_SPLIT = 2, /* tensor cores (tcgen05), BF16 operands split into hi + lo parts, FP32
                           accumulation: W H from the split factors (~FP32 accurate); the numerator as
                           den + G with G the contraction of the weighted residual Wt o (V - WH) (both
                           operands split) and den that of Wt o (WH) (the factor split); FP32 data;
                           weights stored as FP16 with a power-of-two scale (11 significant bits); H
                           carried as three BF16 parts (~FP32) inside the tensor-core loop.  The last
                           polish_iters iterations run in plain FP32.  Requires K <= 128. */
    NMF_BF16_SPLIT_W32 = 3 /* as NMF_BF16_SPLIT with the weights streamed in FP32 (8 instead of 6 bytes per
                              element and pass): for problems whose fit is sensitive to the weights' 11
                              significant bits, typically many components relative to the library size */
} nmf_precision;

typedef struct {
    int64_t N;               /* reference frames (rows of V) */
    int64_t P;               /* pixels per frame */
    int32_t K;               /* components to build */
    int32_t iters_per_stage; /* maximum multiplicative-update iterations per stage (>= 0) */
    int32_t k_start;         /* components already fitted in W, H (0 = start from scratch) */
    int32_t normalize;       /* 1: unit L2 norm for every H row after each stage */
    double tol;              /* stopping rule: relative decrease of Eq. 2 <= tol; 0 = run all iterations */
    double eps;              /* denominator clamp of Eq. 3 (e.g. 1e-30) */
    int32_t precision;       /* nmf_precision */
    int32_t polish_iters;    /* tensor-core forms (NMF_BF16_SPLIT, NMF_BF16_SPLIT_W32): how many of the
                                last stage's iterations (the final ones) run in plain FP32 (>= 0; the
                                total stays iters_per_stage); must be 0 for NMF_FP32 */
} nmf_fit_params;

/* Library version (major * 10000 + minor * 100 + patch). */
NMF_API int32_t nmf_version(void);

/* Human-readable name of a status code (static string, never NULL). */
NMF_API const char *nmf_status_string(nmf_status s);

/* Bytes of device workspace nmf_fit_basis needs for these parameters
 * (0 if the parameters are invalid).  The workspace must be 256-byte aligned. */
NMF_API size_t nmf_fit_workspace_bytes(const nmf_fit_params *prm);

/*
 * nmf_fit_basis -- Sec. 2, Eq. 1-3: sequential construction of the basis.
 *   For k = k_start+1 .. K: component k enters from the initial factors
 *   already in column k of W and row k of H (random initialisation, Sec. 2),
 *   then up to iters_per_stage iterations of Eq. 3 update all k components:
 *     H <- H o [W^T (Wt o V)] / max(W^T [Wt o (W H)], eps)
 *     W <- W o [(Wt o V) H^T] / max([Wt o (W H)] H^T, eps)     (new H)
 *   entries that are exactly 0 stay 0.  The stage ends early once the
 *   relative decrease of Eq. 2 between consecutive iterations is <= tol
 *   (tol > 0, from the second iteration on); the state of that iteration is
 *   kept.  With normalize, each H row is then scaled to unit L2 norm (FP64
 *   norm) and the matching W column by the inverse.
 *
 *   V, Wt      device, N x P, read-only; must be >= 0 and finite.
 *   W          device, N x K: in = initial W0 (columns > k_start unfitted),
 *              out = fitted coefficients.
 *   H          device, K x P: in = initial H0, out = fitted basis.
 *   chi2_hist  device, K doubles: entry k-1 = Eq. 2 at the kept state of
 *              stage k (before the rescale); entries < k_start untouched.
 *   iters_done device, K int32: iterations kept in stage k.
 *   ws         device workspace of nmf_fit_workspace_bytes(prm) bytes,
 *              256-byte aligned, owned by the caller; it must not be shared
 *              with work that may run concurrently.
 * Returns NMF_OK once all work is enqueued on `stream`.
 */
NMF_API nmf_status nmf_fit_basis(const float *V, const float *Wt, float *W, float *H, double *chi2_hist,
                         int32_t *iters_done, void *ws, size_t ws_bytes, const nmf_fit_params *prm,
                         void *stream);

/* Bytes of device workspace nmf_project_target needs (0 if invalid). */
NMF_API size_t nmf_project_workspace_bytes(int64_t M, int64_t P, int32_t K, int32_t precision);

/*
 * nmf_project_target -- Sec. 4.1, target modelling: each science frame is
 * modelled on the fixed basis H by Eq. 3's coefficient rule with H held fixed:
 *     C <- C o [(WtT o T) H^T] / max([WtT o (C H)] H^T, eps),   `iters` times.
 *   H        device, K x P, read-only (the fitted basis).
 *   T, WtT   device, M x P, read-only; >= 0 and finite.
 *   C        device, M x K: in = initial C0 (> 0 entries), out = coefficients.
 *   tol      reserved, must be 0 (fixed iteration count).
 *   precision, polish_iters
 *            as for the fit: the tensor-core forms (NMF_BF16_SPLIT,
 *            NMF_BF16_SPLIT_W32) run the first
 *            iters - polish_iters iterations on tensor cores and the last
 *            polish_iters in plain FP32 (K <= 128); NMF_FP32 requires
 *            polish_iters == 0.
 *   ws       device workspace of nmf_project_workspace_bytes() bytes.
 */
NMF_API nmf_status nmf_project_target(const float *H, int32_t K, int64_t P, const float *T, const float *WtT,
                              int64_t M, float *C, int32_t iters, double tol, double eps, int32_t precision,
                              int32_t polish_iters, void *ws, size_t ws_bytes, void *stream);

/*
 * nmf_project_target_noalloc -- the FP32 target modelling of
 * nmf_project_target (same update, same result within FP32 rounding) for
 * callers that cannot allocate device memory: no workspace argument, and
 * neither the library nor the caller allocates anything.  It exists for
 * programs whose device memory is fixed at start-up or owned by another
 * framework, and for loops that must never reach cudaMalloc; the paper has
 * no counterpart to it.
 *   Scratch: a fixed array of 2,113,792 bytes (about 2.1 MB) compiled into
 *   the library, present on every GPU that loads it until the process exits.
 *   The first call on a device looks up its address (once per device); make
 *   that first call before any stream capture.  The address is cached for
 *   the device's primary context: a device reset after the first call is not
 *   supported.  All calls share the array and each call clears the part that
 *   must start at zero, so calls that can overlap on the GPU (other streams
 *   or host threads on the same device) race and must be serialised by the
 *   caller.
 *   Limits: 1 <= M <= 64, 1 <= K <= 64, K <= P; otherwise NMF_EINVAL.
 *   H (K x P), T, WtT (M x P): device, read-only, used in place (no padding
 *   needed); C (M x K): device, in = C0, out = coefficients, updated in place.
 *   iters >= 0, 0 < eps <= 1.  No device-side validation of the data: T, WtT
 *   and H must be finite and >= 0.
 */
NMF_API nmf_status nmf_project_target_noalloc(const float *H, int32_t K, int64_t P, const float *T,
                                              const float *WtT, int64_t M, float *C, int32_t iters, double eps,
                                              void *stream);

/*
 * nmf_subtract -- Sec. 4.1, PSF subtraction:  R[m,p] = T[m,p] - f_m (C H)[m,p].
 *   T        device, M x P;  C device, M x K;  H device, K x P.
 *   factor   device, M floats, or NULL for f_m = 1 (the best-factor search of
 *            Ren et al. 2018 that the paper applies here is not defined in the
 *            paper; the caller supplies f).
 *   R        device, M x P output.
 *   scatter_idx, img_pixels, img
 *            optional: if scatter_idx (device, P int32 flat image indices,
 *            each in [0, img_pixels)) and img (device, M x img_pixels) are both
 *            non-NULL, img[m, scatter_idx[p]] = R[m,p] and every other image
 *            pixel (masked, missing data) is set to 0.
 */
NMF_API nmf_status nmf_subtract(const float *T, const float *C, const float *H, int64_t M, int32_t K, int64_t P,
                        const float *factor, float *R, const int32_t *scatter_idx, int64_t img_pixels,
                        float *img, void *stream);

/*
 * One independent reduction of a batch: the fit of a reference library and,
 * optionally, the modelling and subtraction of its science frames.
 * All pointers are device pointers owned by the caller (the array of
 * descriptors itself lives in host memory).
 */
typedef struct {
    const float *V, *Wt;  /* N x P reference library and weights */
    float *W, *H;         /* in: W0 (N x K), H0 (K x P); out: fitted factors */
    double *chi2_hist;    /* K: Eq. 2 at the kept state of every stage */
    int32_t *iters_done;  /* K: iterations kept in every stage */
    nmf_fit_params prm;   /* sizes and options of this reduction */
    const float *T, *WtT; /* M x P science frames and weights (NULL if M == 0) */
    float *C;             /* M x K: in C0, out coefficients */
    float *R;             /* M x P residual images T - C H */
    int64_t M;            /* science frames (0: fit only) */
    int32_t proj_iters;   /* projection iterations (same precision and polish as the fit) */
    int32_t reserved;     /* must be 0 */
} nmf_problem;

/* Bytes of device workspace nmf_fit_batched needs (0 if any descriptor is
 * invalid).  The descriptor array is host memory. */
NMF_API size_t nmf_batched_workspace_bytes(const nmf_problem *problems, int32_t count);

/*
 * nmf_fit_batched -- many independent reductions (Sec. 2 fit, Sec. 4.1
 * modelling and subtraction per problem; e.g. several targets with their own
 * reference libraries, of uneven N, P and K) in one call.  Each problem runs
 * on its own concurrent branch; with graphs enabled the whole batch is one
 * CUDA graph launch whose per-stage iteration loops run on the device.
 * Results are identical to separate nmf_fit_basis / nmf_project_target /
 * nmf_subtract calls on each problem.
 *   problems   host array of `count` descriptors (1 <= count <= 1024).
 *   ws         device workspace of nmf_batched_workspace_bytes() bytes,
 *              256-byte aligned.
 * Returns NMF_OK once all work is enqueued on `stream`, NMF_EINVAL for an
 * invalid descriptor or workspace (nothing enqueued), NMF_ECUDA on a launch
 * failure.  Device-side errors (NMF_EDATA, NMF_ETIMEOUT) are recorded per
 * problem in its slice of the workspace: read them with nmf_batched_status.
 * The descriptors' device arrays must not overlap between problems.
 */
NMF_API nmf_status nmf_fit_batched(const nmf_problem *problems, int32_t count, void *ws, size_t ws_bytes,
                                   void *stream);

/* Synchronises `stream` and reads every problem's device status after
 * nmf_fit_batched with the same descriptors and workspace.  `status` (host,
 * `count` entries, may be NULL) receives each problem's status; the return
 * value is the first non-OK status, or NMF_OK. */
NMF_API nmf_status nmf_batched_status(const nmf_problem *problems, int32_t count, const void *ws, void *stream,
                                      int32_t *status);

/*
 * nmf_select_references -- reference selection (Sec. 4.1: the target PSFs
 * are compared with the reference library and the closest frames, by the
 * Euclidean norm that NMF minimises, are kept to build the basis).  For
 * every target frame m and library frame n
 *     dist[m, n] = sum_p WtT[m, p] (T[m, p] - V[n, p])^2
 * (the Eq. 2 cost of modelling T_m by V_n; FP32 per pixel, FP64 over the
 * partial sums in a fixed order, so the result is reproducible), and
 * idx[m, 0 .. n_keep) = the n_keep closest library frames
 * of target m, closest first, equal distances in library order.
 *   T, WtT   device, M x P, row-major, read-only: finite values, weights
 *            WtT >= 0 (with a negative weight the ranking is unspecified).
 *   V        device, N x P, row-major, read-only: the library.
 *   dist     device, M x N doubles (written).
 *   idx      device, M x n_keep int32 (written).
 *   Limits: M, N, P >= 1, M <= 262140, N <= 8192, 1 <= n_keep <= N,
 *   P < 2^28; otherwise
 *   NMF_EINVAL with nothing launched.  Asynchronous on `stream`.
 */
NMF_API nmf_status nmf_select_references(const float *T, const float *WtT, int64_t M, const float *V, int64_t N,
                                         int64_t P, int32_t n_keep, double *dist, int32_t *idx, void *stream);

/* Combination rule of nmf_derotate_combine. */
typedef enum {
    NMF_COMBINE_MEAN = 0,  /* mean of the frames covering the pixel */
    NMF_COMBINE_MEDIAN = 1 /* their median (mean of the two middle values for an even count) */
} nmf_combine_method;

/*
 * nmf_derotate_combine -- North-up rotation and stacking of the subtracted
 * frames (Sec. 4.1 and 4.2: every PSF-subtracted frame is rotated by its
 * position angle, and the rotated frames are combined for signal-to-noise
 * ratio and sky coverage).  Frame f's content is rotated by angle_deg[f]
 * about (cx, cy), x = column, y = row:
 *     rot_f(x, y) = img_f(xs, ys),  xs = cx + (c (x - cx) + s (y - cy)),
 *                                   ys = cy + (c (y - cy) - s (x - cx)),
 *     c = (float)cos(angle_deg[f] * pi / 180), s = (float)sin(...) (host libm),
 * i.e. content on the +x axis turns towards +y (counter-clockwise with row 0
 * drawn at the bottom).  The source position, its floor and fraction are
 * computed in float, each operation rounded (no fused multiply-add); img_f
 * between pixel centres is the bilinear interpolation of its four
 * neighbours, a neighbour of zero weight being unused.  A used neighbour
 * outside the frame, NaN, or with valid == 0 makes rot_f(x, y) NaN (missing).
 * The stacked image is, per pixel, the mean (float, compensated summation in
 * frame order) or the median (the mean of the two middle values for an even
 * count) of the frames whose rot_f is not NaN; NaN where none is.
 *   img        device, F x ny x nx floats, row-major; NaN = missing data.
 *   valid      device, ny x nx bytes (0 = missing in every frame), or NULL.
 *   angle_deg  HOST, F doubles, finite.
 *   cx, cy     rotation centre in pixel coordinates (column, row), |cx|, |cy| <= 2^20.
 *   method     nmf_combine_method.
 *   rot        device, F x ny x nx rotated frames (written), or NULL.
 *   out        device, ny x nx stacked image (written), or NULL (no stacking).
 *   count      device, ny x nx int32: frames covering each pixel, or NULL.
 *   Limits: 1 <= F <= 1024, 1 <= ny, nx <= 16384, at least one of rot, out,
 *   count non-NULL, valid method; otherwise NMF_EINVAL with nothing launched.
 *   One kernel launch, asynchronous on `stream`; img must not overlap the
 *   outputs.
 */
NMF_API nmf_status nmf_derotate_combine(const float *img, int64_t F, int32_t ny, int32_t nx, const uint8_t *valid,
                                        const double *angle_deg, float cx, float cy, int32_t method, float *rot,
                                        float *out, int32_t *count, void *stream);

/*
 * nmf_workspace_status -- synchronises `stream` and returns the device-side
 * status recorded in a workspace by nmf_fit_basis or nmf_project_target
 * (NMF_OK, NMF_EDATA if the data failed validation, NMF_ETIMEOUT if a
 * bounded device-side wait gave up).  Synchronous.
 */
NMF_API nmf_status nmf_workspace_status(const void *ws, void *stream);

/* Text of the most recent CUDA runtime error seen by a library call on the
 * calling thread (after NMF_ECUDA), or "" if none.  Static per-thread
 * storage, valid until the next library call on this thread. */
NMF_API const char *nmf_last_cuda_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all devices, all threads).  Diagnostic: read before and after a region
 * to count the kernels launched inside it. */
NMF_API uint64_t nmf_launch_count(void);

/* Self-test of the failure handling (no step of the paper's method): one
 * kernel waits on an mbarrier nobody arrives at and on a global counter
 * nobody raises, each wait bounded by limit_ns (1 us .. 100 ms), exactly as
 * the tensor-core kernels bound theirs (1 s there).  status (host, 2
 * entries) receives the status each wait recorded: NMF_ETIMEOUT expected.
 * The device stays usable.  Synchronises `stream`.  NMF_EINVAL for a NULL
 * status or a limit out of range (nothing launched). */
NMF_API nmf_status nmf_wait_selftest(int64_t limit_ns, int32_t *status, void *stream);

/* Measurement aid (no step of the paper's method): the FP32 fused
 * multiply-add rate of the current device's CUDA cores, the ceiling of the
 * plain FP32 form.  One kernel of 4 blocks per SM x 512 threads, each thread
 * running eight independent chains of `iters` FMAs (1 .. 2^24), timed with
 * CUDA events on `stream` after a shorter warm-up launch; *tflops (host)
 * receives 2 flop x FMAs / time in TFLOP/s.  Synchronous.  NMF_EINVAL for a
 * NULL tflops or iters out of range. */
NMF_API nmf_status nmf_fp32_fma_rate(int32_t iters, double *tflops, void *stream);

/* Failure-handling test aid (no step of the paper's method).  With
 * t_fault >= 0, every tensor-core fit (either form) enqueued afterwards
 * plants one missing arrival: at iteration t_fault of each stage's loop,
 * block 0 of the W pass waits for an H-pass tile count that is never
 * reached.  The wait gives up after limit_ns (1 us .. 100 ms), records
 * NMF_ETIMEOUT in the workspace status word, the block lets the copies and
 * MMAs it has issued complete and frees its TMEM, the iteration loop stops
 * and the call's remaining kernels return at once; nothing faults, traps or
 * hangs.  t_fault < 0 removes the plant (limit_ns ignored).  Process-wide,
 * for calls made after it.  NMF_EINVAL for a limit out of range. */
NMF_API nmf_status nmf_debug_plant_timeout(int32_t t_fault, int64_t limit_ns);

/* Diagnostic, host only (no device use): the W-pass block schedule the
 * tensor-core fit of a rows x P problem uses on a GPU with `sms` SMs (an
 * implementation detail of nmf_fit_basis, not a step of the paper's
 * method).  Block b streams the 64-pixel chunks [c0[b], c1[b]) of row tile
 * tile[b] (128 rows each) into partial slot split[b] of that tile.  Returns
 * the number of blocks written (at most max_blocks; the arrays are host
 * memory of max_blocks entries), 0 when the fit uses equal splits instead,
 * -1 for invalid arguments or max_blocks too small. */
NMF_API int32_t nmf_w_schedule(int64_t rows, int64_t P, int32_t sms, int32_t max_blocks, int32_t *tile,
                               int32_t *split, int32_t *c0, int32_t *c1);

/*
 * nmf_reduce_host -- the whole hot path from HOST buffers: copies V, Wt, the
 * initial factors and the science frames to the device, runs nmf_fit_basis,
 * nmf_project_target and nmf_subtract, and copies W, H, C, the residuals R
 * (M x P) and the per-stage costs and iteration counts back.  Device memory
 * comes from a cache inside the library that grows as needed and lives until
 * process exit.  Synchronous.  Host buffers may be pageable or pinned
 * (pinned is faster).  Pointers W0/H0/C0 are inputs; W/H/C/R/chi2_hist/
 * iters_done are outputs (host).  proj_iters = iterations of the projection.
 */
NMF_API nmf_status nmf_reduce_host(const float *V, const float *Wt, const float *W0, const float *H0,
                           const float *T, const float *WtT, const float *C0, int64_t M,
                           const nmf_fit_params *prm, int32_t proj_iters, float *W, float *H, float *C,
                           float *R, double *chi2_hist, int32_t *iters_done);

#ifdef __cplusplus
}
#endif

#endif /* NMF_GB300_H */
