/*
 * FP64 CPU oracle for the weighted-NMF coronagraphy hot path
 * (arXiv:2309.04623, "NMF-based GPU accelerated coronagraphy pipeline").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the CUDA
 * path is checked against.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Notation (the paper's X is our V, the paper's weighting term V is our Wt):
 *   V   N x P   reference library, one masked frame per row, pixels contiguous
 *   Wt  N x P   per-pixel weights (missing data = 0)
 *   W   N x K   coefficients,   H  K x P  basis components
 * All arithmetic is double; float inputs are promoted exactly.
 *
 * What each function follows:
 *   nmf_chi2        Eq. 2   weighted Frobenius cost  sum Wt (V - WH)^2
 *   nmf_iterate     Eq. 3   H-step with W fixed, then W-step with the new H
 *   tiny entries    (reading) factor entries below 2^-126 become exact zeros
 *   nmf_fit         Sec. 2  random start, iterate until the decrease of the
 *                           cost reaches a set value or the iteration cap;
 *                           components added one at a time (k = 1..K) with
 *                           warm start, each H row normalised after a stage
 *   nmf_project     Sec. 4.1 modelling of every science frame: Eq. 3's coefficient
 *                           update with the basis H held fixed
 *   nmf_subtract    Sec. 4.1 PSF subtraction: residual = target - model
 *   distances,      Sec. 4.1 reference selection: the library frames closest
 *   select                  to each target frame by the Euclidean norm of the
 *                           difference, weighted as in the NMF cost (Eq. 2),
 *                           the n_keep closest kept (ties by library order)
 *   rotate          Sec. 4.1/4.2 North-up: each subtracted frame rotated by
 *                           its angle about the star by bilinear
 *                           interpolation; missing data stay missing (NaN)
 *   combine         Sec. 4.1/4.2 stacking of the rotated frames: per pixel the
 *                           mean or the median of the frames that cover it
 *
 * Loop orders are chosen so that every sum runs over its index in increasing
 * order; OpenMP only splits independent output rows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(r, c, ld) ((int64_t)(r) * (int64_t)(ld) + (int64_t)(c))

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* R = W[:, :k] H[:k, :]   (W has leading dimension ldw). */
static void product_WH(int64_t N, int64_t P, int k, const double *W, int ldw, const double *H, double *R) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        double *r = R + IDX(n, 0, P);
        for (int64_t p = 0; p < P; ++p) r[p] = 0.0;
        for (int i = 0; i < k; ++i) {
            const double w = W[IDX(n, i, ldw)];
            const double *h = H + IDX(i, 0, P);
            for (int64_t p = 0; p < P; ++p) r[p] += w * h[p];
        }
    }
}

/* out (k x P) = W[:, :k]^T X   with X N x P:  out[i,p] = sum_n W[n,i] X[n,p]. */
static void product_WtX(int64_t N, int64_t P, int k, const double *W, int ldw, const double *X, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < k; ++i) {
        double *o = out + IDX(i, 0, P);
        for (int64_t p = 0; p < P; ++p) o[p] = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            const double w = W[IDX(n, i, ldw)];
            const double *x = X + IDX(n, 0, P);
            for (int64_t p = 0; p < P; ++p) o[p] += w * x[p];
        }
    }
}

/* out (N x k, ld ldo) = X H[:k]^T :  out[n,i] = sum_p X[n,p] H[i,p]. */
static void product_XHt(int64_t N, int64_t P, int k, const double *X, const double *H, double *out, int ldo) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        const double *x = X + IDX(n, 0, P);
        for (int i = 0; i < k; ++i) {
            const double *h = H + IDX(i, 0, P);
            double s = 0.0;
            for (int64_t p = 0; p < P; ++p) s += x[p] * h[p];
            out[IDX(n, i, ldo)] = s;
        }
    }
}

/* Eq. 2: sum_{n,p} Wt (V - R)^2 in natural row-major order. */
static double chi2_of(int64_t N, int64_t P, const double *V, const double *Wt, const double *R) {
    double s = 0.0;
    for (int64_t n = 0; n < N; ++n)
        for (int64_t p = 0; p < P; ++p) {
            const double e = V[IDX(n, p, P)] - R[IDX(n, p, P)];
            s += Wt[IDX(n, p, P)] * e * e;
        }
    return s;
}

/* Smallest magnitude a factor entry keeps (reading of the paper, which is
 * silent on underflow): an entry of W, H or C that an update or the
 * per-stage normalisation leaves below it becomes exactly 0 and, like every
 * zero entry, stays 0.  The default is 2^-126, the smallest normal single
 * precision value, the range the factors are stored in on the GPU; entries
 * this small are dozens of orders of magnitude below any that contributes to
 * W H.  0 turns the rule off (plain double precision). */
static double g_tiny = 0x1p-126;

void oracle_set_tiny(double t) { g_tiny = t >= 0.0 ? t : 0.0; }
double oracle_get_tiny(void) { return g_tiny; }

static inline double flush_tiny(double x) { return x < g_tiny ? 0.0 : x; }

/* The multiplicative rule with the zero-preserving guard and the epsilon
 * clamp on the denominator:  x <- 0 if x == 0, else x * num / max(den, eps),
 * then the tiny-entry rule above. */
static inline double mu_update(double x, double num, double den, double eps) {
    if (x == 0.0) return 0.0;
    return flush_tiny(x * num / (den > eps ? den : eps));
}

typedef struct {
    int64_t N, P;
    double *V, *Wt, *A; /* A = Wt o V */
    double *R, *D;      /* N x P scratch: reconstruction and Wt o R */
    double *NH, *DH;    /* K x P */
    double *NW, *DW;    /* N x K */
} work_t;

static int work_init(work_t *w, int64_t N, int64_t P, int K, const float *V, const float *Wt) {
    memset(w, 0, sizeof(*w));
    w->N = N;
    w->P = P;
    size_t np = (size_t)N * (size_t)P;
    w->V = malloc(np * sizeof(double));
    w->Wt = malloc(np * sizeof(double));
    w->A = malloc(np * sizeof(double));
    w->R = malloc(np * sizeof(double));
    w->D = malloc(np * sizeof(double));
    w->NH = malloc((size_t)K * P * sizeof(double));
    w->DH = malloc((size_t)K * P * sizeof(double));
    w->NW = malloc((size_t)N * K * sizeof(double));
    w->DW = malloc((size_t)N * K * sizeof(double));
    if (!w->V || !w->Wt || !w->A || !w->R || !w->D || !w->NH || !w->DH || !w->NW || !w->DW) return -1;
    for (size_t i = 0; i < np; ++i) {
        w->V[i] = (double)V[i];
        w->Wt[i] = (double)Wt[i];
        w->A[i] = w->Wt[i] * w->V[i];
    }
    return 0;
}

static void work_free(work_t *w) {
    free(w->V);
    free(w->Wt);
    free(w->A);
    free(w->R);
    free(w->D);
    free(w->NH);
    free(w->DH);
    free(w->NW);
    free(w->DW);
}

/* One iteration of Eq. 3 at rank k (first k columns of W, first k rows of H):
 *   H <- H o [W^T (Wt o V)] / [W^T (Wt o (W H))]
 *   W <- W o [(Wt o V) H^T] / [(Wt o (W H)) H^T]      (with the new H)
 * Returns the cost Eq. 2 of the updated pair. */
static double iterate_once(work_t *w, int k, double *W, int ldw, double *H, double eps) {
    const int64_t N = w->N, P = w->P;
    /* H-step */
    product_WH(N, P, k, W, ldw, H, w->R);
    for (int64_t i = 0; i < N * P; ++i) w->D[i] = w->Wt[i] * w->R[i];
    product_WtX(N, P, k, W, ldw, w->A, w->NH);
    product_WtX(N, P, k, W, ldw, w->D, w->DH);
    for (int i = 0; i < k; ++i)
        for (int64_t p = 0; p < P; ++p)
            H[IDX(i, p, P)] = mu_update(H[IDX(i, p, P)], w->NH[IDX(i, p, P)], w->DH[IDX(i, p, P)], eps);
    /* W-step with the new H */
    product_WH(N, P, k, W, ldw, H, w->R);
    for (int64_t i = 0; i < N * P; ++i) w->D[i] = w->Wt[i] * w->R[i];
    product_XHt(N, P, k, w->A, H, w->NW, ldw);
    product_XHt(N, P, k, w->D, H, w->DW, ldw);
    for (int64_t n = 0; n < N; ++n)
        for (int i = 0; i < k; ++i)
            W[IDX(n, i, ldw)] = mu_update(W[IDX(n, i, ldw)], w->NW[IDX(n, i, ldw)], w->DW[IDX(n, i, ldw)], eps);
    /* Eq. 2 on the updated pair */
    product_WH(N, P, k, W, ldw, H, w->R);
    return chi2_of(N, P, w->V, w->Wt, w->R);
}

/* Stopping rule (Sec. 2): stop once the relative decrease of the cost from one
 * iteration to the next is at most tol (tol <= 0: run all iterations). */
static int should_stop(int t, double prev, double cur, double tol) {
    return tol > 0.0 && t >= 2 && (prev - cur) <= tol * prev;
}

/* Weighted cost of the pair (W[:, :k] with ld ldw, H[:k]). */
double oracle_chi2(int64_t N, int64_t P, int k, const float *V, const float *Wt, const double *W, int ldw,
                   const double *H) {
    work_t w;
    if (work_init(&w, N, P, k > 0 ? k : 1, V, Wt)) {
        work_free(&w);
        return NAN;
    }
    product_WH(N, P, k, W, ldw, H, w.R);
    double c = chi2_of(N, P, w.V, w.Wt, w.R);
    work_free(&w);
    return c;
}

/* n_iter iterations of Eq. 3 at fixed rank k from the state (W, H), in place.
 * chi2_trace[t] (length n_iter, may be NULL) receives the cost after
 * iteration t+1.  With tol > 0 the stopping rule applies and the state
 * returned is the one after the iteration that met it.  Returns the number of
 * iterations done, or -1 on allocation failure. */
int oracle_iterate(int64_t N, int64_t P, int k, const float *V, const float *Wt, double *W, int ldw, double *H,
                   int n_iter, double tol, double eps, double *chi2_trace) {
    work_t w;
    if (work_init(&w, N, P, k, V, Wt)) {
        work_free(&w);
        return -1;
    }
    double prev = 0.0;
    int t;
    for (t = 1; t <= n_iter; ++t) {
        double c = iterate_once(&w, k, W, ldw, H, eps);
        if (chi2_trace) chi2_trace[t - 1] = c;
        if (should_stop(t, prev, c, tol)) break;
        prev = c;
    }
    work_free(&w);
    return t > n_iter ? n_iter : t;
}

/* Sequential construction of the basis, stages k = k_start+1 .. K.
 *   W (N x K) and H (K x P) hold, on entry, the converted initial factors W0,
 *   H0 (and, for k_start > 0, the first k_start fitted components).  Stage k
 *   brings in column k of W0 and row k of H0 (already in place), then runs
 *   up to n_iter iterations on all k components, then (normalize != 0)
 *   rescales each H row to unit L2 norm and the matching W column by the
 *   inverse, which leaves W H unchanged.
 *   chi2_hist[k-1]: cost after the last iteration of stage k (before the
 *   rescale); iters_done[k-1]: iterations run in stage k; chi2_trace (may be
 *   NULL): K x n_iter, the cost after every iteration (NaN after a stop). */
int oracle_fit(int64_t N, int64_t P, int K, const float *V, const float *Wt, double *W, double *H, int n_iter,
               double tol, double eps, int normalize, int k_start, double *chi2_hist, int *iters_done,
               double *chi2_trace) {
    work_t w;
    if (work_init(&w, N, P, K, V, Wt)) {
        work_free(&w);
        return -1;
    }
    for (int k = k_start + 1; k <= K; ++k) {
        double prev = 0.0, c = NAN;
        int t, done = 0;
        if (chi2_trace)
            for (int s = 0; s < n_iter; ++s) chi2_trace[IDX(k - 1, s, n_iter)] = NAN;
        for (t = 1; t <= n_iter; ++t) {
            c = iterate_once(&w, k, W, K, H, eps);
            if (chi2_trace) chi2_trace[IDX(k - 1, t - 1, n_iter)] = c;
            done = t;
            if (should_stop(t, prev, c, tol)) break;
            prev = c;
        }
        if (n_iter == 0) {
            product_WH(N, P, k, W, K, H, w.R);
            c = chi2_of(N, P, w.V, w.Wt, w.R);
        }
        chi2_hist[k - 1] = c;
        iters_done[k - 1] = done;
        if (normalize) {
            for (int i = 0; i < k; ++i) {
                double s = 0.0;
                for (int64_t p = 0; p < P; ++p) s += H[IDX(i, p, P)] * H[IDX(i, p, P)];
                s = sqrt(s);
                if (s > 0.0) {
                    for (int64_t p = 0; p < P; ++p) H[IDX(i, p, P)] = flush_tiny(H[IDX(i, p, P)] / s);
                    for (int64_t n = 0; n < N; ++n) W[IDX(n, i, K)] = flush_tiny(W[IDX(n, i, K)] * s);
                }
            }
        }
    }
    work_free(&w);
    return 0;
}

/* Target modelling (Sec. 4.1): coefficients C (M x K) of the science frames T
 * on the fixed basis H (K x P) by Eq. 3's W-rule with H held fixed:
 *   C <- C o [(WtT o T) H^T] / [(WtT o (C H)) H^T],  n_iter times, in place. */
int oracle_project(int64_t M, int64_t P, int K, const double *H, const float *T, const float *WtT, double *C,
                   int n_iter, double eps) {
    work_t w;
    if (work_init(&w, M, P, K, T, WtT)) {
        work_free(&w);
        return -1;
    }
    /* (WtT o T) H^T does not change while H is fixed. */
    product_XHt(M, P, K, w.A, H, w.NW, K);
    for (int t = 0; t < n_iter; ++t) {
        product_WH(M, P, K, C, K, H, w.R);
        for (int64_t i = 0; i < M * P; ++i) w.D[i] = w.Wt[i] * w.R[i];
        product_XHt(M, P, K, w.D, H, w.DW, K);
        for (int64_t m = 0; m < M; ++m)
            for (int i = 0; i < K; ++i)
                C[IDX(m, i, K)] = mu_update(C[IDX(m, i, K)], w.NW[IDX(m, i, K)], w.DW[IDX(m, i, K)], eps);
    }
    work_free(&w);
    return 0;
}

/* PSF subtraction (Sec. 4.1): Res[m,p] = T[m,p] - f_m * sum_i C[m,i] H[i,p]
 * (factor NULL means f_m = 1). */
void oracle_subtract(int64_t M, int64_t P, int K, const float *T, const double *C, const double *H,
                     const double *factor, double *Res) {
    for (int64_t m = 0; m < M; ++m) {
        const double f = factor ? factor[m] : 1.0;
        for (int64_t p = 0; p < P; ++p) {
            double model = 0.0;
            for (int i = 0; i < K; ++i) model += C[IDX(m, i, K)] * H[IDX(i, p, P)];
            Res[IDX(m, p, P)] = (double)T[IDX(m, p, P)] - f * model;
        }
    }
}

/* Reference selection (Sec. 4.1): D[m,n] = sum_p WtT[m,p] (T[m,p] - V[n,p])^2,
 * the squared Euclidean norm of target frame m minus library frame n with
 * the target's weights (the NMF cost, Eq. 2, of modelling T_m by V_n). */
void oracle_distances(int64_t M, int64_t N, int64_t P, const float *T, const float *WtT, const float *V, double *D) {
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < M; ++m)
        for (int64_t n = 0; n < N; ++n) {
            double s = 0.0;
            for (int64_t p = 0; p < P; ++p) {
                const double d = (double)T[IDX(m, p, P)] - (double)V[IDX(n, p, P)];
                s += (double)WtT[IDX(m, p, P)] * d * d;
            }
            D[IDX(m, n, N)] = s;
        }
}

/* The n_keep closest library frames of every target frame, closest first;
 * equal distances are ordered by library index.  Selection by repeated
 * minimum: the plainest reading of keeping the nearest frames. */
void oracle_select(int64_t M, int64_t N, const double *D, int32_t n_keep, int32_t *idx) {
    char *taken = (char *)malloc((size_t)N);
    for (int64_t m = 0; m < M; ++m) {
        memset(taken, 0, (size_t)N);
        for (int32_t r = 0; r < n_keep; ++r) {
            int64_t best = -1;
            for (int64_t n = 0; n < N; ++n)
                if (!taken[n] && (best < 0 || D[IDX(m, n, N)] < D[IDX(m, best, N)])) best = n;
            taken[best] = 1;
            idx[IDX(m, r, n_keep)] = (int32_t)best;
        }
    }
    free(taken);
}

/* North-up rotation (Sec. 4.1 and 4.2: the subtracted frames are rotated by
 * their position angles before they are combined).  Frame f's content is
 * rotated by angle_deg[f] about (cx, cy) (x = column, y = row):
 *
 *   out_f(x, y) = in_f(xs, ys),  xs = cx + ( c (x - cx) + s (y - cy)),
 *                                ys = cy + ( c (y - cy) - s (x - cx)),
 *   c = cos(angle), s = sin(angle) rounded to float,
 *
 * in_f between pixel centres by bilinear interpolation of its four
 * neighbours.  A neighbour whose interpolation weight is zero is not used;
 * if a used neighbour lies outside the frame, is NaN, or is flagged invalid
 * in `valid` (ny x nx bytes, 0 = missing, NULL = all valid), out is NaN.
 * The source position, its floor and its fractional part are the decision
 * of which pixels are used; they are computed in float, in the order written
 * above (no fused multiply-add), so that any float implementation of the
 * same formula takes the same decision.  The interpolation is double. */
#define ORACLE_PI 3.14159265358979323846

void oracle_rotate(int64_t F, int32_t ny, int32_t nx, const float *img, const uint8_t *valid,
                   const double *angle_deg, float cx, float cy, double *out) {
    const int64_t npix = (int64_t)ny * nx;
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < F; ++f) {
        const double th = angle_deg[f] * (ORACLE_PI / 180.0);
        const float c = (float)cos(th), s = (float)sin(th);
        const float *in = img + f * npix;
        double *o = out + f * npix;
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x) {
                const float dx = (float)x - cx, dy = (float)y - cy;
                const float cdx = c * dx, sdy = s * dy, cdy = c * dy, sdx = s * dx;
                const float xs = cx + (cdx + sdy), ys = cy + (cdy - sdx);
                const float x0f = floorf(xs), y0f = floorf(ys);
                const float fx = xs - x0f, fy = ys - y0f;
                double val = NAN;
                /* the neighbours used: (x0, y0) always, x0 + 1 iff fx > 0, y0 + 1 iff fy > 0 */
                const int ux = fx > 0.0f, uy = fy > 0.0f;
                if (x0f >= 0.0f && y0f >= 0.0f && x0f + (float)ux <= (float)(nx - 1) &&
                    y0f + (float)uy <= (float)(ny - 1)) {
                    const int64_t x0 = (int64_t)x0f, y0 = (int64_t)y0f;
                    const double wx[2] = {1.0 - (double)fx, (double)fx};
                    const double wy[2] = {1.0 - (double)fy, (double)fy};
                    double acc = 0.0;
                    int ok = 1;
                    for (int j = 0; j <= uy && ok; ++j)
                        for (int i = 0; i <= ux; ++i) {
                            const int64_t q = (y0 + j) * nx + (x0 + i);
                            const float v = in[q];
                            if (isnan(v) || (valid && !valid[q])) { ok = 0; break; }
                            acc += wy[j] * wx[i] * (double)v;
                        }
                    if (ok) val = acc;
                }
                o[(int64_t)y * nx + x] = val;
            }
    }
}

static int cmp_double(const void *a, const void *b) {
    const double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Stacking of the rotated frames (Sec. 4.1 and 4.2: the rotated frames are
 * combined to raise the signal-to-noise ratio and the sky coverage).  For
 * every pixel, over the frames whose value there is not NaN (count[p] of
 * them): method 0 = their mean, method 1 = their median (the mean of the two
 * middle values when the count is even).  A pixel no frame covers is NaN. */
void oracle_combine(int64_t F, int64_t npix, const double *frames, int32_t method, double *out, int32_t *count) {
#pragma omp parallel
    {
        double *buf = (double *)malloc((size_t)(F > 0 ? F : 1) * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t p = 0; p < npix; ++p) {
            int64_t n = 0;
            for (int64_t f = 0; f < F; ++f) {
                const double v = frames[f * npix + p];
                if (!isnan(v)) buf[n++] = v;
            }
            double r = NAN;
            if (n > 0 && method == 0) {
                double sum = 0.0;
                for (int64_t i = 0; i < n; ++i) sum += buf[i];
                r = sum / (double)n;
            } else if (n > 0) {
                qsort(buf, (size_t)n, sizeof(double), cmp_double);
                r = 0.5 * (buf[(n - 1) / 2] + buf[n / 2]);
            }
            out[p] = r;
            if (count) count[p] = (int32_t)n;
        }
        free(buf);
    }
}
