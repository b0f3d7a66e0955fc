// C-ABI entry points of libnmfgb (declared in include/nmf.h).
//
// Host orchestration only: argument checks, workspace carving, tensor-map
// encoding, and the enqueueing of the kernels of nmf_simt.cu (FP32 form) and
// nmf_tc.cu (tensor-core form) on the caller's stream.  No arithmetic of the
// method runs on the host.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <list>
#include <mutex>
#include <string>
#include <vector>
#include <unordered_map>

#include "nmf_internal.cuh"
#include "nmf_tc.cuh"

using namespace nmfgb;

namespace nmfgb {
static std::atomic<unsigned long long> g_launches{0};
// While a graph is being recorded, launches are tallied for the graph (loop
// bodies times their iteration count) instead of the process counter; each
// launch of the graph then adds its tally.
thread_local bool t_recording = false;
thread_local unsigned long long t_recorded = 0, t_multiplier = 1;
void count_launches(unsigned long long n) {
    if (t_recording)
        t_recorded += n * t_multiplier;
    else
        g_launches.fetch_add(n, std::memory_order_relaxed);
}

thread_local char t_last_error[256] = "";

nmf_status cuda_fail(cudaError_t e, const char *what) {
    snprintf(t_last_error, sizeof(t_last_error), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    return NMF_ECUDA;
}

// Pixel splits of the W pass: enough blocks for ~4 per SM, each split a
// multiple of the pass chunk, at most max_splits of them.
void choose_splits(long long rows, int k, long long Pp, int max_splits, int *nsplit, int *split_len) {
    const int chunk = wpass_chunk_pixels();
    const long long tiles = wpass_row_tiles(k, rows);
    long long want = (4LL * 152 + tiles - 1) / tiles;
    const long long max_by_p = (Pp + chunk - 1) / chunk;
    if (want > max_by_p) want = max_by_p;
    if (want > max_splits) want = max_splits;
    if (want < 1) want = 1;
    long long len = (Pp + want - 1) / want;
    len = (len + chunk - 1) / chunk * chunk;
    *split_len = (int)len;
    *nsplit = (int)((Pp + len - 1) / len);
}
}  // namespace nmfgb

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
inline bool aligned256(const void *p) { return (reinterpret_cast<uintptr_t>(p) & (kAlign - 1)) == 0; }

// Leading dimension of the internal coefficient arrays: a power of two >= 32
// that covers every per-stage component tile (8, 16, 32, 64, 128).
inline int ldw_of(int K) { return K <= 32 ? 32 : (K <= 64 ? 64 : 128); }

constexpr int kMaxSplits = 128;

// Planted missing arrival of nmf_debug_plant_timeout (iteration, wait limit);
// -1 = none.  Read when a fit is emitted and part of its graph key.
std::atomic<int> g_fault_t{-1};
std::atomic<long long> g_fault_ns{0};
// Most tensor-core iterations per recorded loop body: the WHILE node's
// turnaround and the loop-control launch are paid once per body, and the
// iterations of the last body past the loop's count are launched but return
// at once; the body size (16, 8, 4, ... up to this) is chosen per loop to
// minimise the two counts together.
#ifndef NMF_TC_UNROLL
#define NMF_TC_UNROLL 16
#endif
constexpr int kTcUnroll = NMF_TC_UNROLL;

int body_size(int n, int max_unroll) {
    int best = 1;
    long long best_cost = n;  // one iteration per body: n turnarounds, nothing skipped
    for (int u = 2; u <= max_unroll; u *= 2) {
        const long long bodies = (n + u - 1) / u, skipped = bodies * u - n;
        if (bodies + skipped < best_cost) {
            best_cost = bodies + skipped;
            best = u;
        }
    }
    return best;
}
static_assert(kMaxSplits == kMaxWSplits, "the W update reads at most kMaxWSplits partials per row");

// Row tiles of the W pass are never smaller than 8 rows.
inline long long max_row_tiles(long long rows) { return (rows + 7) / 8; }


// Pixel splits of the tensor-core W pass when it has no explicit schedule
// (w_schedule): at most one block per SM (each block holds a whole SM's
// shared memory), splits a multiple of the 64-pixel chunk, the shortest
// for which all blocks fit on the SMs.  The last row tile holds r <= 128
// rows; its splits may be made longer in proportion to its cheaper chunks,
// down to NMF_TC_PHI of a full chunk's cost.  Measured on GB300 a chunk costs
// the same time whatever its rows (the pipeline's per-chunk latency, not its
// bytes, sets the pace), so the default is 1: equal splits everywhere.
#ifndef NMF_TC_PHI
#define NMF_TC_PHI 1.0
#endif
void choose_splits_tc(long long rows, long long Pp, TcArgs &ta) {
    const long long chunk = tc_split_granule();
    const long long tile = tc_tile();
    const long long ntr = (rows + tile - 1) / tile;
    const long long r_last = rows - (ntr - 1) * tile;
    const long long sms = tc_num_sms() > 0 ? tc_num_sms() : 152;
    const long long nchunks = (Pp + chunk - 1) / chunk;
    double c_last = (double)r_last / (double)tile;
    if (c_last < NMF_TC_PHI) c_last = NMF_TC_PHI;
    auto splits = [&](long long nch) { return (nchunks + nch - 1) / nch; };
    for (long long nch = 1; nch <= nchunks; ++nch) {
        long long nch_l = (long long)((double)nch / c_last);
        if (nch_l < 1) nch_l = 1;
        if (nch_l > nchunks) nch_l = nchunks;
        const long long nf = ntr > 1 ? splits(nch) : 0, nl = splits(nch_l);
        if ((ntr - 1) * nf + nl <= sms && nf <= kMaxSplits && nl <= kMaxSplits) {
            ta.split_len = (int)(nch * chunk);
            ta.nsplit = (int)(ntr > 1 ? nf : nl);
            ta.split_len_last = (int)(nch_l * chunk);
            ta.nsplit_last = (int)nl;
            return;
        }
    }
    // more row tiles than SMs: one split per block
    ta.split_len = ta.split_len_last = (int)(nchunks * chunk);
    ta.nsplit = ta.nsplit_last = 1;
}

// Explicit W-pass schedule for a W pass that overlaps its H pass (see
// TcArgs::w_nblk).  The H pass gives its hb blocks ntiles 128-pixel tiles
// round-robin; when ntiles is not a multiple of hb, the rem blocks with an
// extra tile finish a tile's time after the others, whose SMs (and the SMs
// the H pass leaves unused) take the first W blocks.  Those E "early" blocks
// get ranges longer by about one H tile's time (its row chunks plus the tile
// transition, NMF_TC_WHEAD chunks beyond them) over pixels whose tiles are
// written before the last round; the rem "late" blocks share the rest.
// Returns false (equal splits instead) when the shape does not fit.
#ifndef NMF_TC_WHEAD
#define NMF_TC_WHEAD 2
#endif
bool w_schedule(long long rows, long long Pp, long long S, TcArgs &ta) {
    const long long unit = tc_split_granule();
    const long long ntr = (rows + tc_tile() - 1) / tc_tile();
    const long long nch = Pp / unit;  // chunks per row tile
    const long long ntiles = Pp / 128, hb = ntiles < S ? ntiles : S;  // the H pass's blocks (tc_hpass_blocks)
    if (hb <= 0 || ntr > kMaxWRowTiles || nch > 65535 || S > kMaxWBlocks) return false;
    const long long rem = ntiles % hb, rounds = ntiles / hb;
    if (rem == 0 || rounds < 1) return false;
    const long long E = S - rem;                          // early SMs
    const long long early_lim = rounds * hb * 128 / unit;  // chunks written before the last round
    const long long head = (rows + unit - 1) / unit + NMF_TC_WHEAD;
    const long long total = ntr * nch;
    long long Ll = (total - E * head) / S;
    if (Ll < 1) Ll = 1;
    for (; Ll <= nch; ++Ll) {
        const long long Le = Ll + head;
        long long nblk = 0;
        int nsplit[kMaxWRowTiles] = {};
        long long xe[kMaxWRowTiles] = {};
        // the early blocks shared among the row tiles, each over the tile's first pixels
        for (long long t = 0; t < ntr; ++t) {
            const long long et = E / ntr + (t < E % ntr ? 1 : 0);
            long long x = et * Le;
            if (x > early_lim) x = early_lim;
            if (x > nch) x = nch;
            xe[t] = x;
        }
        long long late = 0;
        for (long long t = 0; t < ntr; ++t) late += (nch - xe[t] + Ll - 1) / Ll;
        for (long long t = 0; t < ntr; ++t) nblk += (xe[t] + Le - 1) / Le;
        nblk += late;
        if (nblk > S) continue;
        // emit: early blocks first (tile-major), then late blocks (tile-major)
        int b = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (long long t = 0; t < ntr; ++t) {
                const long long lo = pass == 0 ? 0 : xe[t], hi = pass == 0 ? xe[t] : nch;
                const long long len = pass == 0 ? Le : Ll;
                for (long long c = lo; c < hi; c += len) {
                    ta.w_tile[b] = (uint8_t)t;
                    ta.w_split[b] = (uint8_t)nsplit[t]++;
                    ta.w_c0[b] = (uint16_t)c;
                    ta.w_c1[b] = (uint16_t)(c + len < hi ? c + len : hi);
                    ++b;
                }
            }
        for (long long t = 0; t < ntr; ++t) {
            if (nsplit[t] > kMaxWSplits || nsplit[t] > 255) return false;
            ta.w_nsplit[t] = (uint8_t)nsplit[t];
        }
        ta.w_nblk = b;
        return true;
    }
    return false;
}

struct TcLayout {
    size_t Wtb, img[8], part, flags, total_extra;
};

// Extra workspace of the tensor-core forms, appended after a base layout:
// the 16-bit weights (written and read by the FP16-weights form only; the
// FP32-weights form streams the padded FP32 copy and leaves this region
// unused), the operand images (coefficient rows hi/lo, two sets of basis
// hi/lo, then the basis's two third-part sets) and the W-pass partials.
TcLayout tc_layout(size_t off, long long rows, long long Pp, int K) {
    TcLayout L;
    const size_t start = off;
    L.Wtb = off;
    off = align_up(off + 2 * (size_t)rows * Pp);
    for (int i = 0; i < 2; ++i) {
        L.img[i] = off;
        off = align_up(off + tc_image_bytes(rows, K));
    }
    for (int i = 2; i < 8; ++i) {
        L.img[i] = off;
        off = align_up(off + tc_image_bytes(Pp, K));
    }
    L.part = off;
    off = align_up(off + sizeof(float) * 2 * (size_t)tc_kp(K) * kMaxSplits * rows);
    L.flags = off;  // per 128-pixel tile of the basis: H passes that have written it
    off = align_up(off + sizeof(unsigned) * (size_t)((Pp + 127) / 128));
    L.total_extra = off - start;
    return L;
}

struct FitLayout {
    size_t state, tickets, chi2_part, norm_part, Vp, Wtp, Hb0, Hb1, Wp, part, total;
    TcLayout tc;
};

FitLayout fit_layout(long long N, long long P, int K, int prec) {
    FitLayout L;
    const long long Pp = pad_p(P);
    const int ldw = ldw_of(K);
    size_t off = 0;
    L.state = off;
    off = align_up(off + sizeof(FitState));
    L.tickets = off;
    off = align_up(off + sizeof(unsigned) * (size_t)max_row_tiles(N));
    L.chi2_part = off;
    off = align_up(off + sizeof(double) * (size_t)(Pp / 32 + 1));
    L.norm_part = off;
    off = align_up(off + sizeof(double) * (size_t)kMaxK * 16);
    L.Vp = off;
    off = align_up(off + sizeof(float) * (size_t)N * Pp);
    L.Wtp = off;
    off = align_up(off + sizeof(float) * (size_t)N * Pp);
    L.Hb0 = off;
    off = align_up(off + sizeof(float) * (size_t)K * Pp);
    L.Hb1 = off;
    off = align_up(off + sizeof(float) * (size_t)K * Pp);
    L.Wp = off;
    off = align_up(off + sizeof(float) * (size_t)N * ldw);
    L.part = off;
    off = align_up(off + sizeof(float) * 2 * (size_t)kMaxSplits * N * ldw);
    L.tc = tc_layout(off, N, Pp, K);
    L.total = off;
    if (prec == NMF_BF16_SPLIT || prec == NMF_BF16_SPLIT_W32) L.total += L.tc.total_extra;
    return L;
}

struct ProjLayout {
    size_t state, tickets, Tp, WtTp, Hp, Cp, num, part, total;
    TcLayout tc;
};

ProjLayout proj_layout(long long M, long long P, int K, int prec) {
    ProjLayout L;
    const long long Pp = pad_p(P);
    const int ldw = ldw_of(K);
    size_t off = 0;
    L.state = off;
    off = align_up(off + sizeof(FitState));
    L.tickets = off;
    off = align_up(off + sizeof(unsigned) * (size_t)max_row_tiles(M));
    L.Tp = off;
    off = align_up(off + sizeof(float) * (size_t)M * Pp);
    L.WtTp = off;
    off = align_up(off + sizeof(float) * (size_t)M * Pp);
    L.Hp = off;
    off = align_up(off + sizeof(float) * (size_t)K * Pp);
    L.Cp = off;
    off = align_up(off + sizeof(float) * (size_t)M * ldw);
    L.num = off;
    off = align_up(off + sizeof(float) * (size_t)M * ldw);
    L.part = off;
    off = align_up(off + sizeof(float) * 2 * (size_t)kMaxSplits * M * ldw);
    L.tc = tc_layout(off, M, Pp, K);
    L.total = off;
    if (prec == NMF_BF16_SPLIT || prec == NMF_BF16_SPLIT_W32) L.total += L.tc.total_extra;
    return L;
}

bool fit_params_ok(const nmf_fit_params *p) {
    if (!p) return false;
    if (p->N < 1 || p->P < 1 || p->K < 1 || p->K > kMaxK) return false;
    if (p->N >= (1LL << 31) || p->P >= (1LL << 31) - kPadP) return false;
    if ((long long)p->K > p->N || (long long)p->K > p->P) return false;
    if (p->iters_per_stage < 0 || p->k_start < 0 || p->k_start > p->K) return false;
    if (!(p->tol >= 0.0) || !isfinite(p->tol)) return false;
    if (!(p->eps > 0.0) || !(p->eps <= 1.0)) return false;
    if (p->precision == NMF_FP32) {
        if (p->polish_iters != 0) return false;
    } else if (p->precision == NMF_BF16_SPLIT || p->precision == NMF_BF16_SPLIT_W32) {
        if (p->K > tc_max_k() || p->polish_iters < 0) return false;
    } else {
        return false;
    }
    return true;
}

// Work of one call is emitted either as direct launches on the caller's
// stream or recorded into a CUDA graph in which every stage's iteration loop
// is a WHILE node (its body ends with a loop-control kernel that keeps going
// while iterations remain and the stopping rule has not fired).
struct Emitter {
    cudaStream_t s = nullptr;     // receives the launches (caller's stream, or the recording stream)
    bool graph = false;
    cudaStream_t body = nullptr;  // records loop bodies

    // n iterations of fn; recorded as a WHILE node whose body holds `unroll`
    // iterations (the kernels of an iteration past the count must do nothing
    // for unroll > 1: the tensor-core passes with t_end set)
    template <class F>
    nmf_status loop(int n, int t_limit, const FitState *st, F fn, int unroll = 1) {
        if (n <= 0) return NMF_OK;
        if (!graph) {
            for (int i = 0; i < n; ++i) {
                const nmf_status r = fn(s);
                if (r != NMF_OK) return r;
            }
            return NMF_OK;
        }
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        NMF_CUDA_TRY(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
        cudaGraphConditionalHandle h;
        NMF_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        NMF_CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
        NMF_CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        NMF_CUDA_TRY(cudaStreamBeginCaptureToGraph(body, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeRelaxed));
        const int u = body_size(n, unroll < 1 ? 1 : unroll);
        t_multiplier = (unsigned long long)((n + u - 1) / u);
        nmf_status r = NMF_OK;
        for (int i = 0; i < u && r == NMF_OK; ++i) r = fn(body);
        const cudaError_t e = launch_loop_ctl(st, t_limit, h, body);
        t_multiplier = 1;
        cudaGraph_t out = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(body, &out);
        if (r != NMF_OK) return r;
        NMF_CUDA_TRY(e);
        NMF_CUDA_TRY(e2);
        return NMF_OK;
    }
};

// Recorded graphs, keyed by every argument of the call (pointers and
// parameters), most recently used first.
struct GraphEntry {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    unsigned long long kernels = 0;
};
std::mutex g_graph_mu;
std::list<std::pair<std::string, GraphEntry>> g_graphs;
constexpr size_t kMaxGraphs = 16;
cudaStream_t g_rec_stream[64] = {}, g_body_stream[64] = {};

bool graphs_enabled(cudaStream_t caller) {
    if (getenv("NMF_NO_GRAPH")) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(caller, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    return true;
}

template <class T>
void key_add(std::string &k, const T &v) {
    k.append(reinterpret_cast<const char *>(&v), sizeof(T));
}

// Emit the work through `emit(Emitter&)`: direct launches when graphs are
// off, otherwise the cached (or newly recorded) graph of this argument set.
template <class F>
nmf_status run_emitted(const std::string &key, cudaStream_t caller, F emit) {
    if (!graphs_enabled(caller)) {
        Emitter em;
        em.s = caller;
        return emit(em);
    }
    int dev = 0;
    NMF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return NMF_ECUDA;
    std::string k = key;
    key_add(k, dev);
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
        if (it->first == k) {
            g_graphs.splice(g_graphs.begin(), g_graphs, it);
            NMF_CUDA_TRY(cudaGraphLaunch(it->second.ex, caller));
            g_launches.fetch_add(it->second.kernels, std::memory_order_relaxed);
            return NMF_OK;
        }
    }
    if (!g_rec_stream[dev]) {
        NMF_CUDA_TRY(cudaStreamCreateWithFlags(&g_rec_stream[dev], cudaStreamNonBlocking));
        NMF_CUDA_TRY(cudaStreamCreateWithFlags(&g_body_stream[dev], cudaStreamNonBlocking));
    }
    Emitter em;
    em.s = g_rec_stream[dev];
    em.graph = true;
    em.body = g_body_stream[dev];
    NMF_CUDA_TRY(cudaStreamBeginCapture(em.s, cudaStreamCaptureModeRelaxed));
    t_recording = true;
    t_recorded = 0;
    t_multiplier = 1;
    const nmf_status r = emit(em);
    t_recording = false;
    GraphEntry ge;
    const cudaError_t e = cudaStreamEndCapture(em.s, &ge.g);
    if (r != NMF_OK) {
        if (ge.g) cudaGraphDestroy(ge.g);
        return r;
    }
    NMF_CUDA_TRY(e);
    ge.kernels = t_recorded;
    const cudaError_t ei = cudaGraphInstantiate(&ge.ex, ge.g, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(ge.g);
        return cuda_fail(ei, "cudaGraphInstantiate");
    }
    if (g_graphs.size() >= kMaxGraphs) {
        GraphEntry old = g_graphs.back().second;
        g_graphs.pop_back();
        cudaGraphExecDestroy(old.ex);  // freed after any launch in flight completes
        cudaGraphDestroy(old.g);
    }
    g_graphs.emplace_front(k, ge);
    NMF_CUDA_TRY(cudaGraphLaunch(ge.ex, caller));
    g_launches.fetch_add(ge.kernels, std::memory_order_relaxed);
    return NMF_OK;
}

// The fit (nmf_fit_basis).  With `ext` the work is emitted into that
// emitter (a branch of a batched graph); otherwise it runs as a cached graph
// or direct launches on `stream`.
nmf_status fit_impl(const float *V, const float *Wt, float *W, float *H, double *chi2_hist, int32_t *iters_done,
                    void *ws, size_t ws_bytes, const nmf_fit_params *prm, void *stream, Emitter *ext) {
    if (!fit_params_ok(prm)) return NMF_EINVAL;
    if (!V || !Wt || !W || !H || !chi2_hist || !iters_done || !ws) return NMF_EINVAL;
    const long long N = prm->N, P = prm->P;
    const int K = prm->K;
    const bool tcp = prm->precision == NMF_BF16_SPLIT || prm->precision == NMF_BF16_SPLIT_W32;
    const bool wt32 = prm->precision == NMF_BF16_SPLIT_W32;
    const FitLayout L = fit_layout(N, P, K, prm->precision);
    if (ws_bytes < L.total || !aligned256(ws)) return NMF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(ws);
    FitState *st = reinterpret_cast<FitState *>(base + L.state);
    const long long Pp = pad_p(P);
    const int ldw = ldw_of(K);

    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.V = reinterpret_cast<float *>(base + L.Vp);
    a.Wt = reinterpret_cast<float *>(base + L.Wtp);
    a.W = reinterpret_cast<float *>(base + L.Wp);
    a.Hb0 = reinterpret_cast<float *>(base + L.Hb0);
    a.Hb1 = reinterpret_cast<float *>(base + L.Hb1);
    a.part = reinterpret_cast<float *>(base + L.part);
    a.chi2_part = reinterpret_cast<double *>(base + L.chi2_part);
    a.norm_part = reinterpret_cast<double *>(base + L.norm_part);
    a.tickets = reinterpret_cast<unsigned *>(base + L.tickets);
    a.st = st;
    a.rows = N;
    a.P = P;
    a.Pp = Pp;
    a.ldw = ldw;
    a.eps = (float)prm->eps;
    a.tol = prm->tol;

    TcArgs ta;
    memset(&ta, 0, sizeof(ta));
    uint8_t *img[8] = {};
    void *Wtb = nullptr;
    TcMaps maps[2];  // component widths 64 and 128 (the stages above 64 use the wider kernels)
    if (tcp) {
        Wtb = base + L.tc.Wtb;
        for (int i = 0; i < 8; ++i) img[i] = reinterpret_cast<uint8_t *>(base + L.tc.img[i]);
        for (int w = 0; w < (K > 64 ? 2 : 1); ++w)
            if (!tc_make_maps(&maps[w], a.V, wt32 ? static_cast<const void *>(a.Wt) : Wtb, N, Pp, 64 << w, wt32))
                return cuda_fail(cudaErrorInvalidValue, "cuTensorMapEncodeTiled");
        ta.W = a.W;
        ta.part = reinterpret_cast<float *>(base + L.tc.part);
        ta.chi2_part = a.chi2_part;
        ta.st = st;
        ta.wk_h = img[0];
        ta.wk_l = img[1];
        for (int i = 0; i < 2; ++i) {
            ta.hk_h[i] = img[2 + 2 * i];
            ta.hk_l[i] = img[3 + 2 * i];
            ta.hk_l2[i] = img[6 + i];
        }
        ta.rows = N;
        ta.Pp = Pp;
        ta.ldw = ldw;
        ta.eps = a.eps;
        ta.tol = a.tol;
        ta.wt32 = wt32 ? 1 : 0;
        ta.fault_t = g_fault_t.load();
        ta.fault_ns = (unsigned long long)g_fault_ns.load();
        choose_splits_tc(N, Pp, ta);
    }
    const int iters = prm->iters_per_stage, polish = tcp ? prm->polish_iters : 0;

    auto emit = [&](Emitter &em) -> nmf_status {
        const cudaStream_t s = em.s;
        NMF_CUDA_TRY(cudaMemsetAsync(base, 0, L.Vp, s));  // control block, tickets, partials
        NMF_CUDA_TRY(launch_prologue_copy(V, N, P, P, const_cast<float *>(a.V), Pp, Pp, st, 1, s));
        NMF_CUDA_TRY(launch_prologue_copy(Wt, N, P, P, const_cast<float *>(a.Wt), Pp, Pp, st, 1, s));
        NMF_CUDA_TRY(launch_prologue_copy(W, N, K, K, a.W, ldw, ldw, st, 1, s));
        NMF_CUDA_TRY(launch_prologue_copy(H, K, P, P, a.Hb0, Pp, Pp, st, 1, s));
        NMF_CUDA_TRY(cudaMemsetAsync(a.Hb1, 0, sizeof(float) * (size_t)K * Pp, s));
        if (tcp) {
            if (!wt32) NMF_CUDA_TRY(tc_weights_bf16(Wt, N, P, Wtb, Pp, st, s));
            NMF_CUDA_TRY(cudaMemsetAsync(img[0], 0, L.tc.part - L.tc.img[0], s));
        }
        for (int k = prm->k_start + 1; k <= K; ++k) {
            a.k = k;
            choose_splits(N, k, Pp, kMaxSplits, &a.nsplit, &a.split_len);
            NMF_CUDA_TRY(launch_stage_begin(st, s));
            const bool last = (k == K);
            nmf_status r;
            if (tcp) {
                ta.k = k;
                const int layout_prev = ta.kp == 0 ? 0 : (ta.packed ? 32 : ta.kp);
                ta.kp = tc_kp(k);
                ta.packed = tc_packed(k) ? 1 : 0;
                const TcMaps &mp = maps[ta.kp == 64 ? 0 : 1];
                // the image layout changes at k = 33 (packed to separate hi
                // and lo images) and at k = 65 (two 64-component blocks):
                // clear the images so every component >= k reads as zero
                if (layout_prev != 0 && layout_prev != (ta.packed ? 32 : ta.kp))
                    NMF_CUDA_TRY(cudaMemsetAsync(img[0], 0, L.tc.part - L.tc.img[0], s));
                // operand images of the stage's starting point (t = 0, state in Hb0)
                NMF_CUDA_TRY(tc_images(a.W, N, k, ldw, false, ta.wk_h, ta.wk_l, ta.kp, ta.packed, s));
                NMF_CUDA_TRY(tc_images(a.Hb0, Pp, k, Pp, true, ta.hk_h[0], ta.hk_l[0], ta.kp, ta.packed, s,
                                       ta.hk_l2[0]));
                // the final stage's last `polish` iterations run in FP32
                const int fp32_tail = last ? (polish < iters ? polish : iters) : 0;
                const int tc_iters = iters - fp32_tail;
                ta.t_end = tc_iters;
                ta.h_blocks = tc_hpass_blocks(Pp);  // the W pass records each iteration's Eq. 2
                if (!ext) {
                    // a single reduction: the W pass overlaps the H pass's
                    // last tiles (a batch's problems share the SMs, so their
                    // passes keep the plain order)
                    ta.h_flags = reinterpret_cast<unsigned *>(base + L.tc.flags);
                    NMF_CUDA_TRY(cudaMemsetAsync(ta.h_flags, 0, sizeof(unsigned) * (size_t)(Pp / 128), s));
                }
                // the same pixel splits with and without the overlap, so a
                // batch's members give the same sums as separate calls
                if (!w_schedule(N, Pp, tc_num_sms(), ta)) ta.w_nblk = 0;
                r = em.loop(tc_iters, tc_iters, st, [&](cudaStream_t bs) -> nmf_status {
                    NMF_CUDA_TRY(tc_hpass(mp, ta, false, bs));
                    NMF_CUDA_TRY(tc_wpass(mp, ta, bs));
                    return NMF_OK;
                }, kTcUnroll);
                ta.t_end = 0;
                ta.h_blocks = 0;
                ta.h_flags = nullptr;
                ta.w_nblk = 0;
                if (r != NMF_OK) return r;
                if (tc_iters > 0) NMF_CUDA_TRY(tc_h_from_images(ta, a.Hb0, a.Hb1, s));  // the iterate back in FP32
                if (fp32_tail > 0) {
                    // FP32 refinement continues from the kept state
                    NMF_CUDA_TRY(launch_clear_stop(st, fp32_tail, s));
                    r = em.loop(fp32_tail, -1, st, [&](cudaStream_t bs) -> nmf_status {
                        NMF_CUDA_TRY(launch_hpass_f32(a, false, bs));
                        NMF_CUDA_TRY(launch_wpass_f32(a, WP_FIT, bs));
                        return NMF_OK;
                    });
                    if (r != NMF_OK) return r;
                    NMF_CUDA_TRY(launch_hpass_f32(a, true, s));
                } else {
                    NMF_CUDA_TRY(tc_hpass(mp, ta, true, s));  // Eq. 2 of the final iterate
                }
            } else {
                r = em.loop(iters, iters, st, [&](cudaStream_t bs) -> nmf_status {
                    NMF_CUDA_TRY(launch_hpass_f32(a, false, bs));
                    NMF_CUDA_TRY(launch_wpass_f32(a, WP_FIT, bs));
                    return NMF_OK;
                });
                if (r != NMF_OK) return r;
                NMF_CUDA_TRY(launch_hpass_f32(a, true, s));  // Eq. 2 of the final iterate
            }
            NMF_CUDA_TRY(launch_stage_end(a, prm->normalize, chi2_hist, iters_done, k - 1, s));
        }
        NMF_CUDA_TRY(launch_copy_out(a.W, N, K, ldw, W, K, s));
        NMF_CUDA_TRY(launch_copy_out(a.Hb0, K, P, Pp, H, P, s));
        return NMF_OK;
    };
    if (ext) return emit(*ext);
    std::string key("fit");
    key_add(key, V);
    key_add(key, Wt);
    key_add(key, W);
    key_add(key, H);
    key_add(key, chi2_hist);
    key_add(key, iters_done);
    key_add(key, ws);
    key_add(key, *prm);
    key_add(key, ta.fault_t);
    key_add(key, ta.fault_ns);
    return run_emitted(key, s, emit);
}

// Target modelling (nmf_project_target); `ext` as for fit_impl.
nmf_status project_impl(const float *H, int32_t K, int64_t P, const float *T, const float *WtT, int64_t M, float *C,
                        int32_t iters, double tol, double eps, int32_t precision, int32_t polish_iters, void *ws,
                        size_t ws_bytes, void *stream, Emitter *ext) {
    const size_t need = nmf_project_workspace_bytes(M, P, K, precision);
    if (need == 0 || !H || !T || !WtT || !C || !ws) return NMF_EINVAL;
    if (iters < 0 || tol != 0.0 || !(eps > 0.0) || !(eps <= 1.0)) return NMF_EINVAL;
    if (polish_iters < 0 || (precision == NMF_FP32 && polish_iters != 0)) return NMF_EINVAL;
    if (ws_bytes < need || !aligned256(ws)) return NMF_EINVAL;
    const bool tcp = precision == NMF_BF16_SPLIT || precision == NMF_BF16_SPLIT_W32;
    const bool wt32 = precision == NMF_BF16_SPLIT_W32;
    const ProjLayout L = proj_layout(M, P, K, precision);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(ws);
    FitState *st = reinterpret_cast<FitState *>(base + L.state);
    const long long Pp = pad_p(P);
    const int ldw = ldw_of(K);

    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.V = reinterpret_cast<float *>(base + L.Tp);
    a.Wt = reinterpret_cast<float *>(base + L.WtTp);
    a.W = reinterpret_cast<float *>(base + L.Cp);
    a.Hb0 = a.Hb1 = reinterpret_cast<float *>(base + L.Hp);
    a.part = reinterpret_cast<float *>(base + L.part);
    a.num_const = reinterpret_cast<float *>(base + L.num);
    a.tickets = reinterpret_cast<unsigned *>(base + L.tickets);
    a.st = st;
    a.rows = M;
    a.P = P;
    a.Pp = Pp;
    a.k = K;
    a.ldw = ldw;
    a.eps = (float)eps;
    choose_splits(M, K, Pp, kMaxSplits, &a.nsplit, &a.split_len);

    uint8_t *img[8] = {};
    void *Wtb = nullptr;
    TcMaps maps;
    TcArgs ta;
    memset(&ta, 0, sizeof(ta));
    if (tcp) {
        for (int i = 0; i < 8; ++i) img[i] = reinterpret_cast<uint8_t *>(base + L.tc.img[i]);
        Wtb = base + L.tc.Wtb;
        if (!tc_make_maps(&maps, a.V, wt32 ? static_cast<const void *>(a.Wt) : Wtb, M, Pp, tc_kp(K), wt32))
            return cuda_fail(cudaErrorInvalidValue, "cuTensorMapEncodeTiled");
        ta.W = a.W;
        ta.part = reinterpret_cast<float *>(base + L.tc.part);
        ta.st = st;
        ta.wk_h = img[0];
        ta.wk_l = img[1];
        ta.hk_h[0] = ta.hk_h[1] = img[2];  // the fixed basis
        ta.hk_l[0] = ta.hk_l[1] = img[3];
        ta.rows = M;
        ta.Pp = Pp;
        ta.k = K;
        ta.kp = tc_kp(K);
        ta.packed = tc_packed(K) ? 1 : 0;
        ta.ldw = ldw;
        ta.eps = a.eps;
        ta.fault_t = -1;
        ta.wt32 = wt32 ? 1 : 0;
        choose_splits_tc(M, Pp, ta);
    }

    auto emit = [&](Emitter &em) -> nmf_status {
        const cudaStream_t s = em.s;
        NMF_CUDA_TRY(cudaMemsetAsync(base, 0, L.Tp, s));
        NMF_CUDA_TRY(launch_prologue_copy(T, M, P, P, const_cast<float *>(a.V), Pp, Pp, st, 1, s));
        NMF_CUDA_TRY(launch_prologue_copy(WtT, M, P, P, const_cast<float *>(a.Wt), Pp, Pp, st, 1, s));
        NMF_CUDA_TRY(launch_prologue_copy(H, K, P, P, a.Hb0, Pp, Pp, st, 1, s));
        NMF_CUDA_TRY(launch_prologue_copy(C, M, K, K, a.W, ldw, ldw, st, 1, s));
        NMF_CUDA_TRY(launch_stage_begin(st, s));
        int fp32_iters = iters;
        if (tcp) {
            if (!wt32) NMF_CUDA_TRY(tc_weights_bf16(WtT, M, P, Wtb, Pp, st, s));
            NMF_CUDA_TRY(cudaMemsetAsync(img[0], 0, L.tc.part - L.tc.img[0], s));
            NMF_CUDA_TRY(tc_images(a.W, M, K, ldw, false, img[0], img[1], ta.kp, ta.packed, s));
            NMF_CUDA_TRY(tc_images(a.Hb0, Pp, K, Pp, true, img[2], img[3], ta.kp, ta.packed, s));
            // the last `polish_iters` iterations run in FP32
            fp32_iters = polish_iters < iters ? polish_iters : iters;
            const int tc_iters = iters - fp32_iters;
            ta.t_end = tc_iters;
            const nmf_status r = em.loop(tc_iters, tc_iters, st, [&](cudaStream_t bs) -> nmf_status {
                NMF_CUDA_TRY(tc_wpass(maps, ta, bs));
                return NMF_OK;
            }, kTcUnroll);
            ta.t_end = 0;
            if (r != NMF_OK) return r;
            if (fp32_iters > 0) NMF_CUDA_TRY(launch_clear_stop(st, fp32_iters, s));
        }
        if (fp32_iters > 0) {
            // the constant numerator is formed by the first FP32 iteration
            NMF_CUDA_TRY(launch_wpass_f32(a, WP_PROJ_FIRST, s));
            const nmf_status r = em.loop(fp32_iters - 1, tcp ? -1 : iters, st, [&](cudaStream_t bs) -> nmf_status {
                NMF_CUDA_TRY(launch_wpass_f32(a, WP_PROJ_NEXT, bs));
                return NMF_OK;
            });
            if (r != NMF_OK) return r;
        }
        NMF_CUDA_TRY(launch_copy_out(a.W, M, K, ldw, C, K, s));
        return NMF_OK;
    };
    if (ext) return emit(*ext);
    std::string key("project");
    key_add(key, H);
    key_add(key, T);
    key_add(key, WtT);
    key_add(key, C);
    key_add(key, ws);
    key_add(key, M);
    key_add(key, P);
    key_add(key, K);
    key_add(key, iters);
    key_add(key, eps);
    key_add(key, precision);
    key_add(key, polish_iters);
    return run_emitted(key, s, emit);
}

// Workspace slice of one batched problem: its fit's workspace followed by,
// if it has science frames, its projection's (kept apart so that each keeps
// its own device status).  Returns 0 for an invalid descriptor; *fit_bytes
// receives the offset of the projection part.
size_t batched_slice_bytes(const nmf_problem &q, size_t *fit_bytes = nullptr) {
    if (!fit_params_ok(&q.prm) || q.reserved != 0 || q.M < 0 || q.proj_iters < 0) return 0;
    if (!q.V || !q.Wt || !q.W || !q.H || !q.chi2_hist || !q.iters_done) return 0;
    const size_t fb = align_up(fit_layout(q.prm.N, q.prm.P, q.prm.K, q.prm.precision).total);
    if (fit_bytes) *fit_bytes = fb;
    if (q.M == 0) return fb;
    if (!q.T || !q.WtT || !q.C || !q.R) return 0;
    const size_t pb = nmf_project_workspace_bytes(q.M, q.prm.P, q.prm.K, q.prm.precision);
    if (pb == 0) return 0;
    return fb + align_up(pb);
}

constexpr int kBranchStreams = 16;
cudaStream_t g_branch[64][kBranchStreams] = {};

}  // namespace

extern "C" {

int32_t nmf_version(void) { return 100; }

const char *nmf_last_cuda_error(void) { return t_last_error; }

uint64_t nmf_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int32_t nmf_w_schedule(int64_t rows, int64_t P, int32_t sms, int32_t max_blocks, int32_t *tile, int32_t *split,
                       int32_t *c0, int32_t *c1) {
    if (rows < 1 || P < 1 || sms < 1 || max_blocks < 0) return -1;
    if (max_blocks > 0 && (!tile || !split || !c0 || !c1)) return -1;
    TcArgs ta;
    memset(&ta, 0, sizeof(ta));
    if (!w_schedule(rows, pad_p(P), sms, ta)) return 0;
    if (ta.w_nblk > max_blocks) return -1;
    for (int b = 0; b < ta.w_nblk; ++b) {
        tile[b] = ta.w_tile[b];
        split[b] = ta.w_split[b];
        c0[b] = ta.w_c0[b];
        c1[b] = ta.w_c1[b];
    }
    return ta.w_nblk;
}

nmf_status nmf_debug_plant_timeout(int32_t t_fault, int64_t limit_ns) {
    if (t_fault < 0) {
        g_fault_t.store(-1);
        g_fault_ns.store(0);
        return NMF_OK;
    }
    if (limit_ns < 1000 || limit_ns > 100000000) return NMF_EINVAL;
    g_fault_ns.store(limit_ns);
    g_fault_t.store(t_fault);
    return NMF_OK;
}

const char *nmf_status_string(nmf_status s) {
    switch (s) {
        case NMF_OK: return "NMF_OK";
        case NMF_EINVAL: return "NMF_EINVAL: invalid argument";
        case NMF_ENOMEM: return "NMF_ENOMEM: device allocation failed";
        case NMF_ECUDA: return "NMF_ECUDA: CUDA runtime error";
        case NMF_ETIMEOUT: return "NMF_ETIMEOUT: device wait timed out";
        case NMF_ENOTCONV: return "NMF_ENOTCONV: not converged";
        case NMF_EDATA: return "NMF_EDATA: negative or non-finite input data";
        default: return "unknown nmf_status";
    }
}

size_t nmf_fit_workspace_bytes(const nmf_fit_params *prm) {
    if (!fit_params_ok(prm)) return 0;
    return fit_layout(prm->N, prm->P, prm->K, prm->precision).total;
}

nmf_status nmf_fit_basis(const float *V, const float *Wt, float *W, float *H, double *chi2_hist,
                         int32_t *iters_done, void *ws, size_t ws_bytes, const nmf_fit_params *prm,
                         void *stream) {
    return fit_impl(V, Wt, W, H, chi2_hist, iters_done, ws, ws_bytes, prm, stream, nullptr);
}

size_t nmf_project_workspace_bytes(int64_t M, int64_t P, int32_t K, int32_t precision) {
    if (M < 1 || P < 1 || K < 1 || K > kMaxK) return 0;
    if (precision != NMF_FP32 && precision != NMF_BF16_SPLIT && precision != NMF_BF16_SPLIT_W32) return 0;
    if (precision != NMF_FP32 && K > tc_max_k()) return 0;
    if (M >= (1LL << 31) || P >= (1LL << 31) - kPadP || (long long)K > P) return 0;
    return proj_layout(M, P, K, precision).total;
}

nmf_status nmf_project_target(const float *H, int32_t K, int64_t P, const float *T, const float *WtT,
                              int64_t M, float *C, int32_t iters, double tol, double eps, int32_t precision,
                              int32_t polish_iters, void *ws, size_t ws_bytes, void *stream) {
    return project_impl(H, K, P, T, WtT, M, C, iters, tol, eps, precision, polish_iters, ws, ws_bytes, stream,
                        nullptr);
}

nmf_status nmf_subtract(const float *T, const float *C, const float *H, int64_t M, int32_t K, int64_t P,
                        const float *factor, float *R, const int32_t *scatter_idx, int64_t img_pixels,
                        float *img, void *stream) {
    if (!T || !C || !H || !R || M < 0 || P < 0 || K < 1 || K > kMaxK) return NMF_EINVAL;
    if (M >= (1LL << 31) || P >= (1LL << 31)) return NMF_EINVAL;
    if ((scatter_idx == nullptr) != (img == nullptr)) return NMF_EINVAL;
    if (img && img_pixels < P) return NMF_EINVAL;
    NMF_CUDA_TRY(launch_subtract(T, C, H, M, K, P, factor, R, scatter_idx, img_pixels, img,
                                 static_cast<cudaStream_t>(stream)));
    return NMF_OK;
}

size_t nmf_batched_workspace_bytes(const nmf_problem *problems, int32_t count) {
    if (!problems || count < 1 || count > 1024) return 0;
    size_t total = 0;
    for (int b = 0; b < count; ++b) {
        const size_t sb = batched_slice_bytes(problems[b]);
        if (sb == 0) return 0;
        total += sb;
    }
    return total;
}

nmf_status nmf_fit_batched(const nmf_problem *problems, int32_t count, void *ws, size_t ws_bytes, void *stream) {
    const size_t need = nmf_batched_workspace_bytes(problems, count);
    if (need == 0 || !ws || ws_bytes < need || !aligned256(ws)) return NMF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    NMF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return NMF_ECUDA;
    {
        std::lock_guard<std::mutex> lock(g_graph_mu);
        for (int i = 0; i < kBranchStreams; ++i)
            if (!g_branch[dev][i]) NMF_CUDA_TRY(cudaStreamCreateWithFlags(&g_branch[dev][i], cudaStreamNonBlocking));
    }
    auto emit = [&](Emitter &em) -> nmf_status {
        // fork one branch per problem from the main stream, join them back
        cudaEvent_t fork;
        NMF_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        NMF_CUDA_TRY(cudaEventRecord(fork, em.s));
        // While recording, a reused branch stream would chain problem b + 16
        // behind problem b: every branch instead starts from the fork's
        // dependencies alone.
        std::vector<cudaGraphNode_t> fork_deps;
        if (em.graph) {
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            NMF_CUDA_TRY(cudaStreamGetCaptureInfo(em.s, &cs, nullptr, nullptr, &deps, nullptr, &nd));
            fork_deps.assign(deps, deps + nd);
        }
        char *base = static_cast<char *>(ws);
        nmf_status r = NMF_OK;
        for (int b = 0; b < count && r == NMF_OK; ++b) {
            const nmf_problem &q = problems[b];
            size_t fb = 0;
            const size_t sz = batched_slice_bytes(q, &fb);
            cudaStream_t sb = g_branch[dev][b % kBranchStreams];
            NMF_CUDA_TRY(cudaStreamWaitEvent(sb, fork, 0));
            if (em.graph)
                NMF_CUDA_TRY(cudaStreamUpdateCaptureDependencies(sb, fork_deps.data(), nullptr, fork_deps.size(),
                                                                 cudaStreamSetCaptureDependencies));
            Emitter eb = em;
            eb.s = sb;
            r = fit_impl(q.V, q.Wt, q.W, q.H, q.chi2_hist, q.iters_done, base, fb, &q.prm, sb, &eb);
            if (r == NMF_OK && q.M > 0) {
                r = project_impl(q.H, q.prm.K, q.prm.P, q.T, q.WtT, q.M, q.C, q.proj_iters, 0.0, q.prm.eps,
                                 q.prm.precision, q.prm.polish_iters, base + fb, sz - fb, sb, &eb);
                if (r == NMF_OK) {
                    const cudaError_t e = launch_subtract(q.T, q.C, q.H, q.M, q.prm.K, q.prm.P, nullptr, q.R, nullptr,
                                                          0, nullptr, sb);
                    if (e != cudaSuccess) r = cuda_fail(e, "launch_subtract");
                }
            }
            cudaEvent_t join;
            NMF_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
            NMF_CUDA_TRY(cudaEventRecord(join, sb));
            NMF_CUDA_TRY(cudaStreamWaitEvent(em.s, join, 0));
            cudaEventDestroy(join);
            base += sz;
        }
        cudaEventDestroy(fork);
        return r;
    };
    std::string key("batched");
    key_add(key, count);
    key.append(reinterpret_cast<const char *>(problems), sizeof(nmf_problem) * (size_t)count);
    key_add(key, ws);
    return run_emitted(key, s, emit);
}

nmf_status nmf_batched_status(const nmf_problem *problems, int32_t count, const void *ws, void *stream,
                              int32_t *status) {
    if (nmf_batched_workspace_bytes(problems, count) == 0 || !ws) return NMF_EINVAL;
    NMF_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    const char *base = static_cast<const char *>(ws);
    nmf_status first = NMF_OK;
    for (int b = 0; b < count; ++b) {
        size_t fb = 0;
        const size_t sz = batched_slice_bytes(problems[b], &fb);
        int st_fit = 0, st_proj = 0;
        NMF_CUDA_TRY(cudaMemcpy(&st_fit, base + offsetof(FitState, status), sizeof(int), cudaMemcpyDeviceToHost));
        if (problems[b].M > 0)
            NMF_CUDA_TRY(cudaMemcpy(&st_proj, base + fb + offsetof(FitState, status), sizeof(int),
                                    cudaMemcpyDeviceToHost));
        const int st = st_fit != 0 ? st_fit : st_proj;
        if (status) status[b] = st;
        if (first == NMF_OK && st != 0) first = static_cast<nmf_status>(st);
        base += sz;
    }
    return first;
}

nmf_status nmf_workspace_status(const void *ws, void *stream) {
    if (!ws) return NMF_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int status = 0;
    NMF_CUDA_TRY(cudaStreamSynchronize(s));
    NMF_CUDA_TRY(cudaMemcpy(&status, static_cast<const char *>(ws) + offsetof(FitState, status), sizeof(int),
                            cudaMemcpyDeviceToHost));
    return static_cast<nmf_status>(status);
}

// ---------------------------------------------------------------------------
// host-buffer pipeline with a process-wide device cache

namespace {
std::mutex g_cache_mu;
struct DevCache {
    void *ptr = nullptr;
    size_t bytes = 0;
    int device = -1;
    cudaStream_t stream = nullptr;
} g_cache;
}  // namespace

nmf_status nmf_reduce_host(const float *V, const float *Wt, const float *W0, const float *H0, const float *T,
                           const float *WtT, const float *C0, int64_t M, const nmf_fit_params *prm,
                           int32_t proj_iters, float *W, float *H, float *C, float *R, double *chi2_hist,
                           int32_t *iters_done) {
    if (!fit_params_ok(prm) || !V || !Wt || !W0 || !H0 || !W || !H || !chi2_hist || !iters_done) return NMF_EINVAL;
    if (M < 0 || proj_iters < 0) return NMF_EINVAL;
    if (M > 0 && (!T || !WtT || !C0 || !C || !R)) return NMF_EINVAL;
    const long long N = prm->N, P = prm->P;
    const int K = prm->K;
    const size_t fit_ws = nmf_fit_workspace_bytes(prm);
    const size_t proj_ws = M > 0 ? nmf_project_workspace_bytes(M, P, K, prm->precision) : 0;
    if (M > 0 && proj_ws == 0) return NMF_EINVAL;

    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t oV = take(sizeof(float) * N * P), oWt = take(sizeof(float) * N * P);
    const size_t oW = take(sizeof(float) * N * K), oH = take(sizeof(float) * K * P);
    const size_t oT = take(sizeof(float) * M * P), oWtT = take(sizeof(float) * M * P);
    const size_t oC = take(sizeof(float) * M * K), oR = take(sizeof(float) * M * P);
    const size_t oChi = take(sizeof(double) * K), oIt = take(sizeof(int32_t) * K);
    const size_t oWs = take(fit_ws > proj_ws ? fit_ws : proj_ws);
    const size_t total = off;

    std::lock_guard<std::mutex> lock(g_cache_mu);
    int dev = 0;
    NMF_CUDA_TRY(cudaGetDevice(&dev));
    if (g_cache.device != dev || g_cache.bytes < total) {
        if (g_cache.ptr) {
            cudaSetDevice(g_cache.device);
            cudaFree(g_cache.ptr);
            if (g_cache.stream) cudaStreamDestroy(g_cache.stream);
            cudaSetDevice(dev);
        }
        g_cache = DevCache();
        if (cudaMalloc(&g_cache.ptr, total) != cudaSuccess) {
            g_cache.ptr = nullptr;
            return NMF_ENOMEM;
        }
        NMF_CUDA_TRY(cudaStreamCreateWithFlags(&g_cache.stream, cudaStreamNonBlocking));
        g_cache.bytes = total;
        g_cache.device = dev;
    }
    char *d = static_cast<char *>(g_cache.ptr);
    cudaStream_t s = g_cache.stream;
    auto h2d = [&](size_t o, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(d + o, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    auto d2h = [&](void *dst, size_t o, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, d + o, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
    };
    NMF_CUDA_TRY(h2d(oV, V, sizeof(float) * N * P));
    NMF_CUDA_TRY(h2d(oWt, Wt, sizeof(float) * N * P));
    NMF_CUDA_TRY(h2d(oW, W0, sizeof(float) * N * K));
    NMF_CUDA_TRY(h2d(oH, H0, sizeof(float) * K * P));
    if (M > 0) {
        NMF_CUDA_TRY(h2d(oT, T, sizeof(float) * M * P));
        NMF_CUDA_TRY(h2d(oWtT, WtT, sizeof(float) * M * P));
        NMF_CUDA_TRY(h2d(oC, C0, sizeof(float) * M * K));
    }
    nmf_status st = nmf_fit_basis(reinterpret_cast<float *>(d + oV), reinterpret_cast<float *>(d + oWt),
                                  reinterpret_cast<float *>(d + oW), reinterpret_cast<float *>(d + oH),
                                  reinterpret_cast<double *>(d + oChi), reinterpret_cast<int32_t *>(d + oIt),
                                  d + oWs, fit_ws, prm, s);
    if (st != NMF_OK) return st;
    nmf_status fit_dev = nmf_workspace_status(d + oWs, s);
    if (fit_dev != NMF_OK) return fit_dev;
    if (M > 0) {
        st = nmf_project_target(reinterpret_cast<float *>(d + oH), K, P, reinterpret_cast<float *>(d + oT),
                                reinterpret_cast<float *>(d + oWtT), M, reinterpret_cast<float *>(d + oC),
                                proj_iters, 0.0, prm->eps, prm->precision, prm->polish_iters, d + oWs, proj_ws, s);
        if (st != NMF_OK) return st;
        st = nmf_subtract(reinterpret_cast<float *>(d + oT), reinterpret_cast<float *>(d + oC),
                          reinterpret_cast<float *>(d + oH), M, K, P, nullptr, reinterpret_cast<float *>(d + oR),
                          nullptr, 0, nullptr, s);
        if (st != NMF_OK) return st;
    }
    NMF_CUDA_TRY(d2h(W, oW, sizeof(float) * N * K));
    NMF_CUDA_TRY(d2h(H, oH, sizeof(float) * K * P));
    const int ks = prm->k_start;
    NMF_CUDA_TRY(d2h(chi2_hist + ks, oChi + sizeof(double) * ks, sizeof(double) * (K - ks)));
    NMF_CUDA_TRY(d2h(iters_done + ks, oIt + sizeof(int32_t) * ks, sizeof(int32_t) * (K - ks)));
    if (M > 0) {
        NMF_CUDA_TRY(d2h(C, oC, sizeof(float) * M * K));
        NMF_CUDA_TRY(d2h(R, oR, sizeof(float) * M * P));
    }
    NMF_CUDA_TRY(cudaStreamSynchronize(s));
    if (M > 0) {
        const nmf_status ps = nmf_workspace_status(d + oWs, s);
        if (ps != NMF_OK) return ps;
    }
    return NMF_OK;
}

}  // extern "C"
