// C ABI of libslag: context management and the per-call pipelines.
//
// slag_add_view (Method, "Semantic Embedding": Rasterization, Parameter
// Masking, the view's share of Aggregation):
//   project -> depth sort (stable, caller index breaks ties) -> gather records
//   in depth-rank order -> scan tile counts -> [host waits for this part only:
//   the pair count P and the error flags] -> emit (bin, rank) pairs -> stable
//   sort by bin -> bin ranges -> composite + mask + in-tile segment binning ->
//   consume the per-view (segment, weight) tables into the triple log.
//
// Views are pipelined over kSlots (6) sets of per-view buffers. The front half
// (projection through binning) runs on the slot's front stream, the back half
// (composite, consume) on its back stream, so that the next views' front halves
// and the start of the next composite fill the SMs that a composite's last,
// longest tiles leave idle. Back streams have the higher priority: a view
// whose binning is done composites before more front work is scheduled (the
// same step time at 1920x1080, 1-3% faster on smaller views). Consumes keep view order (they
// update the compensated per-Gaussian sums without atomics) through an event
// chain. Every entry point that reads results or reuses buffers first makes
// the caller's stream wait for all views in flight.
// slag_finalize (Aggregation, E_k formula): sort the log by
//   (block, column, Gaussian) -> distinct columns per block -> blocked
//   contraction with the stored segment embeddings -> divide by sum w.
// slag_query ("Query processing for inference"): cosine scores + top-k.
#include <errno.h>
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <initializer_list>
#include <mutex>
#include <set>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "slag_internal.cuh"

using namespace slag;

namespace slag {
namespace {
std::atomic<unsigned long long> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
// kernels of a replayed graph (k), and the undoing of the count of a capture (which launches nothing)
void note_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void unnote_launches(unsigned long long k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }
unsigned long long launches_now() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t set_max_smem(const void *fn, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({dev, fn})) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert({dev, fn});
    return e;
}
}  // namespace slag

namespace {

constexpr int kSlots = 6;   // views in flight
constexpr int64_t kSpillMin = 1 << 18;   // initial capacity of a slot's spill list
constexpr int kTotals = 5;  // device running totals (see slag_ctx::totals)

// A view's camera and first column in device memory: the kernels of a replayed graph read them
// there (everything else they use is fixed while the graph is valid).
struct ViewParams {
    CamParams cam;
    int32_t view_base;
    int32_t pad[3];
};

// Buffers of one view in flight. Stage A (front stream) and stage B (second
// front stream) fill them; the slot's back stream composites from them; stage A
// reuses them for the view kSlots later once ev_done has fired.
struct ViewSlot {
    // n-sized
    uint32_t *dkey[2] = {nullptr, nullptr}, *dval[2] = {nullptr, nullptr};
    float4 *rec_a = nullptr, *rec_b = nullptr;
    float *rec_t = nullptr;
    uint2 *rect = nullptr, *srect = nullptr;
    uint32_t *stouched = nullptr, *offsets = nullptr;
    HashEntry *hash = nullptr;             // per-view (segment, weight) slots; consume clears them
    // pair-, bin- and image-sized
    uint32_t *pkey[2] = {nullptr, nullptr}, *pval[2] = {nullptr, nullptr};
    int64_t p_cap = 0;
    uint2 *prect = nullptr;
    int64_t prect_cap = 0;
    uint2 *ranges = nullptr;
    int64_t ranges_cap = 0;
    uint32_t *tile_order = nullptr;
    int64_t order_cap = 0;
    int32_t *seg_buf = nullptr;            // the view's segment map (always copied: the caller's buffer
    int64_t seg_cap = 0;                   // is free once slag_add_view returns)
    WeightRecord *recs = nullptr;          // the composite's (Gaussian, segment, weight) sums
    int64_t rec_cap = 0;                   // records (a multiple of kRecChunk)
    unsigned long long *rec_chunks = nullptr;   // chunks reserved by the composite
    uint32_t *rec_fill = nullptr;          // per chunk: records written
    int64_t fill_cap = 0;
    uint64_t *spill_key = nullptr;         // the view's spill list: sums of Gaussians whose table
    float *spill_w = nullptr;              // slots are all taken (log keys and weights)
    int64_t spill_cap = 0;
    const uint32_t *list = nullptr;        // the pair list the view's composite reads
    ViewCounters *ctr = nullptr;           // device: stage A's counters
    ViewCounters *ctr_up = nullptr;        // device: the segment-id check of the view's upload
    struct Host {
        ViewCounters v;                    // stage A's counters
        ViewCounters vu;                   // the segment-id check
        unsigned long long totals[kTotals]; // the context's totals when stage A ended
    } *h = nullptr;                        // mapped pinned host copy
    Host *h_dev = nullptr;                 // its device alias (written by launch_copy_words)
    const uint32_t *sgid = nullptr;        // internal ids in depth order (stage A's output)
    CamParams cp{};                        // the view's camera
    int64_t view_base = 0;                 // its first column in the segment-embedding store
    cudaStream_t front = nullptr;          // the slot's stages A and B (low priority)
    SortScratch scratch;                   // their sorts and scans
    cudaEvent_t ev_front = nullptr;        // the front stream at a join
    cudaStream_t back = nullptr;
    cudaEvent_t ev_a = nullptr;            // stage A of the slot's view done
    cudaEvent_t ev_up = nullptr;           // the view's uploads and segment-id check done
    cudaEvent_t ev_bin = nullptr;          // stage B of the slot's view done
    cudaEvent_t ev_done = nullptr;         // back work of the slot's view done
    int64_t log_bound = 0;                 // triples the slot's view may append after stage A
    bool pending = false;                  // its back half is queued and its counters are not read
    bool count_at_settle = false;          // its view was sized on the device and is not counted
    ViewParams *vp_dev = nullptr;          // the view's camera and first column (replayed graphs)
    ViewParams *vp_host = nullptr;         // pinned staging of vp_dev (rewritten once the slot is settled)
    // the slot's captured graphs: stages A and B (front stream), composite + combine and consume
    // (back stream), with the kernels each holds; valid while gkey matches the slot's buffers
    cudaGraphExec_t gx_front = nullptr, gx_comp = nullptr, gx_cons = nullptr;
    unsigned long long gn_front = 0, gn_comp = 0, gn_cons = 0;
    uint64_t gkey_front = 0, gkey_back = 0;
};

}  // namespace

struct slag_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    int32_t D = 0;
    int32_t weight_mode = 0;
    int32_t precision = 0;
    int32_t opt_flags = 0;                   // SLAG_FLAG_*
    int64_t chunk_gaussians = 1 << 20;       // rows per chunk of the out-of-core contraction
    int64_t force_pair_cap = 0;              // checked builds: pair capacity forced on the next views
    std::string err;

    // Gaussians, internal (Morton) order
    float4 *mean_op = nullptr, *cov_a = nullptr;
    float2 *cov_b = nullptr;
    float *log2_op = nullptr;                // log2 of each opacity (float64, rounded)
    uint32_t *orig_of_int = nullptr, *int_of_orig = nullptr;

    // views in flight
    ViewSlot slot[kSlots];
    cudaEvent_t ev_in = nullptr;             // caller's stream at the start of a call
    cudaStream_t up = nullptr;               // uploads of a view's inputs and their check
    cudaEvent_t ev_consumed = nullptr;       // the last enqueued consume
    int64_t views_enqueued = 0;              // views accepted since create / reset (slot = count % kSlots)
    bool deferred = false;                   // the last accepted view's stage B and back half wait
                                             // for the next call
    int64_t est_P = 0, est_P_tiles = 0;      // the largest pair counts seen (device-sized views)
    int64_t log_fill_seen = 0;               // the triple log's fill level, as last read
    bool graphs = true;                      // device-sized views replay captured graphs (slag_set_graphs)
    float *s_hi = nullptr, *s_lo = nullptr, *s_ovf = nullptr;
    float *dbg_T = nullptr, *dbg_wsum = nullptr;
    int32_t *dbg_count = nullptr;
    int64_t dbg_cap = 0;

    unsigned long long *totals = nullptr;    // device: [0] triples in the log, [1] contributions,
                                             // [2] low word: log overflow flag, [3] evaluations,
                                             // [4] executed lane-pixel evaluations
    unsigned long long *log_count = nullptr; // = totals
    unsigned long long *contrib = nullptr;   // = totals + 1
    struct HostCounters {
        ViewCounters v;                      // validation at create, the last view at finalize
        unsigned long long totals[kTotals];
        unsigned long long touched;
        unsigned long long n_q;              // query candidates (touched rows)
        uint32_t tc_err;
        uint32_t pad;
    } *hc = nullptr;                         // mapped pinned host
    HostCounters *hc_dev = nullptr;          // its device alias (written by launch_copy_words)
    unsigned char *qstage = nullptr, *qstage_dev = nullptr;   // mapped staging of host query results
    int64_t qstage_cap = 0;
    uint32_t *tc_err = nullptr;              // device: a tensor-core kernel gave up waiting

    // triple log + finalize scratch
    uint64_t *log_key = nullptr, *log_key_alt = nullptr;
    float *log_w = nullptr, *log_w_alt = nullptr;
    int64_t log_cap = 0;
    uint32_t *flags = nullptr, *uidx = nullptr, *ucol = nullptr, *ustart = nullptr;
    int64_t fin_cap = 0;
    uint32_t *bstart = nullptr, *bend = nullptr;
    bool log_overflowed = false;

    // stored segment embeddings (columns x D)
    float *table = nullptr;
    int64_t table_rows = 0, table_cap = 0;

    // outputs
    float *E = nullptr, *inv_norm = nullptr, *wsum = nullptr;
    unsigned long long *touched = nullptr;
    uint32_t *qrows = nullptr, *qflags = nullptr, *qpos = nullptr;   // query candidates: touched rows of E
    unsigned long long *d_nq = nullptr;
    unsigned long long *d_thr = nullptr;     // threshold query: number of rows at or above it
    int64_t *thr_ids = nullptr;              // threshold query: ids staged for host outputs
    int64_t thr_cap = 0;
    int64_t n_q = 0;
    bool finalized = false;

    // latent form: autoencoder parameters, codes of the stored segment embeddings, scratch
    float *lat_params = nullptr;
    float *lin_params = nullptr;             // linear code: U (D x 32) then mu (D), and -mu U
    float *lin_enc_bias = nullptr;
    float *ztable = nullptr;                 // columns x kLatent
    int64_t ztable_cap = 0;
    float *lat_hidden = nullptr;             // rows x kLatentHidden
    int64_t lat_hidden_cap = 0;
    float *lat_Z = nullptr, *lat_Y = nullptr;   // finalize: mean codes (n x kLatent), decoded rows
    int64_t lat_Z_cap = 0, lat_Y_cap = 0;

    // queries: split counts chosen by the autotuner per (batch, candidates) shape, and the
    // CUDA graph of the last device-side query (replayed while its buffers and shape repeat)
    std::map<std::pair<int32_t, int64_t>, int32_t> qsplits;
    bool autotune = true;
    cudaStream_t qstream = nullptr;
    cudaEvent_t qev_in = nullptr, qev_out = nullptr;
    // Asynchronous outputs: E and sum w are double-buffered; buf[cur] holds the latest result
    // (ctx->E and ctx->wsum point into it). A finalize moves to the other buffer while
    // copies of the current one are still queued on cstream; ev_copy[b] completes once the
    // copies from buffer b are done.
    float *E_buf[2] = {nullptr, nullptr}, *wsum_buf[2] = {nullptr, nullptr};
    int cur = 0;
    bool copy_pending[2] = {false, false};
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_fin = nullptr, ev_copy[2] = {nullptr, nullptr};
    // The embeddings' download of an asynchronous finalize, still to be issued: a piece after
    // each later view's host sync (a continuous download of the whole matrix would hold the
    // PCIe link and delay every view's sync), the rest at the next finalize or wait.
    const char *pend_src = nullptr;
    char *pend_dst = nullptr;
    size_t pend_left = 0, pend_off = 0, pend_piece = 0;
    cudaMemcpyKind pend_kind = cudaMemcpyDeviceToHost;
    int pend_buf = 0;
    cudaGraphExec_t qgraph = nullptr;
    unsigned long long qgraph_launches = 0;  // kernels in the graph (counted at each replay)
    struct QKey {
        const float *Q;
        int64_t *ids;
        float *scores;
        int32_t *cnt;
        int32_t B, k, splits;
        int64_t nq;
        uint64_t gen;
        bool operator==(const QKey &o) const {
            return Q == o.Q && ids == o.ids && scores == o.scores && cnt == o.cnt && B == o.B && k == o.k &&
                   splits == o.splits && nq == o.nq && gen == o.gen;
        }
    } qkey{};
    uint64_t qgen = 0;                       // bumped by every finalize (candidate list changes)
    float *qbuf = nullptr;
    int64_t qbuf_cap = 0;
    // tensor-core query operands: TF32 hi/lo planes of the candidate rows (rebuilt when qgen moves)
    // and of the current query batch, with the candidates' inverse norms
    float *ehl = nullptr, *qinv = nullptr, *qhl = nullptr;
    int64_t ehl_cap = 0, qinv_cap = 0, qhl_cap = 0;
    uint64_t ehl_gen = ~0ull;
    float *cand_s = nullptr;
    uint32_t *cand_i = nullptr;
    int64_t cand_cap = 0;
    int64_t *qids = nullptr;
    float *qscores = nullptr;
    int32_t *qcount = nullptr;
    int64_t qout_cap = 0;

    SortScratch scratch;                     // finalize, queries, diagnostics (the caller's stream)
    slag_stats stats{};

    // per-stage timing
    struct Span {
        int stage;
        cudaEvent_t a, b;
    };
    uint32_t prof_mask = 0;                                // stages timed (bit s = stage s)
    bool span_open = false;                                // spans.back() waits for its end event
    std::vector<Span> spans;
    std::vector<cudaEvent_t> event_pool;
    slag_profile prof{};
    cudaEvent_t prof_base = nullptr;                       // origin of the span intervals
    std::vector<std::pair<float, float>> busy[SLAG_STAGE_COUNT];
};

namespace {

slag_status fail(slag_ctx *c, slag_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? SLAG_ERR_OOM : SLAG_ERR_CUDA,       \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
        }                                                                                          \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * (size_t)count);
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree((void *)p);
    p = nullptr;
}

// Grows a device buffer to at least `need` elements (x1.5 headroom); keeps
// the first `keep` elements when asked.
template <typename T>
cudaError_t grow(T *&p, int64_t &cap, int64_t need, cudaStream_t st, int64_t keep = 0) {
    if (need <= cap) return cudaSuccess;
    int64_t nc = need + need / 2 + 1024;
    T *q = nullptr;
    cudaError_t e = dalloc(&q, nc);
    if (e != cudaSuccess) return e;
    if (keep > 0 && p) {
        e = cudaMemcpyAsync(q, p, sizeof(T) * (size_t)keep, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { cudaFree(q); return e; }
        cudaStreamSynchronize(st);
    }
    if (p) cudaFree(p);
    p = q;
    cap = nc;
    return cudaSuccess;
}

bool finite_camera(const slag_camera *c) {
    const float *f = &c->fx;
    for (int i = 0; i < 4; ++i)
        if (!std::isfinite(f[i])) return false;
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(c->R[i])) return false;
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(c->t[i])) return false;
    return std::isfinite(c->near_z) && std::isfinite(c->far_z);
}

slag_status check_camera(slag_ctx *ctx, const slag_camera *cam) {
    if (!cam) return fail(ctx, SLAG_ERR_INVALID_ARG, "camera is NULL");
    if (!finite_camera(cam)) return fail(ctx, SLAG_ERR_INVALID_ARG, "camera has a non-finite value");
    if (cam->width < 1 || cam->height < 1 || cam->width > 65535 || cam->height > 65535)
        return fail(ctx, SLAG_ERR_INVALID_ARG, "camera width/height outside 1..65535");
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(ctx, SLAG_ERR_INVALID_ARG, "camera fx/fy must be > 0");
    if (!(cam->near_z > 0.f) || !(cam->far_z > cam->near_z))
        return fail(ctx, SLAG_ERR_INVALID_ARG, "camera needs 0 < near_z < far_z");
    return SLAG_OK;
}

CamParams cam_params(const slag_camera *c) {
    CamParams p;
    p.fx = c->fx; p.fy = c->fy; p.cx = c->cx; p.cy = c->cy;
    p.width = c->width; p.height = c->height;
    memcpy(p.R, c->R, sizeof(p.R));
    memcpy(p.t, c->t, sizeof(p.t));
    p.near_z = c->near_z; p.far_z = c->far_z;
    p.tiles_x = (c->width + kTile - 1) / kTile;
    p.tiles_y = (c->height + kTile - 1) / kTile;
    return p;
}

cudaEvent_t take_event(slag_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Opens a timing span of `stage` in stream `st` (no-op when profiling is off).
// Spans of views in flight overlap, so stage totals add device time per
// stream, not wall time.
void span_begin(slag_ctx *ctx, int stage, cudaStream_t st) {
    if (!((ctx->prof_mask >> stage) & 1u)) return;
    slag_ctx::Span sp{stage, take_event(ctx), take_event(ctx)};
    cudaEventRecord(sp.a, st);
    ctx->spans.push_back(sp);
    ctx->span_open = true;
}

void span_end(slag_ctx *ctx, cudaStream_t st) {
    if (!ctx->span_open) return;
    cudaEventRecord(ctx->spans.back().b, st);
    ctx->span_open = false;
}

// Spans left open between resolutions. Reading a span's times costs several
// driver calls on the host, and the views' host syncs are on the critical path,
// so routine calls resolve only once this many spans are pending; the totals
// resolve everything.
constexpr size_t kSpanBacklog = 4096;

// Adds every finished span to the totals; spans still in flight stay.
void spans_resolve(slag_ctx *ctx, bool all = true) {
    if (!all && ctx->spans.size() < kSpanBacklog) return;
    size_t keep = 0;
    for (size_t i = 0; i < ctx->spans.size(); ++i) {
        auto &sp = ctx->spans[i];
        if (cudaEventQuery(sp.b) != cudaSuccess) {
            ctx->spans[keep++] = sp;
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) {
            ctx->prof.ms[sp.stage] += ms;
            ctx->prof.spans[sp.stage] += 1;
            float t0 = 0.f, t1 = 0.f;
            if (ctx->prof_base && cudaEventElapsedTime(&t0, ctx->prof_base, sp.a) == cudaSuccess &&
                cudaEventElapsedTime(&t1, ctx->prof_base, sp.b) == cudaSuccess)
                ctx->busy[sp.stage].push_back({t0, t1});
        }
        ctx->event_pool.push_back(sp.a);
        ctx->event_pool.push_back(sp.b);
    }
    ctx->spans.resize(keep);
    (void)cudaGetLastError();   // clears cudaErrorNotReady left by the queries
}

// A tensor-core kernel gave up a bounded wait (the error word is set): clears the word, so that
// the context stays usable, and returns TIMEOUT with msg.
slag_status timeout_reported(slag_ctx *ctx, const char *msg) {
    ctx->hc->tc_err = 0;
    cudaMemsetAsync(ctx->tc_err, 0, sizeof(uint32_t), ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return fail(ctx, SLAG_ERR_TIMEOUT, msg);
}

// Checked builds: reads and clears the bounds-check words after the stream has synchronised;
// a failed check is reported as CAPACITY, naming the stages.
slag_status checks_reported(slag_ctx *ctx) {
    if (!kChecked) return SLAG_OK;
    cudaStream_t st = ctx->stream;
    const uint32_t v = checks_take_bin(st) | checks_take_sort(st) | checks_take_composite(st) |
                       checks_take_aggregate(st);
    if (!v) return SLAG_OK;
    std::string m = "bounds check failed in:";
    if (v & kCheckEmit) m += " pair emission";
    if (v & kCheckSort) m += " sort scatter";
    if (v & kCheckComposite) m += " compositing";
    if (v & kCheckAggregate) m += " aggregation";
    return fail(ctx, SLAG_ERR_CAPACITY, m);
}

// The caller's stream waits for every view in flight and for both front streams.
cudaError_t join_views(slag_ctx *ctx) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) {
        ViewSlot &vs = ctx->slot[i];
        e = cudaEventRecord(vs.ev_front, vs.front);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, vs.ev_front, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, vs.ev_done, 0);
    }
    return e;
}

// Host waits for every internal stream of the views (the caller's stream is not waited for).
cudaError_t drain_views(slag_ctx *ctx) {
    cudaError_t e = cudaStreamSynchronize(ctx->up);
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) e = cudaStreamSynchronize(ctx->slot[i].front);
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) e = cudaStreamSynchronize(ctx->slot[i].back);
    return e;
}

int ceil_log2(uint64_t v) {
    int b = 0;
    while ((1ull << b) < v) ++b;
    return b;
}

// Projection through the bin ranges of one view, into slot `vs` on stream
// `st`: leaves the depth-sorted records, the bin-sorted pair list and ranges
// in the slot; returns the pair count in *P_out and the list buffer in
// *list_out. The host waits for `st` once (pair count, error flags) and
// copies the log's fill level of that moment into vs.h->totals.
// Stage A of a view: projection, depth sort, depth-rank gather and the scan of the
// per-Gaussian tile counts (Method: the rasterizer's per-view preprocessing). Reads neither
// the segment map nor the table. The counters and the log's fill level are copied to the
// slot's mapped host struct; the host reads them once the stage has ended.
slag_status stage_a(slag_ctx *ctx, ViewSlot &vs, cudaStream_t st, const CamParams &cp, int shift,
                    SortScratch &scr, const CamParams *cam_dev = nullptr) {
    const int64_t n = ctx->n;
    CK(cudaMemsetAsync(vs.ctr, 0, sizeof(ViewCounters), st));
    span_begin(ctx, SLAG_STAGE_PROJECT, st);
    launch_project(cp, ctx->mean_op, ctx->log2_op, ctx->cov_a, ctx->cov_b, n, ctx->orig_of_int, vs.dkey[0], vs.dval[0],
                   vs.rec_a, vs.rec_b, vs.rec_t, vs.rect, vs.ctr, st, cam_dev);
    int shifts[8], widths[8];
    const int np = digit_passes(0, 32, shifts, widths, n);
    const bool alt = radix_sort_u32(vs.dkey[0], vs.dkey[1], vs.dval[0], vs.dval[1], n, shifts, widths, np,
                                    scr, st);
    vs.sgid = vs.dval[alt ? 1 : 0];
    launch_gather_sorted(vs.sgid, n, vs.ctr, vs.rect, vs.srect, vs.stouched, shift, st);
    exclusive_scan_u32(vs.stouched, vs.offsets, n, &vs.ctr->P, scr, st);
    span_end(ctx, st);
    launch_copy_words(vs.ctr, &vs.h_dev->v, sizeof(ViewCounters), st);
    launch_copy_words(ctx->totals, vs.h_dev->totals, kTotals * sizeof(unsigned long long), st);
    CK(cudaGetLastError());
    return SLAG_OK;
}

// Stage B, once stage A's counters are on the host: pair emission, the stable sort of the
// pairs by bin (tile or super-tile), bin ranges and the tile order; sorts with `scr`.
slag_status stage_b(slag_ctx *ctx, ViewSlot &vs, cudaStream_t st, const CamParams &cp, int shift,
                    SortScratch &scr, int64_t *P_out, uint32_t **list_out) {
    int64_t P = (int64_t)vs.h->v.P;         // pairs at the binning granularity
    // checked builds only: a capacity forced below P; the emission's checks refuse the pairs
    // beyond it and the later stages see only the first pairs
    if (kChecked && ctx->force_pair_cap > 0 && ctx->force_pair_cap < P) P = ctx->force_pair_cap;
    if (P > 0x7fffffffLL || vs.h->v.P_tiles > 0x7fffffffULL)
        return fail(ctx, SLAG_ERR_CAPACITY, "more than 2^31-1 Gaussian-tile pairs in one view");
    if (P > vs.p_cap) {
        int64_t cap = vs.p_cap;
        for (int b = 0; b < 2; ++b) {
            int64_t c1 = cap, c2 = cap;
            CK(grow(vs.pkey[b], c1, P, st));
            CK(grow(vs.pval[b], c2, P, st));
            vs.p_cap = c1;
        }
    }
    CK(scratch_reserve(scr, vs.p_cap));
    const int bins_x = ((cp.tiles_x - 1) >> shift) + 1, bins_y = ((cp.tiles_y - 1) >> shift) + 1;
    const int64_t bins = (int64_t)bins_x * bins_y;
    const int64_t tiles = (int64_t)cp.tiles_x * cp.tiles_y;
    CK(grow(vs.ranges, vs.ranges_cap, bins, st));
    const uint32_t nv = vs.h->v.n_visible;
    span_begin(ctx, SLAG_STAGE_BIN, st);
    // the tile rectangle of each sorted pair (the composite's per-tile filter), for super-tile bins
    if (shift > 0) CK(grow(vs.prect, vs.prect_cap, P, st));
    uint32_t *list = vs.pval[0];
    if (P == 0) {
        CK(cudaMemsetAsync(vs.ranges, 0, sizeof(uint2) * (size_t)bins, st));
    } else if (!bin_sort_fused(vs.srect, vs.offsets, vs.stouched, nv, &vs.ctr->n_visible, &vs.ctr->P, P,
                               P < (int64_t)vs.h->v.P ? 1 : 0, &vs.ctr->overflow, shift, bins_x, (int)bins,
                               vs.sgid, list, shift > 0 ? vs.prect : nullptr, vs.ranges, scr, st)) {
        // more than 2048 bins: emit the pairs, then a radix sort of them by bin
        launch_emit(vs.srect, vs.offsets, nv, shift, bins_x, P, vs.pkey[0], vs.pval[0], st);
        int shifts[8], widths[8];
        const int np = digit_passes(0, ceil_log2((uint64_t)bins), shifts, widths, P);
        CK(cudaMemsetAsync(vs.ranges, 0, sizeof(uint2) * (size_t)bins, st));
        const bool alt = radix_sort_u32(vs.pkey[0], vs.pkey[1], vs.pval[0], vs.pval[1], P, shifts, widths, np, scr,
                                        st, nullptr, 0, shift > 0 ? vs.srect : nullptr,
                                        shift > 0 ? vs.prect : nullptr, vs.sgid);
        launch_ranges(vs.pkey[alt ? 1 : 0], P, vs.ranges, st);
        list = vs.pval[alt ? 1 : 0];
    }
    CK(grow(vs.tile_order, vs.order_cap, tiles, st));
    launch_tile_order(vs.ranges, cp.tiles_x, cp.tiles_y, shift, vs.tile_order, st);
    span_end(ctx, st);
    CK(cudaGetLastError());
    *P_out = P;
    *list_out = list;
    return SLAG_OK;
}

// Both stages in one stream with a host sync between them (the diagnostic entry points).
slag_status bin_view(slag_ctx *ctx, ViewSlot &vs, cudaStream_t st, const CamParams &cp, int64_t *P_out,
                     uint32_t **list_out, int shift) {
    slag_status s = stage_a(ctx, vs, st, cp, shift, ctx->scratch);
    if (s != SLAG_OK) return s;
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    spans_resolve(ctx, false);
    return stage_b(ctx, vs, st, cp, shift, ctx->scratch, P_out, list_out);
}

cudaError_t slot_alloc(ViewSlot &vs, int64_t n) {
    cudaError_t e = cudaSuccess;
#define SA(call) do { if (e == cudaSuccess) e = (call); } while (0)
    for (int b = 0; b < 2; ++b) { SA(dalloc(&vs.dkey[b], n)); SA(dalloc(&vs.dval[b], n)); }
    SA(dalloc(&vs.rec_a, n)); SA(dalloc(&vs.rec_b, n)); SA(dalloc(&vs.rec_t, n));
    SA(dalloc(&vs.rect, n)); SA(dalloc(&vs.srect, n));
    SA(dalloc(&vs.stouched, n)); SA(dalloc(&vs.offsets, n));
    SA(dalloc(&vs.hash, n));
    SA(dalloc(&vs.ctr, 1));
    SA(dalloc(&vs.ctr_up, 1));
    SA(dalloc(&vs.rec_chunks, 1));
    SA(cudaHostAlloc((void **)&vs.h, sizeof(ViewSlot::Host), cudaHostAllocMapped));
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&vs.h_dev, vs.h, 0);
    int lo = 0, hi = 0;
    SA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    SA(cudaStreamCreateWithPriority(&vs.back, cudaStreamNonBlocking, hi));
    SA(cudaStreamCreateWithPriority(&vs.front, cudaStreamNonBlocking, lo));
    SA(cudaEventCreateWithFlags(&vs.ev_front, cudaEventDisableTiming));
    SA(scratch_reserve(vs.scratch, n));
    SA(dalloc(&vs.vp_dev, 1));
    SA(cudaHostAlloc((void **)&vs.vp_host, sizeof(ViewParams), cudaHostAllocDefault));
    SA(cudaEventCreateWithFlags(&vs.ev_a, cudaEventDisableTiming));
    SA(cudaEventCreateWithFlags(&vs.ev_up, cudaEventDisableTiming));
    SA(cudaEventCreateWithFlags(&vs.ev_bin, cudaEventDisableTiming));
    SA(cudaEventCreateWithFlags(&vs.ev_done, cudaEventDisableTiming));
#undef SA
    if (e == cudaSuccess && vs.h) memset(vs.h, 0, sizeof(ViewSlot::Host));
    return e;
}

void slot_free(ViewSlot &vs) {
    for (int b = 0; b < 2; ++b) { dfree(vs.dkey[b]); dfree(vs.dval[b]); dfree(vs.pkey[b]); dfree(vs.pval[b]); }
    dfree(vs.rec_a); dfree(vs.rec_b); dfree(vs.rec_t); dfree(vs.rect); dfree(vs.srect);
    dfree(vs.stouched); dfree(vs.offsets); dfree(vs.hash);
    dfree(vs.prect); dfree(vs.ranges); dfree(vs.tile_order); dfree(vs.seg_buf); dfree(vs.ctr);
    dfree(vs.ctr_up); dfree(vs.recs); dfree(vs.rec_chunks); dfree(vs.rec_fill); dfree(vs.spill_key); dfree(vs.spill_w);
    if (vs.h) cudaFreeHost(vs.h);
    vs.h = nullptr;
    if (vs.back) cudaStreamDestroy(vs.back);
    if (vs.front) cudaStreamDestroy(vs.front);
    vs.front = nullptr;
    scratch_free(vs.scratch);
    dfree(vs.vp_dev);
    if (vs.vp_host) cudaFreeHost(vs.vp_host);
    vs.vp_host = nullptr;
    for (cudaGraphExec_t *g : {&vs.gx_front, &vs.gx_comp, &vs.gx_cons}) {
        if (*g) cudaGraphExecDestroy(*g);
        *g = nullptr;
    }
    for (cudaEvent_t *e : {&vs.ev_a, &vs.ev_up, &vs.ev_bin, &vs.ev_done, &vs.ev_front}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
    }
    vs.back = nullptr;
}

// issues pieces of a pending asynchronous download (defined with the finalize helpers)
slag_status issue_pending(slag_ctx *ctx, int pieces);

}  // namespace

extern "C" {

slag_status slag_create(const slag_gaussians *g, const slag_options *opt, slag_ctx **out) {
    if (!out) return SLAG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!g || !opt) return SLAG_ERR_INVALID_ARG;
    if (g->n < 1 || g->n >= (1LL << 31)) return SLAG_ERR_INVALID_ARG;
    if (!g->means || !g->scales || !g->quats || !g->opacities) return SLAG_ERR_INVALID_ARG;
    if (opt->dim < 128 || opt->dim > 4096 || opt->dim % 128 != 0) return SLAG_ERR_INVALID_ARG;
    if (opt->precision != SLAG_PREC_FP32 && opt->precision != SLAG_PREC_BF16 && opt->precision != SLAG_PREC_LATENT32 &&
        opt->precision != SLAG_PREC_LINEAR32)
        return SLAG_ERR_INVALID_ARG;
    if (opt->weight_mode != SLAG_WEIGHT_ALPHA_T && opt->weight_mode != SLAG_WEIGHT_KERNEL) return SLAG_ERR_INVALID_ARG;
    if ((opt->flags & ~SLAG_FLAG_EMBEDDINGS_ON_HOST) != 0) return SLAG_ERR_INVALID_ARG;

    slag_ctx *ctx = new (std::nothrow) slag_ctx();
    if (!ctx) return SLAG_ERR_OOM;
    float *dm = nullptr, *ds = nullptr, *dq = nullptr, *dop = nullptr;
    uint32_t *bb = nullptr;
    auto free_inputs = [&]() { dfree(dm); dfree(ds); dfree(dq); dfree(dop); dfree(bb); };
    auto bail = [&](slag_status s) {
        slag_destroy(ctx);   // first: it waits for the stream, where copies from g may be queued
        free_inputs();
        return s;
    };
    const int64_t n = g->n;
    ctx->n = n;
    ctx->D = opt->dim;
    ctx->weight_mode = opt->weight_mode;
    ctx->precision = opt->precision;
    ctx->opt_flags = opt->flags;
    ctx->stream = (cudaStream_t)opt->cuda_stream;
    if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(SLAG_ERR_CUDA);
    cudaStream_t st = ctx->stream;

#define CA(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess)                                        \
            return bail(e_ == cudaErrorMemoryAllocation ? SLAG_ERR_OOM : SLAG_ERR_CUDA); \
    } while (0)

    // inputs on the device
    const float *im = g->means, *is = g->scales, *iq = g->quats, *io = g->opacities;
    if (!g->on_device) {
        CA(dalloc(&dm, 3 * n)); CA(dalloc(&ds, 3 * n)); CA(dalloc(&dq, 4 * n)); CA(dalloc(&dop, n));
        CA(cudaMemcpyAsync(dm, g->means, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
        CA(cudaMemcpyAsync(ds, g->scales, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
        CA(cudaMemcpyAsync(dq, g->quats, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, st));
        CA(cudaMemcpyAsync(dop, g->opacities, sizeof(float) * n, cudaMemcpyHostToDevice, st));
        im = dm; is = ds; iq = dq; io = dop;
    }
    CA(cudaHostAlloc((void **)&ctx->hc, sizeof(slag_ctx::HostCounters), cudaHostAllocMapped));
    CA(cudaHostGetDevicePointer((void **)&ctx->hc_dev, ctx->hc, 0));
    for (int i = 0; i < kSlots; ++i) CA(slot_alloc(ctx->slot[i], n));
    {
        int lo = 0, hi = 0;
        CA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        // the segment-id check runs here and slag_add_view waits for it: it must not queue
        // behind the composites' CTAs
        CA(cudaStreamCreateWithPriority(&ctx->up, cudaStreamNonBlocking, hi));
    }
    CA(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
    CA(cudaEventCreateWithFlags(&ctx->ev_consumed, cudaEventDisableTiming));
    CA(cudaStreamCreateWithFlags(&ctx->qstream, cudaStreamNonBlocking));
    CA(cudaEventCreateWithFlags(&ctx->qev_in, cudaEventDisableTiming));
    CA(cudaEventCreateWithFlags(&ctx->qev_out, cudaEventDisableTiming));
    CA(dalloc(&ctx->totals, kTotals));
    ctx->log_count = ctx->totals;
    ctx->contrib = ctx->totals + 1;
    CA(dalloc(&ctx->touched, 1));
    CA(dalloc(&ctx->tc_err, 1));
    ViewCounters *vctr = ctx->slot[0].ctr;
    CA(cudaMemsetAsync(ctx->tc_err, 0, sizeof(uint32_t), st));
    CA(cudaMemsetAsync(vctr, 0, sizeof(ViewCounters), st));
    CA(cudaMemsetAsync(ctx->totals, 0, kTotals * sizeof(unsigned long long), st));
    CA(scratch_reserve(ctx->scratch, n));

    // validation
    launch_check_gaussians(im, is, iq, io, n, &vctr->bad_seg, st);
    CA(cudaMemcpyAsync(&ctx->hc->v, vctr, sizeof(ViewCounters), cudaMemcpyDeviceToHost, st));
    CA(cudaStreamSynchronize(st));
    CA(cudaGetLastError());
    if (ctx->hc->v.bad_seg) return bail(SLAG_ERR_INVALID_ARG);

    // Morton order
    CA(dalloc(&ctx->orig_of_int, n)); CA(dalloc(&ctx->int_of_orig, n));
    CA(dalloc(&bb, 6));
    ViewSlot &s0 = ctx->slot[0];
    launch_bbox(im, n, bb, st);
    launch_morton(im, n, bb, s0.dkey[0], s0.dval[0], st);
    int shifts[8], widths[8];
    int np = digit_passes(0, 30, shifts, widths, n);
    bool alt = radix_sort_u32(s0.dkey[0], s0.dkey[1], s0.dval[0], s0.dval[1], n, shifts, widths, np,
                              ctx->scratch, st);
    CA(cudaMemcpyAsync(ctx->orig_of_int, s0.dval[alt ? 1 : 0], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    CA(dalloc(&ctx->mean_op, n)); CA(dalloc(&ctx->cov_a, n)); CA(dalloc(&ctx->cov_b, n));
    CA(dalloc(&ctx->log2_op, n));
    launch_pack_gaussians(im, is, iq, io, n, ctx->orig_of_int, ctx->mean_op, ctx->cov_a, ctx->cov_b,
                          ctx->int_of_orig, ctx->log2_op, st);

    // accumulators and outputs
    CA(dalloc(&ctx->s_hi, n)); CA(dalloc(&ctx->s_lo, n)); CA(dalloc(&ctx->s_ovf, n));
    if (!(ctx->opt_flags & SLAG_FLAG_EMBEDDINGS_ON_HOST)) CA(dalloc(&ctx->E, n * (int64_t)ctx->D));
    CA(dalloc(&ctx->inv_norm, n)); CA(dalloc(&ctx->wsum, n));
    ctx->E_buf[0] = ctx->E;
    ctx->wsum_buf[0] = ctx->wsum;
    CA(dalloc(&ctx->qrows, n)); CA(dalloc(&ctx->qflags, n)); CA(dalloc(&ctx->qpos, n)); CA(dalloc(&ctx->d_nq, 1));
    CA(dalloc(&ctx->bstart, (n + kBlockG - 1) / kBlockG)); CA(dalloc(&ctx->bend, (n + kBlockG - 1) / kBlockG));
    for (int i = 0; i < kSlots; ++i) launch_hash_init(ctx->slot[i].hash, n, st);
    CA(cudaMemsetAsync(ctx->s_hi, 0, sizeof(float) * n, st));
    CA(cudaMemsetAsync(ctx->s_lo, 0, sizeof(float) * n, st));
    CA(cudaMemsetAsync(ctx->s_ovf, 0, sizeof(float) * n, st));
    CA(cudaStreamSynchronize(st));
    CA(cudaGetLastError());
    free_inputs();
#undef CA
    *out = ctx;
    return SLAG_OK;
}

}  // extern "C"

namespace {

// Room in the triple log and in the record list for the back half of the slot's view. P_tiles
// bounds the view's Gaussian-tile pairs (exact, or an estimate for a view sized on the device).
slag_status prepare_back_half(slag_ctx *ctx, ViewSlot &vs, int64_t P_tiles) {
    const CamParams &cp = vs.cp;
    cudaStream_t fb = vs.front;
    if (vs.spill_cap < kSpillMin) {
        int64_t c1 = vs.spill_cap, c2 = vs.spill_cap;
        CK(grow(vs.spill_key, c1, kSpillMin, fb));
        CK(grow(vs.spill_w, c2, kSpillMin, fb));
        vs.spill_cap = c1;
    }
    // room in the triple log: its fill level as last seen, plus what the other views in flight
    // may still append, plus this view's bound: at most kHashSlots triples per Gaussian from its
    // tables and its spill list's capacity (a view whose spills exceed it appends nothing)
    vs.log_bound = ctx->n * kHashSlots + vs.spill_cap + (1 << 20);
    int64_t others = 0;
    for (int i = 0; i < kSlots; ++i)
        if (&ctx->slot[i] != &vs) others += ctx->slot[i].log_bound;
    if (ctx->log_fill_seen + others + vs.log_bound > ctx->log_cap) {
        // no view may append while the log moves: wait for all, then read the exact
        // fill level; the new capacity keeps room for a full pipeline of views, so
        // that the next views pass this test without waiting
        CK(drain_views(ctx));
        launch_copy_words(ctx->totals, vs.h_dev->totals, kTotals * sizeof(unsigned long long), fb);
        CK(cudaStreamSynchronize(fb));
        const int64_t used = (int64_t)vs.h->totals[0];
        ctx->log_fill_seen = used;
        const int64_t need = used + others + vs.log_bound;
        int64_t c1 = ctx->log_cap, c2 = ctx->log_cap;
        CK(grow(ctx->log_key, c1, need, fb, used));
        CK(grow(ctx->log_w, c2, need, fb, used));
        ctx->log_cap = c1;
    }

    // record list of the composite: one record per (Gaussian, tile, segment) with a
    // non-zero sum (per batch of the tile's CTA); sums beyond the capacity go to the
    // tables directly, so the capacity only bounds the fast path
    // (plus two chunks per tile: a CTA's partly filled and reserved chunks)
    const int64_t tiles = (int64_t)cp.tiles_x * cp.tiles_y;
    int64_t rec_need = P_tiles + ctx->n + 2 * kRecChunk * tiles;
    rec_need = (rec_need + kRecChunk - 1) / kRecChunk * kRecChunk;
    if (rec_need > vs.rec_cap) {
        CK(grow(vs.recs, vs.rec_cap, rec_need, fb));
        vs.rec_cap = vs.rec_cap / kRecChunk * kRecChunk;
        CK(grow(vs.rec_fill, vs.fill_cap, vs.rec_cap / kRecChunk, fb));
    }
    return SLAG_OK;
}

// The composite and the combine pass of the slot's view on its back stream (after its binning
// and its upload). A non-null skip makes both do nothing when *skip is set; a non-null
// view_base_dev gives the view's first column in device memory (replayed graphs).
slag_status enqueue_composite(slag_ctx *ctx, ViewSlot &vs, const uint32_t *list, const uint32_t *skip,
                              const int32_t *view_base_dev) {
    const CamParams &cp = vs.cp;
    cudaStream_t bk = vs.back;
    CK(cudaMemsetAsync(vs.rec_chunks, 0, sizeof(unsigned long long), bk));
    CompositeArgs a;
    a.cam = cp;
    a.ranges = vs.ranges;
    a.bin_shift = kSuperShift;
    a.bins_x = ((cp.tiles_x - 1) >> kSuperShift) + 1;
    a.tile_order = vs.tile_order;
    a.list = list;
    a.prect = vs.prect;
    a.rec_a = vs.rec_a;
    a.rec_b = vs.rec_b;
    a.rec_t = vs.rec_t;
    a.n_ids = (uint32_t)ctx->n;
    a.seg = vs.seg_buf;
    a.view_base = (int32_t)vs.view_base;
    a.view_base_dev = view_base_dev;
    a.weight_mode = ctx->weight_mode;
    a.hash = vs.hash;
    a.spill_count = &vs.ctr->spills;
    a.spill_cap = (unsigned long long)vs.spill_cap;
    a.spill_key = vs.spill_key;
    a.spill_w = vs.spill_w;
    a.ctr = vs.ctr;
    a.contrib = &vs.ctr->contributions;
    a.evals = ctx->totals + 3;
    a.evals_exec = ctx->totals + 4;
    a.dbg_T = a.dbg_wsum = nullptr;
    a.dbg_count = nullptr;
    a.accumulate = 1;
    a.recs = vs.recs;
    a.rec_chunks = vs.rec_chunks;
    a.rec_fill = vs.rec_fill;
    a.chunk_cap = (unsigned long long)(vs.rec_cap / kRecChunk);
    a.dbg_list = nullptr;
    a.dbg_off = nullptr;
    a.dbg_staged = nullptr;
    a.dbg_bad = nullptr;
    a.err = ctx->tc_err;
    a.skip = skip;
    span_begin(ctx, SLAG_STAGE_COMPOSITE, bk);
    launch_composite(a, bk);
    span_end(ctx, bk);
    const HashSink sink{vs.hash, &vs.ctr->spills, (unsigned long long)vs.spill_cap, vs.spill_key, vs.spill_w,
                        (int32_t)vs.view_base};
    span_begin(ctx, SLAG_STAGE_CONSUME, bk);
    launch_combine(vs.recs, vs.rec_chunks, vs.rec_fill, (unsigned long long)(vs.rec_cap / kRecChunk), sink, skip,
                   bk, view_base_dev);
    span_end(ctx, bk);
    CK(cudaGetLastError());
    return SLAG_OK;
}

// The consume pass of the slot's view on its back stream (after the previous view's consume),
// then the copy of the view's counters and the log's fill level to the slot's mapped host struct.
slag_status enqueue_consume(slag_ctx *ctx, ViewSlot &vs, const uint32_t *skip, const int32_t *view_base_dev) {
    cudaStream_t bk = vs.back;
    ConsumeArgs c;
    c.hash = vs.hash;
    c.n = ctx->n;
    c.view_base = (int32_t)vs.view_base;
    c.view_base_dev = view_base_dev;
    c.s_hi = ctx->s_hi;
    c.s_lo = ctx->s_lo;
    c.s_ovf = ctx->s_ovf;
    c.log_count = ctx->log_count;
    c.log_cap = (unsigned long long)ctx->log_cap;
    c.log_key = ctx->log_key;
    c.log_w = ctx->log_w;
    c.overflow = reinterpret_cast<uint32_t *>(ctx->totals + 2);
    c.spill_count = &vs.ctr->spills;
    c.spill_cap = (unsigned long long)vs.spill_cap;
    c.spill_key = vs.spill_key;
    c.spill_w = vs.spill_w;
    c.view_contrib = &vs.ctr->contributions;
    c.total_contrib = ctx->contrib;
    c.skip = skip;
    span_begin(ctx, SLAG_STAGE_CONSUME, bk);
    launch_consume(c, bk);
    span_end(ctx, bk);
    launch_copy_words(vs.ctr, &vs.h_dev->v, sizeof(ViewCounters), bk);
    launch_copy_words(ctx->totals, vs.h_dev->totals, kTotals * sizeof(unsigned long long), bk);
    CK(cudaGetLastError());
    return SLAG_OK;
}

// The back half of a view whose binning is queued (ev_bin): room in the triple log and in the
// record list, then the composite, the combine pass and (in view order: the compensated sums are
// updated without atomics) the consume pass on the slot's back stream, and a copy of the view's
// counters to the slot's mapped host struct at its end. P_tiles bounds the view's Gaussian-tile
// pairs; a non-null skip makes the passes do nothing when *skip is set.
slag_status queue_back_half(slag_ctx *ctx, ViewSlot &vs, const uint32_t *list, int64_t P_tiles,
                            const uint32_t *skip) {
    slag_status s = prepare_back_half(ctx, vs, P_tiles);
    if (s != SLAG_OK) return s;
    vs.list = list;
    vs.pending = true;
    cudaStream_t bk = vs.back;
    CK(cudaStreamWaitEvent(bk, vs.ev_bin, 0));
    CK(cudaStreamWaitEvent(bk, vs.ev_up, 0));   // the segment map
    s = enqueue_composite(ctx, vs, list, skip, nullptr);
    if (s != SLAG_OK) return s;
    CK(cudaStreamWaitEvent(bk, ctx->ev_consumed, 0));
    s = enqueue_consume(ctx, vs, skip, nullptr);
    if (s != SLAG_OK) return s;
    CK(cudaEventRecord(ctx->ev_consumed, bk));
    CK(cudaEventRecord(vs.ev_done, bk));
    return SLAG_OK;
}

// A view's exact counts join the statistics and the sizing estimates of later views.
void count_view(slag_ctx *ctx, const ViewCounters &v) {
    ctx->stats.pairs += (int64_t)v.P_tiles;
    ctx->stats.last_pairs = (int64_t)v.P_tiles;
    ctx->est_P = std::max(ctx->est_P, (int64_t)v.P);
    ctx->est_P_tiles = std::max(ctx->est_P_tiles, (int64_t)v.P_tiles);
}

// The second half of the last accepted view sized on the host: stage B on its own stream once
// stage A's counters are on the host, then the back half. It runs in the next call (the next
// view's slag_add_view, or any call that joins the views), so that stage A of the next view is
// already queued while the host waits for this view's counters.
slag_status launch_deferred_view(slag_ctx *ctx) {
    if (!ctx->deferred) return SLAG_OK;
    ctx->deferred = false;
    ViewSlot &vs = ctx->slot[(ctx->views_enqueued - 1) % kSlots];
    CK(cudaEventSynchronize(vs.ev_a));
    CK(cudaGetLastError());
    spans_resolve(ctx, false);
    cudaStream_t fb = vs.front;
    CK(cudaStreamWaitEvent(fb, vs.ev_a, 0));
    int64_t P = 0;
    uint32_t *list = nullptr;
    slag_status s = stage_b(ctx, vs, fb, vs.cp, kSuperShift, vs.scratch, &P, &list);
    if (s != SLAG_OK) return s;
    CK(cudaEventRecord(vs.ev_bin, fb));
    ctx->log_fill_seen = std::max(ctx->log_fill_seen, (int64_t)vs.h->totals[0]);
    s = queue_back_half(ctx, vs, list, (int64_t)vs.h->v.P_tiles, nullptr);
    if (s != SLAG_OK) return s;
    count_view(ctx, vs.h->v);
    return SLAG_OK;
}

// The pair capacity of a view sized on the device: the largest pair count seen so far, with a
// quarter more, rounded up to a sixteenth of its power of two (so that it changes rarely).
int64_t device_pair_cap(const slag_ctx *ctx) {
    int64_t c = ctx->est_P + ctx->est_P / 4 + 4096;
    int b = 0;
    while ((1ll << (b + 1)) <= c) ++b;
    const int64_t step = b >= 4 ? (1ll << (b - 4)) : 1;
    return (c + step - 1) / step * step;
}

// The buffers of stage B of a view sized on the device, for `cap` pairs.
slag_status prepare_stage_b_async(slag_ctx *ctx, ViewSlot &vs, int64_t cap) {
    const CamParams &cp = vs.cp;
    cudaStream_t st = vs.front;
    if (cap > 0x7fffffffLL) return fail(ctx, SLAG_ERR_CAPACITY, "more than 2^31-1 Gaussian-tile pairs in one view");
    if (cap > vs.p_cap) {
        int64_t c0 = vs.p_cap;
        for (int b = 0; b < 2; ++b) {
            int64_t c1 = c0, c2 = c0;
            CK(grow(vs.pkey[b], c1, cap, st));
            CK(grow(vs.pval[b], c2, cap, st));
            vs.p_cap = c1;
        }
    }
    CK(scratch_reserve(vs.scratch, vs.p_cap));
    const int bins_x = ((cp.tiles_x - 1) >> kSuperShift) + 1, bins_y = ((cp.tiles_y - 1) >> kSuperShift) + 1;
    CK(grow(vs.ranges, vs.ranges_cap, (int64_t)bins_x * bins_y, st));
    CK(grow(vs.prect, vs.prect_cap, cap, st));
    CK(grow(vs.tile_order, vs.order_cap, (int64_t)cp.tiles_x * cp.tiles_y, st));
    return SLAG_OK;
}

// Stage B of a view sized on the device: the binning reads the view's counts from device
// memory and holds at most `cap` pairs; a view with more sets its overflow flag, which makes its
// binning leave every bin empty and its back half do nothing. The host finds the flag when it
// settles the view. Buffers from prepare_stage_b_async.
slag_status enqueue_stage_b_async(slag_ctx *ctx, ViewSlot &vs, int64_t cap, uint32_t **list_out) {
    const CamParams &cp = vs.cp;
    cudaStream_t st = vs.front;
    const int shift = kSuperShift;
    const int bins_x = ((cp.tiles_x - 1) >> shift) + 1, bins_y = ((cp.tiles_y - 1) >> shift) + 1;
    const int64_t bins = (int64_t)bins_x * bins_y;
    span_begin(ctx, SLAG_STAGE_BIN, st);
    if (!bin_sort_fused(vs.srect, vs.offsets, vs.stouched, ctx->n, &vs.ctr->n_visible, &vs.ctr->P, cap, 0,
                        &vs.ctr->overflow, shift, bins_x, (int)bins, vs.sgid, vs.pval[0], vs.prect, vs.ranges,
                        vs.scratch, st))
        return fail(ctx, SLAG_ERR_STATE, "device-sized binning needs at most 2048 bins");
    launch_tile_order(vs.ranges, cp.tiles_x, cp.tiles_y, shift, vs.tile_order, st);
    span_end(ctx, st);
    CK(cudaGetLastError());
    *list_out = vs.pval[0];
    return SLAG_OK;
}

// Stream capture of enqueue() on st into *exec (replacing it) and the number of kernels it holds
// in *nk; the capture launches nothing, so its count is taken back from the launch counter.
template <typename F>
slag_status capture_graph(slag_ctx *ctx, cudaStream_t st, cudaGraphExec_t *exec, unsigned long long *nk, F enqueue) {
    if (*exec) cudaGraphExecDestroy(*exec);
    *exec = nullptr;
    const unsigned long long before = launches_now();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const slag_status s = enqueue();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    const unsigned long long k = launches_now() - before;
    unnote_launches(k);
    if (s == SLAG_OK && e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (s != SLAG_OK) return s;
    if (e != cudaSuccess) {
        *exec = nullptr;
        (void)cudaGetLastError();
        return fail(ctx, SLAG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    *nk = k;
    return SLAG_OK;
}

// A hash of the values a slot's captured graphs depend on (FNV-1a over 64-bit words).
uint64_t graph_key(std::initializer_list<uint64_t> vals) {
    uint64_t h = 1469598103934665603ull;
    for (uint64_t v : vals)
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xffu;
            h *= 1099511628211ull;
        }
    return h;
}

uint64_t front_key(const slag_ctx *ctx, const ViewSlot &vs, int64_t cap) {
    auto P = [](const void *p) { return (uint64_t)(uintptr_t)p; };
    return graph_key({1, (uint64_t)vs.cp.width, (uint64_t)vs.cp.height, (uint64_t)ctx->n, (uint64_t)cap,
                      (uint64_t)vs.p_cap, P(vs.pval[0]), P(vs.prect), P(vs.ranges), P(vs.tile_order),
                      P(vs.scratch.hist), P(vs.scratch.tstart), P(vs.scratch.digit_tot), P(vs.scratch.partials)});
}

uint64_t back_key(const slag_ctx *ctx, const ViewSlot &vs) {
    auto P = [](const void *p) { return (uint64_t)(uintptr_t)p; };
    return graph_key({2, (uint64_t)vs.cp.width, (uint64_t)vs.cp.height, (uint64_t)ctx->n, P(vs.pval[0]),
                      P(vs.prect), P(vs.ranges), P(vs.tile_order), P(vs.seg_buf), P(vs.recs), P(vs.rec_fill),
                      (uint64_t)vs.rec_cap, P(ctx->log_key), P(ctx->log_w), (uint64_t)ctx->log_cap,
                      (uint64_t)ctx->weight_mode, P(vs.spill_key), P(vs.spill_w), (uint64_t)vs.spill_cap});
}

// Settles the slot's view: waits for its back half and reads its counters. A view sized on the
// device is counted here; when its pairs exceeded its binning's capacity, its binning (its
// stage A results, segment map and columns are still in place) and its back half run again with
// the exact count. A view whose spills exceeded its slot's spill list gets a list that holds
// them and is composited again (its consume pass changed nothing but its cleared tables).
slag_status settle_slot(slag_ctx *ctx, ViewSlot &vs) {
    while (vs.pending) {
        vs.pending = false;
        CK(cudaEventSynchronize(vs.ev_done));
        CK(cudaGetLastError());
        const ViewCounters v = vs.h->v;   // copied at the end of its back half
        ctx->log_fill_seen = std::max(ctx->log_fill_seen, (int64_t)vs.h->totals[0]);
        const bool sized_on_device = vs.count_at_settle;
        vs.count_at_settle = false;
        if (sized_on_device) count_view(ctx, v);
        cudaStream_t fb = vs.front;
        if (sized_on_device && v.overflow) {
            ctx->stats.pairs -= (int64_t)v.P_tiles;   // counted again below
            CK(cudaMemsetAsync(&vs.ctr->overflow, 0, sizeof(uint32_t), fb));
            int64_t P = 0;
            uint32_t *list = nullptr;
            slag_status s = stage_b(ctx, vs, fb, vs.cp, kSuperShift, vs.scratch, &P, &list);
            if (s != SLAG_OK) return s;
            CK(cudaEventRecord(vs.ev_bin, fb));
            s = queue_back_half(ctx, vs, list, (int64_t)v.P_tiles, nullptr);
            if (s != SLAG_OK) return s;
            ctx->stats.pairs += (int64_t)v.P_tiles;
            ctx->stats.resized_views += 1;
        } else if (v.spills > (unsigned long long)vs.spill_cap) {
            int64_t c1 = vs.spill_cap, c2 = vs.spill_cap;
            CK(grow(vs.spill_key, c1, (int64_t)v.spills, fb));
            CK(grow(vs.spill_w, c2, (int64_t)v.spills, fb));
            vs.spill_cap = c1;
            CK(cudaMemsetAsync(&vs.ctr->spills, 0, sizeof(unsigned long long), fb));
            CK(cudaMemsetAsync(&vs.ctr->contributions, 0, sizeof(unsigned long long), fb));
            CK(cudaEventRecord(vs.ev_bin, fb));
            const slag_status s = queue_back_half(ctx, vs, vs.list, (int64_t)v.P_tiles, nullptr);
            if (s != SLAG_OK) return s;
            ctx->stats.recomposited_views += 1;
        }
    }
    return SLAG_OK;
}

// Settles every view (before a join reads the accumulated state).
slag_status settle_views(slag_ctx *ctx) {
    for (int i = 0; i < kSlots; ++i) {
        slag_status s = settle_slot(ctx, ctx->slot[i]);
        if (s != SLAG_OK) return s;
    }
    return SLAG_OK;
}

}  // namespace

extern "C" {

slag_status slag_add_view(slag_ctx *ctx, const slag_camera *cam, const int32_t *seg_ids, const float *seg_table,
                          int32_t M, int32_t on_device) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    slag_status s = check_camera(ctx, cam);
    if (s != SLAG_OK) return s;
    if (!seg_ids || !seg_table) return fail(ctx, SLAG_ERR_INVALID_ARG, "seg_ids / seg_table is NULL");
    if (M < 1 || M >= (1 << 24)) return fail(ctx, SLAG_ERR_INVALID_ARG, "M outside [1, 2^24)");
    if (ctx->table_rows + M >= (1LL << 32)) return fail(ctx, SLAG_ERR_CAPACITY, "more than 2^32 segment columns");
    CK(cudaSetDevice(ctx->device));
    // latent form: the segment embeddings are encoded to 32-d codes at finalize, all views' rows
    // in one pass (the codes are only read there)
    if (ctx->precision == SLAG_PREC_LATENT32 && !ctx->lat_params)
        return fail(ctx, SLAG_ERR_STATE, "latent form: slag_set_latent before the first view");
    if (ctx->precision == SLAG_PREC_LINEAR32 && !ctx->lin_params)
        return fail(ctx, SLAG_ERR_STATE, "linear code: slag_set_linear_code before the first view");
    ViewSlot &vs = ctx->slot[ctx->views_enqueued % kSlots];
    cudaStream_t fr = vs.front, up = ctx->up;
    const CamParams cp = cam_params(cam);
    const int64_t npx = (int64_t)cam->width * cam->height;
    const int64_t D = ctx->D;
    // the slot's previous view, if it was sized on the device, is settled before its buffers go
    s = settle_slot(ctx, vs);
    if (s != SLAG_OK) return s;
    // the view's second half: sized on the device and queued by this call when earlier views give
    // an estimate of its pair count (and its bins fit the single-pass binning), as replays of the
    // slot's captured graphs unless stages are being timed; otherwise sized on the host, in the
    // next call
    const int64_t bins = (int64_t)(((cp.tiles_x - 1) >> kSuperShift) + 1) * (((cp.tiles_y - 1) >> kSuperShift) + 1);
    const bool device_sized = ctx->est_P > 0 && bins <= 2048 && !(kChecked && ctx->force_pair_cap > 0);
    const bool graphed = device_sized && ctx->graphs && ctx->prof_mask == 0;
    const int64_t cap = device_sized ? device_pair_cap(ctx) : 0;
    vs.cp = cp;
    vs.view_base = ctx->table_rows;

    // stage A and the uploads start after the caller's work so far (inputs written on the
    // caller's stream) and after the slot's previous view has been composited and consumed
    CK(cudaEventRecord(ctx->ev_in, ctx->stream));
    CK(cudaStreamWaitEvent(fr, ctx->ev_in, 0));
    CK(cudaStreamWaitEvent(fr, vs.ev_done, 0));
    CK(cudaStreamWaitEvent(up, ctx->ev_in, 0));
    CK(cudaStreamWaitEvent(up, vs.ev_done, 0));

    // segment embeddings -> rows [table_rows, table_rows + M) of the column store; the segment
    // map -> the slot; then the check of its ids. All on the upload stream: stage A does not
    // read them, and the composite waits for them.
    if (ctx->table_rows + M > ctx->table_cap / D) {
        CK(drain_views(ctx));   // growing frees the old store
        CK(grow(ctx->table, ctx->table_cap, (ctx->table_rows + M) * D, fr, ctx->table_rows * D));
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // everything from the first copy on; on an error the call still waits for the upload stream
    // before it returns, since the caller may free its buffers once the call returns
    auto queue_view = [&]() -> slag_status {
        CK(cudaMemcpyAsync(ctx->table + ctx->table_rows * D, seg_table, sizeof(float) * (size_t)(M * D), kind,
                           up));
        if (npx > vs.seg_cap) {
            CK(cudaStreamSynchronize(up));   // the slot's previous composite has read the old map
            CK(grow(vs.seg_buf, vs.seg_cap, npx, fr));
        }
        CK(cudaMemcpyAsync(vs.seg_buf, seg_ids, sizeof(int32_t) * (size_t)npx, kind, up));
        CK(cudaMemsetAsync(vs.ctr_up, 0, sizeof(ViewCounters), up));
        launch_check_seg(vs.seg_buf, npx, M, vs.ctr_up, up);
        launch_copy_words(vs.ctr_up, &vs.h_dev->vu, sizeof(ViewCounters), up);
        CK(cudaEventRecord(vs.ev_up, up));
        // one piece of an earlier asynchronous finalize's download, queued behind this view's
        // upload so that the two do not share the PCIe link
        if (ctx->pend_left) {
            CK(cudaStreamWaitEvent(ctx->cstream, vs.ev_up, 0));
            const slag_status sp = issue_pending(ctx, 1);
            if (sp != SLAG_OK) return sp;
        }
        // stage A of this view (and stage B when it is sized on the device), then the previous
        // view's second half
        if (device_sized) {
            const slag_status sp = prepare_stage_b_async(ctx, vs, cap);
            if (sp != SLAG_OK) return sp;
        }
        bool front_graph = graphed;
        if (graphed) {
            vs.vp_host->cam = cp;
            vs.vp_host->view_base = (int32_t)vs.view_base;
            CK(cudaMemcpyAsync(vs.vp_dev, vs.vp_host, sizeof(ViewParams), cudaMemcpyHostToDevice, fr));
            const uint64_t key = front_key(ctx, vs, cap);
            if (!vs.gx_front || vs.gkey_front != key) {
                vs.gkey_front = 0;
                const slag_status sc = capture_graph(ctx, fr, &vs.gx_front, &vs.gn_front, [&]() -> slag_status {
                    const slag_status sa = stage_a(ctx, vs, fr, cp, kSuperShift, vs.scratch, &vs.vp_dev->cam);
                    if (sa != SLAG_OK) return sa;
                    uint32_t *list = nullptr;
                    return enqueue_stage_b_async(ctx, vs, cap, &list);
                });
                if (sc == SLAG_OK) vs.gkey_front = key;
                else front_graph = false;   // launched kernel by kernel instead
            }
        }
        if (front_graph) {
            CK(cudaGraphLaunch(vs.gx_front, fr));
            note_launches(vs.gn_front);
            CK(cudaEventRecord(vs.ev_a, fr));
        } else {
            const slag_status sa = stage_a(ctx, vs, fr, cp, kSuperShift, vs.scratch);
            if (sa != SLAG_OK) return sa;
            CK(cudaEventRecord(vs.ev_a, fr));
            if (device_sized) {
                uint32_t *list = nullptr;
                const slag_status sb = enqueue_stage_b_async(ctx, vs, cap, &list);
                if (sb != SLAG_OK) return sb;
            }
        }
        if (device_sized) CK(cudaEventRecord(vs.ev_bin, fr));
        return launch_deferred_view(ctx);
    };
    s = queue_view();
    if (s != SLAG_OK) {
        cudaStreamSynchronize(up);
        return s;
    }

    // the caller's buffers are free once the uploads are done; the check's result came with them
    CK(cudaEventSynchronize(vs.ev_up));
    CK(cudaGetLastError());
    if (vs.h->vu.bad_seg) return fail(ctx, SLAG_ERR_INVALID_ARG, "segment id outside [-1, M)");
    if (device_sized) {
        // the back half: queued now (the composite waits for the binning and the upload; its
        // passes do nothing if the binning overflowed)
        const int64_t tiles_bound = ctx->est_P_tiles + ctx->est_P_tiles / 4 + 4096;
        bool back_graph = graphed;
        if (graphed) {
            s = prepare_back_half(ctx, vs, tiles_bound);
            if (s != SLAG_OK) return s;
            const uint64_t key = back_key(ctx, vs);
            if (!vs.gx_comp || !vs.gx_cons || vs.gkey_back != key) {
                vs.gkey_back = 0;
                slag_status sc = capture_graph(ctx, vs.back, &vs.gx_comp, &vs.gn_comp, [&]() {
                    return enqueue_composite(ctx, vs, vs.pval[0], &vs.ctr->overflow, &vs.vp_dev->view_base);
                });
                if (sc == SLAG_OK)
                    sc = capture_graph(ctx, vs.back, &vs.gx_cons, &vs.gn_cons, [&]() {
                        return enqueue_consume(ctx, vs, &vs.ctr->overflow, &vs.vp_dev->view_base);
                    });
                if (sc == SLAG_OK) vs.gkey_back = key;
                else back_graph = false;   // launched kernel by kernel instead
            }
        }
        if (back_graph) {
            cudaStream_t bk = vs.back;
            CK(cudaStreamWaitEvent(bk, vs.ev_bin, 0));
            CK(cudaStreamWaitEvent(bk, vs.ev_up, 0));   // the segment map
            CK(cudaGraphLaunch(vs.gx_comp, bk));
            note_launches(vs.gn_comp);
            CK(cudaStreamWaitEvent(bk, ctx->ev_consumed, 0));   // consumes in view order
            CK(cudaGraphLaunch(vs.gx_cons, bk));
            note_launches(vs.gn_cons);
            CK(cudaEventRecord(ctx->ev_consumed, bk));
            CK(cudaEventRecord(vs.ev_done, bk));
        } else {
            s = queue_back_half(ctx, vs, vs.pval[0], tiles_bound, &vs.ctr->overflow);
            if (s != SLAG_OK) return s;
        }
        vs.list = vs.pval[0];
        vs.pending = true;
        vs.count_at_settle = true;
    }
    ctx->views_enqueued += 1;
    ctx->table_rows += M;
    ctx->deferred = !device_sized;
    ctx->stats.views += 1;
    ctx->stats.columns = ctx->table_rows;
    ctx->finalized = false;
    return SLAG_OK;
}

}  // extern "C"

namespace {

// Everything finalize does before the contraction: join the views in flight,
// read the totals, sort the triple log by (block, column, Gaussian) and list
// the distinct columns of every block.
slag_status finalize_prepare(slag_ctx *ctx) {
    if (ctx->stats.views == 0) return fail(ctx, SLAG_ERR_STATE, "finalize before any view");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    slag_status s0 = launch_deferred_view(ctx);
    if (s0 == SLAG_OK) s0 = settle_views(ctx);
    if (s0 != SLAG_OK) return s0;
    CK(join_views(ctx));
    const ViewSlot &last = ctx->slot[(ctx->views_enqueued + kSlots - 1) % kSlots];
    launch_copy_words(ctx->totals, ctx->hc_dev->totals, kTotals * sizeof(unsigned long long), st);
    launch_copy_words(last.ctr, &ctx->hc_dev->v, sizeof(ViewCounters), st);
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    {
        const slag_status sc = checks_reported(ctx);
        if (sc != SLAG_OK) return sc;
    }
    ctx->stats.contributions = (int64_t)ctx->hc->totals[1];
    ctx->stats.evaluations = (int64_t)ctx->hc->totals[3];
    ctx->stats.executed = (int64_t)ctx->hc->totals[4];
    ctx->stats.last_contributions = (int64_t)ctx->hc->v.contributions;
    if (ctx->hc->totals[2]) ctx->log_overflowed = true;
    if (ctx->log_overflowed) return fail(ctx, SLAG_ERR_CAPACITY, "the triple log overflowed in some view");
    const int64_t Z = (int64_t)ctx->hc->totals[0];
    ctx->stats.triples = Z;
    ctx->log_fill_seen = Z;
    const int64_t n = ctx->n;
    const int64_t nblocks = (n + kBlockG - 1) / kBlockG;
    CK(cudaMemsetAsync(ctx->bstart, 0, sizeof(uint32_t) * nblocks, st));
    CK(cudaMemsetAsync(ctx->bend, 0, sizeof(uint32_t) * nblocks, st));
    CK(cudaMemsetAsync(ctx->touched, 0, sizeof(unsigned long long), st));
    if (Z > 0) {
        if (Z > ctx->fin_cap) {
            int64_t c = ctx->fin_cap;
            int64_t c1 = c, c2 = c, c3 = c, c4 = c, c5 = c, c6 = c;
            CK(grow(ctx->log_key_alt, c1, Z, st));
            CK(grow(ctx->log_w_alt, c2, Z, st));
            CK(grow(ctx->flags, c3, Z, st));
            CK(grow(ctx->uidx, c4, Z, st));
            CK(grow(ctx->ucol, c5, Z, st));
            CK(grow(ctx->ustart, c6, Z, st));
            ctx->fin_cap = c1;
            CK(scratch_reserve(ctx->scratch, Z));
        }
        span_begin(ctx, SLAG_STAGE_LOG_SORT, st);
        // sort by (block, column) -- the order of a group's Gaussians is free, the aggregation
        // adds them in any order -- on the compact key layout, whose sorted fields are one
        // contiguous range of col_bits + block_bits bits
        const int cb = ceil_log2((uint64_t)ctx->table_rows);
        launch_repack_keys(ctx->log_key, ctx->log_key, nullptr, nullptr, Z, cb, true, st);
        int shifts[16], widths[16];
        int np = digit_passes(7, cb + ceil_log2((uint64_t)nblocks), shifts, widths, Z);
        const bool alt = radix_sort_u64(ctx->log_key, ctx->log_key_alt, reinterpret_cast<uint32_t *>(ctx->log_w),
                                        reinterpret_cast<uint32_t *>(ctx->log_w_alt), Z, shifts, widths, np,
                                        ctx->scratch, st);
        const uint64_t *sk = alt ? ctx->log_key_alt : ctx->log_key;
        const float *sw = alt ? ctx->log_w_alt : ctx->log_w;
        launch_unique_flags(sk, Z, ctx->flags, st);
        exclusive_scan_u32(ctx->flags, ctx->uidx, Z, nullptr, ctx->scratch, st);
        launch_uniques(sk, ctx->flags, ctx->uidx, Z, cb, ctx->ucol, ctx->ustart, ctx->bstart, ctx->bend, st);
        // the sorted log, back in pack_key's layout, becomes the log (its order is free; later
        // views append to it and the aggregations read it); the log keeps its own buffers, so
        // its capacity for the views in flight stays as it was
        launch_repack_keys(sk, ctx->log_key, alt ? sw : nullptr, ctx->log_w, Z, cb, false, st);
        span_end(ctx, st);
    }
    return SLAG_OK;
}

AggArgs agg_args(slag_ctx *ctx) {
    AggArgs g;
    memset(&g, 0, sizeof(g));
    g.keys = ctx->log_key;
    g.w = ctx->log_w;
    g.flags = ctx->flags;
    g.uidx = ctx->uidx;
    g.ucol = ctx->ucol;
    g.ustart = ctx->ustart;
    g.bstart = ctx->bstart;
    g.bend = ctx->bend;
    g.table = ctx->table;
    g.columns = ctx->table_rows;
    g.s_hi = ctx->s_hi;
    g.s_lo = ctx->s_lo;
    g.s_ovf = ctx->s_ovf;
    g.orig_of_int = ctx->orig_of_int;
    g.n = ctx->n;
    g.D = ctx->D;
    g.E = ctx->E;
    g.inv_norm = ctx->inv_norm;
    g.wsum = ctx->wsum;
    g.touched = ctx->touched;
    g.bf16 = ctx->precision == SLAG_PREC_BF16 ? 1 : 0;
    return g;
}

// The contraction in chunks of blocks, for outputs that need not be resident on
// the device: each chunk's rows (Morton order), their caller ids, weight sums and
// means are copied to pinned host memory and handed to `sink` (rows with id
// 0xffffffff lie past the last Gaussian). At most chunk_gaussians rows are
// resident on the device at a time.
struct ChunkView {
    const float *E;          // rows x D
    const uint32_t *ids;     // rows
    const float *wsum;       // rows
    const float4 *means;     // rows: (x, y, z, opacity)
    int64_t rows;
};

template <typename Sink>
slag_status aggregate_chunks(slag_ctx *ctx, int64_t chunk_gaussians, Sink &&sink) {
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->n, D = ctx->D;
    const int64_t nblocks = (n + kBlockG - 1) / kBlockG;
    int64_t cb = chunk_gaussians / kBlockG;
    if (cb < 1) cb = 1;
    if (cb > nblocks) cb = nblocks;
    const int64_t rows = cb * kBlockG;
    float *dE = nullptr, *dW = nullptr, *hE = nullptr, *hW = nullptr;
    uint32_t *dI = nullptr, *hI = nullptr;
    float4 *hM = nullptr;
    slag_status rc = SLAG_OK;
    auto release = [&]() {
        dfree(dE); dfree(dW); dfree(dI);
        if (hE) cudaFreeHost(hE);
        if (hW) cudaFreeHost(hW);
        if (hI) cudaFreeHost(hI);
        if (hM) cudaFreeHost(hM);
    };
#define CC(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            release();                                                                              \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? SLAG_ERR_OOM : SLAG_ERR_CUDA,        \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
        }                                                                                           \
    } while (0)
    CC(dalloc(&dE, rows * D));
    CC(dalloc(&dW, rows));
    CC(dalloc(&dI, rows));
    CC(cudaMallocHost((void **)&hE, sizeof(float) * (size_t)(rows * D)));
    CC(cudaMallocHost((void **)&hW, sizeof(float) * (size_t)rows));
    CC(cudaMallocHost((void **)&hI, sizeof(uint32_t) * (size_t)rows));
    CC(cudaMallocHost((void **)&hM, sizeof(float4) * (size_t)rows));
    AggArgs g = agg_args(ctx);
    g.E_chunk = dE;
    g.ids_chunk = dI;
    g.wsum_chunk = dW;
    for (int64_t b0 = 0; b0 < nblocks && rc == SLAG_OK; b0 += cb) {
        const int64_t nb = (b0 + cb <= nblocks) ? cb : nblocks - b0;
        g.block0 = b0;
        launch_aggregate(g, nb, ctx->tc_err, st);
        const int64_t r = nb * kBlockG;
        const int64_t first = b0 * kBlockG;
        const int64_t valid = (first + r <= n) ? r : n - first;
        CC(cudaMemcpyAsync(hE, dE, sizeof(float) * (size_t)(r * D), cudaMemcpyDeviceToHost, st));
        CC(cudaMemcpyAsync(hW, dW, sizeof(float) * (size_t)r, cudaMemcpyDeviceToHost, st));
        CC(cudaMemcpyAsync(hI, dI, sizeof(uint32_t) * (size_t)r, cudaMemcpyDeviceToHost, st));
        CC(cudaMemcpyAsync(hM, ctx->mean_op + first, sizeof(float4) * (size_t)valid, cudaMemcpyDeviceToHost, st));
        CC(cudaMemcpyAsync(&ctx->hc->tc_err, ctx->tc_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        CC(cudaStreamSynchronize(st));
        if (ctx->hc->tc_err) {
            release();
            return timeout_reported(ctx, "the tensor-core aggregation gave up waiting");
        }
        rc = sink(ChunkView{hE, hI, hW, hM, valid});
    }
#undef CC
    release();
    return rc;
}

// Issues up to `pieces` pieces of the pending download on the copy stream (all of them when
// pieces < 0); with the last one, the download's buffer gets its copy event.
slag_status issue_pending(slag_ctx *ctx, int pieces) {
    if (!ctx->pend_left) return SLAG_OK;
    for (int i = 0; (pieces < 0 || i < pieces) && ctx->pend_left > 0; ++i) {
        const size_t b = std::min(ctx->pend_piece, ctx->pend_left);
        CK(cudaMemcpyAsync(ctx->pend_dst + ctx->pend_off, ctx->pend_src + ctx->pend_off, b, ctx->pend_kind,
                           ctx->cstream));
        ctx->pend_off += b;
        ctx->pend_left -= b;
    }
    if (!ctx->pend_left) CK(cudaEventRecord(ctx->ev_copy[ctx->pend_buf], ctx->cstream));
    return SLAG_OK;
}

// Makes ctx->E / ctx->wsum writable by this finalize: when copies of the current buffers are
// still queued, the finalize moves to the other pair (allocated on first use) after the copies
// that last read it.
slag_status claim_output_buffers(slag_ctx *ctx, cudaStream_t st) {
    if (!ctx->copy_pending[ctx->cur]) return SLAG_OK;
    const int nx = 1 - ctx->cur;
    if (!ctx->E_buf[nx]) {
        CK(dalloc(&ctx->E_buf[nx], ctx->n * (int64_t)ctx->D));
        CK(dalloc(&ctx->wsum_buf[nx], ctx->n));
    }
    if (ctx->copy_pending[nx]) CK(cudaStreamWaitEvent(st, ctx->ev_copy[nx], 0));
    ctx->copy_pending[nx] = false;
    ctx->cur = nx;
    ctx->E = ctx->E_buf[nx];
    ctx->wsum = ctx->wsum_buf[nx];
    return SLAG_OK;
}

// Queues the copies of E and sum w of this finalize on the copy stream, after the work queued on
// st so far.
slag_status queue_output_copies(slag_ctx *ctx, cudaStream_t st, float *out_emb, float *out_wsum,
                                cudaMemcpyKind kind) {
    if (!ctx->cstream) {
        CK(cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ctx->ev_fin, cudaEventDisableTiming));
        for (int b = 0; b < 2; ++b) CK(cudaEventCreateWithFlags(&ctx->ev_copy[b], cudaEventDisableTiming));
    }
    const int64_t n = ctx->n;
    slag_status s = issue_pending(ctx, -1);
    if (s != SLAG_OK) return s;
    CK(cudaEventRecord(ctx->ev_fin, st));
    CK(cudaStreamWaitEvent(ctx->cstream, ctx->ev_fin, 0));
    if (out_wsum) CK(cudaMemcpyAsync(out_wsum, ctx->wsum, sizeof(float) * (size_t)n, kind, ctx->cstream));
    ctx->copy_pending[ctx->cur] = true;
    if (!out_emb) {
        CK(cudaEventRecord(ctx->ev_copy[ctx->cur], ctx->cstream));
        return SLAG_OK;
    }
    // the embeddings in pieces of about 1/64 (at least 4 MB), issued by later calls
    const size_t total = sizeof(float) * (size_t)(n * ctx->D);
    ctx->pend_src = reinterpret_cast<const char *>(ctx->E);
    ctx->pend_dst = reinterpret_cast<char *>(out_emb);
    ctx->pend_left = total;
    ctx->pend_off = 0;
    ctx->pend_piece = std::max<size_t>((size_t)4 << 20, (total + 63) / 64);
    ctx->pend_kind = kind;
    ctx->pend_buf = ctx->cur;
    return SLAG_OK;
}

slag_status finalize_impl(slag_ctx *ctx, float *out_emb, float *out_wsum, int32_t on_device, bool async_out) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    slag_status s = issue_pending(ctx, -1);   // an earlier download's remaining pieces
    if (s != SLAG_OK) return s;
    s = finalize_prepare(ctx);
    if (s != SLAG_OK) return s;
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->n;
    const int64_t nblocks = (n + kBlockG - 1) / kBlockG;
    if (ctx->opt_flags & SLAG_FLAG_EMBEDDINGS_ON_HOST) {
        // no resident n x D copy: the rows arrive in chunks and are placed in caller order here
        if (out_emb && on_device) return fail(ctx, SLAG_ERR_INVALID_ARG, "embeddings are kept on the host: out_emb must be host memory");
        const int64_t D = ctx->D;
        s = aggregate_chunks(ctx, ctx->chunk_gaussians, [&](const ChunkView &c) {
            for (int64_t r = 0; r < c.rows; ++r) {
                const uint32_t id = c.ids[r];
                if (id == 0xffffffffu) continue;
                if (out_emb) memcpy(out_emb + (int64_t)id * D, c.E + r * D, sizeof(float) * (size_t)D);
                if (out_wsum && !on_device) out_wsum[id] = c.wsum[r];
            }
            return SLAG_OK;
        });
        if (s != SLAG_OK) return s;
        if (out_wsum && on_device) CK(cudaMemcpyAsync(out_wsum, ctx->wsum, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(&ctx->hc->touched, ctx->touched, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        spans_resolve(ctx, false);
        ctx->stats.touched = (int64_t)ctx->hc->touched;
        ctx->n_q = 0;
        ctx->finalized = false;   // queries need the embeddings on the device
        return SLAG_OK;
    }
    if (async_out || ctx->copy_pending[ctx->cur]) {
        s = claim_output_buffers(ctx, st);
        if (s != SLAG_OK) return s;
    }
    AggArgs g = agg_args(ctx);
    span_begin(ctx, SLAG_STAGE_AGGREGATE, st);
    if (ctx->precision == SLAG_PREC_LATENT32 || ctx->precision == SLAG_PREC_LINEAR32) {
        const bool linear = ctx->precision == SLAG_PREC_LINEAR32;
        // the segment embeddings of every view -> codes; mean codes per Gaussian; the decoder in
        // chunks of rows (internal order) -> E in caller order
        const int64_t chunk = std::min<int64_t>(n, 1 << 18);
        const int64_t rows_t = ctx->table_rows;
        CK(grow(ctx->ztable, ctx->ztable_cap, rows_t * kLatent, st));
        CK(grow(ctx->lat_hidden, ctx->lat_hidden_cap,
                linear ? linear_decode_scratch((int)chunk, ctx->D)
                       : std::max(rows_t * kLatentHidden, latent_decode_scratch((int)chunk, ctx->D)), st));
        CK(grow(ctx->lat_Z, ctx->lat_Z_cap, n * kLatent, st));
        CK(grow(ctx->lat_Y, ctx->lat_Y_cap, chunk * ctx->D, st));
        float *Z = ctx->lat_Z, *Y = ctx->lat_Y;
        if (linear)
            linear_encode(ctx->lin_params, ctx->lin_enc_bias, ctx->D, ctx->table, (int)rows_t, ctx->ztable, st);
        else
            latent_encode(ctx->lat_params, ctx->D, ctx->table, (int)rows_t, ctx->lat_hidden, ctx->ztable, st);
        CK(cudaMemsetAsync(ctx->touched, 0, sizeof(unsigned long long), st));
        launch_latent_aggregate(g, ctx->ztable, Z, nblocks, st);
        for (int64_t g0 = 0; g0 < n; g0 += chunk) {
            const int64_t rows = std::min<int64_t>(chunk, n - g0);
            if (linear)
                CK(linear_decode(ctx->lin_params, ctx->D, Z + g0 * kLatent, (int)rows, ctx->lat_hidden, Y, ctx->tc_err,
                                 st));
            else
                CK(latent_decode(ctx->lat_params, ctx->D, Z + g0 * kLatent, (int)rows, ctx->lat_hidden, Y, ctx->tc_err,
                             st));
            launch_latent_finish(g, Y, g0, rows, st);
        }
    } else {
        launch_aggregate(g, nblocks, ctx->tc_err, st);
    }
    // query candidates: the rows of E with a non-zero embedding, in caller order
    launch_touched_rows(ctx->inv_norm, n, ctx->qflags, ctx->qpos, ctx->qrows, ctx->d_nq, ctx->scratch, st);
    span_end(ctx, st);
    CK(cudaGetLastError());
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (async_out) {
        s = queue_output_copies(ctx, st, out_emb, out_wsum, kind);
        if (s != SLAG_OK) return s;
    } else {
        if (out_emb) CK(cudaMemcpyAsync(out_emb, ctx->E, sizeof(float) * (size_t)(n * ctx->D), kind, st));
        if (out_wsum) CK(cudaMemcpyAsync(out_wsum, ctx->wsum, sizeof(float) * (size_t)n, kind, st));
    }
    // small results through the SMs: the copy engine may be busy with an earlier step's outputs
    launch_copy_words(ctx->touched, &ctx->hc_dev->touched, sizeof(unsigned long long), st);
    launch_copy_words(ctx->d_nq, &ctx->hc_dev->n_q, sizeof(unsigned long long), st);
    launch_copy_words(ctx->tc_err, &ctx->hc_dev->tc_err, sizeof(uint32_t), st);
    CK(cudaStreamSynchronize(st));
    if (ctx->hc->tc_err) return timeout_reported(ctx, "a bounded device wait gave up (compositing or aggregation)");
    {
        const slag_status sc = checks_reported(ctx);
        if (sc != SLAG_OK) return sc;
    }
    spans_resolve(ctx, false);
    ctx->stats.touched = (int64_t)ctx->hc->touched;
    ctx->n_q = (int64_t)ctx->hc->n_q;
    ctx->finalized = true;
    ++ctx->qgen;
    return SLAG_OK;
}

}  // namespace

extern "C" {

slag_status slag_finalize(slag_ctx *ctx, float *out_emb, float *out_wsum, int32_t on_device) {
    return finalize_impl(ctx, out_emb, out_wsum, on_device, false);
}

slag_status slag_finalize_async(slag_ctx *ctx, float *out_emb, float *out_wsum, int32_t on_device) {
    if (ctx && (ctx->opt_flags & SLAG_FLAG_EMBEDDINGS_ON_HOST))
        return fail(ctx, SLAG_ERR_INVALID_ARG, "asynchronous outputs need the embeddings on the device");
    return finalize_impl(ctx, out_emb, out_wsum, on_device, true);
}

slag_status slag_wait_outputs(slag_ctx *ctx) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    if (!ctx->cstream) return SLAG_OK;
    CK(cudaSetDevice(ctx->device));
    slag_status s = issue_pending(ctx, -1);
    if (s != SLAG_OK) return s;
    CK(cudaStreamSynchronize(ctx->cstream));
    ctx->copy_pending[0] = ctx->copy_pending[1] = false;
    return SLAG_OK;
}

slag_status slag_query_batch(slag_ctx *ctx, const float *Q, int32_t B, int32_t k, int64_t *out_ids,
                             float *out_scores, int32_t *out_count, int32_t on_device) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    if (!ctx->finalized) return fail(ctx, SLAG_ERR_STATE, "query before finalize");
    if (!Q || !out_ids || !out_scores) return fail(ctx, SLAG_ERR_INVALID_ARG, "NULL query or output");
    if (k < 1 || k > kMaxK) return fail(ctx, SLAG_ERR_INVALID_ARG, "k outside [1, 1024]");
    if (B < 1) return fail(ctx, SLAG_ERR_INVALID_ARG, "B < 1");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int64_t D = ctx->D;
    const float *dQ = Q;
    // host queries: an error return after the upload is queued still waits for the stream, since
    // the caller may free or rewrite Q once the call returns
    struct StreamGuard {
        cudaStream_t st = nullptr;
        ~StreamGuard() {
            if (st) cudaStreamSynchronize(st);
        }
    } guard;
    if (!on_device) {
        CK(grow(ctx->qbuf, ctx->qbuf_cap, (int64_t)B * D, st));
        CK(cudaMemcpyAsync(ctx->qbuf, Q, sizeof(float) * (size_t)(B * D), cudaMemcpyHostToDevice, st));
        guard.st = st;
        dQ = ctx->qbuf;
    }
    if (((uintptr_t)dQ & 15u) != 0) return fail(ctx, SLAG_ERR_INVALID_ARG, "Q must be 16-byte aligned");
    const bool tc = query_tc_supported(ctx->D, k);
    const int64_t nq = ctx->n_q;
    const int64_t nc = tc ? (int64_t)B * (nq > 0 ? query_tc_splits(B, nq) : 0) * (k < 16 ? k : 16)
                          : (int64_t)query_cand_entries(B, nq, k);
    if (nc > ctx->cand_cap) {
        int64_t c1 = ctx->cand_cap, c2 = ctx->cand_cap;
        CK(grow(ctx->cand_s, c1, nc, st));
        CK(grow(ctx->cand_i, c2, nc, st));
        ctx->cand_cap = c1;
    }
    int64_t *ids = out_ids;
    float *scores = out_scores;
    int32_t *cnt = out_count;
    if (!on_device) {
        if ((int64_t)B * k > ctx->qout_cap) {
            int64_t c1 = ctx->qout_cap, c2 = ctx->qout_cap, c3 = ctx->qout_cap;
            CK(grow(ctx->qids, c1, (int64_t)B * k, st));
            CK(grow(ctx->qscores, c2, (int64_t)B * k, st));
            CK(grow(ctx->qcount, c3, (int64_t)B * k, st));
            ctx->qout_cap = c1;
        }
        ids = ctx->qids;
        scores = ctx->qscores;
        cnt = ctx->qcount;
    }
    int32_t splits = 0;
    if (tc && nq > 0) {
        if (ctx->ehl_gen != ctx->qgen) {
            const int64_t np = query_tc_pad_rows(nq);
            CK(grow(ctx->ehl, ctx->ehl_cap, 2 * np * D, st));
            CK(grow(ctx->qinv, ctx->qinv_cap, np, st));
            launch_query_split_e(ctx->E, ctx->inv_norm, ctx->qrows, nq, ctx->D, ctx->ehl, ctx->qinv, st);
            ctx->ehl_gen = ctx->qgen;
        }
        CK(grow(ctx->qhl, ctx->qhl_cap, 2 * query_tc_pad_queries(B) * D, st));
        const int64_t ntiles = query_tc_tiles(nq);
        const int32_t d = std::min<int64_t>(query_tc_splits(B, nq), ntiles);
        auto it = ctx->qsplits.find({B, nq});
        if (it != ctx->qsplits.end()) {
            splits = it->second;
        } else if (ctx->autotune && (double)B * (double)nq >= 2e7) {
            // autotuner: time the default split, half and double (once per shape, after a warm run)
            const int32_t cands[3] = {d, std::max(1, d / 2), (int32_t)std::min<int64_t>(ntiles, 2 * (int64_t)d)};
            const int kk = k < 16 ? k : 16;
            const int64_t need = (int64_t)B * cands[2] * kk;
            if (need > ctx->cand_cap) {
                int64_t c1 = ctx->cand_cap, c2 = ctx->cand_cap;
                CK(grow(ctx->cand_s, c1, need, st));
                CK(grow(ctx->cand_i, c2, need, st));
                ctx->cand_cap = c1;
            }
            cudaEvent_t t0 = take_event(ctx), t1 = take_event(ctx);
            float best = INFINITY;
            int32_t pick = d;
            for (int32_t c : cands) {
                CK(launch_query_topk_tc(dQ, B, ctx->qhl, ctx->ehl, ctx->qinv, ctx->qrows, nq, ctx->D, k,
                                        ctx->cand_s, ctx->cand_i, ids, scores, cnt, ctx->tc_err, st, c));
                CK(cudaEventRecord(t0, st));
                CK(launch_query_topk_tc(dQ, B, ctx->qhl, ctx->ehl, ctx->qinv, ctx->qrows, nq, ctx->D, k,
                                        ctx->cand_s, ctx->cand_i, ids, scores, cnt, ctx->tc_err, st, c));
                CK(cudaEventRecord(t1, st));
                CK(cudaEventSynchronize(t1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, t0, t1));
                if (ms < best) { best = ms; pick = c; }
            }
            ctx->event_pool.push_back(t0);
            ctx->event_pool.push_back(t1);
            ctx->qsplits[{B, nq}] = pick;
            splits = pick;
        } else {
            splits = d;
        }
        const int64_t need = (int64_t)B * splits * (k < 16 ? k : 16);
        if (need > ctx->cand_cap) {
            int64_t c1 = ctx->cand_cap, c2 = ctx->cand_cap;
            CK(grow(ctx->cand_s, c1, need, st));
            CK(grow(ctx->cand_i, c2, need, st));
            ctx->cand_cap = c1;
        }
    }
    auto launch = [&](cudaStream_t s2) -> cudaError_t {
        if (tc)
            return launch_query_topk_tc(dQ, B, ctx->qhl, ctx->ehl, ctx->qinv, ctx->qrows, nq, ctx->D, k,
                                        ctx->cand_s, ctx->cand_i, ids, scores, cnt, ctx->tc_err, s2, splits);
        launch_query_topk(dQ, B, ctx->E, ctx->inv_norm, ctx->qrows, nq, ctx->D, k, ctx->cand_s, ctx->cand_i, ids,
                          scores, cnt, s2);
        return cudaGetLastError();
    };
    if (on_device && !((ctx->prof_mask >> SLAG_STAGE_QUERY) & 1u)) {
        // device buffers: the launches run as a CUDA graph on the query stream, captured for this
        // (buffers, shape, split, finalize) and replayed while they repeat
        const slag_ctx::QKey key{dQ, ids, scores, cnt, B, k, splits, nq, ctx->qgen};
        if (!ctx->qgraph || !(ctx->qkey == key)) {
            if (ctx->qgraph) { cudaGraphExecDestroy(ctx->qgraph); ctx->qgraph = nullptr; }
            cudaGraph_t graph = nullptr;
            const unsigned long long l0 = g_launches.load(std::memory_order_relaxed);
            CK(cudaStreamBeginCapture(ctx->qstream, cudaStreamCaptureModeRelaxed));
            const cudaError_t le = launch(ctx->qstream);
            CK(cudaStreamEndCapture(ctx->qstream, &graph));
            if (le != cudaSuccess) {
                cudaGraphDestroy(graph);
                CK(le);
            }
            // the capture counted its kernels once; replays count them below
            const unsigned long long l1 = g_launches.load(std::memory_order_relaxed);
            ctx->qgraph_launches = l1 - l0;
            g_launches.fetch_sub(l1 - l0, std::memory_order_relaxed);
            cudaError_t e = cudaGraphInstantiate(&ctx->qgraph, graph, 0);
            cudaGraphDestroy(graph);
            CK(e);
            ctx->qkey = key;
        }
        CK(cudaEventRecord(ctx->qev_in, st));
        CK(cudaStreamWaitEvent(ctx->qstream, ctx->qev_in, 0));
        CK(cudaGraphLaunch(ctx->qgraph, ctx->qstream));
        g_launches.fetch_add(ctx->qgraph_launches, std::memory_order_relaxed);
        CK(cudaEventRecord(ctx->qev_out, ctx->qstream));
        CK(cudaStreamWaitEvent(st, ctx->qev_out, 0));
    } else {
        span_begin(ctx, SLAG_STAGE_QUERY, st);
        const cudaError_t le = launch(st);
        span_end(ctx, st);
        CK(le);
    }
    CK(cudaGetLastError());
    launch_copy_words(ctx->tc_err, &ctx->hc_dev->tc_err, sizeof(uint32_t), st);
    if (!on_device) {
        // the results go through mapped staging written by the SMs, so that they do not queue
        // behind an earlier finalize's output copies on the copy engine
        const size_t bi = sizeof(int64_t) * (size_t)B * k, bs = sizeof(float) * (size_t)B * k,
                     bc = sizeof(int32_t) * (size_t)B;
        if ((int64_t)(bi + bs + bc) > ctx->qstage_cap) {
            if (ctx->qstage) cudaFreeHost(ctx->qstage);
            ctx->qstage = nullptr;
            ctx->qstage_cap = 0;
            const size_t cap = (bi + bs + bc) * 3 / 2;
            CK(cudaHostAlloc((void **)&ctx->qstage, cap, cudaHostAllocMapped));
            CK(cudaHostGetDevicePointer((void **)&ctx->qstage_dev, ctx->qstage, 0));
            ctx->qstage_cap = (int64_t)cap;
        }
        launch_copy_words(ids, ctx->qstage_dev, (int64_t)bi, st);
        launch_copy_words(scores, ctx->qstage_dev + bi, (int64_t)bs, st);
        launch_copy_words(cnt, ctx->qstage_dev + bi + bs, (int64_t)bc, st);
        CK(cudaStreamSynchronize(st));
        guard.st = nullptr;
        memcpy(out_ids, ctx->qstage, bi);
        memcpy(out_scores, ctx->qstage + bi, bs);
        if (out_count) memcpy(out_count, ctx->qstage + bi + bs, bc);
        if (ctx->hc->tc_err) return timeout_reported(ctx, "a tensor-core query kernel gave up waiting");
    }
    return SLAG_OK;
}

slag_status slag_query_threshold(slag_ctx *ctx, const float *q, float threshold, int64_t *out_ids, int64_t cap,
                                 int64_t *out_count, int32_t on_device) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    if (!ctx->finalized) return fail(ctx, SLAG_ERR_STATE, "query before finalize");
    if (!q || (!out_ids && cap > 0) || cap < 0 || !out_count)
        return fail(ctx, SLAG_ERR_INVALID_ARG, "NULL query or output, or cap < 0");
    if (!std::isfinite(threshold)) return fail(ctx, SLAG_ERR_INVALID_ARG, "threshold is not finite");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int64_t D = ctx->D, nq = ctx->n_q;
    struct StreamGuard {
        cudaStream_t st = nullptr;
        ~StreamGuard() {
            if (st) cudaStreamSynchronize(st);
        }
    } guard;
    const float *dq = q;
    if (!on_device) {
        CK(grow(ctx->qbuf, ctx->qbuf_cap, D, st));
        CK(cudaMemcpyAsync(ctx->qbuf, q, sizeof(float) * (size_t)D, cudaMemcpyHostToDevice, st));
        guard.st = st;
        dq = ctx->qbuf;
    }
    if (((uintptr_t)dq & 15u) != 0) return fail(ctx, SLAG_ERR_INVALID_ARG, "q must be 16-byte aligned");
    // flags and positions per candidate: the finalize's n-sized scratch (n_q <= n), free after it
    if (!ctx->d_thr) CK(dalloc(&ctx->d_thr, 1));
    int64_t *dids = out_ids;
    if (!on_device && cap > 0) {
        CK(grow(ctx->thr_ids, ctx->thr_cap, cap, st));
        dids = ctx->thr_ids;
    }
    CK(scratch_reserve(ctx->scratch, nq));
    launch_threshold_query(dq, ctx->E, ctx->inv_norm, ctx->qrows, nq, ctx->D, threshold, ctx->qflags, ctx->qpos,
                           ctx->d_thr, cap, dids, ctx->scratch, st);
    unsigned long long total = 0;
    CK(cudaMemcpyAsync(&total, ctx->d_thr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    *out_count = (int64_t)total;
    const int64_t got = std::min<int64_t>((int64_t)total, cap);
    if (!on_device && got > 0) {
        CK(cudaMemcpyAsync(out_ids, dids, sizeof(int64_t) * (size_t)got, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return SLAG_OK;
}

slag_status slag_query(slag_ctx *ctx, const float *q, int32_t k, int64_t *out_ids, float *out_scores,
                       int32_t *out_count) {
    return slag_query_batch(ctx, q, 1, k, out_ids, out_scores, out_count, 0);
}

slag_status slag_reset(slag_ctx *ctx) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->n;
    ctx->deferred = false;   // the last view's second half is dropped with the rest
    CK(join_views(ctx));
    for (int i = 0; i < kSlots; ++i) ctx->slot[i].pending = ctx->slot[i].count_at_settle = false;   // dropped too
    // a view that failed after its first half can leave entries in its slot's table
    for (int i = 0; i < kSlots; ++i) {
        launch_hash_init(ctx->slot[i].hash, n, st);
        CK(cudaMemsetAsync(ctx->slot[i].ctr, 0, sizeof(ViewCounters), st));
        ctx->slot[i].log_bound = 0;
    }
    CK(cudaMemsetAsync(ctx->s_hi, 0, sizeof(float) * n, st));
    CK(cudaMemsetAsync(ctx->s_lo, 0, sizeof(float) * n, st));
    CK(cudaMemsetAsync(ctx->s_ovf, 0, sizeof(float) * n, st));
    CK(cudaMemsetAsync(ctx->totals, 0, kTotals * sizeof(unsigned long long), st));
    CK(cudaGetLastError());
    ctx->views_enqueued = 0;
    ctx->table_rows = 0;
    ctx->log_fill_seen = 0;
    ctx->log_overflowed = false;
    ctx->finalized = false;
    ctx->hc->v = ViewCounters{};
    ctx->stats = slag_stats{};
    return SLAG_OK;
}

slag_status slag_export_partitions(slag_ctx *ctx, const char *dir, int32_t cells_x, int32_t cells_y,
                                   int64_t chunk_gaussians, int64_t *out_written) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    if (!dir || !dir[0]) return fail(ctx, SLAG_ERR_INVALID_ARG, "no directory");
    if (cells_x < 1 || cells_y < 1 || (int64_t)cells_x * cells_y > (1 << 20))
        return fail(ctx, SLAG_ERR_INVALID_ARG, "grid must have 1 .. 2^20 cells");
    if (out_written) *out_written = 0;
    slag_status s = finalize_prepare(ctx);
    if (s != SLAG_OK) return s;
    if (mkdir(dir, 0755) != 0 && errno != EEXIST)
        return fail(ctx, SLAG_ERR_INVALID_ARG, std::string("cannot create ") + dir);
    const int64_t n = ctx->n;
    const int32_t D = ctx->D;
    // x-y bounds of all means
    std::vector<float4> means((size_t)n);
    CK(cudaMemcpyAsync(means.data(), ctx->mean_op, sizeof(float4) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (const float4 &m : means) {
        x0 = fminf(x0, m.x); x1 = fmaxf(x1, m.x);
        y0 = fminf(y0, m.y); y1 = fmaxf(y1, m.y);
    }
    const float sx = x1 > x0 ? (float)cells_x / (x1 - x0) : 0.f, sy = y1 > y0 ? (float)cells_y / (y1 - y0) : 0.f;
    const float cwx = x1 > x0 ? (x1 - x0) / (float)cells_x : 0.f, cwy = y1 > y0 ? (y1 - y0) / (float)cells_y : 0.f;
    const size_t ncell = (size_t)cells_x * (size_t)cells_y;
    const size_t rec_bytes = 8 + 4 + 4 * (size_t)D;
    const size_t hdr_bytes = 8 + 4 + 4 + 8 + 16;
    std::vector<int64_t> count(ncell, 0);
    std::vector<std::vector<char>> pend(ncell);
    auto path_of = [&](size_t c) {
        return std::string(dir) + "/cell_" + std::to_string(c % cells_x) + "_" + std::to_string(c / cells_x) + ".slag";
    };
    auto flush = [&](size_t c) -> bool {
        if (pend[c].empty()) return true;
        const std::string p = path_of(c);
        FILE *f = fopen(p.c_str(), count[c] == (int64_t)(pend[c].size() / rec_bytes) ? "wb" : "ab");
        if (!f) return false;
        bool ok = true;
        if (count[c] == (int64_t)(pend[c].size() / rec_bytes)) {   // new file: header with count 0 for now
            const uint32_t ver = 1, d = (uint32_t)D;
            const int64_t zero = 0;
            const float b[4] = {x0 + cwx * (float)(c % cells_x), x0 + cwx * (float)(c % cells_x + 1),
                                y0 + cwy * (float)(c / cells_x), y0 + cwy * (float)(c / cells_x + 1)};
            ok = fwrite("SLAGPART", 1, 8, f) == 8 && fwrite(&ver, 4, 1, f) == 1 && fwrite(&d, 4, 1, f) == 1 &&
                 fwrite(&zero, 8, 1, f) == 1 && fwrite(b, 4, 4, f) == 4;
        }
        ok = ok && fwrite(pend[c].data(), 1, pend[c].size(), f) == pend[c].size();
        ok = (fclose(f) == 0) && ok;
        pend[c].clear();
        return ok;
    };
    int64_t written = 0;
    s = aggregate_chunks(ctx, chunk_gaussians > 0 ? chunk_gaussians : (int64_t)1 << 20, [&](const ChunkView &v) {
        std::vector<size_t> touched_cells;
        for (int64_t r = 0; r < v.rows; ++r) {
            const uint32_t id = v.ids[r];
            if (id == 0xffffffffu || !(v.wsum[r] > 0.f)) continue;
            int cx = (int)floorf((v.means[r].x - x0) * sx), cy = (int)floorf((v.means[r].y - y0) * sy);
            cx = cx < 0 ? 0 : (cx >= cells_x ? cells_x - 1 : cx);
            cy = cy < 0 ? 0 : (cy >= cells_y ? cells_y - 1 : cy);
            const size_t c = (size_t)cy * cells_x + cx;
            std::vector<char> &buf = pend[c];
            if (buf.empty()) touched_cells.push_back(c);
            const size_t at = buf.size();
            buf.resize(at + rec_bytes);
            const int64_t id64 = id;
            memcpy(buf.data() + at, &id64, 8);
            memcpy(buf.data() + at + 8, &v.wsum[r], 4);
            memcpy(buf.data() + at + 12, v.E + r * D, 4 * (size_t)D);
            ++count[c];
            ++written;
        }
        for (size_t c : touched_cells)
            if (!flush(c)) return fail(ctx, SLAG_ERR_CUDA, "cannot write " + path_of(c));
        return SLAG_OK;
    });
    if (s != SLAG_OK) return s;
    // final counts in the headers, and the index
    FILE *idx = fopen((std::string(dir) + "/index.txt").c_str(), "w");
    if (!idx) return fail(ctx, SLAG_ERR_CUDA, std::string("cannot write ") + dir + "/index.txt");
    for (size_t c = 0; c < ncell; ++c) {
        if (!count[c]) continue;
        FILE *f = fopen(path_of(c).c_str(), "r+b");
        bool ok = f && fseek(f, 16, SEEK_SET) == 0 && fwrite(&count[c], 8, 1, f) == 1;
        if (f) ok = (fclose(f) == 0) && ok;
        if (!ok) {
            fclose(idx);
            return fail(ctx, SLAG_ERR_CUDA, "cannot write " + path_of(c));
        }
        fprintf(idx, "%zu %zu %lld %.9g %.9g %.9g %.9g cell_%zu_%zu.slag\n", c % cells_x, c / cells_x,
                (long long)count[c], x0 + cwx * (float)(c % cells_x), x0 + cwx * (float)(c % cells_x + 1),
                y0 + cwy * (float)(c / cells_x), y0 + cwy * (float)(c / cells_x + 1), c % cells_x, c / cells_x);
    }
    if (fclose(idx) != 0) return fail(ctx, SLAG_ERR_CUDA, std::string("cannot write ") + dir + "/index.txt");
    (void)hdr_bytes;
    if (out_written) *out_written = written;
    return SLAG_OK;
}

// ---- accumulated state: save, load, merge --------------------------------------------------

}  // extern "C"

namespace {

// Serialised state (little-endian), see slag_save_state in slag.h.
struct StateHeader {
    char magic[8];                 // "SLAGSTAT"
    uint32_t version;              // 1
    uint32_t dim;
    int64_t n;
    int64_t columns;
    int64_t triples;
    uint64_t fingerprint;          // of the Gaussian set the state belongs to
    int64_t views, pairs, contributions, evaluations, executed;
    int32_t weight_mode;
    int32_t reserved;
};
static_assert(sizeof(StateHeader) == 96, "state header layout");
constexpr char kStateMagic[8] = {'S', 'L', 'A', 'G', 'S', 'T', 'A', 'T'};

int64_t state_bytes(int64_t n, int64_t D, int64_t columns, int64_t triples) {
    return (int64_t)sizeof(StateHeader) + 4 * columns * D + 12 * n + 12 * triples;
}

// Whether buf holds a well-formed state of `bytes` bytes; fills *h.
bool parse_state(const void *buf, int64_t bytes, StateHeader *h) {
    if (!buf || bytes < (int64_t)sizeof(StateHeader)) return false;
    memcpy(h, buf, sizeof(StateHeader));
    if (memcmp(h->magic, kStateMagic, 8) != 0 || h->version != 1) return false;
    if (h->n < 1 || h->dim < 1 || h->columns < 0 || h->triples < 0 || h->columns >= (1LL << 32)) return false;
    return state_bytes(h->n, h->dim, h->columns, h->triples) == bytes;
}

// FNV-1a over the Gaussian set in the context's internal layout (deterministic for a given input).
slag_status gaussian_fingerprint(slag_ctx *ctx, uint64_t *out) {
    const int64_t n = ctx->n;
    std::vector<float4> a((size_t)n), b((size_t)n);
    std::vector<float2> c((size_t)n);
    CK(cudaMemcpyAsync(a.data(), ctx->mean_op, sizeof(float4) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(b.data(), ctx->cov_a, sizeof(float4) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(c.data(), ctx->cov_b, sizeof(float2) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    uint64_t hsh = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t len) {
        const unsigned char *q = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < len; ++i) hsh = (hsh ^ q[i]) * 1099511628211ull;
    };
    mix(&n, sizeof(n));
    mix(a.data(), sizeof(float4) * (size_t)n);
    mix(b.data(), sizeof(float4) * (size_t)n);
    mix(c.data(), sizeof(float2) * (size_t)n);
    *out = hsh;
    return SLAG_OK;
}

// Joins every view in flight and reads the device totals into ctx->hc->totals.
slag_status join_and_read_totals(slag_ctx *ctx) {
    cudaStream_t st = ctx->stream;
    slag_status s = launch_deferred_view(ctx);
    if (s == SLAG_OK) s = settle_views(ctx);
    if (s != SLAG_OK) return s;
    CK(join_views(ctx));
    launch_copy_words(ctx->totals, ctx->hc_dev->totals, kTotals * sizeof(unsigned long long), st);
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    ctx->log_fill_seen = (int64_t)ctx->hc->totals[0];
    if (ctx->hc->totals[2]) ctx->log_overflowed = true;
    if (ctx->log_overflowed) return fail(ctx, SLAG_ERR_CAPACITY, "the triple log overflowed in some view");
    return SLAG_OK;
}

}  // namespace

extern "C" {

slag_status slag_save_state(slag_ctx *ctx, void *buf, int64_t cap, int64_t *out_bytes) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    slag_status s = join_and_read_totals(ctx);
    if (s != SLAG_OK) return s;
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->n, D = ctx->D, cols = ctx->table_rows;
    const int64_t Z = (int64_t)ctx->hc->totals[0];
    const int64_t need = state_bytes(n, D, cols, Z);
    if (out_bytes) *out_bytes = need;
    if (!buf) return SLAG_OK;
    if (cap < need) return fail(ctx, SLAG_ERR_CAPACITY, "state buffer smaller than the state");
    StateHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kStateMagic, 8);
    h.version = 1;
    h.dim = (uint32_t)D;
    h.n = n;
    h.columns = cols;
    h.triples = Z;
    s = gaussian_fingerprint(ctx, &h.fingerprint);
    if (s != SLAG_OK) return s;
    h.views = ctx->stats.views;
    h.pairs = ctx->stats.pairs;
    h.contributions = (int64_t)ctx->hc->totals[1];
    h.evaluations = (int64_t)ctx->hc->totals[3];
    h.executed = (int64_t)ctx->hc->totals[4];
    h.weight_mode = ctx->weight_mode;
    char *out = static_cast<char *>(buf);
    memcpy(out, &h, sizeof(h));
    char *p = out + sizeof(h);
    // the stored segment embeddings
    if (cols > 0) CK(cudaMemcpyAsync(p, ctx->table, sizeof(float) * (size_t)(cols * D), cudaMemcpyDeviceToHost, st));
    p += 4 * cols * D;
    // the compensated sums in caller order
    std::vector<float> hi((size_t)n), lo((size_t)n), ovf((size_t)n);
    std::vector<uint32_t> orig((size_t)n);
    CK(cudaMemcpyAsync(hi.data(), ctx->s_hi, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(lo.data(), ctx->s_lo, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(ovf.data(), ctx->s_ovf, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(orig.data(), ctx->orig_of_int, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, st));
    // the triples: (caller index, column) unpacked on the device, then W
    uint32_t *dg = nullptr, *dc = nullptr;
    if (Z > 0) {
        cudaError_t e = dalloc(&dg, Z);
        if (e == cudaSuccess) e = dalloc(&dc, Z);
        if (e != cudaSuccess) {
            dfree(dg); dfree(dc);
            return fail(ctx, SLAG_ERR_OOM, "state: triple staging");
        }
        launch_state_unpack(ctx->log_key, Z, ctx->orig_of_int, dg, dc, st);
    }
    CK(cudaStreamSynchronize(st));
    float *fs = reinterpret_cast<float *>(p);
    for (int64_t g = 0; g < n; ++g) {
        const uint32_t c = orig[(size_t)g];
        fs[c] = hi[(size_t)g];
        fs[n + c] = lo[(size_t)g];
        fs[2 * n + c] = ovf[(size_t)g];
    }
    p += 12 * n;
    cudaError_t e = cudaSuccess;
    if (Z > 0) {
        e = cudaMemcpyAsync(p, dg, sizeof(uint32_t) * (size_t)Z, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p + 4 * Z, dc, sizeof(uint32_t) * (size_t)Z, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p + 8 * Z, ctx->log_w, sizeof(float) * (size_t)Z, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    dfree(dg);
    dfree(dc);
    if (e != cudaSuccess) return fail(ctx, SLAG_ERR_CUDA, cudaGetErrorString(e));
    return SLAG_OK;
}

slag_status slag_merge_state(slag_ctx *ctx, const void *buf, int64_t bytes) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    StateHeader h;
    if (!parse_state(buf, bytes, &h)) return fail(ctx, SLAG_ERR_INVALID_ARG, "not a state of this library");
    if (h.n != ctx->n || (int64_t)h.dim != ctx->D) return fail(ctx, SLAG_ERR_INVALID_ARG, "state of another n or dim");
    if (h.weight_mode != ctx->weight_mode) return fail(ctx, SLAG_ERR_INVALID_ARG, "state of another weight mode");
    CK(cudaSetDevice(ctx->device));
    uint64_t fp = 0;
    slag_status s = gaussian_fingerprint(ctx, &fp);
    if (s != SLAG_OK) return s;
    if (fp != h.fingerprint) return fail(ctx, SLAG_ERR_INVALID_ARG, "state of another Gaussian set");
    if (ctx->table_rows + h.columns >= (1LL << 32)) return fail(ctx, SLAG_ERR_CAPACITY, "more than 2^32 segment columns");
    s = join_and_read_totals(ctx);
    if (s != SLAG_OK) return s;
    cudaStream_t st = ctx->stream;
    const int64_t n = ctx->n, D = ctx->D;
    const int64_t used = (int64_t)ctx->hc->totals[0];
    const int64_t Zb = h.triples;
    const char *p = static_cast<const char *>(buf) + sizeof(StateHeader);
    // segment embeddings after the context's own
    if (h.columns > 0) {
        if (ctx->table_rows + h.columns > ctx->table_cap / D)
            CK(grow(ctx->table, ctx->table_cap, (ctx->table_rows + h.columns) * D, st, ctx->table_rows * D));
        CK(cudaMemcpyAsync(ctx->table + ctx->table_rows * D, p, sizeof(float) * (size_t)(h.columns * D),
                           cudaMemcpyHostToDevice, st));
    }
    p += 4 * h.columns * D;
    // sums: caller order -> internal order, added with compensation
    std::vector<uint32_t> orig((size_t)n);
    CK(cudaMemcpyAsync(orig.data(), ctx->orig_of_int, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<float> sums((size_t)(3 * n));
    const float *fs = reinterpret_cast<const float *>(p);
    for (int64_t g = 0; g < n; ++g) {
        const uint32_t c = orig[(size_t)g];
        sums[(size_t)g] = fs[c];
        sums[(size_t)(n + g)] = fs[n + c];
        sums[(size_t)(2 * n + g)] = fs[2 * n + c];
    }
    p += 12 * n;
    float *dsum = nullptr;
    uint32_t *dg = nullptr, *dc = nullptr, *dbad = nullptr;
    float *dw = nullptr;
    auto release = [&]() { dfree(dsum); dfree(dg); dfree(dc); dfree(dw); dfree(dbad); };
    cudaError_t e = dalloc(&dsum, 3 * n);
    if (e == cudaSuccess) e = dalloc(&dbad, 1);
    if (e == cudaSuccess && Zb > 0) e = dalloc(&dg, Zb);
    if (e == cudaSuccess && Zb > 0) e = dalloc(&dc, Zb);
    if (e == cudaSuccess && Zb > 0) e = dalloc(&dw, Zb);
    // room in the log for the other state's triples
    if (e == cudaSuccess && used + Zb > ctx->log_cap) {
        int64_t c1 = ctx->log_cap, c2 = ctx->log_cap;
        e = grow(ctx->log_key, c1, used + Zb, st, used);
        if (e == cudaSuccess) e = grow(ctx->log_w, c2, used + Zb, st, used);
        if (e == cudaSuccess) ctx->log_cap = c1;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(dsum, sums.data(), sizeof(float) * (size_t)(3 * n), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dbad, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess && Zb > 0) {
        e = cudaMemcpyAsync(dg, p, sizeof(uint32_t) * (size_t)Zb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dc, p + 4 * Zb, sizeof(uint32_t) * (size_t)Zb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dw, p + 8 * Zb, sizeof(float) * (size_t)Zb, cudaMemcpyHostToDevice, st);
    }
    uint32_t bad = 0;
    if (e == cudaSuccess) {
        launch_state_pack(dg, dc, dw, Zb, ctx->int_of_orig, n, (uint32_t)ctx->table_rows, (uint32_t)h.columns,
                          ctx->log_key + used, ctx->log_w + used, dbad, st);
        launch_state_sums(ctx->s_hi, ctx->s_lo, ctx->s_ovf, dsum, dsum + n, dsum + 2 * n, n, st);
        // the device totals: triples in the log and the counters the state carries
        unsigned long long *tot = ctx->hc->totals;
        tot[0] = (unsigned long long)(used + Zb);
        ctx->log_fill_seen = used + Zb;
        tot[1] += (unsigned long long)h.contributions;
        tot[3] += (unsigned long long)h.evaluations;
        tot[4] += (unsigned long long)h.executed;
        e = cudaMemcpyAsync(ctx->totals, tot, kTotals * sizeof(unsigned long long), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, dbad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    release();
    if (e != cudaSuccess)
        return fail(ctx, e == cudaErrorMemoryAllocation ? SLAG_ERR_OOM : SLAG_ERR_CUDA, cudaGetErrorString(e));
    ctx->table_rows += h.columns;
    ctx->stats.views += h.views;
    ctx->stats.columns = ctx->table_rows;
    ctx->stats.pairs += h.pairs;
    ctx->finalized = false;
    if (bad) return fail(ctx, SLAG_ERR_INVALID_ARG, "state: a triple names a Gaussian or column out of range "
                                                    "(its weight was dropped; reset the context)");
    return SLAG_OK;
}

slag_status slag_load_state(slag_ctx *ctx, const void *buf, int64_t bytes) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    StateHeader h;
    if (!parse_state(buf, bytes, &h)) return fail(ctx, SLAG_ERR_INVALID_ARG, "not a state of this library");
    slag_status s = slag_reset(ctx);
    if (s != SLAG_OK) return s;
    return slag_merge_state(ctx, buf, bytes);
}

slag_status slag_state_merge_host(const void *a, int64_t a_bytes, const void *b, int64_t b_bytes, void *out,
                                  int64_t cap, int64_t *out_bytes) {
    StateHeader ha, hb;
    if (!parse_state(a, a_bytes, &ha) || !parse_state(b, b_bytes, &hb)) return SLAG_ERR_INVALID_ARG;
    if (ha.n != hb.n || ha.dim != hb.dim || ha.fingerprint != hb.fingerprint || ha.weight_mode != hb.weight_mode)
        return SLAG_ERR_INVALID_ARG;
    if (ha.columns + hb.columns >= (1LL << 32)) return SLAG_ERR_CAPACITY;
    const int64_t n = ha.n, D = ha.dim, ca = ha.columns, cb = hb.columns, za = ha.triples, zb = hb.triples;
    const int64_t need = state_bytes(n, D, ca + cb, za + zb);
    if (out_bytes) *out_bytes = need;
    if (!out) return SLAG_OK;
    if (cap < need) return SLAG_ERR_CAPACITY;
    StateHeader h = ha;
    h.columns = ca + cb;
    h.triples = za + zb;
    h.views += hb.views;
    h.pairs += hb.pairs;
    h.contributions += hb.contributions;
    h.evaluations += hb.evaluations;
    h.executed += hb.executed;
    const char *pa = static_cast<const char *>(a) + sizeof(StateHeader);
    const char *pb = static_cast<const char *>(b) + sizeof(StateHeader);
    char *po = static_cast<char *>(out);
    memcpy(po, &h, sizeof(h));
    po += sizeof(h);
    memcpy(po, pa, (size_t)(4 * ca * D));
    memcpy(po + 4 * ca * D, pb, (size_t)(4 * cb * D));
    po += 4 * (ca + cb) * D;
    pa += 4 * ca * D;
    pb += 4 * cb * D;
    const float *sa = reinterpret_cast<const float *>(pa), *sb = reinterpret_cast<const float *>(pb);
    float *so = reinterpret_cast<float *>(po);
    for (int64_t g = 0; g < n; ++g) {
        const float x = sa[g], y = sb[g];
        const float t = x + y;
        const float err = std::fabs(x) >= std::fabs(y) ? (x - t) + y : (y - t) + x;
        so[g] = t;
        so[n + g] = (sa[n + g] + sb[n + g]) + err;
        so[2 * n + g] = sa[2 * n + g] + sb[2 * n + g];
    }
    po += 12 * n;
    pa += 12 * n;
    pb += 12 * n;
    // triples: a's, then b's with columns shifted past a's
    uint32_t *og = reinterpret_cast<uint32_t *>(po), *oc = og + (za + zb);
    float *ow = reinterpret_cast<float *>(oc + (za + zb));
    const uint32_t *ag = reinterpret_cast<const uint32_t *>(pa), *ac = ag + za;
    const float *aw = reinterpret_cast<const float *>(ac + za);
    const uint32_t *bg = reinterpret_cast<const uint32_t *>(pb), *bc = bg + zb;
    const float *bw = reinterpret_cast<const float *>(bc + zb);
    memcpy(og, ag, (size_t)(4 * za));
    memcpy(og + za, bg, (size_t)(4 * zb));
    memcpy(oc, ac, (size_t)(4 * za));
    for (int64_t i = 0; i < zb; ++i) oc[za + i] = bc[i] + (uint32_t)ca;
    memcpy(ow, aw, (size_t)(4 * za));
    memcpy(ow + za, bw, (size_t)(4 * zb));
    return SLAG_OK;
}

slag_status slag_set_device_budget(slag_ctx *ctx, int64_t bytes) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    if (bytes < 0) return fail(ctx, SLAG_ERR_INVALID_ARG, "budget < 0");
    // a chunk's device rows: E (4 D bytes), sum w and the caller index (4 bytes each)
    const int64_t per_row = 4 * (int64_t)ctx->D + 8;
    int64_t rows = bytes > 0 ? bytes / per_row : ((int64_t)1 << 20);
    rows = rows / kBlockG * kBlockG;
    if (rows < kBlockG) rows = kBlockG;
    ctx->chunk_gaussians = rows;
    return SLAG_OK;
}

slag_status slag_set_linear_code(slag_ctx *ctx, const float *params) {
    if (!ctx || !params) return SLAG_ERR_INVALID_ARG;
    if (ctx->precision != SLAG_PREC_LINEAR32) return fail(ctx, SLAG_ERR_STATE, "context is not SLAG_PREC_LINEAR32");
    if (ctx->stats.views > 0) return fail(ctx, SLAG_ERR_STATE, "slag_set_linear_code before the first view");
    CK(cudaSetDevice(ctx->device));
    const int64_t D = ctx->D, P = linear_param_count(ctx->D);
    for (int64_t i = 0; i < P; ++i)
        if (!std::isfinite(params[i])) return fail(ctx, SLAG_ERR_INVALID_ARG, "linear code: non-finite parameter");
    // the encoder's constant: -mu U
    std::vector<float> bias((size_t)kLatent);
    for (int j = 0; j < kLatent; ++j) {
        double acc = 0.0;
        for (int64_t d = 0; d < D; ++d) acc += (double)params[D * kLatent + d] * (double)params[d * kLatent + j];
        bias[(size_t)j] = (float)-acc;
    }
    if (!ctx->lin_params) CK(dalloc(&ctx->lin_params, P));
    if (!ctx->lin_enc_bias) CK(dalloc(&ctx->lin_enc_bias, kLatent));
    CK(cudaMemcpyAsync(ctx->lin_params, params, sizeof(float) * (size_t)P, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->lin_enc_bias, bias.data(), sizeof(float) * kLatent, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SLAG_OK;
}

slag_status slag_set_latent(slag_ctx *ctx, const float *params) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    if (!params) return fail(ctx, SLAG_ERR_INVALID_ARG, "params is NULL");
    if (ctx->precision != SLAG_PREC_LATENT32) return fail(ctx, SLAG_ERR_STATE, "context not created with SLAG_PREC_LATENT32");
    if (ctx->stats.views > 0) return fail(ctx, SLAG_ERR_STATE, "slag_set_latent after the first view");
    CK(cudaSetDevice(ctx->device));
    const int64_t P = latent_layout(ctx->D).total;
    if (!ctx->lat_params) CK(dalloc(&ctx->lat_params, P));
    CK(cudaMemcpyAsync(ctx->lat_params, params, sizeof(float) * (size_t)P, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SLAG_OK;
}

slag_status slag_add_views_batched(int32_t n_ctx, slag_ctx *const *ctxs, const slag_view *const *views,
                                   const int32_t *n_views, int32_t *failed_ctx) {
    if (failed_ctx) *failed_ctx = -1;
    if (n_ctx < 0 || (n_ctx > 0 && (!ctxs || !views || !n_views))) return SLAG_ERR_INVALID_ARG;
    for (int32_t c = 0; c < n_ctx; ++c) {
        if (!ctxs[c] || n_views[c] < 0 || (n_views[c] > 0 && !views[c])) {
            if (failed_ctx) *failed_ctx = c;
            return SLAG_ERR_INVALID_ARG;
        }
    }
    // scene after scene: each context's own pipeline keeps the GPU busy, and its last view's
    // second half is queued before the next scene starts
    for (int32_t c = 0; c < n_ctx; ++c) {
        slag_status s = SLAG_OK;
        for (int32_t v = 0; v < n_views[c] && s == SLAG_OK; ++v) {
            const slag_view &w = views[c][v];
            s = slag_add_view(ctxs[c], w.camera, w.seg_ids, w.seg_table, w.M, w.on_device);
        }
        if (s == SLAG_OK && n_views[c] > 0) {
            slag_ctx *ctx = ctxs[c];
            if (cudaSetDevice(ctx->device) != cudaSuccess) s = fail(ctx, SLAG_ERR_CUDA, "cudaSetDevice");
            else s = launch_deferred_view(ctx);
        }
        if (s != SLAG_OK) {
            if (failed_ctx) *failed_ctx = c;
            return s;
        }
    }
    return SLAG_OK;
}

slag_status slag_set_graphs(slag_ctx *ctx, int32_t enable) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    ctx->graphs = enable != 0;
    return SLAG_OK;
}

slag_status slag_set_autotune(slag_ctx *ctx, int32_t enable) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    ctx->autotune = enable != 0;
    if (!ctx->autotune) ctx->qsplits.clear();
    return SLAG_OK;
}

uint64_t slag_kernel_launches(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

slag_status slag_debug_force_pair_capacity(slag_ctx *ctx, int64_t cap) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    if (!kChecked) return fail(ctx, SLAG_ERR_STATE, "not a checked build (-DSLAG_CHECKS)");
    if (cap < 0) return fail(ctx, SLAG_ERR_INVALID_ARG, "cap < 0");
    ctx->force_pair_cap = cap;
    return SLAG_OK;
}

int32_t slag_is_checked_build(void) { return kChecked ? 1 : 0; }

slag_status slag_check_wait_timeout(slag_ctx *ctx, int32_t limit_us, int32_t complete) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    if (limit_us < 1 || limit_us > 1000000) return fail(ctx, SLAG_ERR_INVALID_ARG, "limit_us outside 1 .. 1,000,000");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    slag_status s = launch_deferred_view(ctx);
    if (s == SLAG_OK) s = settle_views(ctx);
    if (s != SLAG_OK) return s;
    CK(join_views(ctx));
    launch_wait_check((uint64_t)limit_us * 1000ull, complete ? 1 : 0, ctx->tc_err, st);
    launch_copy_words(ctx->tc_err, &ctx->hc_dev->tc_err, sizeof(uint32_t), st);
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if (ctx->hc->tc_err) return timeout_reported(ctx, "a bounded mbarrier wait gave up (wait check)");
    return SLAG_OK;
}

slag_status slag_get_stats(const slag_ctx *ctx, slag_stats *out) {
    if (!ctx || !out) return SLAG_ERR_INVALID_ARG;
    *out = ctx->stats;
    return SLAG_OK;
}

const char *slag_last_error(const slag_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

void slag_destroy(slag_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream); else cudaDeviceSynchronize();
    if (ctx->up) cudaStreamSynchronize(ctx->up);
    for (int i = 0; i < kSlots; ++i) {
        if (ctx->slot[i].front) cudaStreamSynchronize(ctx->slot[i].front);
        if (ctx->slot[i].back) cudaStreamSynchronize(ctx->slot[i].back);
    }
    for (int i = 0; i < kSlots; ++i) slot_free(ctx->slot[i]);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->up) cudaStreamDestroy(ctx->up);
    if (ctx->ev_consumed) cudaEventDestroy(ctx->ev_consumed);
    if (ctx->qgraph) cudaGraphExecDestroy(ctx->qgraph);
    if (ctx->qstream) { cudaStreamSynchronize(ctx->qstream); cudaStreamDestroy(ctx->qstream); }
    if (ctx->qev_in) cudaEventDestroy(ctx->qev_in);
    if (ctx->qev_out) cudaEventDestroy(ctx->qev_out);
    if (ctx->cstream) { cudaStreamSynchronize(ctx->cstream); cudaStreamDestroy(ctx->cstream); }
    if (ctx->ev_fin) cudaEventDestroy(ctx->ev_fin);
    for (int b = 0; b < 2; ++b)
        if (ctx->ev_copy[b]) cudaEventDestroy(ctx->ev_copy[b]);
    ctx->E = ctx->wsum = nullptr;
    for (int b = 0; b < 2; ++b) { dfree(ctx->E_buf[b]); dfree(ctx->wsum_buf[b]); }
    dfree(ctx->mean_op); dfree(ctx->cov_a); dfree(ctx->cov_b); dfree(ctx->log2_op);
    dfree(ctx->orig_of_int); dfree(ctx->int_of_orig);
    dfree(ctx->s_hi); dfree(ctx->s_lo); dfree(ctx->s_ovf);
    dfree(ctx->dbg_T); dfree(ctx->dbg_wsum); dfree(ctx->dbg_count);
    dfree(ctx->totals); dfree(ctx->touched); dfree(ctx->tc_err);
    dfree(ctx->log_key); dfree(ctx->log_key_alt); dfree(ctx->log_w); dfree(ctx->log_w_alt);
    dfree(ctx->flags); dfree(ctx->uidx); dfree(ctx->ucol); dfree(ctx->ustart); dfree(ctx->bstart); dfree(ctx->bend);
    dfree(ctx->table); dfree(ctx->inv_norm);
    dfree(ctx->qrows); dfree(ctx->qflags); dfree(ctx->qpos); dfree(ctx->d_nq); dfree(ctx->d_thr); dfree(ctx->thr_ids);
    dfree(ctx->lat_params); dfree(ctx->lin_params); dfree(ctx->lin_enc_bias); dfree(ctx->ztable); dfree(ctx->lat_hidden); dfree(ctx->lat_Z); dfree(ctx->lat_Y);
    dfree(ctx->ehl); dfree(ctx->qinv); dfree(ctx->qhl);
    dfree(ctx->qbuf); dfree(ctx->cand_s); dfree(ctx->cand_i); dfree(ctx->qids); dfree(ctx->qscores); dfree(ctx->qcount);
    scratch_free(ctx->scratch);
    for (auto &sp : ctx->spans) { cudaEventDestroy(sp.a); cudaEventDestroy(sp.b); }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->prof_base) cudaEventDestroy(ctx->prof_base);
    if (ctx->hc) cudaFreeHost(ctx->hc);
    if (ctx->qstage) cudaFreeHost(ctx->qstage);
    delete ctx;
}

slag_status slag_set_profiling_stages(slag_ctx *ctx, uint32_t stages) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    stages &= (1u << SLAG_STAGE_COUNT) - 1;
    if (stages && !ctx->prof_mask) {
        if (!ctx->prof_base) CK(cudaEventCreate(&ctx->prof_base));
        // events for a full backlog of spans, created here rather than inside the timed work
        while (ctx->event_pool.size() < 2 * kSpanBacklog + 64) {
            cudaEvent_t e = nullptr;
            CK(cudaEventCreate(&e));
            ctx->event_pool.push_back(e);
        }
        CK(cudaEventRecord(ctx->prof_base, ctx->stream));
        for (auto &b : ctx->busy) b.clear();
    }
    ctx->prof_mask = stages;
    return SLAG_OK;
}

slag_status slag_set_profiling(slag_ctx *ctx, int32_t enable) {
    return slag_set_profiling_stages(ctx, enable ? (1u << SLAG_STAGE_COUNT) - 1 : 0u);
}

slag_status slag_get_profile(slag_ctx *ctx, slag_profile *out, int32_t reset) {
    if (!ctx || !out) return SLAG_ERR_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    slag_status s0 = launch_deferred_view(ctx);
    if (s0 == SLAG_OK) s0 = settle_views(ctx);
    if (s0 != SLAG_OK) return s0;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(drain_views(ctx));
    spans_resolve(ctx);
    for (int s = 0; s < SLAG_STAGE_COUNT; ++s) {
        // union of the stage's intervals
        auto &v = ctx->busy[s];
        std::sort(v.begin(), v.end());
        double total = 0.0, lo = 0.0, hi = -1.0;
        for (const auto &iv : v) {
            if (iv.first > hi) {
                if (hi > lo) total += hi - lo;
                lo = iv.first;
                hi = iv.second;
            } else if (iv.second > hi) {
                hi = iv.second;
            }
        }
        if (hi > lo) total += hi - lo;
        ctx->prof.busy_ms[s] = total;
    }
    *out = ctx->prof;
    if (reset) {
        ctx->prof = slag_profile{};
        for (auto &b : ctx->busy) b.clear();
        if (ctx->prof_base) CK(cudaEventRecord(ctx->prof_base, ctx->stream));
    }
    return SLAG_OK;
}

}  // extern "C"

namespace {

// The pair list of one binning (depth ranks) -> caller indices, on the host.
slag_status ids_to_callers(slag_ctx *ctx, cudaStream_t st, const uint32_t *d_ids, int64_t count, int32_t *out) {
    const int64_t n = ctx->n;
    std::vector<uint32_t> h_list((size_t)(count > 0 ? count : 1)), h_orig((size_t)n);
    if (count > 0) CK(cudaMemcpyAsync(h_list.data(), d_ids, sizeof(uint32_t) * count, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_orig.data(), ctx->orig_of_int, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < count; ++i) {
        const uint32_t g = h_list[(size_t)i];
        out[i] = g < (uint32_t)n ? (int32_t)h_orig[g] : -1;
    }
    return SLAG_OK;
}

// Binning of one view at 2^shift x 2^shift tiles per bin, without compositing (slag_bin_view,
// slag_bin_view_bins).
slag_status bin_view_diag(slag_ctx *ctx, const slag_camera *cam, int shift, uint32_t *out_touched, int64_t *out_P,
                          int32_t *out_list, int64_t list_cap, int64_t *out_ranges) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    slag_status s = check_camera(ctx, cam);
    if (s != SLAG_OK) return s;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    s = launch_deferred_view(ctx);
    if (s == SLAG_OK) s = settle_views(ctx);
    if (s != SLAG_OK) return s;
    CK(join_views(ctx));
    ViewSlot &vs = ctx->slot[ctx->views_enqueued % kSlots];
    const CamParams cp = cam_params(cam);
    int64_t P = 0;
    uint32_t *list = nullptr;
    s = bin_view(ctx, vs, st, cp, &P, &list, shift);
    if (s != SLAG_OK) return s;
    CK(cudaStreamSynchronize(st));
    s = checks_reported(ctx);
    if (s != SLAG_OK) return s;
    if (out_P) *out_P = P;
    const int64_t n = ctx->n;
    const int64_t bins = (int64_t)(((cp.tiles_x - 1) >> shift) + 1) * (((cp.tiles_y - 1) >> shift) + 1);
    if (out_touched) {
        // tiles touched per Gaussian, caller order: depth-sorted values hold internal indices
        std::vector<uint32_t> h_orig((size_t)n);
        std::vector<uint2> h_rect((size_t)n);
        CK(cudaMemcpyAsync(h_rect.data(), vs.rect, sizeof(uint2) * n, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(h_orig.data(), ctx->orig_of_int, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int64_t gI = 0; gI < n; ++gI) {
            const uint2 rc = h_rect[(size_t)gI];
            out_touched[h_orig[(size_t)gI]] = ((rc.x >> 16) - (rc.x & 0xffffu)) * ((rc.y >> 16) - (rc.y & 0xffffu));
        }
    }
    if (out_list) {
        if (list_cap < P) return fail(ctx, SLAG_ERR_CAPACITY, "list_cap < P");
        // the list holds internal indices; map them to caller indices on the host
        s = ids_to_callers(ctx, st, list, P, out_list);
        if (s != SLAG_OK) return s;
    }
    if (out_ranges) {
        std::vector<uint2> h_r((size_t)bins);
        CK(cudaMemcpyAsync(h_r.data(), vs.ranges, sizeof(uint2) * bins, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        // an empty bin is reported as [e, e) with e the end of the bins before it
        int64_t at = 0;
        for (int64_t t = 0; t < bins; ++t) {
            const uint2 r = h_r[(size_t)t];
            if (r.y > r.x) at = r.y;
            out_ranges[2 * t] = r.y > r.x ? (int64_t)r.x : at;
            out_ranges[2 * t + 1] = r.y > r.x ? (int64_t)r.y : at;
        }
    }
    return SLAG_OK;
}

}  // namespace

extern "C" {

slag_status slag_bin_view(slag_ctx *ctx, const slag_camera *cam, uint32_t *out_touched, int64_t *out_P,
                          int32_t *out_list, int64_t list_cap, int64_t *out_ranges) {
    return bin_view_diag(ctx, cam, 0, out_touched, out_P, out_list, list_cap, out_ranges);
}

slag_status slag_bin_view_bins(slag_ctx *ctx, const slag_camera *cam, int32_t bin_shift, int64_t *out_P,
                               int32_t *out_list, int64_t list_cap, int64_t *out_ranges) {
    if (ctx && bin_shift != 0 && bin_shift != kSuperShift)
        return fail(ctx, SLAG_ERR_INVALID_ARG, "bin_shift must be 0 or the compositing's super-tile shift");
    return bin_view_diag(ctx, cam, bin_shift, nullptr, out_P, out_list, list_cap, out_ranges);
}

slag_status slag_composite_trace(slag_ctx *ctx, const slag_camera *cam, int64_t *out_P, int32_t *out_list,
                                 int64_t list_cap, int64_t *out_ranges) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    slag_status s = check_camera(ctx, cam);
    if (s != SLAG_OK) return s;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    s = launch_deferred_view(ctx);
    if (s == SLAG_OK) s = settle_views(ctx);
    if (s != SLAG_OK) return s;
    CK(join_views(ctx));
    ViewSlot &vs = ctx->slot[ctx->views_enqueued % kSlots];
    const CamParams cp = cam_params(cam);
    const int64_t tiles = (int64_t)cp.tiles_x * cp.tiles_y;
    // room per tile: the Gaussians whose tile rectangle holds it (the flat per-tile binning)
    int64_t P = 0;
    uint32_t *list = nullptr;
    s = bin_view(ctx, vs, st, cp, &P, &list, 0);
    if (s != SLAG_OK) return s;
    std::vector<uint2> h_r((size_t)tiles);
    CK(cudaMemcpyAsync(h_r.data(), vs.ranges, sizeof(uint2) * tiles, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int64_t> off((size_t)tiles + 1, 0);
    for (int64_t t = 0; t < tiles; ++t) {
        const uint2 r = h_r[(size_t)t];
        off[(size_t)t + 1] = off[(size_t)t] + (r.y > r.x ? (int64_t)(r.y - r.x) : 0);
    }
    if (out_P) *out_P = off[(size_t)tiles];
    if (!out_list && !out_ranges) return SLAG_OK;
    if (out_list && list_cap < off[(size_t)tiles]) return fail(ctx, SLAG_ERR_CAPACITY, "list_cap < P");
    // the super-tile binning slag_add_view composites from, then the composite with a trace
    int64_t Ps = 0;
    s = bin_view(ctx, vs, st, cp, &Ps, &list, kSuperShift);
    if (s != SLAG_OK) return s;
    uint32_t *d_list = nullptr, *d_staged = nullptr, *d_bad = nullptr;
    int64_t *d_off = nullptr;
    auto release = [&]() { dfree(d_list); dfree(d_staged); dfree(d_bad); dfree(d_off); };
    cudaError_t e = dalloc(&d_list, off[(size_t)tiles]);
    if (e == cudaSuccess) e = dalloc(&d_staged, tiles);
    if (e == cudaSuccess) e = dalloc(&d_bad, 1);
    if (e == cudaSuccess) e = dalloc(&d_off, tiles + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * (tiles + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_staged, 0, sizeof(uint32_t) * tiles, st);
    const int64_t npx = (int64_t)cam->width * cam->height;
    if (e == cudaSuccess && npx > ctx->dbg_cap) {
        int64_t c1 = ctx->dbg_cap, c2 = ctx->dbg_cap, c3 = ctx->dbg_cap;
        e = grow(ctx->dbg_T, c1, npx, st);
        if (e == cudaSuccess) e = grow(ctx->dbg_wsum, c2, npx, st);
        if (e == cudaSuccess) e = grow(ctx->dbg_count, c3, npx, st);
        if (e == cudaSuccess) ctx->dbg_cap = c1;
    }
    if (e != cudaSuccess) {
        release();
        return fail(ctx, e == cudaErrorMemoryAllocation ? SLAG_ERR_OOM : SLAG_ERR_CUDA, cudaGetErrorString(e));
    }
    CompositeArgs a;
    memset(&a, 0, sizeof(a));
    a.cam = cp;
    a.ranges = vs.ranges;
    a.bin_shift = kSuperShift;
    a.bins_x = ((cp.tiles_x - 1) >> kSuperShift) + 1;
    a.tile_order = vs.tile_order;
    a.list = list;
    a.prect = vs.prect;
    a.rec_a = vs.rec_a;
    a.rec_b = vs.rec_b;
    a.rec_t = vs.rec_t;
    a.n_ids = (uint32_t)ctx->n;
    a.weight_mode = ctx->weight_mode;
    a.ctr = vs.ctr;
    a.contrib = &vs.ctr->contributions;
    a.dbg_T = ctx->dbg_T;
    a.dbg_wsum = ctx->dbg_wsum;
    a.dbg_count = ctx->dbg_count;
    a.dbg_list = d_list;
    a.dbg_off = d_off;
    a.dbg_staged = d_staged;
    a.dbg_bad = d_bad;
    a.err = ctx->tc_err;
    a.accumulate = 0;
    launch_composite(a, st);
    e = cudaGetLastError();
    std::vector<uint32_t> staged((size_t)tiles);
    uint32_t bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(staged.data(), d_staged, sizeof(uint32_t) * tiles, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        release();
        return fail(ctx, SLAG_ERR_CUDA, cudaGetErrorString(e));
    }
    if (out_list) {
        s = ids_to_callers(ctx, st, d_list, off[(size_t)tiles], out_list);
        if (s != SLAG_OK) { release(); return s; }
    }
    if (out_ranges)
        for (int64_t t = 0; t < tiles; ++t) {
            out_ranges[2 * t] = off[(size_t)t];
            out_ranges[2 * t + 1] = off[(size_t)t] + (int64_t)staged[(size_t)t];
        }
    release();
    if (bad) return fail(ctx, SLAG_ERR_CAPACITY, "a tile staged more Gaussians than its tile list holds");
    return checks_reported(ctx);
}

slag_status slag_render_debug(slag_ctx *ctx, const slag_camera *cam, float *out_T, float *out_wsum,
                              int32_t *out_count) {
    if (!ctx) return SLAG_ERR_INVALID_ARG;
    slag_status s = check_camera(ctx, cam);
    if (s != SLAG_OK) return s;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    s = launch_deferred_view(ctx);
    if (s == SLAG_OK) s = settle_views(ctx);
    if (s != SLAG_OK) return s;
    CK(join_views(ctx));
    ViewSlot &vs = ctx->slot[ctx->views_enqueued % kSlots];
    const CamParams cp = cam_params(cam);
    const int64_t npx = (int64_t)cam->width * cam->height;
    int64_t P = 0;
    uint32_t *list = nullptr;
    s = bin_view(ctx, vs, st, cp, &P, &list, kSuperShift);
    if (s != SLAG_OK) return s;
    if (npx > ctx->dbg_cap) {
        int64_t c1 = ctx->dbg_cap, c2 = ctx->dbg_cap, c3 = ctx->dbg_cap;
        CK(grow(ctx->dbg_T, c1, npx, st));
        CK(grow(ctx->dbg_wsum, c2, npx, st));
        CK(grow(ctx->dbg_count, c3, npx, st));
        ctx->dbg_cap = c1;
    }
    CompositeArgs a;
    memset(&a, 0, sizeof(a));
    a.cam = cp;
    a.ranges = vs.ranges;
    a.bin_shift = kSuperShift;
    a.bins_x = ((cp.tiles_x - 1) >> kSuperShift) + 1;
    a.tile_order = vs.tile_order;
    a.list = list;
    a.prect = vs.prect;
    a.rec_a = vs.rec_a;
    a.rec_b = vs.rec_b;
    a.rec_t = vs.rec_t;
    a.n_ids = (uint32_t)ctx->n;
    a.seg = nullptr;
    a.weight_mode = ctx->weight_mode;
    a.ctr = vs.ctr;
    a.contrib = &vs.ctr->contributions;
    a.dbg_T = ctx->dbg_T;
    a.dbg_wsum = ctx->dbg_wsum;
    a.dbg_count = ctx->dbg_count;
    a.err = ctx->tc_err;
    a.accumulate = 0;
    a.recs = nullptr;
    a.rec_chunks = nullptr;
    a.rec_fill = nullptr;
    a.chunk_cap = 0;
    launch_composite(a, st);
    CK(cudaGetLastError());
    if (out_T) CK(cudaMemcpyAsync(out_T, ctx->dbg_T, sizeof(float) * npx, cudaMemcpyDeviceToHost, st));
    if (out_wsum) CK(cudaMemcpyAsync(out_wsum, ctx->dbg_wsum, sizeof(float) * npx, cudaMemcpyDeviceToHost, st));
    if (out_count) CK(cudaMemcpyAsync(out_count, ctx->dbg_count, sizeof(int32_t) * npx, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return checks_reported(ctx);
}

}  // extern "C"
