// Front-to-back compositing, parameter masking and in-tile segment binning.
//
// Rasterizer_SLAG (Method, "Semantic Embedding"): for every pixel p, walk the
// tile's Gaussians in ascending (depth, index); q = d^T conic d with
// d = mu' - p, alpha = min(0.99, opacity * exp(-q/2)); skip alpha < 1/255;
// stop the pixel before the Gaussian whose (1 - alpha) would take the
// transmittance T below 1e-4; otherwise record w = alpha * T (or exp(-q/2))
// and T *= 1 - alpha. Parameter Masking keeps w only where the pixel lies in a
// segment. The Aggregation sums need, per Gaussian k and segment j of this
// view, B[k][j] = sum over the pixels of j of w_{k,p}: because every pixel of
// a segment carries the same embedding E_j, the D-wide product B . E is
// deferred to the aggregation (this view only emits B).
//
// One CTA per 16x16 tile: four consumer warps own the tile's 256 pixels (two
// per thread) and one producer warp feeds them. The tile's Gaussians are those
// of its bin's list (a 4x4-tile super-tile) whose tile rectangle holds the
// tile, taken in list order.
//   * Producer: fills one of kNB record buffers at a time (a ring) with the hits among
//     the bin's list, 128 candidates at a time (the following 128 are loaded
//     meanwhile; the list holds Gaussian indices), as many groups as the buffer's
//     128 records hold, copying each hit's record
//     (36 bytes, written by the projection) asynchronously and publishing the
//     buffer on an mbarrier that completes once the copies have landed, so the
//     producer never waits for them; it refills a buffer once all consumers
//     have released it, first moving that buffer's per-(segment, Gaussian)
//     sums to the view's record list. It stops when the list ends or no
//     consumer warp has a live pixel.
//   * Consumers: the tile's pixels are reordered by segment ("slot"), and
//     within a segment by 8x8 block; a thread takes two neighbours in that
//     order (almost always one segment), so each warp's 64 pixels usually
//     share one segment and form a square block. A warp composites each
//     published buffer in chunks of 32 Gaussians, keeping only those whose
//     alpha >= 1/255 reaches its pixel box (the record's mean made tile-local),
//     expands the survivors' exponents into tile-local polynomials, composites
//     them, then sums each Gaussian's weights
//     over its lanes per slot (a transposition through shared memory) into
//     the buffer's (slot x Gaussian) table, and releases the buffer. Warps run
//     independently: a warp whose pixels have all stopped only releases the
//     buffers, and no warp waits for another at a CTA barrier.
//   * Every wait is an mbarrier wait bounded by ~1 s of globaltimer; a wait
//     that gives up sets the context's error word and an abort flag that
//     releases every other wait of the CTA; the producer waits for its copies
//     in flight before it exits.
// A combine pass (many records in flight per SM) adds the records to the
// per-view (segment, weight) table of each Gaussian (4 slots per Gaussian;
// sums of further segments go to the view's spill list).
#include "slag_internal.cuh"
#include "tc_util.cuh"

namespace slag {

SLAG_CHECKS_WORD

namespace {

constexpr int kPix = kTile * kTile;                   // 256 pixels per CTA (one tile)
constexpr int kConsumers = 4;                         // compositing warps, 64 pixels each
constexpr int kPixThreads = 32 * kConsumers;          // two pixels per consumer thread
constexpr int kThreads = kPixThreads + 32;            // + the producer warp
constexpr int kProducer = kConsumers;                 // warp index of the producer
constexpr int kCtasPerSm = 5;                         // resident CTAs per SM (shared memory)
constexpr int kPerLane = 4;                           // candidates per producer lane and batch
constexpr int kBuf = 32 * kPerLane;                   // candidates per batch = record capacity of a buffer
constexpr int kNB = 2;                                // record buffers (a ring)
constexpr int kSmemSlots = 4;
// A pixel stops before the Gaussian that would take its transmittance below kTStop. Its T keeps
// being multiplied by (1 - alpha) afterwards, so it stays below kTStop (a product with a factor
// in [0.01, 1] does not round above its operand): T >= kTStop is "the pixel is live", and the
// transmittance chain is one packed FMA per Gaussian.
constexpr float kTStop = 1e-4f;
static_assert(kBuf < kRecChunk, "one slot's sums of a buffer must fit in two record chunks");
constexpr int kWStride = 36;                          // transposition rows: 16-byte aligned, conflict-free
constexpr uint32_t kBarConsumers = 1;                 // named barrier of the consumer warps

struct Smem {
    float4 q0[kNB][kBuf];                 // records: (mu'x, mu'y, a', b')
    float4 q1[kNB][kBuf];                 //          (c', log2 opacity, r1, r2)
    float qt[kNB][kBuf];                  //          culling threshold t
    uint32_t gid[kNB][kBuf];              // internal Gaussian index of each record
    float wb[kNB][kSmemSlots][kBuf];      // per (buffer, slot, Gaussian of the buffer)
    union {
        float wbuf[kConsumers][32 * kWStride];   // per warp: (survivor of the chunk) x lane
        uint32_t keys[kPix];                     // the prologue's segment sort
    };
    float4 stage[kConsumers][16 * 3];     // per warp: survivors' polynomials, two Gaussians interleaved
    int32_t clist[kConsumers][32];        // per warp: chunk position of each survivor
    uint32_t split_min[2][kConsumers];    // prologue multi-split: per-warp minimum segment
    int32_t split_cnt[2][kConsumers];     // and per-warp counts (first | second pixel << 16)
    int16_t slot_lane[kPixThreads];       // slot of the sums each lane stores (its first pixel's)
    int32_t seg_of_slot[kPix];
    int32_t group_slot[kConsumers];       // slot shared by all of a warp's pixels, -2 = mixed
    int32_t warp_tot[kConsumers];
    int32_t scalar[4];                    // [0] first pixel's segment, [1] slots in shared memory
    int32_t count[kNB];                   // records in each buffer (-1: no more)
    int32_t warp_live[kConsumers];        // a consumer warp still has a live pixel
    uint32_t abort_flag;                  // a wait gave up: every other wait gives up too
    int32_t view_base;                    // column of the view's segment 0
    unsigned long long totals[kConsumers][3];   // per consumer warp: contributions, visited, executed
    __align__(8) uint64_t full[kNB];      // a buffer is published (32 producer arrivals)
    __align__(8) uint64_t empty[kNB];     // a buffer is released (128 consumer arrivals)
    __align__(8) uint64_t ready;          // the consumers' prologue is done (128 arrivals)
};
// kCtasPerSm CTAs per SM (228 KB of shared memory, 1 KB of it reserved per CTA)
static_assert(sizeof(Smem) + 1024 <= 233472 / kCtasPerSm, "composite shared memory above the CTA budget");

__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two floats as one 64-bit operand of the packed FP32 instructions (lane-pair arithmetic of
// fma/mul .f32x2: each half rounds like the scalar instruction).
__device__ __forceinline__ uint64_t pk(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float2 unpk(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// 1.0f where a >= b, else 0.0f (false for NaN)
__device__ __forceinline__ float set_ge(float a, float b) {
    float d;
    asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// The coefficients K0, K1, K2 of the exponent e = K0 + K1 X + K2 Y + A X^2 + Bc X Y + C Y^2 of a
// Gaussian with tile-local mean (mx, my): e = lo + A dx^2 + Bc dx dy + C dy^2 with dx = mx - X,
// dy = my - Y, expanded.
__device__ __forceinline__ void poly_coeffs(float mx, float my, float A, float Bc, float C, float lo, float &K0,
                                            float &K1, float &K2) {
    K1 = -fmaf(2.f * A, mx, Bc * my);
    K2 = -fmaf(Bc, mx, 2.f * C * my);
    K0 = fmaf(fmaf(A, mx, Bc * my), mx, fmaf(C * my, my, lo));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src));
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src));
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Arrival on bar once this thread's cp.async copies so far have landed (counted in the barrier's
// arrival count: .noinc).
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Barriers of the consumer warps only (the producer never takes part).
__device__ __forceinline__ void cbar() { asm volatile("bar.sync %0, %1;" ::"n"(kBarConsumers), "n"(kPixThreads) : "memory"); }

__device__ __forceinline__ bool cbar_and(bool p) {
    uint32_t r;
    asm volatile(
        "{\n"
        " .reg .pred a, b;\n"
        " setp.ne.u32 a, %1, 0;\n"
        " bar.red.and.pred b, %2, %3, a;\n"
        " selp.u32 %0, 1, 0, b;\n"
        "}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "n"(kBarConsumers), "n"(kPixThreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ HashSink sink_of(const CompositeArgs &a, const Smem &sm) {
    return HashSink{a.hash, a.spill_count, a.spill_cap, a.spill_key, a.spill_w, sm.view_base};
}

__device__ __forceinline__ void flush_slot(const CompositeArgs &a, Smem &sm, int b, int slot, int gi, float acc) {
    if (slot < kSmemSlots) atomicAdd(&sm.wb[b][slot][gi], acc);
    else sink_add(sink_of(a, sm), sm.gid[b][gi], sm.seg_of_slot[slot], acc);
}

// The producer's place in the view's record list: chunk `cur` is being filled (`used` records),
// chunk `next` follows it. A chunk index comes from an atomicAdd issued one chunk ahead (lane 0
// holds the result in `pend` until it is needed), so that no store waits for the reservation.
struct RecRes {
    unsigned long long cur, next, pend;   // pend: lane 0 only
    int used;
    bool requested, have_cur, have_next;
};

__device__ __forceinline__ void res_request(const CompositeArgs &a, RecRes &rr, int lane, unsigned long long k) {
    if (lane == 0) rr.pend = atomicAdd(a.rec_chunks, k);
}

__device__ __forceinline__ void res_fill(const CompositeArgs &a, unsigned long long chunk, int lane, uint32_t fill) {
    if (lane == 0 && chunk < a.chunk_cap) a.rec_fill[chunk] = fill;
}

// The producer's last act: the fills of its current and reserved chunks.
__device__ void res_close(const CompositeArgs &a, RecRes &rr, int lane) {
    if (!rr.requested) return;
    if (!rr.have_cur) {   // reserved, never written
        const unsigned long long c = __shfl_sync(0xffffffffu, rr.pend, 0);
        res_fill(a, c, lane, 0u);
        res_fill(a, c + 1ull, lane, 0u);
        return;
    }
    res_fill(a, rr.cur, lane, (uint32_t)rr.used);
    const unsigned long long nx = rr.have_next ? rr.next : __shfl_sync(0xffffffffu, rr.pend, 0);
    res_fill(a, nx, lane, 0u);
}

// Whether the exponent e(X, Y) = lo + A dx^2 + Bc dx dy + C dy^2 (dx = mx - X, dy = my - Y; A, C < 0
// and 4AC > Bc^2: a concave quadratic) reaches lo + t anywhere on the box (x0, x1, y0, y1) of a warp's
// pixel centres. The maximum over the box is lo at the mean when the mean lies inside; otherwise it
// lies on the box's boundary, where each edge is a concave parabola maximised at its clamped vertex:
// dy = r1 dx on a vertical edge (r1 = -Bc / 2C), dx = r2 dy on a horizontal one (r2 = -Bc / 2A). An
// empty box (x0 = +inf) reaches nothing.
__device__ __forceinline__ bool reaches(float mx, float my, float r1, float r2, float A, float Bc, float C, float t,
                                        float4 box) {
    if (!(box.x <= box.y)) return false;
    if (mx >= box.x && mx <= box.y && my >= box.z && my <= box.w) return 0.f >= t;
    const float dx0 = mx - box.y, dx1 = mx - box.x;   // dx range over the box
    const float dy0 = my - box.w, dy1 = my - box.z;
    float best = -INFINITY;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        // vertical edges: dx fixed, dy free in [dy0, dy1]
        const float dx = e ? dx1 : dx0;
        const float dy = fminf(fmaxf(r1 * dx, dy0), dy1);
        best = fmaxf(best, fmaf(fmaf(A, dx, Bc * dy), dx, C * dy * dy));
        // horizontal edges: dy fixed, dx free in [dx0, dx1]
        const float dy2 = e ? dy1 : dy0;
        const float dx2 = fminf(fmaxf(r2 * dy2, dx0), dx1);
        best = fmaxf(best, fmaf(fmaf(A, dx2, Bc * dy2), dx2, C * dy2 * dy2));
    }
    return best >= t;
}

// The box (x0, x1, y0, y1) of the pixel centres (X0, Y0) and (X1, Y1) of the warp's lanes for
// which l0 and l1 hold (x0 = +inf when there are none), in every lane.
__device__ __forceinline__ float4 live_box(bool l0, bool l1, float X0, float Y0, float X1, float Y1) {
    float x0 = fminf(l0 ? X0 : INFINITY, l1 ? X1 : INFINITY);
    float x1 = fmaxf(l0 ? X0 : -INFINITY, l1 ? X1 : -INFINITY);
    float y0 = fminf(l0 ? Y0 : INFINITY, l1 ? Y1 : INFINITY);
    float y1 = fmaxf(l0 ? Y0 : -INFINITY, l1 ? Y1 : -INFINITY);
    for (int o = 16; o; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    return make_float4(x0, x1, y0, y1);
}

// Pixel index p of the tile in block order: four 8x8 blocks (row-major), each row-major, so that
// a warp's 64 pixels of one segment form an 8x8 block.
__device__ __forceinline__ int pix_x(int p) { return ((p >> 3) & 8) | (p & 7); }
__device__ __forceinline__ int pix_y(int p) { return ((p >> 4) & 8) | ((p >> 3) & 7); }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// A bounded wait on the phase `parity` of bar; on giving up, the error word is set and every other
// wait of the CTA gives up through the abort flag.
__device__ __forceinline__ bool wait_phase(const CompositeArgs &a, Smem &sm, uint64_t *bar, uint32_t parity) {
    if (tc::wait_or_abort(bar, parity, &sm.abort_flag)) return true;
    if (a.err) atomicOr(a.err, 1u);
    return false;
}

// ---- the producer warp ---------------------------------------------------------------------

// Moves buffer b's non-zero (slot, Gaussian) sums of its n records (n <= kBuf) to the view's
// record list, clearing the table for the buffer's next use. Per slot, lane l takes records
// l, l + 32, ...; a warp scan of the lanes' counts places them, so the records of one slot
// (at most kBuf < kRecChunk) always fit in chunks cur and next.
__device__ void drain_sums(const CompositeArgs &a, Smem &sm, int b, int n, int ns_smem, int lane, RecRes &rr) {
    for (int s2 = 0; s2 < ns_smem; ++s2) {
        float v[kPerLane];
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
            const int i = lane + 32 * j;
            v[j] = 0.f;
            if (i < n) {
                v[j] = sm.wb[b][s2][i];
                sm.wb[b][s2][i] = 0.f;
            }
            cnt += v[j] != 0.f ? 1 : 0;
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        if (tot == 0) continue;
        const int32_t seg = sm.seg_of_slot[s2];
        if (!a.recs) {   // no record list: the sums go to the tables directly
#pragma unroll
            for (int j = 0; j < kPerLane; ++j)
                if (v[j] != 0.f) sink_add(sink_of(a, sm), sm.gid[b][lane + 32 * j], seg, v[j]);
            continue;
        }
        if (!rr.have_cur) {   // the first records: the two chunks reserved at the start
            rr.cur = __shfl_sync(0xffffffffu, rr.pend, 0);
            rr.next = rr.cur + 1ull;
            rr.used = 0;
            rr.have_cur = rr.have_next = true;
        }
        if (rr.used + tot >= kRecChunk && !rr.have_next) {   // records go to, or continue in, chunk next
            rr.next = __shfl_sync(0xffffffffu, rr.pend, 0);
            rr.have_next = true;
        }
        int pos = rr.used + incl - cnt;
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
            if (v[j] == 0.f) continue;
            const uint32_t g = sm.gid[b][lane + 32 * j];
            const unsigned long long ch = pos < kRecChunk ? rr.cur : rr.next;
            if (ch < a.chunk_cap) {
                WeightRecord r;
                r.g = g;
                r.seg = seg;
                r.w = v[j];
                r.pad = 0u;
                a.recs[ch * kRecChunk + (pos < kRecChunk ? pos : pos - kRecChunk)] = r;
            } else {
                sink_add(sink_of(a, sm), g, seg, v[j]);
            }
            ++pos;
        }
        rr.used += tot;
        if (rr.used >= kRecChunk) {
            // chunk cur is full: continue in next, and reserve the one after it
            res_fill(a, rr.cur, lane, (uint32_t)kRecChunk);
            rr.cur = rr.next;
            rr.used -= kRecChunk;
            rr.have_next = false;
            res_request(a, rr, lane, 1ull);
        }
    }
}

// Publishes buffer b: every producer lane arrives twice on full[b] (count 64), once for its
// shared-memory writes (release) and once, asynchronously, when its record copies have landed.
__device__ __forceinline__ void publish(Smem &sm, int b) {
    cp_async_arrive(&sm.full[b]);
    tc::arrive(&sm.full[b]);
}

template <bool kDebug>
__device__ void producer(const CompositeArgs &a, Smem &sm, int tile, int tx, int ty, float ox, float oy, int lane) {
    const uint32_t lt = lanemask_lt();
    const bool trace = kDebug && a.dbg_list != nullptr;
    const uint2 rg = a.ranges[(ty >> a.bin_shift) * a.bins_x + (tx >> a.bin_shift)];
    const int end = (int)rg.y;
    int cursor = (int)rg.x;
    int staged = 0;   // Gaussians staged so far (their positions in the tile's own list)
    RecRes rr;        // place in the view's record list
    rr.cur = rr.next = rr.pend = 0ull;
    rr.used = 0;
    rr.requested = rr.have_cur = rr.have_next = false;
    if (a.accumulate && a.recs) {   // two chunks, reserved while the first batch is staged
        res_request(a, rr, lane, 2ull);
        rr.requested = true;
    }
    int ns_smem = 0;  // slots with a shared-memory table (known after the consumers' prologue)
    // a batch is the next kBuf candidates of the bin's list; the candidates of the batch after the
    // current one are loaded into registers while the current one is staged
    uint32_t r_nx[kPerLane];
    uint2 rc_nx[kPerLane];
#pragma unroll
    for (int k = 0; k < kPerLane; ++k) {
        const int c = cursor + k * 32 + lane;
        r_nx[k] = c < end ? a.list[c] : 0u;
        rc_nx[k] = c < end ? a.prect[c] : make_uint2(0u, 0u);
    }
    bool ok = true, have_slots = false;
    // batch it is filled in buffer it % kNB; taking a buffer for batch it >= kNB waits until the
    // consumers have released batch it - kNB and moves that batch's sums out
    int it = 0, nb = 0;
    bool held = false;   // batch it has its buffer
    auto take = [&]() -> bool {
        const int b = it % kNB;
        if (it >= kNB) {
            if (!wait_phase(a, sm, &sm.empty[b], (uint32_t)(it / kNB - 1) & 1u)) return false;
            if (a.accumulate) drain_sums(a, sm, b, sm.count[b], ns_smem, lane, rr);
        }
        held = true;
        return true;
    };
    for (;;) {
        // the next kBuf candidates and their hits; the loads of the group after them are issued now
        uint32_t g[kPerLane];
        bool hit[kPerLane];
#pragma unroll
        for (int k = 0; k < kPerLane; ++k) {
            const int c = cursor + k * 32 + lane;
            g[k] = r_nx[k];
            const uint2 rc = rc_nx[k];
            hit[k] = c < end && (uint32_t)tx >= (rc.x & 0xffffu) && (uint32_t)tx < (rc.x >> 16) &&
                     (uint32_t)ty >= (rc.y & 0xffffu) && (uint32_t)ty < (rc.y >> 16) &&
                     SLAG_IN_BOUNDS(g[k] < a.n_ids, kCheckComposite);
            const int cn = c + kBuf;
            r_nx[k] = cn < end ? a.list[cn] : 0u;
            rc_nx[k] = cn < end ? a.prect[cn] : make_uint2(0u, 0u);
        }
        bool live = trace;
        if (!trace) {
            // the consumers' liveness after the batches they have released
            for (int q = 0; q < kConsumers; ++q) live = live || (*((volatile int32_t *)&sm.warp_live[q]) != 0);
        }
        if (cursor >= end || !live) break;
        uint32_t bal[kPerLane];
        int gh = 0;
#pragma unroll
        for (int k = 0; k < kPerLane; ++k) {
            bal[k] = __ballot_sync(0xffffffffu, hit[k]);
            gh += __popc(bal[k]);
        }
        cursor += kBuf;
        if (gh == 0) continue;
        if (!held && !take()) { ok = false; break; }
        if (nb + gh > kBuf) {
            // the batch is as full as the group allows: publish it and fill the next one
            if (!have_slots) {
                // the number of slots comes from the consumers' prologue (needed by the drains)
                if (!wait_phase(a, sm, &sm.ready, 0u)) { ok = false; break; }
                ns_smem = sm.scalar[1];
                have_slots = true;
            }
            if (lane == 0) sm.count[it % kNB] = nb;
            __syncwarp();
            publish(sm, it % kNB);   // complete once the records' copies have landed
            ++it;
            nb = 0;
            held = false;
            if (!take()) { ok = false; break; }
        }
        // stable compaction of the group's hits (candidate order is (k, lane)) after the batch's
        // records so far; their records are copied asynchronously
        const int b = it % kNB;
        int ng = 0;
#pragma unroll
        for (int k = 0; k < kPerLane; ++k) {
            const int pg = ng + __popc(bal[k] & lt);
            if (hit[k]) {
                const int pos = nb + pg;
                cp_async16(&sm.q0[b][pos], a.rec_a + g[k]);
                cp_async16(&sm.q1[b][pos], a.rec_b + g[k]);
                cp_async4(&sm.qt[b][pos], a.rec_t + g[k]);
                sm.gid[b][pos] = g[k];
                if (trace) {
                    const int64_t at = a.dbg_off[tile] + staged + pg;
                    if (at < a.dbg_off[tile + 1]) a.dbg_list[at] = g[k];
                    else atomicOr(a.dbg_bad, 1u);
                }
            }
            ng += __popc(bal[k]);
        }
        nb += gh;
        staged += gh;
    }
    if (ok) {
        // the last batch with records, then the end mark in the batch after it
        if (nb > 0) {
            if (!have_slots) {
                if (!wait_phase(a, sm, &sm.ready, 0u)) ok = false;
                ns_smem = sm.scalar[1];
                have_slots = true;
            }
            if (ok) {
                if (lane == 0) sm.count[it % kNB] = nb;
                __syncwarp();
                publish(sm, it % kNB);
                ++it;
                held = false;
            }
        }
        if (ok && (held || take())) {
            if (lane == 0) sm.count[it % kNB] = -1;
            __syncwarp();
            publish(sm, it % kNB);
        } else {
            ok = false;
        }
    }
    // the batches still held by the consumers (it - kNB + 1 .. it - 1): their sums once released
    for (int bt = it - kNB + 1 > 0 ? it - kNB + 1 : 0; ok && bt < it; ++bt) {
        const int b = bt % kNB;
        ok = wait_phase(a, sm, &sm.empty[b], (uint32_t)(bt / kNB) & 1u);
        if (ok && a.accumulate) drain_sums(a, sm, b, sm.count[b], ns_smem, lane, rr);
    }
    if (a.accumulate && a.recs) res_close(a, rr, lane);
    if (trace && lane == 0) a.dbg_staged[tile] = (uint32_t)staged;
    cp_async_wait_all();   // no copy into the CTA's shared memory outlives it (after a wait gave up)
}

// kKernel: record Eq. 2's kernel exp(-q/2) instead of alpha * T; kDebug: keep the
// per-pixel weight sums and counts of the diagnostic render (and its staging trace).
template <bool kKernel, bool kDebug>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) composite_k(const CompositeArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    if (a.skip && *a.skip) return;   // the view is not composited (uniform, before any barrier)
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int tile = (int)a.tile_order[blockIdx.x];
    const int tx = tile % a.cam.tiles_x, ty = tile / a.cam.tiles_x;
    const int W = a.cam.width, H = a.cam.height;
    const float ox = (float)(tx * kTile), oy = (float)(ty * kTile);

    if (tid == 0) {
        for (int b = 0; b < kNB; ++b) {
            tc::mbar_init(&sm.full[b], 64);
            tc::mbar_init(&sm.empty[b], kPixThreads);
        }
        tc::mbar_init(&sm.ready, kPixThreads);
        sm.abort_flag = 0u;
        sm.view_base = a.view_base_dev ? *a.view_base_dev : a.view_base;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the (slot x Gaussian) sums start at zero; each buffer's drain clears what it read
    for (int i = tid; i < kNB * kSmemSlots * kBuf; i += kThreads) (&sm.wb[0][0][0])[i] = 0.f;
    if (tid < kConsumers) sm.warp_live[tid] = 1;
    __syncthreads();
    if (w == kProducer) {
        producer<kDebug>(a, sm, tile, tx, ty, ox, oy, lane);
        return;
    }

    const uint32_t lt = lanemask_lt();
    // ---- segment of each of the CTA's pixels; positions sorted by segment --------
    // (thread t reads pixels t and t + 128; a pixel index fits in the low 8 bits of a key)
    int32_t s_nat[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p = tid + h * kPixThreads;
        const int px = tx * kTile + pix_x(p), py = ty * kTile + pix_y(p);
        const bool inside = px < W && py < H;
        int32_t sg = (inside && a.seg && a.accumulate) ? a.seg[(int64_t)py * W + px] : -1;
        if (sg < -1) sg = -1;
        s_nat[h] = sg;
        sm.keys[p] = ((uint32_t)(sg + 1) << 8) | (uint32_t)p;
    }
    if (tid == 0) sm.scalar[0] = s_nat[0];
    cbar();
    const bool uniform = cbar_and(s_nat[0] == sm.scalar[0] && s_nat[1] == sm.scalar[0]);
    int pos0 = tid, pos1 = tid + kPixThreads;
    if (!uniform) {
        // stable multi-split into (segment, pixel) order: one round per distinct segment of the
        // tile, smallest first; pixel tid precedes pixel tid + 128 of the same segment
        const uint32_t g0 = (uint32_t)(s_nat[0] + 1), g1 = (uint32_t)(s_nat[1] + 1);
        bool left0 = true, left1 = true;
        int placed = 0;
        for (int rnd = 0;; rnd ^= 1) {
            const uint32_t mine = min(left0 ? g0 : 0xffffffffu, left1 ? g1 : 0xffffffffu);
            const uint32_t wmin = __reduce_min_sync(0xffffffffu, mine);
            const bool t0 = left0 && g0 == wmin, t1 = left1 && g1 == wmin;
            if (lane == 0) sm.split_min[rnd][w] = wmin;
            cbar();
            uint32_t mn = 0xffffffffu;
#pragma unroll
            for (int q = 0; q < kConsumers; ++q) mn = min(mn, sm.split_min[rnd][q]);
            if (mn == 0xffffffffu) break;
            const bool u0 = t0 && wmin == mn, u1 = t1 && wmin == mn;
            const uint32_t b0 = __ballot_sync(0xffffffffu, u0), b1 = __ballot_sync(0xffffffffu, u1);
            if (lane == 0) sm.split_cnt[rnd][w] = __popc(b0) | (__popc(b1) << 16);
            cbar();
            int before0 = 0, before1 = 0, tot0 = 0, tot1 = 0;
#pragma unroll
            for (int q = 0; q < kConsumers; ++q) {
                const int c = sm.split_cnt[rnd][q], c0 = c & 0xffff, c1 = c >> 16;
                before0 += q < w ? c0 : 0;
                before1 += q < w ? c1 : 0;
                tot0 += c0;
                tot1 += c1;
            }
            if (u0) {
                pos0 = placed + before0 + __popc(b0 & lt);
                left0 = false;
            }
            if (u1) {
                pos1 = placed + tot0 + before1 + __popc(b1 & lt);
                left1 = false;
            }
            placed += tot0 + tot1;
        }
    }
    cbar();
    sm.keys[pos0] = ((uint32_t)(s_nat[0] + 1) << 8) | (uint32_t)tid;
    sm.keys[pos1] = ((uint32_t)(s_nat[1] + 1) << 8) | (uint32_t)(tid + kPixThreads);
    cbar();
    // this thread's pixels: positions 2 tid and 2 tid + 1 (adjacent in segment order, so
    // they almost always share a segment)
    const uint32_t k0 = sm.keys[2 * tid], k1 = sm.keys[2 * tid + 1];
    const int pix0 = (int)(k0 & 255u), pix1 = (int)(k1 & 255u);
    const int32_t seg0 = (int32_t)(k0 >> 8) - 1, seg1 = (int32_t)(k1 >> 8) - 1;
    // slots: the distinct segments in position order
    const int32_t seg_before = tid > 0 ? (int32_t)(sm.keys[2 * tid - 1] >> 8) - 1 : -2;
    const int new0 = (seg0 >= 0 && seg0 != seg_before) ? 1 : 0;
    const int new1 = (seg1 >= 0 && seg1 != seg0) ? 1 : 0;
    int incl = new0 + new1;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sm.warp_tot[w] = incl;
    cbar();   // the keys are read: the transposition buffers may reuse them from here on
    int before = incl - new0 - new1, nslots = 0;
#pragma unroll
    for (int q = 0; q < kConsumers; ++q) {
        before += q < w ? sm.warp_tot[q] : 0;
        nslots += sm.warp_tot[q];
    }
    const int slot0 = seg0 >= 0 ? before + new0 - 1 : -1;
    const int slot1 = seg1 >= 0 ? before + new0 + new1 - 1 : -1;
    if (new0) sm.seg_of_slot[slot0] = seg0;
    if (new1) sm.seg_of_slot[slot1] = seg1;
    sm.slot_lane[tid] = (int16_t)slot0;   // the slot of the sums this lane stores (< 256, or -1)
    const bool pair_same = slot0 == slot1;
    // the second pixel of a pair that straddles a segment boundary adds its weights to its own
    // slot directly
    const bool split1 = !pair_same && slot1 >= 0 && a.accumulate;
    {
        const int first = __shfl_sync(0xffffffffu, slot0, 0);
        const bool same = __all_sync(0xffffffffu, slot0 == first && slot1 == first);
        if (lane == 0) sm.group_slot[w] = same ? first : -2;
    }
    if (tid == 0) sm.scalar[1] = nslots < kSmemSlots ? nslots : kSmemSlots;

    const int px0 = tx * kTile + pix_x(pix0), py0 = ty * kTile + pix_y(pix0);
    const int px1 = tx * kTile + pix_x(pix1), py1 = ty * kTile + pix_y(pix1);
    const bool inside0 = px0 < W && py0 < H, inside1 = px1 < W && py1 < H;
    // pixel centres relative to the tile's origin, and their monomials: the exponent of a
    // Gaussian is a quadratic polynomial in them (see the producer's record conversion)
    const float X0 = (float)pix_x(pix0) + 0.5f, Y0 = (float)pix_y(pix0) + 0.5f;
    const float X1 = (float)pix_x(pix1) + 0.5f, Y1 = (float)pix_y(pix1) + 0.5f;
    // each pixel's monomials in both halves of a packed pair: one packed product evaluates two
    // Gaussians (whose coefficients are staged interleaved) at one pixel
    const uint64_t X0d = pk(X0, X0), Y0d = pk(Y0, Y0), XX0d = pk(X0 * X0, X0 * X0), XY0d = pk(X0 * Y0, X0 * Y0),
                   YY0d = pk(Y0 * Y0, Y0 * Y0);
    const uint64_t X1d = pk(X1, X1), Y1d = pk(Y1, Y1), XX1d = pk(X1 * X1, X1 * X1), XY1d = pk(X1 * Y1, X1 * Y1),
                   YY1d = pk(Y1 * Y1, Y1 * Y1);
    // bounding box of this warp's pixel centres (culling of Gaussians per warp), tile-local
    const float4 wbox = live_box(inside0, inside1, X0, Y0, X1, Y1);   // every lane holds the warp's box
    // T (both pixels, packed) below kTStop marks a pixel that has stopped (T = 0 one outside the
    // image): every later Gaussian keeps it there, so no flag is needed
    uint64_t PT = pk(inside0 ? 1.f : 0.f, inside1 ? 1.f : 0.f);
    {
        const bool any = __any_sync(0xffffffffu, inside0 || inside1);
        if (lane == 0) sm.warp_live[w] = any ? 1 : 0;
    }
    cbar();   // slots and group slots are complete
    tc::arrive(&sm.ready);
    const int gs = sm.group_slot[w];
    // the stored weight of a lane is its first pixel's, plus its second's when they share a slot
    const float s1 = pair_same ? 1.f : 0.f;

    float wsum0 = 0.f, wsum1 = 0.f, Tf0 = 0.f, Tf1 = 0.f;   // diagnostics: weight sum, T at the stop
    uint64_t CNT = pk(0.f, 0.f);   // contributions of both pixels (exact: counts below 2^24)
    // examined pairs: a stopped pixel examined the list up to the end of the chunk (32 candidates
    // of the tile's list) in which it stopped (position evp in the tile's candidate order); the
    // others examined every candidate the warp went through (seen)
    int evp0 = 0, evp1 = 0, seen = 0;
    unsigned long long executed = 0;   // Gaussians this warp evaluated for all 64 of its pixels
    float *wb_warp = sm.wbuf[w];
    int32_t *cl = sm.clist[w];
    float4 *stg = sm.stage[w];

    for (int it = 0;; ++it) {
        const int b = it % kNB;
        if (!wait_phase(a, sm, &sm.full[b], (uint32_t)(it / kNB) & 1u)) break;
        const int nb = sm.count[b];
        if (nb < 0) break;
        const float4 *q0 = sm.q0[b];
        const float4 *q1 = sm.q1[b];
        const float *qt = sm.qt[b];
        for (int c = 0; c * 32 < nb; ++c) {
            const float2 T = unpk(PT);
            const bool alive0 = T.x >= kTStop, alive1 = T.y >= kTStop;
            if (!__any_sync(0xffffffffu, alive0 || alive1)) break;
            const int nvalid = min(32, nb - c * 32);
            // which of the chunk's Gaussians can reach alpha >= 1/255 inside this warp's pixels: lane
            // j tests Gaussian c*32 + j against the warp's box
            bool hitw = false;
            float4 qa, qb;
            float mx = 0.f, my = 0.f;
            if (lane < nvalid) {
                // the record (mu'x, mu'y, a', b'), (c', log2 o, r1, r2) and t; mean tile-local
                qa = q0[c * 32 + lane];
                qb = q1[c * 32 + lane];
                mx = qa.x - ox;
                my = qa.y - oy;
                hitw = reaches(mx, my, qb.z, qb.w, qa.z, qa.w, qb.x, qt[c * 32 + lane], wbox);
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, hitw);
            if (mask == 0) continue;
            const int n = __popc(mask);
            executed += (unsigned long long)n;
            // the survivors in chunk order: survivor r's coefficients go to half (r & 1) of staged
            // pair r / 2; an odd count is padded with a Gaussian that reaches no pixel (e = -inf).
            // With pixel centres X = px + 0.5 - ox, Y likewise, and the tile-local mean (mx, my),
            // the exponent q2 + log2 o = a' dx^2 + b' dx dy + c' dy^2 + log2 o (dx = mx - X,
            // dy = my - Y) is K0 + K1 X + K2 Y + A X^2 + Bc X Y + C Y^2 (poly_coeffs).
            if (hitw) {
                const int r = __popc(mask & lt);
                float K0, K1, K2;
                poly_coeffs(mx, my, qa.z, qa.w, qb.x, qb.y, K0, K1, K2);
                float *sp = reinterpret_cast<float *>(stg + (r >> 1) * 3) + (r & 1);
                sp[0] = K0;
                sp[2] = K1;
                sp[4] = K2;
                sp[6] = qa.z;
                sp[8] = qa.w;
                sp[10] = qb.x;
                cl[r] = lane;
            }
            if (lane == 0 && (n & 1)) {
                float *sp = reinterpret_cast<float *>(stg + (n >> 1) * 3) + 1;
                sp[0] = -INFINITY;
                sp[2] = sp[4] = sp[6] = sp[8] = sp[10] = 0.f;
                cl[n] = 0;   // a valid chunk position: the kernel weight reads the pad's record
            }
            __syncwarp();
            // A: composite the survivors for this thread's two pixels, two Gaussians at a time: the
            // packed exponents of a pair at each pixel and the four exp2 are independent; only each
            // pixel's transmittance updates run in order. Floor and stop decisions are 0/1 factors.
            for (int i = 0; i < n; i += 2) {
                const ulonglong2 *cp = reinterpret_cast<const ulonglong2 *>(stg + (i >> 1) * 3);
                const ulonglong2 c0 = cp[0], c1 = cp[1], c2 = cp[2];   // (K0, K1), (K2, A), (Bc, C) pairs
                const float2 E0 = unpk(fma2(c2.y, YY0d, fma2(c2.x, XY0d, fma2(c1.y, XX0d, fma2(c1.x, Y0d,
                                       fma2(c0.y, X0d, c0.x))))));
                const float2 E1 = unpk(fma2(c2.y, YY1d, fma2(c2.x, XY1d, fma2(c1.y, XX1d, fma2(c1.x, Y1d,
                                       fma2(c0.y, X1d, c0.x))))));
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    // e = q2 + log2 opacity of Gaussian i + k at both pixels; q2 <= 0 holds exactly
                    // (positive definite conic)
                    const float e0 = k ? E0.y : E0.x, e1 = k ? E1.y : E1.x;
                    // FL: alpha >= 1/255; NAL = -alpha (0 below the floor)
                    const uint64_t FL = pk(set_ge(e0, kLog2AlphaMin), set_ge(e1, kLog2AlphaMin));
                    const uint64_t NAL = mul2(pk(fmaxf(-0.99f, -fast_exp2(e0)), fmaxf(-0.99f, -fast_exp2(e1))), FL);
                    // the Gaussian whose (1 - alpha) takes T below kTStop stops the pixel and
                    // contributes nothing (M = 0), nor does any later one; alpha = 0 leaves T as it
                    // is. Weights are kept negated (nw = -w), as the packed products give them.
                    const uint64_t Tn = fma2(NAL, PT, PT);   // T - alpha T
                    const float2 tn = unpk(Tn);
                    const uint64_t M = pk(set_ge(tn.x, kTStop), set_ge(tn.y, kTStop));
                    float2 nw;
                    if (kKernel) {
                        const float lo = q1[c * 32 + cl[i + k]].y;
                        nw = unpk(mul2(mul2(pk(-fast_exp2(e0 - lo), -fast_exp2(e1 - lo)), FL), M));
                    } else {
                        nw = unpk(mul2(mul2(NAL, PT), M));   // -alpha T, or 0 at the stop
                    }
                    if (kDebug) {
                        const float2 Tb = unpk(PT);
                        Tf0 = (tn.x < kTStop && Tb.x >= kTStop) ? Tb.x : Tf0;
                        Tf1 = (tn.y < kTStop && Tb.y >= kTStop) ? Tb.y : Tf1;
                        wsum0 -= nw.x;
                        wsum1 -= nw.y;
                    }
                    PT = Tn;
                    CNT = fma2(FL, M, CNT);
                    wb_warp[(i + k) * kWStride + lane] = fmaf(nw.y, s1, nw.x);
                    if (split1 && nw.y != 0.f) flush_slot(a, sm, b, slot1, c * 32 + cl[i + k], -nw.y);
                }
            }
            {
                const float2 Ta = unpk(PT);
                evp0 = (alive0 && !(Ta.x >= kTStop)) ? seen + c * 32 + nvalid : evp0;
                evp1 = (alive1 && !(Ta.y >= kTStop)) ? seen + c * 32 + nvalid : evp1;
            }
            __syncwarp();
            // B: lane r = survivor r, sum over this warp's 32 lanes per slot
            if (a.accumulate && gs != -1 && lane < n) {
                const float *row = wb_warp + lane * kWStride;
                const int gi = c * 32 + cl[lane];
                if (gs >= 0) {
                    // four running sums (lanes q mod 4), two per packed add
                    const float4 *row4 = reinterpret_cast<const float4 *>(row);
                    uint64_t s01 = pk(0.f, 0.f), s23 = pk(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 v = row4[q];
                        s01 = add2(s01, pk(v.x, v.y));
                        s23 = add2(s23, pk(v.z, v.w));
                    }
                    const float2 a01 = unpk(s01), a23 = unpk(s23);
                    const float acc = -((a01.x + a01.y) + (a23.x + a23.y));   // the buffer holds -w
                    if (acc != 0.f) flush_slot(a, sm, b, gs, gi, acc);
                } else {
                    int cur = sm.slot_lane[w * 32];
                    float acc = 0.f;
                    for (int q = 0; q < 32; ++q) {
                        const int sl = sm.slot_lane[w * 32 + q];
                        if (sl != cur) {
                            if (cur >= 0 && acc != 0.f) flush_slot(a, sm, b, cur, gi, acc);
                            acc = 0.f;
                            cur = sl;
                        }
                        acc -= row[q];   // the buffer holds -w
                    }
                    if (cur >= 0 && acc != 0.f) flush_slot(a, sm, b, cur, gi, acc);
                }
            }
            __syncwarp();
        }
        seen += nb;
        {
            const float2 T = unpk(PT);
            const bool any = __any_sync(0xffffffffu, T.x >= kTStop || T.y >= kTStop);
            if (lane == 0) sm.warp_live[w] = any ? 1 : 0;
        }
        __syncwarp();
        tc::arrive(&sm.empty[b]);   // every lane: each releases its own reads and sums
    }

    const float2 Tfin = unpk(PT);
    const float T0 = Tfin.x, T1 = Tfin.y;
    const float2 cntf = unpk(CNT);
    const int count0 = (int)cntf.x, count1 = (int)cntf.y;
    if (inside0) {
        const int64_t pi = (int64_t)py0 * W + px0;
        if (a.dbg_T) a.dbg_T[pi] = T0 >= kTStop ? T0 : Tf0;
        if (a.dbg_wsum) a.dbg_wsum[pi] = wsum0;
        if (a.dbg_count) a.dbg_count[pi] = count0;
    }
    if (inside1) {
        const int64_t pi = (int64_t)py1 * W + px1;
        if (a.dbg_T) a.dbg_T[pi] = T1 >= kTStop ? T1 : Tf1;
        if (a.dbg_wsum) a.dbg_wsum[pi] = wsum1;
        if (a.dbg_count) a.dbg_count[pi] = count1;
    }
    const int ev0 = inside0 ? (T0 >= kTStop ? seen : evp0) : 0, ev1 = inside1 ? (T1 >= kTStop ? seen : evp1) : 0;
    unsigned long long cnt = (unsigned long long)(count0 + count1), ev = (unsigned long long)(ev0 + ev1);
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
    }
    // one atomic per CTA and counter (counters shared by the whole grid)
    if (lane == 0) {
        sm.totals[w][0] = cnt;
        sm.totals[w][1] = ev;
        sm.totals[w][2] = executed * (unsigned long long)(2 * 32);
    }
    cbar();
    if (tid < 3) {
        unsigned long long t = 0;
#pragma unroll
        for (int q = 0; q < kConsumers; ++q) t += sm.totals[q][tid];
        unsigned long long *dst = tid == 0 ? a.contrib : (tid == 1 ? a.evals : a.evals_exec);
        if (t && dst) atomicAdd(dst, t);
    }
}

}  // namespace

void launch_composite(const CompositeArgs &a, cudaStream_t st) {
    const int tiles = a.cam.tiles_x * a.cam.tiles_y;
    const bool kernel = a.weight_mode == SLAG_WEIGHT_KERNEL;
    const bool debug = a.dbg_T || a.dbg_wsum || a.dbg_count;
    auto *kfn = kernel ? (debug ? composite_k<true, true> : composite_k<true, false>)
                       : (debug ? composite_k<false, true> : composite_k<false, false>);
    // on failure the error stays recorded for the caller's cudaGetLastError check
    if (set_max_smem((const void *)kfn, (int)sizeof(Smem)) != cudaSuccess) return;
    kfn<<<tiles, kThreads, sizeof(Smem), st>>>(a); note_launch();
}

SLAG_CHECKS_TAKE(checks_take_composite)

}  // namespace slag
