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
// One CTA (64 threads, one pixel each) per 16x4 quarter of a 16x16 tile; the
// tile's Gaussians are those of its bin's list (a 4x4-tile super-tile) whose
// tile rectangle holds the tile, taken in list order:
//   * the quarter's pixels are reordered by segment ("slot"), so that each
//     warp's 32 pixels usually share one segment;
//   * records of up to 192 Gaussians at a time are staged in shared memory; a
//     record holds mu', the conic scaled by -log2(e)/2 (so that alpha =
//     min(0.99, 2^(q2 + log2 opacity)) needs one SFU exp2 and the alpha
//     floor is tested on the exponent before it), and the half extents of
//     the alpha >= 1/255 ellipse;
//   * per chunk of 32 Gaussians, each warp keeps (ballot) only those whose
//     alpha >= 1/255 ellipse box meets the box of its 32 pixel centres --
//     the others cannot contribute to any of its pixels -- composites its
//     32 pixels against them, storing the weights in a padded shared 32 x 32
//     buffer, then reads the buffer transposed: lane j sums Gaussian j over
//     the warp's pixels per slot and adds the partial into a shared
//     (slot x Gaussian) table;
//   * after each batch the non-zero table entries are queued in shared memory
//     and moved, a block at a time, to the view's record list; a separate
//     combine pass (many records in flight per SM) adds them to the per-view
//     (segment, weight) table of each Gaussian (4 slots per Gaussian; further
//     segments are appended directly as triples). Probing the tables here
//     would leave each CTA waiting on a dependent chain of L2 round trips.
#include "slag_internal.cuh"

namespace slag {

namespace {

constexpr int kRows = 4;                              // tile rows per CTA: a 16x16 tile = 4 CTAs
constexpr int kThreads = kTile * kRows;               // 64: one pixel per thread
constexpr int kSubTiles = kTile / kRows;
constexpr int kRound = 128;                           // candidates examined per fill round
constexpr int kBatch = 64 + kRound;                   // record capacity of a batch
constexpr int kSmemSlots = 4;
constexpr int kRecBuf = 256;                          // queued (Gaussian, slot) sums of a CTA
constexpr int kRecFlush = 128;                        // queue level that triggers a flush after a batch
constexpr int kWStride = 33;
constexpr float kLog2AlphaMin = -7.99435343685886f;   // log2(1/255)

struct Smem {
    float4 rec_a[kBatch];                 // (mu'x, mu'y, a', b')
    float4 rec_b[kBatch];                 // (c', log2 opacity, ex, ey)
    uint32_t gid[kBatch];                 // internal Gaussian index
    int32_t fill[4];                      // per-warp hit counts of a fill round
    float wb[kSmemSlots][kBatch];         // per (slot, Gaussian of the batch)
    float wbuf[kThreads / 32][32 * kWStride];
    uint32_t keys[kThreads];
    int32_t slot_of_pos[kThreads];
    int32_t seg_of_slot[kThreads];
    int32_t group_slot[kThreads / 32];    // slot shared by a warp's 32 positions, -2 = mixed
    int32_t scalar[4];
    uint32_t rec_g[kRecBuf];              // queued sums: Gaussian, weight, shared slot
    float rec_w[kRecBuf];
    uint8_t rec_s[kRecBuf];
    int32_t nrec;
    unsigned long long rec_base;
};
// 10 CTAs per SM (228 KB of shared memory, 1 KB of it reserved per CTA)
static_assert(sizeof(Smem) + 1024 <= 233472 / 10, "composite shared memory above the 10-CTA budget");

__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
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

__device__ __forceinline__ HashSink sink_of(const CompositeArgs &a) {
    return HashSink{a.hash, a.log_count, a.log_cap, a.log_key, a.log_w, a.s_ovf, a.overflow, a.view_base};
}

__device__ __forceinline__ void flush_slot(const CompositeArgs &a, Smem &sm, int slot, int gi, float acc) {
    if (slot < kSmemSlots) atomicAdd(&sm.wb[slot][gi], acc);
    else sink_add(sink_of(a), sm.gid[gi], sm.seg_of_slot[slot], acc);
}

// Moves the queued records to the view's record list: one reservation for
// all of them. Every thread of the CTA calls it (after a barrier).
__device__ void flush_queue(const CompositeArgs &a, Smem &sm, int tid) {
    const int nr = min(sm.nrec, kRecBuf);
    if (tid == 0) sm.rec_base = nr ? atomicAdd(a.rec_count, (unsigned long long)nr) : 0ull;
    __syncthreads();
    const unsigned long long base = sm.rec_base;
    for (int k = tid; k < nr; k += kThreads) {
        const uint32_t g = sm.rec_g[k];
        const int32_t seg = sm.seg_of_slot[sm.rec_s[k]];
        const float w = sm.rec_w[k];
        if (base + (unsigned long long)k < a.rec_cap) {
            WeightRecord r;
            r.g = g;
            r.seg = seg;
            r.w = w;
            r.pad = 0u;
            a.recs[base + k] = r;
        } else {
            sink_add(sink_of(a), g, seg, w);
        }
    }
    __syncthreads();
    if (tid == 0) sm.nrec = 0;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(kThreads, 14) composite_k(const CompositeArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int tile = (int)a.tile_order[blockIdx.x / kSubTiles];
    const int row0 = (int)(blockIdx.x % kSubTiles) * kRows;    // first tile row of this CTA
    const int tx = tile % a.cam.tiles_x, ty = tile / a.cam.tiles_x;
    const int W = a.cam.width, H = a.cam.height;

    // ---- segment of each pixel, slot-sorted positions --------------------------------
    int32_t s_nat;
    {
        int px = tx * kTile + (tid & 15), py = ty * kTile + row0 + (tid >> 4);
        bool inside = px < W && py < H;
        s_nat = (inside && a.seg && a.accumulate) ? a.seg[(int64_t)py * W + px] : -1;
        if (s_nat < -1) s_nat = -1;
        sm.keys[tid] = ((uint32_t)(s_nat + 1) << 8) | (uint32_t)tid;
    }
    // (pixel index within the CTA fits in the low 8 bits of a key)
    if (tid == 0) {
        sm.scalar[0] = s_nat;
        sm.nrec = 0;
    }
    __syncthreads();
    const bool uniform = __syncthreads_and(s_nat == sm.scalar[0]);
    int pos;
    if (uniform) {
        pos = tid;
    } else {
        const uint32_t mine = sm.keys[tid];
        int rank = 0;
#pragma unroll 8
        for (int q = 0; q < kThreads; ++q) rank += sm.keys[q] < mine ? 1 : 0;
        pos = rank;
    }
    __syncthreads();
    sm.keys[pos] = ((uint32_t)(s_nat + 1) << 8) | (uint32_t)tid;   // position -> (segment, pixel)
    __syncthreads();
    // my position is tid from here on
    const uint32_t kp = sm.keys[tid];
    const int pix = (int)(kp & 255u);
    const int32_t my_seg = (int32_t)(kp >> 8) - 1;
    bool is_new = my_seg >= 0 && (tid == 0 || (int32_t)(sm.keys[tid - 1] >> 8) - 1 != my_seg);
    // inclusive prefix count of is_new over positions
    uint32_t bal = __ballot_sync(0xffffffffu, is_new);
    if (lane == 0) sm.group_slot[w] = __popc(bal);
    __syncthreads();
    int before = 0, nslots = 0;
    for (int q = 0; q < kThreads / 32; ++q) {
        int c = sm.group_slot[q];
        if (q < w) before += c;
        nslots += c;
    }
    const int my_slot = my_seg >= 0 ? before + __popc(bal & ((2u << lane) - 1u)) - 1 : -1;
    __syncthreads();
    sm.slot_of_pos[tid] = my_slot;
    if (is_new) sm.seg_of_slot[my_slot] = my_seg;
    {
        int first = __shfl_sync(0xffffffffu, my_slot, 0);
        bool same = __all_sync(0xffffffffu, my_slot == first);
        if (lane == 0) sm.group_slot[w] = same ? first : -2;
    }
    const int ns_smem = nslots < kSmemSlots ? nslots : kSmemSlots;

    const int px = tx * kTile + (pix & 15), py = ty * kTile + row0 + (pix >> 4);
    const bool inside = px < W && py < H;
    const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
    // bounding box of this warp's pixel centres (culling of Gaussians per warp)
    float wx0 = inside ? pxc : INFINITY, wx1 = inside ? pxc : -INFINITY;
    float wy0 = inside ? pyc : INFINITY, wy1 = inside ? pyc : -INFINITY;
    for (int o = 16; o; o >>= 1) {
        wx0 = fminf(wx0, __shfl_xor_sync(0xffffffffu, wx0, o));
        wx1 = fmaxf(wx1, __shfl_xor_sync(0xffffffffu, wx1, o));
        wy0 = fminf(wy0, __shfl_xor_sync(0xffffffffu, wy0, o));
        wy1 = fmaxf(wy1, __shfl_xor_sync(0xffffffffu, wy1, o));
    }
    float T = 1.f, wsum = 0.f;
    int count = 0, evals = 0;
    bool done = !inside;
    const bool kernel_mode = a.weight_mode == SLAG_WEIGHT_KERNEL;

    // this tile's candidates: the depth-ordered list of its bin (a 2^shift x
    // 2^shift square of tiles); the Gaussians whose tile rectangle holds this tile
    // form, in the same order, the tile's own list
    const uint2 rg = a.ranges[(ty >> a.bin_shift) * a.bins_x + (tx >> a.bin_shift)];
    const int end = (int)rg.y;
    int cursor = (int)rg.x;
    float *wb_warp = sm.wbuf[w];
    const uint32_t lt = lanemask_lt();

    // candidates of the next fill round, prefetched into registers
    constexpr int kPer = kRound / kThreads;
    uint32_t r_nx[kPer];
    uint2 rc_nx[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int c = cursor + k * kThreads + tid;
        r_nx[k] = c < end ? a.list[c] : 0u;
        rc_nx[k] = c < end ? a.prect[c] : make_uint2(0u, 0u);
    }

    while (true) {
        int live = __syncthreads_count(!done);   // also: the previous batch is fully consumed
        if (live == 0 || cursor >= end) break;
        // fill: rounds of kRound candidates until at least 64 records are staged; the
        // records of the hits are copied asynchronously, the next round's candidates
        // are loaded while this round is compacted
        int nb = 0;
        while (nb < kBatch - kRound && cursor < end) {
            uint32_t r[kPer];
            bool hit[kPer];
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const int c = cursor + k * kThreads + tid;
                r[k] = r_nx[k];
                const uint2 rc = rc_nx[k];
                hit[k] = c < end && (uint32_t)tx >= (rc.x & 0xffffu) && (uint32_t)tx < (rc.x >> 16) &&
                         (uint32_t)ty >= (rc.y & 0xffffu) && (uint32_t)ty < (rc.y >> 16);
                const int cn = c + kRound;
                r_nx[k] = cn < end ? a.list[cn] : 0u;
                rc_nx[k] = cn < end ? a.prect[cn] : make_uint2(0u, 0u);
            }
            // stable compaction: candidate order is (k, warp, lane)
            uint32_t bal[kPer];
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                bal[k] = __ballot_sync(0xffffffffu, hit[k]);
                if (lane == 0) sm.fill[k * (kThreads / 32) + w] = __popc(bal[k]);
            }
            __syncthreads();
            int nh = 0;
            for (int q = 0; q < kPer * (kThreads / 32); ++q) nh += sm.fill[q];
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                int bk = 0;
                for (int q = 0; q < k * (kThreads / 32) + w; ++q) bk += sm.fill[q];
                if (hit[k]) {
                    const int pos = nb + bk + __popc(bal[k] & lt);
                    cp_async16(&sm.rec_a[pos], a.srec_a + r[k]);
                    cp_async16(&sm.rec_b[pos], a.srec_b + r[k]);
                    cp_async4(&sm.gid[pos], a.sgid + r[k]);
                }
            }
            nb += nh;
            cursor += kRound;
            __syncthreads();
        }
        cp_async_wait_all();
        __syncthreads();
        if (nb == 0) continue;
        if (tid < kBatch)
            for (int s2 = 0; s2 < ns_smem; ++s2) sm.wb[s2][tid] = 0.f;
        for (int i = tid + kThreads; i < nb; i += kThreads)
            for (int s2 = 0; s2 < ns_smem; ++s2) sm.wb[s2][i] = 0.f;
        __syncthreads();
        const float4 *rec_a = sm.rec_a;
        const float4 *rec_b = sm.rec_b;
        const int gs = sm.group_slot[w];
        for (int c = 0; c * 32 < nb; ++c) {
            if (!__any_sync(0xffffffffu, !done)) break;
            const int nvalid = min(32, nb - c * 32);
            // which of the chunk's Gaussians can reach alpha >= 1/255 inside this warp's pixels
            bool hitw = false;
            if (lane < nvalid) {
                const float4 ra = rec_a[c * 32 + lane];
                const float4 rb = rec_b[c * 32 + lane];
                hitw = (ra.x - rb.z <= wx1) && (ra.x + rb.z >= wx0) && (ra.y - rb.w <= wy1) && (ra.y + rb.w >= wy0);
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, hitw);
            if (!done) evals += nvalid;
            if (mask == 0) continue;
            // A: composite the surviving Gaussians for this thread's pixel, four at a time:
            // the exponents and exp2 of a group are independent; only the transmittance
            // updates run in order
            uint32_t m = mask;
            while (m) {
                int jj[4];
                float al[4], kq[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    jj[k] = m ? __ffs(m) - 1 : -1;
                    m &= m ? m - 1 : 0u;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    al[k] = 0.f;
                    kq[k] = 0.f;
                    if (jj[k] >= 0) {
                        const float4 ra = rec_a[c * 32 + jj[k]];
                        const float4 rb = rec_b[c * 32 + jj[k]];
                        const float dx = ra.x - pxc, dy = ra.y - pyc;
                        const float u = fmaf(ra.z, dx, ra.w * dy);
                        const float q2 = fmaf(u, dx, rb.x * dy * dy);
                        const float e = q2 + rb.y;
                        if (q2 <= 0.f && e >= kLog2AlphaMin) {
                            al[k] = fminf(0.99f, fast_exp2(e));
                            kq[k] = q2;
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (jj[k] < 0) break;
                    float wv = 0.f;
                    if (!done && al[k] > 0.f) {
                        const float Tn = T - al[k] * T;
                        if (Tn < 1e-4f) {
                            done = true;
                            evals -= nvalid - 1 - jj[k];
                        } else {
                            wv = kernel_mode ? fast_exp2(kq[k]) : al[k] * T;
                            T = Tn;
                            wsum += wv;
                            ++count;
                        }
                    }
                    wb_warp[jj[k] * kWStride + lane] = wv;
                }
            }
            __syncwarp();
            // B: lane = Gaussian c*32+lane, sum over this warp's 32 positions per slot
            if (a.accumulate && gs != -1 && ((mask >> lane) & 1u)) {
                const float *row = wb_warp + lane * kWStride;
                const int gi = c * 32 + lane;
                if (gs >= 0) {
                    float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
                    for (int q = 0; q < 32; q += 4) {
                        p0 += row[q];
                        p1 += row[q + 1];
                        p2 += row[q + 2];
                        p3 += row[q + 3];
                    }
                    const float acc = (p0 + p1) + (p2 + p3);
                    if (acc != 0.f) flush_slot(a, sm, gs, gi, acc);
                } else {
                    int cur = sm.slot_of_pos[w * 32];
                    float acc = 0.f;
                    for (int q = 0; q < 32; ++q) {
                        const int sl = sm.slot_of_pos[w * 32 + q];
                        if (sl != cur) {
                            if (cur >= 0 && acc != 0.f) flush_slot(a, sm, cur, gi, acc);
                            acc = 0.f;
                            cur = sl;
                        }
                        acc += row[q];
                    }
                    if (cur >= 0 && acc != 0.f) flush_slot(a, sm, cur, gi, acc);
                }
            }
            __syncwarp();
        }
        __syncthreads();
        // C: per Gaussian of the batch, the non-zero (segment, sum) entries are queued;
        // the queue goes to the view's record list in blocks, and the combine pass
        // adds the records to the per-Gaussian tables
        if (a.accumulate) {
            for (int i0 = 0; i0 < nb; i0 += kThreads) {
                const int i = i0 + tid;
                const bool valid = i < nb;
                const uint32_t g = valid ? sm.gid[i] : 0u;
                for (int s2 = 0; s2 < ns_smem; ++s2) {
                    const float v = valid ? sm.wb[s2][i] : 0.f;
                    const uint32_t bal = __ballot_sync(0xffffffffu, v != 0.f);
                    if (bal == 0u) continue;
                    // one queue reservation per warp; without room (or without a record
                    // list) the sum goes to the Gaussian's table directly
                    int base = kRecBuf;
                    if (lane == 0 && a.recs) base = atomicAdd(&sm.nrec, __popc(bal));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (v != 0.f) {
                        const int k = base + __popc(bal & lt);
                        if (k < kRecBuf) {
                            sm.rec_g[k] = g;
                            sm.rec_w[k] = v;
                            sm.rec_s[k] = (uint8_t)s2;
                        } else {
                            sink_add(sink_of(a), g, sm.seg_of_slot[s2], v);
                        }
                    }
                }
            }
            __syncthreads();
            if (sm.nrec >= kRecFlush) flush_queue(a, sm, tid);
        }
    }
    if (a.accumulate && a.recs) flush_queue(a, sm, tid);

    if (inside) {
        const int64_t pi = (int64_t)py * W + px;
        if (a.dbg_T) a.dbg_T[pi] = T;
        if (a.dbg_wsum) a.dbg_wsum[pi] = wsum;
        if (a.dbg_count) a.dbg_count[pi] = count;
    }
    unsigned long long cnt = (unsigned long long)count, ev = (unsigned long long)evals;
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
    }
    if (lane == 0 && cnt) atomicAdd(a.contrib, cnt);
    if (lane == 0 && ev && a.evals) atomicAdd(a.evals, ev);
}

}  // namespace

void launch_composite(const CompositeArgs &a, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(composite_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
        attr_set = true;
    }
    const int tiles = a.cam.tiles_x * a.cam.tiles_y;
    composite_k<<<tiles * kSubTiles, kThreads, sizeof(Smem), st>>>(a); note_launch();
}

}  // namespace slag
