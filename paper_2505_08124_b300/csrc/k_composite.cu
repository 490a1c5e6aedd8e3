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
// One CTA (256 threads) per 16x16 tile:
//   * the tile's pixels are reordered by segment ("slot"), so that each warp's
//     32 pixels usually share one segment;
//   * records of 256 Gaussians at a time are staged in shared memory; a
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
//   * after each batch the non-zero table entries go into the per-view
//     (segment, weight) table of each Gaussian in global memory (4 slots per
//     Gaussian; further segments are appended directly as triples).
#include "slag_internal.cuh"

namespace slag {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 256;
constexpr int kSmemSlots = 8;
constexpr int kWStride = 33;
constexpr float kLog2AlphaMin = -7.99435343685886f;   // log2(1/255)

struct Smem {
    float4 rec_a[kBatch];                 // (mu'x, mu'y, a', b')
    float4 rec_b[kBatch];                 // (c', log2 opacity, ex, ey)
    uint32_t gid[kBatch];                 // internal Gaussian index
    float wb[kSmemSlots][kBatch];         // per (slot, Gaussian of the batch)
    float wbuf[kThreads / 32][32 * kWStride];
    uint32_t keys[kThreads];
    int32_t slot_of_pos[kThreads];
    int32_t seg_of_slot[kThreads];
    int32_t group_slot[kThreads / 32];    // slot shared by a warp's 32 positions, -2 = mixed
    int32_t scalar[4];
};

__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint64_t pack_key(uint32_t g, uint32_t col) {
    return ((uint64_t)(g >> 7) << 39) | ((uint64_t)col << 7) | (uint64_t)(g & 127u);
}

__device__ void append_triple(const CompositeArgs &a, uint32_t g, int32_t seg, float w) {
    unsigned long long idx = atomicAdd(a.log_count, 1ull);
    if (idx < a.log_cap) {
        a.log_key[idx] = pack_key(g, (uint32_t)(a.view_base + seg));
        a.log_w[idx] = w;
        atomicAdd(&a.s_ovf[g], w);
    } else {
        atomicOr(a.overflow, 1u);
    }
}

// Adds w to the (segment, weight) slot of Gaussian g, claiming a free slot if needed.
__device__ void hash_add(const CompositeArgs &a, uint32_t g, int32_t seg, float w) {
    HashEntry *h = a.hash + g;
#pragma unroll
    for (int s = 0; s < kHashSlots; ++s) {
        int32_t cur = *((volatile int32_t *)&h->seg[s]);
        if (cur == -1) {
            cur = atomicCAS(&h->seg[s], -1, seg);
            if (cur == -1) cur = seg;
        }
        if (cur == seg) {
            atomicAdd(&h->w[s], w);
            return;
        }
    }
    append_triple(a, g, seg, w);
}

__device__ __forceinline__ void flush_slot(const CompositeArgs &a, Smem &sm, int slot, int gi, float acc) {
    if (slot < kSmemSlots) atomicAdd(&sm.wb[slot][gi], acc);
    else hash_add(a, sm.gid[gi], sm.seg_of_slot[slot], acc);
}

__global__ void __launch_bounds__(kThreads, 4) composite_k(const CompositeArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x;
    const int tx = tile % a.cam.tiles_x, ty = tile / a.cam.tiles_x;
    const int W = a.cam.width, H = a.cam.height;

    // ---- segment of each pixel, slot-sorted positions --------------------------------
    int32_t s_nat;
    {
        int px = tx * kTile + (tid & 15), py = ty * kTile + (tid >> 4);
        bool inside = px < W && py < H;
        s_nat = (inside && a.seg && a.accumulate) ? a.seg[(int64_t)py * W + px] : -1;
        if (s_nat < -1) s_nat = -1;
        sm.keys[tid] = ((uint32_t)(s_nat + 1) << 8) | (uint32_t)tid;
    }
    if (tid == 0) sm.scalar[0] = s_nat;
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

    const int px = tx * kTile + (pix & 15), py = ty * kTile + (pix >> 4);
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

    const uint2 rg = a.ranges[tile];
    const int start = (int)rg.x, end = (int)rg.y;
    float *wb_warp = sm.wbuf[w];

    for (int b = start; b < end; b += kBatch) {
        int live = __syncthreads_count(!done);   // also: the previous batch is fully consumed
        if (live == 0) break;
        const int nb = min(kBatch, end - b);
        if (tid < nb) {
            const uint32_t r = a.list[b + tid];
            sm.rec_a[tid] = a.srec_a[r];
            sm.rec_b[tid] = a.srec_b[r];
            sm.gid[tid] = a.sgid[r];
        }
        for (int s = 0; s < ns_smem; ++s) sm.wb[s][tid] = 0.f;
        __syncthreads();
        const int gs = sm.group_slot[w];
        for (int c = 0; c * 32 < nb; ++c) {
            if (!__any_sync(0xffffffffu, !done)) break;
            const int nvalid = min(32, nb - c * 32);
            // which of the chunk's Gaussians can reach alpha >= 1/255 inside this warp's pixels
            bool hit = false;
            if (lane < nvalid) {
                const float4 ra = sm.rec_a[c * 32 + lane];
                const float4 rb = sm.rec_b[c * 32 + lane];
                hit = (ra.x - rb.z <= wx1) && (ra.x + rb.z >= wx0) && (ra.y - rb.w <= wy1) && (ra.y + rb.w >= wy0);
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, hit);
            if (!done) evals += nvalid;
            if (mask == 0) continue;
            // A: composite the surviving Gaussians for this thread's pixel
            uint32_t m = mask;
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                float wv = 0.f;
                if (!done) {
                    const float4 ra = sm.rec_a[c * 32 + j];
                    const float4 rb = sm.rec_b[c * 32 + j];
                    const float dx = ra.x - pxc, dy = ra.y - pyc;
                    const float u = fmaf(ra.z, dx, ra.w * dy);
                    const float q2 = fmaf(u, dx, rb.x * dy * dy);
                    const float e = q2 + rb.y;
                    if (q2 <= 0.f && e >= kLog2AlphaMin) {
                        const float alpha = fminf(0.99f, fast_exp2(e));
                        const float Tn = T - alpha * T;
                        if (Tn < 1e-4f) {
                            done = true;
                            evals -= nvalid - 1 - j;
                        } else {
                            wv = kernel_mode ? fast_exp2(q2) : alpha * T;
                            T = Tn;
                            wsum += wv;
                            ++count;
                        }
                    }
                }
                wb_warp[j * kWStride + lane] = wv;
            }
            __syncwarp();
            // B: lane = Gaussian c*32+lane, sum over this warp's 32 positions per slot
            if (a.accumulate && gs != -1 && ((mask >> lane) & 1u)) {
                const float *row = wb_warp + lane * kWStride;
                const int gi = c * 32 + lane;
                if (gs >= 0) {
                    float acc = 0.f;
#pragma unroll
                    for (int q = 0; q < 32; ++q) acc += row[q];
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
        // C: per Gaussian of the batch, push the non-zero (segment, sum) entries
        if (a.accumulate && tid < nb) {
            const uint32_t g = sm.gid[tid];
            for (int s = 0; s < ns_smem; ++s) {
                const float v = sm.wb[s][tid];
                if (v != 0.f) hash_add(a, g, sm.seg_of_slot[s], v);
            }
        }
    }

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
    composite_k<<<tiles, kThreads, sizeof(Smem), st>>>(a);
}

}  // namespace slag
