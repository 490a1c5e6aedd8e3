// Stable LSD radix sort and exclusive scan (no CUB).
//
// Radix sort, one pass per digit of <= 11 bits (256, 512, 1024 or 2048 bins), three
// kernels per pass, over tiles of 256 x ITEMS items (ITEMS = 16, or 4 below
// ~1M items so that the grid still covers the GPU):
//   1. rs_hist:    each CTA counts the digits of its tile into per-warp
//                  shared histograms (one add per distinct digit of a warp
//                  round); writes hist[digit][tile] and adds the digit totals.
//   2. rs_offsets: one CTA per digit scans hist[digit][*] over the tiles and
//                  writes the digit's total.
//   3. rs_scatter: each CTA scans the digit totals (digit starts), ranks its tile stably (warp w owns items
//                  [w*32*ITEMS, (w+1)*32*ITEMS) of the tile in rounds of 32,
//                  so (warp, round, lane) order is input order; equal digits
//                  within a round are found with one ballot per digit bit),
//                  stages the tile in shared memory in digit order and writes
//                  each digit's run contiguously.
// Exclusive scan of uint32: per-tile sums, a single-CTA scan of the sums, and
// a per-tile scan with the carried offset.
#include "slag_internal.cuh"

namespace slag {

SLAG_CHECKS_WORD


namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTileItems = kThreads * kItems;   // 4096
constexpr int kWarps = kThreads / 32;
constexpr int64_t kSmallSort = 1 << 20;         // sorts of fewer items use 1024-item tiles

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp whose digit equals this lane's: one ballot per digit bit.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, int width, bool valid) {
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
    for (int b = 0; b < width; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t ones = __ballot_sync(0xffffffffu, valid && bit);
        peers &= bit ? ones : ~ones;
    }
    return peers;
}

// Per-tile digit counts: per-warp shared histograms, one add per distinct digit of
// each 32-item round (the round's leader adds the popcount of its peers).
template <typename K, int ITEMS, int BINS>
__global__ void __launch_bounds__(kThreads) rs_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                    uint32_t mask, int width, uint32_t *__restrict__ hist,
                                                    int ntiles) {
    extern __shared__ __align__(16) uint32_t hsm[];   // kWarps x BINS
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kWarps * BINS; i += kThreads) hsm[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * (kThreads * ITEMS) + (int64_t)w * (32 * ITEMS);
    uint32_t *h = hsm + w * BINS;
#pragma unroll 4
    for (int r = 0; r < ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        const uint32_t d = valid ? (uint32_t)(keys[i] >> shift) & mask : 0u;
        const uint32_t peers = digit_peers(d, width, valid);
        if (valid && lane == __ffs(peers) - 1) h[d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = tid; d < BINS; d += kThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) s += hsm[q * BINS + d];
        hist[(int64_t)d * ntiles + blockIdx.x] = s;
    }
}

// One CTA per digit: exclusive scan of hist[d][*] over the tiles, in place;
// the row total goes to digit_tot[d].
__global__ void __launch_bounds__(1024) rs_offsets(uint32_t *__restrict__ hist, uint32_t *__restrict__ digit_tot,
                                                  int ntiles) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry_s;
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int nw = blockDim.x >> 5;
    uint32_t carry = 0;
    uint32_t *row = hist + (int64_t)d * ntiles;
    for (int base = 0; base < ntiles; base += blockDim.x) {
        int i = base + tid;
        uint32_t v = i < ntiles ? row[i] : 0;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t ws = lane < nw ? warp_sums[lane] : 0u;
            uint32_t wx = ws;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, wx, o);
                if (lane >= o) wx += y;
            }
            warp_sums[lane] = wx - ws;   // exclusive prefix of warp sums
        }
        __syncthreads();
        uint32_t excl = carry + warp_sums[w] + x - v;
        if (i < ntiles) row[i] = excl;
        __syncthreads();
        // carry for the next chunk: the last thread's exclusive value plus its own count
        if (tid == (int)blockDim.x - 1) carry_s = excl + v;
        __syncthreads();
        carry = carry_s;
    }
    if (tid == 0) digit_tot[d] = carry;
}

// One tile of a stable scatter pass, its items already in registers: item r of this thread is
// tile item w * 32 * ITEMS + r * 32 + lane (valid when its global index is below n), so (warp,
// round, lane) order is input order. Ranks the tile's items by digit, stages them in digit order
// in shared memory and writes each digit's run contiguously (keys to kout when it is non-null,
// values through vmap when given, the payload gsrc[value] to gout when given). Shared memory:
// scatter_smem<K, ITEMS, BINS>() bytes at smem_raw; the caller may have used the staging arrays
// (skeys, svals) for its own input, since they are written only after a barrier.
template <typename K, int ITEMS, int BINS>
__device__ __forceinline__ void scatter_tile(K (&key)[ITEMS], uint32_t (&val)[ITEMS], unsigned char *smem_raw,
                                             K *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                                             int shift, uint32_t mask, int width,
                                             const uint32_t *__restrict__ offs,
                                             const uint32_t *__restrict__ digit_tot, int ntiles,
                                             uint2 *__restrict__ ranges, int nranges,
                                             const uint2 *__restrict__ gsrc, uint2 *__restrict__ gout,
                                             const uint32_t *__restrict__ vmap) {
    constexpr int kTileN = kThreads * ITEMS;
    constexpr int kPer = BINS / kThreads;              // digits per thread in the per-tile scans
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem_raw);              // kWarps x BINS
    uint32_t *lstart = cnt + kWarps * BINS;                              // BINS
    uint32_t *gbase = lstart + BINS;                                     // BINS
    uint32_t *wsum = gbase + BINS;                                       // 16
    K *skeys = reinterpret_cast<K *>(wsum + 16);
    uint32_t *svals = reinterpret_cast<uint32_t *>(skeys + kTileN);

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    __syncthreads();   // the caller's reads of the staging arrays are done
    for (int i = tid; i < kWarps * BINS; i += kThreads) cnt[i] = 0;
    __syncthreads();

    const int64_t tile_base = (int64_t)blockIdx.x * kTileN;
    const int64_t base = tile_base + (int64_t)w * (32 * ITEMS);
    uint32_t pos[ITEMS];
    const uint32_t lt = lanemask_lt();
    uint32_t *cw = cnt + w * BINS;
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        const uint32_t d = (uint32_t)(key[r] >> shift) & mask;
        const uint32_t peers = digit_peers(d, width, valid);
        uint32_t c = 0;
        if (valid) c = cw[d];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cw[d] = c + __popc(peers);
        pos[r] = valid ? c + __popc(peers & lt) : 0xffffffffu;
        __syncwarp();
    }
    __syncthreads();
    // global start of each digit: exclusive scan of the digit totals (kept in gbase)
    {
        uint32_t dt[kPer];
        uint32_t dsum = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            dt[k] = digit_tot[tid * kPer + k];
            dsum += dt[k];
        }
        uint32_t x = dsum;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int q = 0; q < w; ++q) before += wsum[q];
        uint32_t run = before + x - dsum;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int d = tid * kPer + k;
            gbase[d] = run + offs[(int64_t)d * ntiles + blockIdx.x];
            if (ranges && blockIdx.x == 0 && d < nranges) ranges[d] = make_uint2(run, run + dt[k]);
            run += dt[k];
        }
        __syncthreads();
    }
    // per digit: exclusive prefix over warps (in place) and the tile's digit total
    uint32_t tot[kPer];
    uint32_t tsum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int d = tid * kPer + k;
        uint32_t s = 0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) {
            const uint32_t t = cnt[q * BINS + d];
            cnt[q * BINS + d] = s;
            s += t;
        }
        tot[k] = s;
        tsum += s;
    }
    // exclusive scan of the digit totals over the tile -> lstart
    {
        uint32_t x = tsum;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int q = 0; q < w; ++q) before += wsum[q];
        uint32_t run = before + x - tsum;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            lstart[tid * kPer + k] = run;
            run += tot[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        if (pos[r] != 0xffffffffu) {
            const uint32_t d = (uint32_t)(key[r] >> shift) & mask;
            const uint32_t lp = lstart[d] + cw[d] + pos[r];
            skeys[lp] = key[r];
            svals[lp] = val[r];
        }
    }
    __syncthreads();
    const int64_t rem = n - tile_base;
    const int tile_n = rem < kTileN ? (int)rem : kTileN;
    // each thread's ITEMS outputs: the gathers of all of them are issued before any store
    uint32_t gpo[ITEMS], vo[ITEMS];
    uint2 po[ITEMS];
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) {
        const int j = tid + q * kThreads;
        gpo[q] = 0xffffffffu;
        if (j < tile_n) {
            const K k = skeys[j];
            const uint32_t d = (uint32_t)(k >> shift) & mask;
            const uint32_t gp = gbase[d] + (uint32_t)j - lstart[d];
            if (SLAG_IN_BOUNDS((int64_t)gp < n, kCheckSort)) {
                gpo[q] = gp;
                if (kout) kout[gp] = k;
                const uint32_t v = svals[j];
                vo[q] = vmap ? vmap[v] : v;   // optionally written through a map of the values
                if (gout) po[q] = gsrc[v];    // a payload that follows the values (gathered by value)
            }
        }
    }
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) {
        if (gpo[q] == 0xffffffffu) continue;
        vout[gpo[q]] = vo[q];
        if (gout) gout[gpo[q]] = po[q];
    }
}

template <typename K, int ITEMS, int BINS>
__global__ void __launch_bounds__(kThreads) rs_scatter(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                       K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                       int64_t n, int shift, uint32_t mask, int width,
                                                       const uint32_t *__restrict__ offs,
                                                       const uint32_t *__restrict__ digit_tot, int ntiles,
                                                       uint2 *__restrict__ ranges, int nranges,
                                                       const uint2 *__restrict__ gsrc, uint2 *__restrict__ gout,
                                                       const uint32_t *__restrict__ vmap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * (kThreads * ITEMS) + (int64_t)w * (32 * ITEMS);
    K key[ITEMS];
    uint32_t val[ITEMS];
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        key[r] = valid ? kin[i] : (K)0;
        val[r] = valid ? vin[i] : 0u;
    }
    scatter_tile<K, ITEMS, BINS>(key, val, smem_raw, kout, vout, n, shift, mask, width, offs, digit_tot, ntiles,
                                 ranges, nranges, gsrc, gout, vmap);
}

// ---- binning by bin without materialised pairs ---------------------------------------------
// The pairs of a view, in emission order, are each visible Gaussian's bins (depth-rank order,
// each Gaussian's bins row-major in its bin rectangle); pair p of Gaussian r is number
// p - offsets[r] of r's rectangle. The fused binning sorts them by bin in one stable pass whose
// tiles (kTileItems consecutive pairs) generate their own pairs from the rectangles, so the
// emitted pair list is never written or read back.

// The sizes of a fused binning, read on the device (so that the host need not wait for the
// stage that counts them): nv visible Gaussians and P pairs. The pass holds at most cap pairs;
// a larger P sets *overflow and leaves every bin empty, or, with truncate (checked builds'
// forced capacities), keeps the first cap pairs.
struct BinCounts {
    const uint32_t *nv;
    const unsigned long long *P;
    int64_t cap;
    int truncate;
    uint32_t *overflow;
};

__device__ __forceinline__ int64_t pairs_held(const BinCounts &c) {
    const unsigned long long p = *c.P;
    if (p <= (unsigned long long)c.cap) return (int64_t)p;
    return c.truncate ? c.cap : 0;
}

// The Gaussian whose pairs hold the first pair of each tile: tstart[t] for t < the tiles of the
// pairs held. In the checked build, pairs beyond a forced capacity are refused here.
__global__ void __launch_bounds__(256) tile_starts_k(const uint32_t *__restrict__ offsets,
                                                     const uint32_t *__restrict__ counts, const BinCounts c,
                                                     uint32_t *__restrict__ tstart) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t P = pairs_held(c);
    if (r == 0 && !c.truncate && c.overflow && *c.P > (unsigned long long)c.cap) *c.overflow = 1u;
    const uint32_t nv = *c.nv;
    if (r >= nv) return;
    const int64_t ntiles = (P + kTileItems - 1) / kTileItems;
    const int64_t off = offsets[r], cnt = counts[r];
    if (r == (int64_t)nv - 1) (void)SLAG_IN_BOUNDS(off + cnt <= P || !c.truncate, kCheckEmit);
    if (cnt == 0) return;
    for (int64_t t = (off + kTileItems - 1) / kTileItems; t * kTileItems < off + cnt && t < ntiles; ++t)
        tstart[t] = (uint32_t)r;
}

// Calls f(j, bin, r) for every pair of this CTA's tile (below P, of ntiles tiles): j = its place
// in the tile, r = its Gaussian's depth rank. Threads take the tile's Gaussians in turn.
template <typename F>
__device__ __forceinline__ void for_tile_pairs(const uint2 *__restrict__ srect, const uint32_t *__restrict__ offsets,
                                               const uint32_t *__restrict__ tstart, uint32_t nv, int64_t P,
                                               int64_t ntiles, int shift, int bins_x, F f) {
    const int64_t P0 = (int64_t)blockIdx.x * kTileItems;
    const int64_t P1 = P0 + kTileItems < P ? P0 + kTileItems : P;
    const uint32_t r_lo = tstart[blockIdx.x];
    const uint32_t r_hi = (int64_t)blockIdx.x + 1 < ntiles ? tstart[blockIdx.x + 1] : nv - 1u;
    for (uint32_t r = r_lo + threadIdx.x; r <= r_hi; r += kThreads) {
        const uint2 rc = srect[r];
        const uint32_t x0 = (rc.x & 0xffffu) >> shift, x1 = (((rc.x >> 16) - 1u) >> shift) + 1u;
        const uint32_t y0 = (rc.y & 0xffffu) >> shift, y1 = (((rc.y >> 16) - 1u) >> shift) + 1u;
        const uint32_t wx = x1 - x0;
        const int64_t cnt = (int64_t)wx * (y1 - y0);
        const int64_t off = offsets[r];
        const int64_t e0 = P0 - off > 0 ? P0 - off : 0;
        const int64_t e1 = P1 - off < cnt ? P1 - off : cnt;
        if (e0 >= e1) continue;
        uint32_t by = y0 + (uint32_t)(e0 / wx), bx = x0 + (uint32_t)(e0 % wx);
        for (int64_t e = e0; e < e1; ++e) {
            f((int)(off + e - P0), by * (uint32_t)bins_x + bx, r);
            if (++bx == x1) {
                bx = x0;
                ++by;
            }
        }
    }
}

// Per tile: the count of each bin among its pairs, to hist[bin][tile] (the layout of rs_hist,
// ntiles_cap tiles; the tiles beyond the pairs held count nothing).
template <int BINS>
__global__ void __launch_bounds__(kThreads) bin_hist_k(const uint2 *__restrict__ srect,
                                                       const uint32_t *__restrict__ offsets,
                                                       const uint32_t *__restrict__ tstart, const BinCounts c,
                                                       int ntiles_cap, int shift, int bins_x,
                                                       uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[BINS];
    for (int d = threadIdx.x; d < BINS; d += kThreads) h[d] = 0;
    const int64_t P = pairs_held(c);
    const int64_t ntiles = (P + kTileItems - 1) / kTileItems;
    __syncthreads();
    if ((int64_t)blockIdx.x < ntiles)
        for_tile_pairs(srect, offsets, tstart, *c.nv, P, ntiles, shift, bins_x,
                       [&](int, uint32_t bin, uint32_t) { atomicAdd(&h[bin], 1u); });
    __syncthreads();
    for (int d = threadIdx.x; d < BINS; d += kThreads) hist[(int64_t)d * ntiles_cap + blockIdx.x] = h[d];
}

// Per tile: its pairs, generated into the staging arrays in emission order, then scattered
// stably by bin (scatter_tile); values leave as vmap[rank], with the Gaussian's tile rectangle.
// Block 0 always runs: it writes every bin's range.
template <int BINS>
__global__ void __launch_bounds__(kThreads) bin_place_k(const uint2 *__restrict__ srect,
                                                        const uint32_t *__restrict__ offsets,
                                                        const uint32_t *__restrict__ tstart, const BinCounts c,
                                                        int ntiles_cap, int shift, int bins_x, uint32_t mask, int width,
                                                        const uint32_t *__restrict__ offs,
                                                        const uint32_t *__restrict__ digit_tot,
                                                        uint2 *__restrict__ ranges, int nranges,
                                                        const uint2 *__restrict__ rect_src, uint2 *__restrict__ rect_out,
                                                        const uint32_t *__restrict__ vmap,
                                                        uint32_t *__restrict__ vout) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t P = pairs_held(c);
    const int64_t ntiles = (P + kTileItems - 1) / kTileItems;
    if (blockIdx.x > 0 && (int64_t)blockIdx.x >= ntiles) return;   // (uniform per CTA)
    uint32_t *skeys = reinterpret_cast<uint32_t *>(smem_raw) + (kWarps + 2) * BINS + 16;
    uint32_t *svals = skeys + kTileItems;
    if ((int64_t)blockIdx.x < ntiles)
        for_tile_pairs(srect, offsets, tstart, *c.nv, P, ntiles, shift, bins_x, [&](int j, uint32_t bin, uint32_t r) {
            skeys[j] = bin;
            svals[j] = r;
        });
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tile_base = (int64_t)blockIdx.x * kTileItems;
    uint32_t key[kItems], val[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int j = w * (32 * kItems) + r * 32 + lane;
        const bool valid = tile_base + j < P;
        key[r] = valid ? skeys[j] : 0u;
        val[r] = valid ? svals[j] : 0u;
    }
    scatter_tile<uint32_t, kItems, BINS>(key, val, smem_raw, nullptr, vout, P, 0, mask, width, offs, digit_tot,
                                         ntiles_cap, ranges, nranges, rect_src, rect_out, vmap);
}

template <typename K, int ITEMS, int BINS>
size_t scatter_smem() {
    return (size_t)(kWarps + 2) * BINS * 4 + 64 + (size_t)kThreads * ITEMS * (sizeof(K) + 4);
}

template <typename K, int ITEMS, int BINS>
void radix_pass(const K *ki, const uint32_t *vi, K *ko, uint32_t *vo, int64_t n, int shift, int width, SortScratch &s,
                cudaStream_t st, uint2 *ranges, int nranges, const uint2 *gsrc, uint2 *gout, const uint32_t *vmap) {
    constexpr int kTileN = kThreads * ITEMS;
    const int ntiles = (int)((n + kTileN - 1) / kTileN);
    // on failure the error stays recorded for the caller's cudaGetLastError check
    if (set_max_smem((const void *)rs_scatter<K, ITEMS, BINS>, (int)scatter_smem<K, ITEMS, BINS>()) != cudaSuccess ||
        set_max_smem((const void *)rs_hist<K, ITEMS, BINS>, kWarps * BINS * 4) != cudaSuccess)
        return;
    const uint32_t mask = (width >= 32) ? 0xffffffffu : ((1u << width) - 1u);
    rs_hist<K, ITEMS, BINS><<<ntiles, kThreads, kWarps * BINS * 4, st>>>(ki, n, shift, mask, width, s.hist, ntiles); note_launch();
    rs_offsets<<<BINS, ntiles >= 1024 ? 1024 : (ntiles >= 256 ? 256 : 64), 0, st>>>(s.hist, s.digit_tot, ntiles); note_launch();
    rs_scatter<K, ITEMS, BINS><<<ntiles, kThreads, scatter_smem<K, ITEMS, BINS>(), st>>>(
        ki, vi, ko, vo, n, shift, mask, width, s.hist, s.digit_tot, ntiles, ranges, nranges, gsrc, gout, vmap);
    note_launch();
}

// Inputs below ~1M items use 1024-item tiles so that the grid still covers the GPU;
// a pass of w bits uses the smallest of 256, 512, 1024 and 2048 bins that holds its digits
// (fewer bins: smaller per-tile histograms to clear, write and scan).
template <typename K>
bool radix_sort_impl(K *keys, K *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n, const int *shifts,
                     const int *widths, int npass, SortScratch &s, cudaStream_t st, uint2 *ranges, int nranges,
                     const uint2 *gsrc = nullptr, uint2 *gout = nullptr, const uint32_t *vmap = nullptr) {
    if (n <= 0 || npass <= 0) return false;
    const bool small = n < kSmallSort;
    K *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int p = 0; p < npass; ++p) {
        uint2 *rg = (npass == 1) ? ranges : nullptr;
        const uint2 *gs = (p == npass - 1) ? gsrc : nullptr;   // the payload follows the last pass
        uint2 *go = (p == npass - 1) ? gout : nullptr;
        const uint32_t *vm = (p == npass - 1) ? vmap : nullptr;   // the map applies to the last pass's output
        if (widths[p] > 10) {
            if (small) radix_pass<K, 4, 2048>(ki, vi, ko, vo, n, shifts[p], widths[p], s, st, rg, nranges, gs, go, vm);
            else radix_pass<K, kItems, 2048>(ki, vi, ko, vo, n, shifts[p], widths[p], s, st, rg, nranges, gs, go, vm);
        } else if (widths[p] > 9) {
            if (small) radix_pass<K, 4, 1024>(ki, vi, ko, vo, n, shifts[p], widths[p], s, st, rg, nranges, gs, go, vm);
            else radix_pass<K, kItems, 1024>(ki, vi, ko, vo, n, shifts[p], widths[p], s, st, rg, nranges, gs, go, vm);
        } else if (widths[p] > 8) {
            if (small) radix_pass<K, 4, 512>(ki, vi, ko, vo, n, shifts[p], widths[p], s, st, rg, nranges, gs, go, vm);
            else radix_pass<K, kItems, 512>(ki, vi, ko, vo, n, shifts[p], widths[p], s, st, rg, nranges, gs, go, vm);
        } else {
            if (small) radix_pass<K, 4, 256>(ki, vi, ko, vo, n, shifts[p], widths[p], s, st, rg, nranges, gs, go, vm);
            else radix_pass<K, kItems, 256>(ki, vi, ko, vo, n, shifts[p], widths[p], s, st, rg, nranges, gs, go, vm);
        }
        K *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
    }
    return (npass & 1) != 0;
}

// ---------------------------------------------------------------------------
// exclusive scan
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *wsum, uint32_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t ws = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        uint32_t wx = ws;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wx, o);
            if (lane >= o) wx += y;
        }
        wsum[lane] = wx - ws;
        if (lane == 31) wsum[32] = wx;
    }
    __syncthreads();
    uint32_t r = wsum[w] + x - v;
    total = wsum[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads) scan_partials(const uint32_t *__restrict__ in, int64_t n,
                                                          uint32_t *__restrict__ partials) {
    const int64_t base = (int64_t)blockIdx.x * kTileItems;
    uint32_t s = 0;
    for (int j = threadIdx.x; j < kTileItems; j += kThreads) {
        int64_t i = base + j;
        if (i < n) s += in[i];
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ uint32_t ws[kWarps];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int q = 0; q < kWarps; ++q) t += ws[q];
        partials[blockIdx.x] = t;
    }
}

// Single CTA: in-place exclusive scan of the per-tile sums; total to *d_total.
__global__ void __launch_bounds__(1024) scan_spine(uint32_t *__restrict__ partials, int64_t np,
                                                   unsigned long long *__restrict__ d_total) {
    __shared__ uint32_t wsum[33];
    unsigned long long carry = 0;
    for (int64_t base = 0; base < np; base += 1024) {
        int64_t i = base + threadIdx.x;
        uint32_t v = i < np ? partials[i] : 0;
        uint32_t tot;
        uint32_t e = block_excl_scan(v, wsum, tot);
        if (i < np) partials[i] = (uint32_t)(carry + e);
        carry += tot;
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

// buffer index with one pad word per 32, so that thread t reading its 16
// consecutive items hits distinct banks
__device__ __forceinline__ int padded(int j) { return j + (j >> 5); }

__global__ void __launch_bounds__(kThreads) scan_tiles(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                       int64_t n, const uint32_t *__restrict__ partials) {
    __shared__ uint32_t buf[kTileItems + kTileItems / 32];
    __shared__ uint32_t wsum[33];
    const int64_t base = (int64_t)blockIdx.x * kTileItems;
    for (int j = threadIdx.x; j < kTileItems; j += kThreads) {
        int64_t i = base + j;
        buf[padded(j)] = i < n ? in[i] : 0;
    }
    __syncthreads();
    uint32_t v[kItems];
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        v[q] = buf[padded(threadIdx.x * kItems + q)];
        s += v[q];
    }
    uint32_t tot;
    uint32_t e = block_excl_scan(s, wsum, tot) + partials[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        buf[padded(threadIdx.x * kItems + q)] = e;
        e += v[q];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kTileItems; j += kThreads) {
        int64_t i = base + j;
        if (i < n) out[i] = buf[padded(j)];
    }
}

}  // namespace

cudaError_t scratch_reserve(SortScratch &s, int64_t n) {
    // 2048 bins x the largest tile count of a sort of at most n items: 1024-item tiles below
    // ~1M items (up to 1025 tiles), kTileItems-item tiles above, so the count is not monotonic
    // in the size and a reservation for n must cover every smaller sort too
    const int64_t small_max = n < kSmallSort ? (n + 1023) / 1024 + 1 : (kSmallSort - 1 + 1023) / 1024 + 1;
    const int64_t large = n < kSmallSort ? 0 : (n + kTileItems - 1) / kTileItems + 1;
    const int64_t tiles = small_max > large ? small_max : large;
    size_t need_hist = (size_t)2048 * tiles;
    if (!s.digit_tot) {
        cudaError_t e = cudaMalloc(&s.digit_tot, 2048 * sizeof(uint32_t));
        if (e != cudaSuccess) return e;
    }
    if (need_hist > s.hist_cap) {
        cudaFree(s.hist);
        s.hist = nullptr;
        s.hist_cap = 0;
        cudaError_t e = cudaMalloc(&s.hist, need_hist * sizeof(uint32_t));
        if (e != cudaSuccess) return e;
        s.hist_cap = need_hist;
    }
    const int64_t scan_tiles_n = (n + kTileItems - 1) / kTileItems + 1;
    if ((size_t)scan_tiles_n > s.partials_cap) {
        cudaFree(s.partials);
        s.partials = nullptr;
        s.partials_cap = 0;
        cudaError_t e = cudaMalloc(&s.partials, (size_t)scan_tiles_n * sizeof(uint32_t));
        if (e != cudaSuccess) return e;
        s.partials_cap = (size_t)scan_tiles_n;
    }
    if ((size_t)scan_tiles_n > s.tstart_cap) {   // the fused binning's tiles (kTileItems pairs each)
        cudaFree(s.tstart);
        s.tstart = nullptr;
        s.tstart_cap = 0;
        cudaError_t e = cudaMalloc(&s.tstart, (size_t)scan_tiles_n * sizeof(uint32_t));
        if (e != cudaSuccess) return e;
        s.tstart_cap = (size_t)scan_tiles_n;
    }
    return cudaSuccess;
}

void scratch_free(SortScratch &s) {
    cudaFree(s.hist);
    cudaFree(s.digit_tot);
    cudaFree(s.partials);
    cudaFree(s.tstart);
    s = SortScratch{};
}

int digit_passes(int lo, int bits, int *shifts, int *widths, int64_t n) {
    if (bits <= 0) return 0;
    // 2048-bin passes pay off only on large inputs; small ones use 8-bit digits
    const int maxw = n >= (1 << 21) ? 11 : 8;
    int np = (bits + maxw - 1) / maxw;
    int base = bits / np, extra = bits % np, at = lo;
    for (int p = 0; p < np; ++p) {
        int wdt = base + (p < extra ? 1 : 0);
        shifts[p] = at;
        widths[p] = wdt;
        at += wdt;
    }
    return np;
}

bool radix_sort_u32(uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                    const int *shifts, const int *widths, int npass, SortScratch &s, cudaStream_t st,
                    uint2 *ranges, int nranges, const uint2 *gather_src, uint2 *gather_out,
                    const uint32_t *val_map) {
    return radix_sort_impl<uint32_t>(keys, keys_alt, vals, vals_alt, n, shifts, widths, npass, s, st, ranges,
                                     nranges, gather_src, gather_out, val_map);
}

bool radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                    const int *shifts, const int *widths, int npass, SortScratch &s, cudaStream_t st) {
    return radix_sort_impl<uint64_t>(keys, keys_alt, vals, vals_alt, n, shifts, widths, npass, s, st, nullptr, 0);
}

namespace {

template <int BINS>
void bin_sort_fused_impl(const uint2 *srect, const uint32_t *offsets, const uint32_t *counts, int64_t n_cap,
                         const BinCounts &c, int shift, int bins_x, int bins, const uint32_t *val_map,
                         uint32_t *vals_out, uint2 *rect_out, uint2 *ranges, SortScratch &s, cudaStream_t st) {
    const int ntiles_cap = (int)((c.cap + kTileItems - 1) / kTileItems);
    const size_t smem = scatter_smem<uint32_t, kItems, BINS>();
    // on failure the error stays recorded for the caller's cudaGetLastError check
    if (set_max_smem((const void *)bin_place_k<BINS>, (int)smem) != cudaSuccess) return;
    int width = 0;
    while ((1 << width) < bins) ++width;
    if (width == 0) width = 1;
    const uint32_t mask = (1u << width) - 1u;
    tile_starts_k<<<(unsigned)((n_cap + 255) / 256), 256, 0, st>>>(offsets, counts, c, s.tstart);
    note_launch();
    bin_hist_k<BINS><<<ntiles_cap, kThreads, 0, st>>>(srect, offsets, s.tstart, c, ntiles_cap, shift, bins_x, s.hist);
    note_launch();
    rs_offsets<<<BINS, ntiles_cap >= 1024 ? 1024 : (ntiles_cap >= 256 ? 256 : 64), 0, st>>>(s.hist, s.digit_tot,
                                                                                          ntiles_cap);
    note_launch();
    bin_place_k<BINS><<<ntiles_cap, kThreads, smem, st>>>(srect, offsets, s.tstart, c, ntiles_cap, shift, bins_x, mask,
                                                          width, s.hist, s.digit_tot, ranges, bins, srect, rect_out,
                                                          val_map, vals_out);
    note_launch();
}

}  // namespace

bool bin_sort_fused(const uint2 *srect, const uint32_t *offsets, const uint32_t *counts, int64_t n_cap,
                    const uint32_t *d_nv, const unsigned long long *d_P, int64_t cap, int truncate,
                    uint32_t *d_overflow, int shift, int bins_x, int bins, const uint32_t *val_map,
                    uint32_t *vals_out, uint2 *rect_out, uint2 *ranges, SortScratch &s, cudaStream_t st) {
    if (cap <= 0 || n_cap <= 0 || bins < 1 || bins > 2048) return false;
    const BinCounts c{d_nv, d_P, cap, truncate, d_overflow};
    if (bins <= 256)
        bin_sort_fused_impl<256>(srect, offsets, counts, n_cap, c, shift, bins_x, bins, val_map, vals_out, rect_out,
                                 ranges, s, st);
    else if (bins <= 512)
        bin_sort_fused_impl<512>(srect, offsets, counts, n_cap, c, shift, bins_x, bins, val_map, vals_out, rect_out,
                                 ranges, s, st);
    else if (bins <= 1024)
        bin_sort_fused_impl<1024>(srect, offsets, counts, n_cap, c, shift, bins_x, bins, val_map, vals_out, rect_out,
                                  ranges, s, st);
    else
        bin_sort_fused_impl<2048>(srect, offsets, counts, n_cap, c, shift, bins_x, bins, val_map, vals_out, rect_out,
                                  ranges, s, st);
    return true;
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, unsigned long long *d_total,
                        SortScratch &s, cudaStream_t st) {
    if (n <= 0) {
        if (d_total) cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), st);
        return;
    }
    int64_t tiles = (n + kTileItems - 1) / kTileItems;
    scan_partials<<<(unsigned)tiles, kThreads, 0, st>>>(in, n, s.partials); note_launch();
    scan_spine<<<1, 1024, 0, st>>>(s.partials, tiles, d_total); note_launch();
    scan_tiles<<<(unsigned)tiles, kThreads, 0, st>>>(in, out, n, s.partials); note_launch();
}

SLAG_CHECKS_TAKE(checks_take_sort)

}  // namespace slag
