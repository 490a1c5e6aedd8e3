// Tile binning: emit one (bin, depth rank) pair per Gaussian-bin overlap, and
// find each bin's range in the bin-sorted pairs. A bin is a 16x16 tile (the
// flat lists of the integer-stage diagnostics) or a 4x4-tile super-tile (the
// lists the compositing kernel filters per tile, see k_composite.cu).
//
// Pairs are emitted in depth-rank order (rank = position in the stable sort
// by (float32 depth, caller index)), each Gaussian's tiles in row-major order.
// A stable sort of the pairs by tile id alone then yields, per tile, the
// Gaussians in ascending (depth, index): the order a sort by the 64-bit key
// (tile << 32 | depth bits) with ties by index would give, with a key of only
// ceil(log2(tiles)) bits.
#include "slag_internal.cuh"

namespace slag {

SLAG_CHECKS_WORD

namespace {

// One thread per Gaussian (in depth-rank order): the pairs of the bins its tile rectangle meets,
// row-major; a bin is a 2^shift x 2^shift square of tiles. A warp's 32 Gaussians own one
// contiguous run of the output (their offsets are an exclusive scan of their pair counts): the
// warp writes its pairs into shared memory in windows of kEmitStage and copies each window out
// with coalesced stores.
constexpr int kEmitThreads = 256;
constexpr int kEmitStage = 256;

__global__ void __launch_bounds__(kEmitThreads) emit_k(const uint2 *__restrict__ srect,
                                                       const uint32_t *__restrict__ offsets, uint32_t n_visible,
                                                       int shift, int bins_x, int64_t cap,
                                                       uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    __shared__ uint32_t sk[kEmitThreads / 32][kEmitStage], sv[kEmitThreads / 32][kEmitStage];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t r0 = blockIdx.x * kEmitThreads + w * 32;   // the warp's first Gaussian
    if (r0 >= n_visible) return;                               // (warp-uniform)
    const uint32_t r = r0 + lane;
    const bool valid = r < n_visible;
    uint32_t x0 = 0, wx = 1, y0 = 0, cnt = 0, off = 0;
    if (valid) {
        const uint2 rc = srect[r];
        x0 = (rc.x & 0xffffu) >> shift;
        const uint32_t x1 = (((rc.x >> 16) - 1) >> shift) + 1;
        y0 = (rc.y & 0xffffu) >> shift;
        const uint32_t y1 = (((rc.y >> 16) - 1) >> shift) + 1;
        wx = x1 - x0;
        cnt = wx * (y1 - y0);
        off = offsets[r];
    }
    const uint32_t base = __shfl_sync(0xffffffffu, off, 0);
    const uint32_t p = off - base;                             // this lane's first place in the run
    uint32_t total = valid ? p + cnt : 0u;
    for (int o = 16; o; o >>= 1) total = max(total, __shfl_xor_sync(0xffffffffu, total, o));
    // this lane's next pair: index e of its rectangle, at bin (bx, by)
    uint32_t e = 0, bx = x0, by = y0;
    for (uint32_t s = 0; s < total; s += kEmitStage) {
        const uint32_t lim = s + kEmitStage;
        while (e < cnt && p + e < lim) {
            const uint32_t at = p + e - s;
            sk[w][at] = by * (uint32_t)bins_x + bx;
            sv[w][at] = r;
            ++e;
            if (++bx == x0 + wx) {
                bx = x0;
                ++by;
            }
        }
        __syncwarp();
        const uint32_t m = min((uint32_t)kEmitStage, total - s);
        for (uint32_t j = lane; j < m; j += 32) {
            const int64_t g = (int64_t)base + s + j;
            if (!SLAG_IN_BOUNDS(g < cap, kCheckEmit)) continue;
            keys[g] = sk[w][j];
            vals[g] = sv[w][j];
        }
        __syncwarp();
    }
}

__global__ void ranges_k(const uint32_t *__restrict__ keys, int64_t P, uint2 *__restrict__ ranges) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == P - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
}

// One CTA: order = tiles grouped by descending floor(log2(pair count + 1)), so
// that compositing starts the longest lists first (order within a group is
// the order in which the threads claim places).
__device__ __forceinline__ uint2 bin_range(const uint2 *ranges, int t, int tiles_x, int shift) {
    const int tx = t % tiles_x, ty = t / tiles_x;
    const int bins_x = ((tiles_x - 1) >> shift) + 1;
    return ranges[(ty >> shift) * bins_x + (tx >> shift)];
}

__global__ void __launch_bounds__(1024) tile_order_k(const uint2 *__restrict__ ranges, int tiles_x, int tiles,
                                                     int shift, uint32_t *__restrict__ order) {
    __shared__ uint32_t cnt[33], start[33];
    if (threadIdx.x < 33) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
        const uint2 r = bin_range(ranges, t, tiles_x, shift);
        const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
        atomicAdd(&cnt[32 - __clz(len + 1u)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int b = 32; b >= 0; --b) {
            start[b] = acc;
            acc += cnt[b];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
        const uint2 r = bin_range(ranges, t, tiles_x, shift);
        const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
        order[atomicAdd(&start[32 - __clz(len + 1u)], 1u)] = (uint32_t)t;
    }
}

}  // namespace

void launch_tile_order(const uint2 *ranges, int tiles_x, int tiles_y, int shift, uint32_t *order,
                       cudaStream_t st) {
    const int tiles = tiles_x * tiles_y;
    if (tiles <= 0) return;
    tile_order_k<<<1, 1024, 0, st>>>(ranges, tiles_x, tiles, shift, order); note_launch();
}

void launch_emit(const uint2 *srect, const uint32_t *offsets, uint32_t n_visible, int shift, int bins_x, int64_t cap,
                 uint32_t *keys, uint32_t *vals, cudaStream_t st) {
    if (n_visible == 0) return;
    emit_k<<<(n_visible + kEmitThreads - 1) / kEmitThreads, kEmitThreads, 0, st>>>(srect, offsets, n_visible, shift,
                                                                               bins_x, cap, keys, vals);
    note_launch();
}

SLAG_CHECKS_TAKE(checks_take_bin)

void launch_ranges(const uint32_t *keys, int64_t P, uint2 *ranges, cudaStream_t st) {
    if (P <= 0) return;
    ranges_k<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(keys, P, ranges); note_launch();
}

}  // namespace slag
