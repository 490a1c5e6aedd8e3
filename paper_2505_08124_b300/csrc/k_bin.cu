// Tile binning: emit one (tile, depth rank) pair per Gaussian-tile overlap,
// and find each tile's range in the tile-sorted pairs.
//
// Pairs are emitted in depth-rank order (rank = position in the stable sort
// by (float32 depth, caller index)), each Gaussian's tiles in row-major order.
// A stable sort of the pairs by tile id alone then yields, per tile, the
// Gaussians in ascending (depth, index): the order a sort by the 64-bit key
// (tile << 32 | depth bits) with ties by index would give, with a key of only
// ceil(log2(tiles)) bits.
#include "slag_internal.cuh"

namespace slag {

namespace {

// One warp per Gaussian: the lanes write consecutive pairs of its rectangle.
__global__ void __launch_bounds__(256) emit_k(const uint2 *__restrict__ srect, const uint32_t *__restrict__ offsets,
                                              uint32_t n_visible, int tiles_x, uint32_t *__restrict__ keys,
                                              uint32_t *__restrict__ vals) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t r = warp; r < n_visible; r += nwarps) {
        uint2 rc = srect[r];
        uint32_t x0 = rc.x & 0xffffu, x1 = rc.x >> 16, y0 = rc.y & 0xffffu, y1 = rc.y >> 16;
        uint32_t wdt = x1 - x0, cnt = wdt * (y1 - y0);
        uint32_t off = offsets[r];
        for (uint32_t i = lane; i < cnt; i += 32) {
            uint32_t y = y0 + i / wdt, x = x0 + i % wdt;
            keys[off + i] = y * (uint32_t)tiles_x + x;
            vals[off + i] = r;
        }
    }
}

__global__ void ranges_k(const uint32_t *__restrict__ keys, int64_t P, uint2 *__restrict__ ranges) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == P - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
}

}  // namespace

void launch_emit(const uint2 *srect, const uint32_t *offsets, uint32_t n_visible, int tiles_x, uint32_t *keys,
                 uint32_t *vals, cudaStream_t st) {
    if (n_visible == 0) return;
    int64_t blocks = ((int64_t)n_visible * 32 + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    emit_k<<<(unsigned)blocks, 256, 0, st>>>(srect, offsets, n_visible, tiles_x, keys, vals);
}

void launch_ranges(const uint32_t *keys, int64_t P, uint2 *ranges, cudaStream_t st) {
    if (P <= 0) return;
    ranges_k<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(keys, P, ranges);
}

}  // namespace slag
