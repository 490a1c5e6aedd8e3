// Aggregation (Method, "Semantic Embedding", Aggregation step):
//   E_k = sum_views sum_j B_v[k][j] E_{v,j} / sum_views sum_j B_v[k][j].
//
// Per view, the consume pass turns each Gaussian's (segment, weight) table
// into sparse triples (Gaussian k, column c = view base + segment, W) in an
// append-only log -- only non-zero weights leave the view, as in the paper's
// hand-off from the rasterization phase to the aggregation phase -- and adds
// the weights to a compensated (Neumaier) float32 sum per Gaussian. Sums of
// a Gaussian whose table slots are all taken by other segments of the view
// wait in the view's spill list; the consume pass moves them to the log too
// (their weights join a plain per-Gaussian float32 sum).
//
// At finalize, the log is sorted by (Gaussian block of 128, column,
// Gaussian), so that each block of 128 spatially adjacent Gaussians (Morton
// order) sees its distinct columns in order; the distinct columns of each
// block are listed here. The contraction itself (W_block x E_cols on the
// tensor cores) is in k_aggregate_tc.cu.
#include "slag_internal.cuh"

namespace slag {

namespace {

__global__ void hash_init_k(HashEntry *h, int64_t n) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    HashEntry e;
#pragma unroll
    for (int s = 0; s < kHashSlots; ++s) {
        e.seg[s] = -1;
        e.w[s] = 0.f;
    }
    h[g] = e;
}

// Grid-stride over the view's records; many records per SM in flight hide the
// latency of the table probes.
__global__ void __launch_bounds__(256) combine_k(const WeightRecord *__restrict__ recs,
                                                 const unsigned long long *__restrict__ rec_chunks,
                                                 const uint32_t *__restrict__ rec_fill,
                                                 unsigned long long chunk_cap, const HashSink sink_in,
                                                 const uint32_t *__restrict__ skip,
                                                 const int32_t *__restrict__ view_base_dev) {
    if (skip && *skip) return;
    HashSink sink = sink_in;
    if (view_base_dev) sink.view_base = *view_base_dev;
    unsigned long long nc = *rec_chunks;
    if (nc > chunk_cap) nc = chunk_cap;
    const unsigned long long nr = nc * kRecChunk;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < nr;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        if ((uint32_t)(i % kRecChunk) >= rec_fill[i / kRecChunk]) continue;
        const WeightRecord r = recs[i];
        sink_add(sink, r.g, r.seg, r.w);
    }
}

// The view's spill list to the log: grid-stride over chunks of 256 entries, one reservation in
// the log per chunk. Nothing when the list overflowed (the view is composited again).
__global__ void __launch_bounds__(256) spill_commit_k(const ConsumeArgs a) {
    if (a.skip && *a.skip) return;
    const unsigned long long ns = *a.spill_count;
    if (ns == 0 || ns > a.spill_cap) return;
    __shared__ unsigned long long base_s;
    for (unsigned long long c0 = (unsigned long long)blockIdx.x * 256; c0 < ns;
         c0 += (unsigned long long)gridDim.x * 256) {
        const unsigned long long cnt = ns - c0 < 256 ? ns - c0 : 256;
        if (threadIdx.x == 0) base_s = atomicAdd(a.log_count, cnt);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const unsigned long long at = base_s + threadIdx.x;
            const uint64_t key = a.spill_key[c0 + threadIdx.x];
            const float w = a.spill_w[c0 + threadIdx.x];
            if (at < a.log_cap) {
                a.log_key[at] = key;
                a.log_w[at] = w;
                atomicAdd(&a.s_ovf[key_gaussian(key)], w);
            } else {
                atomicOr(a.overflow, 1u);
            }
        }
        __syncthreads();   // base_s is rewritten by the next chunk
    }
}

__global__ void __launch_bounds__(256) consume_k(const ConsumeArgs a) {
    if (a.skip && *a.skip) return;   // (uniform: before any barrier)
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = a.n;
    if (*a.spill_count > a.spill_cap) {
        // the view is composited again: its tables are cleared, nothing is counted
        if (g < n) {
            HashEntry clear;
#pragma unroll
            for (int s = 0; s < kHashSlots; ++s) {
                clear.seg[s] = -1;
                clear.w[s] = 0.f;
            }
            a.hash[g] = clear;
        }
        return;
    }
    const int32_t view_base = a.view_base_dev ? *a.view_base_dev : a.view_base;
    // the view's composited pairs join the running total (the view's composite has finished)
    if (g == 0 && a.view_contrib) atomicAdd(a.total_contrib, *a.view_contrib);
    const int lane = threadIdx.x & 31;
    HashEntry e;
    int cnt = 0;
    if (g < n) {
        e = a.hash[g];
#pragma unroll
        for (int s = 0; s < kHashSlots; ++s) cnt += e.seg[s] >= 0 ? 1 : 0;
    }
    // block-aggregated reservation in the log (one atomic per block on the shared counter)
    __shared__ int wtot_s[8];
    __shared__ unsigned long long base_s;
    const int w = threadIdx.x >> 5;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wtot_s[w] = incl;
    __syncthreads();
    int before = 0, btot = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        before += q < w ? wtot_s[q] : 0;
        btot += wtot_s[q];
    }
    if (threadIdx.x == 0) base_s = btot ? atomicAdd(a.log_count, (unsigned long long)btot) : 0ull;
    __syncthreads();
    if (g >= n || cnt == 0) return;
    unsigned long long at = base_s + (unsigned long long)(before + incl - cnt);
    float sh = a.s_hi[g], sl = a.s_lo[g];
    bool overflow = false;
    HashEntry clear;
#pragma unroll
    for (int s = 0; s < kHashSlots; ++s) {
        clear.seg[s] = -1;
        clear.w[s] = 0.f;
        if (e.seg[s] < 0) continue;
        if (at < a.log_cap) {
            a.log_key[at] = pack_key((uint32_t)g, (uint32_t)(view_base + e.seg[s]));
            a.log_w[at] = e.w[s];
            const float w = e.w[s];
            const float t = sh + w;
            sl += fabsf(sh) >= fabsf(w) ? (sh - t) + w : (w - t) + sh;
            sh = t;
        } else {
            overflow = true;
        }
        ++at;
    }
    a.s_hi[g] = sh;
    a.s_lo[g] = sl;
    a.hash[g] = clear;
    if (overflow) atomicOr(a.overflow, 1u);
}

__global__ void unique_flags_k(const uint64_t *__restrict__ keys, int64_t Z, uint32_t *__restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Z) return;
    flags[i] = (i == 0 || (keys[i] >> 7) != (keys[i - 1] >> 7)) ? 1u : 0u;
}

// keys in the compact layout of repack_keys_k (block above cb column bits)
__global__ void uniques_k(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ flags,
                          const uint32_t *__restrict__ uidx, int64_t Z, int cb, uint32_t *__restrict__ ucol,
                          uint32_t *__restrict__ ustart, uint32_t *__restrict__ bstart,
                          uint32_t *__restrict__ bend) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Z) return;
    const uint64_t k = keys[i];
    if (flags[i]) {
        const uint32_t u = uidx[i];
        ucol[u] = (uint32_t)((k >> 7) & ((1ull << cb) - 1ull));
        ustart[u] = (uint32_t)i;
    }
    const int sb = 7 + cb;
    const uint32_t blk = (uint32_t)(k >> sb);
    if (i == 0 || (uint32_t)(keys[i - 1] >> sb) != blk) bstart[blk] = (uint32_t)i;
    if (i == Z - 1 || (uint32_t)(keys[i + 1] >> sb) != blk) bend[blk] = (uint32_t)(i + 1);
}

// The log key of pack_key, (block << 39) | (column << 7) | (Gaussian & 127), to the compact
// layout (block << (7 + cb)) | (column << 7) | (Gaussian & 127) for columns < 2^cb (forward), and
// back. The compact layout puts the sorted fields (block, column) in 7 + cb + block bits
// without a gap, so the radix sort needs fewer passes.
// keys_out[i] = the repacked keys_in[i] (in place when they alias); with w_in, w_out[i] = w_in[i].
__global__ void repack_keys_k(const uint64_t *keys_in, uint64_t *keys_out, const float *w_in, float *w_out,
                              int64_t Z, int cb, int forward) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Z) return;
    const uint64_t k = keys_in[i];
    const uint64_t cmask = (1ull << cb) - 1ull;
    if (forward)
        keys_out[i] = ((k >> 39) << (7 + cb)) | (((k >> 7) & cmask) << 7) | (k & 127ull);
    else
        keys_out[i] = ((k >> (7 + cb)) << 39) | (((k >> 7) & cmask) << 7) | (k & 127ull);
    if (w_in) w_out[i] = w_in[i];
}

// Saved state: each log entry as (caller index, column).
__global__ void state_unpack_k(const uint64_t *__restrict__ keys, int64_t Z, const uint32_t *__restrict__ orig_of_int,
                               uint32_t *__restrict__ gauss, uint32_t *__restrict__ col) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Z) return;
    const uint64_t k = keys[i];
    const uint32_t g = (uint32_t)(((k >> 39) << 7) | (k & 127ull));
    gauss[i] = orig_of_int[g];
    col[i] = (uint32_t)((k >> 7) & 0xffffffffull);
}

// Merged state: entries (caller index, column, W) appended to the log, the columns shifted past
// the context's own; an index or column out of range is not written and sets *bad.
__global__ void state_pack_k(const uint32_t *__restrict__ gauss, const uint32_t *__restrict__ col,
                             const float *__restrict__ w, int64_t Z, const uint32_t *__restrict__ int_of_orig,
                             int64_t n, uint32_t col_shift, uint32_t cols_in, uint64_t *__restrict__ log_key,
                             float *__restrict__ log_w, uint32_t *bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Z) return;
    const uint32_t c = gauss[i], j = col[i];
    if (c >= (uint64_t)n || j >= cols_in) {
        atomicOr(bad, 1u);
        log_key[i] = pack_key(0u, col_shift);   // a harmless entry: weight 0 on a valid column
        log_w[i] = 0.f;
        return;
    }
    log_key[i] = pack_key(int_of_orig[c], col_shift + j);
    log_w[i] = w[i];
}

// Merged state: the compensated sums (hi, lo) and the overflow sums of another state added,
// per Gaussian (internal order).
__global__ void state_sums_k(float *__restrict__ hi, float *__restrict__ lo, float *__restrict__ ovf,
                             const float *__restrict__ bhi, const float *__restrict__ blo,
                             const float *__restrict__ bovf, int64_t n) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float a = hi[g], b = bhi[g];
    const float t = a + b;
    const float err = fabsf(a) >= fabsf(b) ? (a - t) + b : (b - t) + a;
    hi[g] = t;
    lo[g] = (lo[g] + blo[g]) + err;
    ovf[g] = ovf[g] + bovf[g];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_state_unpack(const uint64_t *keys, int64_t Z, const uint32_t *orig_of_int, uint32_t *gauss, uint32_t *col,
                         cudaStream_t st) {
    if (Z <= 0) return;
    state_unpack_k<<<blocks_for(Z, 256), 256, 0, st>>>(keys, Z, orig_of_int, gauss, col); note_launch();
}

void launch_state_pack(const uint32_t *gauss, const uint32_t *col, const float *w, int64_t Z,
                       const uint32_t *int_of_orig, int64_t n, uint32_t col_shift, uint32_t cols_in,
                       uint64_t *log_key, float *log_w, uint32_t *bad, cudaStream_t st) {
    if (Z <= 0) return;
    state_pack_k<<<blocks_for(Z, 256), 256, 0, st>>>(gauss, col, w, Z, int_of_orig, n, col_shift, cols_in, log_key,
                                                     log_w, bad); note_launch();
}

void launch_state_sums(float *hi, float *lo, float *ovf, const float *bhi, const float *blo, const float *bovf,
                       int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    state_sums_k<<<blocks_for(n, 256), 256, 0, st>>>(hi, lo, ovf, bhi, blo, bovf, n); note_launch();
}

void launch_hash_init(HashEntry *hash, int64_t n, cudaStream_t st) {
    hash_init_k<<<blocks_for(n, 256), 256, 0, st>>>(hash, n); note_launch();
}

namespace {

// dst[i] = src[i] for n 32-bit words; dst may be mapped (zero-copy) host memory.
__global__ void __launch_bounds__(256) copy_words_k(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                                    int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

}  // namespace

void launch_copy_words(const void *src, void *dst, int64_t bytes, cudaStream_t st) {
    const int64_t n = bytes / 4;
    if (n <= 0) return;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 64);
    copy_words_k<<<(unsigned)blocks, 256, 0, st>>>(static_cast<const uint32_t *>(src), static_cast<uint32_t *>(dst),
                                                   n); note_launch();
}

void launch_combine(const WeightRecord *recs, const unsigned long long *rec_chunks, const uint32_t *rec_fill,
                    unsigned long long chunk_cap, const HashSink &sink, const uint32_t *skip, cudaStream_t st,
                    const int32_t *view_base_dev) {
    if (chunk_cap == 0) return;
    const unsigned long long rec_cap = chunk_cap * kRecChunk;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned blocks = (unsigned)sms * 8u;
    const unsigned long long need = (rec_cap + 255) / 256;
    if (need < blocks) blocks = (unsigned)need;
    combine_k<<<blocks, 256, 0, st>>>(recs, rec_chunks, rec_fill, chunk_cap, sink, skip, view_base_dev);
    note_launch();
}

void launch_consume(const ConsumeArgs &a, cudaStream_t st) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    spill_commit_k<<<(unsigned)sms * 2u, 256, 0, st>>>(a);
    note_launch();
    consume_k<<<blocks_for(a.n, 256), 256, 0, st>>>(a);
    note_launch();
}

void launch_unique_flags(const uint64_t *keys, int64_t Z, uint32_t *flags, cudaStream_t st) {
    if (Z <= 0) return;
    unique_flags_k<<<blocks_for(Z, 256), 256, 0, st>>>(keys, Z, flags); note_launch();
}

void launch_uniques(const uint64_t *keys, const uint32_t *flags, const uint32_t *uidx, int64_t Z, int col_bits,
                    uint32_t *ucol, uint32_t *ustart, uint32_t *bstart, uint32_t *bend, cudaStream_t st) {
    if (Z <= 0) return;
    uniques_k<<<blocks_for(Z, 256), 256, 0, st>>>(keys, flags, uidx, Z, col_bits, ucol, ustart, bstart, bend);
    note_launch();
}

void launch_repack_keys(const uint64_t *keys_in, uint64_t *keys_out, const float *w_in, float *w_out, int64_t Z,
                        int col_bits, bool to_compact, cudaStream_t st) {
    if (Z <= 0) return;
    repack_keys_k<<<blocks_for(Z, 256), 256, 0, st>>>(keys_in, keys_out, w_in, w_out, Z, col_bits,
                                                      to_compact ? 1 : 0);
    note_launch();
}

}  // namespace slag
