// Internal declarations shared by the CUDA translation units of libslag.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/slag.h"

namespace slag {

// Counts the kernel launches of the library (process-wide, every device).
void note_launch();

// Raises the dynamic shared-memory limit of kernel `fn` to `bytes` on the current device, once
// per (device, kernel): the attribute belongs to the calling thread's current device, so a
// context on another device needs its own call. Thread-safe; returns the CUDA status of the
// attribute call (cudaSuccess when it was already set on this device).
cudaError_t set_max_smem(const void *fn, int bytes);

// ---- the checked build (-DSLAG_CHECKS, libslag_checks.so) ------------------------------------
// Index checks compiled into pair emission, the sort's scatter, compositing and aggregation: an
// index outside its buffer is not used, and the stage's bit is set in a device word of the
// translation unit; the host reads and clears the words at its synchronisation points and
// returns SLAG_ERR_CAPACITY. In other builds SLAG_IN_BOUNDS is `true` and costs nothing.
enum : uint32_t { kCheckEmit = 1u, kCheckSort = 2u, kCheckComposite = 4u, kCheckAggregate = 8u };
#ifdef SLAG_CHECKS
__device__ __forceinline__ bool check_index(bool ok, uint32_t *word, uint32_t bit) {
    if (!ok) atomicOr(word, bit);
    return ok;
}
#define SLAG_CHECKS_WORD static __device__ uint32_t g_check_word;
#define SLAG_IN_BOUNDS(cond, bit) ::slag::check_index((cond), &g_check_word, (bit))
#define SLAG_CHECKS_TAKE(fn)                                                                         \
    uint32_t fn(cudaStream_t st) {                                                                   \
        uint32_t v = 0, z = 0;                                                                       \
        if (cudaMemcpyFromSymbolAsync(&v, g_check_word, sizeof(v), 0, cudaMemcpyDeviceToHost, st) != \
            cudaSuccess)                                                                             \
            return 0;                                                                                \
        cudaStreamSynchronize(st);                                                                   \
        if (v) {                                                                                     \
            cudaMemcpyToSymbolAsync(g_check_word, &z, sizeof(z), 0, cudaMemcpyHostToDevice, st);     \
            cudaStreamSynchronize(st);                                                               \
        }                                                                                            \
        return v;                                                                                    \
    }
constexpr bool kChecked = true;
#else
#define SLAG_CHECKS_WORD
#define SLAG_IN_BOUNDS(cond, bit) true
#define SLAG_CHECKS_TAKE(fn) \
    uint32_t fn(cudaStream_t) { return 0; }
constexpr bool kChecked = false;
#endif
// Reads and clears the check word of each translation unit (0 in unchecked builds).
uint32_t checks_take_bin(cudaStream_t st);
uint32_t checks_take_sort(cudaStream_t st);
uint32_t checks_take_composite(cudaStream_t st);
uint32_t checks_take_aggregate(cudaStream_t st);

constexpr int kTile = 16;          // screen tile edge in pixels
constexpr float kLog2AlphaMin = -7.99435343685886f;   // log2 of the alpha floor 1/255
constexpr int kBlockG = 128;       // Gaussians per aggregation block (key packs g & 127)
constexpr int kHashSlots = 4;      // per-view (segment, weight) slots per Gaussian
constexpr int kSuperShift = 2;     // compositing lists are binned per 4x4-tile super-tile
constexpr int kMaxK = 1024;        // largest top-k
constexpr uint32_t kCulled = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// device-side records
// ---------------------------------------------------------------------------

// Per-view (segment, weight) table of one Gaussian. seg = -1 marks a free slot.
struct __align__(16) HashEntry {
    int32_t seg[kHashSlots];
    float w[kHashSlots];
};

// Per-view counters written by kernels and read back once per view.
struct ViewCounters {
    uint32_t n_visible;
    uint32_t bad_seg;                 // non-zero: a segment id outside [-1, M)
    unsigned long long P;             // pairs at the binning granularity (tiles or super-tiles)
    unsigned long long P_tiles;       // Gaussian-tile pairs
    unsigned long long contributions; // composited (Gaussian, pixel) pairs (diagnostic render)
    unsigned long long spills;        // (Gaussian, segment) sums that found no free slot in the
                                      // view's table: the spill list's appends, also beyond its
                                      // capacity
    uint32_t overflow;                // the view's pairs exceeded the capacity its binning held
    uint32_t pad;
};

struct CamParams {
    float fx, fy, cx, cy;
    int32_t width, height;
    float R[9];
    float t[3];
    float near_z, far_z;
    int32_t tiles_x, tiles_y;
};

// ---------------------------------------------------------------------------
// primitives (k_sort.cu)
// ---------------------------------------------------------------------------

// Scratch for radix sorts and scans; grows on demand.
struct SortScratch {
    uint32_t *hist = nullptr;      // 256 x tiles
    size_t hist_cap = 0;
    uint32_t *digit_tot = nullptr; // 256
    uint32_t *partials = nullptr;  // scan partials
    size_t partials_cap = 0;
    uint32_t *tstart = nullptr;    // fused binning: the first Gaussian of each tile
    size_t tstart_cap = 0;
};

cudaError_t scratch_reserve(SortScratch &s, int64_t n);
void scratch_free(SortScratch &s);

// Stable LSD radix sort of (key, value) pairs over the bit ranges listed in
// shifts/widths (each width <= 11, applied in order). Ping-pongs between the
// two buffers; returns true when the result is in the *_alt buffers. For a
// single pass whose digit is the whole key, `ranges` (nullable) receives each
// key value's [start, end) in the output for key values < nranges. With
// gather_out (n entries), gather_out[i] = gather_src[sorted value i] as well.
// With val_map, the last pass writes val_map[v] in place of each value v (the
// payload gather still reads gather_src[v]).
bool radix_sort_u32(uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt,
                    int64_t n, const int *shifts, const int *widths, int npass, SortScratch &s,
                    cudaStream_t st, uint2 *ranges = nullptr, int nranges = 0, const uint2 *gather_src = nullptr,
                    uint2 *gather_out = nullptr, const uint32_t *val_map = nullptr);
bool radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt,
                    int64_t n, const int *shifts, const int *widths, int npass, SortScratch &s,
                    cudaStream_t st);

// Binning of a view's Gaussian-bin pairs by bin in one stable pass, without writing the pairs in
// emission order first: the Gaussians of depth rank r < *d_nv (at most n_cap), with bin
// rectangles from srect at 2^shift tiles per bin (bins_x bins per row, `bins` in all), counts[r]
// pairs each and offsets = the exclusive scan of counts; *d_P pairs in all. The counts are read
// on the device, so the host need not know them: the pass holds at most cap pairs, and a larger
// *d_P sets *d_overflow and leaves every bin empty (with truncate, set only by checked builds'
// forced capacities, the first cap pairs are kept and the pair emission's check flags the rest).
// Writes, in bin order and within a bin in emission order, vals_out[i] = val_map[r] and
// rect_out[i] = srect[r] (when rect_out is non-null) of each pair's Gaussian r, and ranges[b] =
// [start, end) of bin b. Returns false (and does nothing) when bins > 2048 or cap is 0; the
// caller then emits the pairs and radix-sorts them.
bool bin_sort_fused(const uint2 *srect, const uint32_t *offsets, const uint32_t *counts, int64_t n_cap,
                    const uint32_t *d_nv, const unsigned long long *d_P, int64_t cap, int truncate,
                    uint32_t *d_overflow, int shift, int bins_x, int bins, const uint32_t *val_map,
                    uint32_t *vals_out, uint2 *rect_out, uint2 *ranges, SortScratch &s, cudaStream_t st);

// Exclusive prefix sum of n uint32 values; writes the total to *d_total (may be null).
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, unsigned long long *d_total,
                        SortScratch &s, cudaStream_t st);

// Splits [lo, lo + bits) into passes for a sort of n items (at most 11 bits
// per pass from 2M items up, 8 below); returns the pass count.
int digit_passes(int lo, int bits, int *shifts, int *widths, int64_t n);

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

// k_project.cu
void launch_check_gaussians(const float *means, const float *scales, const float *quats,
                            const float *opac, int64_t n, uint32_t *d_flag, cudaStream_t st);
void launch_bbox(const float *means, int64_t n, uint32_t *d_bbox6, cudaStream_t st);
void launch_morton(const float *means, int64_t n, const uint32_t *d_bbox6, uint32_t *codes,
                   uint32_t *idx, cudaStream_t st);
void launch_pack_gaussians(const float *means, const float *scales, const float *quats,
                           const float *opac, int64_t n, const uint32_t *orig_of_int,
                           float4 *mean_op, float4 *cov_a, float2 *cov_b, uint32_t *int_of_orig,
                           float *log2_op, cudaStream_t st);
void launch_project(const CamParams &cam, const float4 *mean_op, const float *log2_op, const float4 *cov_a,
                    const float2 *cov_b, int64_t n, const uint32_t *orig_of_int, uint32_t *dkey_orig,
                    uint32_t *dval_orig, float4 *rec_a, float4 *rec_b, float *rec_t, uint2 *rect,
                    ViewCounters *ctr, cudaStream_t st, const CamParams *cam_dev = nullptr);
// Rectangles and bin counts in depth-rank order. With shift s > 0 the count is of
// 2^s x 2^s-tile super-tiles; the tile-pair total goes to ctr->P_tiles.
void launch_gather_sorted(const uint32_t *sorted_vals, int64_t n, ViewCounters *ctr, const uint2 *rect,
                          uint2 *srect, uint32_t *stouched, int shift, cudaStream_t st);
void launch_check_seg(const int32_t *seg, int64_t npx, int32_t M, ViewCounters *ctr, cudaStream_t st);

// k_bin.cu
// One (bin, depth rank) pair per Gaussian-bin overlap; bins are 2^shift-tile squares,
// bins_x of them per row.
void launch_emit(const uint2 *srect, const uint32_t *offsets, uint32_t n_visible, int shift, int bins_x, int64_t cap,
                 uint32_t *keys, uint32_t *vals, cudaStream_t st);
void launch_ranges(const uint32_t *keys, int64_t P, uint2 *ranges, cudaStream_t st);
// Tiles grouped by descending floor(log2(list length + 1)) of their bin.
void launch_tile_order(const uint2 *ranges, int tiles_x, int tiles_y, int shift, uint32_t *order,
                       cudaStream_t st);

// Where a view's per-Gaussian (segment, weight) sums go: the Gaussian's
// kHashSlots-entry table, or, once its slots hold other segments, a triple
// (Gaussian, column, weight) appended to the log, whose weight also goes to
// the Gaussian's overflow sum.
// Where a view's (Gaussian, segment) sums go: the view's table of kHashSlots slots per Gaussian,
// and, for a Gaussian whose slots are all taken by other segments, the view's spill list (log
// keys and weights, moved to the triple log by the view's consume pass). The spill count keeps
// counting beyond the list's capacity, so that the host learns how much room the view needed.
struct HashSink {
    HashEntry *hash;               // n entries (internal order)
    unsigned long long *spill_count;
    unsigned long long spill_cap;
    uint64_t *spill_key;
    float *spill_w;
    int32_t view_base;             // column of segment 0 of this view
};

// Log key of (internal Gaussian g, column col): block of 128 Gaussians, column, offset in the block.
__device__ __forceinline__ uint64_t pack_key(uint32_t g, uint32_t col) {
    return ((uint64_t)(g >> 7) << 39) | ((uint64_t)col << 7) | (uint64_t)(g & 127u);
}

__device__ __forceinline__ uint32_t key_gaussian(uint64_t key) {
    return ((uint32_t)(key >> 39) << 7) | (uint32_t)(key & 127u);
}

__device__ __forceinline__ void sink_append(const HashSink &k, uint32_t g, int32_t seg, float w) {
    const unsigned long long idx = atomicAdd(k.spill_count, 1ull);
    if (idx < k.spill_cap) {
        k.spill_key[idx] = pack_key(g, (uint32_t)(k.view_base + seg));
        k.spill_w[idx] = w;
    }
}

// Adds w to the (segment, weight) slot of Gaussian g, claiming a free slot if needed.
__device__ __forceinline__ void sink_add(const HashSink &k, uint32_t g, int32_t seg, float w) {
    HashEntry *h = k.hash + g;
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
    sink_append(k, g, seg, w);
}

// One per-(Gaussian, sub-tile, segment) sum of a view, on its way from the
// compositing kernel to the combine pass. The record list is reserved in chunks
// of kRecChunk records: a CTA reserves its next chunk one chunk ahead (so that no
// store waits for the reservation) and writes each chunk's fill (its first
// fill records are valid) once it is done with it; every reserved chunk gets a
// fill, zero when it was never used.
constexpr int kRecChunk = 256;
struct __align__(16) WeightRecord {
    uint32_t g;                    // internal Gaussian index
    int32_t seg;
    float w;
    uint32_t pad;
};

// k_composite.cu
struct CompositeArgs {
    CamParams cam;
    const uint2 *ranges;           // per bin (tile, or super-tile when bin_shift > 0)
    int32_t bin_shift, bins_x;
    const uint32_t *tile_order;    // CTAs of tile_order[i] come i-th
    const uint32_t *list;          // sorted pairs' values: the internal index of each pair's Gaussian
    const uint2 *prect;            // tile rectangle of the Gaussian of each sorted pair
    const float4 *rec_a, *rec_b;   // records in internal order: (mu'x, mu'y, a', b'), (c', log2 o, r1, r2)
    const float *rec_t;            // and the culling threshold t of each (k_project.cu)
    uint32_t n_ids;                // Gaussians (records in rec_a / rec_b)
    const int32_t *seg;            // H x W
    int32_t view_base;             // column of segment 0 of this view
    const int32_t *view_base_dev;  // nullable: the same, read on the device (replayed graphs)
    int32_t weight_mode;
    HashEntry *hash;               // n entries (internal order)
    unsigned long long *spill_count;// the view's spill list (see HashSink)
    unsigned long long spill_cap;
    uint64_t *spill_key;
    float *spill_w;
    ViewCounters *ctr;
    unsigned long long *contrib;   // running count of composited (Gaussian, pixel) pairs
    unsigned long long *evals;     // running count of visited (Gaussian, pixel) pairs
    unsigned long long *evals_exec;// running count of evaluated lane-pixel pairs (nullable): per warp,
                                   // the Gaussians that survived its culling x its 64 pixels
    float *dbg_T, *dbg_wsum;       // nullable, H x W
    int32_t *dbg_count;            // nullable
    // trace of the Gaussians each tile stages (diagnostics; nullable): the internal index of every
    // staged Gaussian at dbg_list[dbg_off[tile] + i], i < dbg_off[tile + 1] - dbg_off[tile]
    // (beyond that *dbg_bad is set and nothing is written); dbg_staged[tile] = how many were
    // staged. With a trace the kernel keeps staging after all of a tile's pixels have stopped.
    uint32_t *dbg_list;
    const int64_t *dbg_off;
    uint32_t *dbg_staged;
    uint32_t *dbg_bad;
    uint32_t *err;                 // set when a bounded wait gave up (nullable)
    int accumulate;                // 0: compositing only (diagnostics)
    WeightRecord *recs;            // record list of the view (nullable: sums go to the tables directly)
    unsigned long long *rec_chunks;// chunks of kRecChunk records reserved (zeroed before the launch)
    uint32_t *rec_fill;            // per chunk: records written (every reserved chunk below chunk_cap)
    unsigned long long chunk_cap;  // chunks the record list holds (beyond: sums go to the tables)
    const uint32_t *skip;          // nullable: the launch does nothing when *skip is non-zero
};
void launch_composite(const CompositeArgs &a, cudaStream_t st);

// k_accum.cu
void launch_hash_init(HashEntry *hash, int64_t n, cudaStream_t st);
// Copies `bytes` (a multiple of 4) from device memory to dst with the SMs. dst may be the device
// alias of mapped pinned host memory: small results then reach the host without queueing behind
// bulk copies on the copy engines.
void launch_copy_words(const void *src, void *dst, int64_t bytes, cudaStream_t st);
// Adds the view's records to the per-Gaussian tables: of the first min(*rec_chunks, chunk_cap)
// chunks, the first rec_fill[c] records of chunk c. Nothing when *skip (nullable) is non-zero.
void launch_combine(const WeightRecord *recs, const unsigned long long *rec_chunks, const uint32_t *rec_fill,
                    unsigned long long chunk_cap, const HashSink &sink, const uint32_t *skip, cudaStream_t st,
                    const int32_t *view_base_dev = nullptr);
// The consume pass of a view (k_accum.cu): its spill list and its per-Gaussian tables to triples
// of the log, the tables' weights to the compensated sums, the spilled weights to s_ovf. A view
// whose spills exceeded the list's capacity is not consumed: its tables are cleared and nothing
// else changes, so that the view can be composited again with a larger list. Nothing at all when
// *skip (nullable) is non-zero.
struct ConsumeArgs {
    HashEntry *hash;                        // n entries (internal order)
    int64_t n;
    int32_t view_base;                      // column of segment 0 of the view
    const int32_t *view_base_dev;           // nullable: the same, read on the device
    float *s_hi, *s_lo, *s_ovf;
    unsigned long long *log_count;          // the triple log
    unsigned long long log_cap;
    uint64_t *log_key;
    float *log_w;
    uint32_t *overflow;                     // set when the log is full (never reset by a view)
    const unsigned long long *spill_count;  // the view's spill list
    unsigned long long spill_cap;
    const uint64_t *spill_key;
    const float *spill_w;
    const unsigned long long *view_contrib; // the view's composited pairs (nullable)
    unsigned long long *total_contrib;      // their running total
    const uint32_t *skip;
};
void launch_consume(const ConsumeArgs &a, cudaStream_t st);
void launch_unique_flags(const uint64_t *keys, int64_t Z, uint32_t *flags, cudaStream_t st);
// keys in the compact layout (launch_repack_keys with to_compact) of columns < 2^col_bits
void launch_uniques(const uint64_t *keys, const uint32_t *flags, const uint32_t *uidx, int64_t Z, int col_bits,
                    uint32_t *ucol, uint32_t *ustart, uint32_t *bstart, uint32_t *bend,
                    cudaStream_t st);
// Log keys between pack_key's layout, (block << 39) | (column << 7) | (Gaussian & 127), and the
// compact (block << (7 + col_bits)) | (column << 7) | (Gaussian & 127): keys_out = repacked
// keys_in (in place when they alias); w_in (nullable) is copied to w_out alongside.
void launch_repack_keys(const uint64_t *keys_in, uint64_t *keys_out, const float *w_in, float *w_out, int64_t Z,
                        int col_bits, bool to_compact, cudaStream_t st);
// k_waits.cu: one role waits limit_ns on an mbarrier that completes only when `complete` is set,
// a second role waits until the first releases it or aborts; err |= 1 (the first gave up), 2 (the
// second was aborted).
void launch_wait_check(uint64_t limit_ns, int complete, uint32_t *err, cudaStream_t st);

// Accumulated state (slag_save_state / slag_merge_state): log entries to (caller index, column),
// (caller index, column, W) back into the log with the columns shifted, and the per-Gaussian
// compensated sums of another state added.
void launch_state_unpack(const uint64_t *keys, int64_t Z, const uint32_t *orig_of_int, uint32_t *gauss, uint32_t *col,
                         cudaStream_t st);
void launch_state_pack(const uint32_t *gauss, const uint32_t *col, const float *w, int64_t Z,
                       const uint32_t *int_of_orig, int64_t n, uint32_t col_shift, uint32_t cols_in,
                       uint64_t *log_key, float *log_w, uint32_t *bad, cudaStream_t st);
void launch_state_sums(float *hi, float *lo, float *ovf, const float *bhi, const float *blo, const float *bovf,
                       int64_t n, cudaStream_t st);
struct AggArgs {
    const uint64_t *keys;
    const float *w;
    const uint32_t *flags;         // 1 where a triple starts a new (block, column)
    const uint32_t *uidx;          // exclusive prefix count of flags
    const uint32_t *ucol, *ustart, *bstart, *bend;
    const float *table;            // columns x D
    int64_t columns;
    const float *s_hi, *s_lo, *s_ovf;
    const uint32_t *orig_of_int;
    int64_t n;
    int32_t D;
    float *E;                      // n x D, caller order
    float *inv_norm;               // n, caller order
    float *wsum;                   // n, caller order
    unsigned long long *touched;
    int bf16;                      // BF16 operands (FP32 accumulation) instead of the 3xTF32 split
    // Chunked output (out-of-core finalize): the launch covers blocks block0 .. block0 + grid;
    // with E_chunk set, row r = (b - block0) * 128 + i of E_chunk / ids_chunk / wsum_chunk
    // receives Gaussian i of block b (id 0xffffffff past n) instead of E's caller-order row.
    int64_t block0;
    float *E_chunk;
    uint32_t *ids_chunk;
    float *wsum_chunk;
};
// k_aggregate_tc.cu: one CTA per block of 128 Gaussians on the tensor cores; *err is set
// when a bounded wait gives up
void launch_aggregate(const AggArgs &a, int64_t nblocks, uint32_t *err, cudaStream_t st);

// k_latent.cu: the latent form's autoencoder (D -> kLatentHidden -> kLatent -> kLatentHidden -> D)
constexpr int kLatent = 32;
constexpr int kLatentHidden = 256;
void latent_gemm(bool ta, bool tb, int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C,
                 int ldc, const float *bias, bool gelu_act, float *pre, bool round_a, bool round_b, bool accumulate,
                 cudaStream_t st);
void latent_loss(const float *Y, const float *X, int B, int D, float *dY, float *loss_sum, cudaStream_t st);
void latent_gelu_bwd(float *dH, const float *pre, int64_t n, cudaStream_t st);
void latent_colsum(const float *dC, int M, int N, float *db, cudaStream_t st);
void latent_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, int step, cudaStream_t st);
void latent_gather_rows(const float *src, const uint32_t *idx, int rows, int D, float *dst, cudaStream_t st);
// Z (n x kLatent, internal order) = sum w z_col / sum w per Gaussian from the sorted triple log
void launch_latent_aggregate(const AggArgs &a, const float *ztable, float *Z, int64_t nblocks, cudaStream_t st);
// E[orig] = Y[g] (untouched Gaussians: 0), inv_norm, wsum, touched count
void launch_latent_finish(const AggArgs &a, const float *Y, int64_t g0, int64_t rows, cudaStream_t st);

// slag_latent.cu: parameter layout and inference for input width D
struct LatentLayout {
    int64_t W1, b1, W2, b2, W3, b3, W4, b4, total;
};
LatentLayout latent_layout(int32_t D);
// enc: X (rows x D) -> Z (rows x kLatent); dec: Z -> Y (rows x D); hidden: rows x kLatentHidden scratch
void latent_encode(const float *params, int32_t D, const float *X, int rows, float *hidden, float *Z, cudaStream_t st);
// dec: Z (rows x kLatent) -> Y (rows x D) on the tensor cores; scratch: latent_decode_scratch floats;
// *err is set when a tensor-core wait gave up
int64_t latent_decode_scratch(int rows, int32_t D);
cudaError_t latent_decode(const float *params, int32_t D, const float *Z, int rows, float *scratch, float *Y,
                          uint32_t *err, cudaStream_t st);

// The linear code (SLAG_PREC_LINEAR32): params = U (D x kLatent, row-major, input x output) then
// mu (D). enc: Z = (X - mu) U, with enc_bias = -mu U; dec: Y = Z U^T + mu on the tensor cores
// (the codes as TF32 hi/lo planes times U rounded to TF32); scratch: linear_decode_scratch floats.
int64_t linear_param_count(int32_t D);
void linear_encode(const float *params, const float *enc_bias, int32_t D, const float *X, int rows, float *Z,
                   cudaStream_t st);
int64_t linear_decode_scratch(int rows, int32_t D);
cudaError_t linear_decode(const float *params, int32_t D, const float *Z, int rows, float *scratch, float *Y,
                          uint32_t *err, cudaStream_t st);

// k_query.cu
size_t query_cand_entries(int32_t B, int64_t n, int32_t k);
// per query: the best k of `per_query` candidates (score, index; index 0xffffffff = none);
// with a row list, result ids are rows[index]
void launch_query_merge(const float *cand_s, const uint32_t *cand_i, int64_t per_query, int32_t B, int32_t k,
                        const uint32_t *rows, int64_t *out_ids, float *out_scores, int32_t *out_count,
                        cudaStream_t st);
// The candidates are rows rows[0..n) of E (rows nullable: rows 0..n); ids returned are E rows.
void launch_query_topk(const float *Q, int32_t B, const float *E, const float *inv_norm, const uint32_t *rows,
                       int64_t n, int32_t D, int32_t k, float *cand_s, uint32_t *cand_i, int64_t *out_ids,
                       float *out_scores, int32_t *out_count, cudaStream_t st);
// Threshold query over candidate rows rows[0..n) of E: ids[0..min(count, cap)) = the rows with
// cosine q . E / |E| >= thr, in increasing order; *d_count = their number (flags, pos: n each).
void launch_threshold_query(const float *q, const float *E, const float *inv_norm, const uint32_t *rows, int64_t n,
                            int32_t D, float thr, uint32_t *flags, uint32_t *pos, unsigned long long *d_count,
                            int64_t cap, int64_t *ids, SortScratch &scratch, cudaStream_t st);
// rows[0..*d_count) = the Gaussians with inv_norm > 0, in increasing order (flags, pos: n each)
void launch_touched_rows(const float *inv_norm, int64_t n, uint32_t *flags, uint32_t *pos, uint32_t *rows,
                         unsigned long long *d_count, SortScratch &scratch, cudaStream_t st);

// k_dense_tc.cu: dense layers on tcgen05. out = act(A W + b) for A given as TF32 hi/lo planes
// (2 x rows_pad x K, rows_pad = dense_tc_pad_rows(rows)) and wt = the transposed, bfloat16-rounded
// weights (N x K, launch_weights_t; rounded to TF32 instead with tf32). gelu_planes: out receives gelu(A W + b) as TF32 hi/lo
// planes (2 x rows_pad x N); otherwise float32 rows (rows x ldo). K % 32 == 0, N % 128 == 0.
// *err is set when a wait gave up.
int64_t dense_tc_pad_rows(int64_t rows);
void launch_weights_t(const float *W, int32_t K, int32_t N, float *wt, cudaStream_t st, bool tf32 = false);
cudaError_t launch_dense_tc(const float *a_planes, int64_t rows, int64_t rows_pad, int32_t K, const float *wt,
                            int32_t N, const float *bias, bool gelu_planes, float *out, int64_t ldo, uint32_t *err,
                            cudaStream_t st);

// TF32 hi/lo planes (2 x rows_pad x K floats; rows rows .. rows_pad zero) of a row-major
// rows x K float32 matrix (K a multiple of 4).
void launch_tf32_planes(const float *src, int64_t rows, int64_t rows_pad, int32_t K, float *dst, cudaStream_t st);

// k_query_tc.cu: tensor-core scores (3xTF32 on tcgen05) for k <= 16 and D % 32 == 0
bool query_tc_supported(int32_t D, int32_t k);
// Default split of the Gaussian tiles over CTAs (one wave of 148 CTAs); tiles of n candidates.
int32_t query_tc_splits(int32_t B, int64_t n);
int64_t query_tc_tiles(int64_t n);
// Rows of the split operand planes: n candidates padded to whole tiles, B queries padded likewise.
int64_t query_tc_pad_rows(int64_t n);
int64_t query_tc_pad_queries(int32_t B);
// The TF32 hi/lo planes of the candidates rows[0..n) of E (Ehl: 2 x query_tc_pad_rows(n) x D
// floats) and their inverse norms (qinv: query_tc_pad_rows(n) floats, NaN for zero and padding rows).
void launch_query_split_e(const float *E, const float *inv_norm, const uint32_t *rows, int64_t n, int32_t D,
                          float *Ehl, float *qinv, cudaStream_t st);
// Splits Q into Qhl (2 x query_tc_pad_queries(B) x D floats), scores it against Ehl / qinv and
// merges; result ids are rows[candidate]. splits <= 0: the default split.
cudaError_t launch_query_topk_tc(const float *Q, int32_t B, float *Qhl, const float *Ehl, const float *qinv,
                                 const uint32_t *rows, int64_t n, int32_t D, int32_t k, float *cand_s,
                                 uint32_t *cand_i, int64_t *out_ids, float *out_scores, int32_t *out_count,
                                 uint32_t *err, cudaStream_t st, int32_t splits);

}  // namespace slag
