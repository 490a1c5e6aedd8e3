/*
 * slag.h -- C ABI of the B300 lifting library (libslag.so).
 *
 * The library implements the "Semantic Embedding" stage of SLAG (Method
 * section): 2D language features, one embedding per image segment, are lifted
 * onto the Gaussians of a 3D Gaussian-splatting scene without a loss
 * function. Every Gaussian k receives the normalised weighted average
 *
 *     E_k = sum_i sum_j sum_{p in M_j} w_{k,p} E_j  /  sum_i sum_j sum_{p in M_j} w_{k,p}
 *
 * (Aggregation step), where i runs over views, j over the segments (masks) of
 * view i, p over the pixels of segment j, and w_{k,p} is the weight the
 * rasterizer assigns to Gaussian k at pixel p (Rasterizer_SLAG statement and
 * Eq. 2). Queries are cosine similarity searches over the resulting N x D
 * tensor ("Query processing for inference").
 *
 * Conventions shared by every entry point:
 *   - All compute runs on the CUDA device current at slag_create, in the
 *     stream given in slag_options (NULL = the legacy default stream).
 *   - The caller owns every buffer it passes. Inputs flagged on_device are
 *     read asynchronously in the context's stream and must stay valid until
 *     that stream has passed the call; host inputs are consumed before the
 *     call returns. Outputs are caller-allocated.
 *   - No call throws; each returns a slag_status. slag_last_error() gives a
 *     one-line description of the last failure of a context.
 *   - A context is not thread-safe: one host thread at a time.
 *   - Gaussian indices in every output are the caller's original indices.
 */
#ifndef SLAG_H
#define SLAG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slag_ctx slag_ctx;

typedef enum {
    SLAG_OK = 0,
    SLAG_ERR_INVALID_ARG = 1, /* bad pointer, size, non-finite input, segment id outside [-1, M) */
    SLAG_ERR_STATE = 2,       /* call not allowed now (e.g. query before finalize) */
    SLAG_ERR_OOM = 3,         /* device or pinned host allocation failed */
    SLAG_ERR_CUDA = 4,        /* a CUDA runtime call failed; see slag_last_error */
    SLAG_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    SLAG_ERR_CAPACITY = 6     /* an internal bound was exceeded (see the entry point) */
} slag_status;

/* Weight recorded per (Gaussian, pixel):
 *   SLAG_WEIGHT_ALPHA_T: the front-to-back compositing weight w = alpha * T,
 *     alpha = min(0.99, opacity * exp(-q/2)), T = prod over earlier
 *     contributors of (1 - alpha); the weights of a pixel sum to 1 - T_final.
 *   SLAG_WEIGHT_KERNEL: the raw splat kernel exp(-q/2) of Eq. 2, recorded
 *     for the same contributing set.
 * In both modes a Gaussian contributes to a pixel when alpha >= 1/255 and the
 * transmittance after it stays >= 1e-4 (the first Gaussian that would push it
 * below 1e-4 ends the pixel and is not counted). */
enum { SLAG_WEIGHT_ALPHA_T = 0, SLAG_WEIGHT_KERNEL = 1 };

/* Arithmetic of the aggregation (Aggregation, E_k formula): the per-view
 * weights are always composited in float32 and Sum w is a compensated float32
 * sum. FP32: the contraction of the weights with the segment embeddings runs
 * at float32 accuracy (three-term TF32 split on the tensor cores). BF16: the
 * weights and the segment embeddings enter the tensor cores as bfloat16 with
 * float32 accumulation; the error against float64 is stated per result by the
 * tests (cosine >= 1 - 1e-3 per touched Gaussian at the tested scales). No
 * float64 is used on the GPU in either form. */
enum { SLAG_PREC_FP32 = 0, SLAG_PREC_BF16 = 1, SLAG_PREC_LATENT32 = 2, SLAG_PREC_LINEAR32 = 3 };
/* LATENT32: the learned latent form. The views' segment embeddings are
 * encoded to 32-d codes by a small autoencoder (slag_latent_train; set with
 * slag_set_latent before the first view; finalize encodes every stored
 * segment embedding in one pass), the aggregation runs on the codes,
 * and finalize decodes each touched Gaussian's mean code to D dimensions
 * (the decoder is not linear: dec(mean code) is not the mean of decoded
 * codes; the float32 path is the reference for its error). */

/* LINEAR32: the latent form with a linear 32-d code. With U the top 32
 * principal directions of training embeddings and mu their mean
 * (slag_linear_code_fit; set with slag_set_linear_code before the first
 * view), a segment embedding e is encoded as z = U^T (e - mu) and a code is
 * decoded as mu + U z. The code is linear, so the aggregation of codes is
 * exact: the decoded mean code is mu + U U^T (E_k - mu), the projection of the
 * Aggregation step's E_k onto the code's affine subspace, and its error is the
 * part of E_k outside it (the floor of any 32-d linear code fitted to those
 * embeddings). */

/* SLAG_FLAG_EMBEDDINGS_ON_HOST: the context holds no n x D copy of the
 * embeddings on the device (out-of-core aggregation, after the paper's
 * multi-GPU section, where the aggregation tensor outgrows device memory and
 * is processed in Gaussian-range chunks). slag_finalize then writes host
 * memory only, computing the rows in chunks of spatially adjacent Gaussians,
 * and queries return SLAG_ERR_STATE; slag_export_partitions works in both
 * modes. */
enum { SLAG_FLAG_EMBEDDINGS_ON_HOST = 1 };

/* The Gaussian set G = {G_1..G_N} (Method, Rasterizer_SLAG statement). */
typedef struct {
    int64_t n;               /* number of Gaussians, 1 <= n < 2^31 */
    const float *means;      /* n x 3, world space */
    const float *scales;     /* n x 3, linear standard deviations (>= 0) */
    const float *quats;      /* n x 4, rotation (w, x, y, z), any non-zero norm */
    const float *opacities;  /* n, activated, in [0, 1] */
    int32_t on_device;       /* 1: the four pointers are device pointers */
} slag_gaussians;

/* Pinhole camera (K_i, R_i, t_i). OpenCV axes: x right, y down, z forward.
 * A world point X maps to x_c = R X + t and to pixel (fx x/z + cx, fy y/z + cy);
 * pixel (u, v) covers [u, u+1) x [v, v+1), its centre is (u + 0.5, v + 0.5). */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;   /* 1 .. 65535 */
    float R[9];              /* world -> camera rotation, row-major */
    float t[3];
    float near_z, far_z;     /* a Gaussian is kept when near_z < z_c < far_z; near_z > 0 */
} slag_camera;

typedef struct {
    int32_t dim;             /* D: embedding width, a multiple of 128, 128 .. 4096 */
    int32_t precision;       /* SLAG_PREC_FP32, _BF16, _LATENT32 or _LINEAR32 */
    int32_t weight_mode;     /* SLAG_WEIGHT_ALPHA_T (default) or SLAG_WEIGHT_KERNEL */
    int32_t flags;           /* SLAG_FLAG_* bits, or 0 */
    void *cuda_stream;       /* cudaStream_t, NULL = legacy default stream */
} slag_options;

/* Counters of the views added since create / reset. views and columns count
 * every accepted view; pairs, last_pairs, resized_views and recomposited_views
 * count the views whose counters the host has read (all of them after a
 * finalize); a view is read when its slot is reused or the views are joined;
 * contributions, triples, last_contributions, evaluations and executed are
 * read at finalize. evaluations and executed count the compositing work done,
 * so a view composited twice counts twice there (and once everywhere else). */
typedef struct {
    int64_t views;           /* views added since create / reset */
    int64_t pairs;           /* sum over views of Gaussian-tile pairs P */
    int64_t contributions;   /* sum over views of composited (Gaussian, pixel) pairs */
    int64_t triples;         /* stored (Gaussian, view-segment, W) entries */
    int64_t columns;         /* sum over views of M (segment embeddings kept) */
    int64_t last_pairs;      /* P of the last view */
    int64_t last_contributions;
    int64_t touched;         /* Gaussians with sum w > 0 at the last finalize */
    int64_t evaluations;     /* sum over views of (Gaussian, pixel) pairs visited before each
                                pixel ended (the compositing work, contributing or not): a pixel
                                that stopped counts its tile's candidates up to the end of the
                                chunk of 32 in which it stopped */
    int64_t executed;        /* sum over views of the (Gaussian, pixel) evaluations the
                                compositing kernel carried out: a group of 64 pixels evaluates
                                the Gaussians that can reach alpha >= 1/255 somewhere in it,
                                for all 64 pixels; read at finalize */
    int64_t resized_views;   /* views sized on the device whose pairs exceeded the capacity of
                                their binning, binned again with their exact count */
    int64_t recomposited_views; /* views whose (Gaussian, segment) sums overflowed their slot's
                                spill list (sums of Gaussians that reach more segments of the
                                view than the per-Gaussian table holds), composited again with
                                a list that holds them all */
} slag_stats;

/* Create a context over the Gaussian set (Method, Rasterizer_SLAG statement:
 * G is fixed while views are added). Copies and reorders the Gaussians into
 * device memory and allocates the workspace. Errors: INVALID_ARG for a NULL
 * pointer, n out of range, a non-finite value, a zero quaternion, a negative
 * scale or an opacity outside [0, 1], bad options; OOM; CUDA. *out is set only
 * on success. */
slag_status slag_create(const slag_gaussians *g, const slag_options *opt, slag_ctx **out);

/* Add one view (Method: Rasterization, Parameter Masking and the view's share
 * of the Aggregation sums). seg_ids: height x width int32, row-major, the
 * segment id of each pixel in [0, M) or -1 for a pixel in no segment (the
 * masks M_j of the view as a partition); seg_table: M x dim float32,
 * row-major, the embedding E_j of segment j. A pixel may belong to several
 * overlapping masks by adding the same camera again with a second id map.
 * Runs projection, tile binning, the two sorts, compositing, masking and the
 * per-view reduction, in two halves. This call uploads the inputs, checks the
 * segment ids and queues the first half (projection, depth sort, tile-count
 * scan). The second half (binning, compositing, masking, reduction) is sized
 * by the view's pair count:
 *  - once earlier views give an estimate of it (from the second view of a
 *    context on, when the view has at most 2048 bins of 4x4 tiles), this call
 *    queues it too, sized on the device: a view whose pairs exceed the
 *    estimate is flagged on the device, composites nothing, and is binned
 *    again with its exact count when its slot is reused (kSlots = 6 views
 *    later) or the views are joined (stats.resized_views counts these). Unless
 *    stages are being timed (slag_set_profiling), these views replay CUDA
 *    graphs of the view's work, captured once per slot and image size
 *    (slag_set_graphs);
 *  - otherwise the host reads the count, and the second half is queued by
 *    the next call on the context: the next slag_add_view, or slag_finalize /
 *    slag_finalize_async / slag_export_partitions / slag_get_profile /
 *    slag_bin_view / slag_render_debug.
 * The caller's buffers are free when the call returns. Errors: INVALID_ARG
 * (NULL pointer, camera not finite or out of range, M < 1 or M >= 2^24, a
 * segment id outside [-1, M): the view is then not added); OOM; CUDA. The
 * second half's errors, CAPACITY (more than 2^31 - 1 Gaussian-tile pairs in
 * the view), OOM and CUDA, are returned by the call that queues or settles
 * it, and the context then needs slag_reset. slag_reset drops the views whose
 * second half is not queued or not settled. */
slag_status slag_add_view(slag_ctx *ctx, const slag_camera *cam, const int32_t *seg_ids,
                          const float *seg_table, int32_t M, int32_t on_device);

/* Normalise (Aggregation step, E_k formula) and make the embeddings
 * queryable. out_emb: n x dim float32 (nullable), E_k in the caller's
 * Gaussian order; a Gaussian no view touched (sum w = 0) gets the zero
 * vector. out_wsum: n float32 (nullable), the denominator sum w. on_device
 * says where the two outputs live. May be called again after more views.
 * Errors: STATE before any view; CAPACITY when the triple log overflowed in
 * some view (the log is grown ahead of every view to hold what it can append:
 * 4 triples per Gaussian from its tables plus its spill list, which a view
 * that outgrows it is composited again with); OOM; CUDA. */
slag_status slag_finalize(slag_ctx *ctx, float *out_emb, float *out_wsum, int32_t on_device);

/* slag_finalize with asynchronous outputs: the aggregation runs as in
 * slag_finalize (the call returns once the embeddings are queryable), but the
 * copies into out_emb and out_wsum are queued on the context's copy stream and
 * complete later; the output buffers must not be read (nor freed) before
 * slag_wait_outputs returns. Host outputs overlap with later work only when
 * they are pinned (page-locked) memory. The context keeps two device copies
 * of the embeddings and sum w so that the next finalize does not wait for
 * these copies; the second copy (n x dim + n float32) is allocated by the
 * first finalize that needs it. Errors: as slag_finalize; INVALID_ARG with
 * SLAG_FLAG_EMBEDDINGS_ON_HOST. */
slag_status slag_finalize_async(slag_ctx *ctx, float *out_emb, float *out_wsum, int32_t on_device);

/* Waits until every output copy queued by slag_finalize_async is complete.
 * Errors: CUDA. */
slag_status slag_wait_outputs(slag_ctx *ctx);

/* Cosine top-k of one query vector q (dim float32, host) over the finalized
 * embeddings ("Query processing for inference"). Candidates are Gaussians
 * with sum w > 0 and a non-zero embedding; scores are q . E_k / |E_k| (q is
 * used as given: pass a unit vector for cosine). Results are ordered by
 * descending score, ties to the lower Gaussian index. out_ids (int64) and
 * out_scores (float) hold k entries on the host; *out_count (nullable)
 * receives min(k, candidates); unused slots get id -1. Errors: STATE before
 * finalize; INVALID_ARG for k < 1 or k > 1024. */
slag_status slag_query(slag_ctx *ctx, const float *q, int32_t k, int64_t *out_ids,
                       float *out_scores, int32_t *out_count);

/* Allocation-free cosine top-k over embeddings the caller holds on the
 * device. The paper has no counterpart: this entry point exists for callers
 * that must not allocate device memory once running -- a query service on a
 * robot or embedded board that reserves its memory at start-up (cudaMalloc can
 * synchronise the device and take unbounded time), or an application whose
 * device memory is owned by its own allocator. It runs the same scoring and
 * selection kernels as slag_query_batch and allocates nothing: its scratch is
 * one 16 MiB array inside the library, which every GPU that loads the
 * library holds until the process exits.
 *   E: n x dim float32 row-major (device, 16-byte aligned), e.g. the output of
 *   slag_finalize; wsum: n float32 (device, nullable) -- rows with wsum <= 0
 *   are not candidates; rows with a zero norm never are. Q: B x dim float32
 *   (device, 16-byte aligned). Outputs (device): out_ids B x k int64,
 *   out_scores B x k float32, out_count B int32 (nullable), with the ordering,
 *   candidates and -1 padding of slag_query_batch. dim: a multiple of 16 in
 *   16..4096; 1 <= k <= 1024.
 *   Work is enqueued in cuda_stream (NULL = legacy default stream); the
 *   outputs are ready when that stream has passed the call.
 *   Size limit: 4 n + 8 B ceil(n / 128) min(k, 128) bytes (each of the three
 *   parts rounded up to 256) must not exceed 16 MiB; larger requests return
 *   SLAG_ERR_CAPACITY without launching anything (split the queries).
 *   The first call on a device looks up the array's device address (once per
 *   device and driver context, with that device current; a call after a
 *   device reset looks it up again); make that first call before any stream
 *   capture. Every call uses the same array: nothing in it needs to start at
 *   zero (each call writes all it reads), but calls that overlap on the GPU --
 *   in different streams or from different threads -- race on it.
 *   Every pointer must be memory of the current device (device or managed
 *   allocations); host memory, pinned or not, is refused before any launch.
 * Errors: INVALID_ARG (NULL pointer, sizes out of range, misaligned E or Q, a
 * pointer that is not memory of the current device); CAPACITY (see above);
 * CUDA. */
slag_status slag_noalloc_query_topk(const float *E, int64_t n, int32_t dim, const float *wsum,
                                    const float *Q, int32_t B, int32_t k, int64_t *out_ids,
                                    float *out_scores, int32_t *out_count, void *cuda_stream);

/* Threshold query: the binary response of the paper's open-vocabulary
 * evaluation (Experiments: a Gaussian answers a text query when the cosine of
 * its embedding with the query is at least a threshold, 0.28 there). q: dim
 * float32 (host, or device when on_device; 16-byte aligned); candidates as
 * in slag_query. out_ids (host or device as on_device, cap entries,
 * nullable when cap = 0) receives the ids with q . E_k / |E_k| >= threshold in
 * increasing order, the first cap of them; *out_count their total number
 * (call with cap = 0 to size the output). Errors: STATE before finalize;
 * INVALID_ARG (NULL q or out_count, cap < 0, non-finite threshold). */
slag_status slag_query_threshold(slag_ctx *ctx, const float *q, float threshold, int64_t *out_ids, int64_t cap,
                                 int64_t *out_count, int32_t on_device);

/* Batched form of slag_query: Q is B x dim float32 row-major; out_ids and
 * out_scores are B x k, out_count is B (nullable). on_device says where Q and
 * the outputs live. Same ordering, candidates and errors as slag_query. */
slag_status slag_query_batch(slag_ctx *ctx, const float *Q, int32_t B, int32_t k, int64_t *out_ids,
                             float *out_scores, int32_t *out_count, int32_t on_device);

/* Drop every added view (sums, stored triples and segment embeddings); keep
 * the Gaussians and the workspace. */
slag_status slag_reset(slag_ctx *ctx);

slag_status slag_get_stats(const slag_ctx *ctx, slag_stats *out);
const char *slag_last_error(const slag_ctx *ctx);
void slag_destroy(slag_ctx *ctx);

/* ---- accumulated state: checkpoint, resume, merge -------------------------- */

/* The aggregation sums are additive over views (Aggregation step: numerator
 * and denominator of E_k are sums over views i), which is what lets the
 * paper's multi-GPU section split the views across GPUs and sum the
 * per-GPU tensors. A context's accumulated state -- every view's sparse
 * (Gaussian, view-segment, W) weights, the stored segment embeddings, the
 * compensated sums of w per Gaussian and the counters -- can therefore be
 * saved, restored into another context over the same Gaussians, and merged
 * with the state of a disjoint set of views. Format (little-endian):
 *   header (96 bytes): "SLAGSTAT", uint32 version = 1, uint32 dim, int64 n,
 *     int64 columns, int64 triples Z, uint64 fingerprint of the Gaussian set,
 *     int64 views, pairs, contributions, evaluations, executed, int32
 *     weight_mode, int32 reserved;
 *   float32 segment embeddings, columns x dim;
 *   float32 sum w as (hi, lo, overflow) planes, 3 x n, in caller order (the
 *     sum is hi + lo + overflow; hi + lo is a compensated sum);
 *   Z x uint32 caller index, Z x uint32 column, Z x float32 W.
 * Size: 96 + 4 columns dim + 12 n + 12 Z bytes. */

/* Writes the context's state (after joining the views in flight) into buf
 * (host, cap bytes). *out_bytes (nullable) receives its size; with buf NULL
 * only the size is returned. Errors: CAPACITY when cap is smaller than the
 * state or the triple log overflowed in some view; OOM; CUDA. */
slag_status slag_save_state(slag_ctx *ctx, void *buf, int64_t cap, int64_t *out_bytes);

/* Replaces the context's accumulated state by the one in buf (host, `bytes`
 * bytes): as slag_reset, then slag_merge_state. Later views add to it. */
slag_status slag_load_state(slag_ctx *ctx, const void *buf, int64_t bytes);

/* Adds the state in buf (host) to the context's: its segment embeddings are
 * appended after the context's columns, its triples with their columns
 * shifted past them, and its sums of w added with compensation. The result
 * equals one context that was given both sets of views (the two sets should be
 * disjoint, or views are counted twice). Errors: INVALID_ARG for a buffer that
 * is not a state, or a state of another n, dim, weight mode or Gaussian set,
 * or a triple whose index or column is out of range (its weight is dropped;
 * reset the context); CAPACITY beyond 2^32 columns; OOM; CUDA. The caller's
 * buffer is free when the call returns. */
slag_status slag_merge_state(slag_ctx *ctx, const void *buf, int64_t bytes);

/* Merges two states on the host, without a context or a GPU (for reducing the
 * states of view-sharded jobs where they are stored): out (host, cap bytes)
 * receives the state of both sets of views, a's columns first. *out_bytes
 * (nullable) receives the size; with out NULL only the size is returned.
 * Errors: INVALID_ARG (malformed, or states of other n, dim, weight mode or
 * Gaussian set); CAPACITY (cap too small, or beyond 2^32 columns). */
slag_status slag_state_merge_host(const void *a, int64_t a_bytes, const void *b, int64_t b_bytes, void *out,
                                  int64_t cap, int64_t *out_bytes);

/* ---- diagnostics: the integer stages and per-pixel compositing state ---- */

/* Tile binning of one view without compositing. out_touched: n uint32 (host,
 * nullable), tiles touched per Gaussian in the caller's order (0 = culled);
 * *out_P: number of Gaussian-tile pairs; out_list (host, nullable, list_cap
 * entries): the Gaussian of each pair, grouped by tile in row-major tile
 * order, each tile's Gaussians in ascending (float32 depth, Gaussian index);
 * out_ranges (host, nullable): tiles x 2 int64 [start, end) into out_list.
 * Errors: CAPACITY when out_list is given and list_cap < P (nothing written
 * to out_list). */
slag_status slag_bin_view(slag_ctx *ctx, const slag_camera *cam, uint32_t *out_touched,
                          int64_t *out_P, int32_t *out_list, int64_t list_cap, int64_t *out_ranges);

/* The bins of one view at the granularity the compositing uses, without
 * compositing (the integer stages as they run in slag_add_view). A bin is a
 * 2^bin_shift x 2^bin_shift square of 16x16 tiles: bin_shift 0 gives the
 * lists of slag_bin_view, bin_shift 2 the 4x4-tile super-tiles slag_add_view
 * composites from (other values: INVALID_ARG). A Gaussian belongs to every
 * bin its tile rectangle meets. *out_P: the number of (Gaussian, bin) pairs;
 * out_list (host, nullable, list_cap entries): the caller index of each pair,
 * grouped by bin in row-major bin order, each bin's Gaussians in ascending
 * (float32 depth, Gaussian index); out_ranges (host, nullable): bins x 2 int64
 * [start, end) into out_list, bins = ceil(tiles_x / 2^bin_shift) x
 * ceil(tiles_y / 2^bin_shift); an empty bin is [e, e). Errors: as
 * slag_bin_view. */
slag_status slag_bin_view_bins(slag_ctx *ctx, const slag_camera *cam, int32_t bin_shift, int64_t *out_P,
                               int32_t *out_list, int64_t list_cap, int64_t *out_ranges);

/* The per-tile Gaussian sequences the compositing kernel of slag_add_view
 * stages from the super-tile lists (its filter of each super-tile's list by
 * tile rectangle), recorded by the kernel itself; no view is added. The trace
 * keeps staging after every pixel of a tile has stopped, so that each tile's
 * whole sequence is visible. *out_P: the number of Gaussian-tile pairs;
 * out_list (host, nullable, list_cap >= P entries): caller indices, tile
 * after tile in row-major order; out_ranges (host, nullable): tiles x 2 int64,
 * [start, start + staged) of each tile, start being the tile's place in the
 * flat per-tile lists of slag_bin_view. Errors: as slag_bin_view; CAPACITY
 * when a tile staged more Gaussians than its flat list holds. */
slag_status slag_composite_trace(slag_ctx *ctx, const slag_camera *cam, int64_t *out_P, int32_t *out_list,
                                 int64_t list_cap, int64_t *out_ranges);

/* Composite one view without adding it: per pixel (height x width, host,
 * each nullable) the final transmittance, the sum of the recorded weights
 * over every contributing Gaussian and the number of contributors. */
slag_status slag_render_debug(slag_ctx *ctx, const slag_camera *cam, float *out_T, float *out_wsum,
                              int32_t *out_count);

/* ---- batched scenes ------------------------------------------------------- */

/* One view of a batched call (the arguments of slag_add_view). */
typedef struct {
    const slag_camera *camera;
    const int32_t *seg_ids;
    const float *seg_table;
    int32_t M;
    int32_t on_device;
} slag_view;

/* Adds views to several independent scenes (one context each) in one call:
 * views[c][0 .. n_views[c]) go to ctxs[c], scene after scene. After a scene's
 * last view the call also queues that view's second half (see slag_add_view),
 * so the scene's work runs while the next scene's views are added, with no
 * finalize in between to drain the GPU. The result of each context is that of
 * adding its views in order with slag_add_view. Stops at the first error;
 * *failed_ctx (nullable) receives its context index, or -1. */
slag_status slag_add_views_batched(int32_t n_ctx, slag_ctx *const *ctxs, const slag_view *const *views,
                                   const int32_t *n_views, int32_t *failed_ctx);

/* Replays of captured CUDA graphs for views sized on the device (on by
 * default): per slot of views in flight, the view's first half and binning,
 * its compositing and combine pass, and its consume pass are captured as three
 * graphs at the first such view of an image size (again whenever a buffer they
 * use is reallocated) and replayed for the later ones, with the view's camera
 * and first column read from device memory; the host then issues a handful of
 * calls per view instead of some 60 launches and stream operations. Off: the
 * same work is launched kernel by kernel. The results are the same. */
slag_status slag_set_graphs(slag_ctx *ctx, int32_t enable);

/* Query autotuning (on by default): for a batch shape with enough work, the
 * first device-side query times the tensor-core kernel at the default split of
 * the Gaussian tiles, half and double of it, and keeps the fastest for that
 * (batch, candidates) shape. Device-side queries run as a CUDA graph that is
 * captured once and replayed while the buffers, shape and embeddings repeat. */
slag_status slag_set_autotune(slag_ctx *ctx, int32_t enable);

/* ---- the latent form: autoencoder D -> 256 -> 32 -> 256 -> D ---------------- */

/* Parameters of the autoencoder for input width dim (float32, layout: W1 dim x 256,
 * b1 256, W2 256 x 32, b2 32, W3 32 x 256, b3 256, W4 256 x dim, b4 dim; W row-major
 * input x output). 0 for an unsupported width. */
int64_t slag_latent_param_count(int32_t dim);

/* Trains the autoencoder on n samples (n x dim float32, rows of unit length in
 * the method's use) with Adam at learning rate lr, batches of `batch`, for
 * `epochs` passes over a seeded shuffle. Products take the weights rounded to
 * bfloat16 with float32 accumulation (float32 master weights). The loss per
 * sample is mean((dec(enc(x)) - x)^2) + (1 - cos(dec(enc(x)), x)).
 * samples: host (on_device = 0) or device memory. out_params (host,
 * slag_latent_param_count(dim) floats) receives the trained parameters,
 * out_loss (host, `epochs` floats, nullable) the mean loss of each epoch.
 * dim must be a multiple of 32 in 32 .. 4096. */
slag_status slag_latent_train(const float *samples, int64_t n, int32_t dim, int32_t epochs, int32_t batch,
                              float lr, uint64_t seed, int32_t on_device, float *out_params, float *out_loss,
                              void *cuda_stream);

/* Applies the autoencoder (host parameters) to `rows` host vectors: mode 0
 * encodes (in rows x dim -> out rows x 32), 1 decodes (rows x 32 -> rows x
 * dim), 2 does both (rows x dim -> rows x dim). The decoder runs on the tensor
 * cores (TF32 hi/lo activations times the bfloat16-rounded weights), as at
 * finalize. Errors: INVALID_ARG, OOM, CUDA; TIMEOUT when a tensor-core wait
 * gave up. */
slag_status slag_latent_apply(const float *params, int32_t dim, const float *in, int64_t rows, int32_t mode,
                              float *out, void *cuda_stream);

/* Sets the autoencoder (host parameters, slag_latent_param_count(D) floats) of
 * a context created with SLAG_PREC_LATENT32; before the first view. */
slag_status slag_set_latent(slag_ctx *ctx, const float *params);

/* ---- the linear 32-d code (SLAG_PREC_LINEAR32) --------------------------- */

/* Parameters of the linear code for input width dim: U (dim x 32, row-major,
 * input x output; orthonormal columns) then mu (dim): dim x 33 floats; 0 for
 * an unsupported width. */
int64_t slag_linear_param_count(int32_t dim);

/* Fits the linear code to n samples (n x dim float32, host or device): mu is
 * their mean and U the top 32 eigenvectors of their covariance (principal
 * component analysis: the second moment is accumulated on the device, the
 * eigenvectors found in float64 by subspace iteration with a Rayleigh-Ritz
 * step). out_params (host, slag_linear_param_count(dim) floats); *out_kept
 * (nullable) the fraction of the samples' variance the 32 directions keep.
 * dim a multiple of 32 in 32 .. 4096, 2 <= n < 2^31. */
slag_status slag_linear_code_fit(const float *samples, int64_t n, int32_t dim, int32_t on_device,
                                 float *out_params, float *out_kept, void *cuda_stream);

/* Sets the linear code (host parameters as above) of a context created with
 * SLAG_PREC_LINEAR32; before the first view. */
slag_status slag_set_linear_code(slag_ctx *ctx, const float *params);

/* ---- out-of-core output: per-area embedding files ------------------------- */

/* Device memory the out-of-core finalize of SLAG_FLAG_EMBEDDINGS_ON_HOST may
 * hold for output rows at a time: it then computes the rows in chunks of at
 * most bytes / (4 dim + 8) Gaussians (whole blocks of 128, at least one
 * block). 0 restores the default of 2^20 Gaussians per chunk. Errors:
 * INVALID_ARG for bytes < 0. */
slag_status slag_set_device_budget(slag_ctx *ctx, int64_t bytes);

/* Spatial partition export (the paper stores a large scene's embeddings per
 * area of a grid over the Gaussian means instead of in a vector database).
 * Aggregates the views added so far in chunks of at most chunk_gaussians
 * Gaussians on the device (rounded to blocks of 128 spatially adjacent
 * Gaussians; <= 0 picks 2^20) and appends every touched Gaussian (sum w > 0)
 * to the file of its cell of a cells_x x cells_y grid over the x-y bounding
 * box of all means. The directory is created if missing. Files:
 *   dir/cell_<cx>_<cy>.slag: "SLAGPART" (8 bytes), uint32 version = 1,
 *     uint32 D, int64 count, float x0, x1, y0, y1 (the cell's bounds), then
 *     count records of int64 caller index, float sum w, float E[D];
 *   dir/index.txt: one line per non-empty cell: cx cy count x0 x1 y0 y1 file.
 * *out_written (nullable) receives the number of records. Errors: STATE
 * before any view, INVALID_ARG for a bad grid or path, the CUDA and OOM codes,
 * and SLAG_ERR_CUDA for a file that cannot be written. */
slag_status slag_export_partitions(slag_ctx *ctx, const char *dir, int32_t cells_x, int32_t cells_y,
                                   int64_t chunk_gaussians, int64_t *out_written);

/* ---- diagnostics: per-stage device time ---------------------------------- */

/* Stages timed with CUDA events recorded in the streams that run them. */
enum {
    SLAG_STAGE_PROJECT = 0,    /* projection, depth sort, depth-rank gather, tile-count scan */
    SLAG_STAGE_BIN = 1,        /* pair emission, stable sort by bin, bin ranges */
    SLAG_STAGE_COMPOSITE = 2,  /* compositing, masking, in-tile segment binning */
    SLAG_STAGE_CONSUME = 3,    /* combine pass, per-view (segment, weight) tables -> triple log */
    SLAG_STAGE_LOG_SORT = 4,   /* finalize: sort of the triple log, distinct columns */
    SLAG_STAGE_AGGREGATE = 5,  /* finalize: blocked contraction and normalisation */
    SLAG_STAGE_QUERY = 6,      /* cosine scores and top-k */
    SLAG_STAGE_COUNT = 7
};

typedef struct {
    double ms[SLAG_STAGE_COUNT];       /* summed duration of the stage's spans */
    int64_t spans[SLAG_STAGE_COUNT];   /* number of timed spans per stage */
    double busy_ms[SLAG_STAGE_COUNT];  /* time covered by at least one span of the stage: views in
                                          flight overlap, so ms can exceed it */
} slag_profile;

/* Turn per-stage timing on (1) or off (0). Off by default; when on, every
 * stage is bracketed by two events in the context's stream (no extra
 * synchronisation: spans are resolved at the calls that synchronise). */
slag_status slag_set_profiling(slag_ctx *ctx, int32_t enable);

/* Per-stage timing of the stages in `stages` only (bit s = stage s; bits at
 * or above SLAG_STAGE_COUNT are ignored; 0 turns timing off). Each timed
 * span costs two event records and, when resolved, a few driver calls on
 * the host, so timing only the stage of interest disturbs the rest least.
 * Spans resolve at slag_get_profile, or once 4096 are pending. The first
 * call that turns timing on creates the events for that backlog. With the
 * query stage untimed, device-buffer queries keep their CUDA graph. */
slag_status slag_set_profiling_stages(slag_ctx *ctx, uint32_t stages);

/* Synchronises the context's streams, adds every finished span to *out and,
 * when reset is non-zero, clears the totals. busy_ms covers the spans
 * resolved since profiling was enabled or last reset. */
slag_status slag_get_profile(slag_ctx *ctx, slag_profile *out, int32_t reset);

/* ---- the checked build ------------------------------------------------------
 * libslag_checks.so is this library compiled with -DSLAG_CHECKS: index checks
 * in pair emission, the sort's scatter, compositing and aggregation, in place
 * of the sanitizer that this library's tests cannot use. An index outside its
 * buffer is then not used; the check sets an error word, and the next call
 * that synchronises (slag_finalize, the diagnostics) returns
 * SLAG_ERR_CAPACITY naming the stages. In the regular build the checks are
 * compiled out. */

/* 1 in the checked build, 0 otherwise. */
int32_t slag_is_checked_build(void);

/* Checked build only: the pair buffers of the following views behave as if
 * they held cap pairs (0 = off), so that the emission's checks refuse the
 * pairs beyond cap (a forced capacity overflow; the views' results are then
 * wrong and the next synchronising call returns CAPACITY). In the regular
 * build it returns SLAG_ERR_STATE and changes nothing. Errors: INVALID_ARG
 * for cap < 0. */
slag_status slag_debug_force_pair_capacity(slag_ctx *ctx, int64_t cap);

/* Check of the bounded device waits. Every device-side wait of the library
 * (the mbarrier waits of its tensor-core kernels) gives up after a bound of
 * ~1 s; the kernel then sets the context's error word, the call returns
 * SLAG_ERR_TIMEOUT and the context stays usable. This call runs that path on
 * demand with nothing else in flight: one role waits limit_us microseconds
 * (1 .. 1,000,000) on an mbarrier that nothing completes, and a second role,
 * waiting on another barrier, gives up when the first one aborts. Returns
 * SLAG_ERR_TIMEOUT, or SLAG_OK when `complete` is non-zero (the barrier is
 * completed first and both roles finish normally). Joins the views in flight
 * first. Errors: INVALID_ARG; CUDA. */
slag_status slag_check_wait_timeout(slag_ctx *ctx, int32_t limit_us, int32_t complete);

/* Kernel launches issued by the library so far, over every context and
 * device of the process (a running count; differences give the launches of
 * a region of work). */
uint64_t slag_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* SLAG_H */
