// Cosine top-k on the 5th-generation tensor cores ("Query processing for
// inference": score_k = q . E_k / |E_k|, top-k by descending score, ties to
// the lower Gaussian index).
//
// Float32 accuracy comes from the three-term TF32 split x = hi + lo (hi = x
// rounded to TF32, lo = the rest rounded to TF32): q.e ~ q_hi.e_hi + q_hi.e_lo
// + q_lo.e_hi. Both operands are split once, outside the scoring kernel, into
// two planes (hi, then lo) of rows of D floats: the candidate rows of E once per
// finalize (with their inverse norms, NaN where the row is zero), the queries
// once per batch.
//
// A CTA owns 128 queries (the M = 128 TMEM lanes of a kind::tf32 MMA) and a
// range of Gaussian tiles of N = 256 candidates (256 TMEM columns). Its warps
// have fixed roles:
//   warp 0      one thread issues TMA loads: per K-chunk of 32 values, a 3-D
//               box {32, 128, 2} of the query planes and {32, 256, 2} of the
//               candidate planes, 128-byte swizzled (the canonical K-major
//               layout of the MMA operands), into one of two 96 KB stages;
//   warp 1      owns the TMEM allocation (512 columns: two accumulators) and
//               one thread issues the MMAs: 4 K-steps x 3 products per chunk,
//               freeing the stage by tcgen05.commit and, after a tile's last
//               chunk, signalling the accumulator full;
//   warps 2..5  the epilogue: warp w reads TMEM lanes 32 (w mod 4) .. (one
//               query per thread), 32 columns per tcgen05.ld, scales them by
//               1/|E_k| and keeps a running top-16 in registers; then frees
//               the accumulator for the tile after next.
// So loads, MMAs and the epilogue of the previous tile all overlap. A grid of
// (query tiles x Gaussian splits) writes per-split candidates that the merge
// kernel of k_query.cu reduces to the final top-k.
//
// Every wait on an mbarrier is bounded (about one second of globaltimer) and
// also gives up once another role has given up (a shared abort flag). Before
// the CTA exits, the producer waits for its loads in flight and the MMA
// thread for its MMAs in flight (bounded), then warp 1 releases the TMEM;
// *err is set.
#include <cuda.h>

#include "slag_internal.cuh"
#include "tc_util.cuh"

namespace slag {

namespace {

constexpr int kQM = 128;          // queries per CTA: TMEM lanes of one accumulator
constexpr int kQN = 256;          // candidates per tile: TMEM columns of one accumulator
constexpr int kKC = 32;           // K per stage: one 128-byte swizzle row of TF32
constexpr int kStages = 2;
constexpr int kThreads = 192;     // 6 warps: TMA, MMA, 4 x epilogue
constexpr int kTop = 16;          // running top-k kept per query
constexpr uint32_t kTmemCols = 2 * kQN;

constexpr int kAPlane = kQM * kKC * 4;             // 16 KB: one TF32 plane of the query chunk
constexpr int kBPlane = kQN * kKC * 4;             // 32 KB
constexpr int kStageBytes = 2 * kAPlane + 2 * kBPlane;   // 96 KB
static_assert(kAPlane % 1024 == 0 && kBPlane % 1024 == 0, "swizzle atoms stay 1024-byte aligned");
static_assert(kKC * 4 == 128, "a chunk row is one 128-byte swizzle row");

struct __align__(8) Ctl {
    uint64_t full[kStages];    // TMA -> MMA (transaction bytes)
    uint64_t empty[kStages];   // MMA -> TMA (tcgen05.commit)
    uint64_t tfull[2];         // MMA -> epilogue (tcgen05.commit)
    uint64_t tempty[2];        // epilogue -> MMA (one arrival per epilogue warp)
    uint32_t tmem_addr;
    uint32_t abort;
};

constexpr size_t kSmemBytes = 1024 /* alignment slack */ + (size_t)kStages * kStageBytes + sizeof(Ctl);
static_assert(kSmemBytes <= 232448, "fits the opt-in shared memory of a CTA");

using tc::arrive;
using tc::expect_tx;
using tc::gtimer;
using tc::mbar_init;
using tc::tma_load_3d;
using tc::wait_or_abort;
using tc::mbar_try_wait;
using tc::mma_commit;
using tc::smem_desc;
using tc::smem_u32;
using tc::tmem_ld32;

constexpr uint32_t kIdesc = tc::idesc_tf32<kQN>();

__device__ __forceinline__ bool better(float s, uint32_t i, float s2, uint32_t i2) {
    return s > s2 || (s == s2 && i < i2);
}

// v[j] for a lane-varying j, by a binary tree of selects (no local memory)
__device__ __forceinline__ float select32(const float (&v)[32], int j) {
    float a[16], b[8], c[4], d[2];
#pragma unroll
    for (int t = 0; t < 16; ++t) a[t] = (j & 1) ? v[2 * t + 1] : v[2 * t];
#pragma unroll
    for (int t = 0; t < 8; ++t) b[t] = (j & 2) ? a[2 * t + 1] : a[2 * t];
#pragma unroll
    for (int t = 0; t < 4; ++t) c[t] = (j & 4) ? b[2 * t + 1] : b[2 * t];
#pragma unroll
    for (int t = 0; t < 2; ++t) d[t] = (j & 8) ? c[2 * t + 1] : c[2 * t];
    return (j & 16) ? d[1] : d[0];
}

__global__ void __launch_bounds__(kThreads, 1)
    query_tc_k(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmE, int32_t B,
               const float *__restrict__ qinv, int64_t n, int32_t D, int32_t k, int32_t nsplit,
               float *__restrict__ cand_s, uint32_t *__restrict__ cand_i, uint32_t *err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    Ctl *ctl = reinterpret_cast<Ctl *>(base + kStages * kStageBytes);
    volatile uint32_t *abort = &ctl->abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q0 = blockIdx.x * kQM;
    const int split = blockIdx.y;
    const int64_t ntile = (n + kQN - 1) / kQN;
    const int64_t per = (ntile + nsplit - 1) / nsplit;
    const int64_t t_begin = (int64_t)split * per;
    const int64_t t_end = min(ntile, t_begin + per);
    const int ntl = t_end > t_begin ? (int)(t_end - t_begin) : 0;
    const int nchunk = D / kKC;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&ctl->full[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&ctl->tfull[a], 1);
            mbar_init(&ctl->tempty[a], 4);
        }
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmQ)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmE)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_addr)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = ctl->tmem_addr;

    if (warp == 0) {
        if (lane == 0) {
            // producer: load i goes to stage i % kStages once the MMAs of load i - kStages are done
            int64_t i = 0;
            bool ok = true;
            for (int j = 0; j < ntl && ok; ++j) {
                const int row = (int)((t_begin + j) * kQN);
                for (int c = 0; c < nchunk; ++c, ++i) {
                    const int s = (int)(i % kStages);
                    if (i >= kStages && !wait_or_abort(&ctl->empty[s], (uint32_t)((i / kStages - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    unsigned char *stg = base + s * kStageBytes;
                    expect_tx(&ctl->full[s], (uint32_t)kStageBytes);
                    tma_load_3d(smem_u32(stg), &tmQ, &ctl->full[s], c * kKC, q0, 0);
                    tma_load_3d(smem_u32(stg + 2 * kAPlane), &tmE, &ctl->full[s], c * kKC, row, 0);
                }
            }
            if (ok) {
                // tail: the commits that free the last stages arrive before the CTA exits
                for (int64_t l = i > kStages ? i - kStages : 0; l < i; ++l)
                    if (!wait_or_abort(&ctl->empty[l % kStages], (uint32_t)((l / kStages) & 1), abort)) break;
            } else {
                // loads in flight write this CTA's shared memory: let them land (bounded)
                for (int64_t l = i > kStages ? i - kStages : 0; l < i; ++l) {
                    volatile uint32_t never = 0;
                    wait_or_abort(&ctl->full[l % kStages], (uint32_t)((l / kStages) & 1), &never);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: tile j accumulates into accumulator j & 1
            int64_t i = 0, last = -1;
            bool ok = true;
            for (int j = 0; j < ntl && ok; ++j) {
                const int acc = j & 1;
                if (j >= 2 && !wait_or_abort(&ctl->tempty[acc], (uint32_t)((j / 2 - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dt = tmem + (uint32_t)(acc * kQN);
                for (int c = 0; c < nchunk; ++c, ++i) {
                    const int s = (int)(i % kStages);
                    if (!wait_or_abort(&ctl->full[s], (uint32_t)((i / kStages) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a_hi = smem_u32(base + s * kStageBytes), a_lo = a_hi + kAPlane;
                    const uint32_t b_hi = a_hi + 2 * kAPlane, b_lo = b_hi + kBPlane;
#pragma unroll
                    for (int ks = 0; ks < kKC / 8; ++ks) {
                        const uint32_t ko = ks * 32;   // K = 8 TF32 = 32 bytes along the swizzled row
                        const uint64_t dah = smem_desc(a_hi + ko), dal = smem_desc(a_lo + ko);
                        const uint64_t dbh = smem_desc(b_hi + ko), dbl = smem_desc(b_lo + ko);
                        tc::mma_tf32(dt, dah, dbh, kIdesc, (c > 0 || ks > 0) ? 1u : 0u);
                        tc::mma_tf32(dt, dah, dbl, kIdesc, 1u);
                        tc::mma_tf32(dt, dal, dbh, kIdesc, 1u);
                    }
                    mma_commit(&ctl->empty[s]);
                    last = i;
                }
                if (ok) mma_commit(&ctl->tfull[acc]);
            }
            if (!ok && last >= 0) {
                // MMAs in flight read shared memory and write TMEM: let them finish (bounded)
                volatile uint32_t never = 0;
                wait_or_abort(&ctl->empty[last % kStages], (uint32_t)((last / kStages) & 1), &never);
            }
        }
    } else {
        // epilogue: one query per thread
        const int quarter = warp & 3;
        const int q = q0 + quarter * 32 + lane;
        const int kk = k < kTop ? k : kTop;
        float bs[kTop];
        uint32_t bi[kTop];
#pragma unroll
        for (int p = 0; p < kTop; ++p) {
            bs[p] = -INFINITY;
            bi[p] = 0xffffffffu;
        }
        // Running threshold: the split's k-th best score so far. Columns arrive in increasing
        // candidate index, so a score equal to the k-th best never ranks above it and the test is
        // strict. Rows past the last query take none.
        float thr_run = q < B ? -INFINITY : INFINITY;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        for (int j = 0; j < ntl; ++j) {
            const int acc = j & 1;
            const bool got = wait_or_abort(&ctl->tfull[acc], (uint32_t)((j / 2) & 1), abort);
            if (!__all_sync(0xffffffffu, got)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int64_t g0 = (t_begin + j) * kQN;
            for (int cb = 0; cb < kQN; cb += 32) {
                float v[32];
                tmem_ld32(lane_base + (uint32_t)(acc * kQN + cb), v);
                const int64_t gl = g0 + cb + lane;
                const float inv = __ldg(qinv + gl);   // padded to whole tiles
                uint32_t mask = 0;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    v[jj] *= __shfl_sync(0xffffffffu, inv, jj);   // NaN never passes a threshold
                    mask |= (v[jj] > thr_run ? 1u : 0u) << jj;
                }
                // candidates above the running threshold, one per lane per round, so that the
                // lanes of the warp insert together
                while (__any_sync(0xffffffffu, mask != 0u)) {
                    float sc = -INFINITY;
                    uint32_t gi = 0xffffffffu;
                    if (mask) {
                        const int jj = __ffs(mask) - 1;
                        mask &= mask - 1u;
                        sc = select32(v, jj);
                        gi = (uint32_t)(g0 + cb + jj);
                    }
#pragma unroll
                    for (int p = 0; p < kTop; ++p) {
                        const bool b = better(sc, gi, bs[p], bi[p]);
                        const float ts = b ? bs[p] : sc;
                        const uint32_t ti = b ? bi[p] : gi;
                        bs[p] = b ? sc : bs[p];
                        bi[p] = b ? gi : bi[p];
                        sc = ts;
                        gi = ti;
                    }
                    float kth = bs[0];
#pragma unroll
                    for (int p = 1; p < kTop; ++p) kth = p == kk - 1 ? bs[p] : kth;
                    thr_run = kth;
                }
            }
            // this warp has read the accumulator: it may take the tile after next
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) arrive(&ctl->tempty[acc]);
        }
        if (q < B) {
            float *cs = cand_s + ((int64_t)q * nsplit + split) * kk;
            uint32_t *ci = cand_i + ((int64_t)q * nsplit + split) * kk;
#pragma unroll
            for (int p = 0; p < kTop; ++p)
                if (p < kk) {
                    cs[p] = bs[p];
                    ci[p] = bs[p] == -INFINITY ? 0xffffffffu : bi[p];
                }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *abort) atomicOr(err, 1u);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// The TF32 split of rows (rows[r] of src, or row r without a row list) into two planes of n_pad x D
// floats (hi, then lo); rows n .. n_pad are zero. With qinv, also the rows' inverse norms (NaN
// where not positive, and for the zero rows).
__global__ void __launch_bounds__(256) tf32_split_k(const float *__restrict__ src, const uint32_t *__restrict__ rows,
                                                    int64_t n, int64_t n_pad, int32_t D, float *__restrict__ dst,
                                                    const float *__restrict__ inv_norm, float *__restrict__ qinv) {
    const int64_t d4 = D / 4;
    const int64_t total = n_pad * d4;
    const int64_t plane = n_pad * (int64_t)D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / d4, c = i - r * d4;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
        int64_t sr = -1;
        if (r < n) {
            sr = rows ? (int64_t)__ldg(rows + r) : r;
            const float4 x = __ldg(reinterpret_cast<const float4 *>(src + sr * D) + c);
            h.x = tc::to_tf32(x.x); l.x = tc::to_tf32(x.x - h.x);
            h.y = tc::to_tf32(x.y); l.y = tc::to_tf32(x.y - h.y);
            h.z = tc::to_tf32(x.z); l.z = tc::to_tf32(x.z - h.z);
            h.w = tc::to_tf32(x.w); l.w = tc::to_tf32(x.w - h.w);
        }
        reinterpret_cast<float4 *>(dst + r * D)[c] = h;
        reinterpret_cast<float4 *>(dst + plane + r * D)[c] = l;
        if (qinv && c == 0) {
            const float v = sr >= 0 ? inv_norm[sr] : 0.f;
            qinv[r] = v > 0.f ? v : __int_as_float(0x7fc00000);
        }
    }
}

void launch_split(const float *src, const uint32_t *rows, int64_t n, int64_t n_pad, int32_t D, float *dst,
                  const float *inv_norm, float *qinv, cudaStream_t st) {
    const int64_t total = n_pad * (D / 4);
    if (total <= 0) return;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 148 * 16);
    tf32_split_k<<<(unsigned)blocks, 256, 0, st>>>(src, rows, n, n_pad, D, dst, inv_norm, qinv); note_launch();
}

}  // namespace

bool query_tc_supported(int32_t D, int32_t k) { return k >= 1 && k <= kTop && D % kKC == 0; }

int64_t query_tc_tiles(int64_t n) { return (n + kQN - 1) / kQN; }

int32_t query_tc_splits(int32_t B, int64_t n) {
    const int64_t qt = (B + kQM - 1) / kQM;
    const int64_t nt = (n + kQN - 1) / kQN;
    int64_t s = 148 / qt;
    if (s < 1) s = 1;
    if (s > nt) s = nt;
    return (int32_t)s;
}

void launch_tf32_planes(const float *src, int64_t rows, int64_t rows_pad, int32_t K, float *dst, cudaStream_t st) {
    launch_split(src, nullptr, rows, rows_pad, K, dst, nullptr, nullptr, st);
}

int64_t query_tc_pad_rows(int64_t n) { return (n + kQN - 1) / kQN * kQN; }
int64_t query_tc_pad_queries(int32_t B) { return ((int64_t)B + kQM - 1) / kQM * kQM; }

void launch_query_split_e(const float *E, const float *inv_norm, const uint32_t *rows, int64_t n, int32_t D,
                          float *Ehl, float *qinv, cudaStream_t st) {
    launch_split(E, rows, n, query_tc_pad_rows(n), D, Ehl, inv_norm, qinv, st);
}

cudaError_t launch_query_topk_tc(const float *Q, int32_t B, float *Qhl, const float *Ehl, const float *qinv,
                                 const uint32_t *rows, int64_t n, int32_t D, int32_t k, float *cand_s,
                                 uint32_t *cand_i, int64_t *out_ids, float *out_scores, int32_t *out_count,
                                 uint32_t *err, cudaStream_t st, int32_t splits) {
    {
        const cudaError_t e = set_max_smem((const void *)query_tc_k, (int)kSmemBytes);
        if (e != cudaSuccess) return e;
    }
    const int32_t kk = k < kTop ? k : kTop;
    if (n <= 0) {   // no candidates: every query gets an empty result
        launch_query_merge(cand_s, cand_i, 0, B, k, rows, out_ids, out_scores, out_count, st);
        return cudaGetLastError();
    }
    const int64_t bp = query_tc_pad_queries(B), np = query_tc_pad_rows(n);
    CUtensorMap tq, te;
    if (!tc::encode_planes(&tq, Qhl, bp, D, kQM, 2) || !tc::encode_planes(&te, Ehl, np, D, kQN, 2))
        return cudaErrorInvalidValue;
    launch_split(Q, nullptr, B, bp, D, Qhl, nullptr, nullptr, st);
    int32_t nsplit = splits > 0 ? splits : query_tc_splits(B, n);
    const int64_t ntiles = np / kQN;
    if (nsplit > ntiles) nsplit = (int32_t)ntiles;
    dim3 grid((unsigned)(bp / kQM), (unsigned)nsplit);
    query_tc_k<<<grid, kThreads, kSmemBytes, st>>>(tq, te, B, qinv, n, D, k, nsplit, cand_s, cand_i, err); note_launch();
    launch_query_merge(cand_s, cand_i, (int64_t)nsplit * kk, B, k, rows, out_ids, out_scores, out_count, st);
    return cudaGetLastError();
}

}  // namespace slag
