// Cosine top-k on the 5th-generation tensor cores ("Query processing for
// inference": score_k = q . E_k / |E_k|, top-k by descending score, ties to
// the lower Gaussian index).
//
// A CTA scores 256 queries x 128 Gaussians per tile as two tcgen05.mma
// accumulators of M = 128 TMEM lanes (queries) x N = 128 TMEM columns
// (Gaussians), fp32, over K = D in chunks of 32. Float32 accuracy comes from
// the three-term TF32 split x = hi + lo (hi = x rounded to TF32, lo = the
// rest rounded to TF32): q.e ~ q_hi.e_hi + q_hi.e_lo + q_lo.e_hi, so each
// chunk issues 2 accumulators x 4 K-steps x 3 MMAs of K = 8. The CTA's 512
// threads stage operands into shared memory in the 128-byte-swizzled K-major
// layout (atoms of 8 rows x 128 bytes = 32 TF32 values per row, the 16-byte
// chunk c of row r stored at chunk c ^ (r mod 8), atoms 1024 bytes apart; a
// K-step of 8 advances the descriptor start by 32 bytes), two stages deep
// against the MMAs (mbarriers), with the next chunk's global loads in flight
// while the current one is converted. After a tile's last chunk, the first 8
// warps read one query's 128 scores each from TMEM (tcgen05.ld 32x32b),
// scale them by 1/|E_k| and keep a running top-16 in registers. A grid of
// (query tiles x Gaussian splits) writes per-split candidates that the merge
// kernel of k_query.cu reduces to the final top-k.
//
// Every wait on an mbarrier is bounded (about one second of globaltimer);
// on timeout the kernel sets *err, stops issuing work and releases its TMEM.
#include "slag_internal.cuh"
#include "tc_util.cuh"

namespace slag {

namespace {

constexpr int kM = 256;          // queries per CTA tile: two accumulators of 128 TMEM lanes
constexpr int kMmaM = 128;       // M of one MMA (TMEM lanes of one accumulator)
constexpr int kN = 128;          // Gaussians per tile (TMEM columns of one accumulator)
constexpr int kKC = 32;          // K per staged chunk: one 128-byte swizzle atom row of TF32
constexpr int kStages = 2;
constexpr int kThreadsTC = 512;
constexpr int kTopTC = 16;       // running top-k kept per query
constexpr uint32_t kTmemCols = 256;

// byte sizes of one stage
constexpr int kABytes = kM * kKC * 4;   // 32 KB
constexpr int kBBytes = kN * kKC * 4;   // 16 KB
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
constexpr int kSBO = tc::kSBO;          // bytes between 8-row swizzle atoms
constexpr int kLoadsPerThread = (kM + kN) * (kKC / 4) / kThreadsTC;   // float4 per thread per chunk

struct __align__(8) TcCtl {
    uint64_t bar[kStages];
    uint32_t tmem_addr;
    uint32_t abort;
};

using tc::core_off;
using tc::gtimer;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_commit;
using tc::smem_desc;
using tc::smem_u32;
using tc::split_store;
using tc::tmem_ld32;

constexpr uint32_t kIdesc = tc::idesc_tf32<kN>();
static_assert(kMmaM == 128, "cta_group::1 tf32 MMA shape");
static_assert(kKC * 4 == 128, "a chunk row is one 128-byte swizzle row");

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    tc::mma_tf32(tmem, adesc, bdesc, kIdesc, accum);
}

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

__global__ void __launch_bounds__(kThreadsTC, 1) query_tc_k(const float *__restrict__ Q, int32_t B,
                                                            const float *__restrict__ E,
                                                            const float *__restrict__ inv_norm,
                                                            const uint32_t *__restrict__ rows, int64_t n,
                                                            int32_t D, int32_t k, int32_t nsplit,
                                                            float *__restrict__ cand_s,
                                                            uint32_t *__restrict__ cand_i, uint32_t *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *stage0 = smem_raw;
    TcCtl *ctl = reinterpret_cast<TcCtl *>(smem_raw + kStages * kStageBytes);
    float *sinv = reinterpret_cast<float *>(smem_raw + kStages * kStageBytes + 64);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = blockIdx.x * kM;
    const int split = blockIdx.y;
    const int64_t ntile_g = (n + kN - 1) / kN;
    const int64_t per = (ntile_g + nsplit - 1) / nsplit;
    const int64_t t_begin = split * per;
    const int64_t t_end = min(ntile_g, t_begin + per);
    const int nchunk = D / kKC;
    const int64_t total_chunks = t_end > t_begin ? (t_end - t_begin) * nchunk : 0;

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&ctl->bar[i], 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_addr)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = ctl->tmem_addr;

    float bs[kTopTC];
    uint32_t bi[kTopTC];
#pragma unroll
    for (int i = 0; i < kTopTC; ++i) {
        bs[i] = -INFINITY;
        bi[i] = 0xffffffffu;
    }
    // Running threshold: the split's k-th best score so far. Columns arrive in
    // increasing Gaussian index, so a score equal to the k-th best never ranks
    // above it and the test is strict. Rows past the last query take none.
    const int kk = k < kTopTC ? k : kTopTC;
    float thr_run = -INFINITY;
    if (warp < 8 && q0 + (warp >> 2) * 128 + (warp & 3) * 32 + lane >= B) thr_run = INFINITY;

    // this thread's share of a chunk: kLoadsPerThread float4, A rows first then B rows
    auto fetch = [&](int64_t gc, float4 (&v)[kLoadsPerThread]) {
        const int64_t t = t_begin + gc / nchunk;
        const int d0 = (int)(gc % nchunk) * kKC;
        const int64_t g0 = t * kN;
#pragma unroll
        for (int j = 0; j < kLoadsPerThread; ++j) {
            const int i = tid + j * kThreadsTC;          // 0 .. (kM + kN) * 8
            const int row = i >> 3, kq = i & 7;
            v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < kM) {
                if (q0 + row < B) v[j] = __ldg(reinterpret_cast<const float4 *>(Q + (int64_t)(q0 + row) * D + d0 + kq * 4));
            } else {
                const int64_t g = g0 + (row - kM);
                if (g < n) {
                    const int64_t er = rows ? (int64_t)__ldg(rows + g) : g;
                    v[j] = __ldg(reinterpret_cast<const float4 *>(E + er * D + d0 + kq * 4));
                }
            }
        }
    };

    float4 pf[kLoadsPerThread];
    if (total_chunks > 0) fetch(0, pf);
    bool ok = true;
    int64_t gc = 0;
    for (; gc < total_chunks; ++gc) {
        const int st = (int)(gc % kStages);
        unsigned char *A_hi = stage0 + st * kStageBytes;
        unsigned char *A_lo = A_hi + kABytes;
        unsigned char *B_hi = A_lo + kABytes;
        unsigned char *B_lo = B_hi + kBBytes;
        const int c = (int)(gc % nchunk);
        // the MMAs that last read this stage (chunk gc - kStages) must be done
        if (gc >= kStages) {
            if (!mbar_wait(&ctl->bar[st], (uint32_t)((gc - kStages) / kStages) & 1u)) ok = false;
        }
        if (__syncthreads_or(!ok)) { ok = false; break; }
#pragma unroll
        for (int j = 0; j < kLoadsPerThread; ++j) {
            const int i = tid + j * kThreadsTC;
            const int row = i >> 3, kq = i & 7;
            if (row < kM) split_store(A_hi, A_lo, core_off(row, kq), pf[j]);
            else split_store(B_hi, B_lo, core_off(row - kM, kq), pf[j]);
        }
        if (gc + 1 < total_chunks) fetch(gc + 1, pf);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(A_hi), a_lo = smem_u32(A_lo);
            const uint32_t b_hi = smem_u32(B_hi), b_lo = smem_u32(B_lo);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t ah = a_hi + h * 16 * kSBO, al = a_lo + h * 16 * kSBO;   // rows 128h..
                const uint32_t dt = tmem + (uint32_t)(h * kN);                         // columns 128h..
#pragma unroll
                for (int s2 = 0; s2 < kKC / 8; ++s2) {
                    const uint32_t ko = s2 * 32;    // K = 8 TF32 = 32 bytes along the swizzled row
                    const uint64_t dah = smem_desc(ah + ko), dal = smem_desc(al + ko);
                    const uint64_t dbh = smem_desc(b_hi + ko), dbl = smem_desc(b_lo + ko);
                    mma_tf32(dt, dah, dbh, (c > 0 || s2 > 0) ? 1u : 0u);
                    mma_tf32(dt, dah, dbl, 1u);
                    mma_tf32(dt, dal, dbh, 1u);
                }
            }
            mma_commit(&ctl->bar[st]);
        }
        if (c != nchunk - 1) continue;
        // epilogue of the tile: its last commit follows every earlier MMA
        if (!mbar_wait(&ctl->bar[st], (uint32_t)(gc / kStages) & 1u)) ok = false;
        if (__syncthreads_or(!ok)) { ok = false; ++gc; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int64_t g0 = (t_begin + gc / nchunk) * kN;
        for (int i = tid; i < kN; i += kThreadsTC) {
            const int64_t g = g0 + i;
            const float inv = g < n ? inv_norm[rows ? (int64_t)rows[g] : g] : 0.f;
            sinv[i] = inv > 0.f ? inv : __int_as_float(0x7fc00000);   // NaN: never passes a threshold
        }
        __syncthreads();
        if (warp < 8) {
            // warp w: accumulator w / 4, TMEM lanes 32 (w % 4) ..
            const uint32_t base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * kN);
            for (int cb = 0; cb < kN; cb += 32) {
                float v[32];
                tmem_ld32(base + (uint32_t)cb, v);
                uint32_t mask = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    v[j] *= sinv[cb + j];
                    mask |= (v[j] > thr_run ? 1u : 0u) << j;
                }
                // candidates at or above the running threshold, one per lane per round, so that
                // the lanes of the warp insert together
                while (__any_sync(0xffffffffu, mask != 0u)) {
                    float sc = -INFINITY;
                    uint32_t gi = 0xffffffffu;
                    if (mask) {
                        const int j = __ffs(mask) - 1;
                        mask &= mask - 1u;
                        sc = select32(v, j);
                        gi = (uint32_t)(g0 + cb + j);
                    }
#pragma unroll
                    for (int p = 0; p < kTopTC; ++p) {
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
                    for (int p = 1; p < kTopTC; ++p) kth = p == kk - 1 ? bs[p] : kth;
                    thr_run = kth;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // every thread has read the accumulators before the next tile overwrites them
    }

    if (!ok) {
        if (tid == 0) atomicOr(err, 1u);
        // let MMAs in flight finish (bounded) before TMEM is released
        if (gc > 0) {
            const int64_t last = gc - 1;
            mbar_wait(&ctl->bar[last % kStages], (uint32_t)(last / kStages) & 1u);
        }
    }
    // this query's candidates of this split
    if (warp < 8) {
        const int q = q0 + (warp >> 2) * 128 + (warp & 3) * 32 + lane;
        if (q < B) {
            float *cs = cand_s + ((int64_t)q * nsplit + split) * kk;
            uint32_t *ci = cand_i + ((int64_t)q * nsplit + split) * kk;
#pragma unroll
            for (int p = 0; p < kTopTC; ++p)
                if (p < kk) {
                    cs[p] = bs[p];
                    ci[p] = bs[p] == -INFINITY ? 0xffffffffu : bi[p];
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

size_t tc_smem() { return (size_t)kStages * kStageBytes + 64 + kN * 4; }

}  // namespace

bool query_tc_supported(int32_t D, int32_t k) { return k >= 1 && k <= kTopTC && D % kKC == 0; }

int64_t query_tc_tiles(int64_t n) { return (n + kN - 1) / kN; }

int32_t query_tc_splits(int32_t B, int64_t n) {
    const int64_t qt = (B + kM - 1) / kM;
    const int64_t nt = (n + kN - 1) / kN;
    int64_t s = 148 / qt;
    if (s < 1) s = 1;
    if (s > nt) s = nt;
    return (int32_t)s;
}

void launch_query_topk_tc(const float *Q, int32_t B, const float *E, const float *inv_norm, const uint32_t *rows,
                          int64_t n, int32_t D, int32_t k, float *cand_s, uint32_t *cand_i, int64_t *out_ids,
                          float *out_scores, int32_t *out_count, uint32_t *err, cudaStream_t st, int32_t splits) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(query_tc_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem());
        attr_set = true;
    }
    const int32_t kk = k < kTopTC ? k : kTopTC;
    if (n <= 0) {   // no candidates: every query gets an empty result
        launch_query_merge(cand_s, cand_i, 0, B, k, rows, out_ids, out_scores, out_count, st);
        return;
    }
    int32_t nsplit = splits > 0 ? splits : query_tc_splits(B, n);
    const int64_t ntiles = (n + kN - 1) / kN;
    if (nsplit > ntiles) nsplit = (int32_t)ntiles;
    dim3 grid((unsigned)((B + kM - 1) / kM), (unsigned)nsplit);
    query_tc_k<<<grid, kThreadsTC, tc_smem(), st>>>(Q, B, E, inv_norm, rows, n, D, k, nsplit, cand_s, cand_i, err); note_launch();
    launch_query_merge(cand_s, cand_i, (int64_t)nsplit * kk, B, k, rows, out_ids, out_scores, out_count, st);
}

}  // namespace slag
