// Aggregation on the 5th-generation tensor cores (Method, "Semantic
// Embedding", Aggregation: E_k = sum_{views, segments} B[k][j] E_j / sum w).
//
// After the log sort, each block of 128 spatially adjacent Gaussians (Morton
// order) has its triples grouped by column (view, segment). Its numerator is
// the contraction W_block (128 x K_b) x E_cols (K_b x D), where W_block holds
// the block's weights on its K_b distinct columns and E_cols their segment
// embeddings. One CTA per block computes it with tcgen05.mma kind::tf32 into
// a TMEM accumulator of M = 128 lanes (Gaussians) x N = 256 columns (output
// dimensions; 128 when D is not a multiple of 256), one pass per N dimensions
// of D, K = the block's columns in chunks of 32. Float32 accuracy comes from the three-term TF32 split
// (hi*hi + hi*lo + lo*hi). Per chunk, the CTA:
//   * accumulates the chunk's triples into a float32 128 x 32 tile with
//     shared-memory atomics (a (Gaussian, column) pair may repeat), then
//     splits it into the A operand (rows = Gaussians, 128-byte swizzled);
//   * stages the B operand transposed: lane j of a warp loads 4 dimensions of
//     column j and stores them into 4 rows (dimensions) at K position j, so a
//     warp's 32 stores fill one 128-byte row without bank conflicts;
//   * issues 4 K-steps x 3 MMAs from one thread and commits to the stage's
//     mbarrier; two stages keep staging ahead of the tensor core.
// The next chunk's E values and first triples are loaded into registers while
// the current chunk is stored, and the block's chunk boundaries and column ids
// are read into shared memory once, so the loads' latency overlaps the work.
// After a pass, warps 0-3 read their Gaussians' rows from TMEM, divide by
// sum w, accumulate the squared norm and write the row in the caller's order.
//
// Every mbarrier wait is bounded (about one second of globaltimer); on
// timeout the kernel sets *err, stops issuing MMAs, waits (bounded) for those
// in flight and releases its TMEM.
#include "slag_internal.cuh"
#include "tc_util.cuh"

#include <cuda_bf16.h>

namespace slag {

SLAG_CHECKS_WORD


namespace {

using tc::core_off;
using tc::mbar_init;
using tc::mbar_wait;
using tc::mma_commit;
using tc::smem_desc;
using tc::smem_u32;
using tc::split_store;
using tc::tmem_ld32;

constexpr int kG = kBlockG;              // Gaussians per block = TMEM lanes
constexpr int kMaxChunksS = 512;         // chunk boundaries kept in shared memory
constexpr int kMaxColsS = 2048;          // column ids kept in shared memory
constexpr int kTP = 2;                   // triples per thread prefetched for the next chunk
constexpr int kThreadsA = 256;
constexpr int kWBytes = kG * 128;        // A operand: 128 rows of 128 bytes
static_assert(kG == 128, "one MMA of M = 128 per block");

struct __align__(8) AggCtl {
    uint64_t bar[4];
    uint32_t tmem_addr;
    uint32_t pad;
};

// chunk boundaries + column ids, rounded to 16 bytes (the mbarriers after them need 8-byte alignment)
constexpr size_t kListBytes = (((size_t)(kMaxChunksS + 1) * 4 + (size_t)kMaxColsS * 4) + 15) & ~(size_t)15;

// kNP: output dimensions per pass (TMEM columns, MMA N). kBF: BF16 operands (kind::f16,
// 64 columns per chunk, one MMA per K-step of 16) instead of the 3xTF32 split (32 columns
// per chunk, three MMAs per K-step of 8). A chunk row is one 128-byte swizzle row either way.
template <int kNP, bool kBF>
struct AggShape {
    static constexpr int kKA = kBF ? 64 : 32;                   // columns per chunk
    static constexpr int kPitch = kKA + 1;                      // float32 W tile pitch (conflict-free)
    static constexpr int kStages = kBF ? 3 : 2;
    static constexpr int kEBytes = kNP * 128;                   // B operand: kNP rows of 128 bytes
    static constexpr int kCopies = kBF ? 1 : 2;                 // hi and lo for the TF32 split
    static constexpr int kStageBytes = kCopies * (kWBytes + kEBytes);
    static constexpr size_t kWfBytes = (size_t)kG * kPitch * 4;
    static constexpr uint32_t kIdesc = kBF ? tc::idesc_bf16<kNP>() : tc::idesc_tf32<kNP>();
    static constexpr int kF4 = kNP / 32;                        // float4 of one column per thread per chunk
    static constexpr int kCols = kBF ? 2 : 1;                   // columns staged per lane
    static constexpr size_t smem() { return (size_t)kStages * kStageBytes + kWfBytes + kListBytes + sizeof(AggCtl) + 1024; }
    static_assert(((size_t)kStages * kStageBytes + kWfBytes + kListBytes) % 8 == 0, "mbarrier alignment");
    static_assert(32 * kCols == kKA, "a warp stages one chunk's columns");
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x (lower address) = lo
    return *reinterpret_cast<const uint32_t *>(&v);
}

template <int kNP, bool kBF>
__global__ void __launch_bounds__(kThreadsA, 1) aggregate_tc_k(const AggArgs a, uint32_t *err) {
    using Sh = AggShape<kNP, kBF>;
    constexpr int kKA = Sh::kKA, kPitch = Sh::kPitch, kStages = Sh::kStages;
    constexpr int kStageBytes = Sh::kStageBytes, kEBytes = Sh::kEBytes;
    constexpr uint32_t kIdesc = Sh::kIdesc;
    constexpr int kF4 = Sh::kF4, kCols = Sh::kCols;
    extern __shared__ unsigned char smem_dyn[];
    // 1024-byte alignment for the swizzle atoms
    unsigned char *smem_raw =
        smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    unsigned char *stage0 = smem_raw;
    float *Wf = reinterpret_cast<float *>(smem_raw + kStages * kStageBytes);   // 128 x kPitch float32
    uint32_t *cbound = reinterpret_cast<uint32_t *>(smem_raw + kStages * kStageBytes + Sh::kWfBytes);
    uint32_t *cols = cbound + (kMaxChunksS + 1);
    AggCtl *ctl = reinterpret_cast<AggCtl *>(smem_raw + kStages * kStageBytes + Sh::kWfBytes + kListBytes);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t b = a.block0 + blockIdx.x;
    const uint32_t ts = a.bstart[b], te = a.bend[b];
    const bool any = ts < te;
    // unique (block, column) index of triple t = exclusive count + own flag - 1
    const uint32_t u0 = any ? a.uidx[ts] : 0u, u1 = any ? a.uidx[te - 1] + a.flags[te - 1] : 0u;
    const int nchunks = (int)((u1 - u0 + kKA - 1) / kKA);
    const int npass = a.D / kNP;
    const bool cb_smem = nchunks <= kMaxChunksS, col_smem = (u1 - u0) <= (uint32_t)kMaxColsS;

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&ctl->bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_addr)),
                     "r"((uint32_t)kNP)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the block's chunk boundaries (first triple of each chunk of kKA columns) and column ids
    if (cb_smem)
        for (int i = tid; i <= nchunks; i += kThreadsA) cbound[i] = i < nchunks ? a.ustart[u0 + (uint32_t)i * kKA] : te;
    if (col_smem)
        for (uint32_t i = tid; i < u1 - u0; i += kThreadsA) cols[i] = a.ucol[u0 + i];
    for (int e = tid; e < kG * kPitch; e += kThreadsA) Wf[e] = 0.f;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = ctl->tmem_addr;
    auto chunk_start = [&](int c) -> uint32_t {
        return c >= nchunks ? te : (cb_smem ? cbound[c] : a.ustart[u0 + (uint32_t)c * kKA]);
    };
    auto col_of = [&](uint32_t u) -> uint32_t { return col_smem ? cols[u - u0] : a.ucol[u]; };

    // epilogue threads 0..127: Gaussian g = b * 128 + tid, TMEM lane tid
    const int64_t g = b * kG + (tid & (kG - 1));
    float S = 0.f, norm2 = 0.f;
    if (tid < kG && g < a.n) S = (a.s_hi[g] + a.s_lo[g]) + a.s_ovf[g];
    const float invS = S > 0.f ? 1.f / S : 0.f;

    // operands of one chunk, loaded a chunk ahead: kF4 float4 of E of each of the lane's kCols
    // columns (column kCols lane + i) and the thread's first kTP triples (W tile index, weight)
    float4 ev[kCols][kF4];
    int tw_idx[kTP];
    float tw_w[kTP];
    auto prefetch = [&](int c, int d0) {
        const uint32_t uc = u0 + (uint32_t)c * kKA;
        const uint32_t nk = c < nchunks ? min((uint32_t)kKA, u1 - uc) : 0u;
#pragma unroll
        for (int i = 0; i < kCols; ++i) {
            const uint32_t lc = (uint32_t)(lane * kCols + i);
            const float *row = lc < nk && SLAG_IN_BOUNDS((int64_t)col_of(uc + lc) < a.columns, kCheckAggregate)
                                   ? a.table + (int64_t)col_of(uc + lc) * a.D + d0
                                   : nullptr;
#pragma unroll
            for (int j = 0; j < kF4; ++j)
                ev[i][j] = row ? __ldg(reinterpret_cast<const float4 *>(row) + warp * kF4 + j)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const uint32_t t0 = c < nchunks ? chunk_start(c) : te, t1 = c < nchunks ? chunk_start(c + 1) : te;
#pragma unroll
        for (int j = 0; j < kTP; ++j) {
            const uint32_t t = t0 + tid + j * kThreadsA;
            tw_idx[j] = -1;
            tw_w[j] = 0.f;
            if (t < t1) {
                const uint32_t lc = a.uidx[t] + a.flags[t] - 1u - uc;
                if (SLAG_IN_BOUNDS(lc < (uint32_t)kKA, kCheckAggregate)) {
                    tw_idx[j] = (int)(a.keys[t] & 127u) * kPitch + (int)lc;
                    tw_w[j] = a.w[t];
                }
            }
        }
    };

    bool ok = true;
    int64_t gc = 0;   // chunks issued over all passes (stage = gc % kStages)
    if (nchunks > 0) prefetch(0, 0);
    for (int pass = 0; pass < npass && ok; ++pass) {
        const int d0 = pass * kNP;
        for (int c = 0; c < nchunks; ++c, ++gc) {
            const int st = (int)(gc % kStages);
            unsigned char *W0 = stage0 + st * kStageBytes;   // A (hi)
            unsigned char *W1 = W0 + kWBytes;                // A lo (TF32 split)
            unsigned char *E0 = W0 + Sh::kCopies * kWBytes;  // B (hi)
            unsigned char *E1 = E0 + kEBytes;                // B lo (TF32 split)
            const uint32_t uc = u0 + (uint32_t)c * kKA;
            // the MMAs that last read this stage (chunk gc - kStages) must be done
            if (gc >= kStages && !mbar_wait(&ctl->bar[st], (uint32_t)((gc - kStages) / kStages) & 1u)) ok = false;
            if (__syncthreads_or(!ok)) { ok = false; break; }
            // W: the chunk's triples into the float32 tile (beyond the prefetched ones: loaded here)
#pragma unroll
            for (int j = 0; j < kTP; ++j)
                if (tw_idx[j] >= 0) atomicAdd(&Wf[tw_idx[j]], tw_w[j]);
            {
                const uint32_t t0 = chunk_start(c), t1 = chunk_start(c + 1);
                for (uint32_t t = t0 + tid + kTP * kThreadsA; t < t1; t += kThreadsA) {
                    const uint32_t lc = a.uidx[t] + a.flags[t] - 1u - uc;
                    if (!SLAG_IN_BOUNDS(lc < (uint32_t)kKA, kCheckAggregate)) continue;
                    atomicAdd(&Wf[(int)(a.keys[t] & 127u) * kPitch + (int)lc], a.w[t]);
                }
            }
            // E, transposed: dimensions d0 + 4 (kF4 warp + j) .. + 3 of the lane's columns go to
            // rows (dimensions) of the B operand at the columns' K positions
#pragma unroll
            for (int j = 0; j < kF4; ++j) {
                const int d4 = warp * kF4 + j;
                if constexpr (kBF) {
                    const float v0[4] = {ev[0][j].x, ev[0][j].y, ev[0][j].z, ev[0][j].w};
                    const float v1[4] = {ev[1][j].x, ev[1][j].y, ev[1][j].z, ev[1][j].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        // K positions 2 lane, 2 lane + 1: 4 bytes at byte 4 lane of the 128-byte row
                        const uint32_t off = core_off(d4 * 4 + q, lane >> 2) + (uint32_t)(lane & 3) * 4u;
                        *reinterpret_cast<uint32_t *>(E0 + off) = pack_bf16(v0[q], v1[q]);
                    }
                } else {
                    const float vv[4] = {ev[0][j].x, ev[0][j].y, ev[0][j].z, ev[0][j].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t off = core_off(d4 * 4 + q, lane >> 2) + (uint32_t)(lane & 3) * 4u;
                        const float h = tc::to_tf32(vv[q]);
                        *reinterpret_cast<float *>(E0 + off) = h;
                        *reinterpret_cast<float *>(E1 + off) = tc::to_tf32(vv[q] - h);
                    }
                }
            }
            // the next chunk's operands (the next pass's first chunk after the last one)
            if (c + 1 < nchunks) prefetch(c + 1, d0);
            else if (pass + 1 < npass) prefetch(0, d0 + kNP);
            __syncthreads();
            // W tile -> A operand (16-byte chunks of a 128-byte row); the tile is cleared for the
            // next chunk as it is read
            for (int e = tid; e < kG * 8; e += kThreadsA) {
                const int r = e >> 3, kq = e & 7;
                if constexpr (kBF) {
                    float *src = Wf + r * kPitch + kq * 8;
                    uint4 v;
                    v.x = pack_bf16(src[0], src[1]);
                    v.y = pack_bf16(src[2], src[3]);
                    v.z = pack_bf16(src[4], src[5]);
                    v.w = pack_bf16(src[6], src[7]);
#pragma unroll
                    for (int i = 0; i < 8; ++i) src[i] = 0.f;
                    *reinterpret_cast<uint4 *>(W0 + core_off(r, kq)) = v;
                } else {
                    float *src = Wf + r * kPitch + kq * 4;
                    const float4 v = make_float4(src[0], src[1], src[2], src[3]);
                    src[0] = src[1] = src[2] = src[3] = 0.f;
                    split_store(W0, W1, core_off(r, kq), v);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t w0 = smem_u32(W0), w1 = smem_u32(W1);
                const uint32_t e0 = smem_u32(E0), e1 = smem_u32(E1);
#pragma unroll
                for (int s2 = 0; s2 < 4; ++s2) {
                    const uint32_t ko = s2 * 32;   // one K-step = 32 bytes along the swizzled row
                    const uint32_t acc = (c > 0 || s2 > 0) ? 1u : 0u;
                    if constexpr (kBF) {
                        tc::mma_bf16(tmem, smem_desc(w0 + ko), smem_desc(e0 + ko), kIdesc, acc);
                    } else {
                        const uint64_t dwh = smem_desc(w0 + ko), dwl = smem_desc(w1 + ko);
                        const uint64_t deh = smem_desc(e0 + ko), del = smem_desc(e1 + ko);
                        tc::mma_tf32(tmem, dwh, deh, kIdesc, acc);
                        tc::mma_tf32(tmem, dwh, del, kIdesc, 1u);
                        tc::mma_tf32(tmem, dwl, deh, kIdesc, 1u);
                    }
                }
                mma_commit(&ctl->bar[st]);
            }
        }
        if (!ok) break;
        // epilogue of the pass: its last commit follows every earlier MMA
        if (nchunks > 0) {
            const int64_t last = gc - 1;
            if (!mbar_wait(&ctl->bar[last % kStages], (uint32_t)(last / kStages) & 1u)) ok = false;
        }
        if (__syncthreads_or(!ok)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp < 4) {
            float *out = a.E_chunk ? a.E_chunk + ((int64_t)blockIdx.x * kG + tid) * a.D + d0
                                   : ((g < a.n) ? a.E + (int64_t)a.orig_of_int[g] * a.D + d0 : nullptr);
            const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16);
            for (int cb = 0; cb < kNP; cb += 32) {
                float v[32];
                if (nchunks > 0) {
                    tmem_ld32(base + (uint32_t)cb, v);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0.f;
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    v[j] *= invS;
                    norm2 = fmaf(v[j], v[j], norm2);
                }
                if (out) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *reinterpret_cast<float4 *>(out + cb + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // the accumulator is read before the next pass overwrites it
    }

    if (!ok) {
        if (tid == 0) atomicOr(err, 1u);
        // let MMAs in flight finish (bounded) before TMEM is released
        if (gc > 0) {
            const int64_t last = gc - 1;
            mbar_wait(&ctl->bar[last % kStages], (uint32_t)(last / kStages) & 1u);
        }
    } else if (tid < kG) {
        const uint32_t o = g < a.n ? a.orig_of_int[g] : 0xffffffffu;
        if (g < a.n) {
            const bool nz = S > 0.f && norm2 > 0.f;
            a.inv_norm[o] = nz ? 1.f / sqrtf(norm2) : 0.f;
            a.wsum[o] = S;
        }
        if (a.E_chunk) {
            a.ids_chunk[(int64_t)blockIdx.x * kG + tid] = o;
            a.wsum_chunk[(int64_t)blockIdx.x * kG + tid] = S;
        }
    }
    if (ok && warp < 4) {
        const unsigned touched = __ballot_sync(0xffffffffu, tid < kG && g < a.n && S > 0.f);
        if (lane == 0 && touched) atomicAdd(a.touched, (unsigned long long)__popc(touched));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kNP) : "memory");
    }
}

template <int kNP, bool kBF>
void launch_one(const AggArgs &a, int64_t nblocks, uint32_t *err, cudaStream_t st) {
    // on failure the error stays recorded for the caller's cudaGetLastError check
    if (set_max_smem((const void *)aggregate_tc_k<kNP, kBF>, (int)AggShape<kNP, kBF>::smem()) != cudaSuccess) return;
    aggregate_tc_k<kNP, kBF><<<(unsigned)nblocks, kThreadsA, AggShape<kNP, kBF>::smem(), st>>>(a, err);
}

}  // namespace

void launch_aggregate(const AggArgs &a, int64_t nblocks, uint32_t *err, cudaStream_t st) {
    if (nblocks <= 0) return;
    if (a.bf16)
        launch_one<128, true>(a, nblocks, err, st);
    else if (a.D % 256 == 0)
        launch_one<256, false>(a, nblocks, err, st);
    else
        launch_one<128, false>(a, nblocks, err, st);
    note_launch();
}

SLAG_CHECKS_TAKE(checks_take_aggregate)

}  // namespace slag
