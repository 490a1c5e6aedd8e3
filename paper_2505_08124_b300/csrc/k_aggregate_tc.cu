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

namespace slag {

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
constexpr int kKA = 32;                  // columns per chunk: one 128-byte row of TF32
constexpr int kStagesA = 2;
constexpr int kWPitch = kKA + 1;         // float32 W tile row pitch (conflict-free column atomics)
constexpr int kMaxChunksS = 512;         // chunk boundaries kept in shared memory
constexpr int kMaxColsS = 2048;          // column ids kept in shared memory
constexpr int kTP = 2;                   // triples per thread prefetched for the next chunk
constexpr int kThreadsA = 256;
static_assert(kG == 128, "one MMA of M = 128 per block");
static_assert(kKA * 4 == 128, "a chunk row is one 128-byte swizzle row");

constexpr int kWBytes = kG * kKA * 4;    // 16 KB: A operand (hi or lo)

struct __align__(8) AggCtl {
    uint64_t bar[kStagesA];
    uint32_t tmem_addr;
    uint32_t pad;
};

constexpr size_t kWfBytes = (size_t)kG * kWPitch * 4;
// chunk boundaries + column ids, rounded to 16 bytes (the mbarriers after them need 8-byte alignment)
constexpr size_t kListBytes = (((size_t)(kMaxChunksS + 1) * 4 + (size_t)kMaxColsS * 4) + 15) & ~(size_t)15;

// kNP: output dimensions per pass (TMEM columns, MMA N): 256 when D allows, else 128
template <int kNP>
struct AggShape {
    static constexpr int kEBytes = kNP * kKA * 4;               // B operand (hi or lo)
    static constexpr int kStageBytes = 2 * kWBytes + 2 * kEBytes;
    static constexpr uint32_t kTmemCols = kNP;
    static constexpr uint32_t kIdesc = tc::idesc_tf32<kNP>();
    static constexpr int kF4 = kNP / 32;                        // float4 of E per thread per chunk
    static constexpr size_t smem() { return (size_t)kStagesA * kStageBytes + kWfBytes + kListBytes + sizeof(AggCtl) + 1024; }
    static_assert(((size_t)kStagesA * kStageBytes + kWfBytes + kListBytes) % 8 == 0, "mbarrier alignment");
    static_assert(kF4 * 32 * 8 == kNP * 8, "each warp stages kNP / 8 dimensions");
};

template <int kNP>
__global__ void __launch_bounds__(kThreadsA, 1) aggregate_tc_k(const AggArgs a, uint32_t *err) {
    using Sh = AggShape<kNP>;
    constexpr int kStageBytesA = Sh::kStageBytes;
    constexpr int kEBytes = Sh::kEBytes;
    constexpr uint32_t kTmemColsA = Sh::kTmemCols;
    constexpr uint32_t kIdescA = Sh::kIdesc;
    constexpr int kF4 = Sh::kF4;
    extern __shared__ unsigned char smem_dyn[];
    // 1024-byte alignment for the swizzle atoms
    unsigned char *smem_raw =
        smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    unsigned char *stage0 = smem_raw;
    float *Wf = reinterpret_cast<float *>(smem_raw + kStagesA * kStageBytesA);   // 128 x kWPitch float32
    uint32_t *cbound = reinterpret_cast<uint32_t *>(smem_raw + kStagesA * kStageBytesA + kWfBytes);
    uint32_t *cols = cbound + (kMaxChunksS + 1);
    AggCtl *ctl = reinterpret_cast<AggCtl *>(smem_raw + kStagesA * kStageBytesA + kWfBytes + kListBytes);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t b = blockIdx.x;
    const uint32_t ts = a.bstart[b], te = a.bend[b];
    const bool any = ts < te;
    // unique (block, column) index of triple t = exclusive count + own flag - 1
    const uint32_t u0 = any ? a.uidx[ts] : 0u, u1 = any ? a.uidx[te - 1] + a.flags[te - 1] : 0u;
    const int nchunks = (int)((u1 - u0 + kKA - 1) / kKA);
    const int npass = a.D / kNP;
    const bool cb_smem = nchunks <= kMaxChunksS, col_smem = (u1 - u0) <= (uint32_t)kMaxColsS;

    if (tid == 0) {
        for (int i = 0; i < kStagesA; ++i) mbar_init(&ctl->bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_addr)),
                     "r"(kTmemColsA)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the block's chunk boundaries (first triple of each chunk of 32 columns) and column ids
    if (cb_smem)
        for (int i = tid; i <= nchunks; i += kThreadsA) cbound[i] = i < nchunks ? a.ustart[u0 + (uint32_t)i * kKA] : te;
    if (col_smem)
        for (uint32_t i = tid; i < u1 - u0; i += kThreadsA) cols[i] = a.ucol[u0 + i];
    for (int e = tid; e < kG * kWPitch; e += kThreadsA) Wf[e] = 0.f;
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

    // operands of one chunk, loaded a chunk ahead: 4 float4 of E (lane = column) and the
    // thread's first kTP triples (W tile index, weight)
    float4 ev[kF4];
    int tw_idx[kTP];
    float tw_w[kTP];
    auto prefetch = [&](int c, int d0) {
        const uint32_t uc = u0 + (uint32_t)c * kKA;
        const uint32_t nk = c < nchunks ? min((uint32_t)kKA, u1 - uc) : 0u;
        const float *row = (uint32_t)lane < nk ? a.table + (int64_t)col_of(uc + lane) * a.D + d0 : nullptr;
#pragma unroll
        for (int j = 0; j < kF4; ++j)
            ev[j] = row ? __ldg(reinterpret_cast<const float4 *>(row) + warp * kF4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t t0 = c < nchunks ? chunk_start(c) : te, t1 = c < nchunks ? chunk_start(c + 1) : te;
#pragma unroll
        for (int j = 0; j < kTP; ++j) {
            const uint32_t t = t0 + tid + j * kThreadsA;
            tw_idx[j] = -1;
            tw_w[j] = 0.f;
            if (t < t1) {
                const uint32_t lc = a.uidx[t] + a.flags[t] - 1u - uc;
                tw_idx[j] = (int)(a.keys[t] & 127u) * kWPitch + (int)lc;
                tw_w[j] = a.w[t];
            }
        }
    };

    bool ok = true;
    int64_t gc = 0;   // chunks issued over all passes (stage = gc % kStagesA)
    if (nchunks > 0) prefetch(0, 0);
    for (int pass = 0; pass < npass && ok; ++pass) {
        const int d0 = pass * kNP;
        for (int c = 0; c < nchunks; ++c, ++gc) {
            const int st = (int)(gc % kStagesA);
            unsigned char *W_hi = stage0 + st * kStageBytesA;
            unsigned char *W_lo = W_hi + kWBytes;
            unsigned char *E_hi = W_lo + kWBytes;
            unsigned char *E_lo = E_hi + kEBytes;
            const uint32_t uc = u0 + (uint32_t)c * kKA;
            // the MMAs that last read this stage (chunk gc - kStagesA) must be done
            if (gc >= kStagesA && !mbar_wait(&ctl->bar[st], (uint32_t)((gc - kStagesA) / kStagesA) & 1u)) ok = false;
            if (__syncthreads_or(!ok)) { ok = false; break; }
            // W: the chunk's triples into the float32 tile (beyond the prefetched ones: loaded here)
#pragma unroll
            for (int j = 0; j < kTP; ++j)
                if (tw_idx[j] >= 0) atomicAdd(&Wf[tw_idx[j]], tw_w[j]);
            {
                const uint32_t t0 = chunk_start(c), t1 = chunk_start(c + 1);
                for (uint32_t t = t0 + tid + kTP * kThreadsA; t < t1; t += kThreadsA) {
                    const uint32_t lc = a.uidx[t] + a.flags[t] - 1u - uc;
                    atomicAdd(&Wf[(int)(a.keys[t] & 127u) * kWPitch + (int)lc], a.w[t]);
                }
            }
            // E: the prefetched dimensions d0 + 4 (kF4 warp + j) .. + 3 of column `lane`, transposed
#pragma unroll
            for (int j = 0; j < kF4; ++j) {
                const int d4 = warp * kF4 + j;
                const float vv[4] = {ev[j].x, ev[j].y, ev[j].z, ev[j].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t off = core_off(d4 * 4 + q, lane >> 2) + (uint32_t)(lane & 3) * 4u;
                    const float h = tc::to_tf32(vv[q]);
                    *reinterpret_cast<float *>(E_hi + off) = h;
                    *reinterpret_cast<float *>(E_lo + off) = tc::to_tf32(vv[q] - h);
                }
            }
            // the next chunk's operands (the next pass's first chunk after the last one)
            if (c + 1 < nchunks) prefetch(c + 1, d0);
            else if (pass + 1 < npass) prefetch(0, d0 + kNP);
            __syncthreads();
            // W tile -> A operand; the tile is cleared for the next chunk as it is read
            for (int e = tid; e < kG * (kKA / 4); e += kThreadsA) {
                const int r = e >> 3, kq = e & 7;
                float *src = Wf + r * kWPitch + kq * 4;
                const float4 v = make_float4(src[0], src[1], src[2], src[3]);
                src[0] = src[1] = src[2] = src[3] = 0.f;
                split_store(W_hi, W_lo, core_off(r, kq), v);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t wh = smem_u32(W_hi), wl = smem_u32(W_lo);
                const uint32_t eh = smem_u32(E_hi), el = smem_u32(E_lo);
#pragma unroll
                for (int s2 = 0; s2 < kKA / 8; ++s2) {
                    const uint32_t ko = s2 * 32;   // K = 8 TF32 = 32 bytes along the swizzled row
                    const uint64_t dwh = smem_desc(wh + ko), dwl = smem_desc(wl + ko);
                    const uint64_t deh = smem_desc(eh + ko), del = smem_desc(el + ko);
                    tc::mma_tf32(tmem, dwh, deh, kIdescA, (c > 0 || s2 > 0) ? 1u : 0u);
                    tc::mma_tf32(tmem, dwh, del, kIdescA, 1u);
                    tc::mma_tf32(tmem, dwl, deh, kIdescA, 1u);
                }
                mma_commit(&ctl->bar[st]);
            }
        }
        if (!ok) break;
        // epilogue of the pass: its last commit follows every earlier MMA
        if (nchunks > 0) {
            const int64_t last = gc - 1;
            if (!mbar_wait(&ctl->bar[last % kStagesA], (uint32_t)(last / kStagesA) & 1u)) ok = false;
        }
        if (__syncthreads_or(!ok)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp < 4) {
            float *out = (g < a.n) ? a.E + (int64_t)a.orig_of_int[g] * a.D + d0 : nullptr;
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
            mbar_wait(&ctl->bar[last % kStagesA], (uint32_t)(last / kStagesA) & 1u);
        }
    } else if (tid < kG && g < a.n) {
        const uint32_t o = a.orig_of_int[g];
        const bool nz = S > 0.f && norm2 > 0.f;
        a.inv_norm[o] = nz ? 1.f / sqrtf(norm2) : 0.f;
        a.wsum[o] = S;
    }
    if (ok && warp < 4) {
        const unsigned touched = __ballot_sync(0xffffffffu, tid < kG && g < a.n && S > 0.f);
        if (lane == 0 && touched) atomicAdd(a.touched, (unsigned long long)__popc(touched));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemColsA) : "memory");
    }
}

}  // namespace

void launch_aggregate(const AggArgs &a, int64_t nblocks, uint32_t *err, cudaStream_t st) {
    if (nblocks <= 0) return;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(aggregate_tc_k<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)AggShape<128>::smem());
        cudaFuncSetAttribute(aggregate_tc_k<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)AggShape<256>::smem());
        attr_set = true;
    }
    if (a.D % 256 == 0)
        aggregate_tc_k<256><<<(unsigned)nblocks, kThreadsA, AggShape<256>::smem(), st>>>(a, err);
    else
        aggregate_tc_k<128><<<(unsigned)nblocks, kThreadsA, AggShape<128>::smem(), st>>>(a, err);
    note_launch();
}

}  // namespace slag
