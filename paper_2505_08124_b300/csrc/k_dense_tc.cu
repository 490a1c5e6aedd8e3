// Dense layers on the 5th-generation tensor cores: C = act(A W + b), for the
// decoder of the learned latent form (32 -> 256 -> D, erf-GELU after the hidden
// layer; bfloat16-rounded weights, float32 activations and accumulation).
//
// A (rows x K) arrives as its TF32 hi/lo planes (hi = x rounded to TF32, lo =
// the rest rounded to TF32); the weights arrive transposed (N x K) and rounded
// to bfloat16, which TF32 holds exactly, as one plane. Each product is then
// A_hi W + A_lo W, float32-accurate to about 2^-21 of its magnitude.
//
// The output is cut into tiles of 128 x NT (NT = 256, or 128 when N is not a
// multiple of 256; M = 128 TMEM lanes, NT TMEM columns). A persistent grid of at
// most one CTA per SM walks the tiles; a CTA's warps have fixed roles:
//   warp 0      one thread issues TMA loads of K-chunks of 32 values: a 3-D
//               box {32, 128, 2} of A's planes and {32, NT, 1} of the weights,
//               128-byte swizzled, into one of three stages;
//   warp 1      owns the TMEM allocation (two accumulators of NT columns); one
//               thread issues 4 K-steps x 2 MMAs per chunk, freeing the stage
//               by tcgen05.commit, and tile j accumulates into accumulator j & 1;
//   warps 2..9  the epilogue, two warps per TMEM lane quarter (one row per
//               thread), each on half of the tile's columns, 32 per tcgen05.ld:
//               kGeluPlanes: h = gelu(acc + b), written as the TF32 hi/lo
//                            planes of the next layer's input, or
//               kBiasRows:   acc + b, written as float32 rows;
//               then the accumulator is freed for the tile after next.
// So one tile's epilogue overlaps the next tile's loads and MMAs.
// Every wait on an mbarrier is bounded (about one second of globaltimer) and
// gives up once another role has given up; the producer and the MMA thread
// then wait (bounded) for their operations in flight, TMEM is released and
// *err is set.
#include "slag_internal.cuh"
#include "tc_util.cuh"

#include <cuda_bf16.h>

namespace slag {

namespace {

constexpr int kRowsT = 128;     // rows of A per tile: TMEM lanes
constexpr int kKC = 32;         // K per stage: one 128-byte swizzle row of TF32
constexpr int kStagesD = 3;
constexpr int kEpiWarps = 8;    // two per TMEM lane quarter, one per half of the tile's columns
constexpr int kThreadsD = 32 * (2 + kEpiWarps);   // TMA, MMA, epilogue
constexpr int kAPlaneD = kRowsT * kKC * 4;   // 16 KB

enum { kBiasRows = 0, kGeluPlanes = 1 };

template <int NT>
struct DenseShape {
    static constexpr int kBBytes = NT * kKC * 4;                 // 32 or 16 KB
    static constexpr int kStageBytes = 2 * kAPlaneD + kBBytes;
    static constexpr uint32_t kIdesc = tc::idesc_tf32<NT>();
    static_assert(kBBytes % 1024 == 0, "swizzle atoms stay 1024-byte aligned");
};

struct __align__(8) DenseCtl {
    uint64_t full[kStagesD];
    uint64_t empty[kStagesD];
    uint64_t tfull[2];          // MMA -> epilogue (tcgen05.commit), per accumulator
    uint64_t tempty[2];         // epilogue -> MMA (one arrival per epilogue warp)
    uint32_t tmem_addr;
    uint32_t abort;
};

template <int NT>
constexpr size_t dense_smem() {
    return 1024 + (size_t)kStagesD * DenseShape<NT>::kStageBytes + sizeof(DenseCtl);
}
static_assert(dense_smem<256>() <= 232448, "fits the opt-in shared memory of a CTA");

__device__ __forceinline__ float gelu_d(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

// Persistent: CTA b takes tiles b, b + gridDim.x, ... (tile t: row tile t / ntn, column tile
// t % ntn); tile j of a CTA accumulates into TMEM accumulator j & 1 while the epilogue drains the
// other one.
template <int NT, int kMode>
__global__ void __launch_bounds__(kThreadsD, 1)
    dense_tc_k(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW, int64_t rows,
               int64_t rows_pad, int32_t K, int32_t N, const float *__restrict__ bias, float *__restrict__ out,
               int64_t ldo, uint32_t *err) {
    using Sh = DenseShape<NT>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    DenseCtl *ctl = reinterpret_cast<DenseCtl *>(base + kStagesD * Sh::kStageBytes);
    volatile uint32_t *abort = &ctl->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntn = N / NT;
    const int64_t ntiles = rows_pad / kRowsT * ntn;
    const int ntl = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int nchunk = K / kKC;
    auto tile_of = [&](int j, int64_t *r0, int *n0) {
        const int64_t t = blockIdx.x + (int64_t)j * gridDim.x;
        *r0 = t / ntn * kRowsT;
        *n0 = (int)(t % ntn) * NT;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesD; ++s) {
            tc::mbar_init(&ctl->full[s], 1);
            tc::mbar_init(&ctl->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&ctl->tfull[a], 1);
            tc::mbar_init(&ctl->tempty[a], kEpiWarps);
        }
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmW)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_u32(&ctl->tmem_addr)),
                     "r"((uint32_t)(2 * NT))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = ctl->tmem_addr;
    if (warp == 0) {
        if (lane == 0) {
            // producer: load i goes to stage i % kStagesD once the MMAs of load i - kStagesD are done
            int64_t i = 0;
            bool ok = true;
            for (int j = 0; j < ntl && ok; ++j) {
                int64_t r0;
                int n0;
                tile_of(j, &r0, &n0);
                for (int c = 0; c < nchunk; ++c, ++i) {
                    const int s = (int)(i % kStagesD);
                    if (i >= kStagesD &&
                        !tc::wait_or_abort(&ctl->empty[s], (uint32_t)((i / kStagesD - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    unsigned char *stg = base + s * Sh::kStageBytes;
                    tc::expect_tx(&ctl->full[s], (uint32_t)Sh::kStageBytes);
                    tc::tma_load_3d(tc::smem_u32(stg), &tmA, &ctl->full[s], c * kKC, (int)r0, 0);
                    tc::tma_load_3d(tc::smem_u32(stg + 2 * kAPlaneD), &tmW, &ctl->full[s], c * kKC, n0, 0);
                }
            }
            if (ok) {
                // tail: the commits that free the last stages arrive before the CTA exits
                for (int64_t l = i > kStagesD ? i - kStagesD : 0; l < i; ++l)
                    if (!tc::wait_or_abort(&ctl->empty[l % kStagesD], (uint32_t)((l / kStagesD) & 1), abort)) break;
            } else {
                // loads in flight write this CTA's shared memory: let them land (bounded)
                for (int64_t l = i > kStagesD ? i - kStagesD : 0; l < i; ++l) {
                    volatile uint32_t never = 0;
                    tc::wait_or_abort(&ctl->full[l % kStagesD], (uint32_t)((l / kStagesD) & 1), &never);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int64_t i = 0, last = -1;
            bool ok = true;
            for (int j = 0; j < ntl && ok; ++j) {
                const int acc = j & 1;
                if (j >= 2 && !tc::wait_or_abort(&ctl->tempty[acc], (uint32_t)((j / 2 - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dt = tmem + (uint32_t)(acc * NT);
                for (int c = 0; c < nchunk; ++c, ++i) {
                    const int s = (int)(i % kStagesD);
                    if (!tc::wait_or_abort(&ctl->full[s], (uint32_t)((i / kStagesD) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a_hi = tc::smem_u32(base + s * Sh::kStageBytes), a_lo = a_hi + kAPlaneD;
                    const uint32_t w = a_hi + 2 * kAPlaneD;
#pragma unroll
                    for (int ks = 0; ks < kKC / 8; ++ks) {
                        const uint32_t ko = ks * 32;   // K = 8 TF32 = 32 bytes along the swizzled row
                        const uint64_t dw = tc::smem_desc(w + ko);
                        tc::mma_tf32(dt, tc::smem_desc(a_hi + ko), dw, Sh::kIdesc, (c > 0 || ks > 0) ? 1u : 0u);
                        tc::mma_tf32(dt, tc::smem_desc(a_lo + ko), dw, Sh::kIdesc, 1u);
                    }
                    tc::mma_commit(&ctl->empty[s]);
                    last = i;
                }
                if (ok) tc::mma_commit(&ctl->tfull[acc]);
            }
            if (!ok && last >= 0) {
                // MMAs in flight read shared memory and write TMEM: let them finish (bounded)
                volatile uint32_t never = 0;
                tc::wait_or_abort(&ctl->empty[last % kStagesD], (uint32_t)((last / kStagesD) & 1), &never);
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. (one row per thread) and one half of
        // the tile's columns
        const int quarter = warp & 3;
        const int c0 = ((warp - 2) >> 2) * (NT / 2);
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        for (int j = 0; j < ntl; ++j) {
            const int acc = j & 1;
            int64_t r0;
            int n0;
            tile_of(j, &r0, &n0);
            const int64_t r = r0 + quarter * 32 + lane;
            const bool got = tc::wait_or_abort(&ctl->tfull[acc], (uint32_t)((j / 2) & 1), abort);
            if (!__all_sync(0xffffffffu, got)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int cb = c0; cb < c0 + NT / 2; cb += 32) {
                float v[32];
                tc::tmem_ld32(lane_base + (uint32_t)(acc * NT + cb), v);
                const float bl = __ldg(bias + n0 + cb + lane);
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] += __shfl_sync(0xffffffffu, bl, q);
                if (kMode == kGeluPlanes) {
                    // every row of the padded planes is written (padding rows: gelu(b), never read
                    // into an output)
                    float *hi = out + r * N + n0 + cb;
                    float *lo = hi + rows_pad * N;
#pragma unroll
                    for (int q = 0; q < 32; q += 4) {
                        float4 h, l;
                        float x;
                        x = gelu_d(v[q]);     h.x = tc::to_tf32(x); l.x = tc::to_tf32(x - h.x);
                        x = gelu_d(v[q + 1]); h.y = tc::to_tf32(x); l.y = tc::to_tf32(x - h.y);
                        x = gelu_d(v[q + 2]); h.z = tc::to_tf32(x); l.z = tc::to_tf32(x - h.z);
                        x = gelu_d(v[q + 3]); h.w = tc::to_tf32(x); l.w = tc::to_tf32(x - h.w);
                        *reinterpret_cast<float4 *>(hi + q) = h;
                        *reinterpret_cast<float4 *>(lo + q) = l;
                    }
                } else if (r < rows) {
                    float *o = out + r * ldo + n0 + cb;
#pragma unroll
                    for (int q = 0; q < 32; q += 4)
                        *reinterpret_cast<float4 *>(o + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                }
            }
            // this warp has read the accumulator: it may take the tile after next
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) tc::arrive(&ctl->tempty[acc]);
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *abort) atomicOr(err, 1u);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * NT))
                     : "memory");
    }
}

// wt[n][k] = bfloat16-rounded W[k][n] (W: K x N row-major)
__global__ void __launch_bounds__(256) weights_t_k(const float *__restrict__ W, int32_t K, int32_t N,
                                                   float *__restrict__ wt, int tf32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)K * N) return;
    const int64_t n = i / K, k = i - n * K;
    const float w = W[k * N + n];
    wt[i] = tf32 ? tc::to_tf32(w) : __bfloat162float(__float2bfloat16_rn(w));
}

template <int NT, int kMode>
cudaError_t launch_dense_t(const CUtensorMap &ta, const CUtensorMap &tw, int64_t rows, int64_t rows_pad, int32_t K,
                           int32_t N, const float *bias, float *out, int64_t ldo, uint32_t *err, cudaStream_t st) {
    {
        const cudaError_t e = set_max_smem((const void *)dense_tc_k<NT, kMode>, (int)dense_smem<NT>());
        if (e != cudaSuccess) return e;
    }
    // persistent: one CTA per SM at most (the shared memory admits one)
    int sms = 148;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = rows_pad / kRowsT * (N / NT);
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sms);
    dense_tc_k<NT, kMode><<<grid, kThreadsD, dense_smem<NT>(), st>>>(ta, tw, rows, rows_pad, K, N, bias, out, ldo, err);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

int64_t dense_tc_pad_rows(int64_t rows) { return (rows + kRowsT - 1) / kRowsT * kRowsT; }

void launch_weights_t(const float *W, int32_t K, int32_t N, float *wt, cudaStream_t st, bool tf32) {
    const int64_t n = (int64_t)K * N;
    weights_t_k<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, K, N, wt, tf32 ? 1 : 0); note_launch();
}

cudaError_t launch_dense_tc(const float *a_planes, int64_t rows, int64_t rows_pad, int32_t K, const float *wt,
                            int32_t N, const float *bias, bool gelu_planes, float *out, int64_t ldo, uint32_t *err,
                            cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (K % kKC != 0 || N % 128 != 0 || rows_pad % kRowsT != 0 || rows_pad < rows) return cudaErrorInvalidValue;
    const int nt = N % 256 == 0 ? 256 : 128;
    CUtensorMap ta, tw;
    if (!tc::encode_planes(&ta, a_planes, rows_pad, K, kRowsT, 2) || !tc::encode_planes(&tw, wt, N, K, nt, 1))
        return cudaErrorInvalidValue;
    if (nt == 256)
        return gelu_planes ? launch_dense_t<256, kGeluPlanes>(ta, tw, rows, rows_pad, K, N, bias, out, ldo, err, st)
                           : launch_dense_t<256, kBiasRows>(ta, tw, rows, rows_pad, K, N, bias, out, ldo, err, st);
    return gelu_planes ? launch_dense_t<128, kGeluPlanes>(ta, tw, rows, rows_pad, K, N, bias, out, ldo, err, st)
                       : launch_dense_t<128, kBiasRows>(ta, tw, rows, rows_pad, K, N, bias, out, ldo, err, st);
}

}  // namespace slag
