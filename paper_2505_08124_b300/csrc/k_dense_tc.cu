// Dense layers on the 5th-generation tensor cores: C = act(A W + b), for the
// decoder of the learned latent form (32 -> 256 -> D, erf-GELU after the hidden
// layer; bfloat16-rounded weights, float32 activations and accumulation).
//
// A (rows x K) arrives as its TF32 hi/lo planes (hi = x rounded to TF32, lo =
// the rest rounded to TF32); the weights arrive transposed (N x K) and rounded
// to bfloat16, which TF32 holds exactly, as one plane. Each product is then
// A_hi W + A_lo W, float32-accurate to about 2^-21 of its magnitude.
//
// A CTA computes a 128 x NT tile of C (NT = 256, or 128 when N is not a
// multiple of 256; M = 128 TMEM lanes, NT TMEM columns), its warps in fixed
// roles:
//   warp 0      one thread issues TMA loads of K-chunks of 32 values: a 3-D
//               box {32, 128, 2} of A's planes and {32, NT, 1} of the weights,
//               128-byte swizzled, into one of three stages;
//   warp 1      owns the TMEM allocation; one thread issues 4 K-steps x 2 MMAs
//               per chunk, freeing the stage by tcgen05.commit;
//   warps 2..5  the epilogue: one row of the tile per thread, 32 columns per
//               tcgen05.ld, then either
//               kGeluPlanes: h = gelu(acc + b), written as the TF32 hi/lo
//                            planes of the next layer's input, or
//               kBiasRows:   acc + b, written as float32 rows.
// Every wait on an mbarrier is bounded (about one second of globaltimer) and
// gives up once another role has given up; the producer and the MMA thread
// then wait (bounded) for their operations in flight, TMEM is released and
// *err is set.
#include "slag_internal.cuh"
#include "tc_util.cuh"

#include <cuda_bf16.h>

namespace slag {

namespace {

constexpr int kRowsT = 128;     // rows of A per CTA: TMEM lanes
constexpr int kKC = 32;         // K per stage: one 128-byte swizzle row of TF32
constexpr int kStagesD = 3;
constexpr int kThreadsD = 192;  // 6 warps: TMA, MMA, 4 x epilogue
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
    uint64_t tfull;
    uint32_t tmem_addr;
    uint32_t abort;
};

template <int NT>
constexpr size_t dense_smem() {
    return 1024 + (size_t)kStagesD * DenseShape<NT>::kStageBytes + sizeof(DenseCtl);
}
static_assert(dense_smem<256>() <= 232448, "fits the opt-in shared memory of a CTA");

__device__ __forceinline__ float gelu_d(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

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
    const int64_t r0 = (int64_t)blockIdx.x * kRowsT;
    const int n0 = blockIdx.y * NT;
    const int nchunk = K / kKC;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesD; ++s) {
            tc::mbar_init(&ctl->full[s], 1);
            tc::mbar_init(&ctl->empty[s], 1);
        }
        tc::mbar_init(&ctl->tfull, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmW)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::smem_u32(&ctl->tmem_addr)),
                     "r"((uint32_t)NT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = ctl->tmem_addr;

    if (warp == 0) {
        if (lane == 0) {
            // producer: chunk c goes to stage c % kStagesD once the MMAs of chunk c - kStagesD are done
            int c = 0;
            bool ok = true;
            for (; c < nchunk; ++c) {
                const int s = c % kStagesD;
                if (c >= kStagesD && !tc::wait_or_abort(&ctl->empty[s], (uint32_t)((c / kStagesD - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                unsigned char *stg = base + s * Sh::kStageBytes;
                tc::expect_tx(&ctl->full[s], (uint32_t)Sh::kStageBytes);
                tc::tma_load_3d(tc::smem_u32(stg), &tmA, &ctl->full[s], c * kKC, (int)r0, 0);
                tc::tma_load_3d(tc::smem_u32(stg + 2 * kAPlaneD), &tmW, &ctl->full[s], c * kKC, n0, 0);
            }
            if (ok) {
                // tail: the commits that free the last stages arrive before the CTA exits
                for (int l = c > kStagesD ? c - kStagesD : 0; l < c; ++l)
                    if (!tc::wait_or_abort(&ctl->empty[l % kStagesD], (uint32_t)((l / kStagesD) & 1), abort)) break;
            } else {
                // loads in flight write this CTA's shared memory: let them land (bounded)
                for (int l = c > kStagesD ? c - kStagesD : 0; l < c; ++l) {
                    volatile uint32_t never = 0;
                    tc::wait_or_abort(&ctl->full[l % kStagesD], (uint32_t)((l / kStagesD) & 1), &never);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int last = -1;
            bool ok = true;
            for (int c = 0; c < nchunk; ++c) {
                const int s = c % kStagesD;
                if (!tc::wait_or_abort(&ctl->full[s], (uint32_t)((c / kStagesD) & 1), abort)) {
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
                    tc::mma_tf32(tmem, tc::smem_desc(a_hi + ko), dw, Sh::kIdesc, (c > 0 || ks > 0) ? 1u : 0u);
                    tc::mma_tf32(tmem, tc::smem_desc(a_lo + ko), dw, Sh::kIdesc, 1u);
                }
                tc::mma_commit(&ctl->empty[s]);
                last = c;
            }
            if (ok) {
                tc::mma_commit(&ctl->tfull);
            } else if (last >= 0) {
                // MMAs in flight read shared memory and write TMEM: let them finish (bounded)
                volatile uint32_t never = 0;
                tc::wait_or_abort(&ctl->empty[last % kStagesD], (uint32_t)((last / kStagesD) & 1), &never);
            }
        }
    } else {
        // epilogue: row r0 + 32 (warp mod 4) + lane of the tile
        const int quarter = warp & 3;
        const int64_t r = r0 + quarter * 32 + lane;
        const bool got = tc::wait_or_abort(&ctl->tfull, 0u, abort);
        if (__all_sync(0xffffffffu, got)) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
            for (int cb = 0; cb < NT; cb += 32) {
                float v[32];
                tc::tmem_ld32(lane_base + (uint32_t)cb, v);
                const float bl = __ldg(bias + n0 + cb + lane);
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] += __shfl_sync(0xffffffffu, bl, j);
                if (kMode == kGeluPlanes) {
                    // every row of the padded planes is written (padding rows: gelu(b), never read
                    // into an output)
                    float *hi = out + r * N + n0 + cb;
                    float *lo = hi + rows_pad * N;
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        float4 h, l;
                        float x;
                        x = gelu_d(v[j]);     h.x = tc::to_tf32(x); l.x = tc::to_tf32(x - h.x);
                        x = gelu_d(v[j + 1]); h.y = tc::to_tf32(x); l.y = tc::to_tf32(x - h.y);
                        x = gelu_d(v[j + 2]); h.z = tc::to_tf32(x); l.z = tc::to_tf32(x - h.z);
                        x = gelu_d(v[j + 3]); h.w = tc::to_tf32(x); l.w = tc::to_tf32(x - h.w);
                        *reinterpret_cast<float4 *>(hi + j) = h;
                        *reinterpret_cast<float4 *>(lo + j) = l;
                    }
                } else if (r < rows) {
                    float *o = out + r * ldo + n0 + cb;
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *reinterpret_cast<float4 *>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && *abort) atomicOr(err, 1u);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)NT) : "memory");
    }
}

// wt[n][k] = bfloat16-rounded W[k][n] (W: K x N row-major)
__global__ void __launch_bounds__(256) weights_t_k(const float *__restrict__ W, int32_t K, int32_t N,
                                                   float *__restrict__ wt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)K * N) return;
    const int64_t n = i / K, k = i - n * K;
    wt[i] = __bfloat162float(__float2bfloat16_rn(W[k * N + n]));
}

template <int NT, int kMode>
cudaError_t launch_dense_t(const CUtensorMap &ta, const CUtensorMap &tw, int64_t rows, int64_t rows_pad, int32_t K,
                           int32_t N, const float *bias, float *out, int64_t ldo, uint32_t *err, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(dense_tc_k<NT, kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)dense_smem<NT>());
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((unsigned)(rows_pad / kRowsT), (unsigned)(N / NT));
    dense_tc_k<NT, kMode><<<grid, kThreadsD, dense_smem<NT>(), st>>>(ta, tw, rows, rows_pad, K, N, bias, out, ldo, err);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

int64_t dense_tc_pad_rows(int64_t rows) { return (rows + kRowsT - 1) / kRowsT * kRowsT; }

void launch_weights_t(const float *W, int32_t K, int32_t N, float *wt, cudaStream_t st) {
    const int64_t n = (int64_t)K * N;
    weights_t_k<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, K, N, wt); note_launch();
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
