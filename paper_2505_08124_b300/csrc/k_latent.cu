// The learned latent form: a small autoencoder D -> 256 -> 32 (encoder) and
// 32 -> 256 -> D (decoder) with erf-GELU after the hidden layers, trained on
// segment embeddings, so that the aggregation runs on 32-d latent codes:
// Z_k = sum w z_seg / sum w, decoded per Gaussian to E_k = dec(Z_k) at
// finalize (the decoder is not linear, so dec(mean z) differs from the mean
// of the decoded codes; the plain path is the reference for the error).
//
// Parameters are float32 masters; every product uses them rounded to
// bfloat16 (bfloat16 weights, float32 accumulation). Kernels:
//   * gemm_k: C = act(A' B' + bias) for row-major A (or its transpose) and B
//     (or its transpose), 64 x 64 tiles of C per 256-thread CTA, K in steps
//     of 16 through shared memory, a 4 x 4 register tile per thread;
//   * the loss per sample, mean((y - x)^2) + (1 - cos(y, x)), and its
//     gradient, one warp per sample;
//   * bias gradients (column sums), GELU backward, Adam, row gathers.
// The aggregation in the latent space: a warp per 32 triples at a time (lane =
// latent dimension), the block's 128 x 32 sums in shared memory.
#include <cuda_bf16.h>

#include "slag_internal.cuh"

namespace slag {

namespace {

constexpr int kTM = 64, kTN = 64, kTK = 16;

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// C (M x N) = act(op(A) op(B) + bias); op(A) is M x K, op(B) is K x N. A is M x K row-major
// (lda) or, transposed, K x M; B is K x N (ldb) or, transposed, N x K. When round_b, B's
// values enter as bfloat16 (the weights); pre (nullable) receives the value before act.
template <bool kTA, bool kTB>
__global__ void __launch_bounds__(256) gemm_k(int M, int N, int K, const float *__restrict__ A, int lda,
                                              const float *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                              const float *__restrict__ bias, int act, float *__restrict__ pre,
                                              int round_a, int round_b, int accumulate) {
    __shared__ float As[kTK][kTM + 4];
    __shared__ float Bs[kTK][kTN + 4];
    const int tid = threadIdx.x;
    const int tr = tid >> 4, tc = tid & 15;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kTK) {
        // A tile: kTM x kTK elements, 4 per thread
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * 256;
            int mm, kk;
            if (kTA) { kk = idx / kTM; mm = idx % kTM; } else { mm = idx / kTK; kk = idx % kTK; }
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.f;
            if (m < M && k < K) v = kTA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
            As[kk][mm] = round_a ? bf16_round(v) : v;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * 256;
            int nn, kk;
            if (kTB) { nn = idx / kTK; kk = idx % kTK; } else { kk = idx / kTN; nn = idx % kTN; }
            const int n = n0 + nn, k = k0 + kk;
            float v = 0.f;
            if (n < N && k < K) v = kTB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n];
            Bs[kk][nn] = round_b ? bf16_round(v) : v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kTK; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][tr * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[k][tc * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + tr * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tc * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j] + (bias ? bias[n] : 0.f);
            if (accumulate) v += C[(int64_t)m * ldc + n];
            if (pre) pre[(int64_t)m * ldc + n] = v;
            C[(int64_t)m * ldc + n] = act ? gelu(v) : v;
        }
    }
}

// Per sample r: loss_r = mean_d (y - x)^2 + (1 - cos(y, x)); dY = d(mean_r loss_r)/dY.
__global__ void loss_k(const float *__restrict__ Y, const float *__restrict__ X, int B, int D, float *__restrict__ dY,
                       float *__restrict__ loss_sum) {
    const int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (r >= B) return;
    const float *y = Y + (int64_t)r * D, *x = X + (int64_t)r * D;
    float se = 0.f, yy = 0.f, xx = 0.f, xy = 0.f;
    for (int d = lane; d < D; d += 32) {
        const float e = y[d] - x[d];
        se = fmaf(e, e, se);
        yy = fmaf(y[d], y[d], yy);
        xx = fmaf(x[d], x[d], xx);
        xy = fmaf(x[d], y[d], xy);
    }
    for (int o = 16; o; o >>= 1) {
        se += __shfl_xor_sync(0xffffffffu, se, o);
        yy += __shfl_xor_sync(0xffffffffu, yy, o);
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
        xy += __shfl_xor_sync(0xffffffffu, xy, o);
    }
    const float ny = sqrtf(fmaxf(yy, 1e-30f)), nx = sqrtf(fmaxf(xx, 1e-30f));
    const float cs = xy / (ny * nx);
    const float inv_b = 1.f / (float)B;
    for (int d = lane; d < D; d += 32) {
        const float g_mse = 2.f * (y[d] - x[d]) / (float)D;
        const float g_cos = -(x[d] / (ny * nx) - cs * y[d] / (ny * ny));
        dY[(int64_t)r * D + d] = (g_mse + g_cos) * inv_b;
    }
    if (lane == 0) atomicAdd(loss_sum, se / (float)D + (1.f - cs));
}

__global__ void gelu_bwd_k(float *__restrict__ dH, const float *__restrict__ pre, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dH[i] *= gelu_grad(pre[i]);
}

// db[n] = sum over rows of dC[row][n]
__global__ void colsum_k(const float *__restrict__ dC, int M, int N, float *__restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += dC[(int64_t)m * N + n];
    db[n] = s;
}

__global__ void adam_k(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void gather_rows_k(const float *__restrict__ src, const uint32_t *__restrict__ idx, int rows, int D,
                              float *__restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * D) return;
    const int r = (int)(e / D), d = (int)(e % D);
    dst[e] = src[(int64_t)idx[r] * D + d];
}

// Latent aggregation of one block of 128 Gaussians: Zs[g][c] += w * Zcol[c]; then divide by sum w.
__global__ void __launch_bounds__(256) latent_aggregate_k(const AggArgs a, const float *__restrict__ ztable,
                                                          float *__restrict__ Z) {
    __shared__ float acc[kBlockG][kLatent + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t b = blockIdx.x;
    for (int e = tid; e < kBlockG * (kLatent + 1); e += 256) (&acc[0][0])[e] = 0.f;
    __syncthreads();
    const uint32_t ts = a.bstart[b], te = a.bend[b];
    // a warp takes 32 triples at a time: one coalesced load of their keys and weights, then the
    // code rows of 8 triples in flight together before their adds (lane = latent dimension)
    for (uint32_t t0 = ts + (uint32_t)warp * 32u; t0 < te; t0 += 8u * 32u) {
        const uint32_t t = t0 + (uint32_t)lane;
        uint32_t colv = 0u, gv = 0u;
        float wv = 0.f;
        if (t < te) {
            const uint64_t key = a.keys[t];
            colv = (uint32_t)((key >> 7) & 0xffffffffu);
            gv = (uint32_t)(key & 127u);
            wv = a.w[t];
        }
        const int nt = (int)min(32u, te - t0);
        for (int j = 0; j < nt; j += 8) {
            float z[8], wj[8];
            uint32_t gj[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int src = min(j + u, 31);
                const uint32_t c = __shfl_sync(0xffffffffu, colv, src);
                gj[u] = __shfl_sync(0xffffffffu, gv, src);
                wj[u] = j + u < nt ? __shfl_sync(0xffffffffu, wv, src) : 0.f;
                z[u] = __ldg(ztable + (int64_t)c * kLatent + lane);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (j + u < nt) atomicAdd(&acc[gj[u]][lane], wj[u] * z[u]);
        }
    }
    __syncthreads();
    for (int e = tid; e < kBlockG * kLatent; e += 256) {
        const int i = e / kLatent, c = e % kLatent;
        const int64_t g = b * kBlockG + i;
        if (g >= a.n) continue;
        const float S = (a.s_hi[g] + a.s_lo[g]) + a.s_ovf[g];
        Z[g * kLatent + c] = S > 0.f ? acc[i][c] / S : 0.f;
    }
}

// One warp per Gaussian g0 + r: its decoded row to E in caller order, with the row norm.
__global__ void latent_finish_k(const AggArgs a, const float *__restrict__ Y, int64_t g0, int64_t rows) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const int64_t g = g0 + r;
    if (g >= a.n) return;
    const float S = (a.s_hi[g] + a.s_lo[g]) + a.s_ovf[g];
    const uint32_t o = a.orig_of_int[g];
    float *out = a.E + (int64_t)o * a.D;
    const float *y = Y + r * a.D;
    float n2 = 0.f;
    for (int d = lane; d < a.D; d += 32) {
        const float v = S > 0.f ? y[d] : 0.f;
        out[d] = v;
        n2 = fmaf(v, v, n2);
    }
    for (int o2 = 16; o2; o2 >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o2);
    if (lane == 0) {
        a.inv_norm[o] = (S > 0.f && n2 > 0.f) ? 1.f / sqrtf(n2) : 0.f;
        a.wsum[o] = S;
        if (S > 0.f) atomicAdd(a.touched, 1ull);
    }
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_latent_finish(const AggArgs &a, const float *Y, int64_t g0, int64_t rows, cudaStream_t st) {
    if (rows <= 0) return;
    latent_finish_k<<<blocks(rows * 32, 256), 256, 0, st>>>(a, Y, g0, rows); note_launch();
}

void latent_gemm(bool ta, bool tb, int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C,
                 int ldc, const float *bias, bool gelu_act, float *pre, bool round_a, bool round_b, bool accumulate,
                 cudaStream_t st) {
    dim3 grid((unsigned)((N + kTN - 1) / kTN), (unsigned)((M + kTM - 1) / kTM));
    const int act = gelu_act ? 1 : 0, ra = round_a ? 1 : 0, rb = round_b ? 1 : 0, ac = accumulate ? 1 : 0;
    if (!ta && !tb) gemm_k<false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act, pre, ra, rb, ac);
    else if (ta && !tb) gemm_k<true, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act, pre, ra, rb, ac);
    else if (!ta && tb) gemm_k<false, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act, pre, ra, rb, ac);
    else gemm_k<true, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act, pre, ra, rb, ac);
    note_launch();
}

void latent_loss(const float *Y, const float *X, int B, int D, float *dY, float *loss_sum, cudaStream_t st) {
    loss_k<<<blocks((int64_t)B * 32, 256), 256, 0, st>>>(Y, X, B, D, dY, loss_sum); note_launch();
}

void latent_gelu_bwd(float *dH, const float *pre, int64_t n, cudaStream_t st) {
    gelu_bwd_k<<<blocks(n, 256), 256, 0, st>>>(dH, pre, n); note_launch();
}

void latent_colsum(const float *dC, int M, int N, float *db, cudaStream_t st) {
    colsum_k<<<blocks(N, 128), 128, 0, st>>>(dC, M, N, db); note_launch();
}

void latent_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, int step, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_k<<<blocks(n, 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2); note_launch();
}

void latent_gather_rows(const float *src, const uint32_t *idx, int rows, int D, float *dst, cudaStream_t st) {
    gather_rows_k<<<blocks((int64_t)rows * D, 256), 256, 0, st>>>(src, idx, rows, D, dst); note_launch();
}

void launch_latent_aggregate(const AggArgs &a, const float *ztable, float *Z, int64_t nblocks, cudaStream_t st) {
    if (nblocks <= 0) return;
    latent_aggregate_k<<<(unsigned)nblocks, 256, 0, st>>>(a, ztable, Z); note_launch();
}

}  // namespace slag
