// Cosine top-k ("Query processing for inference"): score_k = q . E_k / |E_k|
// over the Gaussians with sum w > 0 and a non-zero embedding; results by
// descending score, ties to the lower Gaussian index.
//
// The candidates are rows rows[0..n) of E when a row list is given (the
// touched Gaussians in increasing order, so ties still go to the lower
// Gaussian index), else rows 0..n; results are row numbers of E.
//
// Stage 1: a CTA scores 64 queries x 128 Gaussians (K = D in steps of 16,
// a 4 x 8 register tile per thread) and keeps, per query, the best
// min(k, 128) of its 128 Gaussians as candidates. Stage 2: one CTA per query
// selects the k best of all candidates.
#include <float.h>

#include "slag_internal.cuh"

namespace slag {

namespace {

constexpr int kQB = 64;    // queries per CTA
constexpr int kGB = 128;   // Gaussians per CTA
constexpr int kKD = 16;    // depth of a K step

// (score, index) order: higher score first, then lower index.
__device__ __forceinline__ bool better(float s, uint32_t i, float s2, uint32_t i2) {
    return s > s2 || (s == s2 && i < i2);
}

__global__ void __launch_bounds__(256) score_tile_k(const float *__restrict__ Q, int32_t B,
                                                    const float *__restrict__ E, const float *__restrict__ inv_norm,
                                                    const uint32_t *__restrict__ rows, int64_t n, int32_t D,
                                                    int32_t kk, float *__restrict__ cand_s,
                                                    uint32_t *__restrict__ cand_i, int32_t ntiles) {
    __shared__ __align__(16) float Qs[kKD][kQB + 4];
    __shared__ __align__(16) float Es[kKD][kGB + 4];
    __shared__ float Sc[kQB][kGB + 1];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int tq = tid >> 4, tg = tid & 15;
    const int64_t g0 = (int64_t)blockIdx.x * kGB;
    const int q0 = blockIdx.y * kQB;
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    for (int d0 = 0; d0 < D; d0 += kKD) {
        {
            const int q = tid >> 2, d4 = tid & 3;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q0 + q < B) v = *reinterpret_cast<const float4 *>(Q + (int64_t)(q0 + q) * D + d0 + d4 * 4);
            Qs[d4 * 4 + 0][q] = v.x;
            Qs[d4 * 4 + 1][q] = v.y;
            Qs[d4 * 4 + 2][q] = v.z;
            Qs[d4 * 4 + 3][q] = v.w;
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int e = tid + r * 256;
            const int gl = e >> 2, d4 = e & 3;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g0 + gl < n) {
                const int64_t row = rows ? (int64_t)rows[g0 + gl] : g0 + gl;
                v = *reinterpret_cast<const float4 *>(E + row * D + d0 + d4 * 4);
            }
            Es[d4 * 4 + 0][gl] = v.x;
            Es[d4 * 4 + 1][gl] = v.y;
            Es[d4 * 4 + 2][gl] = v.z;
            Es[d4 * 4 + 3][gl] = v.w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kKD; ++k) {
            const float4 qa = *reinterpret_cast<const float4 *>(&Qs[k][tq * 4]);
            const float4 e0 = *reinterpret_cast<const float4 *>(&Es[k][tg * 4]);
            const float4 e1 = *reinterpret_cast<const float4 *>(&Es[k][64 + tg * 4]);
            const float qv[4] = {qa.x, qa.y, qa.z, qa.w};
            const float ev[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(qv[i], ev[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int gl = j < 4 ? tg * 4 + j : 64 + tg * 4 + (j - 4);
        const int64_t g = g0 + gl;
        const float inv = g < n ? inv_norm[rows ? (int64_t)rows[g] : g] : 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) Sc[tq * 4 + i][gl] = inv > 0.f ? acc[i][j] * inv : -INFINITY;
    }
    __syncthreads();
    // per query row: kk rounds of warp arg-max over the 128 scores
    for (int qr = w; qr < kQB; qr += 8) {
        const int q = q0 + qr;
        if (q >= B) break;
        float v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = Sc[qr][lane + 32 * c];
        float *cs = cand_s + ((int64_t)q * ntiles + blockIdx.x) * kk;
        uint32_t *ci = cand_i + ((int64_t)q * ntiles + blockIdx.x) * kk;
        for (int r = 0; r < kk; ++r) {
            float bs = v[0];
            int bc = 0;
#pragma unroll
            for (int c = 1; c < 4; ++c)
                if (v[c] > bs) { bs = v[c]; bc = c; }
            uint32_t bi = (uint32_t)(lane + 32 * bc);
            for (int o = 16; o; o >>= 1) {
                const float s2 = __shfl_xor_sync(0xffffffffu, bs, o);
                const uint32_t i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                if (better(s2, i2, bs, bi)) { bs = s2; bi = i2; }
            }
            if (lane == 0) {
                cs[r] = bs;
                ci[r] = bs == -INFINITY ? 0xffffffffu : (uint32_t)(g0 + bi);
            }
            if ((bi & 31u) == (uint32_t)lane) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if ((uint32_t)c == (bi >> 5)) v[c] = -INFINITY;
            }
        }
    }
}

__global__ void __launch_bounds__(256) merge_k(const float *__restrict__ cand_s, const uint32_t *__restrict__ cand_i,
                                               int64_t per_query, int32_t k, const uint32_t *__restrict__ rows,
                                               int64_t *__restrict__ out_ids,
                                               float *__restrict__ out_scores, int32_t *__restrict__ out_count) {
    __shared__ float ws[8];
    __shared__ uint32_t wi[8];
    __shared__ float last_s;
    __shared__ uint32_t last_i;
    const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const float *cs = cand_s + (int64_t)q * per_query;
    const uint32_t *ci = cand_i + (int64_t)q * per_query;
    // selection by rounds: each round takes the best candidate strictly after the previous pick
    float ps = INFINITY;
    uint32_t pi = 0;
    int found = 0;
    for (int r = 0; r < k; ++r) {
        float bs = -INFINITY;
        uint32_t bi = 0xffffffffu;
        for (int64_t e = tid; e < per_query; e += 256) {
            const float s = cs[e];
            const uint32_t i = ci[e];
            if (i == 0xffffffffu) continue;
            if (!better(ps, pi, s, i)) continue;   // already taken (not strictly after the last pick)
            if (better(s, i, bs, bi)) { bs = s; bi = i; }
        }
        for (int o = 16; o; o >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, bs, o);
            const uint32_t i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (better(s2, i2, bs, bi)) { bs = s2; bi = i2; }
        }
        if (lane == 0) { ws[w] = bs; wi[w] = bi; }
        __syncthreads();
        if (tid == 0) {
            float s = ws[0];
            uint32_t i = wi[0];
            for (int c = 1; c < 8; ++c)
                if (better(ws[c], wi[c], s, i)) { s = ws[c]; i = wi[c]; }
            last_s = s;
            last_i = i;
            out_ids[(int64_t)q * k + r] = i == 0xffffffffu ? -1 : (rows ? (int64_t)rows[i] : (int64_t)i);
            out_scores[(int64_t)q * k + r] = i == 0xffffffffu ? 0.f : s;
        }
        __syncthreads();
        ps = last_s;
        pi = last_i;
        if (pi == 0xffffffffu) {
            for (int r2 = r + 1 + tid; r2 < k; r2 += 256) {
                out_ids[(int64_t)q * k + r2] = -1;
                out_scores[(int64_t)q * k + r2] = 0.f;
            }
            break;
        }
        ++found;
        __syncthreads();
    }
    if (tid == 0 && out_count) out_count[q] = found;
}

}  // namespace

size_t query_cand_entries(int32_t B, int64_t n, int32_t k) {
    const int64_t ntiles = (n + kGB - 1) / kGB;
    const int32_t kk = k < kGB ? k : kGB;
    return (size_t)B * (size_t)ntiles * (size_t)kk;
}

void launch_query_merge(const float *cand_s, const uint32_t *cand_i, int64_t per_query, int32_t B, int32_t k,
                        const uint32_t *rows, int64_t *out_ids, float *out_scores, int32_t *out_count,
                        cudaStream_t st) {
    merge_k<<<B, 256, 0, st>>>(cand_s, cand_i, per_query, k, rows, out_ids, out_scores, out_count); note_launch();
}

void launch_query_topk(const float *Q, int32_t B, const float *E, const float *inv_norm, const uint32_t *rows,
                       int64_t n, int32_t D, int32_t k, float *cand_s, uint32_t *cand_i, int64_t *out_ids,
                       float *out_scores, int32_t *out_count, cudaStream_t st) {
    const int64_t ntiles = (n + kGB - 1) / kGB;
    const int32_t kk = k < kGB ? k : kGB;
    if (ntiles > 0) {
        dim3 grid((unsigned)ntiles, (unsigned)((B + kQB - 1) / kQB));
        score_tile_k<<<grid, 256, 0, st>>>(Q, B, E, inv_norm, rows, n, D, kk, cand_s, cand_i, (int32_t)ntiles); note_launch();
    }
    merge_k<<<B, 256, 0, st>>>(cand_s, cand_i, ntiles * kk, k, rows, out_ids, out_scores, out_count); note_launch();
}

namespace {

// Threshold query: flags[i] = 1 when candidate row rows[i] of E has cosine q . E / |E| >= thr
// (one warp per candidate; inv_norm > 0 on candidates).
__global__ void __launch_bounds__(256) threshold_flags_k(const float *__restrict__ q, const float *__restrict__ E,
                                                         const float *__restrict__ inv_norm,
                                                         const uint32_t *__restrict__ rows, int64_t n, int32_t D,
                                                         float thr, uint32_t *__restrict__ flags) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const uint32_t r = rows[i];
    const float4 *e = reinterpret_cast<const float4 *>(E + (int64_t)r * D);
    const float4 *qq = reinterpret_cast<const float4 *>(q);
    float s = 0.f;
    for (int d = lane; d < D / 4; d += 32) {
        const float4 a = e[d], b = qq[d];
        s = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, s))));
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) flags[i] = (s * inv_norm[r] >= thr) ? 1u : 0u;
}

// out_ids[pos[i]] = rows[i] for the flagged candidates, up to cap; their scores alongside.
__global__ void threshold_ids_k(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos,
                                const uint32_t *__restrict__ rows, int64_t n, int64_t cap, int64_t *__restrict__ ids) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    const int64_t at = pos[i];
    if (at < cap) ids[at] = (int64_t)rows[i];
}

__global__ void touched_flags_k(const float *__restrict__ inv_norm, int64_t n, uint32_t *__restrict__ flags) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) flags[g] = inv_norm[g] > 0.f ? 1u : 0u;
}

__global__ void touched_rows_k(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos, int64_t n,
                               uint32_t *__restrict__ rows) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n && flags[g]) rows[pos[g]] = (uint32_t)g;
}

}  // namespace

void launch_threshold_query(const float *q, const float *E, const float *inv_norm, const uint32_t *rows, int64_t n,
                            int32_t D, float thr, uint32_t *flags, uint32_t *pos, unsigned long long *d_count,
                            int64_t cap, int64_t *ids, SortScratch &scratch, cudaStream_t st) {
    if (n <= 0) {
        cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st);
        return;
    }
    threshold_flags_k<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(q, E, inv_norm, rows, n, D, thr, flags);
    note_launch();
    exclusive_scan_u32(flags, pos, n, d_count, scratch, st);
    threshold_ids_k<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(flags, pos, rows, n, cap, ids); note_launch();
}

void launch_touched_rows(const float *inv_norm, int64_t n, uint32_t *flags, uint32_t *pos, uint32_t *rows,
                         unsigned long long *d_count, SortScratch &scratch, cudaStream_t st) {
    if (n <= 0) return;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    touched_flags_k<<<blocks, 256, 0, st>>>(inv_norm, n, flags); note_launch();
    exclusive_scan_u32(flags, pos, n, d_count, scratch, st);
    touched_rows_k<<<blocks, 256, 0, st>>>(flags, pos, n, rows); note_launch();
}

}  // namespace slag
