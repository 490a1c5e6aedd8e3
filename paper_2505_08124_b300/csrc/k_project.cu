// Gaussian set preparation and per-view projection.
//
// At create time the Gaussians are reordered along a 30-bit Morton curve of
// their means (neighbouring indices are spatial neighbours, which keeps the
// per-block column sets of the aggregation small) and packed as
//   mean_op = (x, y, z, opacity), cov_a = (S00, S01, S02, S11), cov_b = (S12, S22)
// where S = R(q) diag(s) (R(q) diag(s))^T is the world covariance.
//
// The projection (Rasterizer_SLAG: Gaussian -> projected mean mu', 2D
// covariance Sigma' and its conic, tile rectangle) fixes every discrete
// outcome -- visibility, depth key, tile rectangle -- with correctly rounded
// float32 operations in a fixed order (__fmul_rn / __fadd_rn / __fdiv_rn /
// __fsqrt_rn, so nothing is contracted into a fused multiply-add). Constants:
// dilation 0.3, radius ceil(3 sqrt(lambda_max)) with the discriminant floored
// at 0.1, Jacobian clamp 1.3 tan(half fov), rectangle
// [floor((mu'-r)/16), floor((mu'+r)/16)+1) clamped to the tile grid.
#include "slag_internal.cuh"

namespace slag {

namespace {

#define FM __fmul_rn
#define FA __fadd_rn
#define FS __fsub_rn
#define FD __fdiv_rn

__device__ __forceinline__ bool finite3(float a, float b, float c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

__global__ void check_gaussians_k(const float *__restrict__ means, const float *__restrict__ scales,
                                  const float *__restrict__ quats, const float *__restrict__ opac,
                                  int64_t n, uint32_t *flag) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float mx = means[3 * k], my = means[3 * k + 1], mz = means[3 * k + 2];
    float sx = scales[3 * k], sy = scales[3 * k + 1], sz = scales[3 * k + 2];
    float qw = quats[4 * k], qx = quats[4 * k + 1], qy = quats[4 * k + 2], qz = quats[4 * k + 3];
    float o = opac[k];
    bool ok = finite3(mx, my, mz) && finite3(sx, sy, sz) && finite3(qw, qx, qy) && isfinite(qz) &&
              isfinite(o) && sx >= 0.f && sy >= 0.f && sz >= 0.f && o >= 0.f && o <= 1.f &&
              (qw != 0.f || qx != 0.f || qy != 0.f || qz != 0.f);
    if (!ok) atomicOr(flag, 1u);
}

// Order-preserving float <-> uint map (for atomicMin/Max on floats).
__device__ __forceinline__ uint32_t fkey(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float funkey(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void bbox_k(const float *__restrict__ means, int64_t n, uint32_t *bb) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            float v = means[3 * k + a];
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bb[a], fkey(lo[a]));
            atomicMax(&bb[3 + a], fkey(hi[a]));
        }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void morton_k(const float *__restrict__ means, int64_t n, const uint32_t *__restrict__ bb,
                         uint32_t *__restrict__ codes, uint32_t *__restrict__ idx) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        float lo = funkey(bb[a]), hi = funkey(bb[3 + a]);
        float ext = hi - lo;
        float t = ext > 0.f ? (means[3 * k + a] - lo) / ext : 0.f;
        int c = (int)(t * 1024.f);
        q[a] = (uint32_t)min(1023, max(0, c));
    }
    codes[k] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    idx[k] = (uint32_t)k;
}

// World covariance, float32, fixed operation order.
__device__ __forceinline__ void cov3(float sx, float sy, float sz, float qw, float qx, float qy, float qz,
                                     float S[6]) {
    float qq = FA(FA(FA(FM(qw, qw), FM(qx, qx)), FM(qy, qy)), FM(qz, qz));
    float qn = __fsqrt_rn(qq);
    float w = FD(qw, qn), x = FD(qx, qn), y = FD(qy, qn), z = FD(qz, qn);
    float xx = FM(x, x), yy = FM(y, y), zz = FM(z, z);
    float xy = FM(x, y), xz = FM(x, z), yz = FM(y, z);
    float wx = FM(w, x), wy = FM(w, y), wz = FM(w, z);
    float r[9];
    r[0] = FS(1.f, FM(2.f, FA(yy, zz)));
    r[1] = FM(2.f, FS(xy, wz));
    r[2] = FM(2.f, FA(xz, wy));
    r[3] = FM(2.f, FA(xy, wz));
    r[4] = FS(1.f, FM(2.f, FA(xx, zz)));
    r[5] = FM(2.f, FS(yz, wx));
    r[6] = FM(2.f, FS(xz, wy));
    r[7] = FM(2.f, FA(yz, wx));
    r[8] = FS(1.f, FM(2.f, FA(xx, yy)));
    float s[3] = {sx, sy, sz};
    float m[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) m[i * 3 + j] = FM(r[i * 3 + j], s[j]);
    S[0] = FA(FA(FM(m[0], m[0]), FM(m[1], m[1])), FM(m[2], m[2]));
    S[1] = FA(FA(FM(m[0], m[3]), FM(m[1], m[4])), FM(m[2], m[5]));
    S[2] = FA(FA(FM(m[0], m[6]), FM(m[1], m[7])), FM(m[2], m[8]));
    S[3] = FA(FA(FM(m[3], m[3]), FM(m[4], m[4])), FM(m[5], m[5]));
    S[4] = FA(FA(FM(m[3], m[6]), FM(m[4], m[7])), FM(m[5], m[8]));
    S[5] = FA(FA(FM(m[6], m[6]), FM(m[7], m[7])), FM(m[8], m[8]));
}

__global__ void pack_k(const float *__restrict__ means, const float *__restrict__ scales,
                       const float *__restrict__ quats, const float *__restrict__ opac, int64_t n,
                       const uint32_t *__restrict__ orig_of_int, float4 *__restrict__ mean_op,
                       float4 *__restrict__ cov_a, float2 *__restrict__ cov_b,
                       uint32_t *__restrict__ int_of_orig, float *__restrict__ log2_op) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    int64_t k = orig_of_int[g];
    float S[6];
    cov3(scales[3 * k], scales[3 * k + 1], scales[3 * k + 2], quats[4 * k], quats[4 * k + 1],
         quats[4 * k + 2], quats[4 * k + 3], S);
    mean_op[g] = make_float4(means[3 * k], means[3 * k + 1], means[3 * k + 2], opac[k]);
    // log2 of the opacity, rounded to float32 from float64 (the alpha floor is decided on it)
    log2_op[g] = opac[k] > 0.f ? (float)log2((double)opac[k]) : -INFINITY;
    cov_a[g] = make_float4(S[0], S[1], S[2], S[3]);
    cov_b[g] = make_float2(S[4], S[5]);
    int_of_orig[k] = (uint32_t)g;
}

// Per Gaussian (internal order): depth key for the depth sort, written at the
// caller's index so that a stable sort breaks depth ties by that index;
// record (mu', conic, opacity, internal index) and tile rectangle.
__global__ void __launch_bounds__(256) project_k(CamParams cval, const CamParams *__restrict__ cam_dev,
                                                 const float4 *__restrict__ mean_op,
                                                 const float *__restrict__ log2_op,
                                                 const float4 *__restrict__ cov_a, const float2 *__restrict__ cov_b,
                                                 int64_t n, const uint32_t *__restrict__ orig_of_int,
                                                 uint32_t *__restrict__ dkey, uint32_t *__restrict__ dval,
                                                 float4 *__restrict__ rec_a, float4 *__restrict__ rec_b,
                                                 float *__restrict__ rec_t,
                                                 uint2 *__restrict__ rect, ViewCounters *ctr) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const CamParams c = cam_dev ? *cam_dev : cval;   // read on the device in replayed graphs
    bool visible = false;
    if (g < n) {
        float4 mo = mean_op[g];
        const float *R = c.R;
        float tx = FA(FA(FA(FM(R[0], mo.x), FM(R[1], mo.y)), FM(R[2], mo.z)), c.t[0]);
        float ty = FA(FA(FA(FM(R[3], mo.x), FM(R[4], mo.y)), FM(R[5], mo.z)), c.t[1]);
        float tz = FA(FA(FA(FM(R[6], mo.x), FM(R[7], mo.y)), FM(R[8], mo.z)), c.t[2]);
        uint2 rc = make_uint2(0u, 0u);
        float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = make_float4(0.f, 0.f, 0.f, 0.f);
        float rt = INFINITY;
        if (tz > c.near_z && tz < c.far_z) {
            float4 sa = cov_a[g];
            float2 sb = cov_b[g];
            float S0 = sa.x, S1 = sa.y, S2 = sa.z, S3 = sa.w, S4 = sb.x, S5 = sb.y;
            float tanx = FD(FM(0.5f, (float)c.width), c.fx);
            float tany = FD(FM(0.5f, (float)c.height), c.fy);
            float limx = FM(1.3f, tanx), limy = FM(1.3f, tany);
            float xz = FD(tx, tz), yz = FD(ty, tz);
            float cxz = fminf(limx, fmaxf(-limx, xz));
            float cyz = fminf(limy, fmaxf(-limy, yz));
            float j00 = FD(c.fx, tz), j02 = FD(-FM(c.fx, cxz), tz);
            float j11 = FD(c.fy, tz), j12 = FD(-FM(c.fy, cyz), tz);
            float a0 = FA(FM(j00, R[0]), FM(j02, R[6]));
            float a1 = FA(FM(j00, R[1]), FM(j02, R[7]));
            float a2 = FA(FM(j00, R[2]), FM(j02, R[8]));
            float b0 = FA(FM(j11, R[3]), FM(j12, R[6]));
            float b1 = FA(FM(j11, R[4]), FM(j12, R[7]));
            float b2 = FA(FM(j11, R[5]), FM(j12, R[8]));
            float va0 = FA(FA(FM(a0, S0), FM(a1, S1)), FM(a2, S2));
            float va1 = FA(FA(FM(a0, S1), FM(a1, S3)), FM(a2, S4));
            float va2 = FA(FA(FM(a0, S2), FM(a1, S4)), FM(a2, S5));
            float vb0 = FA(FA(FM(b0, S0), FM(b1, S1)), FM(b2, S2));
            float vb1 = FA(FA(FM(b0, S1), FM(b1, S3)), FM(b2, S4));
            float vb2 = FA(FA(FM(b0, S2), FM(b1, S4)), FM(b2, S5));
            float c00 = FA(FA(FA(FM(va0, a0), FM(va1, a1)), FM(va2, a2)), 0.3f);
            float c01 = FA(FA(FM(va0, b0), FM(va1, b1)), FM(va2, b2));
            float c11 = FA(FA(FA(FM(vb0, b0), FM(vb1, b1)), FM(vb2, b2)), 0.3f);
            float det = FS(FM(c00, c11), FM(c01, c01));
            if (det > 0.f) {
                float mid = FM(0.5f, FA(c00, c11));
                float disc = fmaxf(0.1f, FS(FM(mid, mid), det));
                float lam = FA(mid, __fsqrt_rn(disc));
                float r = ceilf(FM(3.f, __fsqrt_rn(lam)));
                float px = FA(FM(c.fx, xz), c.cx);
                float py = FA(FM(c.fy, yz), c.cy);
                float fx0 = floorf(FM(FS(px, r), 0.0625f));
                float fx1 = FA(floorf(FM(FA(px, r), 0.0625f)), 1.f);
                float fy0 = floorf(FM(FS(py, r), 0.0625f));
                float fy1 = FA(floorf(FM(FA(py, r), 0.0625f)), 1.f);
                float ftx = (float)c.tiles_x, fty = (float)c.tiles_y;
                fx0 = fminf(ftx, fmaxf(0.f, fx0));
                fx1 = fminf(ftx, fmaxf(0.f, fx1));
                fy0 = fminf(fty, fmaxf(0.f, fy0));
                fy1 = fminf(fty, fmaxf(0.f, fy1));
                uint32_t x0 = (uint32_t)fx0, x1 = (uint32_t)fx1, y0 = (uint32_t)fy0, y1 = (uint32_t)fy1;
                if (x0 < x1 && y0 < y1) {
                    visible = true;
                    rc = make_uint2(x0 | (x1 << 16), y0 | (y1 << 16));
                    // compositing record: the exponent of alpha in base 2 is
                    //   q2 + log2(o),  q2 = a' dx^2 + b' dx dy + c' dy^2  (d = mu' - pixel)
                    // with (a', b', c') = log2(e) * (-A/2, -B, -C/2) for the conic (A, B, C).
                    // For the compositing kernel's culling: the slopes r1 = -b'/2c', r2 = -b'/2a'
                    // of the lines on which the concave q2 peaks along x and along y, and
                    // t = the floor log2(1/255) less log2(o) and less a rounding margin of the
                    // kernel's tile-local polynomial: 4e-6 S + 0.01 with S a bound on the size of
                    // its terms. In any tile of the rectangle the tile-local mean is within r + 16
                    // of the origin and pixel centres within 16 of it, which gives
                    // S <= |log2 o| + (|a'| + |b'| + |c'|) (r + 32)^2.
                    const float kLog2e = 1.4426950408889634f;
                    const float inv = 1.f / det;
                    const float A = c11 * inv, B = -c01 * inv, C = c00 * inv;
                    const float a2 = -0.5f * kLog2e * A, b2 = -kLog2e * B, c2 = -0.5f * kLog2e * C;
                    const float lo = log2_op[g];
                    const float r1 = -b2 * __frcp_rn(2.f * c2), r2 = -b2 * __frcp_rn(2.f * a2);
                    const float R = r + 32.f;
                    const float S = fabsf(lo) + (fabsf(a2) + fabsf(b2) + fabsf(c2)) * R * R;
                    const float thr = kLog2AlphaMin - fmaf(4e-6f, S, 0.01f);
                    ra = make_float4(px, py, a2, b2);
                    rb = make_float4(c2, lo, r1, r2);
                    rt = lo > -INFINITY ? thr - lo : INFINITY;
                }
            }
        }
        uint32_t o = orig_of_int[g];
        dkey[o] = visible ? __float_as_uint(tz) : kCulled;
        dval[o] = (uint32_t)g;
        rec_a[g] = ra;
        rec_b[g] = rb;
        rec_t[g] = rt;
        rect[g] = rc;
    }
    // one atomic per block (a counter shared by the whole grid)
    __shared__ uint32_t wcnt[8];
    const uint32_t b = __ballot_sync(0xffffffffu, visible);
    if ((threadIdx.x & 31) == 0) wcnt[threadIdx.x >> 5] = (uint32_t)__popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int q = 0; q < 8; ++q) t += wcnt[q];
        if (t) atomicAdd(&ctr->n_visible, t);
    }
}

// r < n_visible: rectangle and bin count of the Gaussian of depth rank r (the records stay in the
// internal order; the compositing kernel reads them through the rank -> Gaussian map).
__global__ void __launch_bounds__(256) gather_sorted_k(const uint32_t *__restrict__ sorted_vals, int64_t n, ViewCounters *ctr,
                                const uint2 *__restrict__ rect, uint2 *__restrict__ srect,
                                uint32_t *__restrict__ stouched, int shift) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t tiles = 0;
    if (r < n) {
        const uint32_t nv = ctr->n_visible;
        if (r < nv) {
            const uint32_t g = sorted_vals[r];
            const uint2 rc = rect[g];
            srect[r] = rc;
            const uint32_t x0 = rc.x & 0xffffu, x1 = rc.x >> 16, y0 = rc.y & 0xffffu, y1 = rc.y >> 16;
            tiles = (x1 - x0) * (y1 - y0);
            stouched[r] = ((((x1 - 1) >> shift) - (x0 >> shift)) + 1) * ((((y1 - 1) >> shift) - (y0 >> shift)) + 1);
        } else {
            stouched[r] = 0;
        }
    }
    // one atomic per block (a counter shared by the whole grid)
    __shared__ unsigned long long wsum[8];
    unsigned long long t = tiles;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long u = 0;
        for (int q = 0; q < 8; ++q) u += wsum[q];
        if (u) atomicAdd(&ctr->P_tiles, u);
    }
}

__global__ void check_seg_k(const int32_t *__restrict__ seg, int64_t npx, int32_t M, ViewCounters *ctr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    for (; i < npx; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = seg[i];
        bad |= (s < -1) || (s >= M);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctr->bad_seg, 1u);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_check_gaussians(const float *means, const float *scales, const float *quats, const float *opac,
                            int64_t n, uint32_t *d_flag, cudaStream_t st) {
    check_gaussians_k<<<blocks_for(n, 256), 256, 0, st>>>(means, scales, quats, opac, n, d_flag); note_launch();
}

void launch_bbox(const float *means, int64_t n, uint32_t *d_bbox6, cudaStream_t st) {
    static const uint32_t init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    cudaMemcpyAsync(d_bbox6, init, sizeof(init), cudaMemcpyHostToDevice, st);
    unsigned nb = blocks_for(n, 256);
    if (nb > 1184) nb = 1184;
    bbox_k<<<nb, 256, 0, st>>>(means, n, d_bbox6); note_launch();
}

void launch_morton(const float *means, int64_t n, const uint32_t *d_bbox6, uint32_t *codes, uint32_t *idx,
                   cudaStream_t st) {
    morton_k<<<blocks_for(n, 256), 256, 0, st>>>(means, n, d_bbox6, codes, idx); note_launch();
}

void launch_pack_gaussians(const float *means, const float *scales, const float *quats, const float *opac,
                           int64_t n, const uint32_t *orig_of_int, float4 *mean_op, float4 *cov_a,
                           float2 *cov_b, uint32_t *int_of_orig, float *log2_op, cudaStream_t st) {
    pack_k<<<blocks_for(n, 256), 256, 0, st>>>(means, scales, quats, opac, n, orig_of_int, mean_op, cov_a,
                                               cov_b, int_of_orig, log2_op); note_launch();
}

void launch_project(const CamParams &cam, const float4 *mean_op, const float *log2_op, const float4 *cov_a,
                    const float2 *cov_b, int64_t n, const uint32_t *orig_of_int, uint32_t *dkey_orig, uint32_t *dval_orig,
                    float4 *rec_a, float4 *rec_b, float *rec_t, uint2 *rect, ViewCounters *ctr, cudaStream_t st,
                    const CamParams *cam_dev) {
    project_k<<<blocks_for(n, 256), 256, 0, st>>>(cam, cam_dev, mean_op, log2_op, cov_a, cov_b, n, orig_of_int, dkey_orig,
                                                  dval_orig, rec_a, rec_b, rec_t, rect, ctr); note_launch();
}

void launch_gather_sorted(const uint32_t *sorted_vals, int64_t n, ViewCounters *ctr, const uint2 *rect, uint2 *srect,
                          uint32_t *stouched, int shift, cudaStream_t st) {
    gather_sorted_k<<<blocks_for(n, 256), 256, 0, st>>>(sorted_vals, n, ctr, rect, srect, stouched, shift);
    note_launch();
}

void launch_check_seg(const int32_t *seg, int64_t npx, int32_t M, ViewCounters *ctr, cudaStream_t st) {
    unsigned nb = blocks_for(npx, 256);
    if (nb > 2368) nb = 2368;
    check_seg_k<<<nb, 256, 0, st>>>(seg, npx, M, ctr); note_launch();
}

}  // namespace slag
