/*
 * Plain CPU oracle for loss-free language lifting onto 3D Gaussians.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product path never
 * calls it and shares no code with it.
 *
 * What it computes (SLAG, Method section, "Semantic Embedding"):
 *   - Rasterizer_SLAG: for each pixel p of view i, the set K_p of Gaussians
 *     that contribute and their weights w_{k,p}. The paper states the splat
 *     kernel exp(-1/2 (p - mu'_k)^T Sigma_k^{-1} (p - mu'_k)) (Eq. 2) and a
 *     "modified Gaussian rasterizer" that captures the weights; the weight
 *     recorded here is the front-to-back compositing weight w = alpha * T
 *     (weight_mode 0), or the raw kernel of Eq. 2 for the same contributing
 *     set (weight_mode 1).
 *   - Parameter Masking: w'_{k,p} = w_{k,p} * M_j(p), with the masks of a view
 *     given as a segment-id map (one id per pixel, -1 = no mask).
 *   - Aggregation: E_k = (sum_i sum_j sum_{p in M_j} w_{k,p} E_j) /
 *     (sum_i sum_j sum_{p in M_j} w_{k,p}). The oracle returns, per view, the
 *     per-(Gaussian, segment) weight sums B[k][j] = sum_{p in M_j} w_{k,p}
 *     (the factored form; the caller forms B.E and sum_j B with a matmul), or
 *     accumulates numerator and denominator one contribution at a time (the
 *     literal form, a D-wide multiply-add per contributing pixel).
 *
 * Precision. Continuous quantities (projected mean, 2D covariance, conic,
 * alpha, transmittance, weights, sums) are float64. The discrete decisions
 * whose outcome is an integer (visibility, tile rectangle, depth order, and
 * whether a Gaussian's alpha reaches the floor 1/255 at a pixel) are taken in
 * float32 by a mirror written out below with a fixed operation order (build
 * with -ffp-contract=off; fused multiply-adds only where written as fmaf);
 * tile lists are sorted by (float32 depth, Gaussian index). The floor test
 * compares the base-2 exponent of alpha, log2(o) - (log2 e / 2) q, with
 * log2(1/255), evaluating it as a quadratic polynomial in the pixel centre's
 * offset from its tile's origin, with log2(o) rounded from float64. The stop
 * test (transmittance below 1e-4) is taken in float64. The paper gives no rasterizer constants; the ones used are: 2D
 * dilation 0.3, radius ceil(3 sqrt(lambda_max)) with the eigenvalue
 * discriminant floored at 0.1, Jacobian clamp 1.3 * tan(half fov), alpha cap
 * 0.99, alpha floor 1/255 (skip), stop when the next transmittance would fall
 * below 1e-4 (that Gaussian is not composited), pixel centres at +0.5,
 * 16x16-pixel tiles, tile rectangle [floor((mu'-r)/16), floor((mu'+r)/16)+1)
 * clamped to the tile grid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TILE 16

typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
    float R[9];   /* world -> camera, row-major */
    float t[3];
    float near_z, far_z;
} ocam;

/* ------------------------------------------------------------------------- */
/* float32 mirror: visibility, depth, tile rectangle                          */
/* ------------------------------------------------------------------------- */

/* World covariance Sigma = M M^T with M = R(q) diag(s), q normalised. */
static void cov3_f32(const float *s, const float *q, float out[6]) {
    float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    float qq = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
    float qn = sqrtf(qq);
    float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float r[9];
    r[0] = 1.0f - 2.0f * (yy + zz); r[1] = 2.0f * (xy - wz);        r[2] = 2.0f * (xz + wy);
    r[3] = 2.0f * (xy + wz);        r[4] = 1.0f - 2.0f * (xx + zz); r[5] = 2.0f * (yz - wx);
    r[6] = 2.0f * (xz - wy);        r[7] = 2.0f * (yz + wx);        r[8] = 1.0f - 2.0f * (xx + yy);
    float m[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m[i * 3 + j] = r[i * 3 + j] * s[j];
    out[0] = (m[0] * m[0] + m[1] * m[1]) + m[2] * m[2];
    out[1] = (m[0] * m[3] + m[1] * m[4]) + m[2] * m[5];
    out[2] = (m[0] * m[6] + m[1] * m[7]) + m[2] * m[8];
    out[3] = (m[3] * m[3] + m[4] * m[4]) + m[5] * m[5];
    out[4] = (m[3] * m[6] + m[4] * m[7]) + m[5] * m[8];
    out[5] = (m[6] * m[6] + m[7] * m[7]) + m[8] * m[8];
}

/* Returns tiles touched (0 = culled); writes depth and rect [x0,y0,x1,y1), and, when rec is
 * non-null, the float32 floor-test record (projected mean, then the conic scaled to base-2
 * exponent coefficients: -(log2 e / 2) A, -(log2 e) B, -(log2 e / 2) C for the conic (A, B, C)). */
static uint32_t bin_one_f32(const float *mu, const float *s, const float *q, const ocam *c,
                            float *depth, int32_t rect[4], float *rec) {
    const float *R = c->R;
    float tx = ((R[0] * mu[0] + R[1] * mu[1]) + R[2] * mu[2]) + c->t[0];
    float ty = ((R[3] * mu[0] + R[4] * mu[1]) + R[5] * mu[2]) + c->t[1];
    float tz = ((R[6] * mu[0] + R[7] * mu[1]) + R[8] * mu[2]) + c->t[2];
    *depth = tz;
    rect[0] = rect[1] = rect[2] = rect[3] = 0;
    if (!(tz > c->near_z) || !(tz < c->far_z)) return 0;
    float S[6];
    cov3_f32(s, q, S);
    float tanx = (0.5f * (float)c->width) / c->fx;
    float tany = (0.5f * (float)c->height) / c->fy;
    float limx = 1.3f * tanx, limy = 1.3f * tany;
    float xz = tx / tz, yz = ty / tz;
    float cxz = fminf(limx, fmaxf(-limx, xz));
    float cyz = fminf(limy, fmaxf(-limy, yz));
    float j00 = c->fx / tz, j02 = -(c->fx * cxz) / tz;
    float j11 = c->fy / tz, j12 = -(c->fy * cyz) / tz;
    float a0 = j00 * R[0] + j02 * R[6], a1 = j00 * R[1] + j02 * R[7], a2 = j00 * R[2] + j02 * R[8];
    float b0 = j11 * R[3] + j12 * R[6], b1 = j11 * R[4] + j12 * R[7], b2 = j11 * R[5] + j12 * R[8];
    float va0 = (a0 * S[0] + a1 * S[1]) + a2 * S[2];
    float va1 = (a0 * S[1] + a1 * S[3]) + a2 * S[4];
    float va2 = (a0 * S[2] + a1 * S[4]) + a2 * S[5];
    float vb0 = (b0 * S[0] + b1 * S[1]) + b2 * S[2];
    float vb1 = (b0 * S[1] + b1 * S[3]) + b2 * S[4];
    float vb2 = (b0 * S[2] + b1 * S[4]) + b2 * S[5];
    float c00 = ((va0 * a0 + va1 * a1) + va2 * a2) + 0.3f;
    float c01 = (va0 * b0 + va1 * b1) + va2 * b2;
    float c11 = ((vb0 * b0 + vb1 * b1) + vb2 * b2) + 0.3f;
    float det = c00 * c11 - c01 * c01;
    if (!(det > 0.0f)) return 0;
    float mid = 0.5f * (c00 + c11);
    float disc = fmaxf(0.1f, mid * mid - det);
    float lam = mid + sqrtf(disc);
    float r = ceilf(3.0f * sqrtf(lam));
    float px = c->fx * xz + c->cx;
    float py = c->fy * yz + c->cy;
    int32_t tilesx = (c->width + TILE - 1) / TILE, tilesy = (c->height + TILE - 1) / TILE;
    float fx0 = floorf((px - r) * 0.0625f), fx1 = floorf((px + r) * 0.0625f) + 1.0f;
    float fy0 = floorf((py - r) * 0.0625f), fy1 = floorf((py + r) * 0.0625f) + 1.0f;
    fx0 = fminf((float)tilesx, fmaxf(0.0f, fx0));
    fx1 = fminf((float)tilesx, fmaxf(0.0f, fx1));
    fy0 = fminf((float)tilesy, fmaxf(0.0f, fy0));
    fy1 = fminf((float)tilesy, fmaxf(0.0f, fy1));
    int32_t x0 = (int32_t)fx0, x1 = (int32_t)fx1, y0 = (int32_t)fy0, y1 = (int32_t)fy1;
    if (x0 >= x1 || y0 >= y1) return 0;
    rect[0] = x0; rect[1] = y0; rect[2] = x1; rect[3] = y1;
    if (rec) {
        const float kLog2e = 1.4426950408889634f;
        float inv = 1.0f / det;
        float A = c11 * inv, B = -c01 * inv, C = c00 * inv;
        rec[0] = px;
        rec[1] = py;
        rec[2] = -0.5f * kLog2e * A;
        rec[3] = -kLog2e * B;
        rec[4] = -0.5f * kLog2e * C;
    }
    return (uint32_t)((x1 - x0) * (y1 - y0));
}

/* log2 of an opacity, rounded to float32 from float64 (-inf for 0). */
static float log2_opacity_f32(float o) { return o > 0.0f ? (float)log2((double)o) : -INFINITY; }

/* Whether alpha reaches the floor 1/255 at the pixel centre (X, Y) = (pixel - tile origin) + 0.5
 * of tile origin (ox, oy), in float32: the exponent e = q2 + log2 o, q2 = a' dx^2 + b' dx dy +
 * c' dy^2 with d = (mean - origin) - (X, Y), expanded as K0 + K1 X + K2 Y + a' X^2 + b' X Y +
 * c' Y^2 and evaluated in that order (Horner form by fused multiply-adds). */
static int floor_reached_f32(const float *rec, float lo, float ox, float oy, float X, float Y) {
    const float mx = rec[0] - ox, my = rec[1] - oy;
    const float A = rec[2], Bc = rec[3], C = rec[4];
    const float K1 = -fmaf(2.0f * A, mx, Bc * my);
    const float K2 = -fmaf(Bc, mx, 2.0f * C * my);
    const float K0 = fmaf(fmaf(A, mx, Bc * my), mx, fmaf(C * my, my, lo));
    const float XX = X * X, XY = X * Y, YY = Y * Y;
    const float e = fmaf(C, YY, fmaf(Bc, XY, fmaf(A, XX, fmaf(K2, Y, fmaf(K1, X, K0)))));
    return e >= -7.99435343685886f;   /* log2(1/255) */
}

void oracle_bin_f32(int64_t n, const float *means, const float *scales, const float *quats,
                    const ocam *cam, float *depth, int32_t *rect, uint32_t *touched) {
    for (int64_t k = 0; k < n; ++k)
        touched[k] = bin_one_f32(means + 3 * k, scales + 3 * k, quats + 4 * k, cam, depth + k,
                                 rect + 4 * k, NULL);
}

/* ------------------------------------------------------------------------- */
/* per-tile lists sorted by (float32 depth, index)                            */
/* ------------------------------------------------------------------------- */

typedef struct { float d; int32_t k; } dk_t;

static int cmp_dk(const void *a, const void *b) {
    const dk_t *x = (const dk_t *)a, *y = (const dk_t *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->k > y->k) - (x->k < y->k);
}

typedef struct {
    int32_t tilesx, tilesy;
    int64_t P;
    int64_t *start;   /* tiles + 1 */
    dk_t *items;      /* P */
} tile_lists;

/* Lists of the tiles in rows [ty0, ty1) of the tile grid (the others stay empty). */
static int build_lists(int64_t n, const float *depth, const int32_t *rect, const uint32_t *touched,
                       const ocam *c, int32_t ty0, int32_t ty1, tile_lists *L) {
    L->tilesx = (c->width + TILE - 1) / TILE;
    L->tilesy = (c->height + TILE - 1) / TILE;
    int64_t T = (int64_t)L->tilesx * L->tilesy;
    L->start = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
    if (!L->start) return -1;
    for (int64_t k = 0; k < n; ++k) {
        if (!touched[k]) continue;
        for (int32_t y = rect[4 * k + 1]; y < rect[4 * k + 3]; ++y) {
            if (y < ty0 || y >= ty1) continue;
            for (int32_t x = rect[4 * k]; x < rect[4 * k + 2]; ++x) L->start[(int64_t)y * L->tilesx + x + 1]++;
        }
    }
    for (int64_t t = 0; t < T; ++t) L->start[t + 1] += L->start[t];
    L->P = L->start[T];
    L->items = (dk_t *)malloc(sizeof(dk_t) * (size_t)(L->P > 0 ? L->P : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)T);
    if (!L->items || !fill) { free(fill); return -1; }
    memcpy(fill, L->start, sizeof(int64_t) * (size_t)T);
    for (int64_t k = 0; k < n; ++k) {
        if (!touched[k]) continue;
        for (int32_t y = rect[4 * k + 1]; y < rect[4 * k + 3]; ++y) {
            if (y < ty0 || y >= ty1) continue;
            for (int32_t x = rect[4 * k]; x < rect[4 * k + 2]; ++x) {
                int64_t t = (int64_t)y * L->tilesx + x;
                L->items[fill[t]].d = depth[k];
                L->items[fill[t]].k = (int32_t)k;
                fill[t]++;
            }
        }
    }
    free(fill);
    for (int64_t t = 0; t < T; ++t)
        qsort(L->items + L->start[t], (size_t)(L->start[t + 1] - L->start[t]), sizeof(dk_t), cmp_dk);
    return 0;
}

static void free_lists(tile_lists *L) { free(L->start); free(L->items); }

/* Full per-tile lists: list_out[P] = Gaussian index, ranges[2*T] = [start, end). Returns P
 * (or -1 on allocation failure / -(P+2) when cap < P, nothing written). */
int64_t oracle_tile_lists_f32(int64_t n, const float *means, const float *scales, const float *quats,
                              const ocam *cam, int64_t cap, int32_t *list_out, int64_t *ranges) {
    float *depth = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    int32_t *rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!depth || !rect || !touched) { free(depth); free(rect); free(touched); return -1; }
    oracle_bin_f32(n, means, scales, quats, cam, depth, rect, touched);
    tile_lists L;
    if (build_lists(n, depth, rect, touched, cam, 0, (cam->height + TILE - 1) / TILE, &L)) {
        free(depth); free(rect); free(touched); return -1;
    }
    int64_t P = L.P;
    if (cap >= P) {
        for (int64_t i = 0; i < P; ++i) list_out[i] = L.items[i].k;
        int64_t T = (int64_t)L.tilesx * L.tilesy;
        for (int64_t t = 0; t < T; ++t) { ranges[2 * t] = L.start[t]; ranges[2 * t + 1] = L.start[t + 1]; }
    }
    free_lists(&L); free(depth); free(rect); free(touched);
    return cap >= P ? P : -(P + 2);
}

/* ------------------------------------------------------------------------- */
/* float64 projection                                                         */
/* ------------------------------------------------------------------------- */

typedef struct { double mx, my, A, B, C, op, c00, c01, c11, depth; } proj64;

static void project_f64(const float *mu, const float *s, const float *q, float op, const ocam *c,
                        proj64 *o) {
    const float *Rf = c->R;
    double R[9];
    for (int i = 0; i < 9; ++i) R[i] = Rf[i];
    double tx = R[0] * mu[0] + R[1] * mu[1] + R[2] * mu[2] + c->t[0];
    double ty = R[3] * mu[0] + R[4] * mu[1] + R[5] * mu[2] + c->t[1];
    double tz = R[6] * mu[0] + R[7] * mu[1] + R[8] * mu[2] + c->t[2];
    double qn = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
    double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    double r[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                   2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                   2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    double S[9];  /* world covariance r diag(s^2) r^T */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += r[i * 3 + k] * (double)s[k] * (double)s[k] * r[j * 3 + k];
            S[i * 3 + j] = acc;
        }
    double tanx = 0.5 * c->width / (double)c->fx, tany = 0.5 * c->height / (double)c->fy;
    double limx = 1.3 * tanx, limy = 1.3 * tany;
    double xz = tx / tz, yz = ty / tz;
    double cxz = fmin(limx, fmax(-limx, xz)), cyz = fmin(limy, fmax(-limy, yz));
    /* Jacobian of (fx x/z + cx, fy y/z + cy) at the (clamped) mean */
    double J[6] = {c->fx / tz, 0.0, -c->fx * cxz / tz, 0.0, c->fy / tz, -c->fy * cyz / tz};
    double Tm[6];  /* J R */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) Tm[i * 3 + j] = J[i * 3] * R[j] + J[i * 3 + 1] * R[3 + j] + J[i * 3 + 2] * R[6 + j];
    double C2[4];  /* Tm S Tm^T */
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 2; ++k) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += Tm[i * 3 + a] * S[a * 3 + b] * Tm[k * 3 + b];
            C2[i * 2 + k] = acc;
        }
    double a = C2[0] + 0.3, b = C2[1], cc = C2[3] + 0.3;
    double det = a * cc - b * b;
    o->A = cc / det; o->B = -b / det; o->C = a / det;
    o->c00 = a; o->c01 = b; o->c11 = cc; o->depth = tz;
    o->mx = c->fx * xz + c->cx;
    o->my = c->fy * yz + c->cy;
    o->op = op;
}

/* Per Gaussian: projected mean, conic, opacity, 2D covariance (dilated), depth:
 * out[10*k + (0..9)] = mx, my, A, B, C, opacity, c00, c01, c11, depth. */
void oracle_project_f64(int64_t n, const float *means, const float *scales, const float *quats,
                        const float *opac, const ocam *cam, double *out) {
    for (int64_t k = 0; k < n; ++k) {
        proj64 p;
        project_f64(means + 3 * k, scales + 3 * k, quats + 4 * k, opac[k], cam, &p);
        double *o = out + 10 * k;
        o[0] = p.mx; o[1] = p.my; o[2] = p.A; o[3] = p.B; o[4] = p.C; o[5] = p.op;
        o[6] = p.c00; o[7] = p.c01; o[8] = p.c11; o[9] = p.depth;
    }
}

/* ------------------------------------------------------------------------- */
/* compositing                                                                */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t n;
    const float *means, *scales, *quats, *opac;
    const ocam *cam;
    const int32_t *seg;
    int32_t M;
    int weight_mode;
    int32_t ty0, ty1;   /* tile rows composited: [ty0, ty1) */
} view_in;

/* Composite every pixel of one view front to back. For each contributing
 * (Gaussian, pixel) with the pixel in segment j >= 0, calls sink(k, j, w).
 * Optional per-pixel outputs: final transmittance, sum of weights over all
 * contributing Gaussians (masked or not), number of contributions.
 * tile_mask (nullable): only tiles with a non-zero entry are composited; only the
 * tile rows [v->ty0, v->ty1) are composited in any case (a bounded sample of a
 * view: the pixels of those rows get exactly the results of the whole view). */
typedef void (*sink_fn)(void *ctx, int32_t k, int32_t j, double w);

static int composite_view(const view_in *v, const uint8_t *tile_mask, sink_fn sink, void *sctx,
                          double *T_final, double *wsum_px, int32_t *count_px, int64_t *stats) {
    int64_t n = v->n;
    float *depth = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    int32_t *rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    proj64 *pj = (proj64 *)malloc(sizeof(proj64) * (size_t)(n > 0 ? n : 1));
    float *rec = (float *)malloc(sizeof(float) * 6 * (size_t)(n > 0 ? n : 1));   /* floor-test record, log2 o */
    if (!depth || !rect || !touched || !pj || !rec) {
        free(depth); free(rect); free(touched); free(pj); free(rec); return -1;
    }
    for (int64_t k = 0; k < n; ++k) {
        touched[k] = bin_one_f32(v->means + 3 * k, v->scales + 3 * k, v->quats + 4 * k, v->cam, depth + k,
                                 rect + 4 * k, rec + 6 * k);
        rec[6 * k + 5] = log2_opacity_f32(v->opac[k]);
        if (touched[k]) project_f64(v->means + 3 * k, v->scales + 3 * k, v->quats + 4 * k, v->opac[k], v->cam, pj + k);
    }
    tile_lists L;
    if (build_lists(n, depth, rect, touched, v->cam, v->ty0, v->ty1, &L)) {
        free(depth); free(rect); free(touched); free(pj); free(rec); return -1;
    }
    const int32_t W = v->cam->width, H = v->cam->height;
    int64_t contributions = 0;
    for (int32_t ty = v->ty0; ty < v->ty1 && ty < L.tilesy; ++ty)
        for (int32_t tx = 0; tx < L.tilesx; ++tx) {
            int64_t t = (int64_t)ty * L.tilesx + tx;
            if (tile_mask && !tile_mask[t]) continue;
            for (int32_t py = ty * TILE; py < ty * TILE + TILE && py < H; ++py)
                for (int32_t px = tx * TILE; px < tx * TILE + TILE && px < W; ++px) {
                    double T = 1.0, wsum = 0.0;
                    int32_t cnt = 0;
                    int32_t j = v->seg ? v->seg[(int64_t)py * W + px] : -1;
                    double cxp = px + 0.5, cyp = py + 0.5;
                    const float ox = (float)(tx * TILE), oy = (float)(ty * TILE);
                    const float X = (float)(px - tx * TILE) + 0.5f, Y = (float)(py - ty * TILE) + 0.5f;
                    for (int64_t i = L.start[t]; i < L.start[t + 1]; ++i) {
                        const int32_t k = L.items[i].k;
                        const proj64 *g = pj + k;
                        double dx = g->mx - cxp, dy = g->my - cyp;
                        double power = -0.5 * (g->A * dx * dx + g->C * dy * dy) - g->B * dx * dy;
                        if (power > 0.0) continue;
                        if (!floor_reached_f32(rec + 6 * k, rec[6 * k + 5], ox, oy, X, Y)) continue;
                        double kern = exp(power);
                        double alpha = fmin(0.99, g->op * kern);
                        double Tn = T * (1.0 - alpha);
                        if (Tn < 1e-4) break;
                        double w = v->weight_mode == 1 ? kern : alpha * T;
                        if (j >= 0 && sink) sink(sctx, L.items[i].k, j, w);
                        wsum += w;
                        ++cnt;
                        T = Tn;
                    }
                    contributions += cnt;
                    int64_t pi = (int64_t)py * W + px;
                    if (T_final) T_final[pi] = T;
                    if (wsum_px) wsum_px[pi] = wsum;
                    if (count_px) count_px[pi] = cnt;
                }
        }
    if (stats) { stats[0] = L.P; stats[1] = contributions; }
    free_lists(&L); free(depth); free(rect); free(touched); free(pj); free(rec);
    return 0;
}

/* --- factored form: per-(Gaussian, segment) weight sums of one view ------- */

typedef struct { const int64_t *sub_of; int32_t M; double *B; } fact_ctx;

static void fact_sink(void *c, int32_t k, int32_t j, double w) {
    fact_ctx *f = (fact_ctx *)c;
    int64_t s = f->sub_of ? f->sub_of[k] : k;
    if (s < 0) return;
    f->B[s * f->M + j] += w;
}

/* B (n_sub x M) += per-(Gaussian, segment) sums of masked weights for one view,
 * over the pixels of tile rows [ty0, ty1) (the whole view: 0 and the tile-grid
 * height). sub_ids (nullable): accumulate only for these Gaussians (row r of B
 * is Gaussian sub_ids[r]); tiles not touched by any of them are skipped.
 * Returns 0, -1 on allocation failure, -2 on a segment id outside [-1, M). */
int oracle_view_weights_rows(int64_t n, const float *means, const float *scales, const float *quats,
                             const float *opac, const ocam *cam, const int32_t *seg, int32_t M,
                             int weight_mode, int64_t n_sub, const int64_t *sub_ids, double *B,
                             double *T_final, double *wsum_px, int32_t *count_px, int64_t *stats,
                             int32_t ty0, int32_t ty1) {
    int64_t npx = (int64_t)cam->width * cam->height;
    for (int64_t p = 0; p < npx; ++p)
        if (seg && (seg[p] < -1 || seg[p] >= M)) return -2;
    view_in v = {n, means, scales, quats, opac, cam, seg, M, weight_mode, ty0, ty1};
    int64_t *sub_of = NULL;
    uint8_t *tile_mask = NULL;
    if (sub_ids) {
        sub_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        int32_t tilesx = (cam->width + TILE - 1) / TILE, tilesy = (cam->height + TILE - 1) / TILE;
        tile_mask = (uint8_t *)calloc((size_t)tilesx * tilesy, 1);
        if (!sub_of || !tile_mask) { free(sub_of); free(tile_mask); return -1; }
        for (int64_t k = 0; k < n; ++k) sub_of[k] = -1;
        for (int64_t r = 0; r < n_sub; ++r) {
            int64_t k = sub_ids[r];
            sub_of[k] = r;
            float d; int32_t rc[4];
            if (bin_one_f32(means + 3 * k, scales + 3 * k, quats + 4 * k, cam, &d, rc, NULL))
                for (int32_t y = rc[1]; y < rc[3]; ++y)
                    for (int32_t x = rc[0]; x < rc[2]; ++x) tile_mask[(int64_t)y * tilesx + x] = 1;
        }
    }
    fact_ctx f = {sub_of, M, B};
    int rc = composite_view(&v, tile_mask, fact_sink, &f, T_final, wsum_px, count_px, stats);
    free(sub_of); free(tile_mask);
    return rc;
}

/* The whole view. */
int oracle_view_weights(int64_t n, const float *means, const float *scales, const float *quats,
                        const float *opac, const ocam *cam, const int32_t *seg, int32_t M,
                        int weight_mode, int64_t n_sub, const int64_t *sub_ids, double *B,
                        double *T_final, double *wsum_px, int32_t *count_px, int64_t *stats) {
    return oracle_view_weights_rows(n, means, scales, quats, opac, cam, seg, M, weight_mode, n_sub, sub_ids, B,
                                    T_final, wsum_px, count_px, stats, 0, (cam->height + TILE - 1) / TILE);
}

/* --- literal form: one D-wide multiply-add per contributing pixel --------- */

typedef struct { const float *table; int32_t D; double *num; double *den; } lit_ctx;

static void lit_sink(void *c, int32_t k, int32_t j, double w) {
    lit_ctx *l = (lit_ctx *)c;
    const float *e = l->table + (int64_t)j * l->D;
    double *a = l->num + (int64_t)k * l->D;
    for (int32_t d = 0; d < l->D; ++d) a[d] += w * (double)e[d];
    l->den[k] += w;
}

/* num (n x D) += sum_p w_{k,p} E_{seg(p)}, den (n) += sum_p w_{k,p}, for one view. */
int oracle_view_literal(int64_t n, const float *means, const float *scales, const float *quats,
                        const float *opac, const ocam *cam, const int32_t *seg, int32_t M,
                        const float *table, int32_t D, int weight_mode, double *num, double *den) {
    int64_t npx = (int64_t)cam->width * cam->height;
    for (int64_t p = 0; p < npx; ++p)
        if (seg && (seg[p] < -1 || seg[p] >= M)) return -2;
    view_in v = {n, means, scales, quats, opac, cam, seg, M, weight_mode, 0, (cam->height + TILE - 1) / TILE};
    lit_ctx l = {table, D, num, den};
    return composite_view(&v, NULL, lit_sink, &l, NULL, NULL, NULL, NULL);
}
