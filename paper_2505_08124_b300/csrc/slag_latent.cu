// The latent form's autoencoder: parameter layout, inference and training
// (C ABI: slag_latent_param_count, slag_latent_train, slag_latent_apply).
//
// Architecture for input width D: enc(x) = W2^T gelu(W1^T x + b1) + b2 and
// dec(z) = W4^T gelu(W3^T z + b3) + b4 with W1: D x 256, W2: 256 x 32,
// W3: 32 x 256, W4: 256 x D (row-major, input x output), erf-GELU. The
// products take the weights rounded to bfloat16 with float32 accumulation;
// training keeps float32 masters and updates them with Adam (beta 0.9 / 0.999,
// eps 1e-8) on the per-sample loss mean((dec(enc(x)) - x)^2) + (1 - cos).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "slag_internal.cuh"

namespace slag {

LatentLayout latent_layout(int32_t D) {
    const int64_t H = kLatentHidden, L = kLatent;
    LatentLayout o;
    int64_t at = 0;
    o.W1 = at; at += (int64_t)D * H;
    o.b1 = at; at += H;
    o.W2 = at; at += H * L;
    o.b2 = at; at += L;
    o.W3 = at; at += L * H;
    o.b3 = at; at += H;
    o.W4 = at; at += H * D;
    o.b4 = at; at += D;
    o.total = at;
    return o;
}

void latent_encode(const float *p, int32_t D, const float *X, int rows, float *hidden, float *Z, cudaStream_t st) {
    const LatentLayout o = latent_layout(D);
    latent_gemm(false, false, rows, kLatentHidden, D, X, D, p + o.W1, kLatentHidden, hidden, kLatentHidden, p + o.b1,
                true, nullptr, false, true, false, st);
    latent_gemm(false, false, rows, kLatent, kLatentHidden, hidden, kLatentHidden, p + o.W2, kLatent, Z, kLatent,
                p + o.b2, false, nullptr, false, true, false, st);
}

int64_t latent_decode_scratch(int rows, int32_t D) {
    const int64_t rp = dense_tc_pad_rows(rows);
    return rp * 2 * (kLatent + kLatentHidden) + (int64_t)kLatentHidden * kLatent + (int64_t)D * kLatentHidden;
}

// The decoder on the tensor cores (k_dense_tc.cu): the codes' TF32 planes, then
// gelu(Z W3 + b3) as the TF32 planes of the hidden layer, then H W4 + b4 as float32 rows.
cudaError_t latent_decode(const float *p, int32_t D, const float *Z, int rows, float *scratch, float *Y,
                          uint32_t *err, cudaStream_t st) {
    const LatentLayout o = latent_layout(D);
    const int64_t rp = dense_tc_pad_rows(rows);
    float *Zp = scratch;                                   // 2 x rp x kLatent
    float *Hp = Zp + rp * 2 * kLatent;                     // 2 x rp x kLatentHidden
    float *W3t = Hp + rp * 2 * kLatentHidden;              // kLatentHidden x kLatent
    float *W4t = W3t + (int64_t)kLatentHidden * kLatent;   // D x kLatentHidden
    launch_tf32_planes(Z, rows, rp, kLatent, Zp, st);
    launch_weights_t(p + o.W3, kLatent, kLatentHidden, W3t, st);
    launch_weights_t(p + o.W4, kLatentHidden, D, W4t, st);
    cudaError_t e = launch_dense_tc(Zp, rows, rp, kLatent, W3t, kLatentHidden, p + o.b3, true, Hp, 0, err, st);
    if (e != cudaSuccess) return e;
    return launch_dense_tc(Hp, rows, rp, kLatentHidden, W4t, D, p + o.b4, false, Y, D, err, st);
}

int64_t linear_param_count(int32_t D) { return (int64_t)D * (kLatent + 1); }

void linear_encode(const float *params, const float *enc_bias, int32_t D, const float *X, int rows, float *Z,
                   cudaStream_t st) {
    latent_gemm(false, false, rows, kLatent, D, X, D, params, kLatent, Z, kLatent, enc_bias, false, nullptr, false, false,
                false, st);
}

int64_t linear_decode_scratch(int rows, int32_t D) {
    return dense_tc_pad_rows(rows) * 2 * kLatent + 2 * (int64_t)D * kLatent;
}

// The dense layer takes its weights transposed, output x input: for the decoder (input 32, output
// D) that is U itself (D x 32), rounded to TF32 (the first of its two TF32 planes).
cudaError_t linear_decode(const float *params, int32_t D, const float *Z, int rows, float *scratch, float *Y,
                          uint32_t *err, cudaStream_t st) {
    const int64_t rp = dense_tc_pad_rows(rows);
    float *Zp = scratch;                         // 2 x rp x kLatent
    float *Up = Zp + rp * 2 * kLatent;           // 2 x D x kLatent: U rounded to TF32, then the rest
    launch_tf32_planes(Z, rows, rp, kLatent, Zp, st);
    launch_tf32_planes(params, D, D, kLatent, Up, st);
    return launch_dense_tc(Zp, rows, rp, kLatent, Up, D, params + (int64_t)D * kLatent, false, Y, D, err, st);
}

}  // namespace slag

using namespace slag;

namespace {

// Symmetric eigenpairs of a small matrix by cyclic Jacobi rotations (float64): A (k x k, row-major,
// overwritten) -> eigenvalues in w, eigenvectors in the columns of V.
void jacobi_eigen(std::vector<double> &A, int k, std::vector<double> &w, std::vector<double> &V) {
    V.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) V[(size_t)i * k + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) off += A[(size_t)p * k + q] * A[(size_t)p * k + q];
        if (off < 1e-30) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = A[(size_t)p * k + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double app = A[(size_t)p * k + p], aqq = A[(size_t)q * k + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {   // A <- A J (columns p, q)
                    const double arp = A[(size_t)r * k + p], arq = A[(size_t)r * k + q];
                    A[(size_t)r * k + p] = c * arp - s * arq;
                    A[(size_t)r * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {   // A <- J^T A (rows p, q)
                    const double apr = A[(size_t)p * k + r], aqr = A[(size_t)q * k + r];
                    A[(size_t)p * k + r] = c * apr - s * aqr;
                    A[(size_t)q * k + r] = s * apr + c * aqr;
                }
                for (int r = 0; r < k; ++r) {   // V <- V J
                    const double vrp = V[(size_t)r * k + p], vrq = V[(size_t)r * k + q];
                    V[(size_t)r * k + p] = c * vrp - s * vrq;
                    V[(size_t)r * k + q] = s * vrp + c * vrq;
                }
            }
    }
    w.resize((size_t)k);
    for (int i = 0; i < k; ++i) w[(size_t)i] = A[(size_t)i * k + i];
}

// Orthonormal columns of V (D x k, row-major) by modified Gram-Schmidt.
void orthonormalise(std::vector<double> &V, int D, int k) {
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i < j; ++i) {
            double d = 0.0;
            for (int r = 0; r < D; ++r) d += V[(size_t)r * k + i] * V[(size_t)r * k + j];
            for (int r = 0; r < D; ++r) V[(size_t)r * k + j] -= d * V[(size_t)r * k + i];
        }
        double nrm = 0.0;
        for (int r = 0; r < D; ++r) nrm += V[(size_t)r * k + j] * V[(size_t)r * k + j];
        nrm = std::sqrt(nrm);
        for (int r = 0; r < D; ++r) V[(size_t)r * k + j] = nrm > 0 ? V[(size_t)r * k + j] / nrm : 0.0;
    }
}

}  // namespace

namespace {

template <typename T>
cudaError_t dmalloc(T **p, int64_t count) {
    *p = nullptr;
    return cudaMalloc((void **)p, sizeof(T) * (size_t)(count > 0 ? count : 1));
}

}  // namespace

extern "C" {

int64_t slag_latent_param_count(int32_t dim) { return dim >= 32 ? latent_layout(dim).total : 0; }

int64_t slag_linear_param_count(int32_t dim) { return dim >= 32 ? linear_param_count(dim) : 0; }

slag_status slag_linear_code_fit(const float *samples, int64_t n, int32_t dim, int32_t on_device, float *out_params,
                                 float *out_kept, void *cuda_stream) {
    if (!samples || !out_params || n < 2 || n >= (1LL << 31) || dim < 32 || dim > 4096 || dim % 32 != 0)
        return SLAG_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int D = dim, k = kLatent;
    float *dX = nullptr, *dsum = nullptr, *dC = nullptr;
    auto cleanup = [&]() {
        if (dX && !on_device) cudaFree(dX);
        if (dsum) cudaFree(dsum);
        if (dC) cudaFree(dC);
    };
#define CF(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            cleanup();                                                                                   \
            return e_ == cudaErrorMemoryAllocation ? SLAG_ERR_OOM : SLAG_ERR_CUDA;                       \
        }                                                                                                \
    } while (0)
    if (on_device) {
        dX = const_cast<float *>(samples);
    } else {
        CF(dmalloc(&dX, n * D));
        CF(cudaMemcpyAsync(dX, samples, sizeof(float) * (size_t)(n * D), cudaMemcpyHostToDevice, st));
    }
    CF(dmalloc(&dsum, D));
    CF(dmalloc(&dC, (int64_t)D * D));
    // column sums and the second moment X^T X on the device (float32 accumulation)
    latent_colsum(dX, (int)n, D, dsum, st);
    latent_gemm(true, false, D, D, (int)n, dX, D, dX, D, dC, D, nullptr, false, nullptr, false, false, false, st);
    std::vector<float> hs((size_t)D), hC((size_t)D * D);
    CF(cudaMemcpyAsync(hs.data(), dsum, sizeof(float) * D, cudaMemcpyDeviceToHost, st));
    CF(cudaMemcpyAsync(hC.data(), dC, sizeof(float) * (size_t)D * D, cudaMemcpyDeviceToHost, st));
    CF(cudaStreamSynchronize(st));
    CF(cudaGetLastError());
#undef CF
    cleanup();
    // covariance in float64, then its top-k eigenvectors by subspace iteration with a Rayleigh-Ritz
    // step (the principal directions of the samples)
    std::vector<double> mu((size_t)D), C((size_t)D * D);
    for (int i = 0; i < D; ++i) mu[(size_t)i] = (double)hs[(size_t)i] / (double)n;
    double trace = 0.0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            const double c = 0.5 * ((double)hC[(size_t)i * D + j] + (double)hC[(size_t)j * D + i]) / (double)n -
                             mu[(size_t)i] * mu[(size_t)j];
            C[(size_t)i * D + j] = c;
            if (i == j) trace += c;
        }
    std::vector<double> V((size_t)D * k), W((size_t)D * k), H((size_t)k * k), ev, R;
    std::mt19937_64 rng(12345);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (auto &x : V) x = nd(rng);
    orthonormalise(V, D, k);
    std::vector<double> prev((size_t)k, 0.0);
    for (int it = 0; it < 1000; ++it) {
        for (int r = 0; r < D; ++r)
            for (int j = 0; j < k; ++j) {
                double acc = 0.0;
                for (int c = 0; c < D; ++c) acc += C[(size_t)r * D + c] * V[(size_t)c * k + j];
                W[(size_t)r * k + j] = acc;
            }
        // Rayleigh quotients of the current basis, for the convergence test
        double change = 0.0;
        for (int j = 0; j < k; ++j) {
            double q = 0.0;
            for (int r = 0; r < D; ++r) q += V[(size_t)r * k + j] * W[(size_t)r * k + j];
            change = std::max(change, std::fabs(q - prev[(size_t)j]) / std::max(std::fabs(q), 1e-300));
            prev[(size_t)j] = q;
        }
        V.swap(W);
        orthonormalise(V, D, k);
        if (it > 8 && change < 1e-12) break;
    }
    // Rayleigh-Ritz: H = V^T C V, rotate V onto its eigenvectors, largest first
    for (int r = 0; r < D; ++r)
        for (int j = 0; j < k; ++j) {
            double acc = 0.0;
            for (int c = 0; c < D; ++c) acc += C[(size_t)r * D + c] * V[(size_t)c * k + j];
            W[(size_t)r * k + j] = acc;
        }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double acc = 0.0;
            for (int r = 0; r < D; ++r) acc += V[(size_t)r * k + i] * W[(size_t)r * k + j];
            H[(size_t)i * k + j] = acc;
        }
    jacobi_eigen(H, k, ev, R);
    std::vector<int> order((size_t)k);
    for (int i = 0; i < k; ++i) order[(size_t)i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return ev[(size_t)a] > ev[(size_t)b]; });
    double kept = 0.0;
    for (int j = 0; j < k; ++j) {
        const int src = order[(size_t)j];
        kept += ev[(size_t)src];
        for (int r = 0; r < D; ++r) {
            double acc = 0.0;
            for (int i = 0; i < k; ++i) acc += V[(size_t)r * k + i] * R[(size_t)i * k + src];
            out_params[(int64_t)r * k + j] = (float)acc;
        }
    }
    for (int r = 0; r < D; ++r) out_params[(int64_t)D * k + r] = (float)mu[(size_t)r];
    if (out_kept) *out_kept = trace > 0 ? (float)(kept / trace) : 0.f;
    return SLAG_OK;
}

slag_status slag_latent_train(const float *samples, int64_t n, int32_t dim, int32_t epochs, int32_t batch, float lr,
                              uint64_t seed, int32_t on_device, float *out_params, float *out_loss,
                              void *cuda_stream) {
    if (!samples || !out_params || n < 1 || dim < 32 || dim > 4096 || dim % 32 != 0 || epochs < 1 || batch < 1 ||
        !(lr > 0.f) || n >= (1LL << 31))
        return SLAG_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const LatentLayout o = latent_layout(dim);
    const int64_t P = o.total;
    const int Bt = (int)std::min<int64_t>(batch, n);
    const int H = kLatentHidden, L = kLatent, D = dim;

    // initial parameters: uniform(-a, a) with a = sqrt(6 / (fan_in + fan_out)), zero biases
    std::vector<float> h(P, 0.f);
    std::mt19937_64 rng(seed);
    auto init = [&](int64_t at, int fin, int fout) {
        std::uniform_real_distribution<float> u(-sqrtf(6.f / (float)(fin + fout)), sqrtf(6.f / (float)(fin + fout)));
        for (int64_t i = 0; i < (int64_t)fin * fout; ++i) h[at + i] = u(rng);
    };
    init(o.W1, D, H);
    init(o.W2, H, L);
    init(o.W3, L, H);
    init(o.W4, H, D);

    float *dX = nullptr, *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *Xb = nullptr;
    float *H1 = nullptr, *A1 = nullptr, *Z = nullptr, *H3 = nullptr, *A3 = nullptr, *Y = nullptr;
    float *dY = nullptr, *dH3 = nullptr, *dZ = nullptr, *dH1 = nullptr, *loss = nullptr;
    uint32_t *idx = nullptr;
    slag_status rc = SLAG_OK;
    auto cleanup = [&]() {
        float *bufs[] = {p, g, m, v, Xb, H1, A1, Z, H3, A3, Y, dY, dH3, dZ, dH1, loss};
        for (float *b : bufs) if (b) cudaFree(b);
        if (dX && !on_device) cudaFree(dX);
        if (idx) cudaFree(idx);
    };
#define CT(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            cleanup();                                                                                   \
            return e_ == cudaErrorMemoryAllocation ? SLAG_ERR_OOM : SLAG_ERR_CUDA;                       \
        }                                                                                                \
    } while (0)
    if (on_device) {
        dX = const_cast<float *>(samples);
    } else {
        CT(dmalloc(&dX, n * D));
        CT(cudaMemcpyAsync(dX, samples, sizeof(float) * (size_t)(n * D), cudaMemcpyHostToDevice, st));
    }
    CT(dmalloc(&p, P)); CT(dmalloc(&g, P)); CT(dmalloc(&m, P)); CT(dmalloc(&v, P));
    CT(dmalloc(&Xb, (int64_t)Bt * D)); CT(dmalloc(&Y, (int64_t)Bt * D)); CT(dmalloc(&dY, (int64_t)Bt * D));
    CT(dmalloc(&H1, (int64_t)Bt * H)); CT(dmalloc(&A1, (int64_t)Bt * H)); CT(dmalloc(&dH1, (int64_t)Bt * H));
    CT(dmalloc(&H3, (int64_t)Bt * H)); CT(dmalloc(&A3, (int64_t)Bt * H)); CT(dmalloc(&dH3, (int64_t)Bt * H));
    CT(dmalloc(&Z, (int64_t)Bt * L)); CT(dmalloc(&dZ, (int64_t)Bt * L));
    CT(dmalloc(&loss, 1));
    CT(dmalloc(&idx, n));
    CT(cudaMemcpyAsync(p, h.data(), sizeof(float) * (size_t)P, cudaMemcpyHostToDevice, st));
    CT(cudaMemsetAsync(m, 0, sizeof(float) * (size_t)P, st));
    CT(cudaMemsetAsync(v, 0, sizeof(float) * (size_t)P, st));

    std::vector<uint32_t> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    int step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        CT(cudaMemcpyAsync(idx, perm.data(), sizeof(uint32_t) * (size_t)n, cudaMemcpyHostToDevice, st));
        CT(cudaMemsetAsync(loss, 0, sizeof(float), st));
        int64_t seen = 0;
        for (int64_t b0 = 0; b0 + Bt <= n; b0 += Bt) {   // full batches; the tail waits for the next shuffle
            const int B = Bt;
            latent_gather_rows(dX, idx + b0, B, D, Xb, st);
            // forward
            latent_gemm(false, false, B, H, D, Xb, D, p + o.W1, H, H1, H, p + o.b1, true, A1, false, true, false, st);
            latent_gemm(false, false, B, L, H, H1, H, p + o.W2, L, Z, L, p + o.b2, false, nullptr, false, true, false, st);
            latent_gemm(false, false, B, H, L, Z, L, p + o.W3, H, H3, H, p + o.b3, true, A3, false, true, false, st);
            latent_gemm(false, false, B, D, H, H3, H, p + o.W4, D, Y, D, p + o.b4, false, nullptr, false, true, false, st);
            latent_loss(Y, Xb, B, D, dY, loss, st);
            // backward (weights rounded as in the forward pass)
            latent_gemm(true, false, H, D, B, H3, H, dY, D, g + o.W4, D, nullptr, false, nullptr, false, false, false, st);
            latent_colsum(dY, B, D, g + o.b4, st);
            latent_gemm(false, true, B, H, D, dY, D, p + o.W4, D, dH3, H, nullptr, false, nullptr, false, true, false, st);
            latent_gelu_bwd(dH3, A3, (int64_t)B * H, st);
            latent_gemm(true, false, L, H, B, Z, L, dH3, H, g + o.W3, H, nullptr, false, nullptr, false, false, false, st);
            latent_colsum(dH3, B, H, g + o.b3, st);
            latent_gemm(false, true, B, L, H, dH3, H, p + o.W3, H, dZ, L, nullptr, false, nullptr, false, true, false, st);
            latent_gemm(true, false, H, L, B, H1, H, dZ, L, g + o.W2, L, nullptr, false, nullptr, false, false, false, st);
            latent_colsum(dZ, B, L, g + o.b2, st);
            latent_gemm(false, true, B, H, L, dZ, L, p + o.W2, L, dH1, H, nullptr, false, nullptr, false, true, false, st);
            latent_gelu_bwd(dH1, A1, (int64_t)B * H, st);
            latent_gemm(true, false, D, H, B, Xb, D, dH1, H, g + o.W1, H, nullptr, false, nullptr, false, false, false, st);
            latent_colsum(dH1, B, H, g + o.b1, st);
            latent_adam(p, g, m, v, P, lr, ++step, st);
            seen += B;
        }
        if (out_loss) {
            float ls = 0.f;
            CT(cudaMemcpyAsync(&ls, loss, sizeof(float), cudaMemcpyDeviceToHost, st));
            CT(cudaStreamSynchronize(st));
            out_loss[ep] = seen > 0 ? ls / (float)seen : 0.f;
        }
    }
    CT(cudaMemcpyAsync(out_params, p, sizeof(float) * (size_t)P, cudaMemcpyDeviceToHost, st));
    CT(cudaStreamSynchronize(st));
    CT(cudaGetLastError());
#undef CT
    cleanup();
    return rc;
}

slag_status slag_latent_apply(const float *params, int32_t dim, const float *in, int64_t rows, int32_t mode,
                              float *out, void *cuda_stream) {
    if (!params || !in || !out || rows < 0 || rows >= (1LL << 31) || dim < 32 || dim > 4096 || dim % 32 != 0 ||
        mode < 0 || mode > 2)
        return SLAG_ERR_INVALID_ARG;
    if (rows == 0) return SLAG_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t P = latent_layout(dim).total;
    const int64_t din = mode == 1 ? kLatent : dim, dout = mode == 0 ? kLatent : dim;
    float *p = nullptr, *X = nullptr, *Hd = nullptr, *Z = nullptr, *Y = nullptr, *Sd = nullptr;
    uint32_t *derr = nullptr;
    auto cleanup = [&]() {
        float *bufs[] = {p, X, Hd, Z, Y, Sd};
        for (float *b : bufs) if (b) cudaFree(b);
        if (derr) cudaFree(derr);
    };
#define CA2(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            cleanup();                                                                                   \
            return e_ == cudaErrorMemoryAllocation ? SLAG_ERR_OOM : SLAG_ERR_CUDA;                       \
        }                                                                                                \
    } while (0)
    CA2(dmalloc(&p, P)); CA2(dmalloc(&X, rows * din)); CA2(dmalloc(&Hd, rows * kLatentHidden));
    CA2(dmalloc(&Z, rows * kLatent)); CA2(dmalloc(&Y, rows * dim));
    CA2(dmalloc(&Sd, latent_decode_scratch((int)rows, dim)));
    CA2(cudaMalloc((void **)&derr, sizeof(uint32_t)));
    CA2(cudaMemsetAsync(derr, 0, sizeof(uint32_t), st));
    CA2(cudaMemcpyAsync(p, params, sizeof(float) * (size_t)P, cudaMemcpyHostToDevice, st));
    CA2(cudaMemcpyAsync(X, in, sizeof(float) * (size_t)(rows * din), cudaMemcpyHostToDevice, st));
    if (mode == 0) {
        latent_encode(p, dim, X, (int)rows, Hd, Z, st);
    } else if (mode == 1) {
        CA2(latent_decode(p, dim, X, (int)rows, Sd, Y, derr, st));
    } else {
        latent_encode(p, dim, X, (int)rows, Hd, Z, st);
        CA2(latent_decode(p, dim, Z, (int)rows, Sd, Y, derr, st));
    }
    uint32_t herr = 0;
    CA2(cudaMemcpyAsync(out, mode == 0 ? Z : Y, sizeof(float) * (size_t)(rows * dout), cudaMemcpyDeviceToHost, st));
    CA2(cudaMemcpyAsync(&herr, derr, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CA2(cudaStreamSynchronize(st));
    CA2(cudaGetLastError());
    if (herr) {
        cleanup();
        return SLAG_ERR_TIMEOUT;
    }
#undef CA2
    cleanup();
    return SLAG_OK;
}

}  // extern "C"
