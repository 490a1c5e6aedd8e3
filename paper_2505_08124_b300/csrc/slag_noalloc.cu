// Cosine top-k that allocates nothing.
//
// Some callers cannot allocate device memory once they are running: a query
// service on a robot or an embedded board that reserves all of its memory at
// start-up and must not call cudaMalloc afterwards (it may synchronise the
// device and take unbounded time), or a host application whose device memory
// is owned and budgeted by its own allocator. slag_noalloc_query_topk serves
// them: it runs the same scoring and selection kernels as slag_query_batch,
// on embeddings the caller already holds on the device, with all of its
// scratch (the inverse row norms and the per-tile candidates) in one
// fixed-size array in this file.
#include <cuda.h>
#include <stdint.h>

#include <mutex>

#include "slag_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;   // 16 MiB, held by every device that loads the library
constexpr int kMaxDevices = 64;

// The scratch itself. In host code this name is only a stand-in for the
// device symbol; kernels receive the device address looked up below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// The array's device address per device, with the context it was looked up in: a device reset
// (or another context made current on the device) makes the address stale, so a change of the
// current context triggers a new lookup.
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);

// The calling thread's current driver context (nullptr when it cannot be read).
CUcontext current_context() {
    static CtxGetCurrentFn fn = []() -> CtxGetCurrentFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(p);
    }();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Whether p is memory of device `dev` (device or managed), so that the kernels may read or
// write it; host memory, pinned or not, is refused.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// 1 / |E_k| for rows with a positive weight sum (or any weight when wsum is
// NULL) and a non-zero norm; 0 marks a row that is not a candidate. One warp per row.
__global__ void row_inv_norm_k(const float *__restrict__ E, const float *__restrict__ wsum, int64_t n, int32_t D,
                               float *__restrict__ inv_norm) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *e = E + row * D;
    float s = 0.f;
    for (int d = lane; d < D; d += 32) s = fmaf(e[d], e[d], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const bool ok = (wsum == nullptr || wsum[row] > 0.f) && s > 0.f;
        inv_norm[row] = ok ? 1.f / sqrtf(s) : 0.f;
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" slag_status slag_noalloc_query_topk(const float *E, int64_t n, int32_t dim, const float *wsum,
                                               const float *Q, int32_t B, int32_t k, int64_t *out_ids,
                                               float *out_scores, int32_t *out_count, void *cuda_stream) {
    if (!E || !Q || !out_ids || !out_scores) return SLAG_ERR_INVALID_ARG;
    if (n < 1 || n >= (1LL << 31) || B < 1 || k < 1 || k > slag::kMaxK) return SLAG_ERR_INVALID_ARG;
    if (dim < 16 || dim > 4096 || dim % 16 != 0) return SLAG_ERR_INVALID_ARG;
    if (((uintptr_t)E & 15u) || ((uintptr_t)Q & 15u)) return SLAG_ERR_INVALID_ARG;
    const size_t norm_bytes = align256((size_t)n * sizeof(float));
    const size_t cand = slag::query_cand_entries(B, n, k);
    const size_t need = norm_bytes + align256(cand * sizeof(float)) + align256(cand * sizeof(uint32_t));
    if (need > kScratchBytes) return SLAG_ERR_CAPACITY;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SLAG_ERR_CUDA;
    // every buffer the kernels touch must be memory of this device: a host address would be
    // read or written by the GPU
    if (!on_device(E, dev) || !on_device(Q, dev) || !on_device(out_ids, dev) || !on_device(out_scores, dev) ||
        (wsum && !on_device(wsum, dev)) || (out_count && !on_device(out_count, dev)))
        return SLAG_ERR_INVALID_ARG;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        const CUcontext ctx = current_context();
        if (!g_scratch_ptr[dev] || ctx != g_scratch_ctx[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return SLAG_ERR_CUDA;
            g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
            g_scratch_ctx[dev] = ctx;
        }
        base = g_scratch_ptr[dev];
    }
    float *inv_norm = reinterpret_cast<float *>(base);
    float *cand_s = reinterpret_cast<float *>(base + norm_bytes);
    uint32_t *cand_i = reinterpret_cast<uint32_t *>(base + norm_bytes + align256(cand * sizeof(float)));

    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t threads = n * 32;
    row_inv_norm_k<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(E, wsum, n, dim, inv_norm); slag::note_launch();
    slag::launch_query_topk(Q, B, E, inv_norm, nullptr, n, dim, k, cand_s, cand_i, out_ids, out_scores, out_count, st);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SLAG_OK : SLAG_ERR_CUDA;
}
