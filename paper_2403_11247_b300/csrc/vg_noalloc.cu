// vg_noalloc.cu -- L1 loss gradients for callers that cannot allocate device
// memory.
//
// vg_loss_l1 keeps its valid-pixel counter in a vg_ctx, and making a ctx
// allocates.  Some callers cannot call cudaMalloc at all: code running while
// another framework owns the device allocator, real-time threads that must
// not take the implicit device synchronisation an allocation can cause, or
// code that only records work into streams it does not own.  This variant
// keeps its scratch -- one valid-pixel counter per view -- in a file-scope
// device array instead, so it allocates nothing.
//
// The array lives in every GPU that loads this library, for the life of the
// process (NOALLOC_MAX_VIEWS words).  All calls share it: two calls that
// overlap on the GPU (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "vg.h"
#include "vg_internal.h"

namespace vgk {

constexpr int NOALLOC_MAX_VIEWS = VG_NOALLOC_MAX_VIEWS;
constexpr int NOALLOC_MAX_DEVICES = 64;

// per-view valid-pixel counts, cleared by every call before use
static __device__ __align__(256) uint32_t g_noalloc_counts[NOALLOC_MAX_VIEWS];

// device addresses of g_noalloc_counts, looked up once per device
static uint32_t* g_noalloc_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

__global__ void noalloc_count_valid_kernel(const float* __restrict__ Dt, int64_t n_pix, uint32_t* counts) {
    const int64_t v = blockIdx.y;
    uint32_t c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pix; i += (int64_t)gridDim.x * blockDim.x)
        c += Dt[v * n_pix + i] > 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(counts + v, c);
}

__global__ void noalloc_loss_l1_kernel(int n_views, int64_t n_pix, const float* __restrict__ C,
                                       const float* __restrict__ D, const float* __restrict__ S,
                                       const float* __restrict__ Ct, const float* __restrict__ Dt, float w_depth,
                                       float gate, const uint32_t* __restrict__ counts, float* __restrict__ dC,
                                       float* __restrict__ dD, float* __restrict__ loss) {
    __shared__ float s_tmp[8];
    uint32_t nvalid = 0;
    for (int v = 0; v < n_views; ++v) nvalid += counts[v];
    const float total = (float)((int64_t)n_views * n_pix);
    const float inv_c = 1.f / (3.f * total);
    const float inv_d = nvalid > 0 ? w_depth / (float)nvalid : 0.f;
    const int64_t v = blockIdx.y;
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pix; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = v * n_pix + i;
        const float m = (gate >= 0.f && !(S[e] > gate)) ? 0.f : 1.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t k = (v * 3 + c) * n_pix + i;
            const float r = C[k] - Ct[k];
            const float sg = (r > 0.f) ? 1.f : ((r < 0.f) ? -1.f : 0.f);
            dC[k] = m * sg * inv_c;
            acc += m * fabsf(r) * inv_c;
        }
        const float rd = D[e] - Dt[e];
        const bool valid = Dt[e] > 0.f;
        const float sd = (rd > 0.f) ? 1.f : ((rd < 0.f) ? -1.f : 0.f);
        dD[e] = valid ? m * sd * inv_d : 0.f;
        acc += valid ? m * fabsf(rd) * inv_d : 0.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_tmp[w];
        atomicAdd(loss, t);
    }
}

}  // namespace vgk

using namespace vgk;

namespace {
vg_status noalloc_fail(vg_status s, const std::string& m) { return set_error(s, m.c_str()); }

// Device address of the static counter array on the current device; looked
// up (cudaGetSymbolAddress) on the first call made with that device current.
vg_status noalloc_scratch(uint32_t** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(VG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return noalloc_fail(VG_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_counts);
        if (e != cudaSuccess || !p)
            return noalloc_fail(VG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return VG_OK;
}
}  // namespace

extern "C" {

vg_status vg_loss_l1_noalloc(int32_t n_views, int64_t n_pix, const float* C, const float* D, const float* S,
                             const float* Ct, const float* Dt, float w_depth, float gate, float* dC, float* dD,
                             float* dS, float* loss, vg_stream stream) {
    if (!C || !D || !Ct || !Dt || !dC || !dD || !loss || n_views < 1 || n_pix < 1)
        return noalloc_fail(VG_ERR_INVALID_ARG, "vg_loss_l1_noalloc: null argument or empty size");
    if (n_views > NOALLOC_MAX_VIEWS)
        return noalloc_fail(VG_ERR_INVALID_ARG, "vg_loss_l1_noalloc: n_views " + std::to_string(n_views) +
                                                    " exceeds the static scratch limit of " +
                                                    std::to_string(NOALLOC_MAX_VIEWS) + " views");
    if (gate >= 0.f && !S) return noalloc_fail(VG_ERR_INVALID_ARG, "vg_loss_l1_noalloc: gate needs S");
    uint32_t* counts = nullptr;
    vg_status s = noalloc_scratch(&counts);
    if (s != VG_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)n_views * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e == cudaSuccess && dS) e = cudaMemsetAsync(dS, 0, (size_t)n_views * n_pix * sizeof(float), st);
    if (e != cudaSuccess) return noalloc_fail(VG_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    int64_t bx = ceil_div(n_pix, 256);
    if (bx > 148 * 8) bx = 148 * 8;
    const dim3 grid((unsigned)bx, (unsigned)n_views);
    count_launches(2);
    noalloc_count_valid_kernel<<<grid, 256, 0, st>>>(Dt, n_pix, counts);
    noalloc_loss_l1_kernel<<<grid, 256, 0, st>>>(n_views, n_pix, C, D, S, Ct, Dt, w_depth, gate, counts, dC, dD, loss);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(VG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return VG_OK;
}

}  // extern "C"
