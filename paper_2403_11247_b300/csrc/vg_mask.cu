// vg_mask.cu -- the sliding-window online mask (Sec. "Sliding Window-based
// Online Mask"): the mask loss over the Gaussians of the current viewing
// frustum (Eq. 13, L_m = 1/N_w sum Sig(m_n)) with its gradient, and the
// removal at the window bound by hit count and mask.
#include "vg_internal.h"

namespace vgk {

// is Gaussian n visible (an unempty tile rect) in some view of the forward?
__device__ __forceinline__ bool visible_any(const uint32_t* __restrict__ ntiles, int64_t N, int n_views, int64_t n) {
    for (int v = 0; v < n_views; ++v)
        if (ntiles[(int64_t)v * N + n] != 0u) return true;
    return false;
}

// pass 1: N_w and sum of Sig(m) over the visible Gaussians
__global__ void __launch_bounds__(256) mask_count_kernel(const float* __restrict__ m, const uint32_t* __restrict__ ntiles,
                                                         int64_t N, int n_views, uint32_t* __restrict__ nw,
                                                         float* __restrict__ sum) {
    __shared__ float s_f[8];
    __shared__ uint32_t s_u[8];
    uint32_t c = 0;
    float t = 0.f;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        if (visible_any(ntiles, N, n_views, n)) {
            ++c;
            t += 1.f / (1.f + expf(-m[n]));
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_u[threadIdx.x >> 5] = c;
        s_f[threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t cc = 0;
        float tt = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            cc += s_u[w];
            tt += s_f[w];
        }
        if (cc) {
            atomicAdd(nw, cc);
            atomicAdd(sum, tt);
        }
    }
}

// pass 2: dmask[n] += weight Sig'(m_n) / N_w on the visible Gaussians, and the loss
__global__ void __launch_bounds__(256) mask_apply_kernel(const float* __restrict__ m, const uint32_t* __restrict__ ntiles,
                                                         int64_t N, int n_views, const uint32_t* __restrict__ nw,
                                                         const float* __restrict__ sum, float weight,
                                                         float* __restrict__ dmask, float* __restrict__ loss) {
    const uint32_t cnt = *nw;
    if (cnt == 0) {
        if (loss && blockIdx.x == 0 && threadIdx.x == 0) *loss = 0.f;
        return;
    }
    const float inv = weight / (float)cnt;
    if (loss && blockIdx.x == 0 && threadIdx.x == 0) *loss = *sum * inv;
    if (!dmask) return;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        if (visible_any(ntiles, N, n_views, n)) {
            const float sg = 1.f / (1.f + expf(-m[n]));
            dmask[n] += inv * sg * (1.f - sg);
        }
}

// removal: mask off (m <= logit(eps), the renderer's own test) or visible in
// the window but hit fewer than min_hits rays -> m = -inf
__global__ void __launch_bounds__(256) mask_prune_kernel(float* __restrict__ m, float thr, const uint32_t* __restrict__ hits,
                                                         const uint32_t* __restrict__ seen, uint32_t min_hits, int64_t N,
                                                         uint32_t* __restrict__ removed, uint32_t* __restrict__ n_removed) {
    uint32_t c = 0;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const float mv = m[n];
        const bool off = !(mv > thr);
        const bool rare = seen && seen[n] != 0u && hits && hits[n] < min_hits;
        const bool rm = off || rare;
        if (rm) m[n] = -INFINITY;
        if (removed) removed[n] = rm ? 1u : 0u;
        c += rm;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (n_removed && (threadIdx.x & 31) == 0 && c) atomicAdd(n_removed, c);
}

vg_status vg_mask_kernels_loss(const SceneDev& S, const Views& V, const uint32_t* ntiles, float weight, float* dmask,
                               float* loss, uint32_t* scratch_u, float* scratch_f, cudaStream_t st) {
    int64_t blocks = ceil_div(S.N > 0 ? S.N : 1, 256);
    if (blocks > 148 * 4) blocks = 148 * 4;
    cudaError_t e = cudaMemsetAsync(scratch_u, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch_f, 0, 4, st);
    if (e != cudaSuccess) return set_error(VG_ERR_CUDA, cudaGetErrorString(e));
    count_launches(2);
    mask_count_kernel<<<(unsigned)blocks, 256, 0, st>>>(S.mask, ntiles, S.N, V.n, scratch_u, scratch_f);
    mask_apply_kernel<<<(unsigned)blocks, 256, 0, st>>>(S.mask, ntiles, S.N, V.n, scratch_u, scratch_f, weight, dmask,
                                                        loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? VG_OK : set_error(VG_ERR_CUDA, cudaGetErrorString(e));
}

vg_status vg_mask_kernels_prune(float* m, float thr, const uint32_t* hits, const uint32_t* seen, uint32_t min_hits,
                                int64_t N, uint32_t* removed, uint32_t* n_removed, cudaStream_t st) {
    if (n_removed) {
        const cudaError_t e = cudaMemsetAsync(n_removed, 0, 4, st);
        if (e != cudaSuccess) return set_error(VG_ERR_CUDA, cudaGetErrorString(e));
    }
    if (N == 0) return VG_OK;
    int64_t blocks = ceil_div(N, 256);
    if (blocks > 148 * 4) blocks = 148 * 4;
    count_launches(1);
    mask_prune_kernel<<<(unsigned)blocks, 256, 0, st>>>(m, thr, hits, seen, min_hits, N, removed, n_removed);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VG_OK : set_error(VG_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace vgk
