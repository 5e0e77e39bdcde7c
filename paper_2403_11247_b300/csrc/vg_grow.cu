// vg_grow.cu -- sequential anchor growing on multi-resolution voxel grids and
// opacity-based anchor removal (Sec. "Sequential Anchor Point Growing",
// Eq. 10).
//
// Statistics: after each backward, every visible (view, Gaussian) pair adds
// the norm of its projected-mean gradient (du, dv) to its Gaussian and its
// opacity to its anchor, with counts.
// Growing, per level m = 1..M (eps_m = eps_g / 4^(m-1), tau_m = tau_g 2^(m-1)):
// an open-addressing hash table keyed by the packed voxel index collects
// (1) the voxels of the established anchors (scene anchors plus those grown at
// coarser levels), flagged occupied, and (2) for every Gaussian seen in the
// interval, its FP32 average gradient as the integer rint(avg 2^32), clamped
// to +-2^52 (an exact, order-free voxel sum), and a count; Gaussians with a
// non-finite average are skipped.  A slot that is unoccupied, whose mean
// exceeds tau_m and that survives the random elimination (SplitMix64 of the key,
// Steele, Lea and Flood, OOPSLA 2014) emits a new anchor at the voxel centre.
// Removal: an anchor seen in the interval whose mean opacity is below
// tau_alpha gets the mask logit -inf on all its k Gaussians.
#include <cmath>

#include "vg_internal.h"

namespace vgk {

constexpr unsigned long long GROW_EMPTY = ~0ull;
constexpr int GROW_BIAS = 1 << 20;

// packed voxel index of p at voxel size eps, or GROW_EMPTY when a component
// is outside [-2^20, 2^20) or not finite
__device__ __forceinline__ unsigned long long voxel_key(const float p[3], float eps) {
    unsigned long long key = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float q = floorf(__fdiv_rn(p[c], eps));
        if (!(q >= -(float)GROW_BIAS && q < (float)GROW_BIAS)) return GROW_EMPTY;
        key = (key << 21) | (unsigned long long)((int)q + GROW_BIAS);
    }
    return key;
}

struct GrowTable {
    unsigned long long* key;
    unsigned long long* sum;
    uint32_t* cnt;
    uint32_t* occ;
    unsigned long long mask;  // slots - 1 (a power of two)
};

// slot holding `key` (inserted if absent); -1 if the table is full
__device__ __forceinline__ long long table_slot(const GrowTable& T, unsigned long long key) {
    unsigned long long s = splitmix64(key) & T.mask;
    for (unsigned long long probe = 0; probe <= T.mask; ++probe) {
        const unsigned long long prev = atomicCAS(T.key + s, GROW_EMPTY, key);
        if (prev == GROW_EMPTY || prev == key) return (long long)s;
        s = (s + 1) & T.mask;
    }
    return -1;
}

__global__ void __launch_bounds__(256) grow_stats_kernel(SceneDev S, const uint32_t* __restrict__ vis,
                                                         const uint32_t* __restrict__ nvis_dev, uint32_t max_vis,
                                                         const float* __restrict__ g2d, float* gacc, uint32_t* gcnt,
                                                         float* oacc, uint32_t* ocnt) {
    const uint32_t nv = min(*nvis_dev, max_vis);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
        const uint32_t slot = vis[i];
        const int64_t n = (int64_t)(slot % (uint32_t)S.N);  // slots are u32, so a 32-bit remainder
        if (gacc) {
            const float du = g2d[(int64_t)slot * G2D_STRIDE + 0], dv = g2d[(int64_t)slot * G2D_STRIDE + 1];
            atomicAdd(gacc + n, sqrtf(du * du + dv * dv));
            atomicAdd(gcnt + n, 1u);
        }
        if (oacc) {
            float ol;
            decode_attr<1>(S, 2, n, &ol);
            const int64_t a = anchor_of(S, n);
            atomicAdd(oacc + a, 1.f / (1.f + expf(-ol)));
            atomicAdd(ocnt + a, 1u);
        }
    }
}

// established anchors: the scene's and the first min(*n_new, cap) grown ones
__global__ void __launch_bounds__(256) grow_occupy_kernel(GrowTable T, const float* __restrict__ xyz, int64_t A,
                                                          const float* __restrict__ new_xyz, const uint32_t* n_new,
                                                          int64_t cap, float eps, uint32_t* err) {
    const int64_t n_grown = min((int64_t)*n_new, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A + n_grown;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float* src = i < A ? xyz + i * 3 : new_xyz + (i - A) * 3;
        const float p[3] = {src[0], src[1], src[2]};
        const unsigned long long key = voxel_key(p, eps);
        if (key == GROW_EMPTY) continue;
        const long long s = table_slot(T, key);
        if (s < 0) {
            atomicOr(err, 1u);
            continue;
        }
        T.occ[s] = 1u;
    }
}

__global__ void __launch_bounds__(256) grow_voxels_kernel(GrowTable T, SceneDev S, const float* __restrict__ gacc,
                                                          const uint32_t* __restrict__ gcnt, float eps, uint32_t* err) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < S.N; n += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = gcnt[n];
        if (c == 0) continue;
        const float avg = __fdiv_rn(gacc[n], (float)c);
        if (!isfinite(avg)) continue;
        float mu[3];
        anchor_mean(S, n, mu);
        const unsigned long long key = voxel_key(mu, eps);
        if (key == GROW_EMPTY) continue;
        const long long s = table_slot(T, key);
        if (s < 0) {
            atomicOr(err, 1u);
            continue;
        }
        // |avg| above 2^20 is clamped there, so that voxel sums stay far inside 64 bits
        const double q = fmin(fmax(rint((double)avg * 4294967296.0), -4503599627370496.0), 4503599627370496.0);
        atomicAdd(T.sum + s, (unsigned long long)(long long)q);
        atomicAdd(T.cnt + s, 1u);
    }
}

__global__ void __launch_bounds__(256) grow_emit_kernel(GrowTable T, float eps, double tau_scaled,
                                                        unsigned long long seed_m,
                                                        unsigned long long drop_below, int level, float* new_xyz,
                                                        int32_t* new_level, uint32_t* n_new, int64_t cap) {
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s <= T.mask;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long key = T.key[s];
        if (key == GROW_EMPTY || T.occ[s]) continue;
        const uint32_t c = T.cnt[s];
        if (c == 0) continue;
        if (!((double)(long long)T.sum[s] > tau_scaled * (double)c)) continue;
        if ((splitmix64(key ^ seed_m) >> 11) < drop_below) continue;
        const uint32_t o = atomicAdd(n_new, 1u);
        if ((int64_t)o >= cap) continue;
        const int ix = (int)((key >> 42) & 0x1fffff) - GROW_BIAS;
        const int iy = (int)((key >> 21) & 0x1fffff) - GROW_BIAS;
        const int iz = (int)(key & 0x1fffff) - GROW_BIAS;
        new_xyz[o * 3 + 0] = __fmul_rn(__fadd_rn((float)ix, 0.5f), eps);
        new_xyz[o * 3 + 1] = __fmul_rn(__fadd_rn((float)iy, 0.5f), eps);
        new_xyz[o * 3 + 2] = __fmul_rn(__fadd_rn((float)iz, 0.5f), eps);
        if (new_level) new_level[o] = level;
    }
}

__global__ void __launch_bounds__(256) grow_prune_kernel(float* mask, int64_t A, int k, const float* __restrict__ oacc,
                                                         const uint32_t* __restrict__ ocnt, float tau_alpha,
                                                         uint32_t* removed, uint32_t* n_removed) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = ocnt[a];
        const bool rm = c > 0 && oacc[a] < __fmul_rn(tau_alpha, (float)c);
        if (rm)
            for (int j = 0; j < k; ++j) mask[a * k + j] = -INFINITY;
        if (removed) removed[a] = rm ? 1u : 0u;
        if (n_removed) {
            const uint32_t b = __ballot_sync(__activemask(), rm);
            if (rm && (threadIdx.x & 31) == (uint32_t)(__ffs(b) - 1)) atomicAdd(n_removed, (uint32_t)__popc(b));
        }
    }
}

static unsigned grid_for(int64_t n) {
    int64_t b = ceil_div(n, 256);
    if (b < 1) b = 1;
    if (b > 148 * 16) b = 148 * 16;
    return (unsigned)b;
}

int64_t grow_table_slots(int64_t A, int64_t N, int64_t cap) {
    const int64_t need = 2 * (A + N + cap) + 1024;
    int64_t s = 1024;
    while (s < need) s <<= 1;
    return s;
}

cudaError_t launch_grow_stats(const SceneDev& S, const uint32_t* vis, const uint32_t* nvis_dev, uint32_t max_vis,
                              const float* g2d, float* gacc, uint32_t* gcnt, float* oacc, uint32_t* ocnt,
                              cudaStream_t st) {
    count_launches(1);
    grow_stats_kernel<<<grid_for(max_vis), 256, 0, st>>>(S, vis, nvis_dev, max_vis, g2d, gacc, gcnt, oacc, ocnt);
    return cudaGetLastError();
}

cudaError_t launch_grow(const SceneDev& S, const float* gacc, const uint32_t* gcnt, float eps_g, float tau_g, int levels,
                        unsigned long long drop_below, unsigned long long seed, float* new_xyz, int32_t* new_level,
                        uint32_t* n_new, int64_t cap, void* ws, int64_t slots, uint32_t* err, cudaStream_t st) {
    GrowTable T;
    T.key = reinterpret_cast<unsigned long long*>(ws);
    T.sum = T.key + slots;
    T.cnt = reinterpret_cast<uint32_t*>(T.sum + slots);
    T.occ = T.cnt + slots;
    T.mask = (unsigned long long)slots - 1;
    cudaError_t e = cudaMemsetAsync(n_new, 0, 4, st);
    if (e != cudaSuccess) return e;
    float scale = 1.f;
    for (int m = 1; m <= levels; ++m) {
        const float eps = eps_g / scale;                // eps_g / 4^(m-1), exact
        const float tau = tau_g * (float)(1 << (m - 1)); // tau_g * 2^(m-1), exact
        scale *= 4.f;
        e = cudaMemsetAsync(T.key, 0xff, (size_t)slots * 8, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(T.sum, 0, (size_t)slots * 16, st);
        if (e != cudaSuccess) return e;
        count_launches(3);
        grow_occupy_kernel<<<grid_for(S.n_anchors + cap), 256, 0, st>>>(T, S.xyz, S.n_anchors, new_xyz, n_new, cap, eps,
                                                                        err);
        grow_voxels_kernel<<<grid_for(S.N), 256, 0, st>>>(T, S, gacc, gcnt, eps, err);
        const unsigned long long seed_m = seed + (unsigned long long)m * GOLDEN_GAMMA;
        grow_emit_kernel<<<grid_for(slots), 256, 0, st>>>(T, eps, (double)tau * 4294967296.0, seed_m, drop_below, m,
                                                          new_xyz, new_level, n_new, cap);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_anchor_prune(float* mask, int64_t A, int k, const float* oacc, const uint32_t* ocnt, float tau_alpha,
                                uint32_t* removed, uint32_t* n_removed, cudaStream_t st) {
    if (n_removed) {
        cudaError_t e = cudaMemsetAsync(n_removed, 0, 4, st);
        if (e != cudaSuccess) return e;
    }
    if (A == 0) return cudaSuccess;
    count_launches(1);
    grow_prune_kernel<<<grid_for(A), 256, 0, st>>>(mask, A, k, oacc, ocnt, tau_alpha, removed, n_removed);
    return cudaGetLastError();
}

}  // namespace vgk
