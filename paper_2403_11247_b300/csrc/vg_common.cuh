// vg_common.cuh -- device-side types and helpers shared by the libvg kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vg.h"

namespace vgk {

constexpr int TILE = VG_TILE;
constexpr int TILE_PIX = TILE * TILE;

// device status bits (vg_stats.flags)
constexpr uint32_t ERR_WAIT = 1u;      // a bounded spin ran out
constexpr uint32_t ERR_OVERFLOW = 2u;  // pair buffer too small
constexpr uint32_t ERR_TABLE = 4u;     // the anchor-growing hash table was full
constexpr uint32_t ERR_TILE_LIST = 8u; // a tile list longer than the compositing kernel sorts (no long pass)
constexpr uint32_t ERR_TILE_LONG = 16u; // a tile list longer than the long-list pass sorts

// a bounded spin gives up after this many unsuccessful polls (~1 s of L2
// round trips) unless the ctx sets another limit (vg_ctx_set_spin_limit)
constexpr uint32_t SPIN_LIMIT_DEFAULT = 1u << 21;

constexpr int RADIUS_MAX = 1 << 20;

// Per-view launch constants.  Passed by value as a __grid_constant__ kernel
// parameter so that a captured graph keeps them; poses may instead come from
// device memory (pose_dev) for graphs that update poses on the device.
struct ViewInfo {
    float fx, fy, cx, cy;
    float T[12];
    float near_plane;
    float limx, limy;
    int32_t W, H, tiles_x, tiles_y;
    int32_t tile_base;
    int64_t pix_base;
};

struct Views {
    int32_t n;
    int32_t total_tiles;
    const float* pose_dev;
    ViewInfo v[VG_MAX_VIEWS];
};

struct Consts {
    float alpha_max, alpha_min, t_min, dilation, sigma_cull;
    int32_t jacobian_clamp;
    uint32_t* hit_count;  // [N] blended (view, pixel) pairs per Gaussian, added to; NULL = off
    uint32_t* seen;       // [N] set to 1 where a Gaussian is visible in some view; NULL = off
    int64_t n_gauss;      // N, for the two arrays above
    int32_t depth_hist;   // the preprocess accumulates depth-key digit histograms (global depth sort)
    const uint8_t* pix_mask;  // [pixels] 0 = not composited (sampled rays); NULL = every pixel
    int32_t blend_batch;      // Gaussians staged in shared memory per batch by the compositing kernels
    int32_t long_sorted;      // lists over VG_TILE_SORT_CAP were sorted by the long-list pass
    // L1 loss gradient written by the forward compositing (vg_render_fwd_l1);
    // lf_on = 0: off
    int32_t lf_on;
    const float* lf_Ct;        // [3 per pixel] target colour, per-view planar like C
    const float* lf_Dt;        // [pixels] target depth
    float* lf_dC;              // [3 per pixel] dL/dC
    float* lf_dD;              // [pixels] dL/dD
    float* lf_dS;              // [pixels] zeroed (may be NULL)
    float* lf_loss;            // [1] the loss (zeroed by the preprocess, summed by the compositing blocks)
    uint32_t* lf_blk;          // [2][compaction blocks] per-block counts of valid depths, sampled pixels
    const uint32_t* lf_counts; // [2] their totals (written by the ranges kernel)
    int64_t lf_pixels;         // pixels of all views
    float lf_wdepth, lf_gate;
};

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the output for generator state `state` (the
// golden gamma added, then the published finaliser); used as a counter-based
// generator keyed by (seed, counter)
constexpr unsigned long long GOLDEN_GAMMA = 0x9E3779B97F4A7C15ull;
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long state) {
    unsigned long long z = state + GOLDEN_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Scene arrays as the kernels see them (device pointers).
struct SceneDev {
    int64_t n_anchors;
    int32_t k;
    int64_t N;
    const float* xyz;
    const float* l;
    const float* off;
    int32_t L[4], K[4];
    const float* cb[4];
    const uint8_t* idx[4];
    const float* raw[4];
    const float* mask;
    float mask_thr;
    // R-VQ coded offsets (idx [Lo][N]) and scaling factors (idx [Ll][Na]); L = 0: raw arrays
    int32_t Lo, Ko, Ll, Kl;
    const float* cbo;
    const float* cbl;
    const uint8_t* idxo;
    const uint8_t* idxl;
};

// attribute group dims and their offsets in the packed 11-float attribute
// gradient record: log-scale 0..2, quaternion 3..6, opacity 7, rgb 8..10
__host__ __device__ constexpr int gdim(int g) { return g == 0 ? 3 : (g == 1 ? 4 : (g == 2 ? 1 : 3)); }
__host__ __device__ constexpr int goff(int g) { return g == 0 ? 0 : (g == 1 ? 3 : (g == 2 ? 7 : 8)); }
constexpr int ATTR_STRIDE = 11;
constexpr int G2D_STRIDE = 12;  // du dv da db dc dopacity dr dg db ddepth, 2 pad (16-byte rows)

__device__ __forceinline__ int view_of_tile(const Views& V, int gt) {
    int lo = 0, hi = V.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (V.v[mid].tile_base <= gt) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void view_pose(const Views& V, int v, float T[12]) {
    if (V.pose_dev) {
#pragma unroll
        for (int i = 0; i < 12; ++i) T[i] = __ldg(V.pose_dev + v * 12 + i);
    } else {
#pragma unroll
        for (int i = 0; i < 12; ++i) T[i] = V.v[v].T[i];
    }
}

// The 2D covariance of Eq. 3 plus the low-pass dilation, J W Sigma W^T J^T +
// dil I, evaluated as M M^T + dil I with M = J W R diag(s) (2x3, rows m0,
// m1; Sigma = (R diag(s)) (R diag(s))^T, RS = R diag(s)): A = |m0|^2 + dil,
// B = m0.m1, C = |m1|^2 + dil, and the determinant by Lagrange's identity,
// det = |m0 x m1|^2 + dil (|m0|^2 + |m1|^2) + dil^2, a sum of non-negative
// terms (AC - B^2 cancels catastrophically for thin splats seen edge-on).
// T is the row-major 3x4 world->camera pose (W = its 3x3 part).
__device__ __forceinline__ void cov2d(float J00, float J02, float J11, float J12, const float T[12],
                                      const float RS[3][3], float dil, float& A, float& B, float& C, float& det) {
    float jw0[3], jw1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        jw0[c] = J00 * T[c] + J02 * T[8 + c];
        jw1[c] = J11 * T[4 + c] + J12 * T[8 + c];
    }
    float m0[3], m1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        m0[c] = jw0[0] * RS[0][c] + jw0[1] * RS[1][c] + jw0[2] * RS[2][c];
        m1[c] = jw1[0] * RS[0][c] + jw1[1] * RS[1][c] + jw1[2] * RS[2][c];
    }
    const float a0 = m0[0] * m0[0] + m0[1] * m0[1] + m0[2] * m0[2];
    const float c0 = m1[0] * m1[0] + m1[1] * m1[1] + m1[2] * m1[2];
    B = m0[0] * m1[0] + m0[1] * m1[1] + m0[2] * m1[2];
    const float x0 = m0[1] * m1[2] - m0[2] * m1[1];
    const float x1 = m0[2] * m1[0] - m0[0] * m1[2];
    const float x2 = m0[0] * m1[1] - m0[1] * m1[0];
    A = a0 + dil;
    C = c0 + dil;
    det = (x0 * x0 + x1 * x1 + x2 * x2) + dil * (a0 + c0) + dil * dil;
}

// Code indices of one item for its first DECODE_STAGES stages, four bytes
// per word, loaded together before any codeword: the loads go out in
// parallel instead of one dependent round trip per stage.  Further stages
// (never in practice) take a plain loop.
constexpr int DECODE_STAGES = 8;
__device__ __forceinline__ void load_codes(const uint8_t* idx, int L, int64_t stride, int64_t n,
                                           uint32_t kp[DECODE_STAGES / 4]) {
#pragma unroll
    for (int w = 0; w < DECODE_STAGES / 4; ++w) kp[w] = 0u;
#pragma unroll
    for (int s = 0; s < DECODE_STAGES; ++s)
        if (s < L) kp[s >> 2] |= (uint32_t)__ldg(idx + (int64_t)s * stride + n) << (8 * (s & 3));
}
__device__ __forceinline__ uint32_t code_at(const uint32_t kp[DECODE_STAGES / 4], int s) {
    return (kp[s >> 2] >> (8 * (s & 3))) & 255u;
}

// attribute = FP32 sum, in stage order, of the indexed codewords (Eq. 14), or
// the raw value; kp receives the codes of the first DECODE_STAGES stages
template <int D>
__device__ __forceinline__ void decode_attr_codes(const SceneDev& S, int g, int64_t n, float* out,
                                                  uint32_t kp[DECODE_STAGES / 4]) {
    if (S.L[g] > 0) {
        const int L = S.L[g], K = S.K[g];
        load_codes(S.idx[g], L, S.N, n, kp);
#pragma unroll
        for (int c = 0; c < D; ++c) out[c] = 0.f;
#pragma unroll
        for (int s = 0; s < DECODE_STAGES; ++s)
            if (s < L) {
                const float* w = S.cb[g] + ((int64_t)s * K + code_at(kp, s)) * D;
#pragma unroll
                for (int c = 0; c < D; ++c) out[c] += __ldg(w + c);
            }
        for (int s = DECODE_STAGES; s < L; ++s) {
            const float* w = S.cb[g] + ((int64_t)s * K + __ldg(S.idx[g] + (int64_t)s * S.N + n)) * D;
#pragma unroll
            for (int c = 0; c < D; ++c) out[c] += __ldg(w + c);
        }
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) out[c] = __ldg(S.raw[g] + n * D + c);
    }
}

template <int D>
__device__ __forceinline__ void decode_attr(const SceneDev& S, int g, int64_t n, float* out) {
    uint32_t kp[DECODE_STAGES / 4];
    decode_attr_codes<D>(S, g, n, out, kp);
}

// same, with the group's codebook staged in shared memory
template <int D>
__device__ __forceinline__ void decode_attr_smem(const SceneDev& S, int g, int64_t n, const float* cb, float* out) {
    if (S.L[g] > 0) {
        const int L = S.L[g], K = S.K[g];
        uint32_t kp[DECODE_STAGES / 4];
        load_codes(S.idx[g], L, S.N, n, kp);
#pragma unroll
        for (int c = 0; c < D; ++c) out[c] = 0.f;
#pragma unroll
        for (int s = 0; s < DECODE_STAGES; ++s)
            if (s < L) {
                const float* w = cb + (s * K + (int)code_at(kp, s)) * D;
#pragma unroll
                for (int c = 0; c < D; ++c) out[c] += w[c];
            }
        for (int s = DECODE_STAGES; s < L; ++s) {
            const float* w = cb + (s * K + __ldg(S.idx[g] + (int64_t)s * S.N + n)) * D;
#pragma unroll
            for (int c = 0; c < D; ++c) out[c] += w[c];
        }
    } else {
#pragma unroll
        for (int c = 0; c < D; ++c) out[c] = __ldg(S.raw[g] + n * D + c);
    }
}

// offset O_n and scaling factor l_a: raw, or the FP32 stage-order sum of
// their R-VQ codewords (Eq. 14)
__device__ __forceinline__ void coded3(const float* cb, const uint8_t* idx, int L, int K, int64_t stride, int64_t i,
                                       float o[3]) {
    uint32_t kp[DECODE_STAGES / 4];
    load_codes(idx, L, stride, i, kp);
    o[0] = o[1] = o[2] = 0.f;
#pragma unroll
    for (int s = 0; s < DECODE_STAGES; ++s)
        if (s < L) {
            const float* w = cb + ((int64_t)s * K + code_at(kp, s)) * 3;
            o[0] += __ldg(w);
            o[1] += __ldg(w + 1);
            o[2] += __ldg(w + 2);
        }
    for (int s = DECODE_STAGES; s < L; ++s) {
        const float* w = cb + ((int64_t)s * K + __ldg(idx + (int64_t)s * stride + i)) * 3;
        o[0] += __ldg(w);
        o[1] += __ldg(w + 1);
        o[2] += __ldg(w + 2);
    }
}
__device__ __forceinline__ void scene_offset(const SceneDev& S, int64_t n, float o[3]) {
    if (S.Lo > 0) {
        coded3(S.cbo, S.idxo, S.Lo, S.Ko, S.N, n, o);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) o[c] = __ldg(S.off + n * 3 + c);
    }
}
__device__ __forceinline__ void scene_scale(const SceneDev& S, int64_t a, float l[3]) {
    if (S.Ll > 0) {
        coded3(S.cbl, S.idxl, S.Ll, S.Kl, S.n_anchors, a, l);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) l[c] = __ldg(S.l + a * 3 + c);
    }
}

// anchor of Gaussian n (k Gaussians per anchor): a 32-bit division where n
// fits, which costs a fraction of the 64-bit one
__device__ __forceinline__ int64_t anchor_of(const SceneDev& S, int64_t n) {
    return n <= 0x7fffffffll ? (int64_t)((uint32_t)n / (uint32_t)S.k) : n / S.k;
}

// Eq. 7 with the binning rounding: mu_c = xa_c + (O_c * l_c), no FMA
__device__ __forceinline__ void anchor_mean(const SceneDev& S, int64_t n, float mu[3]) {
    const int64_t a = anchor_of(S, n);
    float o[3], l[3];
    scene_offset(S, n, o);
    scene_scale(S, a, l);
#pragma unroll
    for (int c = 0; c < 3; ++c) mu[c] = __fadd_rn(__ldg(S.xyz + a * 3 + c), __fmul_rn(o[c], l[c]));
}

// camera-space point with the binning rounding: ((W0 m0 + W1 m1) + W2 m2) + t
__device__ __forceinline__ void cam_point(const float T[12], const float mu[3], float p[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float e0 = __fmul_rn(T[r * 4 + 0], mu[0]);
        float e1 = __fmul_rn(T[r * 4 + 1], mu[1]);
        float e2 = __fmul_rn(T[r * 4 + 2], mu[2]);
        p[r] = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), e2), T[r * 4 + 3]);
    }
}

__device__ __forceinline__ void quat_rot(const float q[4], float R[3][3]) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z);       R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z);       R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y);       R[2][1] = 2.f * (y * z + w * x);       R[2][2] = 1.f - 2.f * (x * x + y * y);
}

constexpr float LOG2E = 1.4426950408889634f;
constexpr float LN2 = 0.6931471805599453f;

// The per-slot conic record holds the exponent in base 2:
//   A2 = -a/2 log2(e), B2 = -b log2(e), C2 = -c/2 log2(e),
// so that p2 = dx (A2 dx + B2 dy) + C2 dy^2 = log2(e) (-1/2 d^T conic d), and
//   thr = log2(alpha_min / o).
// Then alpha >= alpha_min  <=>  q = p2 - thr >= 0, and alpha = alpha_min 2^q:
// a pixel is rejected before any exponential.  Every rounding is spelled out
// so that the forward and backward kernels take identical decisions.
__device__ __forceinline__ float gauss_p2(float A2, float B2, float C2, float dx, float dy) {
    const float inner = __fmaf_rn(A2, dx, __fmul_rn(B2, dy));
    return __fmaf_rn(dx, inner, __fmul_rn(__fmul_rn(C2, dy), dy));
}

// Overlapped launch of a dependent kernel (programmatic dependent launch):
// the kernel in front lets its dependents be scheduled once each of its CTAs
// has started (allow_dependents), and the dependent kernel runs its
// scene-only prefix, then waits here until the kernel in front has completed
// and its writes are visible.  Both are no-ops for a normal launch.
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// 2^x with the hardware base-2 exponential unit
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// add v to a word of shared memory without reading the result back (the
// reduction form of the atomic add: the thread does not wait for it)
__device__ __forceinline__ void red_add_shared(float* p, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(uint32_t* p, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// One pixel of the L1 loss (mean |C - Ct| + w_depth mean_{Dt > 0} |D - Dt|,
// inv_c = 1 / (3 pixels), inv_d = w_depth / valid depths): writes the
// gradients of the three colour planes and the depth, returns the pixel's
// share of the loss.  A pixel not sampled, or gated out (S <= gate when
// gate >= 0, Eq. 21), contributes nothing.  sign(0) = 0.
__device__ __forceinline__ float loss_pixel(float c0, float c1, float c2, float t0, float t1, float t2, float d,
                                            float dt, float s, float gate, float inv_c, float inv_d, float& g0,
                                            float& g1, float& g2, float& gd, bool sampled = true) {
    const float m = (!sampled || (gate >= 0.f && !(s > gate))) ? 0.f : 1.f;
    const float r0 = c0 - t0, r1 = c1 - t1, r2 = c2 - t2, rd = d - dt;
    auto sgn = [](float r) { return (r > 0.f) ? 1.f : ((r < 0.f) ? -1.f : 0.f); };
    g0 = m * sgn(r0) * inv_c;
    g1 = m * sgn(r1) * inv_c;
    g2 = m * sgn(r2) * inv_c;
    const bool valid = sampled && dt > 0.f;
    gd = valid ? m * sgn(rd) * inv_d : 0.f;
    return m * (fabsf(r0) + fabsf(r1) + fabsf(r2)) * inv_c + (valid ? m * fabsf(rd) * inv_d : 0.f);
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) { return *(const volatile uint32_t*)p; }
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) { *(volatile uint32_t*)p = v; }
__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}
__device__ __forceinline__ void st_volatile64(unsigned long long* p, unsigned long long v) {
    *(volatile unsigned long long*)p = v;
}

// exclusive scan over a 256-thread block; returns the block total in *total
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t x, uint32_t* s_tmp /*[8]*/, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint32_t t = s_tmp[w];
        wpre += (w < warp) ? t : 0u;
        tot += t;
    }
    __syncthreads();
    *total = tot;
    return wpre + inc - x;
}

}  // namespace vgk
