// vg_blend_common.cuh -- pieces shared by the compositing kernels (the
// per-tile kernels and the split-list kernels): warp pixel rectangles, the
// warp-level Gaussian/rectangle test, the per-tile list sort and the
// transposing warp reduction of the backward.
#pragma once
#include "vg_internal.h"

namespace vgk {

constexpr int BLEND_BATCH = 256;

// Each warp owns a rectangle of 32*PPT pixels of the tile, as square as the
// 16x16 tile allows (8x4, 8x8, 16x8 for PPT 1, 2, 4): a square footprint
// meets fewer Gaussians of a given size than a strip of the same area, and
// every Gaussian the warp meets costs a cross-lane reduction in the backward.
template <int PPT>
struct WarpRect {
    static constexpr int W = PPT >= 4 ? 16 : 8;       // rectangle width in pixels
    static constexpr int H = 32 * PPT / W;            // rectangle height
    static constexpr int PER_ROW = TILE / W;          // rectangles per tile row
};

// pixel (lx, ly) in the tile of pixel slot k of thread t
template <int PPT>
__device__ __forceinline__ void pixel_of(int t, int k, int& lx, int& ly) {
    using R = WarpRect<PPT>;
    const int w = t >> 5, j = (t & 31) + 32 * k;
    lx = (w % R::PER_ROW) * R::W + j % R::W;
    ly = (w / R::PER_ROW) * R::H + j / R::W;
}

// pixel bounds [X0, X1] x [Y0, Y1] of warp w's rectangle in tile (tx, ty)
template <int PPT>
__device__ __forceinline__ void warp_rect(int tx, int ty, int w, float& X0, float& X1, float& Y0, float& Y1) {
    using R = WarpRect<PPT>;
    X0 = (float)(tx * TILE + (w % R::PER_ROW) * R::W);
    X1 = X0 + (float)(R::W - 1);
    Y0 = (float)(ty * TILE + (w / R::PER_ROW) * R::H);
    Y1 = Y0 + (float)(R::H - 1);
}

// can a pixel of [X0, X1] x [Y0, Y1] have alpha >= alpha_min for this
// Gaussian?  First its alpha box, then the ellipse itself: the base-2
// exponent p2(dx, dy) = A2 dx^2 + B2 dx dy + C2 dy^2 (dx = u - px, dy = v - py,
// concave) must reach thr somewhere on the rectangle.  Its maximum there is 0
// if the centre lies inside, else it lies on an edge facing the centre,
// where p2 is a concave parabola in the free coordinate (vertex clamped to
// the edge).  The margin covers FP32 rounding of the pixels' own tests, so a
// pixel that passes is never culled.
__device__ __forceinline__ bool warp_hits(const float4 g, const float4 co, float X0, float X1, float Y0, float Y1) {
    const float cx = fminf(fmaxf(g.x, X0), X1), cy = fminf(fmaxf(g.y, Y0), Y1);
    if (!(fabsf(g.x - cx) <= g.z && fabsf(g.y - cy) <= g.w)) return false;
    if (cx == g.x && cy == g.y) return true;
    // each candidate is raised by 1e-5 of its terms' magnitudes: FP32
    // rounding of a pixel's own p2 is far smaller, even where the terms of a
    // thin ellipse cancel
    auto p2up = [&](float dx, float dy) {
        const float t1 = co.x * dx * dx, t2 = co.y * dx * dy, t3 = co.z * dy * dy;
        return (t1 + t2 + t3) + 1e-5f * (fabsf(t1) + fabsf(t2) + fabsf(t3));
    };
    // (the vertex through the fast divide: a vertex off by a few ulp lowers
    // the parabola's value there by far less than the margin)
    float best = -INFINITY;
    if (cx != g.x) {  // edge px = cx, dy over [v - Y1, v - Y0]
        const float dx = g.x - cx;
        best = fmaxf(best, p2up(dx, fminf(fmaxf(__fdividef(-co.y * dx, 2.f * co.z), g.y - Y1), g.y - Y0)));
    }
    if (cy != g.y) {  // edge py = cy, dx over [u - X1, u - X0]
        const float dy = g.y - cy;
        best = fmaxf(best, p2up(fminf(fmaxf(__fdividef(-co.y * dy, 2.f * co.x), g.x - X1), g.x - X0), dy));
    }
    return best >= co.w - (1e-3f + 1e-3f * fabsf(co.w));
}

// (key, slot) pairs compared lexicographically: depth bits, then slot index
__device__ __forceinline__ bool kv_less(uint32_t ka, uint32_t va, uint32_t kb, uint32_t vb) {
    return ka < kb || (ka == kb && va < vb);
}

// ascending bitonic sort of one (key, value) pair per lane across the warp
__device__ __forceinline__ void warp_sort32(uint32_t& k, uint32_t& s, int lane) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
        const bool asc = (lane & size) == 0;
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint32_t ok = __shfl_xor_sync(0xffffffffu, k, stride);
            const uint32_t os = __shfl_xor_sync(0xffffffffu, s, stride);
            const bool lower = (lane & stride) == 0;
            const bool other_less = kv_less(ok, os, k, s);
            // in an ascending run the lower lane keeps the smaller pair
            if ((lower == asc) ? other_less : !other_less) {
                k = ok;
                s = os;
            }
        }
    }
}

// Sorts the tile's list pvals[rg.x, rg.y) by (depth key, slot) in place:
// each warp sorts 32-entry chunks in registers, then every entry's final
// position is its rank in its chunk plus, per other chunk, the number of
// entries below it (a 5-step binary search; keys are unique).  The caller
// guarantees n <= VG_TILE_SORT_CAP; s_kv holds VG_TILE_SORT_CAP pairs.
template <int NT>
__device__ __forceinline__ void tile_sort(uint32_t* __restrict__ pvals, uint2 rg, const uint32_t* __restrict__ dkey,
                                          uint2* s_kv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n = rg.y - rg.x;
    const int nch = (int)((n + 31) >> 5);
    for (int c = warp; c < nch; c += NT / 32) {
        const uint32_t e = (uint32_t)c * 32 + lane;
        uint32_t k = 0xffffffffu, sl = 0xffffffffu;  // padding sorts last
        if (e < n) {
            sl = pvals[rg.x + e];
            k = dkey[sl];
        }
        warp_sort32(k, sl, lane);
        s_kv[e] = make_uint2(k, sl);
    }
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < n; e += NT) {
        const uint2 me = s_kv[e];
        const int c = (int)(e >> 5);
        uint32_t pos = e & 31u;
        for (int c2 = 0; c2 < nch; ++c2) {
            if (c2 == c) continue;
            const uint2* b = s_kv + c2 * 32;
            if (kv_less(b[31].x, b[31].y, me.x, me.y)) {
                pos += 32;
                continue;
            }
            uint32_t lo = 0;  // entries of chunk c2 below me: the longest prefix with b[lo - 1] < me
#pragma unroll
            for (uint32_t step = 16; step > 0; step >>= 1) {
                const uint2 x = b[lo + step - 1];
                if (kv_less(x.x, x.y, me.x, me.y)) lo += step;
            }
            pos += lo;
        }
        pvals[rg.x + pos] = me.y;
    }
    __syncthreads();  // the sorted list (global) and the freed shared memory are ready for the block
}

// Fully transposing butterfly: ten per-lane values summed over the warp in
// 12 shuffles.  Each stage halves the values a lane holds (a lane keeps one
// half and sends the other to its partner), so at the end lane l holds the
// warp's sum of value reduce10_index(l) (or nothing, -1), and the ten owners
// issue one atomic instruction together.
__device__ __forceinline__ float warp_reduce10(const float v[10]) {
    const int lane = threadIdx.x & 31;
    const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0, h4 = (lane & 4) != 0, h2 = (lane & 2) != 0;
    float a[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {  // values k (h16 clear) or k + 5 (h16 set)
        const float send = h16 ? v[k] : v[k + 5];
        const float keep = h16 ? v[k + 5] : v[k];
        a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    // h8 clear keeps a0, a1, a2; h8 set keeps a3, a4
    const float b0 = (h8 ? a[3] : a[0]) + __shfl_xor_sync(0xffffffffu, h8 ? a[0] : a[3], 8);
    const float b1 = (h8 ? a[4] : a[1]) + __shfl_xor_sync(0xffffffffu, h8 ? a[1] : a[4], 8);
    const float b2 = (h8 ? 0.f : a[2]) + __shfl_xor_sync(0xffffffffu, h8 ? a[2] : 0.f, 8);
    // h4 clear keeps b0, b1; h4 set keeps b2
    const float c0 = (h4 ? b2 : b0) + __shfl_xor_sync(0xffffffffu, h4 ? b0 : b2, 4);
    const float c1 = (h4 ? 0.f : b1) + __shfl_xor_sync(0xffffffffu, h4 ? b1 : 0.f, 4);
    // h2 clear keeps c0, h2 set keeps c1
    float d = (h2 ? c1 : c0) + __shfl_xor_sync(0xffffffffu, h2 ? c0 : c1, 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    return d;
}

// the value whose warp sum lane `lane` holds after warp_reduce10 (even lanes
// only; the odd ones hold copies), -1 for none
__device__ __forceinline__ int reduce10_index(int lane) {
    if (lane & 1) return -1;
    const int sub = ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    const int k = sub == 0 ? 0 : sub == 1 ? 1 : sub == 2 ? 2 : sub == 4 ? 3 : sub == 5 ? 4 : -1;
    return k < 0 ? -1 : k + ((lane & 16) ? 5 : 0);
}

}  // namespace vgk
