// vg_frame.cu -- RGB-D frame ingestion: the method's input is a sequence of
// RGB-D frames with known intrinsics (Sec. 3, opening paragraph).  Sensors
// deliver colour as interleaved 8-bit RGB and depth as 16-bit integers; the
// frames travel to the device in that form (5 bytes a pixel instead of the
// 16 of the FP32 images) and are decoded there into the planar FP32 images
// the renderer and the losses take.
#include "vg_internal.h"

namespace vgk {

// four pixels a thread: three 32-bit words of RGB (12 bytes), one 64-bit
// word of depth, a float4 per colour plane and one for depth
__global__ void __launch_bounds__(256) frame_decode4_kernel(int64_t n4, int64_t hw, const uint32_t* __restrict__ rgb,
                                                            const uint2* __restrict__ depth, float depth_scale,
                                                            float* __restrict__ C,
                                                            float* __restrict__ D) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = 4 * q;         // first pixel, over all views
        const int64_t v = p / hw;        // its view (hw is a multiple of 4: the four share it)
        const int64_t i = p - v * hw;    // and its place in the view
        const uint32_t w0 = rgb[3 * q], w1 = rgb[3 * q + 1], w2 = rgb[3 * q + 2];
        // bytes r0 g0 b0 r1 | g1 b1 r2 g2 | b2 r3 g3 b3 (little-endian words)
        const uint32_t b[12] = {w0 & 255u, (w0 >> 8) & 255u, (w0 >> 16) & 255u, w0 >> 24,
                                w1 & 255u, (w1 >> 8) & 255u, (w1 >> 16) & 255u, w1 >> 24,
                                w2 & 255u, (w2 >> 8) & 255u, (w2 >> 16) & 255u, w2 >> 24};
        float* Cv = C + v * 3 * hw + i;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            *reinterpret_cast<float4*>(Cv + c * hw) =
                make_float4((float)b[c] / 255.f, (float)b[3 + c] / 255.f, (float)b[6 + c] / 255.f,
                            (float)b[9 + c] / 255.f);
        const uint2 d = depth[q];
        *reinterpret_cast<float4*>(D + p) =
            make_float4((float)(d.x & 0xffffu) / depth_scale, (float)(d.x >> 16) / depth_scale,
                        (float)(d.y & 0xffffu) / depth_scale, (float)(d.y >> 16) / depth_scale);
    }
}

// any layout: one pixel a thread
__global__ void __launch_bounds__(256) frame_decode1_kernel(int64_t n, int64_t hw, const uint8_t* __restrict__ rgb,
                                                            const uint16_t* __restrict__ depth, float depth_scale,
                                                            float* __restrict__ C, float* __restrict__ D) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = p / hw, i = p - v * hw;
#pragma unroll
        for (int c = 0; c < 3; ++c) C[(v * 3 + c) * hw + i] = (float)rgb[3 * p + c] / 255.f;
        D[p] = (float)depth[p] / depth_scale;
    }
}

cudaError_t launch_frame_decode(int n_views, int64_t hw, const uint8_t* rgb, const uint16_t* depth, float depth_scale,
                                float* C, float* D, cudaStream_t st) {
    const int64_t n = (int64_t)n_views * hw;
    if (n <= 0) return cudaSuccess;
    const bool vec = hw % 4 == 0 && (reinterpret_cast<uintptr_t>(rgb) & 3u) == 0 &&
                     (reinterpret_cast<uintptr_t>(depth) & 7u) == 0 && (reinterpret_cast<uintptr_t>(C) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(D) & 15u) == 0;
    const int64_t items = vec ? n / 4 : n;
    int64_t blocks = ceil_div(items, 256);
    if (blocks > 148 * 8) blocks = 148 * 8;
    count_launches(1);
    if (vec)
        frame_decode4_kernel<<<(unsigned)blocks, 256, 0, st>>>(n / 4, hw, reinterpret_cast<const uint32_t*>(rgb),
                                                               reinterpret_cast<const uint2*>(depth), depth_scale,
                                                               C, D);
    else
        frame_decode1_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, hw, rgb, depth, depth_scale, C, D);
    return cudaGetLastError();
}

}  // namespace vgk
