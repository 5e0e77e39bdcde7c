// vg_ssim.cu -- the SSIM term the local-to-global bundle adjustment adds to
// the RGB rendering (Sec. "Tracking and Local-to-Global Bundle Adjustment"):
// L = 1 - mean SSIM(C, C_target) over views, channels and pixels, with an
// 11x11 Gaussian window (sigma 1.5, separable), zero padding, C1 = 0.01^2,
// C2 = 0.03^2, and its gradient with respect to C.
//
// Forward: a horizontal and a vertical 11-tap pass over x, y, x^2, y^2, xy
// give the local means and second moments; SSIM and the three coefficient
// maps of its gradient (d/dmu_x, d/dsigma_x^2, d/dsigma_xy, pre-combined)
// come out of the vertical pass.  Backward: the same two passes over the
// three coefficient maps; dL/dx = G*A + 2 x (G*B) + y (G*Cc).
#include <cmath>

#include "vg_internal.h"

namespace vgk {

constexpr int SSIM_R = 5;  // window radius (11 taps)

struct SsimWin {
    float w[2 * SSIM_R + 1];
};

// horizontal pass of `nq` quantities derived from (x, y): q = 0..4 -> x, y, x^2, y^2, xy
// (nq = 5), or of the three coefficient maps (nq = 3, read from src)
__global__ void __launch_bounds__(256) ssim_hpass_kernel(int planes, int W, int H, const float* __restrict__ x,
                                                         const float* __restrict__ y, const float* __restrict__ src,
                                                         int nq, float* __restrict__ dst, SsimWin win) {
    const int64_t HW = (int64_t)W * H, total = (int64_t)planes * HW;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / HW, rem = e - p * HW;
        const int r = (int)(rem / W), c = (int)(rem - (int64_t)r * W);
        float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = -SSIM_R; k <= SSIM_R; ++k) {
            const int cc = c + k;
            if (cc < 0 || cc >= W) continue;
            const float wk = win.w[k + SSIM_R];
            const int64_t i = p * HW + (int64_t)r * W + cc;
            if (nq == 5) {
                const float a = x[i], b = y[i];
                acc[0] += wk * a;
                acc[1] += wk * b;
                acc[2] += wk * (a * a);
                acc[3] += wk * (b * b);
                acc[4] += wk * (a * b);
            } else {
                for (int q = 0; q < 3; ++q) acc[q] += wk * src[(int64_t)q * total + i];
            }
        }
        for (int q = 0; q < nq; ++q) dst[(int64_t)q * total + e] = acc[q];
    }
}

// vertical pass of the five statistics; SSIM, its sum, and the coefficient maps
__global__ void __launch_bounds__(256) ssim_vstats_kernel(int planes, int W, int H, const float* __restrict__ hs,
                                                          SsimWin win, float inv_m, float* __restrict__ coef,
                                                          float* __restrict__ ssim_sum) {
    __shared__ float s_tmp[8];
    const int64_t HW = (int64_t)W * H, total = (int64_t)planes * HW;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float local = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / HW, rem = e - p * HW;
        const int r = (int)(rem / W), c = (int)(rem - (int64_t)r * W);
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = -SSIM_R; k <= SSIM_R; ++k) {
            const int rr = r + k;
            if (rr < 0 || rr >= H) continue;
            const float wk = win.w[k + SSIM_R];
            const int64_t i = p * HW + (int64_t)rr * W + c;
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] += wk * hs[(int64_t)q * total + i];
        }
        const float mx = m[0], my = m[1];
        const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
        const float a1 = 2.f * mx * my + C1, a2 = 2.f * sxy + C2;
        const float b1 = mx * mx + my * my + C1, b2 = sxx + syy + C2;
        const float inv_b = 1.f / (b1 * b2);
        const float S = a1 * a2 * inv_b;
        local += S;
        const float dmx = 2.f * my * a2 * inv_b - 2.f * mx * S / b1;
        const float dsxx = -S / b2;
        const float dsxy = 2.f * a1 * inv_b;
        coef[e] = -(dmx - 2.f * mx * dsxx - my * dsxy) * inv_m;  // A
        coef[total + e] = -dsxx * inv_m;                         // B
        coef[2 * total + e] = -dsxy * inv_m;                     // Cc
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_tmp[w];
        atomicAdd(ssim_sum, t);
    }
}

// vertical pass of the three filtered coefficient maps and the gradient
__global__ void __launch_bounds__(256) ssim_vgrad_kernel(int planes, int W, int H, const float* __restrict__ hc,
                                                         const float* __restrict__ x, const float* __restrict__ y,
                                                         SsimWin win, float weight, float* __restrict__ dx) {
    const int64_t HW = (int64_t)W * H, total = (int64_t)planes * HW;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / HW, rem = e - p * HW;
        const int r = (int)(rem / W), c = (int)(rem - (int64_t)r * W);
        float g[3] = {0.f, 0.f, 0.f};
        for (int k = -SSIM_R; k <= SSIM_R; ++k) {
            const int rr = r + k;
            if (rr < 0 || rr >= H) continue;
            const float wk = win.w[k + SSIM_R];
            const int64_t i = p * HW + (int64_t)rr * W + c;
#pragma unroll
            for (int q = 0; q < 3; ++q) g[q] += wk * hc[(int64_t)q * total + i];
        }
        dx[e] += weight * (g[0] + 2.f * x[e] * g[1] + y[e] * g[2]);
    }
}

__global__ void ssim_finish_kernel(const float* ssim_sum, float inv_m, float weight, float* loss) {
    *loss = weight * (1.f - *ssim_sum * inv_m);
}

vg_status launch_ssim(int n_views, int W, int H, const float* C, const float* Ct, float weight, float* dC, float* loss,
                   float* ws, cudaStream_t st) {
    SsimWin win;
    double g[2 * SSIM_R + 1], sum = 0.0;
    for (int k = -SSIM_R; k <= SSIM_R; ++k) sum += g[k + SSIM_R] = std::exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
    for (int k = 0; k < 2 * SSIM_R + 1; ++k) win.w[k] = (float)(g[k] / sum);
    const int planes = 3 * n_views;
    const int64_t total = (int64_t)planes * W * H;
    const float inv_m = 1.f / (float)total;
    float* hs = ws;                 // [5][total] horizontal statistics, reused for [3][total] filtered coefficients
    float* coef = ws + 5 * total;   // [3][total]
    float* ssum = ws + 8 * total;   // [1]
    int64_t blocks = ceil_div(total, 256);
    if (blocks > 148 * 8) blocks = 148 * 8;
    cudaError_t e = cudaMemsetAsync(ssum, 0, 4, st);
    if (e != cudaSuccess) return set_error(VG_ERR_CUDA, cudaGetErrorString(e));
    count_launches(2 + (dC ? 2 : 0) + (loss ? 1 : 0));
    ssim_hpass_kernel<<<(unsigned)blocks, 256, 0, st>>>(planes, W, H, C, Ct, nullptr, 5, hs, win);
    ssim_vstats_kernel<<<(unsigned)blocks, 256, 0, st>>>(planes, W, H, hs, win, inv_m, coef, ssum);
    if (dC) {
        ssim_hpass_kernel<<<(unsigned)blocks, 256, 0, st>>>(planes, W, H, nullptr, nullptr, coef, 3, hs, win);
        ssim_vgrad_kernel<<<(unsigned)blocks, 256, 0, st>>>(planes, W, H, hs, C, Ct, win, weight, dC);
    }
    if (loss) ssim_finish_kernel<<<1, 1, 0, st>>>(ssum, inv_m, weight, loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? VG_OK : set_error(VG_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace vgk
