// vg_ssim.cu -- the SSIM term the local-to-global bundle adjustment adds to
// the RGB rendering (Sec. "Tracking and Local-to-Global Bundle Adjustment"):
// L = 1 - mean SSIM(C, C_target) over views, channels and pixels, with an
// 11x11 Gaussian window (sigma 1.5, separable), zero padding, C1 = 0.01^2,
// C2 = 0.03^2, and its gradient with respect to C.
//
// One kernel per 32x32 output tile of one colour plane, everything in shared
// memory: the inputs with a 10-pixel halo; a horizontal and a vertical 11-tap
// pass over x, y, x^2, y^2, xy give the local means and second moments on the
// tile plus a 5-pixel halo; SSIM there and the three coefficient maps of its
// gradient (d/dmu_x, d/dsigma_x^2, d/dsigma_xy, pre-combined; zero outside the
// image, the adjoint of the zero padding); the same two passes over the
// coefficient maps give dL/dx = G*A + 2 x (G*B) + y (G*Cc) on the tile.  Each
// thread of a pass slides along a strip of outputs with the inputs in
// registers (one shared-memory load per input, not per tap).  The
// halo is recomputed by neighbouring tiles instead of going through memory:
// C and C_target are read (from L2 for the halo) and dC read-modify-written,
// 16 bytes per colour value.
#include <cmath>

#include "vg_internal.h"

namespace vgk {

constexpr int SSIM_R = 5;                   // window radius (11 taps)
constexpr int SSIM_T = 32;                  // output tile side
constexpr int SSIM_S = SSIM_T + 2 * SSIM_R;  // statistics region side (42)
constexpr int SSIM_I = SSIM_T + 4 * SSIM_R;  // input region side (52)
// the coefficient maps reuse the inputs' memory, their horizontal pass the
// statistics': 65 KB, three blocks per SM
constexpr int SSIM_SMEM_FLOATS = 2 * SSIM_I * SSIM_I + 5 * SSIM_I * SSIM_S;
static_assert(3 * SSIM_S * SSIM_S <= 2 * SSIM_I * SSIM_I && 3 * SSIM_S * SSIM_T <= 5 * SSIM_I * SSIM_S, "aliasing");
static_assert(SSIM_S % 7 == 0 && SSIM_T % 8 == 0 && SSIM_T % 4 == 0, "strip lengths of the filter passes");

struct SsimWin {
    float w[2 * SSIM_R + 1];
};

__global__ void __launch_bounds__(256) ssim_tile_kernel(int W, int H, const float* __restrict__ x,
                                                        const float* __restrict__ y, SsimWin win, float inv_m,
                                                        float weight, float* __restrict__ dx,
                                                        float* __restrict__ ssim_sum) {
    extern __shared__ float sm[];
    float* sx = sm;                              // [52][52] inputs, zero outside the image
    float* sy = sx + SSIM_I * SSIM_I;
    float* hs = sy + SSIM_I * SSIM_I;            // [5][52][42] horizontal statistics
    float* coef = sm;                            // [3][42][42] coefficient maps (reuses sx, sy)
    float* hc = hs;                              // [3][42][32] their horizontal pass (reuses hs)
    __shared__ float s_tmp[8];
    const int ox = blockIdx.x * SSIM_T, oy = blockIdx.y * SSIM_T;
    const int64_t HW = (int64_t)W * H;
    const float* xp = x + blockIdx.z * HW;
    const float* yp = y + blockIdx.z * HW;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;

    for (int i = threadIdx.x; i < SSIM_I * SSIM_I; i += blockDim.x) {
        const int r = i / SSIM_I, c = i - r * SSIM_I;
        const int gy = oy - 2 * SSIM_R + r, gx = ox - 2 * SSIM_R + c;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        sx[i] = in ? xp[(int64_t)gy * W + gx] : 0.f;
        sy[i] = in ? yp[(int64_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    // horizontal pass of x, y, x^2, y^2, xy: a thread slides along 7 outputs
    // of one row, every input loaded once from shared memory
    for (int it = threadIdx.x; it < SSIM_I * (SSIM_S / 7); it += blockDim.x) {
        const int r = it / (SSIM_S / 7), c0 = (it - r * (SSIM_S / 7)) * 7;
        float a[7][5];
#pragma unroll
        for (int j = 0; j < 7; ++j)
#pragma unroll
            for (int q = 0; q < 5; ++q) a[j][q] = 0.f;
#pragma unroll
        for (int i = 0; i < 7 + 2 * SSIM_R; ++i) {
            const float u = sx[r * SSIM_I + c0 + i], v = sy[r * SSIM_I + c0 + i];
            const float f[5] = {u, v, u * u, v * v, u * v};
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                const int k = i - j;
                if (k < 0 || k > 2 * SSIM_R) continue;
#pragma unroll
                for (int q = 0; q < 5; ++q) a[j][q] += win.w[k] * f[q];
            }
        }
#pragma unroll
        for (int j = 0; j < 7; ++j)
#pragma unroll
            for (int q = 0; q < 5; ++q) hs[q * SSIM_I * SSIM_S + r * SSIM_S + c0 + j] = a[j][q];
    }
    __syncthreads();
    // vertical pass, SSIM and the coefficient maps: a thread slides down 7
    // outputs of one column (the inputs' memory is free from here on)
    float local = 0.f;
    for (int it = threadIdx.x; it < SSIM_S * (SSIM_S / 7); it += blockDim.x) {
        const int c = it % SSIM_S, r0 = (it / SSIM_S) * 7;
        float m[7][5];
#pragma unroll
        for (int j = 0; j < 7; ++j)
#pragma unroll
            for (int q = 0; q < 5; ++q) m[j][q] = 0.f;
#pragma unroll
        for (int i = 0; i < 7 + 2 * SSIM_R; ++i) {
            float h[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) h[q] = hs[q * SSIM_I * SSIM_S + (r0 + i) * SSIM_S + c];
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                const int k = i - j;
                if (k < 0 || k > 2 * SSIM_R) continue;
#pragma unroll
                for (int q = 0; q < 5; ++q) m[j][q] += win.w[k] * h[q];
            }
        }
        const int gx = ox - SSIM_R + c;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const int r = r0 + j, gy = oy - SSIM_R + r;
            float A = 0.f, B = 0.f, Cc = 0.f;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
                const float mx = m[j][0], my = m[j][1];
                const float sxx = m[j][2] - mx * mx, syy = m[j][3] - my * my, sxy = m[j][4] - mx * my;
                const float a1 = 2.f * mx * my + C1, a2 = 2.f * sxy + C2;
                const float b1 = mx * mx + my * my + C1, b2 = sxx + syy + C2;
                const float inv_b = 1.f / (b1 * b2);
                const float S = a1 * a2 * inv_b;
                // each pixel's SSIM counts once: in the tile that owns it
                if (r >= SSIM_R && r < SSIM_R + SSIM_T && c >= SSIM_R && c < SSIM_R + SSIM_T) local += S;
                const float dmx = 2.f * my * a2 * inv_b - 2.f * mx * S / b1;
                const float dsxx = -S / b2;
                const float dsxy = 2.f * a1 * inv_b;
                A = -(dmx - 2.f * mx * dsxx - my * dsxy) * inv_m;
                B = -dsxx * inv_m;
                Cc = -dsxy * inv_m;
            }
            coef[r * SSIM_S + c] = A;
            coef[SSIM_S * SSIM_S + r * SSIM_S + c] = B;
            coef[2 * SSIM_S * SSIM_S + r * SSIM_S + c] = Cc;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0 && ssim_sum) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_tmp[w];
        atomicAdd(ssim_sum, t);
    }
    if (!dx) return;
    // horizontal pass of the coefficient maps: 8 outputs of one row per thread
    for (int it = threadIdx.x; it < SSIM_S * (SSIM_T / 8); it += blockDim.x) {
        const int r = it % SSIM_S, c0 = (it / SSIM_S) * 8;
        float a[8][3];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 3; ++q) a[j][q] = 0.f;
#pragma unroll
        for (int i = 0; i < 8 + 2 * SSIM_R; ++i) {
            float f[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) f[q] = coef[q * SSIM_S * SSIM_S + r * SSIM_S + c0 + i];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = i - j;
                if (k < 0 || k > 2 * SSIM_R) continue;
#pragma unroll
                for (int q = 0; q < 3; ++q) a[j][q] += win.w[k] * f[q];
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < 3; ++q) hc[q * SSIM_S * SSIM_T + r * SSIM_T + c0 + j] = a[j][q];
    }
    __syncthreads();
    // vertical pass and the gradient: 4 outputs of one column per thread
    float* dp = dx + blockIdx.z * HW;
    for (int it = threadIdx.x; it < SSIM_T * (SSIM_T / 4); it += blockDim.x) {
        const int c = it % SSIM_T, r0 = (it / SSIM_T) * 4;
        float g[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 3; ++q) g[j][q] = 0.f;
#pragma unroll
        for (int i = 0; i < 4 + 2 * SSIM_R; ++i) {
            float f[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) f[q] = hc[q * SSIM_S * SSIM_T + (r0 + i) * SSIM_T + c];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = i - j;
                if (k < 0 || k > 2 * SSIM_R) continue;
#pragma unroll
                for (int q = 0; q < 3; ++q) g[j][q] += win.w[k] * f[q];
            }
        }
        const int gx = ox + c;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + j, gy = oy + r;
            if (gy >= H || gx >= W) continue;
            const int64_t e = (int64_t)gy * W + gx;
            dp[e] += weight * (g[j][0] + 2.f * xp[e] * g[j][1] + yp[e] * g[j][2]);
        }
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
    float* ssum = loss ? ws : nullptr;
    const size_t smem = (size_t)SSIM_SMEM_FLOATS * sizeof(float);
    cudaError_t e = allow_dynamic_smem((const void*)ssim_tile_kernel, smem);
    if (e == cudaSuccess && ssum) e = cudaMemsetAsync(ssum, 0, 4, st);
    if (e != cudaSuccess) return set_error(VG_ERR_CUDA, cudaGetErrorString(e));
    if (!dC && !loss) return VG_OK;
    const dim3 grid((unsigned)ceil_div(W, SSIM_T), (unsigned)ceil_div(H, SSIM_T), (unsigned)planes);
    count_launches(1 + (loss ? 1 : 0));
    ssim_tile_kernel<<<grid, 256, smem, st>>>(W, H, C, Ct, win, inv_m, weight, dC, ssum);
    if (loss) ssim_finish_kernel<<<1, 1, 0, st>>>(ssum, inv_m, weight, loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? VG_OK : set_error(VG_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace vgk
