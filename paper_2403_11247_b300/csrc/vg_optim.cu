// vg_optim.cu -- on-device optimiser steps for map parameters (Adam over up
// to 16 arrays in one launch) and camera poses (Adam on the pose twist, then
// the pose moves by the SE(3) exponential of the step, left-multiplied).
#include "vg_internal.h"

namespace vgk {

struct AdamPack {
    int32_t n;
    uint32_t zero_mask;  // bit t: tensor t's gradient is zeroed once read
    float* p[16];
    float* g[16];
    float* m[16];
    float* v[16];
    int64_t size[16];
    int64_t chunk_end[16];  // running total of ceil(size / 4) over tensors 0..t
};

// The update's square root and quotient go through the hardware reciprocal
// square root and the fast divide (about 2 ulp each; the IEEE forms cost more
// issue slots than the kernel's memory traffic).  sqrt(v) is taken as 0 below
// the smallest normal number, where it is far under any eps.
__device__ __forceinline__ void adam_update(float& p, float& m, float& v, float g, float b1, float b2, float step_size,
                                            float inv_sqrt_bc2, float eps) {
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    const float sv = v >= 1.17549435e-38f ? v * rsqrtf(v) : 0.f;
    p -= __fdividef(step_size * m, sv * inv_sqrt_bc2 + eps);
}

// one index space of four-element chunks over all tensors, so that every
// thread issues the loads of its chunk at once instead of walking the tensors
// one after another (one DRAM round trip per launch, not one per tensor); a
// chunk goes through float4 loads where its tensor's four arrays are 16-byte
// aligned and it is whole.
__global__ void __launch_bounds__(256) adam_kernel(const __grid_constant__ AdamPack A, float lr, float b1, float b2,
                                                   float eps, const int32_t* step_dev, int32_t step_host) {
    // the bias corrections, once per block (the powers cost as many issue
    // slots as a thread's whole update)
    __shared__ float s_bc[2];
    if (threadIdx.x == 0) {
        const int32_t step = step_dev ? step_dev[0] : step_host;
        s_bc[0] = 1.f - powf(b1, (float)step);
        s_bc[1] = 1.f - powf(b2, (float)step);
    }
    __syncthreads();
    const float step_size = lr / s_bc[0];
    const float inv_sqrt_bc2 = rsqrtf(s_bc[1]);
    allow_dependents();  // the step counter's increment may wait on the device
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = A.chunk_end[A.n - 1];
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += nthr) {
        int t = 0;
        while (c >= A.chunk_end[t]) ++t;
        float* __restrict__ P = A.p[t];
        float* __restrict__ G = A.g[t];
        const bool zg = (A.zero_mask >> t) & 1u;
        float* __restrict__ M = A.m[t];
        float* __restrict__ Vv = A.v[t];
        const int64_t n = A.size[t];
        const int64_t i0 = (c - (t ? A.chunk_end[t - 1] : 0)) * 4;
        const bool vec = i0 + 4 <= n && ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(G) |
                                          reinterpret_cast<uintptr_t>(M) | reinterpret_cast<uintptr_t>(Vv)) & 15u) == 0;
        if (vec) {
            const int64_t i = i0 / 4;
            float4 p = reinterpret_cast<float4*>(P)[i];
            float4 m = reinterpret_cast<float4*>(M)[i];
            float4 v = reinterpret_cast<float4*>(Vv)[i];
            const float4 g = reinterpret_cast<const float4*>(G)[i];
            if (zg) reinterpret_cast<float4*>(G)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            adam_update(p.x, m.x, v.x, g.x, b1, b2, step_size, inv_sqrt_bc2, eps);
            adam_update(p.y, m.y, v.y, g.y, b1, b2, step_size, inv_sqrt_bc2, eps);
            adam_update(p.z, m.z, v.z, g.z, b1, b2, step_size, inv_sqrt_bc2, eps);
            adam_update(p.w, m.w, v.w, g.w, b1, b2, step_size, inv_sqrt_bc2, eps);
            reinterpret_cast<float4*>(P)[i] = p;
            reinterpret_cast<float4*>(M)[i] = m;
            reinterpret_cast<float4*>(Vv)[i] = v;
        } else {
            const int64_t i1 = i0 + 4 < n ? i0 + 4 : n;
            for (int64_t i = i0; i < i1; ++i) {
                float p = P[i], m = M[i], v = Vv[i];
                const float g = G[i];
                if (zg) G[i] = 0.f;
                adam_update(p, m, v, g, b1, b2, step_size, inv_sqrt_bc2, eps);
                P[i] = p;
                M[i] = m;
                Vv[i] = v;
            }
        }
    }
}

// (overlapped launch after the optimiser kernel of the same call: resident
// while that kernel runs, it waits on the device for it)
__global__ void step_increment_kernel(int32_t* step_dev) {
    grid_dependency_wait();
    step_dev[0] += 1;
}

cudaError_t launch_adam(int n, float* const* p, float* const* g, float* const* m, float* const* v,
                        const int64_t* size, uint32_t zero_mask, float lr, float b1, float b2, float eps,
                        int32_t* step_dev, int32_t step_host, cudaStream_t st) {
    AdamPack A;
    A.n = n;
    A.zero_mask = zero_mask;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        A.p[i] = p[i];
        A.g[i] = g[i];
        A.m[i] = m[i];
        A.v[i] = v[i];
        A.size[i] = size[i];
        total += ceil_div(size[i], 4);
        A.chunk_end[i] = total;
    }
    if (total > 0) {
        int64_t blocks = ceil_div(total, 256);
        if (blocks > 148 * 16) blocks = 148 * 16;
        count_launches(1);
        adam_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, lr, b1, b2, eps, step_dev, step_host);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (step_dev) return launch_overlapped(step_increment_kernel, dim3(1), dim3(1), 0, st, step_dev);
    return cudaSuccess;
}

// SE(3) exponential of xi = (rho, phi): R = exp([phi]x) (Rodrigues),
// t = V rho with V = I + (1 - cos a)/a^2 [phi]x + (a - sin a)/a^3 [phi]x^2
__device__ void se3_exp(const float xi[6], float R[3][3], float t[3]) {
    const float px = xi[3], py = xi[4], pz = xi[5];
    const float a2 = px * px + py * py + pz * pz;
    const float a = sqrtf(a2);
    float A, B, Cc;
    if (a < 1e-4f) {
        A = 1.f - a2 / 6.f;
        B = 0.5f - a2 / 24.f;
        Cc = 1.f / 6.f - a2 / 120.f;
    } else {
        A = sinf(a) / a;
        B = (1.f - cosf(a)) / a2;
        Cc = (a - sinf(a)) / (a2 * a);
    }
    const float K[3][3] = {{0.f, -pz, py}, {pz, 0.f, -px}, {-py, px, 0.f}};
    float K2[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) K2[r][c] = K[r][0] * K[0][c] + K[r][1] * K[1][c] + K[r][2] * K[2][c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            const float I = r == c ? 1.f : 0.f;
            R[r][c] = I + A * K[r][c] + B * K2[r][c];
        }
    for (int r = 0; r < 3; ++r) {
        float acc = 0.f;
        for (int c = 0; c < 3; ++c) {
            const float I = r == c ? 1.f : 0.f;
            acc += (I + B * K[r][c] + Cc * K2[r][c]) * xi[c];
        }
        t[r] = acc;
    }
}

__global__ void pose_step_kernel(int n_views, float* pose, const float* dxi, float* m, float* v, float lr_rot,
                                 float lr_trans, float b1, float b2, float eps, const int32_t* step_dev,
                                 int32_t step_host) {
    allow_dependents();  // the step counter's increment may wait on the device
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_views) return;
    const int32_t step = step_dev ? step_dev[0] : step_host;
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    float d[6];
    for (int c = 0; c < 6; ++c) {
        const float g = dxi[w * 6 + c];
        const float mm = b1 * m[w * 6 + c] + (1.f - b1) * g;
        const float vv = b2 * v[w * 6 + c] + (1.f - b2) * g * g;
        m[w * 6 + c] = mm;
        v[w * 6 + c] = vv;
        const float lr = c < 3 ? lr_trans : lr_rot;
        d[c] = -lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
    float R[3][3], t[3];
    se3_exp(d, R, t);
    float* T = pose + w * 12;
    float out[12];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 4; ++c) {
            float acc = R[r][0] * T[0 * 4 + c] + R[r][1] * T[1 * 4 + c] + R[r][2] * T[2 * 4 + c];
            if (c == 3) acc += t[r];
            out[r * 4 + c] = acc;
        }
    }
    for (int i = 0; i < 12; ++i) T[i] = out[i];
}

cudaError_t launch_pose_step(int n_views, float* pose, const float* dxi, float* m, float* v, float lr_rot,
                             float lr_trans, float b1, float b2, float eps, int32_t* step_dev, int32_t step_host,
                             cudaStream_t st) {
    count_launches(1);
    pose_step_kernel<<<(unsigned)ceil_div(n_views, 64), 64, 0, st>>>(n_views, pose, dxi, m, v, lr_rot, lr_trans, b1,
                                                                      b2, eps, step_dev, step_host);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (step_dev) return launch_overlapped(step_increment_kernel, dim3(1), dim3(1), 0, st, step_dev);
    return cudaSuccess;
}

}  // namespace vgk
