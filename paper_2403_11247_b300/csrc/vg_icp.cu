// vg_icp.cu -- projective data association for the ICP term (Eq. 20): the
// "closest point" q_i of each Gaussian mean, taken as the target depth map's
// back-projected point at the pixel the mean projects to (Sec. "Tracking and
// Local-to-Global Bundle Adjustment").
#include "vg_internal.h"

namespace vgk {

__global__ void __launch_bounds__(256) icp_associate_kernel(SceneDev S, const __grid_constant__ Views V,
                                                            const float* __restrict__ Dt, float max_dist,
                                                            float weight, float* __restrict__ q,
                                                            float* __restrict__ w) {
    const int v = blockIdx.y;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= S.N) return;
    const int64_t o = (int64_t)v * S.N + n;
    float qq[3] = {0.f, 0.f, 0.f}, ww = 0.f;
    const bool active = S.mask ? (__ldg(S.mask + n) > S.mask_thr) : true;
    if (active) {
        const ViewInfo& vi = V.v[v];
        float mu[3], T[12], p[3];
        anchor_mean(S, n, mu);
        view_pose(V, v, T);
        cam_point(T, mu, p);
        if (p[2] > vi.near_plane) {
            const float u = vi.fx * p[0] / p[2] + vi.cx, vv = vi.fy * p[1] / p[2] + vi.cy;
            const int px = __float2int_rn(u), py = __float2int_rn(vv);
            if (px >= 0 && px < vi.W && py >= 0 && py < vi.H) {
                const float d = Dt[vi.pix_base + (int64_t)py * vi.W + px];
                if (d > 0.f && fabsf(p[2] - d) < max_dist) {
                    qq[0] = ((float)px - vi.cx) * d / vi.fx;
                    qq[1] = ((float)py - vi.cy) * d / vi.fy;
                    qq[2] = d;
                    ww = weight;
                }
            }
        }
    }
    q[o * 3 + 0] = qq[0];
    q[o * 3 + 1] = qq[1];
    q[o * 3 + 2] = qq[2];
    w[o] = ww;
}

vg_status launch_icp_associate(const SceneDev& S, const Views& V, const float* Dt, float max_dist, float weight, float* q,
                               float* w, cudaStream_t st) {
    if (S.N == 0) return VG_OK;
    dim3 grid((unsigned)ceil_div(S.N, 256), (unsigned)V.n);
    count_launches(1);
    icp_associate_kernel<<<grid, 256, 0, st>>>(S, V, Dt, max_dist, weight, q, w);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VG_OK : set_error(VG_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace vgk
