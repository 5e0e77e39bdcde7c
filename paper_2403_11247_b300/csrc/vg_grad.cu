// vg_grad.cu -- per-Gaussian chain rule from 2D gradients to the scene
// (projection Eq. 2-3, anchor decode Eq. 7, codebook decode Eq. 14, mask
// straight-through estimator Eq. 11-12), the camera-pose twist gradient, the
// deterministic codebook-gradient reduction, the ICP term (Eq. 20) and the L1
// photometric/depth loss gradient images.
#include "vg_internal.h"

namespace vgk {

constexpr int CHAIN_THREADS = 256;

__device__ __forceinline__ float block_sum_256(float x, float* s_tmp /*[8]*/) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_tmp[warp] = x;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_tmp[w];
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(CHAIN_THREADS) chain_kernel(SceneDev S, const __grid_constant__ Views V, Consts cs,
                                                             const float* __restrict__ g2d, float* __restrict__ dattr,
                                                             float* raw0, float* raw1, float* raw2, float* raw3,
                                                             float* d_xyz, float* d_l, float* d_off, float* d_mask,
                                                             float* __restrict__ pose_part,
                                                             uint32_t* __restrict__ touched_mask,
                                                             const uint32_t* __restrict__ ntiles) {
    __shared__ float s_red[8][6];
    const int64_t n = (int64_t)blockIdx.x * CHAIN_THREADS + threadIdx.x;
    const bool live = n < S.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float mu[3] = {0, 0, 0}, ls[3] = {0, 0, 0}, q[4] = {1, 0, 0, 0}, ol = 0, rgb[3];
    bool active = false;
    float R[3][3], s[3] = {1, 1, 1}, qn[4] = {1, 0, 0, 0}, qnorm = 1.f, Sig[3][3];
    // most Gaussians reach no pixel of any view: their gradients are zero and
    // they need no decode
    // only slots visible in the last forward carry gradient rows
    bool touched = false;
    if (live) {
        for (int v = 0; v < V.n && !touched; ++v) {
            if (ntiles[(int64_t)v * S.N + n] == 0u) continue;
            const float* gg = g2d + ((int64_t)v * S.N + n) * G2D_STRIDE;
#pragma unroll
            for (int c = 0; c < 10; ++c) touched |= gg[c] != 0.f;
        }
    }
    {
        const uint32_t tm = __ballot_sync(0xffffffffu, live && touched);
        if (lane == 0) touched_mask[n >> 5] = tm;
    }
    if (live && touched) {
        anchor_mean(S, n, mu);
        decode_attr<3>(S, 0, n, ls);
        decode_attr<4>(S, 1, n, q);
        decode_attr<1>(S, 2, n, &ol);
        decode_attr<3>(S, 3, n, rgb);
        active = S.mask ? (__ldg(S.mask + n) > S.mask_thr) : true;
        const float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
        active = active && qq > 0.f;
        if (active) {
            qnorm = sqrtf(qq);
#pragma unroll
            for (int c = 0; c < 4; ++c) qn[c] = q[c] / qnorm;
#pragma unroll
            for (int c = 0; c < 3; ++c) s[c] = expf(ls[c]);
        }
    }
    quat_rot(qn, R);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Sig[r][c] = R[r][0] * R[c][0] * s[0] * s[0] + R[r][1] * R[c][1] * s[1] * s[1] + R[r][2] * R[c][2] * s[2] * s[2];

    float dmu[3] = {0, 0, 0}, dSig[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, dop = 0.f, drgb[3] = {0, 0, 0};
    for (int v = 0; v < V.n; ++v) {
        float pose[6] = {0, 0, 0, 0, 0, 0};
        if (live && active && ntiles[(int64_t)v * S.N + n] != 0u) {
            const float* gg = g2d + ((int64_t)v * S.N + n) * G2D_STRIDE;
            float g[10];
            bool nz = false;
#pragma unroll
            for (int c = 0; c < 10; ++c) {
                g[c] = gg[c];
                nz |= g[c] != 0.f;
            }
            if (nz) {
                const ViewInfo& vi = V.v[v];
                float T[12];
                view_pose(V, v, T);
                float p[3];
                cam_point(T, mu, p);
                const float x = p[0], y = p[1], z = p[2];
                const float fx = vi.fx, fy = vi.fy;
                float txz = x / z, tyz = y / z;
                bool ux = true, uy = true;
                if (cs.jacobian_clamp) {
                    if (txz < -vi.limx || txz > vi.limx) { ux = false; txz = fminf(fmaxf(txz, -vi.limx), vi.limx); }
                    if (tyz < -vi.limy || tyz > vi.limy) { uy = false; tyz = fminf(fmaxf(tyz, -vi.limy), vi.limy); }
                }
                const float J00 = fx / z, J02 = -fx * txz / z, J11 = fy / z, J12 = -fy * tyz / z;
                const float W[3][3] = {{T[0], T[1], T[2]}, {T[4], T[5], T[6]}, {T[8], T[9], T[10]}};
                float T1[3][3], Sc[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) T1[r][c] = W[r][0] * Sig[0][c] + W[r][1] * Sig[1][c] + W[r][2] * Sig[2][c];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) Sc[r][c] = T1[r][0] * W[c][0] + T1[r][1] * W[c][1] + T1[r][2] * W[c][2];
                const float A = J00 * J00 * Sc[0][0] + 2.f * J00 * J02 * Sc[0][2] + J02 * J02 * Sc[2][2] + cs.dilation;
                const float B = J00 * J11 * Sc[0][1] + J00 * J12 * Sc[0][2] + J02 * J11 * Sc[1][2] + J02 * J12 * Sc[2][2];
                const float C = J11 * J11 * Sc[1][1] + 2.f * J11 * J12 * Sc[1][2] + J12 * J12 * Sc[2][2] + cs.dilation;
                const float det = A * C - B * B;
                const float i2 = 1.f / (det * det);
                const float da = g[2], db = g[3], dc = g[4];
                // conic = inverse of [[A,B],[B,C]]
                const float dA = i2 * (-C * C * da + B * C * db - B * B * dc);
                const float dB = i2 * (2.f * B * C * da - (A * C + B * B) * db + 2.f * A * B * dc);
                const float dC = i2 * (-B * B * da + A * B * db - A * A * dc);
                const float hB = 0.5f * dB;
                const float Jr[2][3] = {{J00, 0.f, J02}, {0.f, J11, J12}};
                float dSc[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        dSc[r][c] = dA * Jr[0][r] * Jr[0][c] + hB * (Jr[0][r] * Jr[1][c] + Jr[1][r] * Jr[0][c]) +
                                    dC * Jr[1][r] * Jr[1][c];
                float JS[2][3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    JS[0][c] = J00 * Sc[0][c] + J02 * Sc[2][c];
                    JS[1][c] = J11 * Sc[1][c] + J12 * Sc[2][c];
                }
                const float dJ00 = 2.f * (dA * JS[0][0] + hB * JS[1][0]);
                const float dJ02 = 2.f * (dA * JS[0][2] + hB * JS[1][2]);
                const float dJ11 = 2.f * (hB * JS[0][1] + dC * JS[1][1]);
                const float dJ12 = 2.f * (hB * JS[0][2] + dC * JS[1][2]);
                const float z2 = z * z, z3 = z2 * z;
                const float dJ02_dx = ux ? -fx / z2 : 0.f;
                const float dJ12_dy = uy ? -fy / z2 : 0.f;
                const float dJ02_dz = fx * txz / z2 + (ux ? fx * x / z3 : 0.f);
                const float dJ12_dz = fy * tyz / z2 + (uy ? fy * y / z3 : 0.f);
                const float du = g[0], dv = g[1], ddepth = g[9];
                float dp[3];
                dp[0] = du * fx / z + dJ02 * dJ02_dx;
                dp[1] = dv * fy / z + dJ12 * dJ12_dy;
                dp[2] = -du * fx * x / z2 - dv * fy * y / z2 + ddepth - dJ00 * fx / z2 - dJ11 * fy / z2 +
                        dJ02 * dJ02_dz + dJ12 * dJ12_dz;
#pragma unroll
                for (int c = 0; c < 3; ++c) dmu[c] += W[0][c] * dp[0] + W[1][c] * dp[1] + W[2][c] * dp[2];
                float T2[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) T2[r][c] = dSc[r][0] * W[0][c] + dSc[r][1] * W[1][c] + dSc[r][2] * W[2][c];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) dSig[r][c] += W[0][r] * T2[0][c] + W[1][r] * T2[1][c] + W[2][r] * T2[2][c];
                dop += g[5];
                drgb[0] += g[6];
                drgb[1] += g[7];
                drgb[2] += g[8];
                // left perturbation: p += phi x p + rho ; Sc += [phi]x Sc - Sc [phi]x
                float M[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        M[r][c] = Sc[r][0] * dSc[0][c] + Sc[r][1] * dSc[1][c] + Sc[r][2] * dSc[2][c] -
                                  (dSc[r][0] * Sc[0][c] + dSc[r][1] * Sc[1][c] + dSc[r][2] * Sc[2][c]);
                pose[0] = dp[0];
                pose[1] = dp[1];
                pose[2] = dp[2];
                pose[3] = p[1] * dp[2] - p[2] * dp[1] - 2.f * M[2][1];
                pose[4] = p[2] * dp[0] - p[0] * dp[2] - 2.f * M[0][2];
                pose[5] = p[0] * dp[1] - p[1] * dp[0] - 2.f * M[1][0];
            }
        }
        // block reduction of the six pose components for view v
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float x = pose[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) s_red[warp][c] = x;
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            float t = 0.f;
            for (int w = 0; w < CHAIN_THREADS / 32; ++w) t += s_red[w][threadIdx.x];
            pose_part[((int64_t)v * gridDim.x + blockIdx.x) * 6 + threadIdx.x] = t;
        }
        __syncthreads();
    }

    // Sigma = M M^T with M = R diag(s)
    float dls[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dol = 0.f, ds[3] = {0, 0, 0}, o = 0.f;
    if (live && active) {
        float dM[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float acc = 0.f;
#pragma unroll
                for (int m = 0; m < 3; ++m) acc += (dSig[r][m] + dSig[m][r]) * R[m][c] * s[c];
                dM[r][c] = acc;
            }
        float dR[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ds[c] = dM[0][c] * R[0][c] + dM[1][c] * R[1][c] + dM[2][c] * R[2][c];
            dls[c] = ds[c] * s[c];
#pragma unroll
            for (int r = 0; r < 3; ++r) dR[r][c] = dM[r][c] * s[c];
        }
        const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
        float dqn[4];
        dqn[0] = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
        dqn[1] = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] + z * dR[2][0] +
                        w * dR[2][1] - 2.f * x * dR[2][2]);
        dqn[2] = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] - w * dR[2][0] +
                        z * dR[2][1] - 2.f * y * dR[2][2]);
        dqn[3] = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                        y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
        const float dot = qn[0] * dqn[0] + qn[1] * dqn[1] + qn[2] * dqn[2] + qn[3] * dqn[3];
#pragma unroll
        for (int c = 0; c < 4; ++c) dq[c] = (dqn[c] - qn[c] * dot) / qnorm;
        o = 1.f / (1.f + expf(-ol));
        dol = dop * o * (1.f - o);
    } else {
        drgb[0] = drgb[1] = drgb[2] = 0.f;
    }
    if (live) {
        const float* vals[4] = {dls, dq, &dol, drgb};
        float* raws[4] = {raw0, raw1, raw2, raw3};
#pragma unroll
        for (int gi = 0; gi < 4; ++gi) {
            const int d = gdim(gi);
            if (S.L[gi] > 0) {
                // untouched Gaussians are skipped by the codebook reduction
                if (dattr && touched)
                    for (int c = 0; c < d; ++c) dattr[n * ATTR_STRIDE + goff(gi) + c] = vals[gi][c];
            } else if (raws[gi]) {
                for (int c = 0; c < d; ++c) raws[gi][n * d + c] = vals[gi][c];
            }
        }
        if (d_mask && S.mask) {
            float dm = 0.f;
            if (active) {
                const float sm = 1.f / (1.f + expf(-__ldg(S.mask + n)));
                dm = (ds[0] * s[0] + ds[1] * s[1] + ds[2] * s[2] + dop * o) * sm * (1.f - sm);
            }
            d_mask[n] = dm;
        } else if (d_mask) {
            d_mask[n] = 0.f;
        }
    }
    // Eq. 7: d x_a = sum_i dmu_i, d O_i = dmu_i * l, d l = sum_i dmu_i * O_i
    const int64_t a = live ? n / S.k : 0;
    float gl[3] = {0, 0, 0}, gx[3] = {dmu[0], dmu[1], dmu[2]};
    if (live) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float l = __ldg(S.l + a * 3 + c);
            if (d_off) d_off[n * 3 + c] = dmu[c] * l;
            gl[c] = dmu[c] * __ldg(S.off + n * 3 + c);
        }
    }
    if ((32 % S.k) == 0) {
        for (int off = S.k >> 1; off > 0; off >>= 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gx[c] += __shfl_xor_sync(0xffffffffu, gx[c], off);
                gl[c] += __shfl_xor_sync(0xffffffffu, gl[c], off);
            }
        }
        if (live && (n % S.k) == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (d_xyz) d_xyz[a * 3 + c] = gx[c];
                if (d_l) d_l[a * 3 + c] = gl[c];
            }
        }
    } else if (live) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (d_xyz) atomicAdd(d_xyz + a * 3 + c, gx[c]);
            if (d_l) atomicAdd(d_l + a * 3 + c, gl[c]);
        }
    }
}

int chain_blocks(int64_t N) { return (int)ceil_div(N > 0 ? N : 1, CHAIN_THREADS); }

// zero the gradient rows of the visible slots (the only rows the backward
// blend writes); all other rows are kept at zero
__global__ void zero_visible_g2d_kernel(const uint32_t* __restrict__ vis, const uint32_t* __restrict__ nvis_dev,
                                        uint32_t max_vis, float* __restrict__ g2d) {
    const uint32_t n = min(*nvis_dev, max_vis);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n * 3; e += gridDim.x * blockDim.x) {
        const uint32_t s = vis[e / 3];
        reinterpret_cast<float4*>(g2d + (int64_t)s * G2D_STRIDE)[e % 3] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

cudaError_t launch_zero_visible_g2d(const uint32_t* vis_slots, const uint32_t* nvis_dev, uint32_t max_vis, float* g2d,
                                    cudaStream_t st) {
    int64_t blocks = ceil_div((int64_t)max_vis * 3, 256);
    if (blocks > 148 * 4) blocks = 148 * 4;
    if (blocks < 1) blocks = 1;
    count_launches(1);
    zero_visible_g2d_kernel<<<(unsigned)blocks, 256, 0, st>>>(vis_slots, nvis_dev, max_vis, g2d);
    return cudaGetLastError();
}

cudaError_t launch_chain(const SceneDev& S, const Views& V, const Consts& cs, const float* g2d, float* dattr, float* r0,
                         float* r1, float* r2, float* r3, float* d_xyz, float* d_l, float* d_off, float* d_mask,
                         float* pose_part, uint32_t* touched, const uint32_t* ntiles, int* n_blocks_out,
                         cudaStream_t st) {
    const int blocks = chain_blocks(S.N);
    if (n_blocks_out) *n_blocks_out = blocks;
    count_launches(1);
    chain_kernel<<<blocks, CHAIN_THREADS, 0, st>>>(S, V, cs, g2d, dattr, r0, r1, r2, r3, d_xyz, d_l, d_off, d_mask,
                                                   pose_part, touched, ntiles);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// codebook gradients: dC^s[k] = sum over Gaussians n with idx[s][n] == k of
// the attribute gradient of n, as a segmented sum over a per-stage
// codeword-sorted Gaussian list (deterministic, no atomics)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) codebook_reduce_kernel(const __grid_constant__ CodebookJobs J, int64_t N,
                                                                const float* __restrict__ dattr,
                                                                const uint32_t* __restrict__ touched) {
    __shared__ float s_tmp[8];
    int j = 0;
    while (j + 1 < J.n && (int)blockIdx.x >= J.block_start[j + 1]) ++j;
    const int local = blockIdx.x - J.block_start[j];
    const int K = J.K[j], dim = J.dim[j], off = J.off[j];
    const int s = local / K, k = local % K;
    const uint32_t* perm = J.perm[j] + (int64_t)s * N;
    const uint32_t b = J.seg[j][s * (K + 1) + k], e = J.seg[j][s * (K + 1) + k + 1];
    float acc[4] = {0, 0, 0, 0};
    // four independent gathers in flight per thread
    uint32_t i = b + threadIdx.x;
    for (; i + 3 * 256 < e; i += 4 * 256) {
        uint32_t n4[4], t4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) n4[u] = __ldg(perm + i + u * 256);
#pragma unroll
        for (int u = 0; u < 4; ++u) t4[u] = (__ldg(touched + (n4[u] >> 5)) >> (n4[u] & 31)) & 1u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (t4[u])
                for (int c = 0; c < dim; ++c) acc[c] += __ldg(dattr + (int64_t)n4[u] * ATTR_STRIDE + off + c);
    }
    for (; i < e; i += 256) {
        const uint32_t n = __ldg(perm + i);
        if ((__ldg(touched + (n >> 5)) >> (n & 31)) & 1u)
            for (int c = 0; c < dim; ++c) acc[c] += __ldg(dattr + (int64_t)n * ATTR_STRIDE + off + c);
    }
    for (int c = 0; c < dim; ++c) {
        const float t = block_sum_256(acc[c], s_tmp);
        if (threadIdx.x == 0) J.out[j][((int64_t)s * K + k) * dim + c] = t;
    }
}

cudaError_t launch_codebook_reduce(const CodebookJobs& J, int64_t N, const float* dattr, const uint32_t* touched,
                                   cudaStream_t st) {
    if (J.n == 0 || J.block_start[J.n] == 0) return cudaSuccess;
    count_launches(1);
    codebook_reduce_kernel<<<J.block_start[J.n], 256, 0, st>>>(J, N, dattr, touched);
    return cudaGetLastError();
}

__global__ void seg_from_hist_kernel(const uint32_t* hist, int K, uint32_t* seg) {
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int k = 0; k < K; ++k) {
            seg[k] = acc;
            acc += hist[k];
        }
        seg[K] = acc;
    }
}

cudaError_t launch_seg_from_hist(const uint32_t* hist, int K, uint32_t* seg, cudaStream_t st) {
    count_launches(1);
    seg_from_hist_kernel<<<1, 32, 0, st>>>(hist, K, seg);
    return cudaGetLastError();
}

__global__ void idx_to_keys_kernel(const uint8_t* __restrict__ idx, int64_t n, uint32_t* __restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = idx[i];
}

cudaError_t launch_idx_to_keys(const uint8_t* idx, int64_t n, uint32_t* keys, cudaStream_t st) {
    int64_t blocks = ceil_div(n > 0 ? n : 1, 256);
    if (blocks > 148 * 16) blocks = 148 * 16;
    count_launches(1);
    idx_to_keys_kernel<<<(unsigned)blocks, 256, 0, st>>>(idx, n, keys);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ICP (Eq. 20): per view, sum over kept Gaussians with weight w of
// w |R mu + t - q|^2 and its pose gradient (rho: 2 w r, phi: p x 2 w r)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) icp_kernel(SceneDev S, const __grid_constant__ Views V, const float* __restrict__ q,
                                                 const float* __restrict__ w, float* __restrict__ part) {
    __shared__ float s_tmp[8];
    const int v = blockIdx.y;
    const int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x;
    float vals[7] = {0, 0, 0, 0, 0, 0, 0};
    if (n < S.N) {
        const float wn = w[(int64_t)v * S.N + n];
        bool active = S.mask ? (__ldg(S.mask + n) > S.mask_thr) : true;
        if (active && wn != 0.f) {
            float qr[4];
            decode_attr<4>(S, 1, n, qr);
            active = (qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]) > 0.f;
        }
        if (active && wn != 0.f) {
            float mu[3], T[12], p[3];
            anchor_mean(S, n, mu);
            view_pose(V, v, T);
            cam_point(T, mu, p);
            const float* qq = q + ((int64_t)v * S.N + n) * 3;
            const float r0 = p[0] - qq[0], r1 = p[1] - qq[1], r2 = p[2] - qq[2];
            const float g0 = 2.f * wn * r0, g1 = 2.f * wn * r1, g2 = 2.f * wn * r2;
            vals[0] = g0;
            vals[1] = g1;
            vals[2] = g2;
            vals[3] = p[1] * g2 - p[2] * g1;
            vals[4] = p[2] * g0 - p[0] * g2;
            vals[5] = p[0] * g1 - p[1] * g0;
            vals[6] = wn * (r0 * r0 + r1 * r1 + r2 * r2);
        }
    }
    for (int c = 0; c < 7; ++c) {
        const float t = block_sum_256(vals[c], s_tmp);
        if (threadIdx.x == 0) part[((int64_t)v * gridDim.x + blockIdx.x) * 7 + c] = t;
    }
}

int icp_blocks(int64_t N) { return (int)ceil_div(N > 0 ? N : 1, 256); }

cudaError_t launch_icp(const SceneDev& S, const Views& V, const float* q, const float* w, float* part, int n_blocks,
                       cudaStream_t st) {
    dim3 grid(n_blocks, V.n);
    count_launches(1);
    icp_kernel<<<grid, 256, 0, st>>>(S, V, q, w, part);
    return cudaGetLastError();
}

__global__ void pose_final_kernel(const float* __restrict__ pose_part, int nb, const float* __restrict__ icp_part,
                                  int nbi, float* __restrict__ dxi, float* __restrict__ icp_loss) {
    __shared__ float s_tmp[8];
    const int v = blockIdx.x;
    for (int c = 0; c < 7; ++c) {
        float acc = 0.f;
        if (c < 6)
            for (int j = threadIdx.x; j < nb; j += blockDim.x) acc += pose_part[((int64_t)v * nb + j) * 6 + c];
        if (icp_part)
            for (int j = threadIdx.x; j < nbi; j += blockDim.x) acc += icp_part[((int64_t)v * nbi + j) * 7 + c];
        const float t = block_sum_256(acc, s_tmp);
        if (threadIdx.x == 0) {
            if (c < 6) dxi[v * 6 + c] = t;
            else if (icp_loss) icp_loss[v] = t;
        }
    }
}

cudaError_t launch_pose_final(int n_views, const float* pose_part, int nb, const float* icp_part, int nbi, float* dxi,
                              float* icp_loss, cudaStream_t st) {
    count_launches(1);
    pose_final_kernel<<<n_views, 256, 0, st>>>(pose_part, nb, icp_part, nbi, dxi, icp_loss);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// L1 colour + weighted L1 depth (valid where the target depth > 0)
// ---------------------------------------------------------------------------
__global__ void count_valid_kernel(const float* __restrict__ Dt, int64_t n, uint32_t* count) {
    uint32_t c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += Dt[i] > 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void loss_l1_kernel(int64_t n_pix, int64_t total, const float* __restrict__ C, const float* __restrict__ D,
                               const float* __restrict__ S, const float* __restrict__ Ct, const float* __restrict__ Dt,
                               float w_depth, float gate, const uint32_t* __restrict__ valid_count,
                               float* __restrict__ dC, float* __restrict__ dD, float* __restrict__ loss) {
    __shared__ float s_tmp[8];
    const float nv = (float)(*valid_count);
    const float inv_c = 1.f / (3.f * (float)total);
    const float inv_d = nv > 0.f ? w_depth / nv : 0.f;
    float acc = 0.f;
    const int64_t v = blockIdx.y;
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
    const float t = block_sum_256(acc, s_tmp);
    if (threadIdx.x == 0) atomicAdd(loss, t);
}

cudaError_t launch_loss_l1(int n_views, int64_t n_pix, const float* C, const float* D, const float* S, const float* Ct,
                           const float* Dt, float w_depth, float gate, float* dC, float* dD, float* loss,
                           uint32_t* valid_count, cudaStream_t st) {
    const int64_t total = (int64_t)n_views * n_pix;
    int64_t blocks = ceil_div(total > 0 ? total : 1, 256);
    if (blocks > 148 * 8) blocks = 148 * 8;
    count_launches(2);
    count_valid_kernel<<<(unsigned)blocks, 256, 0, st>>>(Dt, total, valid_count);
    int64_t bx = ceil_div(n_pix, 256);
    if (bx > 148 * 8) bx = 148 * 8;
    loss_l1_kernel<<<dim3((unsigned)bx, (unsigned)n_views), 256, 0, st>>>(n_pix, total, C, D, S, Ct, Dt, w_depth, gate,
                                                                          valid_count, dC, dD, loss);
    return cudaGetLastError();
}

}  // namespace vgk
