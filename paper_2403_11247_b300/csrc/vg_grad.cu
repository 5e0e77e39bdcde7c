// vg_grad.cu -- chain rule from the 2D gradients of the visible slots to the
// scene (projection Eq. 2-3, anchor decode Eq. 7, codebook decode Eq. 14,
// mask straight-through estimator Eq. 11-12) with the codebook gradients
// accumulated in the same pass, the camera-pose twist gradient, the ICP term
// (Eq. 20) and the L1 photometric/depth loss gradient images.
#include <mutex>

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

// codebook accumulators of the chain kernel: group gi's size (0 = none) and
// its global gradient array
__host__ __device__ inline int chain_cb_size(const SceneDev& S, const ChainOut& O, int gi) {
    if (gi < 4) return (S.L[gi] > 0 && O.cb[gi]) ? S.L[gi] * S.K[gi] * gdim(gi) : 0;
    if (gi == 4) return (S.Lo > 0 && O.d_off) ? S.Lo * S.Ko * 3 : 0;
    return (S.Ll > 0 && O.d_l) ? S.Ll * S.Kl * 3 : 0;
}
__host__ __device__ inline float* chain_cb_dst(const ChainOut& O, int gi) {
    return gi < 4 ? O.cb[gi] : (gi == 4 ? O.d_off : O.d_l);
}

// One thread per visible (view, Gaussian) slot: the slot's 2D gradient row
// (from the backward compositing) through the projection (Eq. 3), the
// covariance (Eq. 2), the activations, the anchor decode (Eq. 7), the
// codebook decode (Eq. 14) and the mask (Eq. 11-12) to the scene, plus the
// slot's pose-twist contribution.  The chain rule is linear in the row, so
// a Gaussian seen in several views gets the sum of its slots' contributions:
// every scene gradient is accumulated with atomics into arrays zeroed by
// zero_bwd_kernel.  Codebook gradients accumulate per block in shared
// memory (when the codebooks fit) and are flushed once per block.
__global__ void __launch_bounds__(CHAIN_THREADS) chain_kernel(
    SceneDev S, const __grid_constant__ Views V, Consts cs, const float* __restrict__ g2d,
    const uint32_t* __restrict__ vis, const uint32_t* __restrict__ nvis_dev, uint32_t max_vis, ChainOut O) {
    allow_dependents();  // the pose kernel that reads the sums may wait on the device
    extern __shared__ float s_dyn[];  // [V.n][6] pose sums, then the codebook-gradient accumulators
    float* s_pose = s_dyn;
    float* s_cb = s_dyn + V.n * 6;
    const int n_acc = V.n * 6 + (O.cb_in_smem ? O.cb_total : 0);
    for (int i = threadIdx.x; i < n_acc; i += blockDim.x) s_dyn[i] = 0.f;
    __syncthreads();
    const uint32_t nvis = min(*nvis_dev, max_vis);
    const int lane = threadIdx.x & 31;
    // warp-uniform trip count, so that the pose sums can use warp shuffles;
    // consecutive 32-slot chunks go to consecutive blocks, so that a visible
    // set smaller than the grid still spreads over every SM
    // Only a thread's first slot waits for the backward compositing before
    // loading its gradient row; later slots (scenes with more visible slots
    // than threads) load the row together with the attributes.
    bool waited = false;
    for (uint32_t base = ((threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32u; base < nvis;
         base += gridDim.x * blockDim.x) {
        const uint32_t e = base + lane;
        float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int pv = -1;  // view of this lane's pose contribution, -1 = none
        do {
            if (e >= nvis) break;
            const uint32_t slot = vis[e];
            const int v = slot_view(slot, (uint32_t)S.N, V.n);
            const int64_t n = (int64_t)slot - (int64_t)v * S.N;
            const float4* row = reinterpret_cast<const float4*>(g2d + (int64_t)slot * G2D_STRIDE);
            float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
            if (waited) {  // a slot whose row is zero (seen, never blended) needs nothing else
                r0 = row[0];
                r1 = row[1];
                r2 = row[2];
                if (r0.x == 0.f && r0.y == 0.f && r0.z == 0.f && r0.w == 0.f && r1.x == 0.f && r1.y == 0.f &&
                    r1.z == 0.f && r1.w == 0.f && r2.x == 0.f && r2.y == 0.f)
                    break;
            }
            // Eq. 7's offset and scaling factor, decoded once: the mean here,
            // their own gradients at the end.  Everything up to the 2D
            // covariance depends on the scene alone, so it runs before the
            // wait for the backward compositing (overlapped launch); the codes
            // stay in registers for the codebook gradients.
            const int64_t a = anchor_of(S, n);
            float mu[3], ls[3], q[4], ol, rgb[3], oo[3], la[3];
            uint32_t kp[4][DECODE_STAGES / 4];
            scene_offset(S, n, oo);
            scene_scale(S, a, la);
#pragma unroll
            for (int c = 0; c < 3; ++c) mu[c] = __fadd_rn(__ldg(S.xyz + a * 3 + c), __fmul_rn(oo[c], la[c]));
            decode_attr_codes<3>(S, 0, n, ls, kp[0]);
            decode_attr_codes<4>(S, 1, n, q, kp[1]);
            decode_attr_codes<1>(S, 2, n, &ol, kp[2]);
            decode_attr_codes<3>(S, 3, n, rgb, kp[3]);
            const float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
            if (!(qq > 0.f)) break;
            // one reciprocal per slot for every quotient by |q| and by z below;
            // activations, reciprocals and the sigmoids go through the
            // hardware exp / reciprocal-sqrt and the fast divide (a few ulp,
            // far inside what the gradients are held to)
            const float iq = rsqrtf(qq);  // hardware reciprocal square root
            float qn[4], s[3], R[3][3], Sig[3][3];
#pragma unroll
            for (int c = 0; c < 4; ++c) qn[c] = q[c] * iq;
#pragma unroll
            for (int c = 0; c < 3; ++c) s[c] = __expf(ls[c]);
            quat_rot(qn, R);
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    Sig[r][c] = R[r][0] * R[c][0] * s[0] * s[0] + R[r][1] * R[c][1] * s[1] * s[1] + R[r][2] * R[c][2] * s[2] * s[2];
            float dmu[3] = {0, 0, 0}, dSig[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, dop = 0.f, drgb[3] = {0, 0, 0};
            {
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
                const float iz = __fdividef(1.f, z), iz2 = iz * iz;
                const float J00 = fx * iz, J02 = -fx * txz * iz, J11 = fy * iz, J12 = -fy * tyz * iz;
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
                float A, B, C, det, RS[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) RS[r][c] = R[r][c] * s[c];
                cov2d(J00, J02, J11, J12, T, RS, cs.dilation, A, B, C, det);
                // the slot's 2D gradient row, written by the backward compositing
                if (!waited) {
                    grid_dependency_wait();
                    waited = true;
                    r0 = row[0];
                    r1 = row[1];
                    r2 = row[2];
                }
                float g[12];
                {
                    g[0] = r0.x; g[1] = r0.y; g[2] = r0.z; g[3] = r0.w;
                    g[4] = r1.x; g[5] = r1.y; g[6] = r1.z; g[7] = r1.w;
                    g[8] = r2.x; g[9] = r2.y; g[10] = r2.z; g[11] = r2.w;
                }
                bool nz = false;
#pragma unroll
                for (int c = 0; c < 10; ++c) nz |= g[c] != 0.f;
                if (!nz) break;
                const float i2 = __fdividef(1.f, det * det);
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
                const float dJ02_dx = ux ? -fx * iz2 : 0.f;
                const float dJ12_dy = uy ? -fy * iz2 : 0.f;
                const float dJ02_dz = fx * txz * iz2 + (ux ? fx * x * iz2 * iz : 0.f);
                const float dJ12_dz = fy * tyz * iz2 + (uy ? fy * y * iz2 * iz : 0.f);
                const float du = g[0], dv = g[1], ddepth = g[9];
                float dp[3];
                dp[0] = du * fx * iz + dJ02 * dJ02_dx;
                dp[1] = dv * fy * iz + dJ12 * dJ12_dy;
                dp[2] = -(du * fx * x + dv * fy * y + dJ00 * fx + dJ11 * fy) * iz2 + ddepth + dJ02 * dJ02_dz +
                        dJ12 * dJ12_dz;
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
            pv = v;
            // Sigma = M M^T with M = R diag(s)
            float dls[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dol = 0.f, ds[3] = {0, 0, 0}, o = 0.f;
            {
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
                for (int c = 0; c < 4; ++c) dq[c] = (dqn[c] - qn[c] * dot) * iq;
                o = __fdividef(1.f, 1.f + __expf(-ol));
                dol = dop * o * (1.f - o);
            }
            // attribute gradients: raw arrays, or the indexed codewords of every
            // stage (values picked by compile-time group and component, so that
            // they stay in registers)
            auto gval = [&](int gi, int c) -> float { return gi == 0 ? dls[c] : (gi == 1 ? dq[c] : (gi == 2 ? dol : drgb[c])); };
#pragma unroll
            for (int gi = 0; gi < 4; ++gi) {
                constexpr int dmax = 4;
                const int d = gdim(gi);
                if (S.L[gi] > 0) {
                    if (!O.cb[gi]) continue;
                    auto add_cw = [&](int st, int k) {
                        const int j = (st * S.K[gi] + k) * d;
                        if (O.cb_in_smem) {
#pragma unroll
                            for (int c = 0; c < dmax; ++c)
                                if (c < d) red_add_shared(s_cb + O.cb_off[gi] + j + c, gval(gi, c));
                        } else {
#pragma unroll
                            for (int c = 0; c < dmax; ++c)
                                if (c < d) atomicAdd(O.cb[gi] + j + c, gval(gi, c));
                        }
                    };
#pragma unroll
                    for (int st = 0; st < DECODE_STAGES; ++st)
                        if (st < S.L[gi]) add_cw(st, (int)code_at(kp[gi], st));
                    for (int st = DECODE_STAGES; st < S.L[gi]; ++st)
                        add_cw(st, __ldg(S.idx[gi] + (int64_t)st * S.N + n));
                } else if (O.raw[gi]) {
#pragma unroll
                    for (int c = 0; c < dmax; ++c)
                        if (c < d) atomicAdd(O.raw[gi] + n * d + c, gval(gi, c));
                }
            }
            if (O.d_mask && S.mask) {
                const float sm = __fdividef(1.f, 1.f + __expf(-__ldg(S.mask + n)));
                atomicAdd(O.d_mask + n, (ds[0] * s[0] + ds[1] * s[1] + ds[2] * s[2] + dop * o) * sm * (1.f - sm));
            }
            // Eq. 7: d x_a = sum_i dmu_i, d O_i = dmu_i * l, d l = sum_i dmu_i * O_i;
            // coded O or l pass their gradient to the indexed codeword of every stage
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (O.d_xyz) atomicAdd(O.d_xyz + a * 3 + c, dmu[c]);
            if (O.d_off) {
                if (S.Lo > 0) {
                    for (int st = 0; st < S.Lo; ++st) {
                        const int j = (st * S.Ko + __ldg(S.idxo + (int64_t)st * S.N + n)) * 3;
                        if (O.cb_in_smem)
                            for (int c = 0; c < 3; ++c) red_add_shared(s_cb + O.cb_off[4] + j + c, dmu[c] * la[c]);
                        else
                            for (int c = 0; c < 3; ++c) atomicAdd(O.d_off + j + c, dmu[c] * la[c]);
                    }
                } else {
                    for (int c = 0; c < 3; ++c) atomicAdd(O.d_off + n * 3 + c, dmu[c] * la[c]);
                }
            }
            if (O.d_l) {
                if (S.Ll > 0) {
                    for (int st = 0; st < S.Ll; ++st) {
                        const int j = (st * S.Kl + __ldg(S.idxl + (int64_t)st * S.n_anchors + a)) * 3;
                        if (O.cb_in_smem)
                            for (int c = 0; c < 3; ++c) red_add_shared(s_cb + O.cb_off[5] + j + c, dmu[c] * oo[c]);
                        else
                            for (int c = 0; c < 3; ++c) atomicAdd(O.d_l + j + c, dmu[c] * oo[c]);
                    }
                } else {
                    for (int c = 0; c < 3; ++c) atomicAdd(O.d_l + a * 3 + c, dmu[c] * oo[c]);
                }
            }
        } while (0);
        // pose sums: one butterfly per warp when its lanes share a view (the
        // slots are in view order, so they nearly always do)
        const uint32_t has = __ballot_sync(0xffffffffu, pv >= 0);
        if (has) {
            const int v0 = __shfl_sync(0xffffffffu, pv, __ffs(has) - 1);
            if (__all_sync(0xffffffffu, pv < 0 || pv == v0)) {
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    float x = pose[c];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                    if (lane == 0) red_add_shared(s_pose + v0 * 6 + c, x);
                }
            } else if (pv >= 0) {
#pragma unroll
                for (int c = 0; c < 6; ++c) red_add_shared(s_pose + pv * 6 + c, pose[c]);
            }
        }
    }
    grid_dependency_wait();  // (threads without a slot too, before any global write)
    __syncthreads();
    for (int i = threadIdx.x; i < V.n * 6; i += blockDim.x)
        if (s_pose[i] != 0.f) atomicAdd(O.pose_sum + i, s_pose[i]);
    if (O.cb_in_smem) {
        // every block adds its sums to the same rows: four floats per atomic
        // (vector atomic add, 16-byte aligned rows) quarter the operations
        // the L2 serialises on each address
        for (int gi = 0; gi < 6; ++gi) {
            const int sz = chain_cb_size(S, O, gi);
            float* dst = chain_cb_dst(O, gi);
            const float* src = s_cb + O.cb_off[gi];
            const bool vec = sz % 4 == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
            if (vec) {
                for (int j = 4 * (int)threadIdx.x; j < sz; j += 4 * (int)blockDim.x) {
                    const float4 t = make_float4(src[j], src[j + 1], src[j + 2], src[j + 3]);
                    if (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f)
                        atomicAdd(reinterpret_cast<float4*>(dst + j), t);
                }
            } else {
                for (int j = threadIdx.x; j < sz; j += blockDim.x) {
                    const float t = src[j];
                    if (t != 0.f) atomicAdd(dst + j, t);
                }
            }
        }
    }
}

int chain_blocks(int64_t) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

// before the backward: zero the gradient rows of the visible slots (the only
// rows the backward compositing writes; all other rows stay zero) and every
// scene-gradient array the chain kernel accumulates into
__global__ void zero_bwd_kernel(const uint32_t* __restrict__ vis, const uint32_t* __restrict__ nvis_dev,
                                uint32_t max_vis, float* __restrict__ g2d, ZeroList Z) {
    const uint32_t n = min(*nvis_dev, max_vis);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = tid; e < (int64_t)n * 3; e += nthr) {
        const uint32_t s = vis[e / 3];
        reinterpret_cast<float4*>(g2d + (int64_t)s * G2D_STRIDE)[e % 3] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int j = 0; j < Z.n; ++j) {
        float* p = Z.p[j];
        const int64_t cnt = Z.count[j];
        const bool vec = (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
        const int64_t n4 = vec ? cnt / 4 : 0;
        for (int64_t i = tid; i < n4; i += nthr) reinterpret_cast<float4*>(p)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t i = n4 * 4 + tid; i < cnt; i += nthr) p[i] = 0.f;
    }
}

cudaError_t launch_zero_bwd(const uint32_t* vis_slots, const uint32_t* nvis_dev, uint32_t max_vis, float* g2d,
                            const ZeroList& Z, cudaStream_t st) {
    int64_t work = (int64_t)max_vis * 3;
    for (int j = 0; j < Z.n; ++j) work = work > Z.count[j] / 4 ? work : Z.count[j] / 4;
    int64_t blocks = ceil_div(work > 0 ? work : 1, 256);
    if (blocks > 148 * 4) blocks = 148 * 4;
    count_launches(1);
    zero_bwd_kernel<<<(unsigned)blocks, 256, 0, st>>>(vis_slots, nvis_dev, max_vis, g2d, Z);
    return cudaGetLastError();
}

size_t chain_smem(const SceneDev& S, const Views& V, ChainOut* O) {
    int off = 0;
    for (int gi = 0; gi < 6; ++gi) {
        O->cb_off[gi] = off;
        off += chain_cb_size(S, *O, gi);
    }
    O->cb_total = off;
    const size_t pose_bytes = (size_t)V.n * 6 * sizeof(float);
    const size_t cb_bytes = (size_t)off * sizeof(float);
    // codebook accumulators in shared memory up to 96 KB, else global atomics
    O->cb_in_smem = (off > 0 && pose_bytes + cb_bytes <= 96 * 1024) ? 1 : 0;
    return pose_bytes + (O->cb_in_smem ? cb_bytes : 0);
}

cudaError_t launch_chain(const SceneDev& S, const Views& V, const Consts& cs, const float* g2d, const uint32_t* vis,
                         const uint32_t* nvis_dev, uint32_t max_vis, ChainOut O, int* n_blocks_out, cudaStream_t st) {
    const int blocks = chain_blocks(S.N);
    if (n_blocks_out) *n_blocks_out = blocks;
    const size_t smem = chain_smem(S, V, &O);
    cudaError_t e = allow_dynamic_smem((const void*)chain_kernel, smem);
    if (e != cudaSuccess) return e;
    // overlapped with the backward compositing in front of it (same call):
    // the chain's CTAs start their scene-only prefix as that kernel's last
    // CTAs run
    return launch_overlapped(chain_kernel, dim3((unsigned)blocks), dim3(CHAIN_THREADS), smem, st, S, V, cs, g2d, vis,
                             nvis_dev, max_vis, O);
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

// dxi = the chain's pose sums (+ the ICP term's block partials, if any)
__global__ void pose_final_kernel(const float* __restrict__ pose_sum, const float* __restrict__ icp_part, int nbi,
                                  float* __restrict__ dxi, float* __restrict__ icp_loss) {
    grid_dependency_wait();  // (overlapped launch: nothing is read before the kernel in front completes)
    __shared__ float s_tmp[8];
    const int v = blockIdx.x;
    if (!icp_part) {
        if (threadIdx.x < 6) dxi[v * 6 + threadIdx.x] = pose_sum[v * 6 + threadIdx.x];
        return;
    }
    for (int c = 0; c < 7; ++c) {
        float acc = 0.f;
        for (int j = threadIdx.x; j < nbi; j += blockDim.x) acc += icp_part[((int64_t)v * nbi + j) * 7 + c];
        const float t = block_sum_256(acc, s_tmp);
        if (threadIdx.x == 0) {
            if (c < 6) dxi[v * 6 + c] = pose_sum[v * 6 + c] + t;
            else if (icp_loss) icp_loss[v] = t;
        }
    }
}

cudaError_t launch_pose_final(int n_views, const float* pose_sum, const float* icp_part, int nbi, float* dxi,
                              float* icp_loss, cudaStream_t st) {
    // overlapped: resident as the chain (or ICP) kernel in front runs, it
    // waits on the device instead of being launched after it
    return launch_overlapped(pose_final_kernel, dim3((unsigned)n_views), dim3(icp_part ? 256 : 32), 0, st, pose_sum,
                             icp_part, nbi, dxi, icp_loss);
}

// ---------------------------------------------------------------------------
// L1 colour + weighted L1 depth (valid where the target depth > 0)
// ---------------------------------------------------------------------------
// count[0] += sampled pixels with Dt > 0; with a mask also count[1] += sampled
// pixels; zeroes the loss value the loss kernel then accumulates into
__global__ void count_valid_kernel(const float* __restrict__ Dt, const uint8_t* __restrict__ mask, int64_t n,
                                   uint32_t* count, float* loss) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *loss = 0.f;
    uint32_t c = 0, ns = 0;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
    const bool vec = (reinterpret_cast<uintptr_t>(Dt) & 15u) == 0 && (reinterpret_cast<uintptr_t>(mask) & 3u) == 0;
    const int64_t n4 = vec ? n / 4 : 0;
    for (int64_t i = tid; i < n4; i += nthr) {
        const float4 d = reinterpret_cast<const float4*>(Dt)[i];
        if (mask) {
            const uchar4 m = reinterpret_cast<const uchar4*>(mask)[i];
            c += (m.x && d.x > 0.f) + (m.y && d.y > 0.f) + (m.z && d.z > 0.f) + (m.w && d.w > 0.f);
            ns += (m.x != 0) + (m.y != 0) + (m.z != 0) + (m.w != 0);
        } else {
            c += (d.x > 0.f) + (d.y > 0.f) + (d.z > 0.f) + (d.w > 0.f);
        }
    }
    for (int64_t i = n4 * 4 + tid; i < n; i += nthr) {
        const bool m = mask ? mask[i] != 0 : true;
        c += m && Dt[i] > 0.f;
        ns += m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        ns += __shfl_xor_sync(0xffffffffu, ns, o);
    }
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
    if ((threadIdx.x & 31) == 0 && mask && ns) atomicAdd(count + 1, ns);
}

__global__ void loss_l1_kernel(int64_t n_pix, int64_t total, const float* __restrict__ C, const float* __restrict__ D,
                               const float* __restrict__ S, const float* __restrict__ Ct, const float* __restrict__ Dt,
                               const uint8_t* __restrict__ mask, float w_depth, float gate,
                               uint32_t* valid_count, float* __restrict__ dC,
                               float* __restrict__ dD, float* __restrict__ loss, int vec) {
    __shared__ float s_tmp[8];
    const float nv = (float)valid_count[0];
    const float nsamp = mask ? (float)valid_count[1] : (float)total;
    const float inv_c = nsamp > 0.f ? 1.f / (3.f * nsamp) : 0.f;
    const float inv_d = nv > 0.f ? w_depth / nv : 0.f;
    float acc = 0.f;
    const int64_t v = blockIdx.y;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
    const float* c0p = C + (v * 3 + 0) * n_pix;
    const float* c1p = C + (v * 3 + 1) * n_pix;
    const float* c2p = C + (v * 3 + 2) * n_pix;
    const float* t0p = Ct + (v * 3 + 0) * n_pix;
    const float* t1p = Ct + (v * 3 + 1) * n_pix;
    const float* t2p = Ct + (v * 3 + 2) * n_pix;
    const float* dp = D + v * n_pix;
    const float* dtp = Dt + v * n_pix;
    const float* sp = S + v * n_pix;
    float* g0p = dC + (v * 3 + 0) * n_pix;
    float* g1p = dC + (v * 3 + 1) * n_pix;
    float* g2p = dC + (v * 3 + 2) * n_pix;
    float* gdp = dD + v * n_pix;
    const uint8_t* mp = mask ? mask + v * n_pix : nullptr;
    const int64_t n4 = vec ? n_pix / 4 : 0;  // four pixels per step where every plane is 16-byte aligned
    for (int64_t i = tid; i < n4; i += nthr) {
        const float4 c0 = reinterpret_cast<const float4*>(c0p)[i], c1 = reinterpret_cast<const float4*>(c1p)[i],
                     c2 = reinterpret_cast<const float4*>(c2p)[i];
        const float4 t0 = reinterpret_cast<const float4*>(t0p)[i], t1 = reinterpret_cast<const float4*>(t1p)[i],
                     t2 = reinterpret_cast<const float4*>(t2p)[i];
        const float4 d = reinterpret_cast<const float4*>(dp)[i], dt = reinterpret_cast<const float4*>(dtp)[i];
        float4 s = make_float4(1.f, 1.f, 1.f, 1.f);
        if (gate >= 0.f) s = reinterpret_cast<const float4*>(sp)[i];
        uchar4 ms = make_uchar4(1, 1, 1, 1);
        if (mp) ms = reinterpret_cast<const uchar4*>(mp)[i];
        float4 g0, g1, g2, gd;
        acc += loss_pixel(c0.x, c1.x, c2.x, t0.x, t1.x, t2.x, d.x, dt.x, s.x, gate, inv_c, inv_d, g0.x, g1.x, g2.x, gd.x,
                          ms.x != 0);
        acc += loss_pixel(c0.y, c1.y, c2.y, t0.y, t1.y, t2.y, d.y, dt.y, s.y, gate, inv_c, inv_d, g0.y, g1.y, g2.y, gd.y,
                          ms.y != 0);
        acc += loss_pixel(c0.z, c1.z, c2.z, t0.z, t1.z, t2.z, d.z, dt.z, s.z, gate, inv_c, inv_d, g0.z, g1.z, g2.z, gd.z,
                          ms.z != 0);
        acc += loss_pixel(c0.w, c1.w, c2.w, t0.w, t1.w, t2.w, d.w, dt.w, s.w, gate, inv_c, inv_d, g0.w, g1.w, g2.w, gd.w,
                          ms.w != 0);
        reinterpret_cast<float4*>(g0p)[i] = g0;
        reinterpret_cast<float4*>(g1p)[i] = g1;
        reinterpret_cast<float4*>(g2p)[i] = g2;
        reinterpret_cast<float4*>(gdp)[i] = gd;
    }
    for (int64_t i = n4 * 4 + tid; i < n_pix; i += nthr) {
        float g0, g1, g2, gd;
        acc += loss_pixel(c0p[i], c1p[i], c2p[i], t0p[i], t1p[i], t2p[i], dp[i], dtp[i], gate >= 0.f ? sp[i] : 1.f, gate,
                          inv_c, inv_d, g0, g1, g2, gd, mp ? mp[i] != 0 : true);
        g0p[i] = g0;
        g1p[i] = g1;
        g2p[i] = g2;
        gdp[i] = gd;
    }
    const float t = block_sum_256(acc, s_tmp);
    if (threadIdx.x == 0) {
        atomicAdd(loss, t);
        // the last block to finish clears the counters for the next call
        // (every block has read them by then), so no memset precedes a call
        __threadfence();
        if (atomicAdd(valid_count + 2, 1u) == gridDim.x * gridDim.y - 1) {
            valid_count[0] = 0u;
            valid_count[1] = 0u;
            valid_count[2] = 0u;
        }
    }
}

// The same loss in one cooperative launch (every block resident): the blocks
// count the valid target depths and sampled pixels, meet at a grid-wide
// barrier (bounded: a spin that runs out flags ERR_WAIT), then write the
// gradient images and sum the loss.  ctl: [0] valid depths, [1] sampled
// pixels, [2] blocks arrived, [3] blocks done; the last block done clears
// all four for the next call.  Four pixels per step (16-byte aligned planes).
__global__ void __launch_bounds__(256) loss_l1_coop_kernel(
    int64_t n_pix, int n_views, const float* __restrict__ C, const float* __restrict__ D, const float* __restrict__ S,
    const float* __restrict__ Ct, const float* __restrict__ Dt, const uint8_t* __restrict__ mask, float w_depth,
    float gate, uint32_t* ctl, float* __restrict__ dC, float* __restrict__ dD, float* __restrict__ loss, uint32_t* err,
    uint32_t spin_limit) {
    __shared__ float s_tmp[8];
    __shared__ uint32_t s_cnt[2];
    const uint32_t q_view = (uint32_t)(n_pix / 4), n_q = q_view * (uint32_t)n_views;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    // phase 1: counts over every view's target depth (and ray mask)
    uint32_t c = 0, ns = 0;
    for (uint32_t q = tid; q < n_q; q += nthr) {
        const float4 d = reinterpret_cast<const float4*>(Dt)[q];
        if (mask) {
            const uchar4 m = reinterpret_cast<const uchar4*>(mask)[q];
            c += (m.x && d.x > 0.f) + (m.y && d.y > 0.f) + (m.z && d.z > 0.f) + (m.w && d.w > 0.f);
            ns += (m.x != 0) + (m.y != 0) + (m.z != 0) + (m.w != 0);
        } else {
            c += (d.x > 0.f) + (d.y > 0.f) + (d.z > 0.f) + (d.w > 0.f);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        ns += __shfl_xor_sync(0xffffffffu, ns, o);
    }
    if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        if (c) atomicAdd(&s_cnt[0], c);
        if (ns) atomicAdd(&s_cnt[1], ns);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_cnt[0]) atomicAdd(ctl + 0, s_cnt[0]);
        if (mask && s_cnt[1]) atomicAdd(ctl + 1, s_cnt[1]);
        if (blockIdx.x == 0) *loss = 0.f;
        __threadfence();
        atomicAdd(ctl + 2, 1u);
        const volatile uint32_t* arrived = ctl + 2;
        uint32_t polls = 0;
        while (*arrived < gridDim.x) {
            if (++polls > spin_limit) {  // gives up: the counts may be partial, the call's results wrong
                atomicOr(err, ERR_WAIT);
                break;
            }
        }
        __threadfence();
        s_cnt[0] = *(const volatile uint32_t*)(ctl + 0);
        s_cnt[1] = *(const volatile uint32_t*)(ctl + 1);
    }
    __syncthreads();
    // phase 2: gradient images and the loss
    const float nv = (float)s_cnt[0];
    const float nsamp = mask ? (float)s_cnt[1] : (float)((int64_t)n_views * n_pix);
    const float inv_c = nsamp > 0.f ? 1.f / (3.f * nsamp) : 0.f;
    const float inv_d = nv > 0.f ? w_depth / nv : 0.f;
    float acc = 0.f;
    for (uint32_t q = tid; q < n_q; q += nthr) {
        const uint32_t v = q / q_view, i = q - v * q_view;
        const float4* c4 = reinterpret_cast<const float4*>(C) + (int64_t)v * 3 * q_view;
        const float4* t4 = reinterpret_cast<const float4*>(Ct) + (int64_t)v * 3 * q_view;
        const float4 c0 = c4[i], c1 = c4[q_view + i], c2 = c4[2 * q_view + i];
        const float4 t0 = t4[i], t1 = t4[q_view + i], t2 = t4[2 * q_view + i];
        const float4 d = reinterpret_cast<const float4*>(D)[q], dt = reinterpret_cast<const float4*>(Dt)[q];
        float4 sv = make_float4(1.f, 1.f, 1.f, 1.f);
        if (gate >= 0.f) sv = reinterpret_cast<const float4*>(S)[q];
        uchar4 ms = make_uchar4(1, 1, 1, 1);
        if (mask) ms = reinterpret_cast<const uchar4*>(mask)[q];
        float4 g0, g1, g2, gd;
        acc += loss_pixel(c0.x, c1.x, c2.x, t0.x, t1.x, t2.x, d.x, dt.x, sv.x, gate, inv_c, inv_d, g0.x, g1.x, g2.x,
                          gd.x, ms.x != 0);
        acc += loss_pixel(c0.y, c1.y, c2.y, t0.y, t1.y, t2.y, d.y, dt.y, sv.y, gate, inv_c, inv_d, g0.y, g1.y, g2.y,
                          gd.y, ms.y != 0);
        acc += loss_pixel(c0.z, c1.z, c2.z, t0.z, t1.z, t2.z, d.z, dt.z, sv.z, gate, inv_c, inv_d, g0.z, g1.z, g2.z,
                          gd.z, ms.z != 0);
        acc += loss_pixel(c0.w, c1.w, c2.w, t0.w, t1.w, t2.w, d.w, dt.w, sv.w, gate, inv_c, inv_d, g0.w, g1.w, g2.w,
                          gd.w, ms.w != 0);
        float4* gc4 = reinterpret_cast<float4*>(dC) + (int64_t)v * 3 * q_view;
        gc4[i] = g0;
        gc4[q_view + i] = g1;
        gc4[2 * q_view + i] = g2;
        reinterpret_cast<float4*>(dD)[q] = gd;
    }
    const float t = block_sum_256(acc, s_tmp);
    if (threadIdx.x == 0) {
        atomicAdd(loss, t);
        __threadfence();
        if (atomicAdd(ctl + 3, 1u) == gridDim.x - 1) {
            ctl[0] = 0u;
            ctl[1] = 0u;
            ctl[2] = 0u;
            ctl[3] = 0u;
        }
    }
}

cudaError_t launch_loss_l1(int n_views, int64_t n_pix, const float* C, const float* D, const float* S, const float* Ct,
                           const float* Dt, const uint8_t* mask, float w_depth, float gate, float* dC, float* dD,
                           float* loss, uint32_t* valid_count, uint32_t* err, uint32_t spin_limit, cudaStream_t st) {
    const int64_t total = (int64_t)n_views * n_pix;
    int64_t blocks = ceil_div(ceil_div(total > 0 ? total : 1, 4), 256);
    if (blocks > 148 * 8) blocks = 148 * 8;
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const int vec = (n_pix % 4 == 0) && al(C) && al(D) && al(Ct) && al(Dt) && al(dC) && al(dD) &&
                    (gate < 0.f || al(S)) && (reinterpret_cast<uintptr_t>(mask) & 3u) == 0;
    // one cooperative launch where the device takes them and the planes allow
    // four pixels per step; otherwise a counting kernel, then the loss kernel
    // the co-resident grid, per device (queried once per device, under a lock)
    static std::mutex mu;
    static int coop_of[64];
    static bool known_of[64];
    int dev = 0;
    cudaGetDevice(&dev);
    int coop_blocks = 0;
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lock(mu);
        if (!known_of[dev]) {
            int coop = 0, sms = 0, per = 0;
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, loss_l1_coop_kernel, 256, 0);
            coop_of[dev] = coop ? sms * per : 0;
            known_of[dev] = true;
            cudaGetLastError();
        }
        coop_blocks = coop_of[dev];
    }
    if (vec && coop_blocks > 0 && total / 4 < (int64_t)UINT32_MAX && err) {
        int64_t g = ceil_div(total / 4, 256);
        if (g > coop_blocks) g = coop_blocks;
        if (g < 1) g = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)g);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, loss_l1_coop_kernel, n_pix, n_views, C, D, S, Ct, Dt, mask,
                                                 w_depth, gate, valid_count, dC, dD, loss, err, spin_limit);
        if (e == cudaSuccess) {
            count_launches(1);
            return e;
        }
        // fewer SMs than the occupancy query saw (a shared or partitioned
        // device): the two-launch form below needs no co-residency
        if (e != cudaErrorCooperativeLaunchTooLarge) return e;
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lock(mu);
            coop_of[dev] = 0;
        }
    }
    count_launches(2);
    count_valid_kernel<<<(unsigned)blocks, 256, 0, st>>>(Dt, mask, total, valid_count, loss);
    int64_t bx = ceil_div(vec ? ceil_div(n_pix, 4) : n_pix, 256);
    if (bx > 148 * 8) bx = 148 * 8;
    loss_l1_kernel<<<dim3((unsigned)bx, (unsigned)n_views), 256, 0, st>>>(n_pix, total, C, D, S, Ct, Dt, mask, w_depth,
                                                                          gate, valid_count, dC, dD, loss, vec);
    return cudaGetLastError();
}

__global__ void sample_rays_kernel(uint8_t* __restrict__ mask, int64_t n, unsigned long long seed,
                                   const int32_t* __restrict__ round_dev, int32_t round_host,
                                   unsigned long long keep_below) {
    const unsigned long long r = (unsigned long long)(uint32_t)(round_dev ? round_dev[0] : round_host);
    const unsigned long long key = seed + r * GOLDEN_GAMMA;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        mask[p] = (splitmix64(key ^ (unsigned long long)p) >> 11) < keep_below ? 1 : 0;
}

cudaError_t launch_sample_rays(uint8_t* mask, int64_t n, unsigned long long seed, const int32_t* round_dev,
                               int32_t round_host, unsigned long long keep_below, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = ceil_div(n, 256);
    if (blocks > 148 * 8) blocks = 148 * 8;
    count_launches(1);
    sample_rays_kernel<<<(unsigned)blocks, 256, 0, st>>>(mask, n, seed, round_dev, round_host, keep_below);
    return cudaGetLastError();
}

}  // namespace vgk
