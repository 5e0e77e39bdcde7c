// vg_preprocess.cu -- fused decode + mask + projection of every (view, Gaussian)
// slot, and the standalone residual-codebook decode.
//
// Decode follows Eq. 7 (mu = x_a + O_i * l), Eq. 14 first line (attribute =
// sum over stages of the indexed codewords) and Eq. 11-12 (a Gaussian whose
// mask is off is removed).  Projection follows Eq. 2 (Sigma = R S S^T R^T)
// and Eq. 3 (Sigma' = J W Sigma W^T J^T, plus a low-pass dilation).
#include "vg_internal.h"

namespace vgk {

// One thread per Gaussian of a 256-Gaussian block in the first phase: the
// anchor mean (Eq. 7), the mask, the near plane and a conservative reach test
// (below) decide whether the Gaussian can touch a tile of any view; every
// slot of a Gaussian that cannot is written culled at once.  The candidates
// of the block are then compacted (in Gaussian order) and decoded and
// projected by consecutive threads, so the warps that run the decode and the
// projection are dense: with about a tenth of a scene in view, almost every
// warp has a candidate lane, and without the compaction almost every warp
// would run the whole path.
constexpr int PRE_THREADS = 256;
constexpr int LS_STAGES = 8;  // stages the log-scale bound covers

__global__ void __launch_bounds__(PRE_THREADS, 5) preprocess_kernel(
    SceneDev S, const __grid_constant__ Views V, Consts cs, float4* __restrict__ xy, float4* __restrict__ conic_o,
    float4* __restrict__ rgbd, uint2* __restrict__ rect, uint32_t* __restrict__ ntiles, uint32_t* __restrict__ dkey,
    uint32_t* __restrict__ scratch, uint32_t* state, uint32_t* __restrict__ blk_count) {
    __shared__ uint32_t s_hist[4 * 256];
    __shared__ uint32_t s_cnt[2];
    __shared__ uint32_t s_wn[PRE_THREADS / 32];
    __shared__ uint32_t s_list[PRE_THREADS];  // the block's candidates (Gaussian offsets in the block)
    __shared__ float s_mu[PRE_THREADS * 3];   // and their means
    allow_dependents();  // the compaction's loss normalisers may overlap this kernel's last CTAs
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (cs.depth_hist)
        for (int i = tid; i < 4 * 256; i += PRE_THREADS) s_hist[i] = 0;
    if (tid < 2) s_cnt[tid] = 0;
    if (blockIdx.x == 0 && tid == 0) state[ST_EPOCH] += 16u;  // fresh lookback epochs for this forward
    // the fused L1 loss's value (summed by the compositing) starts from zero
    if (cs.lf_on && blockIdx.x == 0 && tid == 0) *cs.lf_loss = 0.f;
    // A decoded log-scale component is a sum over stages of one codeword
    // entry each, so it is at most the sum of each stage's largest entry:
    // with that scale bound, a Gaussian whose 3-sigma box cannot reach any
    // tile of any view is culled before its attributes are decoded.  The box
    // bound uses |J|_F >= |J|_2, a 1% and 2-pixel margin covers FP32
    // rounding, so no Gaussian the full test keeps is lost.  Every warp
    // computes the bound itself (its loads go out with the lanes' own), so
    // that no warp waits for another before its reach test.
    const bool ls_bound = S.L[0] > 0 && S.L[0] <= LS_STAGES;
    float lsb = 0.f;
    if (ls_bound) {
        const int per = S.K[0] * 3;
        float mx[LS_STAGES];
#pragma unroll
        for (int st = 0; st < LS_STAGES; ++st) {
            mx[st] = -INFINITY;
            if (st < S.L[0])
#pragma unroll 2
                for (int i = lane; i < per; i += 32) mx[st] = fmaxf(mx[st], __ldg(S.cb[0] + st * per + i));
        }
#pragma unroll
        for (int st = 0; st < LS_STAGES; ++st)
            if (st < S.L[0]) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx[st] = fmaxf(mx[st], __shfl_xor_sync(0xffffffffu, mx[st], o));
                lsb += mx[st];
            }
    }

    const int64_t n = (int64_t)blockIdx.x * PRE_THREADS + tid;
    const bool live = n < S.N;
    float mu[3] = {0, 0, 0};
    bool cand = false;
    if (live) {
        anchor_mean(S, n, mu);
        const bool on = S.mask ? (__ldg(S.mask + n) > S.mask_thr) : true;
        // a candidate lies in front of the near plane of some view and (with
        // the scale bound) its widest possible 3-sigma box reaches a tile of
        // that view
        const float smax = ls_bound ? expf(lsb) * 1.001f : 0.f;
        for (int v = 0; v < V.n && on && !cand; ++v) {
            const ViewInfo& vi = V.v[v];
            float T[12], pc[3];
            view_pose(V, v, T);
            cam_point(T, mu, pc);
            if (!(pc[2] > vi.near_plane)) continue;
            if (!ls_bound) {
                cand = true;
                break;
            }
            // (hardware reciprocal and reciprocal square root: a few ulp,
            // far inside the margins)
            const float iz = __fdividef(1.f, pc[2]);
            float tx = pc[0] * iz, ty = pc[1] * iz;
            const float u = vi.fx * tx + vi.cx, vv = vi.fy * ty + vi.cy;
            if (cs.jacobian_clamp) {
                tx = fminf(fmaxf(tx, -vi.limx), vi.limx);
                ty = fminf(fmaxf(ty, -vi.limy), vi.limy);
            }
            const float fz = vi.fx * iz, gz = vi.fy * iz;
            const float jf2 = fz * fz * (1.f + tx * tx) + gz * gz * (1.f + ty * ty);
            const float r2 = fmaxf(jf2 * smax * smax + cs.dilation, 1e-30f);
            const float r = cs.sigma_cull * (r2 * rsqrtf(r2)) * 1.01f + 2.f;
            cand = u + r >= 0.f && u - r < (float)(vi.tiles_x * TILE) && vv + r >= 0.f &&
                   vv - r < (float)(vi.tiles_y * TILE);
        }
    }
    if (live && !cand)
        for (int v = 0; v < V.n; ++v) {
            const int64_t slot = (int64_t)v * S.N + n;
            ntiles[slot] = 0u;
            dkey[slot] = 0xffffffffu;  // culled slots sort last
        }
    // compaction of the candidates, in Gaussian order
    const uint32_t bal = __ballot_sync(0xffffffffu, cand);
    if (lane == 0) s_wn[warp] = (uint32_t)__popc(bal);
    __syncthreads();
    uint32_t pos = (uint32_t)__popc(bal & lanemask_lt()), n_cand = 0;
#pragma unroll
    for (int w = 0; w < PRE_THREADS / 32; ++w) {
        const uint32_t c = s_wn[w];
        pos += w < warp ? c : 0u;
        n_cand += c;
    }
    if (cand) {
        s_list[pos] = (uint32_t)tid;
        s_mu[3 * pos] = mu[0];
        s_mu[3 * pos + 1] = mu[1];
        s_mu[3 * pos + 2] = mu[2];
    }
    __syncthreads();

    uint32_t n_vis = 0, n_pair = 0;
    // (a uniform loop: every lane of a warp takes part in its warp votes)
    for (uint32_t j0 = 0; j0 < n_cand; j0 += PRE_THREADS) {
        const uint32_t j = j0 + (uint32_t)tid;
        const bool valid = j < n_cand;
        const int64_t g = valid ? (int64_t)blockIdx.x * PRE_THREADS + s_list[j] : 0;
        float gm[3] = {0, 0, 0}, ls[3] = {0, 0, 0}, q[4] = {1, 0, 0, 0}, ol = 0.f, rgb[3] = {0, 0, 0};
        float RS[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // R diag(s): Sigma = RS RS^T
        float opac = 0.f;
        bool active = valid;
        if (valid) {
            gm[0] = s_mu[3 * j];
            gm[1] = s_mu[3 * j + 1];
            gm[2] = s_mu[3 * j + 2];
            decode_attr<3>(S, 0, g, ls);
            decode_attr<4>(S, 1, g, q);
            decode_attr<1>(S, 2, g, &ol);
            decode_attr<3>(S, 3, g, rgb);
            const float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
            active = qq > 0.f;
            if (active) {
                const float qn_inv = 1.f / sqrtf(qq);
                const float qn[4] = {q[0] * qn_inv, q[1] * qn_inv, q[2] * qn_inv, q[3] * qn_inv};
                float R[3][3];
                quat_rot(qn, R);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float sc = expf(ls[c]);
#pragma unroll
                    for (int r = 0; r < 3; ++r) RS[r][c] = R[r][c] * sc;
                }
                opac = 1.f / (1.f + expf(-ol));
            }
        }
        for (int v = 0; v < V.n; ++v) {
            uint32_t key = 0xffffffffu;
            if (valid) {
                const int64_t slot = (int64_t)v * S.N + g;
                const ViewInfo& vi = V.v[v];
                bool ok = active;
                float p[3] = {0, 0, 1};
                float u = 0, vv = 0;
                uint32_t cnt = 0;
                int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
                float a = 0, b = 0, c = 0, ex = -1.f, ey = -1.f;
                if (ok) {
                    float T[12];
                    view_pose(V, v, T);
                    cam_point(T, gm, p);
                    const float z = p[2];
                    ok = z > vi.near_plane;
                    if (ok) {
                        u = __fadd_rn(__fdiv_rn(__fmul_rn(vi.fx, p[0]), z), vi.cx);
                        vv = __fadd_rn(__fdiv_rn(__fmul_rn(vi.fy, p[1]), z), vi.cy);
                        float txz = p[0] / z, tyz = p[1] / z;
                        if (cs.jacobian_clamp) {
                            txz = fminf(fmaxf(txz, -vi.limx), vi.limx);
                            tyz = fminf(fmaxf(tyz, -vi.limy), vi.limy);
                        }
                        const float J00 = vi.fx / z, J02 = -vi.fx * txz / z;
                        const float J11 = vi.fy / z, J12 = -vi.fy * tyz / z;
                        float A, B, C, det;
                        cov2d(J00, J02, J11, J12, T, RS, cs.dilation, A, B, C, det);
                        ok = det > 0.f;
                        if (ok) {
                            const float inv = 1.f / det;
                            a = C * inv;
                            b = -B * inv;
                            c = A * inv;
                            // half extents of the box holding every pixel with
                            // o exp(-q/2) >= alpha_min, q = d^T conic d: the
                            // ellipse q <= tau, tau = 2 ln(o / alpha_min), has
                            // half extents sqrt(tau A), sqrt(tau C); widened so
                            // that FP32 rounding of a pixel's own test can never
                            // fall outside
                            if (opac > cs.alpha_min) {
                                const float tau = 2.f * logf(opac / cs.alpha_min) * 1.001f + 1e-3f;
                                ex = sqrtf(tau * A) * 1.0001f + 1e-3f;
                                ey = sqrtf(tau * C) * 1.0001f + 1e-3f;
                            }
                            // largest eigenvalue; mid^2 - det written as a sum of squares
                            const float mid = 0.5f * (A + C), hd = 0.5f * (A - C);
                            const float lam = mid + sqrtf(hd * hd + B * B);
                            const float rr = cs.sigma_cull * sqrtf(lam);
                            const int radius = (rr < (float)RADIUS_MAX) ? (int)ceilf(rr) : RADIUS_MAX;
                            const float rf = (float)radius;
                            const float fx0 = floorf(__fdiv_rn(__fsub_rn(u, rf), (float)TILE));
                            const float fx1 = floorf(__fdiv_rn(__fadd_rn(u, rf), (float)TILE)) + 1.f;
                            const float fy0 = floorf(__fdiv_rn(__fsub_rn(vv, rf), (float)TILE));
                            const float fy1 = floorf(__fdiv_rn(__fadd_rn(vv, rf), (float)TILE)) + 1.f;
                            x0 = (int)fminf(fmaxf(fx0, 0.f), (float)vi.tiles_x);
                            x1 = (int)fminf(fmaxf(fx1, 0.f), (float)vi.tiles_x);
                            y0 = (int)fminf(fmaxf(fy0, 0.f), (float)vi.tiles_y);
                            y1 = (int)fminf(fmaxf(fy1, 0.f), (float)vi.tiles_y);
                            ok = (x1 > x0) && (y1 > y0);
                            cnt = ok ? (uint32_t)((x1 - x0) * (y1 - y0)) : 0u;
                        }
                    }
                }
                if (ok) {
                    xy[slot] = make_float4(u, vv, ex, ey);
                    // base-2 exponent coefficients and the opacity threshold
                    const float thr = opac > 0.f ? log2f(cs.alpha_min / opac) : 3.0e38f;
                    conic_o[slot] = make_float4(-0.5f * LOG2E * a, -LOG2E * b, -0.5f * LOG2E * c, thr);
                    rgbd[slot] = make_float4(rgb[0], rgb[1], rgb[2], p[2]);
                    rect[slot] = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
                    ntiles[slot] = cnt;
                    key = __float_as_uint(p[2]);
                    dkey[slot] = key;
                    ++n_vis;
                    n_pair += cnt;
                    if (cs.seen) cs.seen[g] = 1u;
                } else {
                    ntiles[slot] = 0u;
                    dkey[slot] = 0xffffffffu;
                }
            }
            // depth-key digit histograms of the visible slots; most lanes share
            // the high digits
            if (cs.depth_hist) {
                const uint32_t vis_mask = __ballot_sync(0xffffffffu, key != 0xffffffffu);
                if (key != 0xffffffffu) {
#pragma unroll
                    for (int pass = 0; pass < 4; ++pass) {
                        const uint32_t bk = (key >> (8 * pass)) & 255u;
                        const uint32_t peers = __match_any_sync(vis_mask, bk);
                        if (lane == __ffs(peers) - 1) red_add_shared(&s_hist[pass * 256 + bk], (uint32_t)__popc(peers));
                    }
                }
            }
        }
    }
    if (n_vis) red_add_shared(&s_cnt[0], n_vis);
    if (n_pair) red_add_shared(&s_cnt[1], n_pair);
    __syncthreads();
    if (cs.depth_hist)
        for (int i = tid; i < 4 * 256; i += PRE_THREADS) {
            const uint32_t h = s_hist[i];
            if (h) atomicAdd(scratch + SCR_DEPTH_HIST + i, h);
        }
    if (tid == 0) {
        blk_count[blockIdx.x] = s_cnt[0];
        blk_count[gridDim.x + blockIdx.x] = s_cnt[1];  // the block's (slot, tile) pairs
    }
}

// order-preserving compaction of the visible slots: block b of the preprocess
// grid covers Gaussians [256 b, 256 b + 256) of every view; its visible slots
// go, view by view and in Gaussian order, to [base, base + count[b]), where
// base = count[0] + ... + count[b - 1] is summed by the block itself from the
// preprocess's per-block counts (at most a few thousand words, read from L2:
// cheaper than a separate scan launch).  vals_copy (may be NULL) keeps that
// slot order for the backward's per-slot passes (the depth sort overwrites
// vals_out).  With pair_off (the forms that keep this order for the pairs),
// the slot at position j also gets its first pair, pair_off[j] (exclusive
// scan of the tile counts in this order, from the per-block pair counts that
// follow the slot counts), and marks the 256-pair chunks that start inside
// its pairs; the last block writes the pair count (flagged when above cap)
// and the sentinel pair_off[visible slots].  The last block also writes the
// number of visible slots (scratch[SCR_NVIS]): a plain store, so that word
// needs no zeroing between forwards.
__global__ void __launch_bounds__(256) compact_kernel(const __grid_constant__ Views V, int64_t N,
                                                      const uint32_t* __restrict__ dkey,
                                                      const uint32_t* __restrict__ cnt, uint32_t* __restrict__ keys_out,
                                                      uint32_t* __restrict__ vals_out, uint32_t* __restrict__ vals_copy,
                                                      const uint32_t* __restrict__ ntiles, uint32_t* __restrict__ pair_off,
                                                      uint32_t* __restrict__ chunk_start, uint32_t cap,
                                                      uint32_t* __restrict__ scratch, uint32_t* __restrict__ err,
                                                      float* __restrict__ g2d_rows, float* __restrict__ pose_zero,
                                                      int n_pose, int nb, const Consts cs) {
    __shared__ uint32_t s_tmp[8];
    // (overlapped launch: the loss normalisers read only the caller's target
    // depths and pixel mask, so they are counted while the preprocess
    // drains; everything after the wait reads the preprocess's outputs)
    if (cs.lf_on) {
        // the fused L1 loss's normalisers, counted before any pixel is
        // composited: valid target depths and sampled pixels, per block
        // (plain stores; the ranges kernel sums them).  The grid covers at
        // most 4,096 pixels a block; blocks past the compaction's own only
        // count.
        uint32_t c = 0, ns = 0, ct, nst;
        const int64_t tid = (int64_t)blockIdx.x * 256 + threadIdx.x, nthr = (int64_t)gridDim.x * 256;
        // four pixels a load where the depth plane (and the mask) allow it
        const bool vec = (reinterpret_cast<uintptr_t>(cs.lf_Dt) & 15u) == 0 &&
                         (reinterpret_cast<uintptr_t>(cs.pix_mask) & 3u) == 0;
        const int64_t n4 = vec ? cs.lf_pixels / 4 : 0;
        for (int64_t i = tid; i < n4; i += nthr) {
            const float4 d = __ldg(reinterpret_cast<const float4*>(cs.lf_Dt) + i);
            if (cs.pix_mask) {
                const uchar4 m = reinterpret_cast<const uchar4*>(cs.pix_mask)[i];
                c += (m.x && d.x > 0.f) + (m.y && d.y > 0.f) + (m.z && d.z > 0.f) + (m.w && d.w > 0.f);
                ns += (m.x != 0) + (m.y != 0) + (m.z != 0) + (m.w != 0);
            } else {
                c += (d.x > 0.f) + (d.y > 0.f) + (d.z > 0.f) + (d.w > 0.f);
                ns += 4;
            }
        }
        for (int64_t i = n4 * 4 + tid; i < cs.lf_pixels; i += nthr) {
            const bool smp = cs.pix_mask ? cs.pix_mask[i] != 0 : true;
            c += smp && __ldg(cs.lf_Dt + i) > 0.f;
            ns += smp;
        }
        block_excl_scan_256(c, s_tmp, &ct);
        block_excl_scan_256(ns, s_tmp, &nst);
        if (threadIdx.x == 0) {
            cs.lf_blk[blockIdx.x] = ct;
            cs.lf_blk[gridDim.x + blockIdx.x] = nst;
        }
    }
    grid_dependency_wait();
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < n_pose; i += 256) pose_zero[i] = 0.f;
    if ((int)blockIdx.x >= nb) return;
    const int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int b = (int)blockIdx.x;
    // this block's offsets: the sums of the counts of the blocks in front of
    // it (nb^2 / 2 words over the grid, from L2; on the 3M-Gaussian scene's
    // 11,719 blocks still faster than a separate one-block scan launch)
    uint32_t off, poff = 0;
    {
        uint32_t a = 0, p = 0;
#pragma unroll 4
        for (int j = threadIdx.x; j < b; j += 256) {
            a += cnt[j];
            if (pair_off) p += cnt[nb + j];
        }
        block_excl_scan_256(a, s_tmp, &off);
        if (pair_off) block_excl_scan_256(p, s_tmp, &poff);
    }
    for (int v = 0; v < V.n; ++v) {
        const int64_t slot = (int64_t)v * N + n;
        const uint32_t key = n < N ? dkey[slot] : 0xffffffffu;
        const uint32_t f = key != 0xffffffffu;
        uint32_t tot;
        const uint32_t pre = block_excl_scan_256(f, s_tmp, &tot);
        if (f) {
            keys_out[off + pre] = key;
            vals_out[off + pre] = (uint32_t)slot;
            if (vals_copy) vals_copy[off + pre] = (uint32_t)slot;
            if (g2d_rows) {  // the backward's gradient row of this slot starts at zero
                float4* row = reinterpret_cast<float4*>(g2d_rows + slot * G2D_STRIDE);
                row[0] = row[1] = row[2] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (pair_off) {
            const uint32_t c = f ? ntiles[slot] : 0u;
            uint32_t ctot;
            const uint32_t cpre = block_excl_scan_256(c, s_tmp, &ctot);
            if (f) {
                pair_off[off + pre] = poff + cpre;
                mark_chunks(chunk_start, off + pre, poff + cpre, c, cap);
            }
            poff += ctot;
        }
        off += tot;
    }
    if (b == nb - 1 && threadIdx.x == 0) {
        scratch[SCR_NVIS] = off;
        if (pair_off) {
            scratch[SCR_PAIRS] = poff;
            if (poff > cap) atomicOr(err, ERR_OVERFLOW);
            pair_off[off] = poff;
        }
    }
}

int preprocess_blocks(int64_t N) { return (int)ceil_div(N > 0 ? N : 1, PRE_THREADS); }


// with the fused loss the compaction grid counts its normalisers too: a
// block per 4,096 pixels at least
int compact_grid(int64_t N, const Consts& cs) {
    const int64_t blocks = preprocess_blocks(N);
    return (int)(cs.lf_on ? std::max<int64_t>(blocks, ceil_div(cs.lf_pixels, 4096)) : blocks);
}



cudaError_t launch_preprocess(const SceneDev& S, const Views& V, const Consts& cs, float4* xy, float4* conic_o,
                              float4* rgbd, uint2* rect, uint32_t* ntiles, uint32_t* dkey, uint32_t* scratch,
                              uint32_t* state, uint32_t* blk_count, cudaStream_t st) {
    const int blocks = preprocess_blocks(S.N);
    count_launches(1);
    preprocess_kernel<<<(unsigned)blocks, PRE_THREADS, 0, st>>>(S, V, cs, xy, conic_o, rgbd, rect, ntiles, dkey,
                                                                scratch, state, blk_count);
    return cudaGetLastError();
}

cudaError_t launch_compact(const Views& V, int64_t N, const uint32_t* dkey, const uint32_t* blk_count,
                           uint32_t* keys_out, uint32_t* vals_out, uint32_t* vals_copy, const uint32_t* ntiles,
                           uint32_t* pair_off, uint32_t* chunk_start, uint32_t cap, uint32_t* scratch, uint32_t* err,
                           float* g2d_rows, float* pose_zero, int n_pose, const Consts& cs, cudaStream_t st) {
    const int blocks = preprocess_blocks(N);
    const int64_t grid = compact_grid(N, cs);
    // overlapped with the preprocess in front of it (same call): the
    // compaction's CTAs count the loss normalisers as the preprocess drains
    return launch_overlapped(compact_kernel, dim3((unsigned)grid), dim3(256), 0, st, V, N, dkey, blk_count, keys_out,
                             vals_out, vals_copy, ntiles, pair_off, chunk_start, cap, scratch, err, g2d_rows, pose_zero,
                             pose_zero ? n_pose : 0, blocks, cs);
}

// ---------------------------------------------------------------------------
// standalone residual-codebook decode: one thread per output element
// ---------------------------------------------------------------------------
__global__ void rvq_decode_kernel(int dim, int L, int K, const float* __restrict__ cb, const uint8_t* __restrict__ idx,
                                  const float* __restrict__ raw, int64_t n, float* __restrict__ out) {
    const int64_t total = n * dim;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        if (L == 0) {
            out[e] = raw[e];
            continue;
        }
        const int64_t i = e / dim;
        const int c = (int)(e - i * dim);
        float acc = 0.f;
        for (int s = 0; s < L; ++s) {
            int k = __ldg(idx + (int64_t)s * n + i);
            acc += __ldg(cb + ((int64_t)s * K + k) * dim + c);
        }
        out[e] = acc;
    }
}

cudaError_t launch_rvq_decode(int dim, int L, int K, const float* cb, const uint8_t* idx, const float* raw, int64_t n,
                              float* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = ceil_div(n * dim, 256);
    if (blocks > 148 * 32) blocks = 148 * 32;
    count_launches(1);
    rvq_decode_kernel<<<(unsigned)blocks, 256, 0, st>>>(dim, L, K, cb, idx, raw, n, out);
    return cudaGetLastError();
}

}  // namespace vgk
