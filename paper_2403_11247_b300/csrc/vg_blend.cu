// vg_blend.cu -- per-tile front-to-back compositing (Eq. 16-18) and its
// reverse mode.
//
// Forward, per pixel p over its tile's list in (depth, index) order:
//   power = -1/2 d^T conic d (d = uv - p), skipped if > 0
//   alpha = min(alpha_max, o e^power), skipped if < alpha_min
//   stop (Gaussian not blended) if T (1 - alpha) < t_min
//   C += c alpha T, D += z alpha T, S += alpha T, T *= (1 - alpha)
// Keeps the final T and the list position + 1 of the last blended Gaussian.
//
// Backward walks each pixel's list back to front from that position and
// recovers T_i = T_{i+1} / (1 - alpha_i) from the final T (no per-step
// storage).  With w_i = g . (r, g, b, z, 1)_i for the upstream pixel gradient
// g and B_i = sum_{j > i} w_j alpha_j T_j,
//   dL/dalpha_i = T_i w_i - B_i / (1 - alpha_i).
//
// Thread layout: a block is one 16x16 tile; with PPT pixels per thread a warp
// owns a compact rectangle of 32*PPT pixels, so one test per (warp, Gaussian)
// against the Gaussian's alpha >= alpha_min bounding box (half extents from
// the preprocess, widened for FP32 rounding) skips Gaussians that every
// pixel of the warp would skip anyway; the per-pixel decisions are unchanged.
// In the backward, lanes of a warp hold different pixels of the same
// Gaussian: their ten partials are reduced with a fully transposing butterfly
// (12 shuffles) and ten lanes issue the global atomics in one instruction.
#include "vg_blend_common.cuh"

namespace vgk {

// COUNT: keep the work counters (evaluated and blended pairs); off in the
// timed form, whose per-pixel loop then skips their bookkeeping
// Persistent form (PERSIST): the CTAs of the grid pull (view, tile) items
// from the longest-first order through the counter work[0], one item ahead
// (thread 0 holds the next index in `ahead`, so the atomic's round trip
// overlaps the current item); the last CTA to finish puts work[0] and
// work[1] back to zero.  Otherwise CTA b takes item b.
template <bool PERSIST>
__device__ __forceinline__ bool next_item(uint32_t* work, uint32_t& it, uint32_t& ahead, uint32_t total,
                                          uint32_t* s_item) {
    if (!PERSIST) return it < total;
    __syncthreads();  // the previous item's shared memory is free
    if (threadIdx.x == 0) {
        *s_item = ahead;
        if (ahead < total) ahead = atomicAdd(work, 1u);
    }
    __syncthreads();
    it = *s_item;
    return it < total;
}
template <bool PERSIST>
__device__ __forceinline__ void finish_items(uint32_t* work) {
    if (!PERSIST || threadIdx.x != 0) return;
    __threadfence();
    if (atomicAdd(work + 1, 1u) == gridDim.x - 1) {  // every CTA has taken its last item
        work[0] = 0u;
        work[1] = 0u;
    }
}

template <int PPT, bool HITS, bool TSORT, bool COUNT, bool PERSIST>
__global__ void __launch_bounds__(TILE_PIX / PPT) blend_fwd_kernel(
    const __grid_constant__ Views V, Consts cs, uint32_t* work, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ order,
    uint32_t* __restrict__ pvals, const uint32_t* __restrict__ dkey, uint32_t* __restrict__ err,
    const float4* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
    float* __restrict__ C, float* __restrict__ D, float* __restrict__ S, float* __restrict__ Tfin,
    uint32_t* __restrict__ ncontrib, unsigned long long* evals, unsigned long long* blended,
    uint32_t* __restrict__ neval, int count_evals) {
    constexpr int NT = TILE_PIX / PPT;
    // staging of one batch of the tile's Gaussians; before that, the per-tile
    // sort's buffer (VG_TILE_SORT_CAP x 8 bytes) in the same memory
    __shared__ __align__(16) unsigned char s_raw[BLEND_BATCH * (3 * sizeof(float4) + sizeof(uint32_t))];
    static_assert(sizeof(s_raw) >= VG_TILE_SORT_CAP * sizeof(uint2), "sort buffer");
    float4* s_xy = reinterpret_cast<float4*>(s_raw);
    float4* s_co = s_xy + BLEND_BATCH;
    float4* s_cd = s_co + BLEND_BATCH;
    uint32_t* s_gid = reinterpret_cast<uint32_t*>(s_cd + BLEND_BATCH);  // Gaussian ids, for the optional hit counts
    __shared__ uint32_t s_item;
    const uint32_t BB = (uint32_t)cs.blend_batch;

    uint32_t ahead = (PERSIST && threadIdx.x == 0) ? atomicAdd(work, 1u) : 0u;
    for (uint32_t item = PERSIST ? 0u : blockIdx.x;
         next_item<PERSIST>(work, item, ahead, (uint32_t)V.total_tiles, &s_item);) {
    const int gt = (int)order[item];  // longest tile lists first
    const int v = view_of_tile(V, gt);
    const ViewInfo& vi = V.v[v];
    const int t = gt - vi.tile_base;
    const int tx = t % vi.tiles_x, ty = t / vi.tiles_x;
    const int warp = threadIdx.x >> 5;
    float X0, X1, Y0, Y1;
    warp_rect<PPT>(tx, ty, warp, X0, X1, Y0, Y1);

    int px[PPT], py[PPT];
    float fpx[PPT], fpy[PPT];
    bool done[PPT];
    float T[PPT], acc[PPT][5];
    uint32_t last[PPT], stop_at[PPT], nb[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int lx, ly;
        pixel_of<PPT>(threadIdx.x, k, lx, ly);
        px[k] = tx * TILE + lx;
        py[k] = ty * TILE + ly;
        fpx[k] = (float)px[k];
        fpy[k] = (float)py[k];
        done[k] = !(px[k] < vi.W && py[k] < vi.H);
        // a pixel that is not a sampled ray is left out from the start
        if (!done[k] && cs.pix_mask) done[k] = cs.pix_mask[vi.pix_base + (int64_t)py[k] * vi.W + px[k]] == 0;
        T[k] = 1.f;
        last[k] = 0;
        stop_at[k] = done[k] ? 0xfffffffeu : 0xffffffffu;  // a pixel left out examines nothing
        nb[k] = 0;
#pragma unroll
        for (int c = 0; c < 5; ++c) acc[k][c] = 0.f;
    }
    if (cs.lf_on) {  // the fused loss reads these targets once the pixels are done: start them towards L2
        const int64_t HWp = (int64_t)vi.W * vi.H;
#pragma unroll
        for (int k = 0; k < PPT; ++k)
            if (px[k] < vi.W && py[k] < vi.H) {
                const int64_t i = (int64_t)py[k] * vi.W + px[k], pb = vi.pix_base;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(cs.lf_Ct + 3 * pb + i));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(cs.lf_Ct + 3 * pb + HWp + i));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(cs.lf_Ct + 3 * pb + 2 * HWp + i));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(cs.lf_Dt + pb + i));
            }
    }
    const int lane = threadIdx.x & 31;
    const uint2 rg = ranges[gt];
    if (TSORT && rg.y - rg.x > 1) {
        int alldone = 1;
#pragma unroll
        for (int k = 0; k < PPT; ++k) alldone &= (int)done[k];
        // a tile without a pixel to composite needs no order (its backward walks nothing)
        if (__syncthreads_count(alldone) < NT) {
            if (rg.y - rg.x <= (uint32_t)VG_TILE_SORT_CAP)
                tile_sort<NT>(pvals, rg, dkey, reinterpret_cast<uint2*>(s_raw));
            else if (!cs.long_sorted && threadIdx.x == 0)  // (else sorted by the long-list pass)
                atomicOr(err, ERR_TILE_LIST);  // composited unsorted; the outputs are flagged invalid
        }
    }
    for (uint32_t b = rg.x; b < rg.y; b += BB) {
        int alldone = 1;
#pragma unroll
        for (int k = 0; k < PPT; ++k) alldone &= (int)done[k];
        if (__syncthreads_count(alldone) == NT) break;
#pragma unroll 2
        for (int i = threadIdx.x; i < (int)BB; i += NT) {
            const uint32_t j = b + i;
            if (j < rg.y) {
                const uint32_t s = pvals[j];
                s_xy[i] = xy[s];
                s_co[i] = conic_o[s];
                s_cd[i] = rgbd[s];
                if (HITS) s_gid[i] = (uint32_t)(s % (uint64_t)cs.n_gauss);
            }
        }
        __syncthreads();
        const int cnt = (int)min(BB, rg.y - b);
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            int wdone = 1;
#pragma unroll
            for (int k = 0; k < PPT; ++k) wdone &= (int)done[k];
            if (__all_sync(0xffffffffu, wdone)) break;
            // each lane tests one Gaussian of the chunk against the warp's pixels
            const int il = c0 + lane;
            uint32_t m = __ballot_sync(0xffffffffu, il < cnt && warp_hits(s_xy[il], s_co[il], X0, X1, Y0, Y1));
            while (m) {
                const int i = c0 + __ffs(m) - 1;
                m &= m - 1;
                const float4 g = s_xy[i];
                const float4 co = s_co[i];
                const float4 cd = s_cd[i];
                uint32_t hb = 0;  // this lane's pixels that blend Gaussian i (hit counts)
                if (HITS) {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) hb -= nb[k];
                }
                // branch-free per pixel: a pixel that is done, meets a
                // positive exponent or an alpha below alpha_min gets alpha =
                // 0 by select (Tn = T, w = 0: every update an exact no-op); a
                // pixel that stops is not blended
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const float dx = __fsub_rn(g.x, fpx[k]), dy = __fsub_rn(g.y, fpy[k]);
                    const float p2 = gauss_p2(co.x, co.y, co.z, dx, dy);
                    const float q = __fsub_rn(p2, co.w);
                    const bool live = !done[k] && !(p2 > 0.f) && !(q < 0.f);
                    const float e2 = fast_exp2(q);
                    const float alpha = live ? fminf(cs.alpha_max, __fmul_rn(cs.alpha_min, e2)) : 0.f;
                    const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
                    const bool stop = live && Tn < cs.t_min;
                    const bool blend = live && !stop;
                    if (COUNT) stop_at[k] = stop ? b - rg.x + i : stop_at[k];
                    done[k] = done[k] || stop;
                    const float w = blend ? alpha * T[k] : 0.f;
                    acc[k][0] = fmaf(cd.x, w, acc[k][0]);
                    acc[k][1] = fmaf(cd.y, w, acc[k][1]);
                    acc[k][2] = fmaf(cd.z, w, acc[k][2]);
                    acc[k][3] = fmaf(cd.w, w, acc[k][3]);
                    acc[k][4] += w;
                    T[k] = blend ? Tn : T[k];
                    last[k] = blend ? b - rg.x + i + 1 : last[k];
                    if (HITS || COUNT) nb[k] += blend ? 1u : 0u;
                }
                if (HITS) {
#pragma unroll
                    for (int k = 0; k < PPT; ++k) hb += nb[k];
                    const uint32_t tot = __reduce_add_sync(0xffffffffu, hb);
                    if (lane == 0 && tot) atomicAdd(cs.hit_count + s_gid[i], tot);
                }
            }
        }
    }
    const int64_t HW = (int64_t)vi.W * vi.H;
    uint32_t ev = 0, bl = 0;
    // fused L1 loss (vg_render_fwd_l1): its normalisers were counted before
    // this launch, so each pixel's gradient is final as the pixel is written
    float lsum = 0.f, inv_c = 0.f, inv_d = 0.f;
    if (cs.lf_on) {
        const float nv = (float)cs.lf_counts[0];
        const float nsamp = cs.pix_mask ? (float)cs.lf_counts[1] : (float)cs.lf_pixels;
        inv_c = nsamp > 0.f ? 1.f / (3.f * nsamp) : 0.f;
        inv_d = nv > 0.f ? cs.lf_wdepth / nv : 0.f;
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!(px[k] < vi.W && py[k] < vi.H)) continue;
        const int64_t i = (int64_t)py[k] * vi.W + px[k];
        const int64_t pb = vi.pix_base;
        C[3 * pb + i] = acc[k][0];
        C[3 * pb + HW + i] = acc[k][1];
        C[3 * pb + 2 * HW + i] = acc[k][2];
        D[pb + i] = acc[k][3];
        S[pb + i] = acc[k][4];
        Tfin[pb + i] = T[k];
        ncontrib[pb + i] = last[k];
        if (cs.lf_on) {
            const bool smp = cs.pix_mask ? cs.pix_mask[pb + i] != 0 : true;
            float g0, g1, g2, gd;
            lsum += loss_pixel(acc[k][0], acc[k][1], acc[k][2], __ldg(cs.lf_Ct + 3 * pb + i),
                               __ldg(cs.lf_Ct + 3 * pb + HW + i), __ldg(cs.lf_Ct + 3 * pb + 2 * HW + i), acc[k][3],
                               __ldg(cs.lf_Dt + pb + i), acc[k][4], cs.lf_gate, inv_c, inv_d, g0, g1, g2, gd, smp);
            cs.lf_dC[3 * pb + i] = g0;
            cs.lf_dC[3 * pb + HW + i] = g1;
            cs.lf_dC[3 * pb + 2 * HW + i] = g2;
            cs.lf_dD[pb + i] = gd;
            if (cs.lf_dS) cs.lf_dS[pb + i] = 0.f;
        }
        // examined list entries: up to and including the stopping one
        const uint32_t evk = stop_at[k] == 0xffffffffu ? rg.y - rg.x : stop_at[k] == 0xfffffffeu ? 0u : stop_at[k] + 1;
        if (COUNT && neval) neval[pb + i] = evk;
        ev += evk;
        bl += nb[k];
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ev += __shfl_xor_sync(0xffffffffu, ev, o);
            bl += __shfl_xor_sync(0xffffffffu, bl, o);
        }
        if ((threadIdx.x & 31) == 0 && ev) atomicAdd(evals, (unsigned long long)ev);
        if ((threadIdx.x & 31) == 0 && bl) atomicAdd(blended, (unsigned long long)bl);
    }
    if (cs.lf_on) {  // the block's share of the loss, one atomic per block
        __shared__ float s_red[NT / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = lsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) t += s_red[w];
            atomicAdd(cs.lf_loss, t);
        }
    }
    if (!PERSIST) break;
    }  // items
    finish_items<PERSIST>(work);
}

template <int PPT, bool PERSIST>
__global__ void __launch_bounds__(TILE_PIX / PPT) blend_bwd_kernel(
    const __grid_constant__ Views V, Consts cs, uint32_t* work, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ pvals,
    const float4* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
    const float* __restrict__ Tfin, const uint32_t* __restrict__ ncontrib, const float* __restrict__ dC,
    const float* __restrict__ dD, const float* __restrict__ dS, float* __restrict__ g2d,
    unsigned long long* bwd_pairs, int count) {
    constexpr int NT = TILE_PIX / PPT;
    __shared__ float4 s_xy[BLEND_BATCH];
    __shared__ float4 s_co[BLEND_BATCH];   // base-2 exponent coefficients and threshold
    __shared__ float4 s_nat[BLEND_BATCH];  // inverse 2D covariance a, b, c and 1/opacity
    __shared__ float4 s_cd[BLEND_BATCH];
    __shared__ uint32_t s_slot[BLEND_BATCH];
    __shared__ uint32_t s_max;
    __shared__ uint32_t s_item;
    const uint32_t BB = (uint32_t)cs.blend_batch;

    uint32_t ahead = (PERSIST && threadIdx.x == 0) ? atomicAdd(work, 1u) : 0u;
    for (uint32_t item = PERSIST ? 0u : blockIdx.x;
         next_item<PERSIST>(work, item, ahead, (uint32_t)V.total_tiles, &s_item);) {
    const int gt = (int)order[item];  // longest tile lists first
    const int v = view_of_tile(V, gt);
    const ViewInfo& vi = V.v[v];
    const int t = gt - vi.tile_base;
    const int tx = t % vi.tiles_x, ty = t / vi.tiles_x;
    const int64_t HW = (int64_t)vi.W * vi.H, pb = vi.pix_base;
    const int warp = threadIdx.x >> 5;
    float X0, X1, Y0, Y1;
    warp_rect<PPT>(tx, ty, warp, X0, X1, Y0, Y1);

    int px[PPT], py[PPT];
    float fpx[PPT], fpy[PPT];
    uint32_t nc[PPT];
    float T[PPT], Bk[PPT], gp[PPT][5];
    uint32_t mymax = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int lx, ly;
        pixel_of<PPT>(threadIdx.x, k, lx, ly);
        px[k] = tx * TILE + lx;
        py[k] = ty * TILE + ly;
        fpx[k] = (float)px[k];
        fpy[k] = (float)py[k];
        const bool inside = px[k] < vi.W && py[k] < vi.H;
        const int64_t i = (int64_t)py[k] * vi.W + px[k];
        nc[k] = inside ? ncontrib[pb + i] : 0u;
        T[k] = inside ? Tfin[pb + i] : 1.f;
        Bk[k] = 0.f;
        gp[k][0] = (inside && dC) ? dC[3 * pb + i] : 0.f;
        gp[k][1] = (inside && dC) ? dC[3 * pb + HW + i] : 0.f;
        gp[k][2] = (inside && dC) ? dC[3 * pb + 2 * HW + i] : 0.f;
        gp[k][3] = (inside && dD) ? dD[pb + i] : 0.f;
        gp[k][4] = (inside && dS) ? dS[pb + i] : 0.f;
        mymax = max(mymax, nc[k]);
    }
    if (count) {
        uint32_t walked = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) walked += nc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) walked += __shfl_xor_sync(0xffffffffu, walked, o);
        if ((threadIdx.x & 31) == 0 && walked) atomicAdd(bwd_pairs, (unsigned long long)walked);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, mymax);
    __syncthreads();
    const uint2 rg = ranges[gt];
    const uint32_t end = rg.x + min(s_max, rg.y - rg.x);
    // largest list position this warp still needs
    const uint32_t warp_max = mymax;
    // this lane's reduced value and its factor: dL/d(u, v) = -sum dp (conic d);
    // dL/d(a, b, c) = -sum dp (dx^2/2, dx dy, dy^2/2); dL/do = sum e^power dA
    // with e^power = x / o (the 1/o is the visited Gaussian's); the rest as summed
    const int red_idx = reduce10_index(threadIdx.x & 31);
    const float red_scale = (red_idx == 2 || red_idx == 4) ? -0.5f : (red_idx >= 0 && red_idx <= 3) ? -1.f : 1.f;

    for (uint32_t bend = end; bend > rg.x;) {
        const uint32_t bstart = (bend - rg.x > BB) ? bend - BB : rg.x;
        __syncthreads();
        for (int i = threadIdx.x; i < (int)(bend - bstart); i += NT) {
            const uint32_t s = pvals[bstart + i];
            s_slot[i] = s;
            s_xy[i] = xy[s];
            const float4 co = conic_o[s];
            s_co[i] = co;
            // natural-unit conic and 1/opacity: a = -2 ln2 A2, b = -ln2 B2,
            // c = -2 ln2 C2, 1/o = 2^thr / alpha_min
            s_nat[i] = make_float4(-2.f * LN2 * co.x, -LN2 * co.y, -2.f * LN2 * co.z,
                                   fast_exp2(co.w) / cs.alpha_min);
            s_cd[i] = rgbd[s];
        }
        __syncthreads();
        const int lane = threadIdx.x & 31;
        for (int c1 = (int)(bend - bstart); c1 > 0; c1 -= 32) {
            const int c0 = c1 > 32 ? c1 - 32 : 0;
            // each lane tests one Gaussian of the chunk; hits are then walked
            // back to front (highest set bit first)
            const int il = c0 + lane;
            const bool hit = il < c1 && (bstart - rg.x + (uint32_t)il) < warp_max &&
                             warp_hits(s_xy[il], s_co[il], X0, X1, Y0, Y1);
            uint32_t m = __ballot_sync(0xffffffffu, hit);
            while (m) {
                const int hb = 31 - __clz(m);
                m &= ~(1u << hb);
                const int i = c0 + hb;
                const uint32_t jl = bstart - rg.x + (uint32_t)i;
                const float4 g = s_xy[i];
                const float4 co = s_co[i];
                const float4 nat = s_nat[i];
                const float4 cd = s_cd[i];
                float vals[10];
#pragma unroll
                for (int c = 0; c < 10; ++c) vals[c] = 0.f;
                bool any = false;
                // Branch-free per pixel: a pixel that does not blend this
                // Gaussian (past its last contributor, positive exponent,
                // alpha below alpha_min) gets alpha = x = 0 by select, which
                // makes every update below an exact no-op; a pixel that
                // blends takes exactly the arithmetic of the walk.  (Whole
                // warps rarely skip a visited Gaussian, so branching around
                // the update costs more in reconvergence than it saves.)
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const float dx = __fsub_rn(g.x, fpx[k]), dy = __fsub_rn(g.y, fpy[k]);
                    const float p2 = gauss_p2(co.x, co.y, co.z, dx, dy);
                    const float q = __fsub_rn(p2, co.w);
                    const bool live = jl < nc[k] && !(p2 > 0.f) && !(q < 0.f);
                    const float e2 = fast_exp2(q);
                    const float x = live ? __fmul_rn(cs.alpha_min, e2) : 0.f;  // o e^power before the cap
                    const float alpha = fminf(cs.alpha_max, x);
                    const float inv = __fdividef(1.f, 1.f - alpha);  // hardware reciprocal, ~2 ulp
                    T[k] = live ? T[k] * inv : T[k];  // transmittance in front of this Gaussian
                    const float w = gp[k][0] * cd.x + gp[k][1] * cd.y + gp[k][2] * cd.z + gp[k][3] * cd.w + gp[k][4];
                    const float dA = T[k] * w - Bk[k] * inv;
                    const float wt = alpha * T[k];
                    Bk[k] = fmaf(w, wt, Bk[k]);
                    vals[6] = fmaf(wt, gp[k][0], vals[6]);
                    vals[7] = fmaf(wt, gp[k][1], vals[7]);
                    vals[8] = fmaf(wt, gp[k][2], vals[8]);
                    vals[9] = fmaf(wt, gp[k][3], vals[9]);
                    // capped alpha is constant: no conic, mean or opacity terms.
                    // The per-Gaussian factors (e^power = x / o, the signs and
                    // halves of the conic terms) are applied once per visit below
                    // (uncapped, x is alpha: dp = alpha dA = x dA, and the
                    // opacity sum takes the same dp)
                    const float xu = x <= cs.alpha_max ? x : 0.f;
                    const float dp = xu * dA;
                    const float pdx = dp * dx, pdy = dp * dy;
                    vals[5] += dp;
                    vals[0] = fmaf(nat.x, pdx, fmaf(nat.y, pdy, vals[0]));
                    vals[1] = fmaf(nat.y, pdx, fmaf(nat.z, pdy, vals[1]));
                    vals[2] = fmaf(pdx, dx, vals[2]);
                    vals[3] = fmaf(pdx, dy, vals[3]);
                    vals[4] = fmaf(pdy, dy, vals[4]);
                    any |= live;
                }
                if (__any_sync(0xffffffffu, any)) {
                    const float sum = warp_reduce10(vals);
                    if (red_idx >= 0)
                        atomicAdd(g2d + (int64_t)s_slot[i] * G2D_STRIDE + red_idx,
                                  sum * (red_idx == 5 ? nat.w : red_scale));
                }
            }
        }
        bend = bstart;
    }
    if (!PERSIST) break;
    }  // items
    finish_items<PERSIST>(work);
}

static int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 148;
    }
    return sms;
}

static unsigned blend_grid(const Views& V, int persist, uint32_t*& work) {
    if (persist <= 0) {
        work = nullptr;
        return (unsigned)V.total_tiles;
    }
    const int64_t g = (int64_t)persist * sm_count();
    return (unsigned)(g < V.total_tiles ? g : V.total_tiles);
}

cudaError_t launch_blend_fwd(const Views& V, const Consts& cs, int ppt, int persist, uint32_t* work,
                             const uint2* ranges, const uint32_t* order,
                             uint32_t* pvals, const uint32_t* dkey, uint32_t* err,
                             const float4* xy, const float4* conic_o, const float4* rgbd, float* C, float* D, float* S,
                             float* Tfin, uint32_t* ncontrib, unsigned long long* evals, unsigned long long* blended,
                             uint32_t* neval, int count_evals, cudaStream_t st) {
    if (V.total_tiles <= 0) return cudaSuccess;
    count_launches(1);
    const unsigned grid = blend_grid(V, persist, work);
#define VG_FWD5(P, H, TS, CN, PE)                                                                               \
    blend_fwd_kernel<P, H, TS, CN, PE><<<grid, TILE_PIX / P, 0, st>>>(V, cs, work, ranges, order, pvals, dkey, err, \
                                                                           xy, conic_o, rgbd, C, D, S, Tfin,     \
                                                                           ncontrib, evals, blended, neval,      \
                                                                           count_evals)
#define VG_FWD4(P, H, TS, CN)                                                                                   \
    do {                                                                                                        \
        if (work) VG_FWD5(P, H, TS, CN, true); else VG_FWD5(P, H, TS, CN, false);                                \
    } while (0)
#define VG_FWD3(P, H, TS)                                                                                       \
    do {                                                                                                        \
        if (count_evals) VG_FWD4(P, H, TS, true); else VG_FWD4(P, H, TS, false);                                \
    } while (0)
#define VG_FWD(P)                                                                                               \
    do {                                                                                                        \
        if (cs.hit_count) {                                                                                     \
            if (dkey) VG_FWD3(P, true, true); else VG_FWD3(P, true, false);                                     \
        } else {                                                                                                \
            if (dkey) VG_FWD3(P, false, true); else VG_FWD3(P, false, false);                                   \
        }                                                                                                       \
    } while (0)
    if (ppt == 4) VG_FWD(4);
    else if (ppt == 2) VG_FWD(2);
    else VG_FWD(1);
#undef VG_FWD
#undef VG_FWD3
#undef VG_FWD4
#undef VG_FWD5
    return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const Views& V, const Consts& cs, int ppt, int persist, uint32_t* work,
                             const uint2* ranges, const uint32_t* order,
                             const uint32_t* pvals,
                             const float4* xy, const float4* conic_o, const float4* rgbd, const float* Tfin,
                             const uint32_t* ncontrib, const float* dC, const float* dD, const float* dS, float* g2d,
                             unsigned long long* bwd_pairs, int count, cudaStream_t st) {
    if (V.total_tiles <= 0) return cudaSuccess;
    count_launches(1);
    const unsigned grid = blend_grid(V, persist, work);
#define VG_BWD2(P, PE)                                                                                               \
    blend_bwd_kernel<P, PE><<<grid, TILE_PIX / P, 0, st>>>(V, cs, work, ranges, order, pvals, xy, conic_o, rgbd, Tfin, \
                                                           ncontrib, dC, dD, dS, g2d, bwd_pairs, count)
#define VG_BWD(P)                                                                                                    \
    do {                                                                                                             \
        if (work) VG_BWD2(P, true); else VG_BWD2(P, false);                                                          \
    } while (0)
    if (ppt == 1) VG_BWD(1);
    else if (ppt == 2) VG_BWD(2);
    else VG_BWD(4);
#undef VG_BWD
#undef VG_BWD2
    return cudaGetLastError();
}

}  // namespace vgk
