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
// In the backward, the walk (one pixel per lane) queues each visit's
// per-pixel (dp, wt) in shared memory, and every 16 visits (8 at 4 pixels
// per thread) the warp sums the queued Gaussians' ten gradient partials
// with one Gaussian per lane pair (quad): no reduction across the warp.
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

// Backward gradient queue.  The walk keeps one pixel per lane (a pixel's
// transmittance and its running sum B are sequential in the list), but the
// ten per-Gaussian sums are taken with one Gaussian per lane group: each
// visit stores its pixels' (dp, wt) = (x dL/dalpha, alpha T) in the warp's
// queue column and the Gaussian's staged index, and every QN visits the
// warp turns the queue around -- the LPE = 32/QN lanes of entry e each sum
// its partials over PPL of the warp's pixels, 0-2 shuffle stages fold the
// parts (each part keeps half of the remaining values), and every lane adds
// its sums to the Gaussian's gradient row.  No sum crosses all 32 lanes.
// Rows are padded by one float2, so both the column writes of the walk and
// the row reads of the turn-around are free of bank conflicts.
template <int PPT>
struct BwdQueue {
    static constexpr int NW = TILE_PIX / PPT / 32;  // warps per block
    static constexpr int WP = 32 * PPT;             // pixels per warp
    static constexpr int QN = PPT >= 4 ? 8 : 16;    // visits per turn-around
    static constexpr int LPE = 32 / QN;             // lanes per queued Gaussian
    static constexpr int PPL = WP / LPE;            // pixels each of them sums
    static constexpr int QROW = QN + 1;             // float2 per pixel row
    static constexpr int GROW = PPL + 1;            // float4 per part's pixel gradients
    static constexpr int STAGE = 128;               // Gaussians staged at a time (at most)
    static constexpr int MINB = PPT == 1 ? 3 : PPT == 2 ? 4 : 2;  // blocks per SM the registers must allow
    static constexpr size_t BYTES = (size_t)STAGE * (3 * sizeof(float4) + sizeof(uint32_t)) +
                                    (size_t)NW * LPE * GROW * sizeof(float4) +
                                    (size_t)NW * WP * QROW * sizeof(float2) + (size_t)NW * QN * sizeof(uint32_t);
};

// The turn-around of one warp's queue (nq <= 32 / LPE visits, LPE lanes per
// queued Gaussian).  Sums, for the
// Gaussian at mean (u, v) over the part's pixels (dx = u - px, dy = v - py),
//   s0 = sum dp dx, s1 = sum dp dy, s2 = sum dp dx^2, s3 = sum dp dx dy,
//   s4 = sum dp dy^2, s5 = sum dp, s6..s9 = sum wt (dC_r, dC_g, dC_b, dD);
// then dL/du = -(a s0 + b s1), dL/dv = -(b s0 + c s1) for the natural-unit
// inverse covariance (a, b, c), dL/d(a, b, c) = (-s2/2, -s3, -s4/2),
// dL/do = s5 / o (dp = o e^power dL/dalpha) and the colour and depth
// gradients s6..s9 (Eq. 16-18 in reverse).
template <int PPT, int LPE>
__device__ __forceinline__ void bwd_turn_around(int nq, const float2* __restrict__ sq, const float4* __restrict__ sgp,
                                                const uint32_t* __restrict__ sqi, const float4* __restrict__ s_xy,
                                                const float4* __restrict__ s_co, const uint32_t* __restrict__ s_slot,
                                                float X0, float Y0, float alpha_min, float* __restrict__ g2d) {
    using Q = BwdQueue<PPT>;
    using R = WarpRect<PPT>;
    constexpr int NE = 32 / LPE;     // entries this turn-around takes
    constexpr int PPL = Q::WP / LPE;  // pixels each lane sums
    constexpr int ROWS = PPL / R::W;
    static_assert(LPE >= Q::LPE && LPE <= 4 && ROWS >= 1, "turn-around shape");
    const int lane = threadIdx.x & 31;
    const int e = lane % NE, part = lane / NE;
    const bool valid = e < nq;
    const uint32_t i = sqi[valid ? e : 0];
    const float4 g = s_xy[i];
    float dxs[R::W];
#pragma unroll
    for (int c = 0; c < R::W; ++c) dxs[c] = __fsub_rn(g.x, X0 + (float)c);
    const float Yp = Y0 + (float)(part * ROWS);
    const int j0 = part * PPL;  // the part's first pixel
    const float2* q = sq + j0 * Q::QROW + e;
    const float4* gq = sgp + (j0 / Q::PPL) * Q::GROW + j0 % Q::PPL;
    float s[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) s[c] = 0.f;
    // a pixel row shares dy: per row, sum dp dx, dp dx^2 and dp, then fold
    // in the dy factors once
#pragma unroll 1
    for (int r = 0; r < ROWS; ++r, q += R::W * Q::QROW, gq += R::W) {
        float A = 0.f, B = 0.f, C = 0.f;
#pragma unroll
        for (int c = 0; c < R::W; ++c) {
            const float2 pw = q[c * Q::QROW];
            const float4 gp = gq[c];
            const float pdx = pw.x * dxs[c];
            A += pdx;
            B = fmaf(pdx, dxs[c], B);
            C += pw.x;
            s[6] = fmaf(pw.y, gp.x, s[6]);
            s[7] = fmaf(pw.y, gp.y, s[7]);
            s[8] = fmaf(pw.y, gp.z, s[8]);
            s[9] = fmaf(pw.y, gp.w, s[9]);
        }
        const float dy = __fsub_rn(g.y, Yp + (float)r);
        s[0] += A;
        s[1] = fmaf(C, dy, s[1]);
        s[2] += B;
        s[3] = fmaf(A, dy, s[3]);
        s[4] = fmaf(C * dy, dy, s[4]);
        s[5] += C;
    }
    // fold the parts: value v ends in the lane whose part bits select it
    int first = 0;  // index of this lane's first kept value
    int kept = 10;
    if constexpr (LPE >= 2) {
        const bool h16 = (lane & 16) != 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float send = h16 ? s[k] : s[k + 5];
            const float keep = h16 ? s[k + 5] : s[k];
            s[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
        first = h16 ? 5 : 0;
        kept = 5;
    }
    if constexpr (LPE >= 4) {
        const bool h8 = (lane & 8) != 0;  // clear: values first..first+2, set: first+3, first+4
        const float b0 = (h8 ? s[3] : s[0]) + __shfl_xor_sync(0xffffffffu, h8 ? s[0] : s[3], 8);
        const float b1 = (h8 ? s[4] : s[1]) + __shfl_xor_sync(0xffffffffu, h8 ? s[1] : s[4], 8);
        const float b2 = s[2] + __shfl_xor_sync(0xffffffffu, s[2], 8);  // (kept by the clear lane only)
        s[0] = b0;
        s[1] = b1;
        s[2] = b2;
        first += h8 ? 3 : 0;
        kept = h8 ? 2 : 3;
    }
    if (!valid) return;
    const float4 co = s_co[i];
    float* row = g2d + (int64_t)s_slot[i] * G2D_STRIDE + first;
    // natural-unit inverse covariance from the base-2 coefficients:
    // a = -2 ln2 A2, b = -ln2 B2, c = -2 ln2 C2; 1/o = 2^thr / alpha_min
    const float na = -2.f * LN2 * co.x, nb = -LN2 * co.y, nc = -2.f * LN2 * co.z;
    const float inv_o = fast_exp2(co.w) / alpha_min;
    constexpr int KMAX = LPE == 1 ? 10 : LPE == 2 ? 5 : 3;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < kept) {
            const int v = first + k;
            const float sc = (v == 2 || v == 4) ? -0.5f : v == 3 ? -1.f : v == 5 ? inv_o : 1.f;
            float out = s[k] * sc;
            if (k == 0 && v == 0) out = -(na * s[0] + nb * s[1]);
            if (k == 1 && v == 1) out = -(nb * s[0] + nc * s[1]);
            atomicAdd(row + k, out);
        }
    }
}

template <int PPT, bool PERSIST>
__global__ void __launch_bounds__(TILE_PIX / PPT, BwdQueue<PPT>::MINB) blend_bwd_kernel(
    const __grid_constant__ Views V, Consts cs, uint32_t* work, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ pvals,
    const float4* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
    const float* __restrict__ Tfin, const uint32_t* __restrict__ ncontrib, const float* __restrict__ dC,
    const float* __restrict__ dD, const float* __restrict__ dS, float* __restrict__ g2d,
    unsigned long long* bwd_pairs, int count) {
    allow_dependents();  // the chain kernel's scene-only prefix may overlap this kernel's last CTAs
    using Q = BwdQueue<PPT>;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_xy = reinterpret_cast<float4*>(smem);
    float4* s_co = s_xy + Q::STAGE;  // base-2 exponent coefficients and threshold
    float4* s_cd = s_co + Q::STAGE;  // colour and depth
    float4* s_gp = s_cd + Q::STAGE;  // per warp and part: the pixels' upstream colour and depth gradients
    float2* s_q = reinterpret_cast<float2*>(s_gp + Q::NW * Q::LPE * Q::GROW);  // per warp: [pixel][visit]
    uint32_t* s_slot = reinterpret_cast<uint32_t*>(s_q + Q::NW * Q::WP * Q::QROW);
    uint32_t* s_qi = s_slot + Q::STAGE;  // per warp: staged index of each queued visit
    __shared__ uint32_t s_max;
    __shared__ uint32_t s_item;
    const uint32_t BB = min((uint32_t)cs.blend_batch, (uint32_t)Q::STAGE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* const sgp = s_gp + warp * Q::LPE * Q::GROW;
    float2* const sq = s_q + warp * Q::WP * Q::QROW;
    uint32_t* const sqi = s_qi + warp * Q::QN;

    uint32_t ahead = (PERSIST && threadIdx.x == 0) ? atomicAdd(work, 1u) : 0u;
    for (uint32_t item = PERSIST ? 0u : blockIdx.x;
         next_item<PERSIST>(work, item, ahead, (uint32_t)V.total_tiles, &s_item);) {
    const int gt = (int)order[item];  // longest tile lists first
    const int v = view_of_tile(V, gt);
    const ViewInfo& vi = V.v[v];
    const int t = gt - vi.tile_base;
    const int tx = t % vi.tiles_x, ty = t / vi.tiles_x;
    const int64_t HW = (int64_t)vi.W * vi.H, pb = vi.pix_base;
    float X0, X1, Y0, Y1;
    warp_rect<PPT>(tx, ty, warp, X0, X1, Y0, Y1);

    // a lane's pixels share their column (the warp rectangle's width divides 32)
    static_assert(32 % WarpRect<PPT>::W == 0, "pixel columns per lane");
    float fpx = 0.f, fpy[PPT];
    uint32_t nc[PPT];
    float T[PPT], Bk[PPT], gp[PPT][5];
    uint32_t mymax = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int lx, ly;
        pixel_of<PPT>(threadIdx.x, k, lx, ly);
        const int px = tx * TILE + lx, py = ty * TILE + ly;
        fpx = (float)px;
        fpy[k] = (float)py;
        const bool inside = px < vi.W && py < vi.H;
        const int64_t i = (int64_t)py * vi.W + px;
        nc[k] = inside ? ncontrib[pb + i] : 0u;
        T[k] = inside ? Tfin[pb + i] : 1.f;
        Bk[k] = 0.f;
        gp[k][0] = (inside && dC) ? dC[3 * pb + i] : 0.f;
        gp[k][1] = (inside && dC) ? dC[3 * pb + HW + i] : 0.f;
        gp[k][2] = (inside && dC) ? dC[3 * pb + 2 * HW + i] : 0.f;
        gp[k][3] = (inside && dD) ? dD[pb + i] : 0.f;
        gp[k][4] = (inside && dS) ? dS[pb + i] : 0.f;
        mymax = max(mymax, nc[k]);
        const int j = lane + 32 * k;  // the pixel's row in the warp's queue
        sgp[(j / Q::PPL) * Q::GROW + j % Q::PPL] = make_float4(gp[k][0], gp[k][1], gp[k][2], gp[k][3]);
    }
    if (count) {
        uint32_t walked = 0;
#pragma unroll
        for (int k = 0; k < PPT; ++k) walked += nc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) walked += __shfl_xor_sync(0xffffffffu, walked, o);
        if (lane == 0 && walked) atomicAdd(bwd_pairs, (unsigned long long)walked);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if (lane == 0) atomicMax(&s_max, mymax);
    __syncthreads();
    const uint2 rg = ranges[gt];
    const uint32_t end = rg.x + min(s_max, rg.y - rg.x);
    // largest list position this warp still needs
    const uint32_t warp_max = mymax;
    int qn = 0;  // visits in the warp's queue (warp-uniform)

    for (uint32_t bend = end; bend > rg.x;) {
        // batches start at multiples of BB from the list start, and chunks
        // at multiples of 32 from the batch start (the part-filled chunk is
        // the first walked)
        const uint32_t bstart = rg.x + ((bend - rg.x - 1) / BB) * BB;
        __syncthreads();
        for (int i = threadIdx.x; i < (int)(bend - bstart); i += TILE_PIX / PPT) {
            const uint32_t s = pvals[bstart + i];
            s_slot[i] = s;
            s_xy[i] = xy[s];
            s_co[i] = conic_o[s];
            s_cd[i] = rgbd[s];
        }
        __syncthreads();
        for (int c1 = (int)(bend - bstart); c1 > 0; c1 = (c1 - 1) & ~31) {
            const int c0 = (c1 - 1) & ~31;
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
                const float4 cd = s_cd[i];
                float2* const qc = sq + lane * Q::QROW + qn;
                const float dx = __fsub_rn(g.x, fpx);
                // Branch-free per pixel: a pixel that does not blend this
                // Gaussian (past its last contributor, positive exponent,
                // alpha below alpha_min) gets alpha = x = 0 by select, which
                // makes every update an exact no-op and queues (0, 0); a
                // pixel that blends takes exactly the arithmetic of the walk.
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const float dy = __fsub_rn(g.y, fpy[k]);
                    const float p2 = gauss_p2(co.x, co.y, co.z, dx, dy);
                    const float q = __fsub_rn(p2, co.w);
                    const bool live = jl < nc[k] && !(p2 > 0.f) && !(q < 0.f);
                    const float e2 = fast_exp2(q);
                    const float x = live ? __fmul_rn(cs.alpha_min, e2) : 0.f;  // o e^power before the cap
                    const float alpha = fminf(cs.alpha_max, x);
                    const float inv = __fdividef(1.f, 1.f - alpha);  // hardware reciprocal, ~2 ulp
                    T[k] = live ? T[k] * inv : T[k];  // transmittance in front of this Gaussian
                    const float w =
                        fmaf(gp[k][3], cd.w, fmaf(gp[k][2], cd.z, fmaf(gp[k][1], cd.y, fmaf(gp[k][0], cd.x, gp[k][4]))));
                    const float dA = T[k] * w - Bk[k] * inv;
                    const float wt = alpha * T[k];
                    Bk[k] = fmaf(w, wt, Bk[k]);
                    // a capped alpha is constant: no conic, mean or opacity
                    // terms; uncapped, alpha = x and dp = x dA feeds them all
                    const float xu = x <= cs.alpha_max ? x : 0.f;
                    qc[k * 32 * Q::QROW] = make_float2(xu * dA, wt);
                }
                sqi[qn] = (uint32_t)i;
                if (++qn == Q::QN) {
                    __syncwarp();
                    bwd_turn_around<PPT, Q::LPE>(Q::QN, sq, sgp, sqi, s_xy, s_co, s_slot, X0, Y0, cs.alpha_min, g2d);
                    qn = 0;
                    __syncwarp();
                }
            }
        }
        if (qn) {  // the queue refers to staged Gaussians: empty it before the next batch
            __syncwarp();
            bwd_turn_around<PPT, Q::LPE>(qn, sq, sgp, sqi, s_xy, s_co, s_slot, X0, Y0, cs.alpha_min, g2d);
            qn = 0;
            __syncwarp();
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
    else if (ppt == 1) VG_FWD(1);
    else VG_FWD(2);
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
    do {                                                                                                             \
        const cudaError_t e = allow_dynamic_smem((const void*)blend_bwd_kernel<P, PE>, BwdQueue<P>::BYTES);          \
        if (e != cudaSuccess) return e;                                                                              \
        blend_bwd_kernel<P, PE><<<grid, TILE_PIX / P, BwdQueue<P>::BYTES, st>>>(                                     \
            V, cs, work, ranges, order, pvals, xy, conic_o, rgbd, Tfin, ncontrib, dC, dD, dS, g2d, bwd_pairs, count); \
    } while (0)
#define VG_BWD(P)                                                                                                    \
    do {                                                                                                             \
        if (work) VG_BWD2(P, true); else VG_BWD2(P, false);                                                          \
    } while (0)
    if (ppt == 1) VG_BWD(1);
    else if (ppt == 4) VG_BWD(4);
    else VG_BWD(2);
#undef VG_BWD
#undef VG_BWD2
    return cudaGetLastError();
}

}  // namespace vgk
