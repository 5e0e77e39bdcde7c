// vg_split.cu -- compositing of deep tile lists split across CTAs.
//
// When an image has few tiles (fewer than the GPU has SMs to give one CTA
// each) and their lists are deep, the per-tile kernels leave most SMs idle
// and each CTA walks its whole list alone.  Here each tile's (depth-sorted)
// list is cut into S consecutive segments and every (tile, segment) item is a
// CTA.  The front-to-back sums of Eq. 16-18 split over ordered segments:
// with T_in(s) the transmittance in front of segment s,
//   C = sum_s C_s  where C_s = sum_{i in s} c_i alpha_i T_i  and  T_i = T_in(s) prod_{j in s, j < i} (1 - alpha_j),
//   T_in(s + 1) = T_in(s) P_s,  P_s = prod_{i in s} (1 - alpha_i).
// Three passes:
//   1. split_prod: every segment's P_s per pixel (a pixel stops multiplying
//      once its product is below t_min: the segments behind it then see
//      T_in < t_min whatever the rest of the product is).
//   2. split_walk: T_in(s) = prod_{s' < s} P_s', then the segment is walked
//      exactly as the per-tile forward walks a list (alpha tests, the stop
//      rule against t_min, the blended sums with absolute T), starting from
//      T_in(s).  A pixel with T_in(s) < t_min stopped in an earlier segment
//      and does nothing here.
//   3. split_combine: per pixel, the segments' sums in order, the final T of
//      the last segment the pixel composited, the last contributor, the work
//      counts and (vg_render_fwd_l1) the fused L1 loss gradient.
// The results equal the per-tile forward's up to the rounding of the
// transmittance products (associated per segment); every decision (alpha
// tests, the stop) is the same except where a product lands within rounding
// of t_min.
//
// The backward splits the same way: segment s walks its part of the pixel's
// list back to front from T_out(s) (its own final transmittance, kept by
// pass 2), with the sum of the Gaussians behind it, B = sum_{i behind} w_i
// alpha_i T_i, started at g . (C, D, S) of the later segments (w_i is linear
// in the colour, depth and the constant 1).
#include "vg_blend_common.cuh"

namespace vgk {

constexpr int SPLIT_NT = TILE_PIX;  // one pixel per thread
constexpr uint32_t SPLIT_NONE = 0xffffffffu;

// per (item, field, tile pixel) storage of the split passes
__device__ __forceinline__ size_t sf_idx(uint32_t item, int f, int pid) {
    return ((size_t)item * SPLIT_F + f) * TILE_PIX + pid;
}
__device__ __forceinline__ size_t su_idx(uint32_t item, int f, int pid) {
    return ((size_t)item * SPLIT_U + f) * TILE_PIX + pid;
}

// the list positions [a, b) of segment s of S of the list rg
__device__ __forceinline__ void segment_of(uint2 rg, int s, int S, uint32_t& a, uint32_t& b) {
    const uint64_t len = rg.y - rg.x;
    a = rg.x + (uint32_t)((len * (uint64_t)s) / (uint64_t)S);
    b = rg.x + (uint32_t)((len * (uint64_t)(s + 1)) / (uint64_t)S);
}

struct SplitPixel {
    int px, py, pid;
    float fpx, fpy;
    bool inside;
    float X0, X1, Y0, Y1;  // the warp's pixel rectangle
};

__device__ __forceinline__ SplitPixel split_pixel(const ViewInfo& vi, int t) {
    SplitPixel p;
    const int tx = t % vi.tiles_x, ty = t / vi.tiles_x;
    int lx, ly;
    pixel_of<1>(threadIdx.x, 0, lx, ly);
    p.pid = ly * TILE + lx;
    p.px = tx * TILE + lx;
    p.py = ty * TILE + ly;
    p.fpx = (float)p.px;
    p.fpy = (float)p.py;
    p.inside = p.px < vi.W && p.py < vi.H;
    warp_rect<1>(tx, ty, (int)(threadIdx.x >> 5), p.X0, p.X1, p.Y0, p.Y1);
    return p;
}

// per-tile sort of the lists (the per-tile form) before they are split: the
// same (depth bits, slot) order the per-tile forward builds for itself, by a
// bitonic network over the list padded to a power of two in shared memory
// (the lists here are deep: a network of log^2 steps beats the per-tile
// forward's rank merge, whose work grows with n^2 / 32)
__global__ void __launch_bounds__(SPLIT_NT) split_sort_kernel(Consts cs, const uint2* __restrict__ ranges,
                                                              uint32_t* __restrict__ pvals,
                                                              const uint32_t* __restrict__ dkey,
                                                              uint32_t* __restrict__ err) {
    __shared__ __align__(16) uint2 s_kv[VG_TILE_SORT_CAP];
    const uint2 rg = ranges[blockIdx.x];
    const uint32_t n = rg.y - rg.x;
    if (n <= 1) return;
    if (n > (uint32_t)VG_TILE_SORT_CAP) {
        if (!cs.long_sorted && threadIdx.x == 0) atomicOr(err, ERR_TILE_LIST);  // (else sorted by the long-list pass)
        return;
    }
    uint32_t n2 = 32;
    while (n2 < n) n2 <<= 1;
    for (uint32_t e = threadIdx.x; e < n2; e += SPLIT_NT) {
        uint2 kv = make_uint2(0xffffffffu, 0xffffffffu);  // padding sorts last
        if (e < n) {
            kv.y = pvals[rg.x + e];
            kv.x = dkey[kv.y];
        }
        s_kv[e] = kv;
    }
    __syncthreads();
    for (uint32_t size = 2; size <= n2; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            // each thread takes pairs (lo, lo + stride), lo with the stride bit clear
            for (uint32_t t = threadIdx.x; t < n2 / 2; t += SPLIT_NT) {
                const uint32_t lo = 2 * t - (t & (stride - 1));
                const uint32_t hi = lo + stride;
                const uint2 x = s_kv[lo], y = s_kv[hi];
                const bool asc = (lo & size) == 0;
                if (kv_less(y.x, y.y, x.x, x.y) == asc) {
                    s_kv[lo] = y;
                    s_kv[hi] = x;
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t e = threadIdx.x; e < n; e += SPLIT_NT) pvals[rg.x + e] = s_kv[e].y;
}

// pass 1: P_s per pixel
__global__ void __launch_bounds__(SPLIT_NT) split_prod_kernel(const __grid_constant__ Views V, Consts cs, int S,
                                                              const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ pvals,
                                                              const float4* __restrict__ xy,
                                                              const float4* __restrict__ conic_o,
                                                              float* __restrict__ segf) {
    __shared__ float4 s_xy[BLEND_BATCH];
    __shared__ float4 s_co[BLEND_BATCH];
    const uint32_t item = blockIdx.x;
    const int gt = (int)(item / (uint32_t)S), s = (int)(item % (uint32_t)S);
    const int v = view_of_tile(V, gt);
    const ViewInfo& vi = V.v[v];
    const SplitPixel P = split_pixel(vi, gt - vi.tile_base);
    bool done = !P.inside;
    if (!done && cs.pix_mask) done = cs.pix_mask[vi.pix_base + (int64_t)P.py * vi.W + P.px] == 0;
    float T = 1.f;
    uint32_t a, b;
    segment_of(ranges[gt], s, S, a, b);
    const int lane = threadIdx.x & 31;
    for (uint32_t b0 = a; b0 < b; b0 += BLEND_BATCH) {
        if (__syncthreads_count(done ? 1 : 0) == SPLIT_NT) break;
        const int cnt = (int)min((uint32_t)BLEND_BATCH, b - b0);
        for (int i = threadIdx.x; i < cnt; i += SPLIT_NT) {
            const uint32_t sl = pvals[b0 + i];
            s_xy[i] = xy[sl];
            s_co[i] = conic_o[sl];
        }
        __syncthreads();
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const int il = c0 + lane;
            uint32_t m = __ballot_sync(0xffffffffu, il < cnt && warp_hits(s_xy[il], s_co[il], P.X0, P.X1, P.Y0, P.Y1));
            while (m) {
                const int i = c0 + __ffs(m) - 1;
                m &= m - 1;
                const float4 g = s_xy[i];
                const float4 co = s_co[i];
                const float dx = __fsub_rn(g.x, P.fpx), dy = __fsub_rn(g.y, P.fpy);
                const float p2 = gauss_p2(co.x, co.y, co.z, dx, dy);
                const float q = __fsub_rn(p2, co.w);
                const bool live = !done && !(p2 > 0.f) && !(q < 0.f);
                const float alpha = live ? fminf(cs.alpha_max, __fmul_rn(cs.alpha_min, fast_exp2(q))) : 0.f;
                T = __fmul_rn(T, __fsub_rn(1.f, alpha));
                done = done || T < cs.t_min;
            }
        }
    }
    segf[sf_idx(item, 0, P.pid)] = T;
}

// pass 2: the exact walk of segment s from T_in(s).  Writes the segment's
// sums (C rgb, D, S with absolute T), its final T, its last contributor
// (list position + 1 from the tile's list start, 0 = none), its blended
// count, where the pixel stopped (SPLIT_NONE = not here) and whether the
// pixel composited this segment at all.
template <bool HITS>
__global__ void __launch_bounds__(SPLIT_NT) split_walk_kernel(const __grid_constant__ Views V, Consts cs, int S,
                                                              const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ pvals,
                                                              const float4* __restrict__ xy,
                                                              const float4* __restrict__ conic_o,
                                                              const float4* __restrict__ rgbd,
                                                              float* __restrict__ segf, uint32_t* __restrict__ segu) {
    __shared__ float4 s_xy[BLEND_BATCH];
    __shared__ float4 s_co[BLEND_BATCH];
    __shared__ float4 s_cd[BLEND_BATCH];
    __shared__ uint32_t s_gid[HITS ? BLEND_BATCH : 1];
    const uint32_t item = blockIdx.x;
    const int gt = (int)(item / (uint32_t)S), s = (int)(item % (uint32_t)S);
    const int v = view_of_tile(V, gt);
    const ViewInfo& vi = V.v[v];
    const SplitPixel P = split_pixel(vi, gt - vi.tile_base);
    bool out = !P.inside;
    if (!out && cs.pix_mask) out = cs.pix_mask[vi.pix_base + (int64_t)P.py * vi.W + P.px] == 0;
    // transmittance in front of this segment, from the earlier segments' products
    float T = 1.f;
    const uint32_t item0 = (uint32_t)gt * (uint32_t)S;
    for (int s2 = 0; s2 < s; ++s2) T = __fmul_rn(T, segf[sf_idx(item0 + s2, 0, P.pid)]);
    const bool ran = !out && !(T < cs.t_min);
    bool done = !ran;
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    uint32_t last = 0, nb = 0, stop_at = SPLIT_NONE;
    const uint2 rg = ranges[gt];
    uint32_t a, b;
    segment_of(rg, s, S, a, b);
    const int lane = threadIdx.x & 31;
    for (uint32_t b0 = a; b0 < b; b0 += BLEND_BATCH) {
        if (__syncthreads_count(done ? 1 : 0) == SPLIT_NT) break;
        const int cnt = (int)min((uint32_t)BLEND_BATCH, b - b0);
        for (int i = threadIdx.x; i < cnt; i += SPLIT_NT) {
            const uint32_t sl = pvals[b0 + i];
            s_xy[i] = xy[sl];
            s_co[i] = conic_o[sl];
            s_cd[i] = rgbd[sl];
            if (HITS) s_gid[i] = (uint32_t)(sl % (uint64_t)cs.n_gauss);
        }
        __syncthreads();
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const int il = c0 + lane;
            uint32_t m = __ballot_sync(0xffffffffu, il < cnt && warp_hits(s_xy[il], s_co[il], P.X0, P.X1, P.Y0, P.Y1));
            while (m) {
                const int i = c0 + __ffs(m) - 1;
                m &= m - 1;
                const float4 g = s_xy[i];
                const float4 co = s_co[i];
                const float4 cd = s_cd[i];
                const float dx = __fsub_rn(g.x, P.fpx), dy = __fsub_rn(g.y, P.fpy);
                const float p2 = gauss_p2(co.x, co.y, co.z, dx, dy);
                const float q = __fsub_rn(p2, co.w);
                const bool live = !done && !(p2 > 0.f) && !(q < 0.f);
                const float alpha = live ? fminf(cs.alpha_max, __fmul_rn(cs.alpha_min, fast_exp2(q))) : 0.f;
                const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
                const bool stop = live && Tn < cs.t_min;
                const bool blend = live && !stop;
                const uint32_t pos = b0 - rg.x + (uint32_t)i;
                stop_at = stop ? pos : stop_at;
                done = done || stop;
                const float w = blend ? alpha * T : 0.f;
                acc[0] = fmaf(cd.x, w, acc[0]);
                acc[1] = fmaf(cd.y, w, acc[1]);
                acc[2] = fmaf(cd.z, w, acc[2]);
                acc[3] = fmaf(cd.w, w, acc[3]);
                acc[4] += w;
                T = blend ? Tn : T;
                last = blend ? pos + 1 : last;
                nb += blend ? 1u : 0u;
                if (HITS) {
                    const uint32_t tot = __reduce_add_sync(0xffffffffu, blend ? 1u : 0u);
                    if (lane == 0 && tot) atomicAdd(cs.hit_count + s_gid[i], tot);
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) segf[sf_idx(item, 1 + c, P.pid)] = acc[c];
    segf[sf_idx(item, 6, P.pid)] = T;
    segu[su_idx(item, 0, P.pid)] = last;
    segu[su_idx(item, 1, P.pid)] = nb;
    segu[su_idx(item, 2, P.pid)] = stop_at;
    segu[su_idx(item, 3, P.pid)] = ran ? 1u : 0u;
}

// pass 3: per pixel, the segments in order.  Writes what the per-tile
// forward writes (images, T_final, last contributor, counters, the fused
// loss gradient).
template <bool COUNT>
__global__ void __launch_bounds__(SPLIT_NT) split_combine_kernel(const __grid_constant__ Views V, Consts cs, int S,
                                                                 const uint2* __restrict__ ranges,
                                                                 const float* __restrict__ segf,
                                                                 const uint32_t* __restrict__ segu,
                                                                 float* __restrict__ C, float* __restrict__ D,
                                                                 float* __restrict__ Sout, float* __restrict__ Tfin,
                                                                 uint32_t* __restrict__ ncontrib,
                                                                 unsigned long long* evals,
                                                                 unsigned long long* blended,
                                                                 uint32_t* __restrict__ neval) {
    const int gt = (int)blockIdx.x;
    const int v = view_of_tile(V, gt);
    const ViewInfo& vi = V.v[v];
    const SplitPixel P = split_pixel(vi, gt - vi.tile_base);
    const uint2 rg = ranges[gt];
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float T = 1.f;
    uint32_t last = 0, nb = 0, stop_at = SPLIT_NONE;
    bool any = false, stopped = false;
    const uint32_t item0 = (uint32_t)gt * (uint32_t)S;
    // four segments' fields loaded together, then taken in order
    constexpr int G = 4;
    for (int s0 = 0; s0 < S; s0 += G) {
        float f[G][6];
        uint32_t u[G][4];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const uint32_t it = item0 + (uint32_t)min(s0 + j, S - 1);
#pragma unroll
            for (int c = 0; c < 6; ++c) f[j][c] = segf[sf_idx(it, 1 + c, P.pid)];
#pragma unroll
            for (int c = 0; c < 4; ++c) u[j][c] = segu[su_idx(it, c, P.pid)];
        }
#pragma unroll
        for (int j = 0; j < G; ++j) {
            // skipped: past S, stopped in an earlier segment (a later segment
            // that still saw T_in >= t_min, its product rounded the other
            // way, is not composited), or left out
            if (s0 + j >= S || stopped || !u[j][3]) continue;
            any = true;
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[c] += f[j][c];
            T = f[j][5];
            last = max(last, u[j][0]);
            nb += u[j][1];
            stop_at = u[j][2];
            stopped = stop_at != SPLIT_NONE;
        }
    }
    const int64_t HW = (int64_t)vi.W * vi.H;
    float lsum = 0.f;
    uint32_t ev = 0, bl = 0;
    if (P.inside) {
        const int64_t i = (int64_t)P.py * vi.W + P.px;
        const int64_t pb = vi.pix_base;
        C[3 * pb + i] = acc[0];
        C[3 * pb + HW + i] = acc[1];
        C[3 * pb + 2 * HW + i] = acc[2];
        D[pb + i] = acc[3];
        Sout[pb + i] = acc[4];
        Tfin[pb + i] = T;
        ncontrib[pb + i] = last;
        if (cs.lf_on) {
            const float nv = (float)cs.lf_counts[0];
            const float nsamp = cs.pix_mask ? (float)cs.lf_counts[1] : (float)cs.lf_pixels;
            const float inv_c = nsamp > 0.f ? 1.f / (3.f * nsamp) : 0.f;
            const float inv_d = nv > 0.f ? cs.lf_wdepth / nv : 0.f;
            const bool smp = cs.pix_mask ? cs.pix_mask[pb + i] != 0 : true;
            float g0, g1, g2, gd;
            lsum = loss_pixel(acc[0], acc[1], acc[2], __ldg(cs.lf_Ct + 3 * pb + i), __ldg(cs.lf_Ct + 3 * pb + HW + i),
                              __ldg(cs.lf_Ct + 3 * pb + 2 * HW + i), acc[3], __ldg(cs.lf_Dt + pb + i), acc[4],
                              cs.lf_gate, inv_c, inv_d, g0, g1, g2, gd, smp);
            cs.lf_dC[3 * pb + i] = g0;
            cs.lf_dC[3 * pb + HW + i] = g1;
            cs.lf_dC[3 * pb + 2 * HW + i] = g2;
            cs.lf_dD[pb + i] = gd;
            if (cs.lf_dS) cs.lf_dS[pb + i] = 0.f;
        }
        // examined list entries: up to and including the stopping one (none
        // for a pixel left out)
        ev = !any ? 0u : (stop_at == SPLIT_NONE ? rg.y - rg.x : stop_at + 1);
        bl = nb;
        if (COUNT && neval) neval[pb + i] = ev;
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
        __shared__ float s_red[SPLIT_NT / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = lsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
#pragma unroll
            for (int w = 0; w < SPLIT_NT / 32; ++w) t += s_red[w];
            atomicAdd(cs.lf_loss, t);
        }
    }
}

// backward of segment s: the pixel's list positions [a, min(last, b)) back
// to front from T_out(s), with B started at g . (C, D, S) of the later
// segments the pixel composited; the per-Gaussian partials go through the
// same transposing warp reduction and atomics as the per-tile backward
__global__ void __launch_bounds__(SPLIT_NT) split_bwd_kernel(
    const __grid_constant__ Views V, Consts cs, int S, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ pvals, const float4* __restrict__ xy, const float4* __restrict__ conic_o,
    const float4* __restrict__ rgbd, const float* __restrict__ segf, const uint32_t* __restrict__ segu,
    const uint32_t* __restrict__ ncontrib, const float* __restrict__ dC, const float* __restrict__ dD,
    const float* __restrict__ dS, float* __restrict__ g2d, unsigned long long* bwd_pairs, int count) {
    __shared__ float4 s_xy[BLEND_BATCH];
    __shared__ float4 s_co[BLEND_BATCH];
    __shared__ float4 s_nat[BLEND_BATCH];
    __shared__ float4 s_cd[BLEND_BATCH];
    __shared__ uint32_t s_slot[BLEND_BATCH];
    __shared__ uint32_t s_max;
    const uint32_t item = blockIdx.x;
    const int gt = (int)(item / (uint32_t)S), s = (int)(item % (uint32_t)S);
    const int v = view_of_tile(V, gt);
    const ViewInfo& vi = V.v[v];
    const SplitPixel P = split_pixel(vi, gt - vi.tile_base);
    const int64_t HW = (int64_t)vi.W * vi.H, pb = vi.pix_base;
    const uint2 rg = ranges[gt];
    uint32_t a, b;
    segment_of(rg, s, S, a, b);
    const uint32_t item0 = (uint32_t)gt * (uint32_t)S;
    // this pixel's part of the segment: [a, a + nc) in list positions
    uint32_t nc = 0;
    float T = 1.f, Bk = 0.f, gp[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (P.inside) {
        const int64_t i = (int64_t)P.py * vi.W + P.px;
        const uint32_t last = ncontrib[pb + i];  // position + 1 from rg.x
        const uint32_t lo = a - rg.x, hi = min(last, b - rg.x);
        nc = (hi > lo && segu[su_idx(item, 3, P.pid)]) ? hi - lo : 0u;
        T = segf[sf_idx(item, 6, P.pid)];
        gp[0] = dC ? dC[3 * pb + i] : 0.f;
        gp[1] = dC ? dC[3 * pb + HW + i] : 0.f;
        gp[2] = dC ? dC[3 * pb + 2 * HW + i] : 0.f;
        gp[3] = dD ? dD[pb + i] : 0.f;
        gp[4] = dS ? dS[pb + i] : 0.f;
        if (nc) {  // the later segments' blended sums, weighted by the upstream gradient
            for (int s2 = s + 1; s2 < S; ++s2) {
                const uint32_t it = item0 + (uint32_t)s2;
                if (!segu[su_idx(it, 3, P.pid)]) break;  // the pixel stopped before it
#pragma unroll
                for (int c = 0; c < 5; ++c) Bk = fmaf(gp[c], segf[sf_idx(it, 1 + c, P.pid)], Bk);
                if (segu[su_idx(it, 2, P.pid)] != SPLIT_NONE) break;  // ... or in it (as the combine reads them)
            }
        }
    }
    if (count) {
        uint32_t walked = nc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) walked += __shfl_xor_sync(0xffffffffu, walked, o);
        if ((threadIdx.x & 31) == 0 && walked) atomicAdd(bwd_pairs, (unsigned long long)walked);
    }
    uint32_t mymax = nc;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, mymax);
    __syncthreads();
    const uint32_t end = a + min(s_max, b - a);
    const uint32_t warp_max = mymax;
    const int red_idx = reduce10_index(threadIdx.x & 31);
    const float red_scale = (red_idx == 2 || red_idx == 4) ? -0.5f : (red_idx >= 0 && red_idx <= 3) ? -1.f : 1.f;
    const int lane = threadIdx.x & 31;
    for (uint32_t bend = end; bend > a;) {
        const uint32_t bstart = (bend - a > (uint32_t)BLEND_BATCH) ? bend - BLEND_BATCH : a;
        __syncthreads();
        for (int i = threadIdx.x; i < (int)(bend - bstart); i += SPLIT_NT) {
            const uint32_t sl = pvals[bstart + i];
            s_slot[i] = sl;
            s_xy[i] = xy[sl];
            const float4 co = conic_o[sl];
            s_co[i] = co;
            // natural-unit conic and 1/opacity: a = -2 ln2 A2, b = -ln2 B2,
            // c = -2 ln2 C2, 1/o = 2^thr / alpha_min
            s_nat[i] = make_float4(-2.f * LN2 * co.x, -LN2 * co.y, -2.f * LN2 * co.z, fast_exp2(co.w) / cs.alpha_min);
            s_cd[i] = rgbd[sl];
        }
        __syncthreads();
        for (int c1 = (int)(bend - bstart); c1 > 0; c1 -= 32) {
            const int c0 = c1 > 32 ? c1 - 32 : 0;
            const int il = c0 + lane;
            const bool hit = il < c1 && (bstart - a + (uint32_t)il) < warp_max &&
                             warp_hits(s_xy[il], s_co[il], P.X0, P.X1, P.Y0, P.Y1);
            uint32_t m = __ballot_sync(0xffffffffu, hit);
            while (m) {
                const int hb = 31 - __clz(m);
                m &= ~(1u << hb);
                const int i = c0 + hb;
                const uint32_t jl = bstart - a + (uint32_t)i;
                const float4 g = s_xy[i];
                const float4 co = s_co[i];
                const float4 nat = s_nat[i];
                const float4 cd = s_cd[i];
                float vals[10];
#pragma unroll
                for (int c = 0; c < 10; ++c) vals[c] = 0.f;
                const float dx = __fsub_rn(g.x, P.fpx), dy = __fsub_rn(g.y, P.fpy);
                const float p2 = gauss_p2(co.x, co.y, co.z, dx, dy);
                const float q = __fsub_rn(p2, co.w);
                const bool live = jl < nc && !(p2 > 0.f) && !(q < 0.f);
                const float e2 = fast_exp2(q);
                const float x = live ? __fmul_rn(cs.alpha_min, e2) : 0.f;
                const float alpha = fminf(cs.alpha_max, x);
                const float inv = __fdividef(1.f, 1.f - alpha);
                T = live ? T * inv : T;
                const float w = gp[0] * cd.x + gp[1] * cd.y + gp[2] * cd.z + gp[3] * cd.w + gp[4];
                const float dA = T * w - Bk * inv;
                const float wt = alpha * T;
                Bk = fmaf(w, wt, Bk);
                vals[6] = wt * gp[0];
                vals[7] = wt * gp[1];
                vals[8] = wt * gp[2];
                vals[9] = wt * gp[3];
                const float xu = x <= cs.alpha_max ? x : 0.f;  // (uncapped, x is alpha)
                const float dp = xu * dA;
                const float pdx = dp * dx, pdy = dp * dy;
                vals[5] = dp;
                vals[0] = fmaf(nat.x, pdx, nat.y * pdy);
                vals[1] = fmaf(nat.y, pdx, nat.z * pdy);
                vals[2] = pdx * dx;
                vals[3] = pdx * dy;
                vals[4] = pdy * dy;
                if (__any_sync(0xffffffffu, live)) {
                    const float sum = warp_reduce10(vals);
                    if (red_idx >= 0)
                        atomicAdd(g2d + (int64_t)s_slot[i] * G2D_STRIDE + red_idx,
                                  sum * (red_idx == 5 ? nat.w : red_scale));
                }
            }
        }
        bend = bstart;
    }
}

cudaError_t launch_split_fwd(const Views& V, const Consts& cs, int S, const uint2* ranges, uint32_t* pvals,
                             const uint32_t* dkey, uint32_t* err, const float4* xy, const float4* conic_o,
                             const float4* rgbd, float* segf, uint32_t* segu, float* C, float* D, float* Sout,
                             float* Tfin, uint32_t* ncontrib, unsigned long long* evals, unsigned long long* blended,
                             uint32_t* neval, int count_evals, cudaStream_t st) {
    if (V.total_tiles <= 0) return cudaSuccess;
    const unsigned tiles = (unsigned)V.total_tiles, items = tiles * (unsigned)S;
    if (dkey) {  // per-tile form: order each list first
        count_launches(1);
        split_sort_kernel<<<tiles, SPLIT_NT, 0, st>>>(cs, ranges, pvals, dkey, err);
    }
    count_launches(3);
    split_prod_kernel<<<items, SPLIT_NT, 0, st>>>(V, cs, S, ranges, pvals, xy, conic_o, segf);
    if (cs.hit_count)
        split_walk_kernel<true><<<items, SPLIT_NT, 0, st>>>(V, cs, S, ranges, pvals, xy, conic_o, rgbd, segf, segu);
    else
        split_walk_kernel<false><<<items, SPLIT_NT, 0, st>>>(V, cs, S, ranges, pvals, xy, conic_o, rgbd, segf, segu);
    if (count_evals)
        split_combine_kernel<true><<<tiles, SPLIT_NT, 0, st>>>(V, cs, S, ranges, segf, segu, C, D, Sout, Tfin,
                                                               ncontrib, evals, blended, neval);
    else
        split_combine_kernel<false><<<tiles, SPLIT_NT, 0, st>>>(V, cs, S, ranges, segf, segu, C, D, Sout, Tfin,
                                                                ncontrib, evals, blended, neval);
    return cudaGetLastError();
}

cudaError_t launch_split_bwd(const Views& V, const Consts& cs, int S, const uint2* ranges, const uint32_t* pvals,
                             const float4* xy, const float4* conic_o, const float4* rgbd, const float* segf,
                             const uint32_t* segu, const uint32_t* ncontrib, const float* dC, const float* dD,
                             const float* dS, float* g2d, unsigned long long* bwd_pairs, int count, cudaStream_t st) {
    if (V.total_tiles <= 0) return cudaSuccess;
    count_launches(1);
    split_bwd_kernel<<<(unsigned)V.total_tiles * (unsigned)S, SPLIT_NT, 0, st>>>(
        V, cs, S, ranges, pvals, xy, conic_o, rgbd, segf, segu, ncontrib, dC, dD, dS, g2d, bwd_pairs, count);
    return cudaGetLastError();
}

}  // namespace vgk
