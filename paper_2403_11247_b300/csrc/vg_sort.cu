// vg_sort.cu -- tile binning: an in-house onesweep LSD radix sort (one kernel
// per 8-bit digit, decoupled look-back across partitions, digit histograms
// computed up front by the producer kernels), the fused scan + duplicate
// kernel that emits (tile, Gaussian) pairs in depth order, and per-tile ranges.
//
// Order produced: every tile's list ascending by (FP32 depth bits, slot
// index).  The depth sort is a stable sort of slot ids by depth key (ties keep
// slot order); pairs are then emitted in that order and stably sorted by tile
// key, so within a tile the depth order survives.
//
// Look-back entries are 64-bit: [epoch:32][flag:2][count:30].  The epoch comes
// from device memory (bumped once per forward), so entries left by earlier
// sorts never look ready and no memset of the look-back arrays is needed.
// Every wait on another partition is bounded (spin_limit unsuccessful polls);
// on timeout the kernel sets ERR_WAIT and carries on with the prefix it has
// (too small: every position it writes stays inside the output).
#include "vg_internal.h"

namespace vgk {

constexpr unsigned long long LB_AGG = 1ull << 30;
constexpr unsigned long long LB_INC = 2ull << 30;
constexpr unsigned long long LB_COUNT = (1ull << 30) - 1;

__device__ __forceinline__ unsigned long long lb_make(uint32_t epoch, unsigned long long flag, uint32_t count) {
    return ((unsigned long long)epoch << 32) | flag | (unsigned long long)count;
}

// Walk back from partition pid-1, summing counts until an inclusive prefix.
// Eight predecessors are read per round (independent loads in flight), so a
// chain of P partitions costs about P/8 L2 round trips instead of P.
constexpr int LB_WINDOW = 8;

__device__ __forceinline__ uint32_t lookback_walk(const unsigned long long* lb, int stride, int col, uint32_t pid,
                                                  uint32_t epoch, uint32_t* err, uint32_t spin_limit) {
    uint32_t excl = 0;
    int64_t j = (int64_t)pid - 1;
    uint32_t spins = 0;
    while (j >= 0) {
        unsigned long long w[LB_WINDOW];
#pragma unroll
        for (int u = 0; u < LB_WINDOW; ++u) w[u] = (j - u >= 0) ? ld_volatile64(lb + (j - u) * stride + col) : 0ull;
        int u = 0;
        bool stop = false;
        for (; u < LB_WINDOW && j - u >= 0; ++u) {
            const unsigned long long s = w[u];
            if ((uint32_t)(s >> 32) != epoch || (s & (LB_AGG | LB_INC)) == 0) break;  // not ready: re-read from here
            excl += (uint32_t)(s & LB_COUNT);
            if (s & LB_INC) {
                stop = true;
                break;
            }
        }
        if (stop) break;
        if (u == 0 && ++spins > spin_limit) {
            atomicOr(err, ERR_WAIT);
            break;
        }
        j -= u;
    }
    return excl;
}

// add 1 to bin b of a shared histogram; lanes of a warp adding to the same bin
// are combined first (one atomic per distinct bin)
__device__ __forceinline__ void hist_add_warp(uint32_t* h, uint32_t b, uint32_t active) {
    const uint32_t peers = __match_any_sync(active, b);
    if ((threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) red_add_shared(h + b, (uint32_t)__popc(peers));
}

__global__ void __launch_bounds__(SORT_THREADS) onesweep_pass_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const uint32_t* n_dev, uint32_t n_cap, int shift, const uint32_t* __restrict__ hist,
    unsigned long long* lookback, uint32_t* counter, const uint32_t* state, uint32_t epoch_offset, uint32_t* err,
    uint32_t spin_limit) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_whist[8][256];
    __shared__ uint32_t s_bpre[256];
    __shared__ uint32_t s_gout[256];
    __shared__ uint32_t s_keys[SORT_TILE];
    __shared__ uint32_t s_vals[SORT_TILE];
    __shared__ uint32_t s_tmp[8];
    __shared__ uint32_t s_pid;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = n_dev ? min(*n_dev, n_cap) : n_cap;
    const uint32_t nparts = (n + SORT_TILE - 1) / SORT_TILE;
    const uint32_t epoch = state[ST_EPOCH] + epoch_offset;
    uint32_t tot;
    s_base[tid] = block_excl_scan_256(hist[tid], s_tmp, &tot);
    const uint32_t lt = lanemask_lt();

    for (;;) {
        if (tid == 0) s_pid = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t pid = s_pid;
        if (pid >= nparts) break;
        for (int i = lane; i < 256; i += 32) s_whist[warp][i] = 0;
        __syncwarp();
        const uint32_t base = pid * SORT_TILE + warp * (32 * SORT_ITEMS);
        uint32_t key[SORT_ITEMS], val[SORT_ITEMS], rank[SORT_ITEMS];
#pragma unroll
        for (int i = 0; i < SORT_ITEMS; ++i) {
            const uint32_t idx = base + i * 32 + lane;
            const bool valid = idx < n;
            key[i] = valid ? keys_in[idx] : 0u;
            val[i] = valid ? (vals_in ? vals_in[idx] : idx) : 0u;
            const uint32_t d = valid ? ((key[i] >> shift) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const int leader = __ffs(peers) - 1;
            uint32_t cnt = 0;
            if (valid && lane == leader) {
                cnt = s_whist[warp][d];
                s_whist[warp][d] = cnt + __popc(peers);
            }
            cnt = __shfl_sync(0xffffffffu, cnt, leader);
            rank[i] = cnt + __popc(peers & lt);
            __syncwarp();
        }
        __syncthreads();
        // per digit (thread = digit): warp-exclusive prefix and partition total
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            uint32_t c = s_whist[w][tid];
            s_whist[w][tid] = total;
            total += c;
        }
        unsigned long long* lb = lookback;
        st_volatile64(lb + (int64_t)pid * 256 + tid, lb_make(epoch, pid == 0 ? LB_INC : LB_AGG, total));
        uint32_t btot;
        s_bpre[tid] = block_excl_scan_256(total, s_tmp, &btot);
        uint32_t excl = 0;
        if (pid > 0) {
            excl = lookback_walk(lb, 256, tid, pid, epoch, err, spin_limit);
            st_volatile64(lb + (int64_t)pid * 256 + tid, lb_make(epoch, LB_INC, excl + total));
        }
        s_gout[tid] = s_base[tid] + excl;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < SORT_ITEMS; ++i) {
            const uint32_t idx = base + i * 32 + lane;
            if (idx < n) {
                const uint32_t d = (key[i] >> shift) & 255u;
                const uint32_t pos = s_bpre[d] + s_whist[warp][d] + rank[i];
                s_keys[pos] = key[i];
                s_vals[pos] = val[i];
            }
        }
        __syncthreads();
        const uint32_t nvalid = min((uint32_t)SORT_TILE, n - pid * SORT_TILE);
        for (uint32_t j = tid; j < nvalid; j += SORT_THREADS) {
            const uint32_t k = s_keys[j];
            const uint32_t d = (k >> shift) & 255u;
            const uint32_t g = s_gout[d] + (j - s_bpre[d]);
            keys_out[g] = k;
            vals_out[g] = s_vals[j];
        }
        __syncthreads();
    }
}

int sort_pass_grid(uint32_t n_cap) {
    static int max_grid = 0;
    if (!max_grid) {
        int dev = 0, sms = 148, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, onesweep_pass_kernel, SORT_THREADS, 0);
        max_grid = sms * (per > 0 ? per : 1);
    }
    int64_t parts = ceil_div((int64_t)n_cap, SORT_TILE);
    if (parts < 1) parts = 1;
    return (int)(parts < max_grid ? parts : max_grid);
}

cudaError_t launch_sort_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                             const uint32_t* n_dev, uint32_t n_cap, int shift, const uint32_t* hist,
                             unsigned long long* lookback, uint32_t* counter, const uint32_t* state,
                             uint32_t epoch_offset, uint32_t* err, int grid, uint32_t spin_limit, cudaStream_t st) {
    count_launches(1);
    onesweep_pass_kernel<<<grid, SORT_THREADS, 0, st>>>(keys_in, vals_in, keys_out, vals_out, n_dev, n_cap, shift, hist,
                                                        lookback, counter, state, epoch_offset, err, spin_limit);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// pair offsets: exclusive scan of the tile counts of the depth-sorted visible
// slots, reduce then scan (no waits between blocks): block b first totals
// partition b's DUP_TILE tile counts, then, in a second launch, sums the
// totals of the partitions in front of it (a few thousand words from L2)
// and scans its own.  Blocks past the visible slots (the grid is sized for
// every slot) return at once.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(DUP_THREADS) pair_totals_kernel(const uint32_t* __restrict__ sorted_slots,
                                                                 const uint32_t* __restrict__ ntiles,
                                                                 const uint32_t* __restrict__ scratch,
                                                                 uint32_t* __restrict__ part_total) {
    __shared__ uint32_t s_tmp[8];
    const uint32_t nvis = scratch[SCR_NVIS];
    const uint32_t base = blockIdx.x * DUP_TILE + threadIdx.x * DUP_ITEMS;
    if (blockIdx.x * DUP_TILE >= nvis) return;
    uint32_t local = 0;
#pragma unroll
    for (int i = 0; i < DUP_ITEMS; ++i)
        if (base + i < nvis) local += ntiles[sorted_slots[base + i]];
    uint32_t agg;
    block_excl_scan_256(local, s_tmp, &agg);
    if (threadIdx.x == 0) part_total[blockIdx.x] = agg;
}

__global__ void __launch_bounds__(DUP_THREADS) pair_offsets_kernel(
    const uint32_t* __restrict__ sorted_slots, const uint32_t* __restrict__ ntiles, uint32_t* __restrict__ offsets,
    uint32_t* __restrict__ chunk_start, uint32_t cap, uint32_t* scratch, const uint32_t* __restrict__ part_total,
    uint32_t* err) {
    __shared__ uint32_t s_tmp[8];
    const int tid = threadIdx.x;
    const uint32_t nvis = scratch[SCR_NVIS];
    const uint32_t pid = blockIdx.x, nparts = (nvis + DUP_TILE - 1) / DUP_TILE;
    if (pid >= nparts) return;
    uint32_t excl_part = 0;  // the partitions in front of this one
    for (uint32_t j = tid; j < pid; j += DUP_THREADS) excl_part += part_total[j];
    uint32_t excl;
    block_excl_scan_256(excl_part, s_tmp, &excl);
    uint32_t cnt[DUP_ITEMS];
    uint32_t local = 0;
    const uint32_t base = pid * DUP_TILE + tid * DUP_ITEMS;
#pragma unroll
    for (int i = 0; i < DUP_ITEMS; ++i) {
        const uint32_t pos = base + i;
        cnt[i] = pos < nvis ? ntiles[sorted_slots[pos]] : 0u;
        local += cnt[i];
    }
    uint32_t agg;
    const uint32_t pre = block_excl_scan_256(local, s_tmp, &agg);
    if (tid == 0 && pid == nparts - 1) {
        scratch[SCR_PAIRS] = excl + agg;
        offsets[nvis] = excl + agg;
        if (excl + agg > cap) atomicOr(err, ERR_OVERFLOW);
    }
    uint32_t off = excl + pre;
#pragma unroll
    for (int i = 0; i < DUP_ITEMS; ++i) {
        if (base + i < nvis) {
            offsets[base + i] = off;
            mark_chunks(chunk_start, base + i, off, cnt[i], cap);
        }
        off += cnt[i];
    }
}

// ---------------------------------------------------------------------------
// pair emission: one thread per (Gaussian, tile) pair, balanced however the
// tiles are spread over Gaussians (a Gaussian close to the camera can cover
// thousands of tiles).  A block takes EMIT_R consecutive chunks of
// EMIT_CHUNK pairs at a time; chunk_start names the slot position j0 the
// first pair belongs to.  Every visible slot owns at least one pair, so
// positions j0 .. j0 + EMIT_R * EMIT_CHUNK cover the block's pairs: each
// marks where its pairs start, and an inclusive max-scan over the pairs
// hands every pair its slot (the owner index only grows along the pairs).
// Thread t handles pair t of each chunk, so that a warp still emits 32
// consecutive pairs at a time, and the chain of dependent loads (chunk
// start, slot offsets, slot rect) is paid once per EMIT_R chunks.  Tiles in
// row-major order of the rect.
// ---------------------------------------------------------------------------
constexpr int EMIT_R = 4;
constexpr int EMIT_SPAN = EMIT_R * EMIT_CHUNK;

__global__ void __launch_bounds__(EMIT_CHUNK) emit_pairs_kernel(
    const uint32_t* __restrict__ sorted_slots, const uint32_t* __restrict__ offsets,
    const uint32_t* __restrict__ chunk_start, const uint2* __restrict__ rect, int64_t N,
    const __grid_constant__ Views V, uint32_t* __restrict__ pkeys, uint32_t* __restrict__ pvals, uint32_t cap,
    uint32_t* scratch, int tile_passes, int tiles_in_smem, uint2* __restrict__ ranges_zero) {
    __shared__ uint32_t s_hist[3 * 256];
    __shared__ uint32_t s_own[EMIT_SPAN];
    __shared__ uint32_t s_slot[EMIT_SPAN + 1], s_first[EMIT_SPAN + 1];
    __shared__ uint32_t s_wmax[EMIT_CHUNK / 32];
    extern __shared__ uint32_t s_tiles[];  // per-tile counts when the block's share of pairs pays for them
    for (int i = threadIdx.x; i < tile_passes * 256; i += blockDim.x) s_hist[i] = 0;
    if (tiles_in_smem)
        for (int i = threadIdx.x; i < V.total_tiles; i += blockDim.x) s_tiles[i] = 0;
    uint32_t* tile_counts = scratch + SCR_TILE_COUNTS;
    // global-sort form (ranges_zero): no per-tile counts here -- the ranges
    // come from the sorted keys later -- but their array starts at zero
    if (ranges_zero)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V.total_tiles; i += gridDim.x * blockDim.x)
            ranges_zero[i] = make_uint2(0u, 0u);
    const uint32_t nvis = scratch[SCR_NVIS];
    const uint32_t P = min(scratch[SCR_PAIRS], cap);
    const uint32_t stride = gridDim.x * EMIT_SPAN;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t e0 = blockIdx.x * EMIT_SPAN; e0 < P; e0 += stride) {
        const uint32_t e1 = min(e0 + (uint32_t)EMIT_SPAN, P);
#pragma unroll
        for (int r = 0; r < EMIT_R; ++r) s_own[r * EMIT_CHUNK + threadIdx.x] = 0u;
        __syncthreads();
        const uint32_t j0 = chunk_start[e0 / EMIT_CHUNK];
        for (uint32_t t = threadIdx.x; t <= (uint32_t)EMIT_SPAN; t += EMIT_CHUNK) {
            const uint32_t j = j0 + t;
            if (j < nvis) {
                const uint32_t o = __ldg(offsets + j), o1 = __ldg(offsets + j + 1);
                s_slot[t] = __ldg(sorted_slots + j);
                s_first[t] = o;
                if (o1 > e0 && o < e1) s_own[max(o, e0) - e0] = t;
            }
        }
        __syncthreads();
        // inclusive max-scan of s_own: a thread's EMIT_R consecutive entries,
        // then across the threads in front of it
        uint32_t loc[EMIT_R], run = 0u;
#pragma unroll
        for (int r = 0; r < EMIT_R; ++r) {
            run = max(run, s_own[threadIdx.x * EMIT_R + r]);
            loc[r] = run;
        }
        uint32_t inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = max(inc, y);
        }
        if (lane == 31) s_wmax[warp] = inc;
        uint32_t pre = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) pre = 0u;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < EMIT_CHUNK / 32; ++w)
            if (w < warp) pre = max(pre, s_wmax[w]);
#pragma unroll
        for (int r = 0; r < EMIT_R; ++r) s_own[threadIdx.x * EMIT_R + r] = max(pre, loc[r]);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < EMIT_R; ++r) {
            const uint32_t e = e0 + (uint32_t)(r * EMIT_CHUNK) + threadIdx.x;
            const bool live = e < e1;
            const uint32_t active = __ballot_sync(0xffffffffu, live);
            if (!live) continue;
            const uint32_t own = s_own[r * EMIT_CHUNK + threadIdx.x];
            if (j0 + own >= nvis) continue;  // (only offsets left wrong by a timed-out wait get here)
            const uint32_t s = s_slot[own];
            const uint32_t local = e - s_first[own];
            const uint2 rc = __ldg(rect + s);
            const uint32_t x0 = rc.x & 0xffff, y0 = rc.x >> 16, x1 = rc.y & 0xffff, y1 = rc.y >> 16;
            const uint32_t w = x1 - x0;
            // a pair past its slot's rect only comes of offsets left wrong by
            // a timed-out wait (ERR_WAIT is set): skipped, never an index
            // outside the tiles
            if (w == 0 || local >= w * (y1 - y0)) continue;
            const uint32_t ry = local / w, rx = local - ry * w;
            const int v = slot_view(s, (uint32_t)N, V.n);
            const uint32_t key = (uint32_t)(V.v[v].tile_base + (int)(y0 + ry) * V.v[v].tiles_x + (int)(x0 + rx));
            pkeys[e] = key;
            pvals[e] = s;
            // digit histograms of the tile passes: the low digit of a warp's
            // keys is mostly distinct (consecutive tiles of a rect row), so
            // each lane adds its own; higher digits mostly repeat in a warp
            // and are combined first
            if (tile_passes > 0) red_add_shared(s_hist + (key & 255u), 1u);
            for (int p = 1; p < tile_passes; ++p) hist_add_warp(s_hist + p * 256, (key >> (8 * p)) & 255u, active);
            if (!ranges_zero) {
                const uint32_t peers = __match_any_sync(active, key);
                if ((uint32_t)lane == (uint32_t)(__ffs(peers) - 1)) {
                    if (tiles_in_smem) red_add_shared(s_tiles + key, (uint32_t)__popc(peers));
                    else atomicAdd(tile_counts + key, (uint32_t)__popc(peers));
                }
            }
        }
        __syncthreads();  // s_own, s_slot, s_first are read before the next span reuses them
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tile_passes * 256; i += blockDim.x) {
        const uint32_t h = s_hist[i];
        if (h) atomicAdd(scratch + SCR_TILE_HIST + i, h);
    }
    if (tiles_in_smem)
        for (int i = threadIdx.x; i < V.total_tiles; i += blockDim.x) {
            const uint32_t h = s_tiles[i];
            if (h) atomicAdd(tile_counts + i, h);
        }
}

cudaError_t launch_duplicate(const uint32_t* sorted_slots, uint32_t* offsets, uint32_t* chunk_start,
                             bool offsets_ready, const uint32_t* ntiles, const uint2* rect,
                             int64_t N, const Views& V, uint32_t* pkeys, uint32_t* pvals, uint32_t cap,
                             uint32_t* scratch, int tile_passes, uint32_t* part_total, uint32_t* err,
                             int64_t max_slots, uint2* ranges, cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 148;
    }
    cudaError_t e;
    if (!offsets_ready) {
        const int64_t parts = ceil_div(max_slots > 0 ? max_slots : 1, DUP_TILE);
        count_launches(2);
        pair_totals_kernel<<<(unsigned)parts, DUP_THREADS, 0, st>>>(sorted_slots, ntiles, scratch, part_total);
        pair_offsets_kernel<<<(unsigned)parts, DUP_THREADS, 0, st>>>(sorted_slots, ntiles, offsets, chunk_start, cap,
                                                                    scratch, part_total, err);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    int64_t eg = ceil_div((int64_t)cap, EMIT_SPAN);
    if (eg > (int64_t)sms * 8) eg = (int64_t)sms * 8;
    if (eg < 1) eg = 1;
    // per-tile counts: a per-block histogram in shared memory pays for its
    // zeroing and flush only when a block emits at least as many pairs as
    // there are tiles; otherwise one global atomic per run of equal tiles
    const int64_t spans_per_block = ceil_div(ceil_div((int64_t)cap, EMIT_SPAN), eg);
    const int tiles_in_smem = !offsets_ready ? 0 : (V.total_tiles <= EMIT_SMEM_TILES &&
                              (int64_t)V.total_tiles <= spans_per_block * EMIT_SPAN ? 1 : 0);
    const size_t smem = tiles_in_smem ? (size_t)V.total_tiles * 4 : 0;
    e = allow_dynamic_smem((const void*)emit_pairs_kernel, smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    emit_pairs_kernel<<<(unsigned)eg, EMIT_CHUNK, smem, st>>>(sorted_slots, offsets, chunk_start, rect, N, V, pkeys,
                                                               pvals, cap, scratch, tile_passes, tiles_in_smem,
                                                               offsets_ready ? nullptr : ranges);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// tile ranges of the global-sort form, from the tile-sorted keys: a pair that
// starts a run of equal keys writes the run's start, the pair that ends it
// the end (empty tiles keep the zero the emission wrote)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tile_bounds_kernel(const uint32_t* __restrict__ keys,
                                                         const uint32_t* __restrict__ n_dev, uint32_t cap,
                                                         uint2* __restrict__ ranges) {
    const uint32_t P = min(*n_dev, cap);
    uint32_t* r = reinterpret_cast<uint32_t*>(ranges);
    // four keys per thread (one 16-byte load; the key arrays are 256-byte
    // aligned allocations) and their two neighbours
    const uint32_t q4 = (P + 3) / 4;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < q4; q += gridDim.x * blockDim.x) {
        const uint32_t e0 = 4 * q;
        uint32_t k[6];
        if (e0 + 4 <= P) {
            const uint4 v = reinterpret_cast<const uint4*>(keys)[q];
            k[1] = v.x; k[2] = v.y; k[3] = v.z; k[4] = v.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) k[1 + i] = e0 + i < P ? keys[e0 + i] : 0xffffffffu;
        }
        k[0] = e0 > 0 ? keys[e0 - 1] : 0xffffffffu;
        k[5] = e0 + 4 < P ? keys[e0 + 4] : 0xffffffffu;
#pragma unroll
        for (int i = 1; i <= 4; ++i) {
            const uint32_t e = e0 + (uint32_t)(i - 1);
            if (e >= P) break;
            if (e == 0 || k[i - 1] != k[i]) r[2 * k[i]] = e;
            if (e + 1 == P || k[i + 1] != k[i]) r[2 * k[i] + 1] = e + 1;
        }
    }
}

cudaError_t launch_tile_bounds(const uint32_t* keys, const uint32_t* n_dev, uint32_t cap, uint2* ranges,
                               cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 148;
    }
    int64_t g = ceil_div(ceil_div((int64_t)cap, 4), 256);
    if (g > (int64_t)sms * 16) g = (int64_t)sms * 16;
    if (g < 1) g = 1;
    count_launches(1);
    tile_bounds_kernel<<<(unsigned)g, 256, 0, st>>>(keys, n_dev, cap, ranges);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// per-tile [start, end): exclusive scan of the per-tile pair counts, and the
// order in which the compositing kernels take the tiles: longest lists first
// (256 buckets of list length, descending; any order within a bucket), so
// that the long tiles start early and the short ones fill in behind them
// instead of a cluster of long neighbouring tiles running last (one block)
// ---------------------------------------------------------------------------
constexpr int ORDER_BUCKETS = 256;
constexpr int RANGES_SMEM_TILES = 32768;  // counts staged in shared memory up to this many tiles (128 KB)

__device__ __forceinline__ int order_bucket(uint32_t c, uint32_t cmax) {
    // 0 for the longest lists, ORDER_BUCKETS - 1 for empty ones
    return ORDER_BUCKETS - 1 - (int)(((uint64_t)c * (ORDER_BUCKETS - 1)) / (cmax > 0 ? cmax : 1u));
}

// clear: (global-sort form, where this kernel is the last reader) zero the
// tile counts, the digit histograms and the pass counters afterwards, so the
// next forward starts from clean scratch without a memset
__global__ void __launch_bounds__(1024) ranges_kernel(uint32_t* __restrict__ cnt_g, int n,
                                                      uint2* __restrict__ ranges, uint32_t* __restrict__ order,
                                                      int staged, uint32_t* __restrict__ scratch, int clear,
                                                      const uint32_t* __restrict__ lf_blk, int lf_grid,
                                                      uint32_t* __restrict__ lf_counts,
                                                      uint32_t* __restrict__ long_tiles, int from_ranges) {
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_carry, s_max, s_nlong;
    __shared__ uint32_t s_lf[2];
    __shared__ uint32_t s_bin[ORDER_BUCKETS];
    extern __shared__ uint32_t s_cnt[];  // the counts, when they fit: one coalesced load for all three uses
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (from_ranges) {  // global-sort form: the ranges are final, the counts are their lengths
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const uint2 r = ranges[i];
            const uint32_t c = r.y > r.x ? r.y - r.x : 0u;
            if (staged) s_cnt[i] = c;
            else cnt_g[i] = c;
        }
        __syncthreads();
    } else if (staged) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) s_cnt[i] = cnt_g[i];
    }
    const uint32_t* cnt = staged ? s_cnt : cnt_g;
    if (threadIdx.x == 0) {
        s_carry = 0;
        s_max = 0;
    }
    if (threadIdx.x < 2) s_lf[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_nlong = 0;
    for (int i = threadIdx.x; i < ORDER_BUCKETS; i += blockDim.x) s_bin[i] = 0;
    __syncthreads();
    if (lf_blk) {  // the fused loss's normalisers from the compaction's per-block counts
        uint32_t c = 0, ns = 0;
        for (int i = threadIdx.x; i < lf_grid; i += blockDim.x) {
            c += lf_blk[i];
            ns += lf_blk[lf_grid + i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            ns += __shfl_xor_sync(0xffffffffu, ns, o);
        }
        if (lane == 0) {
            red_add_shared(&s_lf[0], c);
            red_add_shared(&s_lf[1], ns);
        }
    }
    uint32_t mymax = 0;
    for (int c0 = 0; c0 < n; c0 += 1024) {
        const int i = c0 + threadIdx.x;
        const uint32_t x = i < n ? cnt[i] : 0u;
        mymax = max(mymax, x);
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            s_w[lane] = t;
        }
        __syncthreads();
        const uint32_t start = s_carry + (warp ? s_w[warp - 1] : 0u) + inc - x;
        if (i < n && !from_ranges) ranges[i] = make_uint2(start, start + x);
        if (long_tiles && i < n && x > (uint32_t)VG_TILE_SORT_CAP) long_tiles[atomicAdd(&s_nlong, 1u)] = (uint32_t)i;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_w[31];
        __syncthreads();
    }
    if (lf_blk && threadIdx.x == 0) {  // (s_lf is complete: the scan's barriers came after its adds)
        lf_counts[0] = s_lf[0];
        lf_counts[1] = s_lf[1];
    }
    if (long_tiles && threadIdx.x == 0) scratch[SCR_N_LONG] = s_nlong;  // (complete: barriers since)
    if (!order) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if (lane == 0) atomicMax(&s_max, mymax);
    __syncthreads();
    const uint32_t cmax = s_max;
    for (int i = threadIdx.x; i < n; i += blockDim.x) red_add_shared(&s_bin[order_bucket(cnt[i], cmax)], 1u);
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the bucket sizes, 8 buckets per lane
        uint32_t v[ORDER_BUCKETS / 32], tot = 0;
#pragma unroll
        for (int k = 0; k < ORDER_BUCKETS / 32; ++k) {
            v[k] = s_bin[lane * (ORDER_BUCKETS / 32) + k];
            tot += v[k];
        }
        uint32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        uint32_t run = inc - tot;
#pragma unroll
        for (int k = 0; k < ORDER_BUCKETS / 32; ++k) {
            s_bin[lane * (ORDER_BUCKETS / 32) + k] = run;
            run += v[k];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) order[atomicAdd(&s_bin[order_bucket(cnt[i], cmax)], 1u)] = (uint32_t)i;
    if (clear) {
        __syncthreads();  // every count has been read
        for (int i = threadIdx.x; i < n; i += blockDim.x) cnt_g[i] = 0u;
        for (int i = threadIdx.x; i < SCR_NVIS; i += blockDim.x) scratch[i] = 0u;  // digit histograms
        for (int i = SCR_CNT_DEPTH + (int)threadIdx.x; i < SCR_CNT_TILE + 3; i += blockDim.x) scratch[i] = 0u;
    }
}

cudaError_t launch_ranges(uint32_t* scratch, int n_tiles, uint2* ranges, uint32_t* order, int clear,
                          const uint32_t* lf_blk, int lf_grid, uint32_t* lf_counts, uint32_t* long_tiles,
                          int from_ranges, cudaStream_t st) {
    count_launches(1);
    const int staged = n_tiles <= RANGES_SMEM_TILES ? 1 : 0;
    const size_t smem = staged ? (size_t)n_tiles * 4 : 0;
    cudaError_t e = allow_dynamic_smem((const void*)ranges_kernel, smem);
    if (e != cudaSuccess) return e;
    ranges_kernel<<<1, 1024, smem, st>>>(scratch + SCR_TILE_COUNTS, n_tiles, ranges, order, staged, scratch, clear,
                                         lf_blk, lf_grid, lf_counts, long_tiles, from_ranges);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// grouping by tile without order (per-tile sort): pair e goes to a free
// position of its tile's range, claimed by counting the tile's pair count
// down (one atomic per run of equal tiles in a warp); the forward compositing
// kernel then orders each tile's list, so the claim order does not matter
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tile_scatter_kernel(const uint32_t* __restrict__ keys_in,
                                                           const uint32_t* __restrict__ vals_in,
                                                           const uint32_t* __restrict__ n_dev, uint32_t cap,
                                                           const uint2* __restrict__ ranges, uint32_t* counts,
                                                           uint32_t* __restrict__ keys_out,
                                                           uint32_t* __restrict__ vals_out) {
    const uint32_t P = min(*n_dev, cap);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < P; e += gridDim.x * blockDim.x) {
        const uint32_t key = keys_in[e];
        const uint32_t peers = __match_any_sync(__activemask(), key);
        const int leader = __ffs(peers) - 1;
        const uint32_t n = (uint32_t)__popc(peers);
        uint32_t top = 0;
        if ((int)(threadIdx.x & 31) == leader) top = atomicSub(counts + key, n);
        top = __shfl_sync(peers, top, leader);
        const uint32_t pos = ranges[key].x + top - n + (uint32_t)__popc(peers & lanemask_lt());
        keys_out[pos] = key;
        vals_out[pos] = vals_in[e];
    }
}

cudaError_t launch_tile_scatter(const uint32_t* keys_in, const uint32_t* vals_in, const uint32_t* n_dev, uint32_t cap,
                                const uint2* ranges, uint32_t* counts, uint32_t* keys_out, uint32_t* vals_out,
                                cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 148;
    }
    int64_t grid = ceil_div((int64_t)cap, 256);
    if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
    if (grid < 1) grid = 1;
    count_launches(1);
    tile_scatter_kernel<<<(unsigned)grid, 256, 0, st>>>(keys_in, vals_in, n_dev, cap, ranges, counts, keys_out,
                                                       vals_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// per-tile ranges, the longest-first tile order and the grouping of the pairs
// by tile in one launch (per-tile sort without the long-list pass, up to
// PLACE_SMEM_TILES tiles).  Every CTA scans the per-tile pair counts itself (a
// few thousand words from L2) into a shared-memory copy of the tile starts.
// CTA 0 then writes the ranges, the order (longest lists first: 256 buckets
// of list length, descending, any order within a bucket) and the fused
// loss's normalisers; the other CTAs place the pairs: a pair claims a free
// position of its tile's range by counting the tile's fill counter up (one
// atomic per run of equal tiles in a warp, several pairs per thread in
// flight).  The last CTA out puts the counts, the fill counters and its exit
// counter back to zero for the next forward.  This replaces a one-CTA scan
// launch followed by a separate scatter launch.
// ---------------------------------------------------------------------------
constexpr int PLACE_THREADS = 512;
constexpr int PLACE_ITEMS = 4;
constexpr int PLACE_SMEM_TILES = 16384;

// length bucket of a tile list: 0 for the longest, ORDER_BUCKETS - 1 for
// empty ones
__device__ __forceinline__ int place_bucket(uint32_t c, float scale) {
    return ORDER_BUCKETS - 1 - min(ORDER_BUCKETS - 1, (int)((float)c * scale));
}

__global__ void __launch_bounds__(PLACE_THREADS) tile_place_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t cap, uint32_t* scratch,
    int n, uint2* __restrict__ ranges, uint32_t* __restrict__ order, const uint32_t* __restrict__ lf_blk, int lf_grid,
    uint32_t* __restrict__ lf_counts, uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out) {
    extern __shared__ uint32_t s_start[];  // [n + 1]: exclusive scan of the tile counts, the total last
    __shared__ uint32_t s_w[PLACE_THREADS / 32], s_w2[PLACE_THREADS / 32];
    __shared__ uint32_t s_bin[ORDER_BUCKETS];
    __shared__ uint32_t s_max, s_last;
    uint32_t* const cnt_g = scratch + SCR_TILE_COUNTS;
    uint32_t* const fill = cnt_g + n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool lead = blockIdx.x == 0;  // the CTA that writes ranges and order
    // a placing CTA loads and claims its first round of pairs before the
    // scan: the claims need only the fill counters, so their round trips
    // overlap the scan, and only the positions wait for the tile starts
    const uint32_t P = min(scratch[SCR_PAIRS], cap);
    const uint32_t lt = lanemask_lt();
    const uint32_t span = (uint32_t)PLACE_THREADS * PLACE_ITEMS;
    uint32_t key[PLACE_ITEMS], val[PLACE_ITEMS], peers[PLACE_ITEMS], old[PLACE_ITEMS];
    auto claim = [&](uint32_t base) {
#pragma unroll
        for (int k = 0; k < PLACE_ITEMS; ++k) {
            const uint32_t e = base + (uint32_t)(k * PLACE_THREADS + tid);
            key[k] = e < P ? keys_in[e] : 0xffffffffu;
            val[k] = e < P ? vals_in[e] : 0u;
        }
#pragma unroll
        for (int k = 0; k < PLACE_ITEMS; ++k) {
            peers[k] = __match_any_sync(0xffffffffu, key[k]);
            old[k] = 0u;
            if (key[k] < (uint32_t)n && lane == __ffs(peers[k]) - 1)
                old[k] = atomicAdd(fill + key[k], (uint32_t)__popc(peers[k]));
        }
    };
    uint32_t base = lead ? P : (blockIdx.x - 1) * span;
    if (base < P) claim(base);
    // (unrolled: the loads of a thread's counts go out together, not one L2
    // round trip each)
#pragma unroll 8
    for (int i = tid; i < n; i += PLACE_THREADS) s_start[i] = cnt_g[i];
    if (lead) {
        for (int i = tid; i < ORDER_BUCKETS; i += PLACE_THREADS) s_bin[i] = 0u;
        if (tid == 0) s_max = 0u;
    }
    __syncthreads();
    // each thread scans a contiguous stretch of the counts
    const int per = (n + PLACE_THREADS - 1) / PLACE_THREADS;
    const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
    uint32_t sum = 0u, mx = 0u;
    for (int i = i0; i < i1; ++i) {
        const uint32_t c = s_start[i];
        sum += c;
        mx = max(mx, c);
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[warp] = inc;
    if (lead) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(&s_max, mx);
    }
    __syncthreads();
    uint32_t run = inc - sum;
    for (int w = 0; w < warp; ++w) run += s_w[w];
    for (int i = i0; i < i1; ++i) {
        const uint32_t c = s_start[i];
        s_start[i] = run;
        run += c;
    }
    if (tid == PLACE_THREADS - 1) s_start[n] = run;  // (the last stretch ends at n)
    __syncthreads();

    if (lead) {
        const uint32_t cmax = s_max;
        const float scale = cmax > 0u ? (float)(ORDER_BUCKETS - 1) / (float)cmax : 0.f;
        // bucket sizes; the lanes of a warp that share a bucket add once
        // (a uniform loop: every lane takes part in the vote)
        for (int i0b = 0; i0b < n; i0b += PLACE_THREADS) {
            const int i = i0b + tid;
            const int b = i < n ? place_bucket(s_start[i + 1] - s_start[i], scale) : -1;
            const uint32_t peers = __match_any_sync(0xffffffffu, b);
            if (b >= 0 && lane == __ffs(peers) - 1) red_add_shared(&s_bin[b], (uint32_t)__popc(peers));
        }
        __syncthreads();
        if (warp == 0) {  // exclusive scan of the bucket sizes, 8 buckets per lane
            constexpr int BPL = ORDER_BUCKETS / 32;
            uint32_t v[BPL], tot = 0u;
#pragma unroll
            for (int k = 0; k < BPL; ++k) {
                v[k] = s_bin[lane * BPL + k];
                tot += v[k];
            }
            uint32_t bi = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, bi, o);
                if (lane >= o) bi += y;
            }
            uint32_t r = bi - tot;
#pragma unroll
            for (int k = 0; k < BPL; ++k) {
                s_bin[lane * BPL + k] = r;
                r += v[k];
            }
        }
        __syncthreads();
        for (int i0b = 0; i0b < n; i0b += PLACE_THREADS) {
            const int i = i0b + tid;
            uint32_t s0 = 0u, s1 = 0u;
            int b = -1;
            if (i < n) {
                s0 = s_start[i];
                s1 = s_start[i + 1];
                ranges[i] = make_uint2(s0, s1);
                b = place_bucket(s1 - s0, scale);
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, b);
            const int leader = __ffs(peers) - 1;
            uint32_t at = 0u;
            if (b >= 0 && lane == leader) at = atomicAdd(&s_bin[b], (uint32_t)__popc(peers));
            at = __shfl_sync(0xffffffffu, at, leader);
            if (b >= 0) order[at + (uint32_t)__popc(peers & lanemask_lt())] = (uint32_t)i;
        }
        if (lf_blk) {  // the fused loss's normalisers from the compaction's per-block counts
            uint32_t c = 0u, ns = 0u;
#pragma unroll 4
            for (int i = tid; i < lf_grid; i += PLACE_THREADS) {
                c += lf_blk[i];
                ns += lf_blk[lf_grid + i];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c += __shfl_xor_sync(0xffffffffu, c, o);
                ns += __shfl_xor_sync(0xffffffffu, ns, o);
            }
            if (lane == 0) {
                s_w[warp] = c;
                s_w2[warp] = ns;
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t a = 0u, b = 0u;
                for (int w = 0; w < PLACE_THREADS / 32; ++w) {
                    a += s_w[w];
                    b += s_w2[w];
                }
                lf_counts[0] = a;
                lf_counts[1] = b;
            }
        }
    } else {
        // the pairs: PLACE_ITEMS per thread per round, their claims in flight together
        for (bool first = true; base < P; base += (gridDim.x - 1) * span, first = false) {
            if (!first) claim(base);
#pragma unroll
            for (int k = 0; k < PLACE_ITEMS; ++k) {
                const uint32_t o = __shfl_sync(0xffffffffu, old[k], __ffs(peers[k]) - 1);
                if (key[k] < (uint32_t)n) {
                    const uint32_t pos = s_start[key[k]] + o + (uint32_t)__popc(peers[k] & lt);
                    if (pos < cap) {
                        keys_out[pos] = key[k];
                        vals_out[pos] = val[k];
                    }
                }
            }
        }
    }
    // the last CTA out clears the counts and the fill counters
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(scratch + SCR_PLACE_DONE, 1u) == gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int i = tid; i < 2 * n; i += PLACE_THREADS) cnt_g[i] = 0u;
        if (tid == 0) scratch[SCR_PLACE_DONE] = 0u;
    }
}

bool tile_place_fits(int n_tiles) { return n_tiles <= PLACE_SMEM_TILES; }

cudaError_t launch_tile_place(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t cap, uint32_t* scratch,
                              int n_tiles, uint2* ranges, uint32_t* order, const uint32_t* lf_blk, int lf_grid,
                              uint32_t* lf_counts, uint32_t* keys_out, uint32_t* vals_out, cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 148;
    }
    // CTA 0 writes the ranges and the order, the others place the pairs
    int64_t grid = ceil_div((int64_t)cap, (int64_t)PLACE_THREADS * PLACE_ITEMS);
    if (grid > (int64_t)sms * 2 - 1) grid = (int64_t)sms * 2 - 1;
    if (grid < 1) grid = 1;
    grid += 1;
    const size_t smem = (size_t)(n_tiles + 1) * 4;
    cudaError_t e = allow_dynamic_smem((const void*)tile_place_kernel, smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    tile_place_kernel<<<(unsigned)grid, PLACE_THREADS, smem, st>>>(keys_in, vals_in, cap, scratch, n_tiles, ranges,
                                                                   order, lf_blk, lf_grid, lf_counts, keys_out,
                                                                   vals_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// long tile lists (over VG_TILE_SORT_CAP, the forward compositing kernel's
// own sort), one CTA per list.
// Up to RADIX_LONG_CAP entries: a least-significant-digit radix sort on the
// FP32 depth bits in shared memory (four stable passes of 8 bits), then the
// rare runs of equal depth bits put in slot order, which gives the
// (depth bits, slot) order.  Each warp owns a contiguous stretch of the list
// and takes it in rounds of 32 entries: an entry's place among the equal
// digits of its round comes from match_any, its place among earlier rounds
// from the warp's running count of that digit, its place among earlier
// warps and smaller digits from a scan of the warps' digit counts; so every
// pass keeps the order of equal digits (about 110 instructions per entry
// against ~500 for a bitonic network on 2,048).
// Longer lists (up to VG_TILE_SORT_LONG_CAP): keys (depth bits, slot)
// packed as one 64-bit integer, padded to a power of two with the largest
// value and sorted by a bitonic network.
// ---------------------------------------------------------------------------
constexpr int LONG_SORT_THREADS = 512;
constexpr int RADIX_LONG_THREADS = 256;
constexpr int RADIX_LONG_WARPS = RADIX_LONG_THREADS / 32;
constexpr int RADIX_LONG_CAP = 4096;
constexpr int RADIX_LONG_ROUNDS = RADIX_LONG_CAP / RADIX_LONG_THREADS;  // rounds of 32 per warp, at most

__global__ void __launch_bounds__(RADIX_LONG_THREADS, 3) tile_radix_long_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ long_tiles, const uint32_t* __restrict__ n_long_p,
    uint32_t* __restrict__ pvals, const uint32_t* __restrict__ dkey) {
    extern __shared__ uint32_t s_dyn[];
    // buffer b holds keys at s_dyn + b * CAP and slots at s_dyn + (2 + b) * CAP
    auto s_key = [&](int b) { return s_dyn + b * RADIX_LONG_CAP; };
    auto s_val = [&](int b) { return s_dyn + (2 + b) * RADIX_LONG_CAP; };
    uint32_t* s_cnt = s_dyn + 4 * RADIX_LONG_CAP;  // [warp][digit] counts, then offsets
    __shared__ uint32_t s_tmp[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t n_long = *n_long_p;
    for (uint32_t t = blockIdx.x; t < n_long; t += gridDim.x) {
        const uint2 rg = ranges[long_tiles[t]];
        const uint32_t n = rg.y - rg.x;
        if (n > (uint32_t)RADIX_LONG_CAP) continue;  // (the bitonic kernel's)
        for (uint32_t i = threadIdx.x; i < n; i += RADIX_LONG_THREADS) {
            const uint32_t sl = pvals[rg.x + i];
            s_val(0)[i] = sl;
            s_key(0)[i] = dkey[sl];
        }
        // warp w's stretch: [w * seg, min((w + 1) * seg, n)), seg a multiple of 32
        const uint32_t seg = ((n + RADIX_LONG_WARPS * 32 - 1) / (RADIX_LONG_WARPS * 32)) * 32;
        const uint32_t w0 = (uint32_t)warp * seg;
        const int rounds = (int)(seg / 32);
        int cur = 0;
        for (int shift = 0; shift < 32; shift += 8) {
            for (int d = lane; d < 256; d += 32) s_cnt[warp * 256 + d] = 0u;
            __syncthreads();  // (the previous pass's output and this pass's counts)
            uint32_t key[RADIX_LONG_ROUNDS], val[RADIX_LONG_ROUNDS], peers[RADIX_LONG_ROUNDS];
#pragma unroll
            for (int r = 0; r < RADIX_LONG_ROUNDS; ++r) {
                if (r >= rounds) break;
                const uint32_t e = w0 + (uint32_t)r * 32 + (uint32_t)lane;
                const bool ok = e < n;
                key[r] = ok ? s_key(cur)[e] : 0u;
                val[r] = ok ? s_val(cur)[e] : 0u;
                const uint32_t dg = ok ? ((key[r] >> shift) & 255u) : 256u;
                peers[r] = __match_any_sync(0xffffffffu, dg);
                if (ok && (peers[r] & lt) == 0) s_cnt[warp * 256 + dg] += (uint32_t)__popc(peers[r]);
                __syncwarp();
            }
            __syncthreads();
            {  // offsets: digit-major, then warp
                const int dg = threadIdx.x;  // one digit per thread (256 threads)
                uint32_t c[RADIX_LONG_WARPS], tot = 0;
#pragma unroll
                for (int w = 0; w < RADIX_LONG_WARPS; ++w) {
                    c[w] = s_cnt[w * 256 + dg];
                    tot += c[w];
                }
                uint32_t all;
                uint32_t run = block_excl_scan_256(tot, s_tmp, &all);
#pragma unroll
                for (int w = 0; w < RADIX_LONG_WARPS; ++w) {
                    s_cnt[w * 256 + dg] = run;
                    run += c[w];
                }
            }
            __syncthreads();
            const int nxt = cur ^ 1;
#pragma unroll
            for (int r = 0; r < RADIX_LONG_ROUNDS; ++r) {
                if (r >= rounds) break;
                const uint32_t e = w0 + (uint32_t)r * 32 + (uint32_t)lane;
                const bool ok = e < n;
                const uint32_t dg = ok ? ((key[r] >> shift) & 255u) : 0u;
                const uint32_t base = ok ? s_cnt[warp * 256 + dg] : 0u;
                __syncwarp();
                if (ok) {
                    const uint32_t pos = base + (uint32_t)__popc(peers[r] & lt);
                    s_key(nxt)[pos] = key[r];
                    s_val(nxt)[pos] = val[r];
                    if ((peers[r] & lt) == 0) s_cnt[warp * 256 + dg] = base + (uint32_t)__popc(peers[r]);
                }
                __syncwarp();
            }
            cur = nxt;
        }
        __syncthreads();
        // runs of equal depth bits (rare): their slots in increasing order
        for (uint32_t i = threadIdx.x; i < n; i += RADIX_LONG_THREADS) {
            const uint32_t k = s_key(cur)[i];
            if ((i == 0 || s_key(cur)[i - 1] != k) && i + 1 < n && s_key(cur)[i + 1] == k) {
                uint32_t j = i + 1;
                while (j < n && s_key(cur)[j] == k) ++j;
                for (uint32_t a = i + 1; a < j; ++a) {  // insertion sort of s_val(cur)[i, j)
                    const uint32_t v = s_val(cur)[a];
                    uint32_t b = a;
                    while (b > i && s_val(cur)[b - 1] > v) {
                        s_val(cur)[b] = s_val(cur)[b - 1];
                        --b;
                    }
                    s_val(cur)[b] = v;
                }
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += RADIX_LONG_THREADS) pvals[rg.x + i] = s_val(cur)[i];
        __syncthreads();  // shared memory free for the next list
    }
}

__global__ void __launch_bounds__(LONG_SORT_THREADS) tile_sort_long_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ long_tiles, const uint32_t* __restrict__ n_long_p,
    uint32_t* __restrict__ pvals, const uint32_t* __restrict__ dkey, uint32_t* __restrict__ err) {
    extern __shared__ unsigned long long s_k[];  // VG_TILE_SORT_LONG_CAP entries
    const uint32_t n_long = *n_long_p;
    for (uint32_t t = blockIdx.x; t < n_long; t += gridDim.x) {
        const uint2 rg = ranges[long_tiles[t]];
        const uint32_t n = rg.y - rg.x;
        if (n <= (uint32_t)RADIX_LONG_CAP) continue;  // (the radix kernel's)
        if (n > (uint32_t)VG_TILE_SORT_LONG_CAP) {  // left unsorted: the outputs are flagged invalid
            if (threadIdx.x == 0) atomicOr(err, ERR_TILE_LONG);
            continue;
        }
        uint32_t np = 1;
        while (np < n) np <<= 1;
        for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) {
            unsigned long long k = ~0ull;
            if (i < n) {
                const uint32_t sl = pvals[rg.x + i];
                k = ((unsigned long long)dkey[sl] << 32) | sl;
            }
            s_k[i] = k;
        }
        __syncthreads();
        for (uint32_t size = 2; size <= np; size <<= 1)
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t c = threadIdx.x; c < (np >> 1); c += blockDim.x) {
                    // comparator c joins a (bit `stride` clear) and a + stride
                    const uint32_t a = ((c & ~(stride - 1u)) << 1) | (c & (stride - 1u));
                    const bool asc = (a & size) == 0;
                    const unsigned long long x = s_k[a], y = s_k[a + stride];
                    if ((x > y) == asc) {
                        s_k[a] = y;
                        s_k[a + stride] = x;
                    }
                }
                __syncthreads();
            }
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) pvals[rg.x + i] = (uint32_t)s_k[i];
        __syncthreads();  // shared memory free for the next list
    }
}

cudaError_t launch_tile_sort_long(const uint2* ranges, const uint32_t* long_tiles, const uint32_t* n_long,
                                  uint32_t* pvals, const uint32_t* dkey, uint32_t* err, cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 148;
    }
    // lists up to 4,096: the radix kernel, three 72 KB CTAs per SM
    const size_t rsmem = (size_t)(4 * RADIX_LONG_CAP + RADIX_LONG_WARPS * 256) * sizeof(uint32_t);
    cudaError_t e = allow_dynamic_smem((const void*)tile_radix_long_kernel, rsmem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    tile_radix_long_kernel<<<(unsigned)(3 * sms), RADIX_LONG_THREADS, rsmem, st>>>(ranges, long_tiles, n_long, pvals,
                                                                                   dkey);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // longer ones: the bitonic kernel, three 64 KB CTAs per SM; a CTA with no
    // list left exits at once
    const size_t smem = (size_t)VG_TILE_SORT_LONG_CAP * sizeof(unsigned long long);
    e = allow_dynamic_smem((const void*)tile_sort_long_kernel, smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    tile_sort_long_kernel<<<(unsigned)(3 * sms), LONG_SORT_THREADS, smem, st>>>(ranges, long_tiles, n_long, pvals,
                                                                                dkey, err);
    return cudaGetLastError();
}

__global__ void epoch_bump_kernel(uint32_t* state, uint32_t by) { state[ST_EPOCH] += by; }

cudaError_t launch_epoch_bump(uint32_t* state, uint32_t by, cudaStream_t st) {
    count_launches(1);
    epoch_bump_kernel<<<1, 1, 0, st>>>(state, by);
    return cudaGetLastError();
}

}  // namespace vgk
