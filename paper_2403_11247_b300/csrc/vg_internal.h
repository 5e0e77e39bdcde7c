// vg_internal.h -- host-side launchers of the libvg kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "vg_common.cuh"

namespace vgk {

// per-forward scratch words (zeroed by one memset per forward)
constexpr int SCR_DEPTH_HIST = 0;      // [4][256]
constexpr int SCR_TILE_HIST = 1024;    // [3][256]
constexpr int SCR_NVIS = 1792;
constexpr int SCR_PAIRS = 1793;
constexpr int SCR_CNT_DEPTH = 1794;    // 4 pass counters
constexpr int SCR_CNT_DUP = 1798;
constexpr int SCR_CNT_TILE = 1799;     // 3 pass counters
constexpr int SCR_LOSS_VALID = 1802;
constexpr int SCR_N_LONG = 1804;       // tiles with lists over VG_TILE_SORT_CAP (ranges kernel)
constexpr int SCR_PLACE_DONE = 1805;   // CTAs of the tile placement that have finished
constexpr int SCR_WORDS = 1808;
// per-tile pair counts follow, [total_tiles], then the tile placement's fill
// counters, [total_tiles]
constexpr int SCR_TILE_COUNTS = SCR_WORDS;

// persistent state words
constexpr int ST_EPOCH = 0;
constexpr int ST_ERR = 1;
constexpr int ST_EVALS = 2;    // u64 at words 2..3: evaluated (pixel, Gaussian) pairs, forward
constexpr int ST_BLENDED = 4;  // u64 at words 4..5: blended pairs, forward
constexpr int ST_BWD = 6;      // u64 at words 6..7: pairs walked by the backward
// persistent compositing launches: next (view, tile) item, CTAs finished
// (the last CTA out puts both back to zero)
constexpr int ST_WORK_FWD = 8;
constexpr int ST_DONE_FWD = 9;
constexpr int ST_WORK_BWD = 10;
constexpr int ST_DONE_BWD = 11;
constexpr int ST_WORDS = 12;

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int DUP_THREADS = 256;
constexpr int DUP_ITEMS = 4;
constexpr int DUP_TILE = DUP_THREADS * DUP_ITEMS;
constexpr int EMIT_SMEM_TILES = 16384;  // per-tile counts kept in shared memory up to this many tiles

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// view of slot s = v N + n (slots are view-major, views few): by comparisons
// instead of a 64-bit division
__device__ __forceinline__ int slot_view(uint32_t s, uint32_t N, int n_views) {
    int v = 0;
    for (uint32_t next = N; v + 1 < n_views && s >= next; next += N) ++v;
    return v;
}

// pairs are emitted in chunks of EMIT_CHUNK consecutive pairs, one block each
constexpr int EMIT_CHUNK = 256;
// The slot at position j of the pair order owns pairs [o, o + c): every chunk
// k whose first pair EMIT_CHUNK k lies there (and below cap) starts in it.
__device__ __forceinline__ void mark_chunks(uint32_t* chunk_start, uint32_t j, uint32_t o, uint32_t c, uint32_t cap) {
    const uint64_t end = min((uint64_t)o + c, (uint64_t)cap);
    for (uint64_t k = ((uint64_t)o + EMIT_CHUNK - 1) / EMIT_CHUNK; k * EMIT_CHUNK < end; ++k) chunk_start[k] = j;
}

// kernels enqueued by this library in this process (host-side count)
void count_launches(int n);
// Launch kernel<<<grid, block, smem, st>>>(args...) with programmatic stream
// serialization: its CTAs may be scheduled once every CTA of the kernel in
// front of it has started (that kernel calls allow_dependents()), and the
// kernel must call grid_dependency_wait() before it reads anything that
// kernel writes or writes anything that kernel reads.  Used only where the
// kernel in front is this library's own, enqueued by the same call.
template <typename... KArgs, typename... Args>
cudaError_t launch_overlapped(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    count_launches(1);
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
// Raise a kernel's dynamic shared-memory limit when its static plus dynamic
// shared memory passes the 48 KB that launches get without opting in.
cudaError_t allow_dynamic_smem(const void* kernel, size_t dynamic_bytes);
// record the message returned by vg_last_error() and return s
vg_status set_error(vg_status s, const char* msg);

// frame.cu: RGB-D frames (interleaved uint8 RGB, uint16 depth) to planar FP32
cudaError_t launch_frame_decode(int n_views, int64_t hw, const uint8_t* rgb, const uint16_t* depth, float depth_scale,
                                float* C, float* D, cudaStream_t st);

// preprocess.cu
int preprocess_blocks(int64_t N);
// the compaction's grid (preprocess_blocks, widened for the fused loss's
// counts when cs.lf_on)
int compact_grid(int64_t N, const Consts& cs);
cudaError_t launch_preprocess(const SceneDev& S, const Views& V, const Consts& cs, float4* xy, float4* conic_o,
                              float4* rgbd, uint2* rect, uint32_t* ntiles, uint32_t* dkey, uint32_t* scratch,
                              uint32_t* state, uint32_t* blk_count, cudaStream_t st);
// visible slots, in (view, Gaussian) order within each preprocess block, to keys_out / vals_out
// blk_count holds [blocks] visible-slot counts, then (pair_off non-NULL)
// [blocks] pair counts; with pair_off the pair offsets of the compacted
// order, the chunk starts, the pair count and the overflow flag are produced
// here and launch_duplicate skips its own scan
// g2d_rows (may be NULL): the backward's per-slot gradient rows, zeroed here
// for every visible slot; pose_zero [n_pose] (may be NULL): zeroed too.
// With cs.lf_on it also counts the fused loss's normalisers per block into
// cs.lf_blk [2][compact_grid] (the ranges kernel sums them).
cudaError_t launch_compact(const Views& V, int64_t N, const uint32_t* dkey, const uint32_t* blk_count,
                           uint32_t* keys_out, uint32_t* vals_out, uint32_t* vals_copy, const uint32_t* ntiles,
                           uint32_t* pair_off, uint32_t* chunk_start, uint32_t cap, uint32_t* scratch, uint32_t* err,
                           float* g2d_rows, float* pose_zero, int n_pose, const Consts& cs, cudaStream_t st);
cudaError_t launch_rvq_decode(int dim, int L, int K, const float* cb, const uint8_t* idx, const float* raw,
                              int64_t n, float* out, cudaStream_t st);

// sort.cu
// One stable LSD pass on 8-bit digit (key >> shift) & 255 of u32 keys with u32
// values (vals_in NULL: value = index).  n = min(*n_dev, n_cap) if n_dev, else n_cap.
cudaError_t launch_sort_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                             uint32_t* vals_out, const uint32_t* n_dev, uint32_t n_cap, int shift,
                             const uint32_t* hist, unsigned long long* lookback, uint32_t* counter,
                             const uint32_t* state, uint32_t epoch_offset, uint32_t* err, int grid,
                             uint32_t spin_limit, cudaStream_t st);
int sort_pass_grid(uint32_t n_cap);
// offsets has room for [slots + 1] (the last is the pair count) and
// chunk_start for [ceil(cap / EMIT_CHUNK)]; offsets_ready: both were filled by
// launch_compact for this order; else part_total [ceil(slots / 1024)] holds
// the per-partition totals of the reduce-then-scan
cudaError_t launch_duplicate(const uint32_t* sorted_slots, uint32_t* offsets, uint32_t* chunk_start,
                             bool offsets_ready, const uint32_t* ntiles,
                             const uint2* rect, int64_t N, const Views& V, uint32_t* pkeys, uint32_t* pvals,
                             uint32_t cap, uint32_t* scratch, int tile_passes, uint32_t* part_total, uint32_t* err,
                             int64_t max_slots, uint2* ranges, cudaStream_t st);
// global-sort form: tile ranges from the tile-sorted pair keys (the
// emission zeroed them; the per-tile counts are not kept)
cudaError_t launch_tile_bounds(const uint32_t* keys, const uint32_t* n_dev, uint32_t cap, uint2* ranges,
                               cudaStream_t st);
// per-tile [start, end) from the per-tile pair counts at scratch +
// SCR_TILE_COUNTS (one-block scan); clear: zero the counts, the digit
// histograms and the pass counters afterwards (global-sort form).  With
// lf_blk (may be NULL) also the fused loss's counts: lf_counts[c] = sum of
// lf_blk[c * lf_grid + b] over b.  With long_tiles (may be NULL) the tiles
// whose lists pass VG_TILE_SORT_CAP are listed there, their number in
// scratch[SCR_N_LONG].
// from_ranges: the ranges are already final (global-sort form): the counts
// are taken from them and only the order (and the rest) is built.
cudaError_t launch_ranges(uint32_t* scratch, int n_tiles, uint2* ranges, uint32_t* order, int clear,
                          const uint32_t* lf_blk, int lf_grid, uint32_t* lf_counts, uint32_t* long_tiles,
                          int from_ranges, cudaStream_t st);
// sort the lists of the tiles in long_tiles[0 .. *n_long) by (dkey[slot],
// slot), one CTA per list, in shared memory (lists over VG_TILE_SORT_LONG_CAP
// flag ERR_TILE_LONG and stay unsorted)
cudaError_t launch_tile_sort_long(const uint2* ranges, const uint32_t* long_tiles, const uint32_t* n_long,
                                  uint32_t* pvals, const uint32_t* dkey, uint32_t* err, cudaStream_t st);
cudaError_t launch_epoch_bump(uint32_t* state, uint32_t by, cudaStream_t st);
// ranges, longest-first tile order and the grouping of the pairs by tile
// (unordered within a tile) in one launch, from the per-tile pair counts at
// scratch + SCR_TILE_COUNTS (which end at zero, as do the fill counters after
// them); lf_blk / lf_counts as in launch_ranges.  For up to
// tile_place_fits() tiles.
bool tile_place_fits(int n_tiles);
cudaError_t launch_tile_place(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t cap, uint32_t* scratch,
                              int n_tiles, uint2* ranges, uint32_t* order, const uint32_t* lf_blk, int lf_grid,
                              uint32_t* lf_counts, uint32_t* keys_out, uint32_t* vals_out, cudaStream_t st);
// group the pairs by tile (unordered within a tile) into the ranges; counts
// (the per-tile pair counts the ranges came from) end at zero
cudaError_t launch_tile_scatter(const uint32_t* keys_in, const uint32_t* vals_in, const uint32_t* n_dev, uint32_t cap,
                                const uint2* ranges, uint32_t* counts, uint32_t* keys_out, uint32_t* vals_out,
                                cudaStream_t st);

// ssim.cu: workspace ws holds 8 * 3 * n_views * W * H + 1 floats
vg_status launch_ssim(int n_views, int W, int H, const float* C, const float* Ct, float weight, float* dC, float* loss,
                      float* ws, cudaStream_t st);

// icp.cu
vg_status launch_icp_associate(const SceneDev& S, const Views& V, const float* Dt, float max_dist, float weight, float* q,
                               float* w, cudaStream_t st);

// grow.cu
int64_t grow_table_slots(int64_t A, int64_t N, int64_t cap);
cudaError_t launch_grow_stats(const SceneDev& S, const uint32_t* vis, const uint32_t* nvis_dev, uint32_t max_vis,
                              const float* g2d, float* gacc, uint32_t* gcnt, float* oacc, uint32_t* ocnt,
                              cudaStream_t st);
cudaError_t launch_grow(const SceneDev& S, const float* gacc, const uint32_t* gcnt, float eps_g, float tau_g, int levels,
                        unsigned long long drop_below, unsigned long long seed, float* new_xyz, int32_t* new_level,
                        uint32_t* n_new, int64_t cap, void* ws, int64_t slots, uint32_t* err, cudaStream_t st);
cudaError_t launch_anchor_prune(float* mask, int64_t A, int k, const float* oacc, const uint32_t* ocnt, float tau_alpha,
                                uint32_t* removed, uint32_t* n_removed, cudaStream_t st);

// mask.cu
vg_status vg_mask_kernels_loss(const SceneDev& S, const Views& V, const uint32_t* ntiles, float weight, float* dmask,
                               float* loss, uint32_t* scratch_u, float* scratch_f, cudaStream_t st);
vg_status vg_mask_kernels_prune(float* m, float thr, const uint32_t* hits, const uint32_t* seen, uint32_t min_hits,
                                int64_t N, uint32_t* removed, uint32_t* n_removed, cudaStream_t st);

// blend.cu
// dkey non-NULL: sort each tile's list by (dkey[slot], slot) first (VG_SORT_TILE)
// persist > 0: persist CTAs per SM pull tiles from `work` ([0] next item,
// [1] CTAs done, both zero before and after the launch); 0: a CTA per tile
cudaError_t launch_blend_fwd(const Views& V, const Consts& cs, int ppt, int persist, uint32_t* work,
                             const uint2* ranges, const uint32_t* order,
                             uint32_t* pvals, const uint32_t* dkey, uint32_t* err,
                             const float4* xy, const float4* conic_o, const float4* rgbd, float* C, float* D,
                             float* S, float* Tfin, uint32_t* ncontrib, unsigned long long* evals,
                             unsigned long long* blended, uint32_t* neval, int count_evals, cudaStream_t st);
cudaError_t launch_blend_bwd(const Views& V, const Consts& cs, int ppt, int persist, uint32_t* work,
                             const uint2* ranges, const uint32_t* order,
                             const uint32_t* pvals,
                             const float4* xy, const float4* conic_o, const float4* rgbd, const float* Tfin,
                             const uint32_t* ncontrib, const float* dC, const float* dD, const float* dS,
                             float* g2d, unsigned long long* bwd_pairs, int count, cudaStream_t st);

// split.cu: deep tile lists cut into S segments, one CTA per (tile,
// segment); per-segment state in segf [items][SPLIT_F][256] (product of the
// segment, its five blended sums, its final T) and segu [items][SPLIT_U][256]
// (last contributor, blended count, stop position, composited flag), items =
// tiles x S.  dkey non-NULL: sort each tile's list first (per-tile form).
constexpr int SPLIT_F = 8;
constexpr int SPLIT_U = 4;
constexpr int SPLIT_MAX = 32;
cudaError_t launch_split_fwd(const Views& V, const Consts& cs, int S, const uint2* ranges, uint32_t* pvals,
                             const uint32_t* dkey, uint32_t* err, const float4* xy, const float4* conic_o,
                             const float4* rgbd, float* segf, uint32_t* segu, float* C, float* D, float* Sout,
                             float* Tfin, uint32_t* ncontrib, unsigned long long* evals, unsigned long long* blended,
                             uint32_t* neval, int count_evals, cudaStream_t st);
cudaError_t launch_split_bwd(const Views& V, const Consts& cs, int S, const uint2* ranges, const uint32_t* pvals,
                             const float4* xy, const float4* conic_o, const float4* rgbd, const float* segf,
                             const uint32_t* segu, const uint32_t* ncontrib, const float* dC, const float* dD,
                             const float* dS, float* g2d, unsigned long long* bwd_pairs, int count, cudaStream_t st);

// grad.cu
// where the chain kernel accumulates the scene gradients (device pointers;
// NULL = not wanted); cb_off/cb_total/cb_in_smem are filled by the launcher
struct ChainOut {
    float* raw[4];   // per-Gaussian attribute gradients of uncoded groups [N][d]
    float* cb[4];    // codebook gradients of coded groups [L][K][d]
    float *d_xyz, *d_l, *d_off, *d_mask;
    float* pose_sum;   // [views][6], zeroed before the backward
    // shared-memory accumulator offsets: the four attribute codebooks, then the
    // R-VQ offset codebook (4) and scaling-factor codebook (5) when coded
    int32_t cb_off[6], cb_total, cb_in_smem;
};
// arrays the zeroing kernel clears before the backward
struct ZeroList {
    int32_t n;
    float* p[12];
    int64_t count[12];
};
cudaError_t launch_zero_bwd(const uint32_t* vis_slots, const uint32_t* nvis_dev, uint32_t max_vis, float* g2d,
                            const ZeroList& Z, cudaStream_t st);
cudaError_t launch_chain(const SceneDev& S, const Views& V, const Consts& cs, const float* g2d, const uint32_t* vis,
                         const uint32_t* nvis_dev, uint32_t max_vis, ChainOut O, int* n_blocks_out, cudaStream_t st);
int chain_blocks(int64_t N);
cudaError_t launch_icp(const SceneDev& S, const Views& V, const float* q, const float* w, float* part, int n_blocks,
                       cudaStream_t st);
int icp_blocks(int64_t N);
cudaError_t launch_pose_final(int n_views, const float* pose_sum, const float* icp_part, int n_icp_blocks,
                              float* dxi, float* icp_loss, cudaStream_t st);
cudaError_t launch_sample_rays(uint8_t* mask, int64_t n, unsigned long long seed, const int32_t* round_dev,
                               int32_t round_host, unsigned long long keep_below, cudaStream_t st);
// mask non-NULL: only sampled pixels count (vg_loss_l1_masked).  valid_count:
// four words, zero before the first call; the call leaves them zero (no memset
// between calls) and writes loss[0] itself.  err: the ctx's status word (the
// single-launch form's barrier reports a spin that ran out of its spin_limit
// unsuccessful polls there)
cudaError_t launch_loss_l1(int n_views, int64_t n_pix, const float* C, const float* D, const float* S,
                           const float* Ct, const float* Dt, const uint8_t* mask, float w_depth, float gate, float* dC,
                           float* dD, float* loss, uint32_t* valid_count, uint32_t* err, uint32_t spin_limit,
                           cudaStream_t st);

// optim.cu
// zero_mask bit t: tensor t's gradient is zeroed once read
cudaError_t launch_adam(int n, float* const* p, float* const* g, float* const* m, float* const* v,
                        const int64_t* size, uint32_t zero_mask, float lr, float b1, float b2, float eps,
                        int32_t* step_dev, int32_t step_host, cudaStream_t st);
cudaError_t launch_pose_step(int n_views, float* pose, const float* dxi, float* m, float* v, float lr_rot,
                             float lr_trans, float b1, float b2, float eps, int32_t* step_dev, int32_t step_host,
                             cudaStream_t st);

}  // namespace vgk
