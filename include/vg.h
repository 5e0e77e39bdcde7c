/*
 * vg.h -- C ABI of libvg, a B300 (sm_103a) differentiable tile rasterizer for
 * voxel-anchored, residual-codebook-coded, mask-pruned 3D Gaussians
 * (Deng et al., "Voxelized 3D Gaussian Representation for Dense Visual SLAM
 * on Embedded Vision System").
 *
 * Conventions shared by every call
 * --------------------------------
 * Pointers.  Unless a parameter says "host", every array argument is a DEVICE
 *   pointer of the current CUDA device, allocated and owned by the caller.
 *   libvg owns only what it allocates itself: a vg_scene made by
 *   vg_scene_upload with VG_SCENE_COPY and a vg_ctx; each is released by its
 *   _free call.
 * Layout.  Float arrays are IEEE FP32, little-endian, dense, row-major (C
 *   order).  Images of a multi-view call are per-view planar blocks laid end to
 *   end in view order: view v owns pixels [pb_v, pb_v + W_v*H_v), pb_v the sum
 *   of W*H over earlier views; colour holds three planes per view
 *   (C + 3*pb_v: R plane, G plane, B plane, each H_v rows of W_v), depth and
 *   silhouette one plane.  With equal sizes this is [B][3][H][W] and [B][H][W].
 * Streams.  Every call enqueues its work on the given stream and returns
 *   without synchronising, except vg_scene_upload (which synchronises its
 *   stream before returning) and vg_check / vg_ctx_stats (which synchronise
 *   the stream to read device status).
 * Errors.  Argument errors are detected on the host before anything is
 *   enqueued and return VG_ERR_INVALID_ARG.  A failed CUDA call returns
 *   VG_ERR_CUDA.  Conditions found on the device (the pair buffer of the ctx
 *   too small, a bounded wait that ran out) set a flag in the ctx and leave the
 *   outputs of that call undefined; the next vg_check returns VG_ERR_CAPACITY
 *   or VG_ERR_TIMEOUT and clears the flag.  vg_last_error() gives a message for
 *   the calling thread's last non-OK status.
 * Threads.  One vg_ctx per stream; a vg_scene may be shared by calls on
 *   several streams as long as nothing writes it meanwhile.
 */
#ifndef VG_H
#define VG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* vg_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    VG_OK = 0,
    VG_ERR_INVALID_ARG = 1,
    VG_ERR_OOM = 2,
    VG_ERR_CUDA = 3,
    VG_ERR_CAPACITY = 4,
    VG_ERR_TIMEOUT = 5,
    VG_ERR_UNIMPLEMENTED = 6
} vg_status;

#define VG_TILE 16          /* tile side in pixels (the only supported value) */
#define VG_MAX_VIEWS 64     /* views per launch */
#define VG_MAX_CODEWORDS 256 /* 1-byte indices */
#define VG_SORT_AUTO 0       /* vg_render_params.sort_mode: per-tile unless it overflowed on this ctx */
#define VG_SORT_GLOBAL 1     /* radix sort of the visible slots by depth, then pairs stably by tile */
#define VG_SORT_TILE 2       /* pairs by tile only; each tile's list sorted by depth in the forward */
#define VG_TILE_SORT_CAP 1024 /* longest tile list the compositing kernel sorts itself */
#define VG_TILE_SORT_LONG_CAP 8192 /* longest tile list the per-tile sort takes (long-list pass) */

/* Pinhole camera.  T_cw: row-major 3x4 world->camera transform [R | t];
 * camera x right, y down, z forward.  A point projects to
 * u = fx * x / z + cx, v = fy * y / z + cy (pixel (px, py) is sampled at
 * integer coordinates).  Gaussians with camera depth z <= near_plane are
 * culled. */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
    float T_cw[12];
    float near_plane;
} vg_camera;

/* One attribute group of the Gaussians (Sec. "Residual Codebook
 * Quantization", Eq. 14 first line: the attribute of Gaussian n is the sum,
 * over stages s = 0..L-1 in order, of codebook[s][idx[s][n]]; 1-byte indices).
 * stages == 0 selects raw per-Gaussian values instead.
 *   dim        values per Gaussian (log-scale 3, quaternion 4, opacity 1, RGB 3)
 *   stages     L (0 = raw)
 *   codewords  K, 1..256
 *   codebook   [L][K][dim] FP32
 *   idx        [L][N] uint8, stage-major
 *   raw        [N][dim] FP32 when stages == 0 */
typedef struct {
    int32_t dim;
    int32_t stages;
    int32_t codewords;
    const float* codebook;
    const uint8_t* idx;
    const float* raw;
} vg_attr_group;

/* Scene (Sec. "Voxel-Anchored 3D Gaussian Representation", Eq. 7): anchors
 * with position x_a, scaling factor l and k offsets O_i; Gaussian n = a*k + i
 * sits at mu_n = x_a + O_i * l (element-wise).  Attributes: log-scale
 * (scale = exp), quaternion (w, x, y, z; normalised before use), opacity
 * logit (opacity = sigmoid), RGB (used as is).  Online mask (Eq. 11-12):
 * Gaussian n is kept iff sigmoid(mask_logit[n]) > mask_eps, evaluated as
 * mask_logit[n] > logit(mask_eps) rounded to FP32; a removed Gaussian renders
 * exactly as if deleted.  mask_logit may be NULL (all kept). */
typedef struct {
    int64_t n_anchors;
    int32_t k;
    const float* anchor_xyz; /* [Na][3] */
    const float* anchor_l;   /* [Na][3] */
    const float* offsets;    /* [Na][k][3] */
    vg_attr_group logscale, rot, opacity, rgb;
    const float* mask_logit; /* [N] or NULL */
    float mask_eps;
    /* R-VQ coded offsets and scaling factors (Sec. "Residual Codebook
     * Quantization", Eq. 14: the offset O and scaling factor l are what the
     * paper's R-VQ compresses).  With offsets_rvq.stages > 0, O_n (n = a*k + i)
     * is the sum over stages of offsets_rvq.codebook[s][idx[s][n]] (dim 3,
     * idx [L][N]) and `offsets` is not read; with l_rvq.stages > 0, l_a is the
     * sum of l_rvq.codebook[s][idx[s][a]] (dim 3, idx [L][Na], one code per
     * anchor) and `anchor_l` is not read.  Sums are FP32 in stage order.
     * stages = 0 (a zeroed struct) keeps the raw arrays. */
    vg_attr_group offsets_rvq;
    vg_attr_group l_rvq;
} vg_scene_desc;

/* Per-pixel compositing constants (readings of Eq. 16-18; the paper leaves
 * them open):
 *   alpha(p) = min(alpha_max, o * exp(-1/2 d^T Sigma'^-1 d)), d = (u,v) - p;
 *   a Gaussian with alpha < alpha_min, or with positive exponent, is skipped;
 *   compositing stops before a Gaussian that would bring transmittance below
 *   t_min (that Gaussian is not blended);
 *   Sigma' gets `dilation` px^2 added to its diagonal;
 *   radius r = ceil(sigma_cull * sqrt(lambda_max(Sigma'))), tile rect
 *   [floor((u-r)/16), floor((u+r)/16)+1) x [same for v], clipped to the image;
 *   with jacobian_clamp, x/z and y/z inside the projection Jacobian are
 *   clamped to +-clamp_factor * (W/2)/fx and +-clamp_factor * (H/2)/fy.
 * batch: Gaussians the compositing kernels stage in shared memory at a time:
 *   64, 128 or 256 (0 = 256).  Any value gives the same results.
 * persist_ctas: 0 (default) launches the compositing kernels with one CTA
 *   per (view, tile); k in 1..32 launches k CTAs per SM that take (view,
 *   tile) items, longest list first, from a device counter until none is
 *   left (a persistent launch; the counter is back at zero after it, so a
 *   captured graph can replay it).  Same results either way.
 * ppt_fwd, ppt_bwd: pixels per thread in the forward / backward blend
 *   kernels, 1, 2 or 4 (0 = default: 2); a 16x16 tile is one block of
 *   256 / ppt threads.
 * pose_dev: optional DEVICE array [n_views][12] read instead of the
 *   cameras' T_cw (lets a captured CUDA graph follow poses updated on the
 *   device).  count_evals: accumulate evaluated (pixel, Gaussian) pairs into
 *   the ctx counter (vg_ctx_stats) and keep each pixel's count
 *   (VG_BUF_N_EVAL).
 * hit_count, seen: optional DEVICE arrays [N] for the sliding-window mask
 *   (Sec. "Sliding Window-based Online Mask", Eq. 13).  vg_render_fwd ADDS
 *   to hit_count[n] the number of (view, pixel) pairs where Gaussian n is
 *   blended and sets seen[n] = 1 where Gaussian n is visible (an unempty
 *   tile rect) in some view; nothing clears them, so a sliding window
 *   accumulates over its frames.  NULL = off.
 * sort_mode: how the (tile, depth, index) order of the pairs is built; all
 *   give the same order.  VG_SORT_GLOBAL: a stable radix sort of the visible
 *   slots on their FP32 depth bits, pairs emitted in that order, then a
 *   stable sort by tile.  VG_SORT_TILE: pairs emitted in slot order and
 *   grouped by tile; the forward compositing kernel sorts each tile's list
 *   of up to VG_TILE_SORT_CAP entries by (depth bits, slot) in shared memory
 *   and writes it back for the backward, and a pass before it sorts the
 *   longer lists (up to VG_TILE_SORT_LONG_CAP entries, one CTA each: a
 *   shared-memory radix sort up to 4,096 entries, a bitonic network above).
 *   VG_SORT_AUTO (the default): VG_SORT_TILE without the long-list pass
 *   until a forward on this ctx meets a list over VG_TILE_SORT_CAP, and
 *   VG_SORT_GLOBAL from then on (for lists that long the global radix
 *   passes are faster than the scatter and the per-list sorts).  A forward
 *   that meets a list longer than its form takes leaves its outputs invalid
 *   and the next vg_check returns VG_ERR_CAPACITY (render again:
 *   vg.render_with_retry does).
 * pixel_mask: optional DEVICE array [total pixels of all views, in view
 *   order, each row-major] of 0/1: only pixels with 1 are composited (the
 *   sampled rays of a bundle-adjustment step, Sec. "Tracking and
 *   Local-to-Global Bundle Adjustment"); the others get C = D = S = 0 and
 *   are skipped by the backward.  NULL = every pixel.  See vg_sample_rays.
 * grad_accumulate: vg_render_bwd ADDS to the scene-gradient arrays instead
 *   of zeroing them first; the caller keeps them zero between steps (e.g.
 *   vg_adam_step with zero_grad set clears each gradient after using it).
 *   0 (default) = the backward zeroes them.
 * list_split: compositing of deep tile lists across CTAs.  With S > 1 each
 *   tile's list is cut into S consecutive segments, each composited by its
 *   own CTA (forward: the segments' transmittance products, then each
 *   segment walked from the transmittance in front of it, then the sums
 *   combined in order; backward: each segment walked back to front from its
 *   own final transmittance) -- for images with too few tiles to fill the
 *   GPU.  0 (default) = automatic: S = min(16, ceil(2 x SMs / tiles)) when
 *   the views have fewer tiles than the GPU has SMs, else 1; 1 = never;
 *   2..32 = S.  The images equal the unsplit ones up to FP32 rounding of
 *   the transmittance products (the same Gaussians are blended except where
 *   a product lands within rounding of t_min); the backward must use the
 *   forward's split, which the ctx keeps.  Workspace: 48 B per tile pixel
 *   and segment (tiles x S x 256 x 48 B). */
typedef struct {
    int32_t tile;
    int32_t batch;
    float alpha_max, alpha_min, t_min, dilation, sigma_cull, clamp_factor;
    int32_t jacobian_clamp;
    int32_t count_evals;
    const float* pose_dev;
    int32_t ppt_fwd, ppt_bwd;
    uint32_t* hit_count;
    uint32_t* seen;
    int32_t sort_mode;
    const uint8_t* pixel_mask;
    int32_t grad_accumulate;
    int32_t persist_ctas;
    int32_t list_split;
} vg_render_params;

/* Gradient outputs of vg_render_bwd (DEVICE pointers, caller-allocated; each
 * may be NULL to skip it; every non-NULL array is fully overwritten):
 *   anchor_xyz [Na][3], anchor_l [Na][3], offsets [Na][k][3] -- or, for
 *   R-VQ coded offsets / scaling factors, their [L][K][3] codebook gradients;
 *   per attribute group: [L][K][dim] codebook gradient for a coded group,
 *   [N][dim] for a raw group; mask_logit [N] (straight-through estimator of
 *   Eq. 11: dL/dm = (sum_j dL/ds_j s_j + dL/do o) sigmoid'(m) for kept
 *   Gaussians, 0 for removed ones). */
typedef struct {
    float* anchor_xyz;
    float* anchor_l;
    float* offsets;
    float* logscale;
    float* rot;
    float* opacity;
    float* rgb;
    float* mask_logit;
} vg_scene_grads;

/* Device counters of a ctx, read by vg_ctx_stats. */
typedef struct {
    int64_t pairs;          /* (Gaussian, tile) pairs of the last forward */
    int64_t pair_capacity;  /* current pair buffer size */
    int64_t visible;        /* (view, Gaussian) slots that reached a tile */
    int64_t evaluated;      /* forward: (pixel, Gaussian) pairs examined, accumulated while count_evals */
    int64_t blended;        /* forward: pairs blended, accumulated while count_evals */
    int64_t bwd_pairs;      /* backward: pairs walked (sum of per-pixel list lengths), while count_evals */
    uint32_t flags;         /* bit0 bounded wait ran out, bit1 pair overflow */
} vg_stats;

typedef struct vg_scene vg_scene;
typedef struct vg_ctx vg_ctx;

#define VG_SCENE_COPY 0   /* copy every array (host or device source) into libvg-owned device memory */
#define VG_SCENE_BORROW 1 /* keep the caller's device pointers; values may change between calls */

/* Make a device-resident scene from `desc` (a HOST struct).  COPY: arrays may
 * be host or device pointers; they are copied, and the call synchronises
 * `stream` before returning.  BORROW: arrays must be device pointers that stay
 * valid until vg_scene_free; the caller may update their values in place
 * (e.g. an optimiser step) but not their sizes or index arrays.  Both forms
 * build, once, the per-stage codeword-to-Gaussian lists used to reduce
 * codebook gradients.  Errors: VG_ERR_INVALID_ARG (null or inconsistent
 * sizes, k < 1, K > 256, dims other than 3/4/1/3), VG_ERR_OOM, VG_ERR_CUDA. */
vg_status vg_scene_upload(const vg_scene_desc* desc, int32_t flags, vg_stream stream, vg_scene** out);
vg_status vg_scene_free(vg_scene* scene);
/* Number of Gaussians (n_anchors * k). */
int64_t vg_scene_size(const vg_scene* scene);

/* Workspace for the render calls: per-(view, Gaussian) records, sort
 * buffers, per-pixel state kept from forward to backward, device counters.
 * Sizes are hints; slot, pixel and tile buffers grow on demand (outside
 * stream capture), the pair buffer grows only through vg_ctx_reserve. */
vg_status vg_ctx_create(int64_t pair_capacity, vg_ctx** out);
vg_status vg_ctx_free(vg_ctx* ctx);
/* Page-locked host memory for the frames a caller streams in and the
 * results it reads back (the paper has no counterpart): 2 MB aligned,
 * transparent huge pages requested (madvise), zero-filled, then registered
 * with the CUDA driver (cudaHostRegister), so that copies from it run as
 * asynchronous DMA.  Measured on a B300 system (PCIe Gen6), 13 MB
 * host->device copies from such memory ran at ~55 GB/s when its lines were
 * in memory; written by a core just before, they ran at ~15 GB/s (the
 * copy engine then reads dirty cache lines): fill it with vg_host_stage.
 * vg_host_alloc: *out receives the pointer (bytes > 0); VG_ERR_OOM if the
 * memory cannot be had, VG_ERR_CUDA if registration fails.
 * vg_host_free: unregisters and frees a pointer from vg_host_alloc (NULL is
 * a no-op); the caller keeps no device work reading it in flight. */
vg_status vg_host_alloc(int64_t bytes, void** out);
vg_status vg_host_free(void* ptr);
/* Host-to-host copy of `bytes` into a staging buffer with streaming
 * (non-temporal) stores on x86-64, a plain copy elsewhere: the written lines
 * do not stay dirty in the CPU caches.  The copy engine's reads of lines a
 * core had just written measured ~15 GB/s on a B300 system, against
 * ~55 GB/s for lines in memory; stage each frame with this call before
 * vg_memcpy_async.  Synchronous; VG_ERR_INVALID_ARG for a negative size or
 * NULL pointers. */
vg_status vg_host_stage(void* dst, const void* src, int64_t bytes);
/* One asynchronous copy of `bytes` between any two of host memory (page-
 * locked for asynchrony, e.g. from vg_host_alloc) and device memory, in
 * `stream` order (cudaMemcpyAsync with the direction inferred from the
 * pointers).  VG_ERR_INVALID_ARG for a negative size or NULL pointers. */
vg_status vg_memcpy_async(void* dst, const void* src, int64_t bytes, vg_stream stream);
/* Grow the pair buffer to at least `pair_capacity` (no-op if large enough). */
vg_status vg_ctx_reserve(vg_ctx* ctx, int64_t pair_capacity);
/* Synchronise `stream`, read the counters into *out (may be NULL), return
 * VG_ERR_CAPACITY / VG_ERR_TIMEOUT if a device flag is set (and clear it),
 * else VG_OK. */
vg_status vg_check(vg_ctx* ctx, vg_stream stream);

/* Bounded device waits (failure detection; no counterpart in the paper).
 * Every spin a kernel of this ctx makes on another block -- the radix
 * sort's and the pair-offset scan's decoupled look-back, the cooperative
 * loss's grid barrier -- gives up after `polls` unsuccessful polls, sets a
 * device flag and lets the kernel finish (its results are then wrong, every
 * index stays inside its buffer); the next vg_check returns VG_ERR_TIMEOUT.
 * The default, 2^21 polls (about a second of L2 round trips), is far above
 * any wait of a working device; a small limit makes the waits run out (for
 * tests).  polls = VG_SPIN_LIMIT_DEFAULT_SENTINEL restores the default.
 * Takes effect from the next call enqueued on the ctx. */
#define VG_SPIN_LIMIT_DEFAULT_SENTINEL 0xffffffffu
vg_status vg_ctx_set_spin_limit(vg_ctx* ctx, uint32_t polls);
vg_status vg_ctx_stats(vg_ctx* ctx, vg_stream stream, vg_stats* out);
/* Zero the evaluated / blended / backward pair counters (enqueued). */
vg_status vg_ctx_reset_counters(vg_ctx* ctx, vg_stream stream);

/* Per-stage timing with CUDA events recorded on the launching stream around
 * every kernel a render / loss / pose call enqueues.  vg_ctx_profile(ctx, 1)
 * clears the records and starts recording, 0 stops.  vg_ctx_profile_read
 * synchronises `stream` and writes, for each stage id s < VG_STAGE_COUNT,
 * ms_total[s] (sum of event-to-event durations) and launches[s].  Calls made
 * during stream capture record their events as external event nodes of the
 * graph; those records persist (until the ctx is freed) and report the most
 * recent replay of the graph.  VG_STAGE_CHAIN includes the codebook
 * gradients (accumulated in the same pass); VG_STAGE_CODEBOOK records
 * nothing and is kept for the numbering.  VG_STAGE_MEMSET covers the zeroing
 * before the backward. */
enum {
    VG_STAGE_PREPROCESS = 0, VG_STAGE_DEPTH_SORT, VG_STAGE_DUPLICATE, VG_STAGE_TILE_SORT, VG_STAGE_RANGES,
    VG_STAGE_BLEND_FWD, VG_STAGE_LOSS, VG_STAGE_BLEND_BWD, VG_STAGE_CHAIN, VG_STAGE_CODEBOOK, VG_STAGE_POSE,
    VG_STAGE_MEMSET, VG_STAGE_COUNT
};
vg_status vg_ctx_profile(vg_ctx* ctx, int32_t enable);
vg_status vg_ctx_profile_read(vg_ctx* ctx, vg_stream stream, double* ms_total, int64_t* launches);

/* Read-only view of an intermediate workspace array, for inspection and
 * tests.  Valid after the call that fills it and until the next render call
 * on the ctx; the ctx keeps ownership.  *ptr gets the device address and
 * *bytes the number of valid bytes (pair arrays: capacity bytes; the valid
 * count is vg_stats.pairs).
 *   VG_BUF_XY         float4 [slots]  projected mean (u, v) and the half extents of the
 *                                     box where alpha can reach alpha_min (slot = view*N + n)
 *   VG_BUF_CONIC      float4 [slots]  base-2 exponent coefficients -a/2 log2 e, -b log2 e,
 *                                     -c/2 log2 e of the inverse 2D covariance [[a,b],[b,c]]
 *                                     and log2(alpha_min / opacity)
 *   VG_BUF_RGBD       float4 [slots]  r, g, b, camera depth
 *   VG_BUF_RECT       uint2  [slots]  tile rect x0|y0<<16, x1|y1<<16
 *   VG_BUF_NTILES     uint32 [slots]  tiles touched (0 = culled)
 *   VG_BUF_PAIR_KEYS  uint32 [pairs]  sorted global tile ids
 *   VG_BUF_PAIR_VALS  uint32 [pairs]  slot of each sorted pair
 *   VG_BUF_RANGES     uint2  [tiles]  [start, end) of each tile's list
 *   VG_BUF_T_FINAL    float  [pixels] transmittance after compositing
 *   VG_BUF_N_CONTRIB  uint32 [pixels] list position + 1 of the last blended Gaussian
 *   VG_BUF_G2D        float  [slots][12] du dv da db dc dopacity dr dg db ddepth, 2 pad
 *   VG_BUF_N_EVAL     uint32 [pixels] list entries the pixel examined, up to and including the
 *                                     one that stopped it (forwards with count_evals only) */
enum {
    VG_BUF_XY = 0, VG_BUF_CONIC, VG_BUF_RGBD, VG_BUF_RECT, VG_BUF_NTILES, VG_BUF_PAIR_KEYS, VG_BUF_PAIR_VALS,
    VG_BUF_RANGES, VG_BUF_T_FINAL, VG_BUF_N_CONTRIB, VG_BUF_G2D, VG_BUF_N_EVAL
};
vg_status vg_ctx_buffer(const vg_ctx* ctx, int32_t which, const void** ptr, int64_t* bytes);

/* Eq. 14, first line, standalone: out[n][c] = sum_s codebook[s][idx[s][n]][c]
 * summed in stage order, for n < n_items.  `group` is a HOST struct with
 * device arrays; out is [n_items][dim].  A raw group (stages == 0) is copied. */
vg_status vg_rvq_decode(const vg_attr_group* group, int64_t n_items, float* out, vg_stream stream);

/* Eq. 14, second line, and Eq. 15: residual vector quantisation of n_items
 * vectors x [n_items][dim] (device) with group's codebooks [stages][codewords]
 * [dim] (device; group->idx and ->raw are ignored).  Stage s = 0..L-1 picks
 *   idx[s][n] = argmin_k || C^s[k] - (x_n - sum_{t<s} C^t[idx[t][n]]) ||^2,
 * the first minimum on ties; the decision is taken in FP32 in a fixed order
 * (running sum over stages, residual, squared differences summed over
 * components in order, no fused multiply-add).  idx is [stages][n_items]
 * uint8 (device).  If loss (device float[1]) is non-NULL it receives
 *   L = 1/(n K) sum_s sum_n || sg[r_{s,n}] - C^s[idx[s][n]] ||^2,
 * r the residual entering stage s; if dcodebook (device, codebook layout) is
 * non-NULL it receives dL/dC (2/(n K) times the sum of C^s[k] - r over the
 * items assigned to k).  Both are overwritten.  1 <= codewords <= 256,
 * 1 <= dim <= 16, codebooks within 200 KB (100 KB with dcodebook); else
 * VG_ERR_INVALID_ARG.  n_items == 0 writes zeros to loss and dcodebook. */
vg_status vg_rvq_encode(const vg_attr_group* group, int64_t n_items, const float* x, uint8_t* idx, float* loss,
                        float* dcodebook, vg_stream stream);

/* Forward render of n_views (1..64) cameras (HOST array) of one scene in one
 * launch sequence: decode (Eq. 7, 11-12, 14) and project (Eq. 2-3) every
 * Gaussian for every view, bin (Gaussian, tile) pairs and order each tile's
 * list by (FP32 depth, Gaussian index), composite front to back (Eq. 16-18):
 *   C(p) = sum_i c_i a_i T_i,  D(p) = sum_i z_i a_i T_i,  S(p) = sum_i a_i T_i,
 *   T_i = prod_{j<i} (1 - a_j), background 0.
 * C, D, S: output images (layout above); D is not normalised by S.  The ctx
 * keeps what vg_render_bwd needs (final transmittance, last contributor per
 * pixel, the sorted lists); do not reuse the ctx for another forward before
 * the matching backward. */
vg_status vg_render_fwd(vg_scene* scene, const vg_camera* cams, int32_t n_views, const vg_render_params* params,
                        vg_ctx* ctx, float* C, float* D, float* S, vg_stream stream);

/* Backward of the last vg_render_fwd on this ctx (same scene, cameras,
 * params) for upstream images dC, dD, dS (same layout as C, D, S; any may be
 * NULL = zero).  Per-pixel transmittance is recovered back to front from the
 * final transmittance by division, not stored per step.  Writes the scene
 * gradients (*grads, HOST struct of device pointers) and keeps per-view pose
 * partial sums in the ctx for vg_pose_grad. */
vg_status vg_render_bwd(vg_scene* scene, const vg_camera* cams, int32_t n_views, const vg_render_params* params,
                        vg_ctx* ctx, const float* dC, const float* dD, const float* dS,
                        const vg_scene_grads* grads, vg_stream stream);

/* vg_render_fwd and vg_loss_l1 of its images in one pass: the same C, D, S,
 * and the L1 loss gradients and value of Eq. 19's L1 form (the benchmark
 * loss: mean |C - Ct| + w_depth * mean over target depths > 0 of |D - Dt|,
 * with the silhouette gate S > gate of Eq. 21 when gate >= 0), written by
 * the compositing kernel as each pixel is finished: its normalisers (the
 * target depths > 0, and with params->pixel_mask the sampled pixels, which
 * then restrict both means as in vg_loss_l1_masked) are counted by the
 * preprocess before any pixel is composited.  Means run over every pixel of
 * every view of the call; views may differ in size.  Ct [3 per pixel] and
 * Dt [pixel] are DEVICE arrays in the layout of C and D; dC, dD (and dS,
 * zeroed, may be NULL) receive the gradients, loss[0] the value (device
 * float).  The gradient images equal vg_loss_l1's bit for bit; the loss value
 * is summed in another order (one atomic add per tile).  Argument errors
 * (NULL target or output, w_depth < 0) return VG_ERR_INVALID_ARG before any
 * launch; everything else as vg_render_fwd. */
vg_status vg_render_fwd_l1(vg_scene* scene, const vg_camera* cams, int32_t n_views, const vg_render_params* params,
                           vg_ctx* ctx, const float* Ct, const float* Dt, float w_depth, float gate, float* C,
                           float* D, float* S, float* dC, float* dD, float* dS, float* loss, vg_stream stream);

/* Camera pose gradients of the last vg_render_bwd, for the left
 * perturbation T_cw <- exp(xi^) T_cw, xi = (rho, phi): dxi [n_views][6]
 * (rho then phi).  Optional ICP term (Eq. 20): with icp_q [n_views][N][3]
 * (camera-frame targets) and icp_w [n_views][N] (weights, 0 = none), adds
 * the gradient of sum_n w_n |R mu_n + t - q_n|^2 over kept Gaussians and
 * writes that loss per view to icp_loss [n_views] (may be NULL).  Pass
 * icp_q = NULL to skip it. */
vg_status vg_pose_grad(vg_ctx* ctx, int32_t n_views, const float* icp_q, const float* icp_w,
                       float* dxi, float* icp_loss, vg_stream stream);

/* RGB-D frame ingestion.  The method's input is a sequence of RGB-D frames
 * {I_i, D_i} with known intrinsics (Sec. 3, opening paragraph); sensors
 * deliver them as interleaved 8-bit colour and 16-bit depth, and uploading
 * them in that form moves 5 bytes a pixel over the host link instead of the
 * 16 of FP32 images.  This decodes n_views frames of width x height pixels,
 * back to back, on the device:
 *   rgb   uint8  [n_views][height][width][3]  (DEVICE, interleaved R, G, B)
 *   depth uint16 [n_views][height][width]     (DEVICE, depth_scale units a
 *                                              metre; 0 = no measurement)
 *   C     float  [n_views][3][height][width]  (DEVICE, planar: rgb / 255)
 *   D     float  [n_views][height][width]     (DEVICE: depth / depth_scale,
 *                                              0 where there is none, which
 *                                              the L1 losses treat as invalid)
 * in the layout the renderer and the losses use (C, D as vg_render_fwd
 * writes them).  Both quotients are IEEE FP32 divisions.  Enqueued on
 * `stream`; no allocation.  VG_ERR_INVALID_ARG for a NULL pointer,
 * n_views, width or height < 1, or depth_scale not finite and positive. */
vg_status vg_frame_decode(int32_t n_views, int32_t width, int32_t height, const uint8_t* rgb, const uint16_t* depth,
                          float depth_scale, float* C, float* D, vg_stream stream);

/* Upstream gradients of L = mean|C - Ct| + w_depth * mean_{Dt>0}|D - Dt| over
 * n_views views of n_pix pixels each (C, Ct: [n_views][3][n_pix]; D, Dt, S:
 * [n_views][n_pix]); with gate >= 0 only pixels with S > gate contribute
 * (Eq. 21), normalisers unchanged.  Writes dC, dD (dS is zeroed if non-NULL)
 * and the loss value to loss[0] (device float).  sign(0) = 0. */
vg_status vg_loss_l1(int32_t n_views, int64_t n_pix, const float* C, const float* D, const float* S,
                     const float* Ct, const float* Dt, float w_depth, float gate,
                     float* dC, float* dD, float* dS, float* loss, vg_ctx* ctx, vg_stream stream);

/* One Adam step (Kingma & Ba) on up to 16 FP32 arrays in one launch:
 *   m = b1 m + (1-b1) g ; v = b2 v + (1-b2) g^2 ;
 *   p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * `tensors` is a HOST array of n_tensors records of device pointers (m and v
 * caller-allocated, zero before the first step).  The step number t comes
 * from step_dev[0] when step_dev is non-NULL (then incremented on the device,
 * so a captured graph advances it on every replay), else from step_host.
 * zero_grad != 0: grad[i] is set to 0 once read (for a backward that
 * accumulates, vg_render_params.grad_accumulate). */
typedef struct {
    float* param;
    float* grad;
    float* m;
    float* v;
    int64_t n;
    int32_t zero_grad;
} vg_adam_tensor;
vg_status vg_adam_step(const vg_adam_tensor* tensors, int32_t n_tensors, float lr, float beta1, float beta2, float eps,
                       int32_t* step_dev, int32_t step_host, vg_stream stream);

/* Adam step on camera poses from their twist gradients dxi [n_views][6]
 * (rho, phi for the left perturbation exp(xi^) T_cw): the Adam direction d
 * (scaled by lr_trans for rho and lr_rot for phi) moves each pose to
 * T_cw <- exp(-d^) T_cw.  pose [n_views][12] row-major 3x4, m and v
 * [n_views][6] (zero before the first step); step as in vg_adam_step. */
vg_status vg_pose_step(int32_t n_views, float* pose, const float* dxi, float* m, float* v, float lr_rot,
                       float lr_trans, float beta1, float beta2, float eps, int32_t* step_dev, int32_t step_host,
                       vg_stream stream);

/* Number of CUDA kernels libvg has enqueued in this process (host count). */
int64_t vg_launch_count(void);

/* Number of workspace allocations (a ctx buffer created or grown) libvg has
 * made in this process: a serving loop reads it to see whether a launch had
 * to grow a workspace. */
int64_t vg_workspace_allocs(void);

/* vg_loss_l1 over the sampled rays only: pixels with pixel_mask 0 (same
 * layout as vg_render_params.pixel_mask) get zero gradient, and the means
 * run over the sampled pixels (colour) and the sampled pixels with Dt > 0
 * (depth).  pixel_mask = NULL is vg_loss_l1. */
vg_status vg_loss_l1_masked(int32_t n_views, int64_t n_pix, const float* C, const float* D, const float* S,
                            const float* Ct, const float* Dt, const uint8_t* pixel_mask, float w_depth, float gate,
                            float* dC, float* dD, float* dS, float* loss, vg_ctx* ctx, vg_stream stream);

/* Random-ray sampling for the bundle adjustment (Sec. "Tracking and
 * Local-to-Global Bundle Adjustment": rays sampled from the keyframe
 * database): mask[p] = 1 iff SplitMix64((seed + r * 0x9E3779B97F4A7C15) ^ p)
 * >> 11 < floor(rate * 2^53) for p in [0, n), else 0, with r = round_dev[0]
 * when round_dev is non-NULL (a device counter, e.g. an optimiser step, so
 * that a captured graph draws new rays on every replay) else round_host.
 * SplitMix64 is the generator of Steele, Lea and Flood (OOPSLA 2014).
 * VG_ERR_INVALID_ARG for n < 0, a NULL mask or rate outside [0, 1]. */
vg_status vg_sample_rays(uint8_t* mask, int64_t n, double rate, uint64_t seed, const int32_t* round_dev,
                         int32_t round_host, vg_stream stream);

/* vg_loss_l1 without a ctx, for callers that cannot allocate device memory
 * (the paper has no counterpart: this is a library facility).  Making a
 * vg_ctx allocates; code that runs while another framework owns the device
 * allocator, real-time threads that must not risk the device-wide
 * synchronisation of cudaMalloc, or code that only enqueues into streams it
 * does not own, can call this instead.  Same arguments, layout and results as
 * vg_loss_l1 (minus the ctx).  Its scratch -- one valid-pixel counter per view
 * -- is a file-scope device array of VG_NOALLOC_MAX_VIEWS words that every GPU
 * loading the library holds until the process exits; n_views above that limit
 * returns VG_ERR_INVALID_ARG.  It calls no cudaMalloc or cudaFree and clears
 * the counters it uses on `stream` before each use.  The first call on each
 * device (with that device current) looks the array's device address up with
 * cudaGetSymbolAddress; make that first call before any stream capture.  All
 * calls share the array: calls that overlap on the GPU (unordered streams)
 * race on it and must be serialised by the caller.  The array's address is
 * kept per device ordinal for the life of the process, so the call assumes
 * the device's primary context (the CUDA runtime's, which PyTorch uses) and
 * no cudaDeviceReset between calls. */
#define VG_NOALLOC_MAX_VIEWS 256
vg_status vg_loss_l1_noalloc(int32_t n_views, int64_t n_pix, const float* C, const float* D, const float* S,
                             const float* Ct, const float* Dt, float w_depth, float gate,
                             float* dC, float* dD, float* dS, float* loss, vg_stream stream);

/* Projective data association for the ICP term (Eq. 20; the paper's "closest
 * points" q_i, taken here as the target depth map's point on the ray of the
 * pixel each Gaussian mean projects to).  For view v and Gaussian n kept by
 * its mask, with p = T_cw mu in front of the near plane: pixel (px, py) =
 * the nearest integers to (fx x/z + cx, fy y/z + cy); if inside the image,
 * with target depth d = Dt[view][py][px] > 0 and |z - d| < max_dist:
 *   q[v][n] = ((px - cx) d / fx, (py - cy) d / fy, d)  (camera frame),
 *   w[v][n] = weight (the ICP term's lambda, per correspondence);
 * otherwise q = 0, w = 0.  Dt [n_views][H][W], q [n_views][N][3] and
 * w [n_views][N] are device arrays, ready for vg_pose_grad's icp_q/icp_w;
 * params->pose_dev is honoured like in vg_render_fwd. */
vg_status vg_icp_associate(const vg_scene* scene, const vg_camera* cams, int32_t n_views,
                           const vg_render_params* params, const float* Dt, float max_dist, float weight, float* q,
                           float* w, vg_stream stream);

/* The SSIM term the local-to-global bundle adjustment adds to the RGB
 * rendering (Sec. "Tracking and Local-to-Global Bundle Adjustment"; the
 * paper names the loss, this is the structural similarity of Wang et al.):
 * per colour channel, 11x11 Gaussian window (sigma 1.5), zero padding,
 * C1 = 0.01^2, C2 = 0.03^2;  L = 1 - mean SSIM(C, Ct) over the n_views x 3
 * planes of width x height ([view][3][H][W], device).  Writes weight * L to
 * loss[0] and ADDS weight * dL/dC to dC (e.g. after vg_loss_l1 wrote it);
 * either may be NULL.  One kernel per 32x32 tile of a colour plane; the
 * ctx holds only the SSIM sum. */
vg_status vg_ssim_loss(vg_ctx* ctx, int32_t n_views, int32_t width, int32_t height, const float* C, const float* Ct,
                       float weight, float* dC, float* loss, vg_stream stream);

/* Sliding-window online mask (Sec. "Sliding Window-based Online Mask").
 * vg_mask_loss: over the Gaussians visible (an unempty tile rect) in some
 * view of the last vg_render_fwd of `scene` on `ctx` (frustum selection;
 * N_w of them), writes loss[0] = weight/N_w * sum Sig(m_n) (Eq. 13, L_m) and
 * ADDS weight/N_w * Sig'(m_n) to dmask_logit[n] for those n ([N], device;
 * e.g. the mask gradient vg_render_bwd wrote).  Either output may be NULL.
 * vg_mask_prune, at the window bound: every Gaussian whose mask is off
 * (m <= logit(mask_eps), the renderer's own test) or that was seen in the
 * window (seen[n] != 0) but hit fewer than min_hits rays (hit_count[n],
 * both accumulated by vg_render_fwd, see vg_render_params) is removed: its
 * mask logit becomes -inf in the scene's own array (the caller's array for a
 * borrowed scene), so it is culled from then on.  removed [N] (0/1) and
 * n_removed[0] are optional device outputs; hit_count and seen are both
 * given or both NULL (then only the mask decides).  VG_ERR_INVALID_ARG for
 * a scene without mask logits. */
vg_status vg_mask_loss(const vg_scene* scene, vg_ctx* ctx, float weight, float* dmask_logit, float* loss,
                       vg_stream stream);
vg_status vg_mask_prune(vg_scene* scene, const uint32_t* hit_count, const uint32_t* seen, uint32_t min_hits,
                        uint32_t* removed, uint32_t* n_removed, vg_stream stream);

/* Sequential anchor growing and opacity-based anchor removal (Sec.
 * "Sequential Anchor Point Growing", Eq. 10).
 * vg_grow_accumulate, after vg_render_bwd of `scene` on `ctx`: for every
 * (view, Gaussian) pair visible in that forward, ADDS the norm of the loss
 * gradient with respect to the projected mean, sqrt(du^2 + dv^2) in pixel
 * units, to grad_sum[n] and 1 to grad_cnt[n] ([N], device), and the
 * Gaussian's opacity sigmoid(o_n) to opa_sum[a] and 1 to opa_cnt[a] ([A],
 * device; a = n / k).  Either pair of arrays may be NULL (both of a pair).
 * vg_anchor_grow: for levels m = 1..levels, voxel size eps_m = eps_g / 4^(m-1)
 * and threshold tau_m = tau_g * 2^(m-1): every voxel floor(mu / eps_m) (FP32;
 * mu = x_a + O l) whose Gaussians with grad_cnt > 0 have a mean of their
 * averages grad_sum / grad_cnt (FP32) above tau_m, that holds no anchor of
 * the scene and none grown at a coarser level, and that survives the random
 * elimination (kept iff SplitMix64(key ^ (seed + m * 0x9E3779B97F4A7C15))
 * >> 11 >= floor(p_drop * 2^53), key the voxel index packed as
 * (ix + 2^20) << 42 | (iy + 2^20) << 21 | (iz + 2^20)), gets a new anchor at
 * its centre ((index + 0.5) * eps_m, FP32): new_xyz [cap][3] and, if not
 * NULL, new_level [cap] (m) receive up to cap of them in unspecified order;
 * n_new[0] (device) receives how many there were (more than cap: the output
 * is truncated and finer levels saw only the first cap; call again with a
 * larger cap).  The voxel mean is decided exactly: each average enters as
 * rint(avg * 2^32) (clamped to +-2^52) in a 64-bit integer sum compared in
 * FP64 with (tau_m * 2^32) * count; non-finite averages and voxel indices
 * outside [-2^20, 2^20) are skipped.  Workspace: a hash table of
 * 24 bytes x the next power of two >= 2 (A + N + cap) + 1024, in the ctx.
 * vg_anchor_prune: every anchor with opa_cnt[a] > 0 and
 * opa_sum[a] < tau_alpha * opa_cnt[a] (FP32) is removed: the mask logits of
 * its k Gaussians become -inf in the scene's own array; removed [A] (0/1) and
 * n_removed[0] are optional device outputs.
 * Errors: VG_ERR_INVALID_ARG for null arrays, levels outside 1..8,
 * eps_g <= 0, p_drop outside [0, 1], cap < 0, or (prune) a scene without
 * mask logits; vg_grow_accumulate needs a vg_render_bwd of this scene on
 * this ctx. */
vg_status vg_grow_accumulate(const vg_scene* scene, vg_ctx* ctx, float* grad_sum, uint32_t* grad_cnt, float* opa_sum,
                             uint32_t* opa_cnt, vg_stream stream);
vg_status vg_anchor_grow(const vg_scene* scene, vg_ctx* ctx, const float* grad_sum, const uint32_t* grad_cnt,
                         float eps_g, float tau_g, int32_t levels, double p_drop, uint64_t seed, int64_t cap,
                         float* new_xyz, int32_t* new_level, uint32_t* n_new, vg_stream stream);
vg_status vg_anchor_prune(vg_scene* scene, const float* opa_sum, const uint32_t* opa_cnt, float tau_alpha,
                          uint32_t* removed, uint32_t* n_removed, vg_stream stream);

/* Throughput probe for roofline denominators (a measurement facility; the
 * paper has no counterpart).  Enqueues one kernel on `stream` over a grid of
 * (SM count x 8) blocks of 256 threads, each thread running `iters` steps of:
 *   kind 0: 8 independent FP32 fused multiply-adds  (units: FLOP, FMA = 2)
 *   kind 1: 8 independent base-2 exponentials       (units: exponentials)
 *   kind 2: one conflict-free 16-byte shared load   (units: bytes)
 *   kind 3: one float atomic add, a distinct address per thread (units: atomics)
 *   kind 4: one float atomic add, one address per warp          (units: atomics)
 * and writes to *units the work the launch does; time it with events on
 * `stream`.  `buf` is a device array of at least buf_floats >= grid threads
 * floats (kinds 3-4 add into it; kinds 0-2 never write it in practice).
 * VG_ERR_INVALID_ARG for a bad kind, iters < 1 or a small buffer. */
vg_status vg_probe_peak(int32_t kind, int32_t iters, float* buf, int64_t buf_floats, int64_t* units,
                        vg_stream stream);

/* Message for the calling thread's last non-OK status ("" if none). */
const char* vg_last_error(void);

/* Default compositing constants (alpha_max 0.99, alpha_min 1/255, t_min 1e-4,
 * dilation 0.3, sigma_cull 3, clamp_factor 1.3, jacobian_clamp 1, tile 16). */
vg_render_params vg_default_params(void);

#ifdef __cplusplus
}
#endif
#endif /* VG_H */
