/*
 * vg_oracle.h -- plain FP64 CPU oracle of the differentiable tile rasterizer
 * for voxel-anchored, residual-codebook-coded, mask-pruned 3D Gaussians.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this library: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * Everything is double precision except the binning decisions, which the
 * method takes in FP32 (see orc_project): tile membership and the
 * front-to-back order are integers decided by floating point, so both
 * sides decide them in the kernel's precision.
 */
#ifndef VG_ORACLE_H
#define VG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_G_LOGSCALE = 0, ORC_G_ROT = 1, ORC_G_OPACITY = 2, ORC_G_RGB = 3, ORC_NGROUPS = 4 };

typedef struct {
    int64_t n_anchors;
    int k;                               /* Gaussians per anchor */
    const double* anchor_xyz;            /* [Na][3] */
    const double* anchor_l;              /* [Na][3] */
    const double* offsets;               /* [Na][k][3] */
    int L[ORC_NGROUPS], K[ORC_NGROUPS];  /* stages, codewords per stage */
    const double* codebook[ORC_NGROUPS]; /* [L][K][dim] or NULL (raw) */
    const uint8_t* idx[ORC_NGROUPS];     /* [L][N] */
    const double* raw[ORC_NGROUPS];      /* [N][dim] when codebook == NULL */
    const double* mask_logit;            /* [N] or NULL (no mask) */
    double mask_thr;                     /* masked iff mask_logit[n] <= mask_thr */
} orc_scene;

typedef struct {
    double fx, fy, cx, cy;
    int width, height;
    double T_cw[12];                     /* row-major 3x4 world -> camera */
    double near_plane;
} orc_camera;

typedef struct {
    double alpha_max, alpha_min, t_min, dilation, sigma_cull, clamp_factor;
    int jacobian_clamp;
    int tile;                            /* 16 */
    double r_band;                       /* relative band flagging a borderline radius */
    double decision_band;                /* relative error floor of an FP32 alpha (opacity, threshold, exp2) */
    double t_band;                       /* safety factor on the transmittance's FP32 error bound */
    double q_ulps;                       /* FP32 units in the last place of the exponent, per unit of
                                            (1 + condition number of the 2D covariance) */
} orc_params;

typedef struct orc_ctx orc_ctx;

/* Eq. 14, first line: out[n][c] = sum over stages s (in order) of cb[s][idx[s][n]][c]. */
void orc_rvq_decode(int L, int K, int dim, const double* cb, const uint8_t* idx, int64_t n, double* out);

/* Decode, project and bin every (view, Gaussian) slot.  Returns NULL on bad input. */
orc_ctx* orc_create(const orc_scene* scene, const orc_camera* cams, int n_views, const orc_params* prm);
void orc_free(orc_ctx* ctx);

int64_t orc_n_slots(const orc_ctx* ctx);
int64_t orc_n_pairs(const orc_ctx* ctx);
int64_t orc_n_tiles(const orc_ctx* ctx);
int64_t orc_n_pixels(const orc_ctx* ctx);

/* Restrict compositing (forward and backward) of view v to the pixels
 * [x0, x1) x [y0, y1) (clipped to the image); the others are skipped (their
 * outputs untouched, their upstream gradients ignored).  Projection, culling
 * and tile lists are those of the whole image.  Default: the whole image.
 * Returns -1 for a bad view. */
int orc_set_window(orc_ctx* ctx, int v, int x0, int y0, int x1, int y1);

/* Composite (forward, backward, hit counts) only the pixels whose entry of
 * mask [n_pix] (views in order, each row-major) is non-zero: the sampled
 * rays of a bundle-adjustment step; the other pixels' outputs are left
 * untouched and their upstream gradients ignored.  The caller keeps mask
 * alive; NULL restores every pixel. */
void orc_set_pixel_mask(orc_ctx* ctx, const uint8_t* mask);

/* Per-slot projection results (slot = view * N + n); any pointer may be NULL.
 * proj: [slots][16] = u, v, depth, conic a, b, c, opacity, r, g, b, valid,
 *        radius, rect x0, y0, x1, y1.  bin32: [slots][3] = FP32 u, v, depth.
 * flags: [slots] bit0 borderline radius. */
void orc_get_proj(const orc_ctx* ctx, double* proj, float* bin32, int32_t* flags);

/* Tile rects from FP64 against FP32 projected centres: among the slots whose
 * FP32 projection reaches the rect stage (in front, positive determinant),
 * the number whose rect from the FP64 centre (u, v) differs from the rect
 * the binning takes from the FP32 centre (same radius); *n_borderline
 * (nullable) receives the number of slots whose radius itself is
 * borderline (r_band). */
int64_t orc_rect_fp64_diff(const orc_ctx* ctx, int64_t* n_borderline);

/* Per-tile lists: tile_start [n_tiles + 1], list [n_pairs] of slot ids, in the
 * (tile, FP32 depth, Gaussian index) order. */
void orc_get_bins(const orc_ctx* ctx, int64_t* tile_start, int64_t* list);

/* Decoded per-Gaussian attributes [N][15]: mu(3) logscale(3) quat(4)
 * opacity-logit(1) rgb(3) active(1). */
void orc_get_decoded(const orc_ctx* ctx, double* out);

/* Forward compositing (Eq. 16-18).  Images are flat, per-view planar blocks:
 * view v occupies pixels [pix_base[v], pix_base[v] + W*H); C holds three
 * planes per view.  Any output pointer may be NULL.
 * flags: a decision of the pixel lies within the FP32 error bound of its
 * threshold -- bit0 alpha near alpha_min, bit1 alpha near the cap, bit2
 * transmittance stop near t_min, bit3 a Gaussian whose tile membership
 * hangs on a borderline radius reaches the pixel (alpha >= alpha_min there,
 * before the pixel's stop), bit4 exponent near zero; bit5 (work counters
 * only) the pixel's tile list may differ by such a Gaussian.
 * C_abs: [3 per pixel, same layout as C] sum over the blended Gaussians of
 * |colour| alpha T, the magnitude of the sum that C is (equal to |C| when
 * the colours share one sign).  margin: [pixels] the smallest distance of
 * any of the pixel's decisions to its threshold, in units of its error
 * bound (flagged iff <= 1).  Returns total evaluated pairs. */
int64_t orc_forward(orc_ctx* ctx, double* C, double* D, double* S, double* T_final,
                    int32_t* n_contrib, int32_t* n_eval, uint8_t* flags, double* C_abs, double* margin,
                    int threads);

/* Hit counts of the sliding-window mask (Eq. 13): hits[n] += the number of
 * (view, pixel) pairs, within each view's window, where Gaussian n is
 * blended; seen[n] = 1 where Gaussian n is visible (an unempty tile rect) in
 * some view.  Either may be NULL. */
void orc_hit_counts(orc_ctx* ctx, int64_t* hits, int32_t* seen, int threads);

/* Reverse mode of the forward for upstream images dC, dD, dS (same layout).
 * Outputs (any may be NULL; all are overwritten):
 *   g2d     [slots][10]: du dv da db dc dopacity dr dg db ddepth
 *   d_anchor_xyz [Na][3], d_anchor_l [Na][3], d_offsets [Na][k][3]
 *   d_attr[g]   codebook gradient [L][K][dim] for coded groups,
 *               per-Gaussian [N][dim] for raw groups
 *   d_mask_logit [N]  (straight-through estimator, Eq. 11)
 *   d_pose [views][6] (rho, phi) for the left perturbation exp(xi^) T_cw */
void orc_backward(orc_ctx* ctx, const double* dC, const double* dD, const double* dS,
                  double* g2d, double* d_anchor_xyz, double* d_anchor_l, double* d_offsets,
                  double* d_attr0, double* d_attr1, double* d_attr2, double* d_attr3,
                  double* d_mask_logit, double* d_pose, int threads);

/* ICP term (Eq. 20) for given camera-frame targets q [views][N][3] and
 * weights w [views][N]: per view loss and pose gradient (added to d_pose). */
void orc_icp(orc_ctx* ctx, const double* q, const double* w, double* loss, double* d_pose);

/* L1 photometric + weighted L1 depth loss over valid depth (target > 0),
 * mean-normalised; optional silhouette gate (S > gate) when gate >= 0. */
double orc_loss_l1(int64_t n_pix, const double* C, const double* D, const double* S,
                   const double* Ct, const double* Dt, double w_depth, double gate,
                   double* dC, double* dD);

#ifdef __cplusplus
}
#endif
#endif
