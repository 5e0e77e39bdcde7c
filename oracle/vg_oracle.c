/*
 * vg_oracle.c -- plain FP64 CPU oracle of the differentiable tile rasterizer
 * for voxel-anchored, residual-codebook-coded, mask-pruned 3D Gaussians.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  It shares no
 * code with the CUDA library.  It is written for reading, not for speed:
 * every step is the paper's definition spelled out, in the paper's order.
 *
 * What each part follows:
 *   decode      Eq. 7 (anchor + offset * l), Eq. 14 first line (residual
 *               codebook sum over stages), Eq. 11-12 (binary mask: a masked
 *               Gaussian has zero opacity and is removed)
 *   project     Eq. 1-2 (Sigma = R S S^T R^T), Eq. 3 (Sigma' = J W Sigma W^T J^T)
 *   composite   Eq. 16 (colour), Eq. 17 (depth), Eq. 18 (silhouette), front to
 *               back over the per-tile lists of the tile-based splatting the
 *               implementation section names
 *   backward    reverse mode of the above, written by hand, with the per-step
 *               transmittance stored (no division recurrence); pose gradient
 *               for the left perturbation exp(xi^) T_cw
 *   icp         Eq. 20
 *   loss        L1 colour + weighted L1 depth over rays with valid depth
 *               (the benchmark's loss; Eq. 19 has the squared form), optional
 *               silhouette gate of Eq. 21
 *
 * Constants the paper leaves open (per-pixel opacity cap, skip threshold,
 * early-stop transmittance, tile size, 3-sigma radius, low-pass dilation,
 * Jacobian clamp, near plane) arrive as orc_params.
 *
 * Binning decisions are taken in FP32, the kernel's precision, because they
 * turn floating point into integers (tile membership, list order):
 *   mu32_c  = xa_c + (O_c * l_c)
 *   p32_r   = ((W_r0*mu0 + W_r1*mu1) + W_r2*mu2) + t_r
 *   z32     = p32_2 ; the slot is in front iff z32 > near
 *   u32     = (fx * p32_0) / z32 + cx ;  v32 = (fy * p32_1) / z32 + cy
 *   rect    x0 = clamp(floor((u32 - r) / T), 0, TX), x1 = clamp(floor((u32 + r) / T) + 1, 0, TX)
 *   order   ascending (tile, bits of z32, Gaussian index)
 * each operation rounded to nearest FP32, no fused multiply-add.  The radius
 * r = ceil(sigma_cull * sqrt(lambda_max)) uses the FP64 lambda_max; a slot
 * whose sigma_cull*sqrt(lambda_max) lies within r_band (relative) of an
 * integer is flagged "borderline", since an FP32 evaluation may round the
 * other way.
 */
#include "vg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const int GDIM[ORC_NGROUPS] = {3, 4, 1, 3};
#define RADIUS_MAX (1 << 20)

typedef struct {
    double mu[3], ls[3], q[4], ol, rgb[3];
    int active;
} gauss_t;

typedef struct {
    int valid;
    double p[3];          /* camera-space mean */
    double Sc[3][3];      /* camera-frame 3D covariance W Sigma W^T */
    double A, B, C;       /* 2D covariance incl. dilation */
    double conic[3];      /* a, b, c of the inverse 2D covariance */
    double uv[2];
    double opacity;
    double txz, tyz;      /* x/z and y/z as used inside J (after clamping) */
    int unclamped_x, unclamped_y;
    float u32, v32, z32;
    int radius;
    int rect[4];          /* x0 y0 x1 y1 (tiles) */
    int borderline;
    double qerr;          /* relative FP32 error bound of the exponent (per unit of its term magnitudes) */
    int reached;          /* the FP32 projection reached the rect stage */
    int rect64[4];        /* the rect from the FP64 centre, same radius */
} proj_t;

typedef struct {
    double R[3][3], s[3], qn[4], qnorm, Sig[3][3];
} shape_t;

struct orc_ctx {
    orc_scene sc;
    int nv;
    orc_camera* cams;
    orc_params prm;
    int64_t N;
    gauss_t* g;
    shape_t* shp;
    proj_t* pr;
    int* tiles_x;
    int* tiles_y;
    int64_t* tile_base;
    int64_t* pix_base;
    int* win;            /* per view x0, y0, x1, y1: the pixels composited */
    const uint8_t* pmask; /* [n_pix] 0 = pixel not composited (sampled rays); NULL = all (caller-owned) */
    int64_t n_tiles, n_pix;
    int64_t* tile_start;
    int64_t* list;
    int64_t n_pairs;
    uint8_t* tile_ambiguous;
    int64_t* amb_start;   /* [n_tiles + 1]: per tile, the slots whose membership hangs on a borderline radius */
    int64_t* amb_slot;
};

/* ------------------------------------------------------------------------ */
/* decode                                                                    */
/* ------------------------------------------------------------------------ */

void orc_rvq_decode(int L, int K, int dim, const double* cb, const uint8_t* idx, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < dim; ++c) out[i * dim + c] = 0.0;
        for (int s = 0; s < L; ++s) {
            int k = idx[(int64_t)s * n + i];
            if (k >= K) k = K - 1; /* never happens for valid input */
            for (int c = 0; c < dim; ++c) out[i * dim + c] += cb[((int64_t)s * K + k) * dim + c];
        }
    }
}

static void decode_attr(const orc_scene* sc, int grp, int64_t n, int64_t N, double* out)
{
    int d = GDIM[grp];
    if (sc->codebook[grp]) {
        for (int c = 0; c < d; ++c) out[c] = 0.0;
        for (int s = 0; s < sc->L[grp]; ++s) {
            int k = sc->idx[grp][(int64_t)s * N + n];
            for (int c = 0; c < d; ++c) out[c] += sc->codebook[grp][((int64_t)s * sc->K[grp] + k) * d + c];
        }
    } else {
        for (int c = 0; c < d; ++c) out[c] = sc->raw[grp][n * d + c];
    }
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static void quat_to_rot(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------ */
/* projection and binning                                                    */
/* ------------------------------------------------------------------------ */

static void project_slot(const orc_ctx* ctx, int v, int64_t n, proj_t* P)
{
    const orc_camera* cam = &ctx->cams[v];
    const orc_params* prm = &ctx->prm;
    const orc_scene* sc = &ctx->sc;
    const gauss_t* g = &ctx->g[n];
    const shape_t* sh = &ctx->shp[n];
    memset(P, 0, sizeof(*P));
    if (!g->active) return;

    double W[3][3], t[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) W[r][c] = cam->T_cw[r * 4 + c];
        t[r] = cam->T_cw[r * 4 + 3];
    }

    /* FP32 binning quantities */
    int64_t a = n / sc->k, i = n % sc->k;
    float m32[3];
    for (int c = 0; c < 3; ++c) {
        float xa = (float)sc->anchor_xyz[a * 3 + c];
        float o = (float)sc->offsets[(a * sc->k + i) * 3 + c];
        float l = (float)sc->anchor_l[a * 3 + c];
        float ol = o * l;
        m32[c] = xa + ol;
    }
    float p32[3];
    for (int r = 0; r < 3; ++r) {
        float w0 = (float)W[r][0], w1 = (float)W[r][1], w2 = (float)W[r][2], tr = (float)t[r];
        float e0 = w0 * m32[0];
        float e1 = w1 * m32[1];
        float e2 = w2 * m32[2];
        float s01 = e0 + e1;
        float s012 = s01 + e2;
        p32[r] = s012 + tr;
    }
    float z32 = p32[2];
    if (!(z32 > (float)cam->near_plane)) return;
    float fx32 = (float)cam->fx, fy32 = (float)cam->fy, cx32 = (float)cam->cx, cy32 = (float)cam->cy;
    float nu = fx32 * p32[0];
    float nv = fy32 * p32[1];
    float qu = nu / z32;
    float qv = nv / z32;
    P->u32 = qu + cx32;
    P->v32 = qv + cy32;
    P->z32 = z32;

    /* FP64 values */
    double p[3];
    for (int r = 0; r < 3; ++r) p[r] = W[r][0] * g->mu[0] + W[r][1] * g->mu[1] + W[r][2] * g->mu[2] + t[r];
    double x = p[0], y = p[1], z = p[2];
    double limx = prm->clamp_factor * (0.5 * cam->width / cam->fx);
    double limy = prm->clamp_factor * (0.5 * cam->height / cam->fy);
    double txz = x / z, tyz = y / z;
    int ux = 1, uy = 1;
    if (prm->jacobian_clamp) {
        if (txz < -limx) { txz = -limx; ux = 0; }
        if (txz > limx) { txz = limx; ux = 0; }
        if (tyz < -limy) { tyz = -limy; uy = 0; }
        if (tyz > limy) { tyz = limy; uy = 0; }
    }
    double J00 = cam->fx / z, J02 = -cam->fx * txz / z;
    double J11 = cam->fy / z, J12 = -cam->fy * tyz / z;

    double Sc[3][3], T1[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int m = 0; m < 3; ++m) acc += W[r][m] * sh->Sig[m][c];
            T1[r][c] = acc;
        }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int m = 0; m < 3; ++m) acc += T1[r][m] * W[c][m];
            Sc[r][c] = acc;
        }
    /* Sigma' = J Sc J^T with J = [[J00,0,J02],[0,J11,J12]] */
    double Jm[2][3] = {{J00, 0, J02}, {0, J11, J12}};
    double S2[2][2];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double acc = 0;
            for (int m = 0; m < 3; ++m)
                for (int q = 0; q < 3; ++q) acc += Jm[r][m] * Sc[m][q] * Jm[c][q];
            S2[r][c] = acc;
        }
    double A = S2[0][0] + prm->dilation, B = 0.5 * (S2[0][1] + S2[1][0]), C = S2[1][1] + prm->dilation;
    double det = A * C - B * B;
    if (!(det > 0)) return;
    double mid = 0.5 * (A + C);
    double lam = mid + sqrt(fmax(0.0, mid * mid - det));
    double rr = prm->sigma_cull * sqrt(lam);
    if (!(rr < (double)RADIUS_MAX)) rr = RADIUS_MAX;
    int radius = (int)ceil(rr);
    double nearest = floor(rr + 0.5);
    P->borderline = fabs(rr - nearest) <= prm->r_band * rr;
    /* FP32 error of the exponent -1/2 d^T Sigma'^-1 d: a few units in the
     * last place per operation, and rounding the entries of Sigma' (of the
     * size of lambda_max) moves its small eigenvalue by as much, so the
     * error grows with the condition number lambda_max / lambda_min */
    double kappa = lam * lam / det;
    P->qerr = prm->q_ulps * ldexp(1.0, -24) * (1.0 + kappa);
    P->reached = 1;
    {
        double u64 = cam->fx * x / z + cam->cx, v64 = cam->fy * y / z + cam->cy, T = (double)prm->tile;
        int TX = ctx->tiles_x[v], TY = ctx->tiles_y[v];
        int r64[4] = {(int)floor((u64 - radius) / T), (int)floor((v64 - radius) / T),
                      (int)floor((u64 + radius) / T) + 1, (int)floor((v64 + radius) / T) + 1};
        int lim[4] = {TX, TY, TX, TY};
        for (int q = 0; q < 4; ++q) P->rect64[q] = r64[q] < 0 ? 0 : (r64[q] > lim[q] ? lim[q] : r64[q]);
    }

    int TX = ctx->tiles_x[v], TY = ctx->tiles_y[v];
    float Tf = (float)prm->tile, rf = (float)radius;
    float ul = P->u32 - rf, uh = P->u32 + rf, vl = P->v32 - rf, vh = P->v32 + rf;
    int x0 = (int)floorf(ul / Tf), x1 = (int)floorf(uh / Tf) + 1;
    int y0 = (int)floorf(vl / Tf), y1 = (int)floorf(vh / Tf) + 1;
    x0 = x0 < 0 ? 0 : (x0 > TX ? TX : x0);
    x1 = x1 < 0 ? 0 : (x1 > TX ? TX : x1);
    y0 = y0 < 0 ? 0 : (y0 > TY ? TY : y0);
    y1 = y1 < 0 ? 0 : (y1 > TY ? TY : y1);
    P->radius = radius;
    P->rect[0] = x0; P->rect[1] = y0; P->rect[2] = x1; P->rect[3] = y1;
    if (x1 <= x0 || y1 <= y0) return;

    P->valid = 1;
    for (int c = 0; c < 3; ++c) P->p[c] = p[c];
    memcpy(P->Sc, Sc, sizeof(Sc));
    P->A = A; P->B = B; P->C = C;
    P->conic[0] = C / det; P->conic[1] = -B / det; P->conic[2] = A / det;
    P->uv[0] = cam->fx * x / z + cam->cx;
    P->uv[1] = cam->fy * y / z + cam->cy;
    P->opacity = sigmoid(g->ol);
    P->txz = txz; P->tyz = tyz; P->unclamped_x = ux; P->unclamped_y = uy;
}

typedef struct { int64_t key; uint32_t zbits; int64_t n; int64_t slot; } entry_t;

static int cmp_entry(const void* pa, const void* pb)
{
    const entry_t* a = (const entry_t*)pa;
    const entry_t* b = (const entry_t*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->zbits != b->zbits) return a->zbits < b->zbits ? -1 : 1;
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    return 0;
}

static uint32_t float_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

orc_ctx* orc_create(const orc_scene* scene, const orc_camera* cams, int n_views, const orc_params* prm)
{
    if (!scene || !cams || n_views <= 0 || !prm || scene->k <= 0 || scene->n_anchors < 0 || prm->tile <= 0) return NULL;
    orc_ctx* ctx = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    ctx->sc = *scene;
    ctx->nv = n_views;
    ctx->cams = (orc_camera*)malloc(sizeof(orc_camera) * n_views);
    memcpy(ctx->cams, cams, sizeof(orc_camera) * n_views);
    ctx->prm = *prm;
    int64_t N = scene->n_anchors * scene->k;
    ctx->N = N;

    /* decode: Eq. 7, Eq. 14, Eq. 11 */
    ctx->g = (gauss_t*)calloc(N > 0 ? N : 1, sizeof(gauss_t));
    ctx->shp = (shape_t*)calloc(N > 0 ? N : 1, sizeof(shape_t));
    for (int64_t n = 0; n < N; ++n) {
        gauss_t* g = &ctx->g[n];
        int64_t a = n / scene->k, i = n % scene->k;
        for (int c = 0; c < 3; ++c)
            g->mu[c] = scene->anchor_xyz[a * 3 + c] + scene->offsets[(a * scene->k + i) * 3 + c] * scene->anchor_l[a * 3 + c];
        decode_attr(scene, ORC_G_LOGSCALE, n, N, g->ls);
        decode_attr(scene, ORC_G_ROT, n, N, g->q);
        decode_attr(scene, ORC_G_OPACITY, n, N, &g->ol);
        decode_attr(scene, ORC_G_RGB, n, N, g->rgb);
        g->active = scene->mask_logit ? (scene->mask_logit[n] > scene->mask_thr) : 1;

        /* Eq. 2: Sigma = R S S^T R^T */
        shape_t* sh = &ctx->shp[n];
        double qq = g->q[0] * g->q[0] + g->q[1] * g->q[1] + g->q[2] * g->q[2] + g->q[3] * g->q[3];
        sh->qnorm = sqrt(qq);
        if (!(sh->qnorm > 0)) { g->active = 0; continue; }
        for (int c = 0; c < 4; ++c) sh->qn[c] = g->q[c] / sh->qnorm;
        quat_to_rot(sh->qn, sh->R);
        for (int c = 0; c < 3; ++c) sh->s[c] = exp(g->ls[c]);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int m = 0; m < 3; ++m) acc += sh->R[r][m] * sh->s[m] * sh->s[m] * sh->R[c][m];
                sh->Sig[r][c] = acc;
            }
    }

    /* per-view tile grids and image blocks */
    ctx->tiles_x = (int*)malloc(sizeof(int) * n_views);
    ctx->tiles_y = (int*)malloc(sizeof(int) * n_views);
    ctx->tile_base = (int64_t*)malloc(sizeof(int64_t) * (n_views + 1));
    ctx->pix_base = (int64_t*)malloc(sizeof(int64_t) * (n_views + 1));
    ctx->win = (int*)malloc(sizeof(int) * 4 * (n_views > 0 ? n_views : 1));
    for (int v = 0; v < n_views; ++v) {
        ctx->win[4 * v + 0] = 0;
        ctx->win[4 * v + 1] = 0;
        ctx->win[4 * v + 2] = cams[v].width;
        ctx->win[4 * v + 3] = cams[v].height;
    }
    ctx->tile_base[0] = 0;
    ctx->pix_base[0] = 0;
    for (int v = 0; v < n_views; ++v) {
        ctx->tiles_x[v] = (cams[v].width + prm->tile - 1) / prm->tile;
        ctx->tiles_y[v] = (cams[v].height + prm->tile - 1) / prm->tile;
        ctx->tile_base[v + 1] = ctx->tile_base[v] + (int64_t)ctx->tiles_x[v] * ctx->tiles_y[v];
        ctx->pix_base[v + 1] = ctx->pix_base[v] + (int64_t)cams[v].width * cams[v].height;
    }
    ctx->n_tiles = ctx->tile_base[n_views];
    ctx->n_pix = ctx->pix_base[n_views];

    /* projection */
    int64_t slots = (int64_t)n_views * N;
    ctx->pr = (proj_t*)calloc(slots > 0 ? slots : 1, sizeof(proj_t));
    for (int v = 0; v < n_views; ++v)
        for (int64_t n = 0; n < N; ++n) project_slot(ctx, v, n, &ctx->pr[(int64_t)v * N + n]);

    /* binning: every (tile, slot) pair, sorted by (tile, z32 bits, n) */
    int64_t P = 0;
    for (int64_t s = 0; s < slots; ++s)
        if (ctx->pr[s].valid) P += (int64_t)(ctx->pr[s].rect[2] - ctx->pr[s].rect[0]) * (ctx->pr[s].rect[3] - ctx->pr[s].rect[1]);
    entry_t* e = (entry_t*)malloc(sizeof(entry_t) * (P > 0 ? P : 1));
    int64_t w = 0;
    for (int64_t s = 0; s < slots; ++s) {
        const proj_t* pr = &ctx->pr[s];
        if (!pr->valid) continue;
        int v = (int)(s / (N > 0 ? N : 1));
        int64_t n = s - (int64_t)v * N;
        for (int ty = pr->rect[1]; ty < pr->rect[3]; ++ty)
            for (int tx = pr->rect[0]; tx < pr->rect[2]; ++tx) {
                e[w].key = ctx->tile_base[v] + (int64_t)ty * ctx->tiles_x[v] + tx;
                e[w].zbits = float_bits(pr->z32);
                e[w].n = n;
                e[w].slot = s;
                ++w;
            }
    }
    qsort(e, (size_t)P, sizeof(entry_t), cmp_entry);
    ctx->n_pairs = P;
    ctx->list = (int64_t*)malloc(sizeof(int64_t) * (P > 0 ? P : 1));
    ctx->tile_start = (int64_t*)calloc(ctx->n_tiles + 1, sizeof(int64_t));
    for (int64_t j = 0; j < P; ++j) {
        ctx->list[j] = e[j].slot;
        ctx->tile_start[e[j].key + 1]++;
    }
    for (int64_t t = 0; t < ctx->n_tiles; ++t) ctx->tile_start[t + 1] += ctx->tile_start[t];
    free(e);

    /* tiles whose membership depends on a borderline radius: rect(r+1) \ rect(r-1) */
    ctx->tile_ambiguous = (uint8_t*)calloc(ctx->n_tiles > 0 ? ctx->n_tiles : 1, 1);
    for (int64_t s = 0; s < slots; ++s) {
        const proj_t* pr = &ctx->pr[s];
        if (!pr->borderline || pr->z32 == 0.0f) continue;
        int v = (int)(s / (N > 0 ? N : 1));
        int TX = ctx->tiles_x[v], TY = ctx->tiles_y[v];
        int rr[2] = {pr->radius + 1, pr->radius - 1 > 0 ? pr->radius - 1 : 0};
        int rc[2][4];
        float Tf = (float)prm->tile;
        for (int q = 0; q < 2; ++q) {
            float rf = (float)rr[q];
            int x0 = (int)floorf((pr->u32 - rf) / Tf), x1 = (int)floorf((pr->u32 + rf) / Tf) + 1;
            int y0 = (int)floorf((pr->v32 - rf) / Tf), y1 = (int)floorf((pr->v32 + rf) / Tf) + 1;
            rc[q][0] = x0 < 0 ? 0 : (x0 > TX ? TX : x0);
            rc[q][2] = x1 < 0 ? 0 : (x1 > TX ? TX : x1);
            rc[q][1] = y0 < 0 ? 0 : (y0 > TY ? TY : y0);
            rc[q][3] = y1 < 0 ? 0 : (y1 > TY ? TY : y1);
        }
        for (int ty = rc[0][1]; ty < rc[0][3]; ++ty)
            for (int tx = rc[0][0]; tx < rc[0][2]; ++tx) {
                int inner = tx >= rc[1][0] && tx < rc[1][2] && ty >= rc[1][1] && ty < rc[1][3];
                if (!inner) ctx->tile_ambiguous[ctx->tile_base[v] + (int64_t)ty * TX + tx] = 1;
            }
    }
    /* the same (tile, slot) memberships, listed per tile: counted, then filled */
    ctx->amb_start = (int64_t*)calloc(ctx->n_tiles + 1, sizeof(int64_t));
    int64_t n_amb = 0;
    for (int pass = 0; pass < 2; ++pass) {
        int64_t* fill = NULL;
        if (pass == 1) {
            for (int64_t t = 0; t < ctx->n_tiles; ++t) ctx->amb_start[t + 1] += ctx->amb_start[t];
            n_amb = ctx->amb_start[ctx->n_tiles];
            ctx->amb_slot = (int64_t*)malloc(sizeof(int64_t) * (n_amb > 0 ? n_amb : 1));
            fill = (int64_t*)calloc(ctx->n_tiles > 0 ? ctx->n_tiles : 1, sizeof(int64_t));
        }
        for (int64_t s = 0; s < slots; ++s) {
            const proj_t* pr = &ctx->pr[s];
            if (!pr->borderline || pr->z32 == 0.0f) continue;
            int v = (int)(s / (N > 0 ? N : 1));
            int TX = ctx->tiles_x[v], TY = ctx->tiles_y[v];
            int rr[2] = {pr->radius + 1, pr->radius - 1 > 0 ? pr->radius - 1 : 0};
            int rc[2][4];
            float Tf = (float)prm->tile;
            for (int q = 0; q < 2; ++q) {
                float rf = (float)rr[q];
                int x0 = (int)floorf((pr->u32 - rf) / Tf), x1 = (int)floorf((pr->u32 + rf) / Tf) + 1;
                int y0 = (int)floorf((pr->v32 - rf) / Tf), y1 = (int)floorf((pr->v32 + rf) / Tf) + 1;
                rc[q][0] = x0 < 0 ? 0 : (x0 > TX ? TX : x0);
                rc[q][2] = x1 < 0 ? 0 : (x1 > TX ? TX : x1);
                rc[q][1] = y0 < 0 ? 0 : (y0 > TY ? TY : y0);
                rc[q][3] = y1 < 0 ? 0 : (y1 > TY ? TY : y1);
            }
            for (int ty = rc[0][1]; ty < rc[0][3]; ++ty)
                for (int tx = rc[0][0]; tx < rc[0][2]; ++tx) {
                    int inner = tx >= rc[1][0] && tx < rc[1][2] && ty >= rc[1][1] && ty < rc[1][3];
                    if (inner) continue;
                    int64_t t = ctx->tile_base[v] + (int64_t)ty * TX + tx;
                    if (pass == 0) ctx->amb_start[t + 1]++;
                    else ctx->amb_slot[ctx->amb_start[t] + fill[t]++] = s;
                }
        }
        free(fill);
    }
    return ctx;
}

void orc_free(orc_ctx* ctx)
{
    if (!ctx) return;
    free(ctx->cams); free(ctx->g); free(ctx->shp); free(ctx->pr);
    free(ctx->tiles_x); free(ctx->tiles_y); free(ctx->tile_base); free(ctx->pix_base); free(ctx->win);
    free(ctx->tile_start); free(ctx->list); free(ctx->tile_ambiguous);
    free(ctx->amb_start); free(ctx->amb_slot);
    free(ctx);
}

int64_t orc_n_slots(const orc_ctx* ctx) { return (int64_t)ctx->nv * ctx->N; }
int64_t orc_n_pairs(const orc_ctx* ctx) { return ctx->n_pairs; }
int64_t orc_n_tiles(const orc_ctx* ctx) { return ctx->n_tiles; }
int64_t orc_n_pixels(const orc_ctx* ctx) { return ctx->n_pix; }

void orc_set_pixel_mask(orc_ctx* ctx, const uint8_t* mask) { ctx->pmask = mask; }

int orc_set_window(orc_ctx* ctx, int v, int x0, int y0, int x1, int y1)
{
    if (v < 0 || v >= ctx->nv) return -1;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > ctx->cams[v].width) x1 = ctx->cams[v].width;
    if (y1 > ctx->cams[v].height) y1 = ctx->cams[v].height;
    ctx->win[4 * v + 0] = x0;
    ctx->win[4 * v + 1] = y0;
    ctx->win[4 * v + 2] = x1 > x0 ? x1 : x0;
    ctx->win[4 * v + 3] = y1 > y0 ? y1 : y0;
    return 0;
}

void orc_get_proj(const orc_ctx* ctx, double* proj, float* bin32, int32_t* flags)
{
    int64_t slots = (int64_t)ctx->nv * ctx->N;
    for (int64_t s = 0; s < slots; ++s) {
        const proj_t* P = &ctx->pr[s];
        if (proj) {
            double* o = proj + s * 16;
            int64_t n = s % (ctx->N > 0 ? ctx->N : 1);
            o[0] = P->uv[0]; o[1] = P->uv[1]; o[2] = P->p[2];
            o[3] = P->conic[0]; o[4] = P->conic[1]; o[5] = P->conic[2];
            o[6] = P->opacity;
            o[7] = ctx->g[n].rgb[0]; o[8] = ctx->g[n].rgb[1]; o[9] = ctx->g[n].rgb[2];
            o[10] = P->valid; o[11] = P->radius;
            o[12] = P->rect[0]; o[13] = P->rect[1]; o[14] = P->rect[2]; o[15] = P->rect[3];
        }
        if (bin32) { bin32[s * 3 + 0] = P->u32; bin32[s * 3 + 1] = P->v32; bin32[s * 3 + 2] = P->z32; }
        if (flags) flags[s] = P->borderline ? 1 : 0;
    }
}

int64_t orc_rect_fp64_diff(const orc_ctx* ctx, int64_t* n_borderline)
{
    int64_t slots = (int64_t)ctx->nv * ctx->N, diff = 0, nb = 0;
    for (int64_t s = 0; s < slots; ++s) {
        const proj_t* P = &ctx->pr[s];
        if (!P->reached) continue;
        if (P->borderline) ++nb;
        if (memcmp(P->rect, P->rect64, sizeof(P->rect)) != 0) ++diff;
    }
    if (n_borderline) *n_borderline = nb;
    return diff;
}

void orc_get_bins(const orc_ctx* ctx, int64_t* tile_start, int64_t* list)
{
    if (tile_start) memcpy(tile_start, ctx->tile_start, sizeof(int64_t) * (ctx->n_tiles + 1));
    if (list) memcpy(list, ctx->list, sizeof(int64_t) * ctx->n_pairs);
}

void orc_get_decoded(const orc_ctx* ctx, double* out)
{
    for (int64_t n = 0; n < ctx->N; ++n) {
        const gauss_t* g = &ctx->g[n];
        double* o = out + n * 15;
        memcpy(o, g->mu, 3 * sizeof(double));
        memcpy(o + 3, g->ls, 3 * sizeof(double));
        memcpy(o + 6, g->q, 4 * sizeof(double));
        o[10] = g->ol;
        memcpy(o + 11, g->rgb, 3 * sizeof(double));
        o[14] = g->active;
    }
}

/* ------------------------------------------------------------------------ */
/* compositing (Eq. 16-18)                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t slot;
    double alpha, T, G, x, dx, dy;
    int capped;
} step_t;

/* Distance of value x from threshold t in units of the error bound
 * rel * |t| (large when the bound is zero). */
static double band_units(double x, double t, double rel)
{
    double b = rel * fabs(t);
    return b > 0 ? fabs(x - t) / b : 1e300;
}

/* Walk one pixel's list front to back.  Fills steps (if non-NULL) with every
 * blended Gaussian; returns the number of blended steps.
 *
 * Near-threshold bookkeeping (flags, margin): the GPU takes every decision
 * in FP32, this walk in FP64, so each decision is compared with its
 * threshold in units of the FP32 error bound of the quantity that decides it.
 *   exponent power: |error| <= qerr * (sum of the magnitudes of its terms)
 *   alpha (= opacity e^power): relative error <= decision_band + that
 *   transmittance: relative error accumulates alpha / (1 - alpha) times the
 *     relative error of alpha plus two roundings per blended Gaussian.
 * A decision within its bound (margin <= 1) flags the pixel. */
static int walk_pixel(const orc_ctx* ctx, int v, int px, int py, step_t* steps,
                      double out[5], double* T_final, int32_t* n_contrib, int32_t* n_eval, uint8_t* flag,
                      double cabs[3], double* margin_out)
{
    const orc_params* prm = &ctx->prm;
    const double u32 = ldexp(1.0, -24);
    int tile = prm->tile;
    int64_t key = ctx->tile_base[v] + (int64_t)(py / tile) * ctx->tiles_x[v] + px / tile;
    int64_t b = ctx->tile_start[key], e = ctx->tile_start[key + 1];
    double T = 1.0, C0 = 0, C1 = 0, C2 = 0, Dd = 0, Ss = 0, A0 = 0, A1 = 0, A2 = 0;
    double eT = 0.0;         /* relative FP32 error bound of T */
    double margin = 1e300;
    int m = 0;
    int32_t last = 0, evals = 0;
    int64_t stop_slot = -1;  /* the list entry at which the pixel stopped */
    uint8_t f = 0;
    for (int64_t j = b; j < e; ++j) {
        int64_t s = ctx->list[j];
        const proj_t* P = &ctx->pr[s];
        const gauss_t* g = &ctx->g[s % ctx->N];
        ++evals;
        double dx = P->uv[0] - px, dy = P->uv[1] - py;
        double a = P->conic[0], bb = P->conic[1], c = P->conic[2];
        double power = -0.5 * (a * dx * dx + c * dy * dy) - bb * dx * dy;
        double scale = 0.5 * (fabs(a) * dx * dx + fabs(c) * dy * dy) + fabs(bb * dx * dy);
        double perr = P->qerr * scale;                 /* absolute error bound of power */
        double xerr = prm->decision_band + perr;       /* relative error bound of x */
        if (scale > 0) {
            double mu = power < 0 ? -power / perr : 0.0;
            if (mu <= 1.0) f |= 16;
            if (mu < margin) margin = mu;
        }
        if (power > 0) continue;
        double G = exp(power);
        double x = P->opacity * G;
        double m1 = band_units(x, prm->alpha_min, xerr), m2 = band_units(x, prm->alpha_max, xerr);
        if (m1 <= 1.0) f |= 1;
        if (m2 <= 1.0) f |= 2;
        if (m1 < margin) margin = m1;
        if (m2 < margin) margin = m2;
        int capped = x > prm->alpha_max;
        double alpha = capped ? prm->alpha_max : x;
        if (alpha < prm->alpha_min) continue;
        double Tn = T * (1.0 - alpha);
        double ea = capped ? 2.0 * u32 : xerr;
        double eTn = eT + ea * alpha / (1.0 - alpha) + 2.0 * u32;
        double m4 = band_units(Tn, prm->t_min, prm->t_band * eTn);
        if (m4 <= 1.0) f |= 4;
        if (m4 < margin) margin = m4;
        if (Tn < prm->t_min) {
            stop_slot = s;
            break;
        }
        double wgt = alpha * T;
        C0 += g->rgb[0] * wgt; C1 += g->rgb[1] * wgt; C2 += g->rgb[2] * wgt;
        A0 += fabs(g->rgb[0]) * wgt; A1 += fabs(g->rgb[1]) * wgt; A2 += fabs(g->rgb[2]) * wgt;
        Dd += P->p[2] * wgt;
        Ss += wgt;
        if (steps) {
            steps[m].slot = s; steps[m].alpha = alpha; steps[m].T = T; steps[m].G = G; steps[m].x = x;
            steps[m].dx = dx; steps[m].dy = dy; steps[m].capped = capped;
        }
        ++m;
        T = Tn;
        eT = eTn;
        last = (int32_t)(j - b + 1);
    }
    if (ctx->tile_ambiguous[key] && (flag || margin_out)) {
        /* a Gaussian whose membership of this tile hangs on a borderline
         * radius changes the images only where it passes alpha >= alpha_min
         * before the pixel's stop; any of them changes the work counters */
        f |= 32;
        float zs = stop_slot >= 0 ? ctx->pr[stop_slot].z32 : 0.0f;
        int64_t ns = stop_slot >= 0 ? stop_slot % ctx->N : 0;
        for (int64_t q = ctx->amb_start[key]; q < ctx->amb_start[key + 1]; ++q) {
            int64_t s = ctx->amb_slot[q];
            const proj_t* P = &ctx->pr[s];
            if (stop_slot >= 0) {
                int64_t n = s % ctx->N;
                if (P->z32 > zs || (P->z32 == zs && n > ns)) continue;  /* ordered after the stop */
            }
            double dx = P->uv[0] - px, dy = P->uv[1] - py;
            double a = P->conic[0], bb = P->conic[1], c = P->conic[2];
            double power = -0.5 * (a * dx * dx + c * dy * dy) - bb * dx * dy;
            double scale = 0.5 * (fabs(a) * dx * dx + fabs(c) * dy * dy) + fabs(bb * dx * dy);
            double perr = P->qerr * scale;
            if (power > perr) continue;
            double x = P->opacity * exp(power < 0 ? power : 0.0);
            if (x >= prm->alpha_min * (1.0 - prm->decision_band - perr)) {
                f |= 8;
                margin = 0.0;
            }
        }
    }
    out[0] = C0; out[1] = C1; out[2] = C2; out[3] = Dd; out[4] = Ss;
    if (cabs) { cabs[0] = A0; cabs[1] = A1; cabs[2] = A2; }
    if (T_final) *T_final = T;
    if (n_contrib) *n_contrib = last;
    if (n_eval) *n_eval = evals;
    if (flag) *flag = f;
    if (margin_out) *margin_out = margin;
    return m;
}

int64_t orc_forward(orc_ctx* ctx, double* C, double* D, double* S, double* T_final,
                    int32_t* n_contrib, int32_t* n_eval, uint8_t* flags, double* C_abs, double* margin,
                    int threads)
{
    int64_t total = 0;
#ifdef _OPENMP
    if (threads < 1) threads = 1;
#endif
    for (int v = 0; v < ctx->nv; ++v) {
        int Wd = ctx->cams[v].width, Ht = ctx->cams[v].height;
        int64_t pb = ctx->pix_base[v];
        int64_t HW = (int64_t)Wd * Ht;
        int64_t vt = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads) schedule(dynamic, 4) reduction(+ : vt)
#endif
        for (int py = ctx->win[4 * v + 1]; py < ctx->win[4 * v + 3]; ++py)
            for (int px = ctx->win[4 * v + 0]; px < ctx->win[4 * v + 2]; ++px) {
                double out[5], Tf, ca[3], mg;
                int32_t nc, ne;
                uint8_t f;
                int64_t i = (int64_t)py * Wd + px;
                if (ctx->pmask && !ctx->pmask[pb + i]) continue;
                walk_pixel(ctx, v, px, py, NULL, out, &Tf, &nc, &ne, &f, ca, &mg);
                if (C) { C[3 * pb + i] = out[0]; C[3 * pb + HW + i] = out[1]; C[3 * pb + 2 * HW + i] = out[2]; }
                if (C_abs) { C_abs[3 * pb + i] = ca[0]; C_abs[3 * pb + HW + i] = ca[1]; C_abs[3 * pb + 2 * HW + i] = ca[2]; }
                if (margin) margin[pb + i] = mg;
                if (D) D[pb + i] = out[3];
                if (S) S[pb + i] = out[4];
                if (T_final) T_final[pb + i] = Tf;
                if (n_contrib) n_contrib[pb + i] = nc;
                if (n_eval) n_eval[pb + i] = ne;
                if (flags) flags[pb + i] = f;
                vt += ne;
            }
        total += vt;
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* hit counts (sliding-window mask, Eq. 13): per Gaussian, the number of     */
/* (view, pixel) pairs where it is blended; seen: visible (an unempty tile  */
/* rect) in any view.  Both are ADDED to / OR-ed into the caller's arrays.  */
void orc_hit_counts(orc_ctx* ctx, int64_t* hits, int32_t* seen, int threads)
{
    int64_t N = ctx->N;
    if (seen)
        for (int64_t s = 0; s < (int64_t)ctx->nv * N; ++s)
            if (ctx->pr[s].valid) seen[s % N] = 1;
    if (!hits) return;
    int64_t maxlen = 1;
    for (int64_t t = 0; t < ctx->n_tiles; ++t) {
        int64_t l = ctx->tile_start[t + 1] - ctx->tile_start[t];
        if (l > maxlen) maxlen = l;
    }
    if (threads < 1) threads = 1;
    for (int v = 0; v < ctx->nv; ++v) {
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
#endif
        {
            step_t* steps = (step_t*)malloc(sizeof(step_t) * maxlen);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
            for (int py = ctx->win[4 * v + 1]; py < ctx->win[4 * v + 3]; ++py)
                for (int px = ctx->win[4 * v + 0]; px < ctx->win[4 * v + 2]; ++px) {
                    double out[5];
                    if (ctx->pmask && !ctx->pmask[ctx->pix_base[v] + (int64_t)py * ctx->cams[v].width + px]) continue;
                    int m = walk_pixel(ctx, v, px, py, steps, out, NULL, NULL, NULL, NULL, NULL, NULL);
                    for (int i = 0; i < m; ++i) {
                        int64_t n = steps[i].slot % N;
#ifdef _OPENMP
#pragma omp atomic
#endif
                        hits[n] += 1;
                    }
                }
            free(steps);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* backward                                                                  */
/* ------------------------------------------------------------------------ */

/* reverse mode of one pixel's compositing; accumulates into g2d [slots][10] */
static void pixel_backward(const orc_ctx* ctx, int v, int px, int py, step_t* steps,
                           const double gpix[5], double* g2d)
{
    double out[5];
    int m = walk_pixel(ctx, v, px, py, steps, out, NULL, NULL, NULL, NULL, NULL, NULL);
    double suffix = 0.0; /* sum over later steps j of w_j * alpha_j * T_j */
    for (int k = m - 1; k >= 0; --k) {
        const step_t* st = &steps[k];
        const proj_t* P = &ctx->pr[st->slot];
        const gauss_t* g = &ctx->g[st->slot % ctx->N];
        double w = gpix[0] * g->rgb[0] + gpix[1] * g->rgb[1] + gpix[2] * g->rgb[2] + gpix[3] * P->p[2] + gpix[4];
        /* d out / d alpha_k: own term T_k * value, minus every later term
         * scaled by 1/(1-alpha_k) because their transmittance holds (1-alpha_k) */
        double dalpha = st->T * w - suffix / (1.0 - st->alpha);
        suffix += w * st->alpha * st->T;
        double* o = g2d + st->slot * 10;
        double wgt = st->alpha * st->T;
        o[6] += wgt * gpix[0];
        o[7] += wgt * gpix[1];
        o[8] += wgt * gpix[2];
        o[9] += wgt * gpix[3];
        if (st->capped) continue; /* alpha = alpha_max: constant */
        double dpower = st->x * dalpha;      /* d(o e^power)/dpower = o e^power */
        o[5] += st->G * dalpha;              /* d alpha / d opacity */
        double a = P->conic[0], b = P->conic[1], c = P->conic[2];
        double dx = st->dx, dy = st->dy;
        o[0] += dpower * (-(a * dx + b * dy));
        o[1] += dpower * (-(b * dx + c * dy));
        o[2] += dpower * (-0.5 * dx * dx);
        o[3] += dpower * (-dx * dy);
        o[4] += dpower * (-0.5 * dy * dy);
    }
}

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* 2D gradients of one slot -> camera-space mean / covariance gradients,
 * world mean / covariance gradients and the slot's pose-twist gradient. */
static void slot_chain(const orc_ctx* ctx, int v, const proj_t* P, const shape_t* sh, const double* g,
                       double dmu[3], double dSig[3][3], double pose[6])
{
    const orc_camera* cam = &ctx->cams[v];
    double W[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) W[r][c] = cam->T_cw[r * 4 + c];
    double x = P->p[0], y = P->p[1], z = P->p[2];
    double fx = cam->fx, fy = cam->fy;

    /* conic (a,b,c) = inverse of [[A,B],[B,C]] */
    double A = P->A, B = P->B, C = P->C;
    double det = A * C - B * B, i2 = 1.0 / (det * det);
    double da = g[2], db = g[3], dc = g[4];
    double dA = i2 * (-C * C * da + B * C * db - B * B * dc);
    double dB = i2 * (2 * B * C * da - (A * C + B * B) * db + 2 * A * B * dc);
    double dC = i2 * (-B * B * da + A * B * db - A * A * dc);
    double Gp[2][2] = {{dA, 0.5 * dB}, {0.5 * dB, dC}};

    double J00 = fx / z, J02 = -fx * P->txz / z, J11 = fy / z, J12 = -fy * P->tyz / z;
    double J[2][3] = {{J00, 0, J02}, {0, J11, J12}};
    /* dL/dSc = J^T Gp J */
    double dSc[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int m = 0; m < 2; ++m)
                for (int q = 0; q < 2; ++q) acc += J[m][r] * Gp[m][q] * J[q][c];
            dSc[r][c] = acc;
        }
    /* dL/dJ = 2 Gp J Sc */
    double dJ[2][3];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int m = 0; m < 2; ++m)
                for (int q = 0; q < 3; ++q) acc += 2.0 * Gp[r][m] * J[m][q] * P->Sc[q][c];
            dJ[r][c] = acc;
        }
    double du = g[0], dv = g[1], ddepth = g[9];
    double dp[3];
    double dJ02_dx = P->unclamped_x ? -fx / (z * z) : 0.0;
    double dJ12_dy = P->unclamped_y ? -fy / (z * z) : 0.0;
    double dJ02_dz = fx * P->txz / (z * z) + (P->unclamped_x ? fx * x / (z * z * z) : 0.0);
    double dJ12_dz = fy * P->tyz / (z * z) + (P->unclamped_y ? fy * y / (z * z * z) : 0.0);
    dp[0] = du * fx / z + dJ[0][2] * dJ02_dx;
    dp[1] = dv * fy / z + dJ[1][2] * dJ12_dy;
    dp[2] = du * (-fx * x / (z * z)) + dv * (-fy * y / (z * z)) + ddepth
          + dJ[0][0] * (-fx / (z * z)) + dJ[1][1] * (-fy / (z * z)) + dJ[0][2] * dJ02_dz + dJ[1][2] * dJ12_dz;

    /* p = W mu + t ; Sc = W Sigma W^T */
    for (int c = 0; c < 3; ++c) dmu[c] = W[0][c] * dp[0] + W[1][c] * dp[1] + W[2][c] * dp[2];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int m = 0; m < 3; ++m)
                for (int q = 0; q < 3; ++q) acc += W[m][r] * dSc[m][q] * W[q][c];
            dSig[r][c] = acc;
        }
    (void)sh;
    /* left perturbation: p -> p + phi x p + rho ; Sc -> Sc + [phi]x Sc - Sc [phi]x */
    double cr[3];
    cross3(P->p, dp, cr);
    double M[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int m = 0; m < 3; ++m) acc += P->Sc[r][m] * dSc[m][c] - dSc[r][m] * P->Sc[m][c];
            M[r][c] = acc;
        }
    pose[0] = dp[0]; pose[1] = dp[1]; pose[2] = dp[2];
    pose[3] = cr[0] - 2.0 * M[2][1];
    pose[4] = cr[1] - 2.0 * M[0][2];
    pose[5] = cr[2] - 2.0 * M[1][0];
}

void orc_backward(orc_ctx* ctx, const double* dCimg, const double* dDimg, const double* dSimg,
                  double* g2d_out, double* d_anchor_xyz, double* d_anchor_l, double* d_offsets,
                  double* d_attr0, double* d_attr1, double* d_attr2, double* d_attr3,
                  double* d_mask_logit, double* d_pose, int threads)
{
    const orc_scene* sc = &ctx->sc;
    int64_t N = ctx->N, slots = (int64_t)ctx->nv * N;
    if (threads < 1) threads = 1;
#ifndef _OPENMP
    threads = 1;
#endif
    double** part = (double**)malloc(sizeof(double*) * threads);
    for (int t = 0; t < threads; ++t) part[t] = (double*)calloc((slots > 0 ? slots : 1) * 10, sizeof(double));

    int64_t maxlen = 1;
    for (int64_t t = 0; t < ctx->n_tiles; ++t) {
        int64_t l = ctx->tile_start[t + 1] - ctx->tile_start[t];
        if (l > maxlen) maxlen = l;
    }
    for (int v = 0; v < ctx->nv; ++v) {
        int Wd = ctx->cams[v].width, Ht = ctx->cams[v].height;
        int64_t pb = ctx->pix_base[v], HW = (int64_t)Wd * Ht;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
#endif
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            step_t* steps = (step_t*)malloc(sizeof(step_t) * maxlen);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
            for (int py = ctx->win[4 * v + 1]; py < ctx->win[4 * v + 3]; ++py)
                for (int px = ctx->win[4 * v + 0]; px < ctx->win[4 * v + 2]; ++px) {
                    int64_t i = (int64_t)py * Wd + px;
                    if (ctx->pmask && !ctx->pmask[pb + i]) continue;
                    double gp[5];
                    gp[0] = dCimg ? dCimg[3 * pb + i] : 0;
                    gp[1] = dCimg ? dCimg[3 * pb + HW + i] : 0;
                    gp[2] = dCimg ? dCimg[3 * pb + 2 * HW + i] : 0;
                    gp[3] = dDimg ? dDimg[pb + i] : 0;
                    gp[4] = dSimg ? dSimg[pb + i] : 0;
                    pixel_backward(ctx, v, px, py, steps, gp, part[tid]);
                }
            free(steps);
        }
    }
    double* g2d = part[0];
    for (int t = 1; t < threads; ++t)
        for (int64_t j = 0; j < slots * 10; ++j) g2d[j] += part[t][j];
    if (g2d_out) memcpy(g2d_out, g2d, sizeof(double) * slots * 10);

    /* per-Gaussian chain rule, summing over views */
    double* d_attr[4] = {d_attr0, d_attr1, d_attr2, d_attr3};
    for (int grp = 0; grp < 4; ++grp) {
        if (!d_attr[grp]) continue;
        int64_t sz = sc->codebook[grp] ? (int64_t)sc->L[grp] * sc->K[grp] * GDIM[grp] : N * GDIM[grp];
        memset(d_attr[grp], 0, sizeof(double) * sz);
    }
    if (d_anchor_xyz) memset(d_anchor_xyz, 0, sizeof(double) * sc->n_anchors * 3);
    if (d_anchor_l) memset(d_anchor_l, 0, sizeof(double) * sc->n_anchors * 3);
    if (d_offsets) memset(d_offsets, 0, sizeof(double) * N * 3);
    if (d_mask_logit) memset(d_mask_logit, 0, sizeof(double) * N);
    if (d_pose) memset(d_pose, 0, sizeof(double) * ctx->nv * 6);

    for (int64_t n = 0; n < N; ++n) {
        const gauss_t* g = &ctx->g[n];
        const shape_t* sh = &ctx->shp[n];
        if (!g->active) continue;
        double dmu[3] = {0, 0, 0}, dSig[3][3] = {{0}}, dop = 0, drgb[3] = {0, 0, 0};
        for (int v = 0; v < ctx->nv; ++v) {
            int64_t s = (int64_t)v * N + n;
            const proj_t* P = &ctx->pr[s];
            if (!P->valid) continue;
            const double* gg = g2d + s * 10;
            double m1[3], S1[3][3], pose[6];
            slot_chain(ctx, v, P, sh, gg, m1, S1, pose);
            for (int c = 0; c < 3; ++c) dmu[c] += m1[c];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) dSig[r][c] += S1[r][c];
            dop += gg[5];
            drgb[0] += gg[6]; drgb[1] += gg[7]; drgb[2] += gg[8];
            if (d_pose)
                for (int c = 0; c < 6; ++c) d_pose[v * 6 + c] += pose[c];
        }
        /* Sigma = M M^T with M = R diag(s) */
        double Mm[3][3], dM[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Mm[r][c] = sh->R[r][c] * sh->s[c];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int m = 0; m < 3; ++m) acc += (dSig[r][m] + dSig[m][r]) * Mm[m][c];
                dM[r][c] = acc;
            }
        double ds[3], dls[3], dR[3][3];
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int r = 0; r < 3; ++r) acc += dM[r][c] * sh->R[r][c];
            ds[c] = acc;
            dls[c] = acc * sh->s[c];
        }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) dR[r][c] = dM[r][c] * sh->s[c];
        double w = sh->qn[0], x = sh->qn[1], y = sh->qn[2], z = sh->qn[3];
        double Dw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
        double Dx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
        double Dy[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
        double Dz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
        double dqn[4] = {0, 0, 0, 0};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                dqn[0] += dR[r][c] * Dw[r][c];
                dqn[1] += dR[r][c] * Dx[r][c];
                dqn[2] += dR[r][c] * Dy[r][c];
                dqn[3] += dR[r][c] * Dz[r][c];
            }
        double dot = sh->qn[0] * dqn[0] + sh->qn[1] * dqn[1] + sh->qn[2] * dqn[2] + sh->qn[3] * dqn[3];
        double dq[4];
        for (int c = 0; c < 4; ++c) dq[c] = (dqn[c] - sh->qn[c] * dot) / sh->qnorm;
        double o = sigmoid(g->ol);
        double dol = dop * o * (1.0 - o);
        const double* dattr[4] = {dls, dq, &dol, drgb};
        for (int grp = 0; grp < 4; ++grp) {
            if (!d_attr[grp]) continue;
            int d = GDIM[grp];
            if (sc->codebook[grp]) {
                for (int s = 0; s < sc->L[grp]; ++s) {
                    int k = sc->idx[grp][(int64_t)s * N + n];
                    for (int c = 0; c < d; ++c) d_attr[grp][((int64_t)s * sc->K[grp] + k) * d + c] += dattr[grp][c];
                }
            } else {
                for (int c = 0; c < d; ++c) d_attr[grp][n * d + c] = dattr[grp][c];
            }
        }
        /* Eq. 11-12 straight-through mask: hat s = M s, hat alpha = M alpha, M = 1 here */
        if (d_mask_logit && sc->mask_logit) {
            double sm = sigmoid(sc->mask_logit[n]);
            double dM_ = ds[0] * sh->s[0] + ds[1] * sh->s[1] + ds[2] * sh->s[2] + dop * o;
            d_mask_logit[n] = dM_ * sm * (1.0 - sm);
        }
        /* Eq. 7: mu = x_a + O_i * l */
        int64_t a = n / sc->k, i = n % sc->k;
        for (int c = 0; c < 3; ++c) {
            if (d_anchor_xyz) d_anchor_xyz[a * 3 + c] += dmu[c];
            if (d_offsets) d_offsets[(a * sc->k + i) * 3 + c] = dmu[c] * sc->anchor_l[a * 3 + c];
            if (d_anchor_l) d_anchor_l[a * 3 + c] += dmu[c] * sc->offsets[(a * sc->k + i) * 3 + c];
        }
    }
    for (int t = 0; t < threads; ++t) free(part[t]);
    free(part);
}

/* ------------------------------------------------------------------------ */
/* ICP (Eq. 20) and loss                                                     */
/* ------------------------------------------------------------------------ */

void orc_icp(orc_ctx* ctx, const double* q, const double* w, double* loss, double* d_pose)
{
    int64_t N = ctx->N;
    for (int v = 0; v < ctx->nv; ++v) {
        const orc_camera* cam = &ctx->cams[v];
        double L = 0, g[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t n = 0; n < N; ++n) {
            const gauss_t* gs = &ctx->g[n];
            double wn = w[(int64_t)v * N + n];
            if (!gs->active || wn == 0.0) continue;
            double p[3], r[3], cr[3];
            for (int i = 0; i < 3; ++i)
                p[i] = cam->T_cw[i * 4 + 0] * gs->mu[0] + cam->T_cw[i * 4 + 1] * gs->mu[1] + cam->T_cw[i * 4 + 2] * gs->mu[2] + cam->T_cw[i * 4 + 3];
            for (int i = 0; i < 3; ++i) r[i] = p[i] - q[((int64_t)v * N + n) * 3 + i];
            L += wn * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            double gr[3] = {2 * wn * r[0], 2 * wn * r[1], 2 * wn * r[2]};
            cross3(p, gr, cr);
            for (int i = 0; i < 3; ++i) { g[i] += gr[i]; g[3 + i] += cr[i]; }
        }
        if (loss) loss[v] = L;
        if (d_pose)
            for (int i = 0; i < 6; ++i) d_pose[v * 6 + i] += g[i];
    }
}

double orc_loss_l1(int64_t n_pix, const double* C, const double* D, const double* S,
                   const double* Ct, const double* Dt, double w_depth, double gate,
                   double* dC, double* dD)
{
    /* n_pix pixels of a single view: C, Ct are [3][n_pix]; D, S, Dt are [n_pix] */
    int64_t n_valid = 0;
    for (int64_t i = 0; i < n_pix; ++i)
        if (Dt[i] > 0) ++n_valid;
    double Lc = 0, Ld = 0;
    for (int64_t i = 0; i < n_pix; ++i) {
        double m = (gate >= 0 && !(S[i] > gate)) ? 0.0 : 1.0;
        for (int c = 0; c < 3; ++c) {
            double r = C[c * n_pix + i] - Ct[c * n_pix + i];
            Lc += m * fabs(r);
            if (dC) dC[c * n_pix + i] = m * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (3.0 * n_pix);
        }
        double rd = D[i] - Dt[i];
        int valid = Dt[i] > 0;
        if (valid) Ld += m * fabs(rd);
        if (dD) dD[i] = (valid && n_valid > 0) ? m * w_depth * (rd > 0 ? 1.0 : (rd < 0 ? -1.0 : 0.0)) / n_valid : 0.0;
    }
    return Lc / (3.0 * n_pix) + (n_valid > 0 ? w_depth * Ld / n_valid : 0.0);
}
