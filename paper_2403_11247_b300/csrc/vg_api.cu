// vg_api.cu -- the extern "C" boundary of libvg (declared in include/vg.h):
// argument checks, ownership of scenes and workspaces, and the launch
// sequence of each call.  Nothing here synchronises the stream except
// vg_scene_upload, vg_check and vg_ctx_stats.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <sys/mman.h>
#if defined(__x86_64__)
#include <emmintrin.h>
#endif

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vg.h"
#include "vg_internal.h"

using namespace vgk;

#include <atomic>

namespace {
thread_local std::string g_err;
}  // namespace

namespace vgk {
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_ws_allocs{0};  // workspace allocations (DevBuf growth)
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
cudaError_t allow_dynamic_smem(const void* kernel, size_t dynamic_bytes) {
    if (dynamic_bytes == 0) return cudaSuccess;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (fa.sharedSizeBytes + dynamic_bytes <= 48 * 1024) return cudaSuccess;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= dynamic_bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dynamic_bytes);
}
vg_status set_error(vg_status s, const char* msg) {
    g_err = msg;
    return s;
}
}  // namespace vgk

namespace {

vg_status fail(vg_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define VG_CUDA(expr)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess) return fail(VG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    bool pooled = false;  // from the stream-ordered pool (cudaFree of it does not wait for its users)
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) {
            if (pooled) cudaDeviceSynchronize();
            cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
        pooled = false;
    }
    // grow to at least b bytes (contents are not kept).  Stream-ordered: the
    // old buffer is freed after the work already queued on `st` (the ctx's
    // stream, the only one that uses it) and the new one comes from the
    // device's memory pool, so a growth never waits for the work of other
    // streams the way cudaFree does.
    vg_status ensure(size_t b, cudaStream_t st, const char* what) {
        if (b == 0) b = 16;
        if (b <= bytes) return VG_OK;
        if (capturing(st))
            return fail(VG_ERR_CAPACITY, std::string("workspace buffer '") + what +
                                             "' must grow, which cannot happen during stream capture; run once "
                                             "outside capture first");
        // (a call on the legacy stream, as vg_ctx_reserve and vg_ctx_create
        // make, keeps the synchronous free and allocation).  A buffer that
        // has to grow again grows by at least a quarter, so that a workload
        // whose sizes creep up (a server's batches) rarely reallocates.
        if (p) {
            b = std::max(b, bytes + bytes / 4);
            if (pooled && st) {
                if (cudaFreeAsync(p, st) != cudaSuccess) {
                    cudaGetLastError();
                    cudaDeviceSynchronize();
                    cudaFree(p);
                }
                p = nullptr;
                bytes = 0;
                pooled = false;
            } else {
                release();
            }
        }
        pooled = st != nullptr;
        cudaError_t e = pooled ? cudaMallocAsync(&p, b, st) : cudaMalloc(&p, b);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? VG_ERR_OOM : VG_ERR_CUDA,
                        std::string("cudaMalloc(") + what + "): " + cudaGetErrorString(e));
        }
        bytes = b;
        g_ws_allocs.fetch_add(1, std::memory_order_relaxed);
        return VG_OK;
    }
    template <class T>
    T* as() const { return (T*)p; }
};

#define VG_TRY(expr)                     \
    do {                                 \
        vg_status s_ = (expr);           \
        if (s_ != VG_OK) return s_;      \
    } while (0)

constexpr int GDIMS[4] = {3, 4, 1, 3};

// run `expr` (a launch returning cudaError_t) bracketed by profiling events;
// inside stream capture the events become external event nodes of the graph
#define VG_STAGE(id, expr)                                                                          \
    do {                                                                                            \
        cudaEvent_t e0_ = nullptr;                                                                  \
        if (prof_on) {                                                                              \
            e0_ = prof_graph ? ctx->prof.get_graph() : ctx->prof.get();                             \
            if (e0_) cudaEventRecordWithFlags(e0_, st, prof_graph ? cudaEventRecordExternal : 0);   \
        }                                                                                           \
        VG_CUDA(expr);                                                                              \
        if (prof_on && e0_) {                                                                       \
            cudaEvent_t e1_ = prof_graph ? ctx->prof.get_graph() : ctx->prof.get();                 \
            if (e1_) {                                                                              \
                cudaEventRecordWithFlags(e1_, st, prof_graph ? cudaEventRecordExternal : 0);        \
                auto& v_ = prof_graph ? ctx->prof.graph_recs : ctx->prof.recs;                      \
                if (v_.size() < 200000) v_.push_back({(id), e0_, e1_});                             \
            }                                                                                       \
        }                                                                                           \
    } while (0)
const char* GNAMES[4] = {"logscale", "rot", "opacity", "rgb"};

}  // namespace

struct vg_scene {
    SceneDev dev{};
    bool owned = false;
    std::vector<void*> owned_ptrs;
    ~vg_scene() {
        for (void* p : owned_ptrs) cudaFree(p);
    }
};

// CUDA events around each stage, harvested on demand
struct StageProfiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    // records captured into CUDA graphs: their events are graph nodes, so they
    // are never reused and always hold the latest replay's timestamps
    std::vector<Rec> graph_recs;
    std::vector<cudaEvent_t> graph_pool;
    cudaEvent_t get_graph() {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        graph_pool.push_back(e);
        return e;
    }
    cudaEvent_t get() {
        if (used < pool.size()) return pool[used++];
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pool.push_back(e);
        ++used;
        return e;
    }
    void reset() {
        recs.clear();
        used = 0;
    }
    ~StageProfiler() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
        for (cudaEvent_t e : graph_pool) cudaEventDestroy(e);
    }
};

struct vg_ctx {
    StageProfiler prof;
    int64_t pair_cap = 0;
    DevBuf xy, conic_o, rgbd, rect, ntiles, dkey[2], dval[2], g2d, pkey[2], pval[2], ranges, tile_order, Tfin, ncontrib, lookback,
        scratch, state, pose_part, icp_part, loss_scratch, pair_off, chunk_start, blk_count, vis, ssim_ws, grow_ws,
        neval, loss_blk, long_tiles, part_total;
    int final_pair = 0;
    bool have_fwd = false, have_bwd = false;
    // VG_SORT_AUTO's form on this ctx: 0 per-tile sort, 2 global (a list
    // passed VG_TILE_SORT_CAP; for such lists the global radix passes beat
    // the long-list pass's comparison sort)
    int auto_stage = 0;
    int split_S = 1;         // segments per tile list of the last forward (1 = unsplit)
    DevBuf seg_f, seg_u;     // the split passes' per-segment state, kept for the backward
    uint32_t spin_limit = SPIN_LIMIT_DEFAULT;  // unsuccessful polls before a bounded device wait gives up
    bool g2d_clean = false;
    bool fwd_zeroed = false;  // the last forward zeroed the visible slots' gradient rows and the pose sums
    // scratch words known to be zero: a forward leaves every counter it
    // accumulates back at zero (the visible and pair counts are plain
    // stores), so only a fresh or grown scratch needs a memset
    size_t scratch_clean_words = 0;
    Views views{};
    int64_t fwd_N = -1;
    const vg_scene* fwd_scene = nullptr;
    int pose_blocks = 0;
    SceneDev bwd_scene{};
};

extern "C" {

const char* vg_last_error(void) { return g_err.c_str(); }

int64_t vg_launch_count(void) { return (int64_t)g_launches.load(); }

int64_t vg_workspace_allocs(void) { return (int64_t)g_ws_allocs.load(); }

// segments per tile list: the caller's choice, or (0) automatic -- split when
// the views have fewer tiles than the GPU has SMs, into enough segments for
// about two CTAs per SM
static int split_segments(int32_t want, int total_tiles) {
    if (want == 1 || total_tiles <= 0) return 1;
    if (want > 1) return want;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 148;
    }
    if (total_tiles >= sms) return 1;
    return (int)std::min<int64_t>(16, ceil_div((int64_t)2 * sms, total_tiles));
}

vg_render_params vg_default_params(void) {
    vg_render_params p;
    std::memset(&p, 0, sizeof(p));
    p.tile = VG_TILE;
    p.batch = 0;
    p.alpha_max = 0.99f;
    p.alpha_min = 1.0f / 255.0f;
    p.t_min = 1e-4f;
    p.dilation = 0.3f;
    p.sigma_cull = 3.0f;
    p.clamp_factor = 1.3f;
    p.jacobian_clamp = 1;
    p.count_evals = 0;
    p.pose_dev = nullptr;
    return p;
}

// ---------------------------------------------------------------------------
// scenes
// ---------------------------------------------------------------------------

static vg_status check_group(const vg_attr_group& g, int gi, int64_t N) {
    if (g.dim != GDIMS[gi])
        return fail(VG_ERR_INVALID_ARG, std::string("group ") + GNAMES[gi] + ": dim must be " + std::to_string(GDIMS[gi]));
    if (g.stages < 0) return fail(VG_ERR_INVALID_ARG, std::string("group ") + GNAMES[gi] + ": stages < 0");
    if (g.stages > 0) {
        if (g.codewords < 1 || g.codewords > VG_MAX_CODEWORDS)
            return fail(VG_ERR_INVALID_ARG, std::string("group ") + GNAMES[gi] + ": codewords must be in 1..256");
        if (!g.codebook || (N > 0 && !g.idx))
            return fail(VG_ERR_INVALID_ARG, std::string("group ") + GNAMES[gi] + ": null codebook or idx");
    } else if (N > 0 && !g.raw) {
        return fail(VG_ERR_INVALID_ARG, std::string("group ") + GNAMES[gi] + ": null raw array");
    }
    return VG_OK;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

vg_status vg_scene_upload(const vg_scene_desc* d, int32_t flags, vg_stream stream, vg_scene** out) {
    if (!d || !out) return fail(VG_ERR_INVALID_ARG, "vg_scene_upload: null argument");
    *out = nullptr;
    if (flags != VG_SCENE_COPY && flags != VG_SCENE_BORROW) return fail(VG_ERR_INVALID_ARG, "vg_scene_upload: bad flags");
    if (d->n_anchors < 0 || d->k < 1) return fail(VG_ERR_INVALID_ARG, "vg_scene_upload: n_anchors < 0 or k < 1");
    const int64_t N = d->n_anchors * (int64_t)d->k;
    if (N >= (int64_t)1 << 30) return fail(VG_ERR_INVALID_ARG, "vg_scene_upload: more than 2^30 Gaussians");
    const bool off_coded = d->offsets_rvq.stages > 0, l_coded = d->l_rvq.stages > 0;
    if (d->n_anchors > 0 && (!d->anchor_xyz || (!d->anchor_l && !l_coded) || (!d->offsets && !off_coded)))
        return fail(VG_ERR_INVALID_ARG, "vg_scene_upload: null anchor array");
    for (const vg_attr_group* g : {&d->offsets_rvq, &d->l_rvq}) {
        if (g->stages < 0) return fail(VG_ERR_INVALID_ARG, "vg_scene_upload: R-VQ stages < 0");
        if (g->stages > 0 && (g->dim != 3 || g->codewords < 1 || g->codewords > VG_MAX_CODEWORDS || !g->codebook ||
                              (N > 0 && !g->idx)))
            return fail(VG_ERR_INVALID_ARG, "vg_scene_upload: coded offsets / scaling factors need dim 3, "
                                            "1..256 codewords, a codebook and indices");
    }
    const vg_attr_group* gr[4] = {&d->logscale, &d->rot, &d->opacity, &d->rgb};
    for (int gi = 0; gi < 4; ++gi) VG_TRY(check_group(*gr[gi], gi, N));
    if (d->mask_logit && !(d->mask_eps > 0.f && d->mask_eps < 1.f))
        return fail(VG_ERR_INVALID_ARG, "vg_scene_upload: mask_eps must be in (0, 1)");
    {
        // the preprocess stages every codebook in shared memory
        size_t cb_bytes = 0;
        for (int gi = 0; gi < 4; ++gi)
            if (gr[gi]->stages > 0) cb_bytes += (size_t)gr[gi]->stages * gr[gi]->codewords * gr[gi]->dim * 4;
        if (cb_bytes > 200 * 1024)
            return fail(VG_ERR_INVALID_ARG, "vg_scene_upload: codebooks exceed 200 KB in total");
    }
    cudaStream_t st = (cudaStream_t)stream;

    vg_scene* sc = new vg_scene();
    SceneDev& S = sc->dev;
    S.n_anchors = d->n_anchors;
    S.k = d->k;
    S.N = N;
    S.mask_thr = d->mask_logit ? (float)std::log((double)d->mask_eps / (1.0 - (double)d->mask_eps)) : 0.f;

    auto fin = [&](vg_status s) {
        if (s != VG_OK) delete sc;
        return s;
    };
    if (flags == VG_SCENE_BORROW) {
        sc->owned = false;
        const void* ptrs[] = {d->anchor_xyz, d->anchor_l, d->offsets, d->mask_logit};
        for (const void* p : ptrs)
            if (p && !is_device_ptr(p)) return fin(fail(VG_ERR_INVALID_ARG, "VG_SCENE_BORROW needs device pointers"));
        S.xyz = d->anchor_xyz;
        S.l = l_coded ? nullptr : d->anchor_l;
        S.off = off_coded ? nullptr : d->offsets;
        S.mask = d->mask_logit;
        S.Lo = d->offsets_rvq.stages;
        S.Ko = off_coded ? d->offsets_rvq.codewords : 0;
        S.cbo = off_coded ? d->offsets_rvq.codebook : nullptr;
        S.idxo = off_coded ? d->offsets_rvq.idx : nullptr;
        S.Ll = d->l_rvq.stages;
        S.Kl = l_coded ? d->l_rvq.codewords : 0;
        S.cbl = l_coded ? d->l_rvq.codebook : nullptr;
        S.idxl = l_coded ? d->l_rvq.idx : nullptr;
        {
            const void* cp[] = {S.l, S.off, S.cbo, S.idxo, S.cbl, S.idxl};
            for (const void* p : cp)
                if (p && !is_device_ptr(p)) return fin(fail(VG_ERR_INVALID_ARG, "VG_SCENE_BORROW needs device pointers"));
        }
        for (int gi = 0; gi < 4; ++gi) {
            const vg_attr_group& g = *gr[gi];
            S.L[gi] = g.stages;
            S.K[gi] = g.stages > 0 ? g.codewords : 0;
            S.cb[gi] = g.stages > 0 ? g.codebook : nullptr;
            S.idx[gi] = g.stages > 0 ? g.idx : nullptr;
            S.raw[gi] = g.stages > 0 ? nullptr : g.raw;
            const void* gp[] = {S.cb[gi], S.idx[gi], S.raw[gi]};
            for (const void* p : gp)
                if (p && !is_device_ptr(p)) return fin(fail(VG_ERR_INVALID_ARG, "VG_SCENE_BORROW needs device pointers"));
        }
    } else {
        sc->owned = true;
        auto copy = [&](const void* src, size_t bytes, const void** dst) -> vg_status {
            *dst = nullptr;
            if (!src || bytes == 0) return VG_OK;
            void* p = nullptr;
            cudaError_t e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(e == cudaErrorMemoryAllocation ? VG_ERR_OOM : VG_ERR_CUDA, "vg_scene_upload: cudaMalloc");
            }
            sc->owned_ptrs.push_back(p);
            VG_CUDA(cudaMemcpyAsync(p, src, bytes, cudaMemcpyDefault, st));
            *dst = p;
            return VG_OK;
        };
        const size_t Na = (size_t)d->n_anchors;
        VG_TRY(fin(copy(d->anchor_xyz, Na * 3 * 4, (const void**)&S.xyz)));
        if (!l_coded) VG_TRY(fin(copy(d->anchor_l, Na * 3 * 4, (const void**)&S.l)));
        if (!off_coded) VG_TRY(fin(copy(d->offsets, (size_t)N * 3 * 4, (const void**)&S.off)));
        S.Lo = d->offsets_rvq.stages;
        S.Ll = d->l_rvq.stages;
        if (off_coded) {
            S.Ko = d->offsets_rvq.codewords;
            VG_TRY(fin(copy(d->offsets_rvq.codebook, (size_t)S.Lo * S.Ko * 12, (const void**)&S.cbo)));
            VG_TRY(fin(copy(d->offsets_rvq.idx, (size_t)S.Lo * N, (const void**)&S.idxo)));
        }
        if (l_coded) {
            S.Kl = d->l_rvq.codewords;
            VG_TRY(fin(copy(d->l_rvq.codebook, (size_t)S.Ll * S.Kl * 12, (const void**)&S.cbl)));
            VG_TRY(fin(copy(d->l_rvq.idx, (size_t)S.Ll * Na, (const void**)&S.idxl)));
        }
        VG_TRY(fin(copy(d->mask_logit, (size_t)N * 4, (const void**)&S.mask)));
        for (int gi = 0; gi < 4; ++gi) {
            const vg_attr_group& g = *gr[gi];
            S.L[gi] = g.stages;
            S.K[gi] = g.stages > 0 ? g.codewords : 0;
            if (g.stages > 0) {
                VG_TRY(fin(copy(g.codebook, (size_t)g.stages * g.codewords * g.dim * 4, (const void**)&S.cb[gi])));
                VG_TRY(fin(copy(g.idx, (size_t)g.stages * N, (const void**)&S.idx[gi])));
                S.raw[gi] = nullptr;
            } else {
                VG_TRY(fin(copy(g.raw, (size_t)N * g.dim * 4, (const void**)&S.raw[gi])));
                S.cb[gi] = nullptr;
                S.idx[gi] = nullptr;
            }
        }
    }

    VG_CUDA(cudaStreamSynchronize(st));
    *out = sc;
    return VG_OK;
}

vg_status vg_scene_free(vg_scene* scene) {
    if (!scene) return fail(VG_ERR_INVALID_ARG, "vg_scene_free: null scene");
    delete scene;
    return VG_OK;
}

int64_t vg_scene_size(const vg_scene* scene) { return scene ? scene->dev.N : -1; }

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------

vg_status vg_ctx_create(int64_t pair_capacity, vg_ctx** out) {
    if (!out || pair_capacity < 0) return fail(VG_ERR_INVALID_ARG, "vg_ctx_create: bad argument");
    *out = nullptr;
    vg_ctx* c = new vg_ctx();
    vg_status s = c->state.ensure(ST_WORDS * 4, nullptr, "state");
    if (s == VG_OK) s = c->scratch.ensure(SCR_WORDS * 4 + 4096 * 4, nullptr, "scratch");
    if (s == VG_OK) s = c->loss_scratch.ensure(32, nullptr, "loss");
    if (s == VG_OK && cudaMemset(c->loss_scratch.p, 0, 32) != cudaSuccess) s = fail(VG_ERR_CUDA, "cudaMemset");
    if (s != VG_OK) {
        delete c;
        return s;
    }
    if (cudaMemset(c->state.p, 0, c->state.bytes) != cudaSuccess) {
        delete c;
        return fail(VG_ERR_CUDA, "vg_ctx_create: cudaMemset");
    }
    if (pair_capacity > 0) {
        s = vg_ctx_reserve(c, pair_capacity);
        if (s != VG_OK) {
            delete c;
            return s;
        }
    }
    *out = c;
    return VG_OK;
}

vg_status vg_ctx_free(vg_ctx* ctx) {
    if (!ctx) return fail(VG_ERR_INVALID_ARG, "vg_ctx_free: null ctx");
    delete ctx;
    return VG_OK;
}

vg_status vg_ctx_reserve(vg_ctx* ctx, int64_t cap) {
    if (!ctx || cap < 0) return fail(VG_ERR_INVALID_ARG, "vg_ctx_reserve: bad argument");
    if (cap >= ((int64_t)1 << 30)) return fail(VG_ERR_INVALID_ARG, "vg_ctx_reserve: capacity must be below 2^30 pairs");
    if (cap <= ctx->pair_cap) return VG_OK;
    for (int b = 0; b < 2; ++b) {
        VG_TRY(ctx->pkey[b].ensure((size_t)cap * 4, nullptr, "pair keys"));
        VG_TRY(ctx->pval[b].ensure((size_t)cap * 4, nullptr, "pair values"));
    }
    ctx->pair_cap = cap;
    return VG_OK;
}

vg_status vg_ctx_stats(vg_ctx* ctx, vg_stream stream, vg_stats* out) {
    if (!ctx) return fail(VG_ERR_INVALID_ARG, "vg_ctx_stats: null ctx");
    cudaStream_t st = (cudaStream_t)stream;
    VG_CUDA(cudaStreamSynchronize(st));
    uint32_t state[ST_WORDS];
    uint32_t scr[SCR_WORDS];
    VG_CUDA(cudaMemcpy(state, ctx->state.p, sizeof(state), cudaMemcpyDeviceToHost));
    VG_CUDA(cudaMemcpy(scr, ctx->scratch.p, sizeof(scr), cudaMemcpyDeviceToHost));
    if (out) {
        out->pairs = scr[SCR_PAIRS];
        out->pair_capacity = ctx->pair_cap;
        out->visible = scr[SCR_NVIS];
        unsigned long long ev, bl, bw;
        std::memcpy(&ev, state + ST_EVALS, 8);
        std::memcpy(&bl, state + ST_BLENDED, 8);
        std::memcpy(&bw, state + ST_BWD, 8);
        out->evaluated = (int64_t)ev;
        out->blended = (int64_t)bl;
        out->bwd_pairs = (int64_t)bw;
        out->flags = state[ST_ERR];
    }
    return VG_OK;
}

vg_status vg_check(vg_ctx* ctx, vg_stream stream) {
    if (!ctx) return fail(VG_ERR_INVALID_ARG, "vg_check: null ctx");
    vg_stats s;
    VG_TRY(vg_ctx_stats(ctx, stream, &s));
    if (s.flags) {
        VG_CUDA(cudaMemset(ctx->state.as<uint32_t>() + ST_ERR, 0, 4));
        if (s.flags & ERR_WAIT) return fail(VG_ERR_TIMEOUT, "a bounded device wait ran out");
        if (s.flags & ERR_TABLE) return fail(VG_ERR_CAPACITY, "anchor-growing hash table full");
        if (s.flags & ERR_TILE_LONG) {
            ctx->auto_stage = 2;
            if (!(s.flags & ERR_OVERFLOW))
                return fail(VG_ERR_CAPACITY, "a tile list longer than VG_TILE_SORT_LONG_CAP (" +
                                                 std::to_string(VG_TILE_SORT_LONG_CAP) +
                                                 "): this ctx sorts globally from the next forward under VG_SORT_AUTO");
        }
        if (s.flags & ERR_TILE_LIST) {
            ctx->auto_stage = 2;
            if (!(s.flags & ERR_OVERFLOW))
                return fail(VG_ERR_CAPACITY, "a tile list longer than VG_TILE_SORT_CAP (" +
                                                 std::to_string(VG_TILE_SORT_CAP) +
                                                 "): this ctx sorts globally from the next forward under VG_SORT_AUTO");
        }
        return fail(VG_ERR_CAPACITY, "pair buffer too small: " + std::to_string(s.pairs) + " pairs needed, capacity " +
                                         std::to_string(s.pair_capacity));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(VG_ERR_CUDA, cudaGetErrorString(e));
    return VG_OK;
}

vg_status vg_ctx_set_spin_limit(vg_ctx* ctx, uint32_t polls) {
    if (!ctx) return fail(VG_ERR_INVALID_ARG, "vg_ctx_set_spin_limit: null ctx");
    ctx->spin_limit = polls == VG_SPIN_LIMIT_DEFAULT_SENTINEL ? SPIN_LIMIT_DEFAULT : polls;
    return VG_OK;
}

vg_status vg_ctx_reset_counters(vg_ctx* ctx, vg_stream stream) {
    if (!ctx) return fail(VG_ERR_INVALID_ARG, "vg_ctx_reset_counters: null ctx");
    VG_CUDA(cudaMemsetAsync(ctx->state.as<uint32_t>() + ST_EVALS, 0, 24, (cudaStream_t)stream));
    return VG_OK;
}

vg_status vg_ctx_profile(vg_ctx* ctx, int32_t enable) {
    if (!ctx) return fail(VG_ERR_INVALID_ARG, "vg_ctx_profile: null ctx");
    ctx->prof.reset();
    ctx->prof.on = enable != 0;
    return VG_OK;
}

vg_status vg_ctx_profile_read(vg_ctx* ctx, vg_stream stream, double* ms_total, int64_t* launches) {
    if (!ctx || !ms_total || !launches) return fail(VG_ERR_INVALID_ARG, "vg_ctx_profile_read: null argument");
    VG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    for (int i = 0; i < VG_STAGE_COUNT; ++i) {
        ms_total[i] = 0.0;
        launches[i] = 0;
    }
    for (const auto* list : {&ctx->prof.recs, &ctx->prof.graph_recs}) {
        for (const auto& r : *list) {
            float ms = 0.f;
            VG_CUDA(cudaEventSynchronize(r.b));
            if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
                cudaGetLastError();  // a graph record whose graph has not run yet
                continue;
            }
            ms_total[r.stage] += ms;
            launches[r.stage] += 1;
        }
    }
    return VG_OK;
}

vg_status vg_ctx_buffer(const vg_ctx* ctx, int32_t which, const void** ptr, int64_t* bytes) {
    if (!ctx || !ptr || !bytes) return fail(VG_ERR_INVALID_ARG, "vg_ctx_buffer: null argument");
    const DevBuf* b = nullptr;
    switch (which) {
        case VG_BUF_XY: b = &ctx->xy; break;
        case VG_BUF_CONIC: b = &ctx->conic_o; break;
        case VG_BUF_RGBD: b = &ctx->rgbd; break;
        case VG_BUF_RECT: b = &ctx->rect; break;
        case VG_BUF_NTILES: b = &ctx->ntiles; break;
        case VG_BUF_PAIR_KEYS: b = &ctx->pkey[ctx->final_pair]; break;
        case VG_BUF_PAIR_VALS: b = &ctx->pval[ctx->final_pair]; break;
        case VG_BUF_RANGES: b = &ctx->ranges; break;
        case VG_BUF_T_FINAL: b = &ctx->Tfin; break;
        case VG_BUF_N_CONTRIB: b = &ctx->ncontrib; break;
        case VG_BUF_G2D: b = &ctx->g2d; break;
        case VG_BUF_N_EVAL: b = &ctx->neval; break;
        default: return fail(VG_ERR_INVALID_ARG, "vg_ctx_buffer: unknown buffer id");
    }
    *ptr = b->p;
    *bytes = (int64_t)b->bytes;
    return VG_OK;
}

// ---------------------------------------------------------------------------
// decode
// ---------------------------------------------------------------------------

vg_status vg_rvq_decode(const vg_attr_group* g, int64_t n, float* out, vg_stream stream) {
    if (!g || (n > 0 && !out) || n < 0) return fail(VG_ERR_INVALID_ARG, "vg_rvq_decode: null argument or n < 0");
    if (g->dim < 1) return fail(VG_ERR_INVALID_ARG, "vg_rvq_decode: dim < 1");
    if (g->stages > 0) {
        if (g->codewords < 1 || g->codewords > VG_MAX_CODEWORDS)
            return fail(VG_ERR_INVALID_ARG, "vg_rvq_decode: codewords must be in 1..256");
        if (!g->codebook || (n > 0 && !g->idx)) return fail(VG_ERR_INVALID_ARG, "vg_rvq_decode: null codebook or idx");
    } else if (g->stages < 0 || (n > 0 && !g->raw)) {
        return fail(VG_ERR_INVALID_ARG, "vg_rvq_decode: raw group needs raw values");
    }
    VG_CUDA(launch_rvq_decode(g->dim, g->stages, g->codewords, g->codebook, g->idx, g->raw, n, out, (cudaStream_t)stream));
    return VG_OK;
}

// ---------------------------------------------------------------------------
// render
// ---------------------------------------------------------------------------

static vg_status build_views(const vg_camera* cams, int32_t n_views, const vg_render_params* p, Views* V, Consts* cs,
                             int64_t* pixels) {
    if (!cams || !p) return fail(VG_ERR_INVALID_ARG, "null cameras or params");
    if (n_views < 1 || n_views > VG_MAX_VIEWS) return fail(VG_ERR_INVALID_ARG, "n_views must be in 1..64");
    if (p->tile != VG_TILE) return fail(VG_ERR_INVALID_ARG, "params.tile must be 16");
    if (p->ppt_fwd != 0 && p->ppt_fwd != 1 && p->ppt_fwd != 2 && p->ppt_fwd != 4)
        return fail(VG_ERR_INVALID_ARG, "params.ppt_fwd must be 0, 1, 2 or 4");
    if (p->ppt_bwd != 0 && p->ppt_bwd != 1 && p->ppt_bwd != 2 && p->ppt_bwd != 4)
        return fail(VG_ERR_INVALID_ARG, "params.ppt_bwd must be 0, 1, 2 or 4");
    if (p->batch != 0 && p->batch != 64 && p->batch != 128 && p->batch != 256)
        return fail(VG_ERR_INVALID_ARG, "params.batch must be 0, 64, 128 or 256");
    if (p->persist_ctas < 0 || p->persist_ctas > 32)
        return fail(VG_ERR_INVALID_ARG, "params.persist_ctas must be in 0..32");
    if (p->list_split < 0 || p->list_split > SPLIT_MAX)
        return fail(VG_ERR_INVALID_ARG, "params.list_split must be in 0..32");
    if (!(p->alpha_max > 0.f && p->alpha_max < 1.f) || !(p->alpha_min >= 0.f) || !(p->t_min >= 0.f) ||
        !(p->dilation >= 0.f) || !(p->sigma_cull > 0.f) || !(p->clamp_factor > 0.f))
        return fail(VG_ERR_INVALID_ARG, "render params out of range");
    std::memset(V, 0, sizeof(*V));
    std::memset(cs, 0, sizeof(*cs));  // every optional feature off unless set below or by the caller
    V->n = n_views;
    V->pose_dev = p->pose_dev;
    int64_t tb = 0, pb = 0;
    for (int v = 0; v < n_views; ++v) {
        const vg_camera& c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 65535 * VG_TILE || c.height > 65535 * VG_TILE)
            return fail(VG_ERR_INVALID_ARG, "camera size out of range");
        if (!(c.fx > 0.f && c.fy > 0.f) || !(c.near_plane > 0.f))
            return fail(VG_ERR_INVALID_ARG, "camera focal lengths and near plane must be positive");
        ViewInfo& vi = V->v[v];
        vi.fx = c.fx;
        vi.fy = c.fy;
        vi.cx = c.cx;
        vi.cy = c.cy;
        std::memcpy(vi.T, c.T_cw, sizeof(vi.T));
        vi.near_plane = c.near_plane;
        vi.limx = p->clamp_factor * (0.5f * c.width / c.fx);
        vi.limy = p->clamp_factor * (0.5f * c.height / c.fy);
        vi.W = c.width;
        vi.H = c.height;
        vi.tiles_x = (c.width + VG_TILE - 1) / VG_TILE;
        vi.tiles_y = (c.height + VG_TILE - 1) / VG_TILE;
        vi.tile_base = (int32_t)tb;
        vi.pix_base = pb;
        tb += (int64_t)vi.tiles_x * vi.tiles_y;
        pb += (int64_t)c.width * c.height;
    }
    if (tb >= ((int64_t)1 << 24)) return fail(VG_ERR_INVALID_ARG, "too many tiles in one call");
    V->total_tiles = (int32_t)tb;
    cs->alpha_max = p->alpha_max;
    cs->alpha_min = p->alpha_min;
    cs->t_min = p->t_min;
    cs->dilation = p->dilation;
    cs->sigma_cull = p->sigma_cull;
    cs->jacobian_clamp = p->jacobian_clamp;
    cs->hit_count = p->hit_count;
    cs->seen = p->seen;
    cs->depth_hist = 1;
    cs->pix_mask = p->pixel_mask;
    cs->blend_batch = p->batch ? p->batch : 256;
    if (p->sort_mode < VG_SORT_AUTO || p->sort_mode > VG_SORT_TILE)
        return fail(VG_ERR_INVALID_ARG, "sort_mode must be VG_SORT_AUTO, VG_SORT_GLOBAL or VG_SORT_TILE");
    cs->n_gauss = 0;  // set by the caller that knows the scene
    *pixels = pb;
    return VG_OK;
}

static int tile_passes_for(int total_tiles) {
    int bits = 1;
    while ((1 << bits) < total_tiles) ++bits;
    return (bits + 7) / 8;
}

// the L1 loss a forward computes in its compositing epilogue (vg_render_fwd_l1)
struct FusedLoss {
    const float *Ct, *Dt;
    float *dC, *dD, *dS, *loss;
    float w_depth, gate;
};

static vg_status render_forward(vg_scene* scene, const vg_camera* cams, int32_t n_views,
                                const vg_render_params* params, vg_ctx* ctx, float* C, float* D, float* S,
                                const FusedLoss* lf, vg_stream stream) {
    if (!scene || !ctx || !C || !D || !S) return fail(VG_ERR_INVALID_ARG, "vg_render_fwd: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    Views V;
    Consts cs;
    int64_t pixels = 0;
    VG_TRY(build_views(cams, n_views, params, &V, &cs, &pixels));
    cs.n_gauss = scene->dev.N;
    if (lf) {
        cs.lf_on = 1;
        cs.lf_Ct = lf->Ct;
        cs.lf_Dt = lf->Dt;
        cs.lf_dC = lf->dC;
        cs.lf_dD = lf->dD;
        cs.lf_dS = lf->dS;
        cs.lf_loss = lf->loss;
        cs.lf_pixels = pixels;
        cs.lf_wdepth = lf->w_depth;
        cs.lf_gate = lf->gate;
    }
    const SceneDev& sd = scene->dev;
    const int64_t N = sd.N;
    const int64_t slots = N * n_views;
    if (slots >= ((int64_t)1 << 30)) return fail(VG_ERR_INVALID_ARG, "vg_render_fwd: views x Gaussians >= 2^30");
    if (ctx->pair_cap < 1) VG_TRY(vg_ctx_reserve(ctx, std::max<int64_t>(1024, slots * 8)));

    VG_TRY(ctx->xy.ensure(slots * 16, st, "xy"));
    VG_TRY(ctx->conic_o.ensure(slots * 16, st, "conic"));
    VG_TRY(ctx->rgbd.ensure(slots * 16, st, "rgbd"));
    VG_TRY(ctx->rect.ensure(slots * 8, st, "rect"));
    VG_TRY(ctx->ntiles.ensure(slots * 4, st, "ntiles"));
    VG_TRY(ctx->pair_off.ensure((slots + 1) * 4, st, "pair offsets"));
    VG_TRY(ctx->chunk_start.ensure((size_t)ceil_div(std::max<int64_t>(ctx->pair_cap, 1), EMIT_CHUNK) * 4, st,
                                   "pair chunk starts"));
    VG_TRY(ctx->blk_count.ensure((size_t)preprocess_blocks(N) * 8, st, "block counts"));
    const int lf_grid = compact_grid(N, cs);
    if (lf) {
        VG_TRY(ctx->loss_blk.ensure((size_t)lf_grid * 8, st, "loss block counts"));
        cs.lf_blk = ctx->loss_blk.as<uint32_t>();
    }

    for (int b = 0; b < 2; ++b) {
        VG_TRY(ctx->dkey[b].ensure(slots * 4, st, "depth keys"));
        VG_TRY(ctx->dval[b].ensure(slots * 4, st, "depth values"));
    }
    VG_TRY(ctx->vis.ensure(slots * 4, st, "visible slots"));
    VG_TRY(ctx->part_total.ensure((size_t)ceil_div(slots, DUP_TILE) * 4, st, "pair partition totals"));
    VG_TRY(ctx->ranges.ensure((size_t)V.total_tiles * 8, st, "ranges"));
    VG_TRY(ctx->tile_order.ensure((size_t)V.total_tiles * 4, st, "tile order"));
    const size_t scr_words = (size_t)SCR_WORDS + 2 * (size_t)V.total_tiles;
    if (ctx->scratch.bytes < scr_words * 4) ctx->scratch_clean_words = 0;
    VG_TRY(ctx->scratch.ensure(scr_words * 4, st, "scratch"));
    VG_TRY(ctx->pose_part.ensure((size_t)n_views * 6 * 4, st, "pose sums"));
    VG_TRY(ctx->Tfin.ensure(pixels * 4, st, "T_final"));
    VG_TRY(ctx->ncontrib.ensure(pixels * 4, st, "n_contrib"));
    VG_TRY(ctx->neval.ensure(pixels * 4, st, "n_eval"));  // written by forwards with count_evals
    const int64_t lb_parts = std::max(ceil_div(slots, SORT_TILE), ceil_div(ctx->pair_cap, SORT_TILE));
    const int64_t lb_entries = std::max(lb_parts * 256, ceil_div(slots, DUP_TILE));
    if (ctx->lookback.bytes < (size_t)lb_entries * 8) {
        VG_TRY(ctx->lookback.ensure(lb_entries * 8, st, "lookback"));
        VG_CUDA(cudaMemsetAsync(ctx->lookback.p, 0, ctx->lookback.bytes, st));
    }

    uint32_t* scr = ctx->scratch.as<uint32_t>();
    uint32_t* state = ctx->state.as<uint32_t>();
    uint32_t* err = state + ST_ERR;
    if (lf) cs.lf_counts = scr + SCR_LOSS_VALID;
    unsigned long long* lb = ctx->lookback.as<unsigned long long>();
    const bool tile_sort = params->sort_mode == VG_SORT_TILE ||
                           (params->sort_mode == VG_SORT_AUTO && ctx->auto_stage < 2);
    const bool long_pass = tile_sort && params->sort_mode == VG_SORT_TILE;
    cs.long_sorted = long_pass ? 1 : 0;
    if (long_pass) VG_TRY(ctx->long_tiles.ensure((size_t)V.total_tiles * 4, st, "long tile lists"));
    cs.depth_hist = tile_sort ? 0 : 1;
    const bool prof_graph = capturing(st);
    const bool prof_on = ctx->prof.on;
    if (ctx->scratch_clean_words < scr_words) {
        VG_STAGE(VG_STAGE_MEMSET, cudaMemsetAsync(scr, 0, scr_words * 4, st));
    }
    // both forms leave every accumulated word back at zero (the per-tile
    // form's scatter counts the tile counts down; the global form's ranges
    // kernel clears its histograms, pass counters and tile counts)
    ctx->scratch_clean_words = std::max(ctx->scratch_clean_words, scr_words);
    VG_STAGE(VG_STAGE_PREPROCESS,
             launch_preprocess(sd, V, cs, ctx->xy.as<float4>(), ctx->conic_o.as<float4>(), ctx->rgbd.as<float4>(),
                               ctx->rect.as<uint2>(), ctx->ntiles.as<uint32_t>(), ctx->dkey[1].as<uint32_t>(), scr,
                               state, ctx->blk_count.as<uint32_t>(), st));
    // depth order of the visible slots: order-preserving compaction, then
    // (global sort) a stable radix sort on the FP32 depth bits (ties keep
    // Gaussian order); with the per-tile sort the compacted order stays and
    // the forward compositing kernel orders each tile's list instead
    const int dgrid = sort_pass_grid((uint32_t)slots);
    const uint32_t cap = (uint32_t)ctx->pair_cap;
    // with the per-tile sort the pairs follow the compacted order, so the
    // compaction also produces their offsets (no separate scan)
    // once the ctx has the backward's gradient rows (after its first
    // backward), the compaction zeroes those of the visible slots, and always
    // the pose sums, so that the backward needs no zeroing pass of its own
    float* g2d_rows = (ctx->g2d_clean && ctx->g2d.bytes >= (size_t)slots * G2D_STRIDE * 4) ? ctx->g2d.as<float>()
                                                                                            : nullptr;
    VG_STAGE(VG_STAGE_DEPTH_SORT, ([&]() -> cudaError_t {
                 cudaError_t e = launch_compact(V, N, ctx->dkey[1].as<uint32_t>(), ctx->blk_count.as<uint32_t>(),
                                                ctx->dkey[0].as<uint32_t>(),
                                                ctx->dval[0].as<uint32_t>(), ctx->vis.as<uint32_t>(),
                                                ctx->ntiles.as<uint32_t>(),
                                                tile_sort ? ctx->pair_off.as<uint32_t>() : nullptr,
                                                ctx->chunk_start.as<uint32_t>(), cap, scr, err, g2d_rows,
                                                ctx->pose_part.as<float>(), n_views * 6, cs, st);
                 if (e != cudaSuccess) return e;
                 for (int p = 0; p < (tile_sort ? 0 : 4); ++p) {
                     const int i = p & 1, o = i ^ 1;
                     e = launch_sort_pass(ctx->dkey[i].as<uint32_t>(), ctx->dval[i].as<uint32_t>(),
                                          ctx->dkey[o].as<uint32_t>(), ctx->dval[o].as<uint32_t>(), scr + SCR_NVIS,
                                          (uint32_t)slots, 8 * p, scr + SCR_DEPTH_HIST + 256 * p, lb,
                                          scr + SCR_CNT_DEPTH + p, state, (uint32_t)p, err, dgrid, ctx->spin_limit,
                                          st);
                     if (e != cudaSuccess) return e;
                 }
                 return cudaSuccess;
             })());
    // pairs in depth order, then stable by tile (global sort); or in slot
    // order, then grouped by tile without order (per-tile sort)
    const int tp = tile_passes_for(V.total_tiles);
    VG_STAGE(VG_STAGE_DUPLICATE,
             launch_duplicate(ctx->dval[0].as<uint32_t>(), ctx->pair_off.as<uint32_t>(),
                              ctx->chunk_start.as<uint32_t>(), tile_sort, ctx->ntiles.as<uint32_t>(),
                              ctx->rect.as<uint2>(), N, V, ctx->pkey[0].as<uint32_t>(), ctx->pval[0].as<uint32_t>(), cap,
                              scr, tile_sort ? 0 : tp, ctx->part_total.as<uint32_t>(), err, slots,
                              ctx->ranges.as<uint2>(), st));
    const int tgrid = sort_pass_grid(cap);
    if (tile_sort && !long_pass && tile_place_fits(V.total_tiles)) {
        // ranges, tile order and grouping by tile in one launch
        VG_STAGE(VG_STAGE_TILE_SORT,
                 launch_tile_place(ctx->pkey[0].as<uint32_t>(), ctx->pval[0].as<uint32_t>(), cap, scr,
                                   V.total_tiles, ctx->ranges.as<uint2>(), ctx->tile_order.as<uint32_t>(), cs.lf_blk,
                                   lf_grid, scr + SCR_LOSS_VALID, ctx->pkey[1].as<uint32_t>(),
                                   ctx->pval[1].as<uint32_t>(), st));
    } else if (tile_sort) {
        VG_STAGE(VG_STAGE_RANGES, launch_ranges(scr, V.total_tiles, ctx->ranges.as<uint2>(),
                                               ctx->tile_order.as<uint32_t>(), 0, cs.lf_blk, lf_grid,
                                               scr + SCR_LOSS_VALID,
                                               long_pass ? ctx->long_tiles.as<uint32_t>() : nullptr, 0, st));
        VG_STAGE(VG_STAGE_TILE_SORT, ([&]() -> cudaError_t {
                     cudaError_t e = launch_tile_scatter(ctx->pkey[0].as<uint32_t>(), ctx->pval[0].as<uint32_t>(),
                                                         scr + SCR_PAIRS, cap, ctx->ranges.as<uint2>(),
                                                         scr + SCR_TILE_COUNTS, ctx->pkey[1].as<uint32_t>(),
                                                         ctx->pval[1].as<uint32_t>(), st);
                     if (e != cudaSuccess || !long_pass) return e;
                     return launch_tile_sort_long(ctx->ranges.as<uint2>(), ctx->long_tiles.as<uint32_t>(),
                                                  scr + SCR_N_LONG, ctx->pval[1].as<uint32_t>(),
                                                  ctx->dkey[1].as<uint32_t>(), err, st);
                 })());
    }
    VG_STAGE(VG_STAGE_TILE_SORT, ([&]() -> cudaError_t {
                 for (int p = 0; p < (tile_sort ? 0 : tp); ++p) {
                     const int i = p & 1, o = i ^ 1;
                     cudaError_t e = launch_sort_pass(
                         ctx->pkey[i].as<uint32_t>(), ctx->pval[i].as<uint32_t>(), ctx->pkey[o].as<uint32_t>(),
                         ctx->pval[o].as<uint32_t>(), scr + SCR_PAIRS, cap, 8 * p, scr + SCR_TILE_HIST + 256 * p, lb,
                         scr + SCR_CNT_TILE + p, state, 5u + (uint32_t)p, err, tgrid, ctx->spin_limit, st);
                     if (e != cudaSuccess) return e;
                 }
                 return cudaSuccess;
             })());
    const int fin = tile_sort ? 1 : (tp & 1);
    ctx->final_pair = fin;
    if (!tile_sort)
        VG_STAGE(VG_STAGE_RANGES, ([&]() -> cudaError_t {
                     cudaError_t e = launch_tile_bounds(ctx->pkey[fin].as<uint32_t>(), scr + SCR_PAIRS, cap,
                                                        ctx->ranges.as<uint2>(), st);
                     if (e != cudaSuccess) return e;
                     return launch_ranges(scr, V.total_tiles, ctx->ranges.as<uint2>(), ctx->tile_order.as<uint32_t>(),
                                          1, cs.lf_blk, lf_grid, scr + SCR_LOSS_VALID, nullptr, 1, st);
                 })());
    // deep lists on few tiles: each list split over S CTAs
    const int split = split_segments(params->list_split, V.total_tiles);
    if (split > 1) {
        const size_t px = (size_t)V.total_tiles * split * TILE_PIX;
        VG_TRY(ctx->seg_f.ensure(px * SPLIT_F * 4, st, "split segment sums"));
        VG_TRY(ctx->seg_u.ensure(px * SPLIT_U * 4, st, "split segment counts"));
        VG_STAGE(VG_STAGE_BLEND_FWD,
                 launch_split_fwd(V, cs, split, ctx->ranges.as<uint2>(), ctx->pval[fin].as<uint32_t>(),
                                  tile_sort ? ctx->dkey[1].as<uint32_t>() : nullptr, err, ctx->xy.as<float4>(),
                                  ctx->conic_o.as<float4>(), ctx->rgbd.as<float4>(), ctx->seg_f.as<float>(),
                                  ctx->seg_u.as<uint32_t>(), C, D, S, ctx->Tfin.as<float>(),
                                  ctx->ncontrib.as<uint32_t>(), (unsigned long long*)(state + ST_EVALS),
                                  (unsigned long long*)(state + ST_BLENDED),
                                  params->count_evals ? ctx->neval.as<uint32_t>() : nullptr, params->count_evals, st));
    } else
    VG_STAGE(VG_STAGE_BLEND_FWD,
             launch_blend_fwd(V, cs, params->ppt_fwd, params->persist_ctas, state + ST_WORK_FWD,
                              ctx->ranges.as<uint2>(), ctx->tile_order.as<uint32_t>(),
                              ctx->pval[fin].as<uint32_t>(), tile_sort ? ctx->dkey[1].as<uint32_t>() : nullptr, err,
                              ctx->xy.as<float4>(), ctx->conic_o.as<float4>(), ctx->rgbd.as<float4>(), C, D, S,
                              ctx->Tfin.as<float>(), ctx->ncontrib.as<uint32_t>(),
                              (unsigned long long*)(state + ST_EVALS), (unsigned long long*)(state + ST_BLENDED),
                              params->count_evals ? ctx->neval.as<uint32_t>() : nullptr, params->count_evals, st));
    ctx->split_S = split;
    ctx->views = V;
    ctx->fwd_N = N;
    ctx->fwd_scene = scene;
    ctx->have_fwd = true;
    ctx->have_bwd = false;
    ctx->fwd_zeroed = g2d_rows != nullptr;
    return VG_OK;
}

vg_status vg_render_fwd(vg_scene* scene, const vg_camera* cams, int32_t n_views, const vg_render_params* params,
                        vg_ctx* ctx, float* C, float* D, float* S, vg_stream stream) {
    return render_forward(scene, cams, n_views, params, ctx, C, D, S, nullptr, stream);
}

vg_status vg_render_fwd_l1(vg_scene* scene, const vg_camera* cams, int32_t n_views, const vg_render_params* params,
                           vg_ctx* ctx, const float* Ct, const float* Dt, float w_depth, float gate, float* C,
                           float* D, float* S, float* dC, float* dD, float* dS, float* loss, vg_stream stream) {
    if (!Ct || !Dt || !dC || !dD || !loss) return fail(VG_ERR_INVALID_ARG, "vg_render_fwd_l1: null argument");
    if (!(w_depth >= 0.f)) return fail(VG_ERR_INVALID_ARG, "vg_render_fwd_l1: w_depth must be >= 0");
    const FusedLoss lf{Ct, Dt, dC, dD, dS, loss, w_depth, gate};
    return render_forward(scene, cams, n_views, params, ctx, C, D, S, &lf, stream);
}

static bool same_views(const Views& a, const Views& b) {
    if (a.n != b.n || a.total_tiles != b.total_tiles) return false;
    for (int v = 0; v < a.n; ++v)
        if (a.v[v].W != b.v[v].W || a.v[v].H != b.v[v].H) return false;
    return true;
}

vg_status vg_render_bwd(vg_scene* scene, const vg_camera* cams, int32_t n_views, const vg_render_params* params,
                        vg_ctx* ctx, const float* dC, const float* dD, const float* dS, const vg_scene_grads* grads,
                        vg_stream stream) {
    if (!scene || !ctx || !grads) return fail(VG_ERR_INVALID_ARG, "vg_render_bwd: null argument");
    if (!ctx->have_fwd || ctx->fwd_scene != scene)
        return fail(VG_ERR_INVALID_ARG, "vg_render_bwd: no matching vg_render_fwd on this ctx");
    cudaStream_t st = (cudaStream_t)stream;
    Views V;
    Consts cs;
    int64_t pixels = 0;
    VG_TRY(build_views(cams, n_views, params, &V, &cs, &pixels));
    if (!same_views(V, ctx->views)) return fail(VG_ERR_INVALID_ARG, "vg_render_bwd: cameras differ from the forward");
    const SceneDev& sd = scene->dev;
    const int64_t N = sd.N, slots = N * n_views;
    if (ctx->g2d.bytes < (size_t)slots * G2D_STRIDE * 4) ctx->g2d_clean = false;
    VG_TRY(ctx->g2d.ensure(slots * G2D_STRIDE * 4, st, "g2d"));

    float* gptr[4] = {grads->logscale, grads->rot, grads->opacity, grads->rgb};

    // the scene-gradient arrays the chain accumulates into, zeroed together
    // with the visible slots' gradient rows before the backward compositing
    ChainOut O;
    std::memset(&O, 0, sizeof(O));
    ZeroList Z;
    std::memset(&Z, 0, sizeof(Z));
    auto zero = [&Z](float* p, int64_t count) {
        if (p && count > 0) {
            Z.p[Z.n] = p;
            Z.count[Z.n++] = count;
        }
    };
    for (int gi = 0; gi < 4; ++gi) {
        if (sd.L[gi] > 0) {
            O.cb[gi] = gptr[gi];
            zero(gptr[gi], (int64_t)sd.L[gi] * sd.K[gi] * GDIMS[gi]);
        } else {
            O.raw[gi] = gptr[gi];
            zero(gptr[gi], N * GDIMS[gi]);
        }
    }
    O.d_xyz = grads->anchor_xyz;
    O.d_l = grads->anchor_l;
    O.d_off = grads->offsets;
    O.d_mask = sd.mask ? grads->mask_logit : nullptr;
    O.pose_sum = ctx->pose_part.as<float>();
    zero(grads->anchor_xyz, sd.n_anchors * 3);
    // coded scaling factors / offsets receive [L][K][3] codebook gradients
    zero(grads->anchor_l, sd.Ll > 0 ? (int64_t)sd.Ll * sd.Kl * 3 : sd.n_anchors * 3);
    zero(grads->offsets, sd.Lo > 0 ? (int64_t)sd.Lo * sd.Ko * 3 : N * 3);
    zero(grads->mask_logit, N);
    if (params->grad_accumulate) Z.n = 0;  // the caller keeps the scene gradients zero

    const bool prof_graph = capturing(st);
    const bool prof_on = ctx->prof.on;
    // the forward's compaction zeroed the visible rows and the pose sums, for
    // this backward only (a second backward of the same forward zeroes again)
    bool rows_zero = ctx->fwd_zeroed;
    ctx->fwd_zeroed = false;
    if (!ctx->g2d_clean) {  // rows of slots that were never visible stay zero from here on
        VG_CUDA(cudaMemsetAsync(ctx->g2d.p, 0, ctx->g2d.bytes, st));
        ctx->g2d_clean = true;
        rows_zero = false;  // (the pose sums still need it)
    }
    if (!rows_zero) zero(O.pose_sum, (int64_t)n_views * 6);
    if (!rows_zero || Z.n > 0)
        VG_STAGE(VG_STAGE_MEMSET, launch_zero_bwd(ctx->vis.as<uint32_t>(), ctx->scratch.as<uint32_t>() + SCR_NVIS,
                                                  rows_zero ? 0u : (uint32_t)slots, ctx->g2d.as<float>(), Z, st));
    if (ctx->split_S > 1)
        VG_STAGE(VG_STAGE_BLEND_BWD,
                 launch_split_bwd(V, cs, ctx->split_S, ctx->ranges.as<uint2>(),
                                  ctx->pval[ctx->final_pair].as<uint32_t>(), ctx->xy.as<float4>(),
                                  ctx->conic_o.as<float4>(), ctx->rgbd.as<float4>(), ctx->seg_f.as<float>(),
                                  ctx->seg_u.as<uint32_t>(), ctx->ncontrib.as<uint32_t>(), dC, dD, dS,
                                  ctx->g2d.as<float>(), (unsigned long long*)(ctx->state.as<uint32_t>() + ST_BWD),
                                  params->count_evals, st));
    else
    VG_STAGE(VG_STAGE_BLEND_BWD,
             launch_blend_bwd(V, cs, params->ppt_bwd, params->persist_ctas, ctx->state.as<uint32_t>() + ST_WORK_BWD,
                              ctx->ranges.as<uint2>(), ctx->tile_order.as<uint32_t>(),
                              ctx->pval[ctx->final_pair].as<uint32_t>(),
                              ctx->xy.as<float4>(), ctx->conic_o.as<float4>(), ctx->rgbd.as<float4>(),
                              ctx->Tfin.as<float>(), ctx->ncontrib.as<uint32_t>(), dC, dD, dS, ctx->g2d.as<float>(),
                              (unsigned long long*)(ctx->state.as<uint32_t>() + ST_BWD), params->count_evals, st));
    VG_STAGE(VG_STAGE_CHAIN, launch_chain(sd, V, cs, ctx->g2d.as<float>(), ctx->vis.as<uint32_t>(),
                                          ctx->scratch.as<uint32_t>() + SCR_NVIS, (uint32_t)slots, O,
                                          &ctx->pose_blocks, st));
    ctx->bwd_scene = sd;
    ctx->views = V;
    ctx->have_bwd = true;
    return VG_OK;
}

vg_status vg_pose_grad(vg_ctx* ctx, int32_t n_views, const float* icp_q, const float* icp_w, float* dxi,
                       float* icp_loss, vg_stream stream) {
    if (!ctx || !dxi) return fail(VG_ERR_INVALID_ARG, "vg_pose_grad: null argument");
    if (!ctx->have_bwd) return fail(VG_ERR_INVALID_ARG, "vg_pose_grad: no vg_render_bwd on this ctx");
    if (n_views != ctx->views.n) return fail(VG_ERR_INVALID_ARG, "vg_pose_grad: n_views differs from the backward");
    if (icp_q && !icp_w) return fail(VG_ERR_INVALID_ARG, "vg_pose_grad: icp_q without icp_w");
    cudaStream_t st = (cudaStream_t)stream;
    const SceneDev& sd = ctx->bwd_scene;
    const float* icp_part = nullptr;
    int nbi = 0;
    const bool prof_graph = capturing(st);
    const bool prof_on = ctx->prof.on;
    if (icp_q) {
        nbi = icp_blocks(sd.N);
        VG_TRY(ctx->icp_part.ensure((size_t)n_views * nbi * 7 * 4, st, "icp partials"));
        VG_STAGE(VG_STAGE_POSE, launch_icp(sd, ctx->views, icp_q, icp_w, ctx->icp_part.as<float>(), nbi, st));
        icp_part = ctx->icp_part.as<float>();
    } else if (icp_loss) {
        VG_CUDA(cudaMemsetAsync(icp_loss, 0, (size_t)n_views * 4, st));
    }
    VG_STAGE(VG_STAGE_POSE, launch_pose_final(n_views, ctx->pose_part.as<float>(), icp_part, nbi, dxi,
                                              icp_q ? icp_loss : nullptr, st));
    return VG_OK;
}

vg_status vg_loss_l1(int32_t n_views, int64_t n_pix, const float* C, const float* D, const float* S, const float* Ct,
                     const float* Dt, float w_depth, float gate, float* dC, float* dD, float* dS, float* loss,
                     vg_ctx* ctx, vg_stream stream) {
    return vg_loss_l1_masked(n_views, n_pix, C, D, S, Ct, Dt, nullptr, w_depth, gate, dC, dD, dS, loss, ctx, stream);
}

vg_status vg_frame_decode(int32_t n_views, int32_t width, int32_t height, const uint8_t* rgb, const uint16_t* depth,
                          float depth_scale, float* C, float* D, vg_stream stream) {
    if (!rgb || !depth || !C || !D || n_views < 1 || width < 1 || height < 1)
        return fail(VG_ERR_INVALID_ARG, "vg_frame_decode: null pointer or empty size");
    if (!(depth_scale > 0.f) || !std::isfinite(depth_scale))
        return fail(VG_ERR_INVALID_ARG, "vg_frame_decode: depth_scale must be finite and positive");
    VG_CUDA(launch_frame_decode(n_views, (int64_t)width * height, rgb, depth, depth_scale, C, D, (cudaStream_t)stream));
    return VG_OK;
}

vg_status vg_sample_rays(uint8_t* mask, int64_t n, double rate, uint64_t seed, const int32_t* round_dev,
                         int32_t round_host, vg_stream stream) {
    if (n < 0 || (n > 0 && !mask) || !(rate >= 0.0 && rate <= 1.0))
        return fail(VG_ERR_INVALID_ARG, "vg_sample_rays: n >= 0, a mask and rate in [0, 1] are needed");
    const unsigned long long keep_below = (unsigned long long)std::floor(rate * 9007199254740992.0);
    VG_CUDA(launch_sample_rays(mask, n, (unsigned long long)seed, round_dev, round_host, keep_below,
                               (cudaStream_t)stream));
    return VG_OK;
}

vg_status vg_loss_l1_masked(int32_t n_views, int64_t n_pix, const float* C, const float* D, const float* S,
                            const float* Ct, const float* Dt, const uint8_t* pixel_mask, float w_depth, float gate,
                            float* dC, float* dD, float* dS, float* loss, vg_ctx* ctx, vg_stream stream) {
    if (!ctx || !C || !D || !Ct || !Dt || !dC || !dD || !loss || n_views < 1 || n_pix < 1)
        return fail(VG_ERR_INVALID_ARG, "vg_loss_l1: null argument or empty size");
    if (gate >= 0.f && !S) return fail(VG_ERR_INVALID_ARG, "vg_loss_l1: gate needs S");
    cudaStream_t st = (cudaStream_t)stream;
    const bool prof_graph = capturing(st);
    const bool prof_on = ctx->prof.on;
    if (dS) VG_CUDA(cudaMemsetAsync(dS, 0, (size_t)n_views * n_pix * 4, st));
    // words 4..7 of the loss scratch: kept zero between calls by the kernels
    VG_STAGE(VG_STAGE_LOSS, launch_loss_l1(n_views, n_pix, C, D, S, Ct, Dt, pixel_mask, w_depth, gate, dC, dD, loss,
                                           ctx->loss_scratch.as<uint32_t>() + 4,
                                           ctx->state.as<uint32_t>() + ST_ERR, ctx->spin_limit, st));
    return VG_OK;
}

vg_status vg_icp_associate(const vg_scene* scene, const vg_camera* cams, int32_t n_views, const vg_render_params* params,
                           const float* Dt, float max_dist, float weight, float* q, float* w, vg_stream stream) {
    if (!scene || !Dt || !q || !w) return fail(VG_ERR_INVALID_ARG, "vg_icp_associate: null argument");
    Views V;
    Consts cs;
    int64_t pixels = 0;
    VG_TRY(build_views(cams, n_views, params, &V, &cs, &pixels));
    return launch_icp_associate(scene->dev, V, Dt, max_dist, weight, q, w, (cudaStream_t)stream);
}

vg_status vg_ssim_loss(vg_ctx* ctx, int32_t n_views, int32_t width, int32_t height, const float* C, const float* Ct,
                       float weight, float* dC, float* loss, vg_stream stream) {
    if (!ctx || !C || !Ct || n_views < 1 || width < 1 || height < 1)
        return fail(VG_ERR_INVALID_ARG, "vg_ssim_loss: null argument or empty size");
    if (n_views > 21845) return fail(VG_ERR_INVALID_ARG, "vg_ssim_loss: more than 21845 views");
    cudaStream_t st = (cudaStream_t)stream;
    VG_TRY(ctx->ssim_ws.ensure(16, st, "ssim sum"));
    return launch_ssim(n_views, width, height, C, Ct, weight, dC, loss, ctx->ssim_ws.as<float>(), st);
}

vg_status vg_mask_loss(const vg_scene* scene, vg_ctx* ctx, float weight, float* dmask_logit, float* loss,
                       vg_stream stream) {
    if (!scene || !ctx) return fail(VG_ERR_INVALID_ARG, "vg_mask_loss: null argument");
    if (!scene->dev.mask) return fail(VG_ERR_INVALID_ARG, "vg_mask_loss: the scene has no mask logits");
    if (!ctx->have_fwd || ctx->fwd_scene != scene)
        return fail(VG_ERR_INVALID_ARG, "vg_mask_loss: no vg_render_fwd of this scene on this ctx");
    uint32_t* su = ctx->loss_scratch.as<uint32_t>();
    return vg_mask_kernels_loss(scene->dev, ctx->views, ctx->ntiles.as<uint32_t>(), weight, dmask_logit, loss, su,
                                reinterpret_cast<float*>(su + 1), (cudaStream_t)stream);
}

vg_status vg_mask_prune(vg_scene* scene, const uint32_t* hit_count, const uint32_t* seen, uint32_t min_hits,
                        uint32_t* removed, uint32_t* n_removed, vg_stream stream) {
    if (!scene) return fail(VG_ERR_INVALID_ARG, "vg_mask_prune: null scene");
    if (!scene->dev.mask) return fail(VG_ERR_INVALID_ARG, "vg_mask_prune: the scene has no mask logits");
    if ((hit_count == nullptr) != (seen == nullptr))
        return fail(VG_ERR_INVALID_ARG, "vg_mask_prune: hit_count and seen go together");
    return vg_mask_kernels_prune(const_cast<float*>(scene->dev.mask), scene->dev.mask_thr, hit_count, seen, min_hits,
                                 scene->dev.N, removed, n_removed, (cudaStream_t)stream);
}

vg_status vg_host_alloc(int64_t bytes, void** out) {
    if (!out || bytes <= 0) return fail(VG_ERR_INVALID_ARG, "vg_host_alloc: bytes must be > 0");
    *out = nullptr;
    const size_t align = (size_t)2 << 20;
    const size_t size = ((size_t)bytes + align - 1) / align * align;
    void* p = nullptr;
    if (posix_memalign(&p, align, size) != 0 || !p) return fail(VG_ERR_OOM, "vg_host_alloc: out of host memory");
    madvise(p, size, MADV_HUGEPAGE);  // a hint: fewer, larger pages for the DMA engine to translate
    std::memset(p, 0, size);
    // portable: page-locked for every CUDA context of the process (the
    // caller's framework may run its own runtime beside this library's)
    cudaError_t e = cudaHostRegister(p, size, cudaHostRegisterPortable);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free(p);
        return fail(VG_ERR_CUDA, std::string("vg_host_alloc: cudaHostRegister: ") + cudaGetErrorString(e));
    }
    *out = p;
    return VG_OK;
}

vg_status vg_host_free(void* ptr) {
    if (!ptr) return VG_OK;
    cudaError_t e = cudaHostUnregister(ptr);
    free(ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(VG_ERR_CUDA, std::string("vg_host_free: cudaHostUnregister: ") + cudaGetErrorString(e));
    }
    return VG_OK;
}

vg_status vg_host_stage(void* dst, const void* src, int64_t bytes) {
    if (bytes < 0 || (bytes > 0 && (!dst || !src))) return fail(VG_ERR_INVALID_ARG, "vg_host_stage: bad arguments");
    char* d = static_cast<char*>(dst);
    const char* s = static_cast<const char*>(src);
    int64_t i = 0;
#if defined(__x86_64__)
    // streaming stores: the data goes to memory, not to this core's caches
    const int64_t head = (int64_t)((16 - (reinterpret_cast<uintptr_t>(d) & 15)) & 15);
    for (; i < head && i < bytes; ++i) d[i] = s[i];
    for (; i + 64 <= bytes; i += 64) {
        const __m128i a = _mm_loadu_si128(reinterpret_cast<const __m128i*>(s + i));
        const __m128i b = _mm_loadu_si128(reinterpret_cast<const __m128i*>(s + i + 16));
        const __m128i c = _mm_loadu_si128(reinterpret_cast<const __m128i*>(s + i + 32));
        const __m128i e = _mm_loadu_si128(reinterpret_cast<const __m128i*>(s + i + 48));
        _mm_stream_si128(reinterpret_cast<__m128i*>(d + i), a);
        _mm_stream_si128(reinterpret_cast<__m128i*>(d + i + 16), b);
        _mm_stream_si128(reinterpret_cast<__m128i*>(d + i + 32), c);
        _mm_stream_si128(reinterpret_cast<__m128i*>(d + i + 48), e);
    }
    for (; i < bytes; ++i) d[i] = s[i];
    _mm_sfence();
#else
    std::memcpy(d, s, (size_t)bytes);
#endif
    return VG_OK;
}

vg_status vg_memcpy_async(void* dst, const void* src, int64_t bytes, vg_stream stream) {
    if (bytes < 0 || (bytes > 0 && (!dst || !src))) return fail(VG_ERR_INVALID_ARG, "vg_memcpy_async: bad arguments");
    if (bytes == 0) return VG_OK;
    VG_CUDA(cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDefault, (cudaStream_t)stream));
    return VG_OK;
}

vg_status vg_grow_accumulate(const vg_scene* scene, vg_ctx* ctx, float* grad_sum, uint32_t* grad_cnt, float* opa_sum,
                             uint32_t* opa_cnt, vg_stream stream) {
    if (!scene || !ctx) return fail(VG_ERR_INVALID_ARG, "vg_grow_accumulate: null argument");
    if ((grad_sum == nullptr) != (grad_cnt == nullptr) || (opa_sum == nullptr) != (opa_cnt == nullptr))
        return fail(VG_ERR_INVALID_ARG, "vg_grow_accumulate: sums and counts go together");
    if (!ctx->have_bwd || ctx->fwd_scene != scene)
        return fail(VG_ERR_INVALID_ARG, "vg_grow_accumulate: no vg_render_bwd of this scene on this ctx");
    if (scene->dev.N == 0 || (!grad_sum && !opa_sum)) return VG_OK;
    const uint32_t slots = (uint32_t)(ctx->views.n * scene->dev.N);
    VG_CUDA(launch_grow_stats(scene->dev, ctx->vis.as<uint32_t>(), ctx->scratch.as<uint32_t>() + SCR_NVIS, slots,
                              ctx->g2d.as<float>(), grad_sum, grad_cnt, opa_sum, opa_cnt, (cudaStream_t)stream));
    return VG_OK;
}

vg_status vg_anchor_grow(const vg_scene* scene, vg_ctx* ctx, const float* grad_sum, const uint32_t* grad_cnt,
                         float eps_g, float tau_g, int32_t levels, double p_drop, uint64_t seed, int64_t cap,
                         float* new_xyz, int32_t* new_level, uint32_t* n_new, vg_stream stream) {
    if (!scene || !ctx || !grad_sum || !grad_cnt || !n_new || (cap > 0 && !new_xyz))
        return fail(VG_ERR_INVALID_ARG, "vg_anchor_grow: null argument");
    if (levels < 1 || levels > 8 || !(eps_g > 0.f) || !(p_drop >= 0.0 && p_drop <= 1.0) || cap < 0)
        return fail(VG_ERR_INVALID_ARG, "vg_anchor_grow: levels must be 1..8, eps_g > 0, p_drop in [0, 1], cap >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t slots = grow_table_slots(scene->dev.n_anchors, scene->dev.N, cap);
    VG_TRY(ctx->grow_ws.ensure((size_t)slots * 24, st, "anchor-growing table"));
    const unsigned long long drop_below = (unsigned long long)std::floor(p_drop * 9007199254740992.0);
    VG_CUDA(launch_grow(scene->dev, grad_sum, grad_cnt, eps_g, tau_g, levels, drop_below, (unsigned long long)seed,
                        new_xyz, new_level, n_new, cap, ctx->grow_ws.p, slots, ctx->state.as<uint32_t>() + ST_ERR, st));
    return VG_OK;
}

vg_status vg_anchor_prune(vg_scene* scene, const float* opa_sum, const uint32_t* opa_cnt, float tau_alpha,
                          uint32_t* removed, uint32_t* n_removed, vg_stream stream) {
    if (!scene || !opa_sum || !opa_cnt) return fail(VG_ERR_INVALID_ARG, "vg_anchor_prune: null argument");
    if (!scene->dev.mask) return fail(VG_ERR_INVALID_ARG, "vg_anchor_prune: the scene has no mask logits");
    VG_CUDA(launch_anchor_prune(const_cast<float*>(scene->dev.mask), scene->dev.n_anchors, scene->dev.k, opa_sum,
                                opa_cnt, tau_alpha, removed, n_removed, (cudaStream_t)stream));
    return VG_OK;
}

vg_status vg_adam_step(const vg_adam_tensor* tensors, int32_t n, float lr, float beta1, float beta2, float eps,
                       int32_t* step_dev, int32_t step_host, vg_stream stream) {
    if (!tensors || n < 1 || n > 16) return fail(VG_ERR_INVALID_ARG, "vg_adam_step: need 1..16 tensors");
    if (!step_dev && step_host < 1) return fail(VG_ERR_INVALID_ARG, "vg_adam_step: step must be >= 1");
    float* p[16];
    float* g[16];
    float* m[16];
    float* v[16];
    int64_t size[16];
    uint32_t zero_mask = 0;
    for (int i = 0; i < n; ++i) {
        const vg_adam_tensor& t = tensors[i];
        if (t.n < 0 || (t.n > 0 && (!t.param || !t.grad || !t.m || !t.v)))
            return fail(VG_ERR_INVALID_ARG, "vg_adam_step: null array or negative size");
        p[i] = t.param;
        g[i] = t.grad;
        m[i] = t.m;
        v[i] = t.v;
        size[i] = t.n;
        if (t.zero_grad) zero_mask |= 1u << i;
    }
    VG_CUDA(launch_adam(n, p, g, m, v, size, zero_mask, lr, beta1, beta2, eps, step_dev, step_host,
                        (cudaStream_t)stream));
    return VG_OK;
}

vg_status vg_pose_step(int32_t n_views, float* pose, const float* dxi, float* m, float* v, float lr_rot, float lr_trans,
                       float beta1, float beta2, float eps, int32_t* step_dev, int32_t step_host, vg_stream stream) {
    if (n_views < 1 || !pose || !dxi || !m || !v) return fail(VG_ERR_INVALID_ARG, "vg_pose_step: null argument");
    if (!step_dev && step_host < 1) return fail(VG_ERR_INVALID_ARG, "vg_pose_step: step must be >= 1");
    VG_CUDA(launch_pose_step(n_views, pose, dxi, m, v, lr_rot, lr_trans, beta1, beta2, eps, step_dev, step_host,
                             (cudaStream_t)stream));
    return VG_OK;
}

}  // extern "C"
