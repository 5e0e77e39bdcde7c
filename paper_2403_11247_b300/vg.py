"""Thin ctypes binding of libvg (include/vg.h), one Python function per C call
and with the same name.  Argument marshalling only: every step of the render
path runs in the CUDA library; there is no CPU fallback.  PyTorch provides
device memory and streams.

Tensors passed in must be contiguous CUDA tensors of the stated dtype; host
numpy arrays are accepted only where the C call accepts host memory
(vg_scene_upload with VG_SCENE_COPY).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional, Sequence

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libvg.so")

VG_OK, VG_ERR_INVALID_ARG, VG_ERR_OOM, VG_ERR_CUDA, VG_ERR_CAPACITY, VG_ERR_TIMEOUT, VG_ERR_UNIMPLEMENTED = range(7)
STATUS_NAMES = ["VG_OK", "VG_ERR_INVALID_ARG", "VG_ERR_OOM", "VG_ERR_CUDA", "VG_ERR_CAPACITY", "VG_ERR_TIMEOUT",
                "VG_ERR_UNIMPLEMENTED"]
VG_SCENE_COPY, VG_SCENE_BORROW = 0, 1
VG_SORT_AUTO, VG_SORT_GLOBAL, VG_SORT_TILE = 0, 1, 2
VG_TILE_SORT_CAP = 1024
VG_TILE_SORT_LONG_CAP = 8192
VG_MAX_VIEWS = 64
GROUPS = ("logscale", "rot", "opacity", "rgb")
GDIM = {"logscale": 3, "rot": 4, "opacity": 1, "rgb": 3}


class VgError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class vg_camera(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("T_cw", C.c_float * 12), ("near_plane", C.c_float)]


class vg_attr_group(C.Structure):
    _fields_ = [("dim", C.c_int32), ("stages", C.c_int32), ("codewords", C.c_int32),
                ("codebook", C.c_void_p), ("idx", C.c_void_p), ("raw", C.c_void_p)]


class vg_scene_desc(C.Structure):
    _fields_ = [("n_anchors", C.c_int64), ("k", C.c_int32),
                ("anchor_xyz", C.c_void_p), ("anchor_l", C.c_void_p), ("offsets", C.c_void_p),
                ("logscale", vg_attr_group), ("rot", vg_attr_group), ("opacity", vg_attr_group), ("rgb", vg_attr_group),
                ("mask_logit", C.c_void_p), ("mask_eps", C.c_float),
                ("offsets_rvq", vg_attr_group), ("l_rvq", vg_attr_group)]


class vg_render_params(C.Structure):
    _fields_ = [("tile", C.c_int32), ("batch", C.c_int32),
                ("alpha_max", C.c_float), ("alpha_min", C.c_float), ("t_min", C.c_float), ("dilation", C.c_float),
                ("sigma_cull", C.c_float), ("clamp_factor", C.c_float),
                ("jacobian_clamp", C.c_int32), ("count_evals", C.c_int32), ("pose_dev", C.c_void_p),
                ("ppt_fwd", C.c_int32), ("ppt_bwd", C.c_int32), ("hit_count", C.c_void_p), ("seen", C.c_void_p),
                ("sort_mode", C.c_int32), ("pixel_mask", C.c_void_p), ("grad_accumulate", C.c_int32),
                ("persist_ctas", C.c_int32), ("list_split", C.c_int32)]


class vg_scene_grads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("anchor_xyz", "anchor_l", "offsets", "logscale", "rot", "opacity", "rgb",
                                          "mask_logit")]


class vg_stats(C.Structure):
    _fields_ = [("pairs", C.c_int64), ("pair_capacity", C.c_int64), ("visible", C.c_int64),
                ("evaluated", C.c_int64), ("blended", C.c_int64), ("bwd_pairs", C.c_int64), ("flags", C.c_uint32)]


_lib = None


def lib():
    """Load libvg.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libvg.so not found at {LIB_PATH}; build it with paper_2403_11247_b300.build.build()")
        L = C.CDLL(LIB_PATH)
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "vg_scene_upload": [P, I32, P, P],
            "vg_scene_free": [P],
            "vg_ctx_create": [I64, P],
            "vg_ctx_free": [P],
            "vg_ctx_reserve": [P, I64],
            "vg_check": [P, P],
            "vg_ctx_stats": [P, P, P],
            "vg_ctx_reset_counters": [P, P],
            "vg_ctx_set_spin_limit": [P, C.c_uint32],
            "vg_ctx_buffer": [P, I32, P, P],
            "vg_ctx_profile": [P, I32],
            "vg_ctx_profile_read": [P, P, P, P],
            "vg_rvq_decode": [P, I64, P, P],
            "vg_render_fwd": [P, P, I32, P, P, P, P, P, P],
            "vg_render_fwd_l1": [P, P, I32, P, P, P, P, C.c_float, C.c_float, P, P, P, P, P, P, P, P],
            "vg_render_bwd": [P, P, I32, P, P, P, P, P, P, P],
            "vg_pose_grad": [P, I32, P, P, P, P, P],
            "vg_loss_l1": [I32, I64, P, P, P, P, P, C.c_float, C.c_float, P, P, P, P, P, P],
            "vg_loss_l1_masked": [I32, I64, P, P, P, P, P, P, C.c_float, C.c_float, P, P, P, P, P, P],
            "vg_sample_rays": [P, I64, C.c_double, C.c_uint64, P, I32, P],
            "vg_frame_decode": [I32, I32, I32, P, P, C.c_float, P, P, P],
            "vg_loss_l1_noalloc": [I32, I64, P, P, P, P, P, C.c_float, C.c_float, P, P, P, P, P],
            "vg_probe_peak": [I32, I32, P, I64, P, P],
            "vg_rvq_encode": [P, I64, P, P, P, P, P],
            "vg_mask_loss": [P, P, C.c_float, P, P, P],
            "vg_ssim_loss": [P, I32, I32, I32, P, P, C.c_float, P, P, P],
            "vg_icp_associate": [P, P, I32, P, P, C.c_float, C.c_float, P, P, P],
            "vg_mask_prune": [P, P, P, C.c_uint32, P, P, P],
            "vg_grow_accumulate": [P, P, P, P, P, P, P],
            "vg_anchor_grow": [P, P, P, P, C.c_float, C.c_float, I32, C.c_double, C.c_uint64, I64, P, P, P, P],
            "vg_anchor_prune": [P, P, P, C.c_float, P, P, P],
            "vg_host_alloc": [I64, P],
            "vg_host_free": [P],
            "vg_memcpy_async": [P, P, I64, P],
            "vg_host_stage": [P, P, I64],
            "vg_adam_step": [P, I32, C.c_float, C.c_float, C.c_float, C.c_float, P, I32, P],
            "vg_pose_step": [I32, P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, P, I32, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.vg_last_error.restype = C.c_char_p
        L.vg_last_error.argtypes = []
        L.vg_default_params.restype = vg_render_params
        L.vg_default_params.argtypes = []
        L.vg_launch_count.restype = C.c_int64
        L.vg_launch_count.argtypes = []
        L.vg_workspace_allocs.restype = C.c_int64
        L.vg_workspace_allocs.argtypes = []
        L.vg_scene_size.restype = C.c_int64
        L.vg_scene_size.argtypes = [P]
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != VG_OK:
        raise VgError(status, where, lib().vg_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t) -> Optional[int]:
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        raise TypeError("a device tensor is required here, not a numpy array")
    if not t.is_cuda:
        raise TypeError("a CUDA tensor is required")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _host_or_dev_ptr(a):
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, a
    return _ptr(a), a


def default_params(**kw) -> vg_render_params:
    p = lib().vg_default_params()
    for k, v in kw.items():
        if k in ("pose_dev", "hit_count", "seen", "pixel_mask"):
            setattr(p, k, _ptr(v))
        else:
            setattr(p, k, v)
    return p


def cameras(cams: Sequence) -> C.Array:
    arr = (vg_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = c.fx, c.fy, c.cx, c.cy
        arr[i].width, arr[i].height = c.width, c.height
        T = np.asarray(c.T_cw, np.float32).reshape(12)
        for j in range(12):
            arr[i].T_cw[j] = float(T[j])
        arr[i].near_plane = c.near
    return arr


# ---------------------------------------------------------------------------
# scenes and workspaces
# ---------------------------------------------------------------------------

class SceneHandle:
    """An owned vg_scene; keeps borrowed tensors alive."""

    def __init__(self, handle: int, keep, n: int, n_anchors: int, k: int, coded: Dict[str, tuple], masked: bool):
        self.handle = handle
        self._keep = keep
        self.n = n
        self.n_anchors = n_anchors
        self.k = k
        self.coded = coded          # group -> (L, K) for coded groups
        self.masked = masked
        self.coded_geometry = {}    # "offsets" / "anchor_l" -> (L, K) when R-VQ coded

    def free(self):
        if self.handle:
            _check(lib().vg_scene_free(self.handle), "vg_scene_free")
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def vg_scene_upload(scene, flags: int = VG_SCENE_COPY, stream=None) -> SceneHandle:
    """``scene``: a synth.Scene (numpy host arrays, COPY) or any object with the
    same attributes holding CUDA tensors (COPY or BORROW)."""
    desc = vg_scene_desc()
    keep = []

    def put(a):
        p, ref = _host_or_dev_ptr(a)
        if ref is not None:
            keep.append(ref)
        return p

    off_rvq = getattr(scene, "offsets_rvq", None)
    l_rvq = getattr(scene, "l_rvq", None)
    desc.n_anchors = int(scene.anchor_xyz.shape[0])
    desc.k = int(scene.k) if hasattr(scene, "k") else int(scene.offsets.shape[1])
    desc.anchor_xyz = put(scene.anchor_xyz)
    desc.anchor_l = put(scene.anchor_l) if l_rvq is None else None
    desc.offsets = put(scene.offsets) if off_rvq is None else None
    for grp, g in ((desc.offsets_rvq, off_rvq), (desc.l_rvq, l_rvq)):
        if g is not None:
            grp.dim, grp.stages, grp.codewords = 3, int(g.codebook.shape[0]), int(g.codebook.shape[1])
            grp.codebook, grp.idx, grp.raw = put(g.codebook), put(g.idx), None
    coded = {}
    for name in GROUPS:
        g = scene.groups[name]
        grp = getattr(desc, name)
        grp.dim = GDIM[name]
        if g.codebook is not None:
            grp.stages, grp.codewords = int(g.codebook.shape[0]), int(g.codebook.shape[1])
            grp.codebook = put(g.codebook)
            grp.idx = put(g.idx)
            grp.raw = None
            coded[name] = (grp.stages, grp.codewords)
        else:
            grp.stages, grp.codewords = 0, 0
            grp.raw = put(g.raw)
    desc.mask_logit = put(scene.mask_logit)
    desc.mask_eps = float(scene.mask_eps)
    h = C.c_void_p()
    _check(lib().vg_scene_upload(C.byref(desc), flags, _stream(stream), C.byref(h)), "vg_scene_upload")
    n = desc.n_anchors * desc.k
    geom = {}
    if off_rvq is not None:
        geom["offsets"] = tuple(int(x) for x in off_rvq.codebook.shape[:2])
    if l_rvq is not None:
        geom["anchor_l"] = tuple(int(x) for x in l_rvq.codebook.shape[:2])
    h_ = SceneHandle(h.value, keep if flags == VG_SCENE_BORROW else None, n, desc.n_anchors, desc.k, coded,
                     scene.mask_logit is not None)
    h_.coded_geometry = geom
    return h_


class CtxHandle:
    def __init__(self, handle: int):
        self.handle = handle
        self.views = None

    def free(self):
        if self.handle:
            _check(lib().vg_ctx_free(self.handle), "vg_ctx_free")
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def vg_ctx_create(pair_capacity: int = 0) -> CtxHandle:
    h = C.c_void_p()
    _check(lib().vg_ctx_create(int(pair_capacity), C.byref(h)), "vg_ctx_create")
    return CtxHandle(h.value)


def vg_host_alloc(nbytes: int) -> int:
    p = C.c_void_p()
    _check(lib().vg_host_alloc(int(nbytes), C.byref(p)), "vg_host_alloc")
    return p.value


def vg_host_free(ptr: int):
    _check(lib().vg_host_free(C.c_void_p(ptr)), "vg_host_free")


def vg_memcpy_async(dst, src, stream=None):
    """Copies tensor src into tensor dst (same number of bytes; host or
    device) in stream order through the library."""
    nb = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != nb:
        raise ValueError("vg_memcpy_async: sizes differ")
    def any_ptr(t):
        if not t.is_contiguous():
            raise ValueError("vg_memcpy_async: tensors must be contiguous")
        return t.data_ptr()
    _check(lib().vg_memcpy_async(any_ptr(dst), any_ptr(src), int(nb), _stream(stream)), "vg_memcpy_async")


def vg_host_stage(dst, src):
    """Writes CPU tensor (or numpy array) src into CPU tensor dst, e.g. a
    host_empty staging buffer, with streaming stores (see vg.h)."""
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src)
        sp, nb = src.ctypes.data, src.nbytes
    else:
        if not src.is_contiguous() or src.is_cuda:
            raise ValueError("vg_host_stage: src must be a contiguous host tensor")
        sp, nb = src.data_ptr(), src.numel() * src.element_size()
    if dst.is_cuda or not dst.is_contiguous() or dst.numel() * dst.element_size() != nb:
        raise ValueError("vg_host_stage: dst must be a contiguous host tensor of the same size")
    _check(lib().vg_host_stage(C.c_void_p(dst.data_ptr()), C.c_void_p(sp), int(nb)), "vg_host_stage")


def host_empty(shape, dtype=None):
    """A CPU tensor in vg_host_alloc memory (page-locked, huge-page backed):
    the staging buffer for frames streamed to the device.  The memory is
    freed when the last tensor viewing it is gone."""
    import weakref
    torch = _torch()
    dtype = dtype or torch.float32
    shape = (shape,) if isinstance(shape, int) else tuple(shape)
    n = int(np.prod(shape)) if shape else 1
    nbytes = max(1, n * torch.empty((), dtype=dtype).element_size())
    ptr = vg_host_alloc(nbytes)
    buf = (C.c_char * nbytes).from_address(ptr)
    weakref.finalize(buf, vg_host_free, ptr)
    return torch.frombuffer(buf, dtype=dtype, count=n).view(shape)


def vg_ctx_reserve(ctx: CtxHandle, pair_capacity: int):
    _check(lib().vg_ctx_reserve(ctx.handle, int(pair_capacity)), "vg_ctx_reserve")


def vg_ctx_stats(ctx: CtxHandle, stream=None) -> Dict[str, int]:
    s = vg_stats()
    _check(lib().vg_ctx_stats(ctx.handle, _stream(stream), C.byref(s)), "vg_ctx_stats")
    return dict(pairs=s.pairs, pair_capacity=s.pair_capacity, visible=s.visible, evaluated=s.evaluated,
                blended=s.blended, bwd_pairs=s.bwd_pairs, flags=s.flags)


def vg_check(ctx: CtxHandle, stream=None) -> int:
    """Returns the status code (VG_OK, VG_ERR_CAPACITY, ...) without raising."""
    return lib().vg_check(ctx.handle, _stream(stream))


def vg_ctx_reset_counters(ctx: CtxHandle, stream=None):
    _check(lib().vg_ctx_reset_counters(ctx.handle, _stream(stream)), "vg_ctx_reset_counters")


# ---------------------------------------------------------------------------
# compute calls
# ---------------------------------------------------------------------------

def vg_rvq_decode(codebook, idx, out=None, stream=None):
    """codebook [L,K,d] f32 CUDA, idx [L,n] u8 CUDA -> out [n,d] f32."""
    torch = _torch()
    L, K, d = codebook.shape
    n = idx.shape[1]
    if out is None:
        out = torch.empty((n, d), dtype=torch.float32, device=codebook.device)
    g = vg_attr_group(int(d), int(L), int(K), _ptr(codebook), _ptr(idx), None)
    _check(lib().vg_rvq_decode(C.byref(g), int(n), _ptr(out), _stream(stream)), "vg_rvq_decode")
    return out


def vg_rvq_encode(codebook, x, idx=None, loss=None, dcodebook=None, want_loss=True, want_grad=True, stream=None):
    """codebook [L,K,d] f32 CUDA, x [n,d] f32 CUDA -> (idx [L,n] u8, loss [1], dcodebook [L,K,d])."""
    torch = _torch()
    L, K, d = codebook.shape
    n = x.shape[0]
    dev = codebook.device
    if idx is None:
        idx = torch.empty((L, n), dtype=torch.uint8, device=dev)
    if loss is None and want_loss:
        loss = torch.empty(1, dtype=torch.float32, device=dev)
    if dcodebook is None and want_grad:
        dcodebook = torch.empty_like(codebook)
    g = vg_attr_group(int(d), int(L), int(K), _ptr(codebook), None, None)
    _check(lib().vg_rvq_encode(C.byref(g), int(n), _ptr(x), _ptr(idx), _ptr(loss), _ptr(dcodebook),
                               _stream(stream)), "vg_rvq_encode")
    return idx, loss, dcodebook


def vg_mask_loss(scene: SceneHandle, ctx: CtxHandle, weight: float = 1.0, dmask=None, loss=None, stream=None):
    """Mask loss over the last forward's visible Gaussians; adds its gradient to dmask."""
    torch = _torch()
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _check(lib().vg_mask_loss(scene.handle, ctx.handle, float(weight), _ptr(dmask), _ptr(loss), _stream(stream)),
           "vg_mask_loss")
    return loss


def vg_grow_accumulate(scene: SceneHandle, ctx: CtxHandle, grad_sum=None, grad_cnt=None, opa_sum=None, opa_cnt=None,
                       stream=None):
    """Adds the last backward's per-pair growing statistics to the given
    accumulators (grad_sum/grad_cnt [N], opa_sum/opa_cnt [A])."""
    _check(lib().vg_grow_accumulate(scene.handle, ctx.handle, _ptr(grad_sum), _ptr(grad_cnt), _ptr(opa_sum),
                                    _ptr(opa_cnt), _stream(stream)), "vg_grow_accumulate")


def vg_anchor_grow(scene: SceneHandle, ctx: CtxHandle, grad_sum, grad_cnt, eps_g: float, tau_g: float, levels: int = 3,
                   p_drop: float = 0.0, seed: int = 0, cap: int = 65536, new_xyz=None, new_level=None, n_new=None,
                   stream=None):
    """New anchor centres on the multi-resolution voxel grid; returns
    (new_xyz [cap][3], new_level [cap], n_new [1]) device tensors, the first
    min(n_new, cap) rows valid, in unspecified order."""
    torch = _torch()
    if new_xyz is None:
        new_xyz = torch.empty((max(cap, 1), 3), dtype=torch.float32, device="cuda")
    if new_level is None:
        new_level = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    if n_new is None:
        n_new = torch.empty(1, dtype=torch.int32, device="cuda")
    _check(lib().vg_anchor_grow(scene.handle, ctx.handle, _ptr(grad_sum), _ptr(grad_cnt), float(eps_g), float(tau_g),
                                int(levels), float(p_drop), int(seed) & ((1 << 64) - 1), int(cap), _ptr(new_xyz),
                                _ptr(new_level), _ptr(n_new), _stream(stream)), "vg_anchor_grow")
    return new_xyz, new_level, n_new


def vg_anchor_prune(scene: SceneHandle, opa_sum, opa_cnt, tau_alpha: float, removed=None, n_removed=None, stream=None):
    """Removes (mask logit -inf on all k Gaussians) every anchor seen with a
    mean opacity below tau_alpha; returns n_removed [1]."""
    torch = _torch()
    if n_removed is None:
        n_removed = torch.empty(1, dtype=torch.int32, device="cuda")
    _check(lib().vg_anchor_prune(scene.handle, _ptr(opa_sum), _ptr(opa_cnt), float(tau_alpha), _ptr(removed),
                                 _ptr(n_removed), _stream(stream)), "vg_anchor_prune")
    return n_removed


def vg_mask_prune(scene: SceneHandle, hit_count=None, seen=None, min_hits: int = 1, removed=None, n_removed=None,
                  stream=None):
    torch = _torch()
    if n_removed is None:
        n_removed = torch.empty(1, dtype=torch.int32, device="cuda")
    _check(lib().vg_mask_prune(scene.handle, _ptr(hit_count), _ptr(seen), int(min_hits), _ptr(removed),
                               _ptr(n_removed), _stream(stream)), "vg_mask_prune")
    return n_removed


def vg_ssim_loss(ctx: CtxHandle, n_views: int, width: int, height: int, C_, Ct, weight: float = 1.0, dC=None,
                 loss=None, stream=None):
    torch = _torch()
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=C_.device)
    _check(lib().vg_ssim_loss(ctx.handle, int(n_views), int(width), int(height), _ptr(C_), _ptr(Ct), float(weight),
                              _ptr(dC), _ptr(loss), _stream(stream)), "vg_ssim_loss")
    return loss


def vg_icp_associate(scene: SceneHandle, cams, params, Dt, max_dist: float = 0.1, weight: float = 1.0, q=None, w=None,
                     stream=None):
    torch = _torch()
    V_ = len(cams)
    if q is None:
        q = torch.empty((V_, scene.n, 3), dtype=torch.float32, device="cuda")
    if w is None:
        w = torch.empty((V_, scene.n), dtype=torch.float32, device="cuda")
    p = params if params is not None else default_params()
    _check(lib().vg_icp_associate(scene.handle, cameras(cams), V_, C.byref(p), _ptr(Dt), float(max_dist), float(weight),
                                  _ptr(q), _ptr(w), _stream(stream)), "vg_icp_associate")
    return q, w


def image_sizes(cams):
    return [c.width * c.height for c in cams]


def vg_render_fwd(scene: SceneHandle, cams, params: Optional[vg_render_params], ctx: CtxHandle,
                  C_=None, D=None, S=None, stream=None):
    """Returns flat (C [3*P], D [P], S [P]) CUDA tensors (per-view planar blocks)."""
    torch = _torch()
    P = sum(image_sizes(cams))
    dev = torch.device("cuda", torch.cuda.current_device())
    if C_ is None:
        C_ = torch.empty(3 * P, dtype=torch.float32, device=dev)
    if D is None:
        D = torch.empty(P, dtype=torch.float32, device=dev)
    if S is None:
        S = torch.empty(P, dtype=torch.float32, device=dev)
    p = params if params is not None else default_params()
    cc = cameras(cams)
    _check(lib().vg_render_fwd(scene.handle, cc, len(cams), C.byref(p), ctx.handle, _ptr(C_), _ptr(D), _ptr(S),
                               _stream(stream)), "vg_render_fwd")
    return C_, D, S


def vg_render_fwd_l1(scene: SceneHandle, cams, params: Optional[vg_render_params], ctx: CtxHandle, Ct, Dt,
                     w_depth: float = 0.5, gate: float = -1.0, C_=None, D=None, S=None, dC=None, dD=None, dS=None,
                     loss=None, stream=None):
    """Forward with the L1 loss gradient written by the compositing kernel:
    returns (C, D, S, dC, dD, loss) CUDA tensors (dS, if given, is zeroed)."""
    torch = _torch()
    P = sum(image_sizes(cams))
    dev = torch.device("cuda", torch.cuda.current_device())
    f32 = dict(dtype=torch.float32, device=dev)
    C_ = torch.empty(3 * P, **f32) if C_ is None else C_
    D = torch.empty(P, **f32) if D is None else D
    S = torch.empty(P, **f32) if S is None else S
    dC = torch.empty(3 * P, **f32) if dC is None else dC
    dD = torch.empty(P, **f32) if dD is None else dD
    loss = torch.empty(1, **f32) if loss is None else loss
    p = params if params is not None else default_params()
    cc = cameras(cams)
    _check(lib().vg_render_fwd_l1(scene.handle, cc, len(cams), C.byref(p), ctx.handle, _ptr(Ct), _ptr(Dt),
                                  float(w_depth), float(gate), _ptr(C_), _ptr(D), _ptr(S), _ptr(dC), _ptr(dD), _ptr(dS),
                                  _ptr(loss), _stream(stream)), "vg_render_fwd_l1")
    return C_, D, S, dC, dD, loss


def grads_like(scene: SceneHandle, device=None, mask=True):
    """Allocate a full set of gradient tensors for ``scene``."""
    torch = _torch()
    dev = device or torch.device("cuda", torch.cuda.current_device())
    f = dict(dtype=torch.float32, device=dev)
    g = dict(anchor_xyz=torch.empty((scene.n_anchors, 3), **f), anchor_l=torch.empty((scene.n_anchors, 3), **f),
             offsets=torch.empty((scene.n_anchors, scene.k, 3), **f))
    # R-VQ coded offsets / scaling factors: [L][K][3] codebook gradients
    for name, (L, K) in getattr(scene, "coded_geometry", {}).items():
        g[name] = torch.empty((L, K, 3), **f)
    for name in GROUPS:
        if name in scene.coded:
            L, K = scene.coded[name]
            g[name] = torch.empty((L, K, GDIM[name]), **f)
        else:
            g[name] = torch.empty((scene.n, GDIM[name]), **f)
    if mask and scene.masked:
        g["mask_logit"] = torch.empty(scene.n, **f)
    return g


def vg_render_bwd(scene: SceneHandle, cams, params: Optional[vg_render_params], ctx: CtxHandle,
                  dC=None, dD=None, dS=None, grads: Optional[Dict] = None, stream=None):
    if grads is None:
        grads = grads_like(scene)
    sg = vg_scene_grads()
    for name, _ in vg_scene_grads._fields_:
        setattr(sg, name, _ptr(grads.get(name)))
    p = params if params is not None else default_params()
    cc = cameras(cams)
    _check(lib().vg_render_bwd(scene.handle, cc, len(cams), C.byref(p), ctx.handle, _ptr(dC), _ptr(dD), _ptr(dS),
                               C.byref(sg), _stream(stream)), "vg_render_bwd")
    return grads


def vg_pose_grad(ctx: CtxHandle, n_views: int, icp_q=None, icp_w=None, dxi=None, icp_loss=None, stream=None):
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    if dxi is None:
        dxi = torch.empty((n_views, 6), dtype=torch.float32, device=dev)
    if icp_q is not None and icp_loss is None:
        icp_loss = torch.empty(n_views, dtype=torch.float32, device=dev)
    _check(lib().vg_pose_grad(ctx.handle, int(n_views), _ptr(icp_q), _ptr(icp_w), _ptr(dxi), _ptr(icp_loss),
                              _stream(stream)), "vg_pose_grad")
    return dxi, icp_loss


def vg_frame_decode(rgb, depth, width: int, height: int, depth_scale: float, C_=None, D=None, stream=None):
    """RGB-D frames as sensors deliver them -- rgb uint8 [views][H][W][3],
    depth uint16 [views][H][W] (depth_scale units a metre), CUDA tensors --
    decoded on the device into planar FP32 C [views*3*H*W] and D [views*H*W]."""
    torch = _torch()
    hw = int(width) * int(height)
    n_views = rgb.numel() // (3 * hw) if hw > 0 else 0
    if C_ is None:
        C_ = torch.empty(3 * n_views * hw, dtype=torch.float32, device=rgb.device)
    if D is None:
        D = torch.empty(n_views * hw, dtype=torch.float32, device=rgb.device)
    _check(lib().vg_frame_decode(int(n_views), int(width), int(height), _ptr(rgb), _ptr(depth), float(depth_scale),
                                 _ptr(C_), _ptr(D), _stream(stream)), "vg_frame_decode")
    return C_, D


def vg_loss_l1(n_views: int, n_pix: int, C_, D, S, Ct, Dt, w_depth: float, gate: float, ctx: CtxHandle,
               dC=None, dD=None, dS=None, loss=None, stream=None):
    torch = _torch()
    if dC is None:
        dC = torch.empty_like(C_)
    if dD is None:
        dD = torch.empty_like(D)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=C_.device)
    _check(lib().vg_loss_l1(int(n_views), int(n_pix), _ptr(C_), _ptr(D), _ptr(S), _ptr(Ct), _ptr(Dt), float(w_depth),
                            float(gate), _ptr(dC), _ptr(dD), _ptr(dS), _ptr(loss), ctx.handle, _stream(stream)),
           "vg_loss_l1")
    return dC, dD, dS, loss


def vg_loss_l1_masked(n_views: int, n_pix: int, C_, D, S, Ct, Dt, pixel_mask, w_depth: float, gate: float,
                      ctx: CtxHandle, dC=None, dD=None, dS=None, loss=None, stream=None):
    """vg_loss_l1 over the sampled rays (pixel_mask uint8, one entry per pixel of every view)."""
    torch = _torch()
    if dC is None:
        dC = torch.empty_like(C_)
    if dD is None:
        dD = torch.empty_like(D)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=C_.device)
    _check(lib().vg_loss_l1_masked(int(n_views), int(n_pix), _ptr(C_), _ptr(D), _ptr(S), _ptr(Ct), _ptr(Dt),
                                   _ptr(pixel_mask), float(w_depth), float(gate), _ptr(dC), _ptr(dD), _ptr(dS),
                                   _ptr(loss), ctx.handle, _stream(stream)), "vg_loss_l1_masked")
    return dC, dD, dS, loss


def vg_sample_rays(mask, rate: float, seed: int, round_dev=None, round_host: int = 0, stream=None):
    """Fills the uint8 device array mask with the rays sampled at this round
    (see vg.h); round_dev: optional int32 device counter."""
    _check(lib().vg_sample_rays(_ptr(mask), int(mask.numel()), float(rate), int(seed) & ((1 << 64) - 1),
                                _ptr(round_dev), int(round_host), _stream(stream)), "vg_sample_rays")
    return mask


VG_BUF = dict(xy=0, conic=1, rgbd=2, rect=3, ntiles=4, pair_keys=5, pair_vals=6, ranges=7, t_final=8, n_contrib=9,
              g2d=10, n_eval=11)
_BUF_DTYPE = dict(xy=("float32", 4), conic=("float32", 4), rgbd=("float32", 4), rect=("uint32", 2),
                  ntiles=("uint32", 1), pair_keys=("uint32", 1), pair_vals=("uint32", 1), ranges=("uint32", 2),
                  t_final=("float32", 1), n_contrib=("uint32", 1), g2d=("float32", 12), n_eval=("uint32", 1))


SPIN_LIMIT_DEFAULT = 0xFFFFFFFF


def vg_ctx_set_spin_limit(ctx: CtxHandle, polls: int = SPIN_LIMIT_DEFAULT):
    """Unsuccessful polls before a bounded device wait of this ctx gives up
    (then vg_check returns VG_ERR_TIMEOUT); the default restores 2^21."""
    _check(lib().vg_ctx_set_spin_limit(ctx.handle, int(polls) & 0xFFFFFFFF), "vg_ctx_set_spin_limit")


def vg_ctx_buffer(ctx: CtxHandle, which: str, count: int, stream=None) -> np.ndarray:
    """Copy ``count`` records of an intermediate workspace array to the host
    (synchronises the stream)."""
    torch = _torch()
    ptr, nbytes = C.c_void_p(), C.c_int64()
    _check(lib().vg_ctx_buffer(ctx.handle, VG_BUF[which], C.byref(ptr), C.byref(nbytes)), "vg_ctx_buffer")
    dt, width = _BUF_DTYPE[which]
    rec = np.dtype(dt).itemsize * width
    if count * rec > nbytes.value:
        raise ValueError(f"{which}: {count} records exceed the buffer ({nbytes.value} bytes)")
    out = np.empty(count * width, dtype=dt)
    (torch.cuda.current_stream() if stream is None else stream).synchronize()
    if count:
        res = _cudart().cudaMemcpy(C.c_void_p(out.ctypes.data), ptr, C.c_size_t(count * rec), 2)  # device -> host
        if int(res) != 0:
            raise RuntimeError(f"cudaMemcpy failed: {res}")
    return out.reshape(count, width) if width > 1 else out


_cudart_lib = None


def _cudart():
    global _cudart_lib
    if _cudart_lib is None:
        _cudart_lib = C.CDLL("libcudart.so.13")
        _cudart_lib.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
        _cudart_lib.cudaMemcpy.restype = C.c_int
    return _cudart_lib


class vg_adam_tensor(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p), ("n", C.c_int64),
                ("zero_grad", C.c_int32)]


def vg_adam_step(params, grads, ms, vs, lr, beta1=0.9, beta2=0.999, eps=1e-15, step_dev=None, step_host=0,
                 stream=None, zero_grad=False):
    """Adam over lists of equally-shaped CUDA tensors (one launch); with
    zero_grad each gradient is set to zero once read."""
    n = len(params)
    arr = (vg_adam_tensor * n)()
    for i in range(n):
        arr[i].param, arr[i].grad = _ptr(params[i]), _ptr(grads[i])
        arr[i].m, arr[i].v, arr[i].n = _ptr(ms[i]), _ptr(vs[i]), params[i].numel()
        arr[i].zero_grad = 1 if zero_grad else 0
    _check(lib().vg_adam_step(arr, n, lr, beta1, beta2, eps, _ptr(step_dev), int(step_host), _stream(stream)),
           "vg_adam_step")


def vg_pose_step(pose, dxi, m, v, lr_rot, lr_trans, beta1=0.9, beta2=0.999, eps=1e-15, step_dev=None, step_host=0,
                 stream=None):
    _check(lib().vg_pose_step(int(pose.shape[0]), _ptr(pose), _ptr(dxi), _ptr(m), _ptr(v), lr_rot, lr_trans, beta1,
                              beta2, eps, _ptr(step_dev), int(step_host), _stream(stream)), "vg_pose_step")


STAGES = ("preprocess", "depth_sort", "duplicate", "tile_sort", "ranges", "blend_fwd", "loss", "blend_bwd", "chain",
          "codebook", "pose", "memset")


def vg_ctx_profile(ctx: CtxHandle, enable: bool):
    _check(lib().vg_ctx_profile(ctx.handle, 1 if enable else 0), "vg_ctx_profile")


def vg_ctx_profile_read(ctx: CtxHandle, stream=None) -> Dict[str, tuple]:
    """{stage: (total ms, launches)} since profiling was enabled."""
    ms = (C.c_double * len(STAGES))()
    n = (C.c_int64 * len(STAGES))()
    _check(lib().vg_ctx_profile_read(ctx.handle, _stream(stream), ms, n), "vg_ctx_profile_read")
    return {s: (ms[i], n[i]) for i, s in enumerate(STAGES)}


def vg_launch_count() -> int:
    return int(lib().vg_launch_count())


def vg_workspace_allocs() -> int:
    return int(lib().vg_workspace_allocs())


VG_NOALLOC_MAX_VIEWS = 256


def vg_loss_l1_noalloc(n_views: int, n_pix: int, C_, D, S, Ct, Dt, w_depth: float, gate: float,
                       dC=None, dD=None, dS=None, loss=None, stream=None):
    """vg_loss_l1 without a ctx: its scratch is a static device array, so the
    call allocates no device memory (outputs are allocated here only when the
    caller passes none)."""
    torch = _torch()
    if dC is None:
        dC = torch.empty_like(C_)
    if dD is None:
        dD = torch.empty_like(D)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=C_.device)
    _check(lib().vg_loss_l1_noalloc(int(n_views), int(n_pix), _ptr(C_), _ptr(D), _ptr(S), _ptr(Ct), _ptr(Dt),
                                    float(w_depth), float(gate), _ptr(dC), _ptr(dD), _ptr(dS), _ptr(loss),
                                    _stream(stream)), "vg_loss_l1_noalloc")
    return dC, dD, dS, loss


def exported_symbols():
    return ["vg_scene_upload", "vg_scene_free", "vg_scene_size", "vg_ctx_create", "vg_ctx_free", "vg_ctx_reserve",
            "vg_check", "vg_ctx_stats", "vg_ctx_reset_counters", "vg_ctx_buffer", "vg_ctx_profile",
            "vg_ctx_profile_read", "vg_adam_step", "vg_pose_step", "vg_rvq_decode", "vg_render_fwd",
            "vg_render_bwd", "vg_pose_grad", "vg_loss_l1", "vg_loss_l1_noalloc", "vg_last_error", "vg_default_params",
            "vg_launch_count", "vg_probe_peak", "vg_rvq_encode", "vg_mask_loss", "vg_mask_prune", "vg_ssim_loss", "vg_icp_associate",
            "vg_grow_accumulate", "vg_anchor_grow", "vg_anchor_prune", "vg_host_alloc", "vg_host_free", "vg_memcpy_async", "vg_host_stage",
            "vg_loss_l1_masked", "vg_sample_rays", "vg_render_fwd_l1", "vg_ctx_set_spin_limit",
            "vg_workspace_allocs", "vg_frame_decode"]


PROBES = {"fma": (0, 20000, "TFLOP/s", 1e12), "ex2": (1, 2000, "G exp2/s", 1e9), "smem": (2, 5000, "TB/s", 1e12),
          "atomic_distinct": (3, 200, "G atomics/s", 1e9), "atomic_per_warp": (4, 50, "G atomics/s", 1e9)}


def probe_peaks(reps: int = 5) -> Dict[str, dict]:
    """Measured throughput of each vg_probe_peak kind (best of `reps` launches,
    CUDA events on the current stream)."""
    torch = _torch()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    n = sms * 8 * 256
    buf = torch.zeros(n, dtype=torch.float32, device="cuda")
    units = C.c_int64()
    out = {}
    for name, (kind, iters, unit, scale) in PROBES.items():
        best = None
        for _ in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            _check(lib().vg_probe_peak(kind, iters, _ptr(buf), n, C.byref(units), _stream(None)), "vg_probe_peak")
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        out[name] = {"value": units.value / (best / 1e3) / scale, "unit": unit, "ms": best}
    return out


def render_with_retry(scene: SceneHandle, cams, params, ctx: CtxHandle, stream=None, max_tries: int = 4):
    """Forward, and if the pair buffer overflowed, grow it and render again
    (the overflowed outputs are discarded).  Synchronises the stream."""
    for _ in range(max_tries):
        out = vg_render_fwd(scene, cams, params, ctx, stream=stream)
        st = vg_check(ctx, stream)
        if st == VG_OK:
            return out
        if st != VG_ERR_CAPACITY:
            _check(st, "vg_render_fwd")
        need = vg_ctx_stats(ctx, stream)["pairs"]
        vg_ctx_reserve(ctx, int(need * 1.25) + 1024)
    raise VgError(VG_ERR_CAPACITY, "render_with_retry", "pair buffer kept overflowing")
