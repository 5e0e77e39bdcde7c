"""ctypes binding of the FP64 CPU oracle (``vg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It imports nothing
from the CUDA package; scenes and cameras come from the shared seeded
generator module as plain numpy arrays.

Parameter defaults are the readings the method leaves open: per-pixel opacity
cap 0.99, skip below 1/255, early stop when transmittance would fall below
1e-4, 16x16 tiles, 3-sigma radius, 0.3 px^2 low-pass dilation, Jacobian clamp
at 1.3x the half field of view, near plane 0.2 m.

Near-threshold flags mark pixels whose discrete decisions an FP32 evaluation
may take the other way.  Each decision is measured against the FP32 error
bound of the quantity that decides it: the exponent carries q_ulps units in
the last place per unit of (1 + the condition number of the 2D covariance),
relative to the magnitudes of its terms (rounding the entries of Sigma'
moves its small eigenvalue by about lambda_max u); alpha adds a floor of
decision_band (FP32 opacity, base-2 threshold, exp2); the transmittance
accumulates alpha / (1 - alpha) times alpha's error plus two roundings per
blended Gaussian, with a safety factor t_band; the radius 3 sqrt(lambda_max)
carries ~3e-7 (band r_band = 5e-6).  A Gaussian whose tile membership hangs
on a borderline radius flags only the pixels where it could be blended.
Flags are bits 0-4 of ``flags`` (images and gradients); ``ctr_flags`` adds
the pixels whose tile list may differ by a borderline member (work counters).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from typing import Dict, List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vg_oracle.c")
HDR = os.path.join(HERE, "vg_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")

GROUPS = ("logscale", "rot", "opacity", "rgb")
GDIM = (3, 4, 1, 3)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, so the FP32
    binning expressions round exactly as written)."""
    stale = (not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
    if force or stale:
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", LIB, SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return LIB


class _Scene(C.Structure):
    _fields_ = [("n_anchors", C.c_int64), ("k", C.c_int),
                ("anchor_xyz", C.c_void_p), ("anchor_l", C.c_void_p), ("offsets", C.c_void_p),
                ("L", C.c_int * 4), ("K", C.c_int * 4),
                ("codebook", C.c_void_p * 4), ("idx", C.c_void_p * 4), ("raw", C.c_void_p * 4),
                ("mask_logit", C.c_void_p), ("mask_thr", C.c_double)]


class _Camera(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int), ("height", C.c_int), ("T_cw", C.c_double * 12), ("near_plane", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("alpha_max", C.c_double), ("alpha_min", C.c_double), ("t_min", C.c_double),
                ("dilation", C.c_double), ("sigma_cull", C.c_double), ("clamp_factor", C.c_double),
                ("jacobian_clamp", C.c_int), ("tile", C.c_int), ("r_band", C.c_double),
                ("decision_band", C.c_double), ("t_band", C.c_double), ("q_ulps", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_create.restype = P
        _lib.orc_create.argtypes = [P, P, C.c_int, P]
        _lib.orc_free.argtypes = [P]
        for f in ("orc_n_slots", "orc_n_pairs", "orc_n_tiles", "orc_n_pixels"):
            getattr(_lib, f).restype = C.c_int64
            getattr(_lib, f).argtypes = [P]
        _lib.orc_get_proj.argtypes = [P, P, P, P]
        _lib.orc_get_bins.argtypes = [P, P, P]
        _lib.orc_get_decoded.argtypes = [P, P]
        _lib.orc_forward.restype = C.c_int64
        _lib.orc_forward.argtypes = [P] * 10 + [C.c_int]
        _lib.orc_rect_fp64_diff.restype = C.c_int64
        _lib.orc_rect_fp64_diff.argtypes = [P, P]
        _lib.orc_backward.argtypes = [P] * 14 + [C.c_int]
        _lib.orc_icp.argtypes = [P, P, P, P, P]
        _lib.orc_loss_l1.restype = C.c_double
        _lib.orc_loss_l1.argtypes = [C.c_int64, P, P, P, P, P, C.c_double, C.c_double, P, P]
        _lib.orc_rvq_decode.argtypes = [C.c_int, C.c_int, C.c_int, P, P, C.c_int64, P]
        _lib.orc_hit_counts.argtypes = [P, P, P, C.c_int]
        _lib.orc_set_window.restype = C.c_int
        _lib.orc_set_window.argtypes = [P] + [C.c_int] * 5
        _lib.orc_set_pixel_mask.restype = None
        _lib.orc_set_pixel_mask.argtypes = [P, P]
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def default_params(**kw) -> Dict[str, float]:
    p = dict(alpha_max=0.99, alpha_min=1.0 / 255.0, t_min=1e-4, dilation=0.3, sigma_cull=3.0,
             clamp_factor=1.3, jacobian_clamp=1, tile=16, r_band=5e-6, decision_band=2e-6, t_band=4.0,
             q_ulps=64.0)
    p.update(kw)
    return p


def mask_threshold(eps: float) -> float:
    """Eq. 11 keeps Gaussian n iff sigmoid(m_n) > eps; sigmoid is monotone, so
    this is m_n > logit(eps), with logit(eps) rounded to FP32 so that both
    sides compare the same two floats."""
    return float(np.float32(math.log(eps / (1.0 - eps))))


def rvq_decode_fp32(codebook: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Eq. 14, first line, summed in FP32 in stage order (the kernels' order)."""
    cb = np.asarray(codebook, np.float32)
    ix = np.asarray(idx)
    acc = np.zeros((ix.shape[1], cb.shape[2]), np.float32)
    for s in range(cb.shape[0]):
        acc = acc + cb[s][ix[s].astype(np.int64)]
    return acc


def rvq_scatter(grad: np.ndarray, idx: np.ndarray, shape) -> np.ndarray:
    """Gradient of a decoded array [n][d] with respect to its codebook
    [L][K][d]: codeword k of stage s collects the rows whose index is k."""
    out = np.zeros(shape)
    for s in range(shape[0]):
        np.add.at(out[s], np.asarray(idx[s], np.int64), grad)
    return out


def rvq_decode(codebook: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Eq. 14 (first line): sum over stages of the indexed codewords, FP64."""
    cb = np.ascontiguousarray(codebook, np.float64)
    ix = np.ascontiguousarray(idx, np.uint8)
    L, K, d = cb.shape
    n = ix.shape[1]
    out = np.zeros((n, d), np.float64)
    lib().orc_rvq_decode(L, K, d, _p(cb), _p(ix), n, _p(out))
    return out


class Oracle:
    """Decode + project + bin a scene for a list of cameras (FP64)."""

    def __init__(self, scene, cams: Sequence, params: Optional[Dict] = None, overrides: Optional[Dict] = None):
        """``scene``: a synth.Scene (float32 arrays are widened to float64);
        ``overrides`` may replace any scene array by a float64 array (used by
        finite differences)."""
        L = lib()
        prm = default_params(**(params or {}))
        ov = overrides or {}
        self._keep = []

        def f64(name, arr):
            a = np.ascontiguousarray(ov.get(name, arr), np.float64)
            self._keep.append(a)
            return a

        sc = _Scene()
        sc.n_anchors = scene.n_anchors
        sc.k = scene.k
        # R-VQ coded offsets / scaling factors (Eq. 14) enter as their decoded
        # values; the decode is FP32 in stage order because the means decide
        # the binning in FP32
        self.off_rvq = getattr(scene, "offsets_rvq", None)
        self.l_rvq = getattr(scene, "l_rvq", None)
        off_src = scene.offsets if self.off_rvq is None else \
            rvq_decode_fp32(self.off_rvq.codebook, self.off_rvq.idx).reshape(scene.n_anchors, scene.k, 3)
        l_src = scene.anchor_l if self.l_rvq is None else rvq_decode_fp32(self.l_rvq.codebook, self.l_rvq.idx)
        self.anchor_xyz = f64("anchor_xyz", scene.anchor_xyz)
        self.anchor_l = f64("anchor_l", l_src)
        self.offsets = f64("offsets", off_src)
        sc.anchor_xyz, sc.anchor_l, sc.offsets = _p(self.anchor_xyz), _p(self.anchor_l), _p(self.offsets)
        self.coded = []
        for gi, name in enumerate(GROUPS):
            g = scene.groups[name]
            if g.coded:
                cb = f64("cb_" + name, g.codebook)
                ix = np.ascontiguousarray(g.idx, np.uint8)
                self._keep.append(ix)
                sc.L[gi], sc.K[gi] = cb.shape[0], cb.shape[1]
                sc.codebook[gi], sc.idx[gi], sc.raw[gi] = _p(cb), _p(ix), None
            else:
                raw = f64("raw_" + name, g.raw)
                sc.L[gi], sc.K[gi] = 0, 0
                sc.codebook[gi], sc.idx[gi], sc.raw[gi] = None, None, _p(raw)
            self.coded.append(g.coded)
        if scene.mask_logit is not None:
            m = f64("mask_logit", scene.mask_logit)
            sc.mask_logit = _p(m)
        else:
            sc.mask_logit = None
        sc.mask_thr = mask_threshold(scene.mask_eps)
        self.scene = scene
        self._sc = sc

        cams = list(cams)
        self.cams = cams
        cc = (_Camera * len(cams))()
        T_over = ov.get("T_cw")
        for i, c in enumerate(cams):
            cc[i].fx, cc[i].fy, cc[i].cx, cc[i].cy = c.fx, c.fy, c.cx, c.cy
            cc[i].width, cc[i].height = c.width, c.height
            T = np.asarray(T_over[i] if T_over is not None else c.T_cw, np.float64).reshape(12)
            for j in range(12):
                cc[i].T_cw[j] = T[j]
            cc[i].near_plane = c.near
        self._cc = cc
        pp = _Params()
        for k, v in prm.items():
            setattr(pp, k, v)
        self._pp = pp
        self.params = prm
        self.ctx = L.orc_create(C.byref(sc), cc, len(cams), C.byref(pp))
        if not self.ctx:
            raise ValueError("oracle rejected the scene")
        self.N = scene.n
        self.n_views = len(cams)
        self.n_slots = L.orc_n_slots(self.ctx)
        self.n_pairs = L.orc_n_pairs(self.ctx)
        self.n_tiles = L.orc_n_tiles(self.ctx)
        self.n_pixels = L.orc_n_pixels(self.ctx)

    def hit_counts(self, threads: int = 1):
        """Eq. 13's h: per Gaussian, the (view, pixel) pairs where it is
        blended; and whether it is visible in some view."""
        hits = np.zeros(self.N, np.int64)
        seen = np.zeros(self.N, np.int32)
        lib().orc_hit_counts(self.ctx, _p(hits), _p(seen), int(threads))
        return hits, seen

    def set_window(self, view: int, x0: int, y0: int, x1: int, y1: int):
        """Composite (forward and backward) only pixels [x0, x1) x [y0, y1)
        of ``view``; binning stays that of the whole image."""
        if lib().orc_set_window(self.ctx, int(view), int(x0), int(y0), int(x1), int(y1)) != 0:
            raise ValueError("bad view")

    def set_pixel_mask(self, mask: Optional[np.ndarray]):
        """Composite only the pixels where mask (uint8, one entry per pixel of
        every view, views in order) is non-zero; None = all pixels."""
        if mask is None:
            self._pmask = None
            lib().orc_set_pixel_mask(self.ctx, None)
            return
        m = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
        if m.size != self.n_pixels:
            raise ValueError("pixel mask size differs from the views' pixel count")
        self._pmask = m  # kept alive while the oracle uses it
        lib().orc_set_pixel_mask(self.ctx, m.ctypes.data)

    def __del__(self):
        if getattr(self, "ctx", None):
            lib().orc_free(self.ctx)
            self.ctx = None

    # -- projection / binning -------------------------------------------------
    def projection(self):
        proj = np.zeros((self.n_slots, 16), np.float64)
        b32 = np.zeros((self.n_slots, 3), np.float32)
        fl = np.zeros(self.n_slots, np.int32)
        lib().orc_get_proj(self.ctx, _p(proj), _p(b32), _p(fl))
        return proj, b32, fl

    def bins(self):
        ts = np.zeros(self.n_tiles + 1, np.int64)
        lst = np.zeros(max(1, self.n_pairs), np.int64)
        lib().orc_get_bins(self.ctx, _p(ts), _p(lst))
        return ts, lst[: self.n_pairs]

    def decoded(self):
        out = np.zeros((self.N, 15), np.float64)
        lib().orc_get_decoded(self.ctx, _p(out))
        return out

    # -- compositing ----------------------------------------------------------
    def forward(self, threads: int = 1):
        P = self.n_pixels
        out = dict(C=np.zeros(3 * P), D=np.zeros(P), S=np.zeros(P), T_final=np.zeros(P),
                   n_contrib=np.zeros(P, np.int32), n_eval=np.zeros(P, np.int32), flags=np.zeros(P, np.uint8),
                   C_abs=np.zeros(3 * P), margin=np.zeros(P))
        tot = lib().orc_forward(self.ctx, _p(out["C"]), _p(out["D"]), _p(out["S"]), _p(out["T_final"]),
                                _p(out["n_contrib"]), _p(out["n_eval"]), _p(out["flags"]), _p(out["C_abs"]),
                                _p(out["margin"]), threads)
        out["evaluated"] = int(tot)
        raw = out["flags"]
        out["ctr_flags"] = raw != 0            # work counters: any flag, list ambiguity included
        out["flags"] = raw & np.uint8(31)      # images and gradients
        return out

    def rect_fp64_diff(self):
        """(slots whose FP64-centre tile rect differs from the FP32 one the
        binning uses, slots with a borderline radius), over the slots whose
        FP32 projection reaches the rect stage."""
        nb = C.c_int64(0)
        d = lib().orc_rect_fp64_diff(self.ctx, C.byref(nb))
        return int(d), int(nb.value)

    def backward(self, dC, dD, dS, threads: int = 1):
        sc = self.scene
        N = self.N
        dC = np.ascontiguousarray(dC, np.float64)
        dD = np.ascontiguousarray(dD, np.float64)
        dS = np.ascontiguousarray(dS, np.float64)
        g2d = np.zeros((self.n_slots, 10))
        dxyz = np.zeros((sc.n_anchors, 3))
        dl = np.zeros((sc.n_anchors, 3))
        doff = np.zeros((sc.n_anchors, sc.k, 3))
        dattr = []
        for gi, name in enumerate(GROUPS):
            g = sc.groups[name]
            dattr.append(np.zeros(g.codebook.shape) if g.coded else np.zeros((N, GDIM[gi])))
        dm = np.zeros(N)
        dpose = np.zeros((self.n_views, 6))
        lib().orc_backward(self.ctx, _p(dC), _p(dD), _p(dS), _p(g2d), _p(dxyz), _p(dl), _p(doff),
                           _p(dattr[0]), _p(dattr[1]), _p(dattr[2]), _p(dattr[3]),
                           _p(dm) if sc.mask_logit is not None else None, _p(dpose), threads)
        out = dict(g2d=g2d, anchor_xyz=dxyz, anchor_l=dl, offsets=doff, mask_logit=dm, pose=dpose)
        for gi, name in enumerate(GROUPS):
            out[name] = dattr[gi]
        # coded offsets / scaling factors: the indexed codeword of every stage
        # receives the gradient of its value (Eq. 14 is a sum over stages)
        for key, g, raw in (("offsets", self.off_rvq, doff), ("anchor_l", self.l_rvq, dl)):
            if g is not None:
                out[key + "_raw"] = raw
                out[key] = rvq_scatter(raw.reshape(-1, 3), np.asarray(g.idx), g.codebook.shape)
        return out

    def icp(self, q, w):
        q = np.ascontiguousarray(q, np.float64)
        w = np.ascontiguousarray(w, np.float64)
        loss = np.zeros(self.n_views)
        dpose = np.zeros((self.n_views, 6))
        lib().orc_icp(self.ctx, _p(q), _p(w), _p(loss), _p(dpose))
        return loss, dpose


def loss_l1(C_, D_, S_, Ct, Dt, w_depth=0.5, gate=-1.0):
    """Single-view L1 colour + w_depth * L1 depth (valid where target > 0);
    returns (loss, dC, dD)."""
    C_ = np.ascontiguousarray(C_, np.float64)
    D_ = np.ascontiguousarray(D_, np.float64)
    S_ = np.ascontiguousarray(S_, np.float64)
    Ct = np.ascontiguousarray(Ct, np.float64)
    Dt = np.ascontiguousarray(Dt, np.float64)
    n = D_.size
    dC = np.zeros(3 * n)
    dD = np.zeros(n)
    L = lib().orc_loss_l1(n, _p(C_), _p(D_), _p(S_), _p(Ct), _p(Dt), w_depth, gate, _p(dC), _p(dD))
    return L, dC, dD
