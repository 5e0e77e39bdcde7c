"""Seeded synthetic scenes and cameras.

This module only draws random numbers and lays out scene geometry (room
surfaces, boxes, voxel grids, camera placements).  It holds none of the
rasterizer's arithmetic: no decoding, projection, compositing or gradients.
Both the FP64 oracle tests and the CUDA path take their inputs from here, so
that neither side ever feeds the other.

Scene layout (per the voxel-anchored representation, Sec. "Voxel-Anchored 3D
Gaussian Representation", Eq. 7): ``n_anchors`` anchors, ``k`` Gaussians per
anchor; Gaussian ``n`` belongs to anchor ``n // k`` and uses offset slot
``n % k``.  Per-Gaussian attributes come in four groups (log-scale 3,
quaternion 4 in (w, x, y, z) order, opacity logit 1, RGB 3), each either
residual-codebook coded (Eq. 14: ``L`` stages of ``K`` codewords, 1-byte
indices, Sec. "Residual Codebook Quantization") or given raw per Gaussian.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

GROUPS = ("logscale", "rot", "opacity", "rgb")
GROUP_DIMS = {"logscale": 3, "rot": 4, "opacity": 1, "rgb": 3}


@dataclasses.dataclass
class Group:
    """One attribute group: codebook-coded (codebook [L,K,d] f32 + idx [L,N] u8)
    or raw (values [N,d] f32)."""
    dim: int
    codebook: Optional[np.ndarray] = None
    idx: Optional[np.ndarray] = None
    raw: Optional[np.ndarray] = None

    @property
    def coded(self) -> bool:
        return self.codebook is not None


@dataclasses.dataclass
class Scene:
    anchor_xyz: np.ndarray          # [Na,3] f32
    anchor_l: np.ndarray            # [Na,3] f32  (per-anchor scaling factor l)
    offsets: np.ndarray             # [Na,k,3] f32
    groups: Dict[str, Group]
    mask_logit: Optional[np.ndarray] = None   # [N] f32
    mask_eps: float = 0.5
    # R-VQ coded offsets (idx [L][N]) and scaling factors (idx [L][Na]); when
    # set, `offsets` / `anchor_l` are None and only the codes describe them
    offsets_rvq: Optional[Group] = None
    l_rvq: Optional[Group] = None
    k_coded: int = 0                          # k when the offsets are coded

    @property
    def n_anchors(self) -> int:
        return int(self.anchor_xyz.shape[0])

    @property
    def k(self) -> int:
        return int(self.offsets.shape[1]) if self.offsets is not None else int(self.k_coded)

    @property
    def n(self) -> int:
        return self.n_anchors * self.k


@dataclasses.dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    T_cw: np.ndarray               # [3,4] f32, world -> camera, row-major
    near: float = 0.2


# --------------------------------------------------------------------------
# small geometric helpers (input construction only)
# --------------------------------------------------------------------------

def rotation_about(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation matrix for ``angle`` radians about ``axis`` (Rodrigues)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera [3,4] for a camera at ``eye`` looking at ``target``;
    camera x right, y down (image rows), z forward."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = -R @ eye
    return T


def perturb_pose(T_cw: np.ndarray, rng: np.random.Generator,
                 max_angle_deg: float, max_trans: float) -> np.ndarray:
    """Left-multiply a pose by a random rigid motion: rotation of angle
    U[0, max] about a random axis, translation uniform in a ball."""
    axis = rng.normal(size=3)
    ang = math.radians(rng.uniform(0.0, max_angle_deg))
    R = rotation_about(axis, ang)
    d = rng.normal(size=3)
    d = d / np.linalg.norm(d) * max_trans * rng.uniform() ** (1.0 / 3.0)
    T = np.asarray(T_cw, np.float64)
    out = np.zeros((3, 4))
    out[:, :3] = R @ T[:, :3]
    out[:, 3] = R @ T[:, 3] + d
    return out


def camera(fx, fy, cx, cy, w, h, T_cw, near=0.2) -> Camera:
    return Camera(float(fx), float(fy), float(cx), float(cy), int(w), int(h),
                  np.asarray(T_cw, np.float32).reshape(3, 4).copy(), float(near))


def identity_pose() -> np.ndarray:
    T = np.zeros((3, 4), np.float32)
    T[:, :3] = np.eye(3)
    return T


def random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform unit quaternions (normalised N(0, I4) draws), (w,x,y,z)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


# --------------------------------------------------------------------------
# attribute groups
# --------------------------------------------------------------------------

def raw_groups(rng: np.random.Generator, n: int, logscale_lo=-4.0, logscale_hi=-2.0) -> Dict[str, Group]:
    """Free Gaussians with raw attributes (no codebooks): log-scales
    U[lo,hi] per axis, uniform random rotations, opacity logit N(0,1),
    RGB U[0,1]."""
    return {
        "logscale": Group(3, raw=rng.uniform(logscale_lo, logscale_hi, size=(n, 3)).astype(np.float32)),
        "rot": Group(4, raw=random_quats(rng, n).astype(np.float32)),
        "opacity": Group(1, raw=rng.normal(0.0, 1.0, size=(n, 1)).astype(np.float32)),
        "rgb": Group(3, raw=rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)),
    }


def coded_groups(rng: np.random.Generator, n: int, L: int, K: int,
                 logscale_centre: float = -4.2, logscale_spread: float = 0.25) -> Dict[str, Group]:
    """Residual-codebook groups: stage-1 codewords drawn around the raw
    attribute distributions, stage s>1 residual codewords with 1/4^(s-1)
    of the stage-1 spread; indices uniform in {0..K-1}, 1 byte each."""
    assert 1 <= K <= 256

    def book(d, first, spread):
        cb = np.zeros((L, K, d), np.float32)
        cb[0] = first((K, d))
        for s in range(1, L):
            cb[s] = rng.normal(0.0, spread / 4.0 ** s, size=(K, d))
        return cb

    groups = {
        "logscale": Group(3, codebook=book(3, lambda sh: rng.normal(logscale_centre, logscale_spread, size=sh), logscale_spread)),
        "rot": Group(4, codebook=book(4, lambda sh: rng.normal(0.0, 1.0, size=sh), 1.0)),
        "opacity": Group(1, codebook=book(1, lambda sh: rng.normal(0.0, 1.0, size=sh), 1.0)),
        "rgb": Group(3, codebook=book(3, lambda sh: rng.uniform(0.0, 1.0, size=sh), 0.29)),
    }
    for g in groups.values():
        g.idx = rng.integers(0, K, size=(L, n), dtype=np.uint8)
    return groups


def code_geometry(scene: Scene, seed: int, L: int = 3, K: int = 64, l_centre: float = 0.05,
                  offset_std: float = 0.6) -> Scene:
    """The scene with R-VQ coded offsets and scaling factors in place of the
    raw ones: seeded codebooks (stage 1 drawn like the raw values -- offsets
    N(0, offset_std), scaling factors around l_centre -- later stages residual
    codewords with 1/4^(s-1) of the spread) and uniform 1-byte indices.  The
    codes are the scene: no decoded copy is kept."""
    rng = np.random.default_rng(seed)
    na, k = scene.n_anchors, scene.k
    ocb = np.zeros((L, K, 3), np.float32)
    ocb[0] = rng.normal(0.0, offset_std, size=(K, 3))
    lcb = np.zeros((L, K, 3), np.float32)
    lcb[0] = rng.uniform(0.8 * l_centre, 1.2 * l_centre, size=(K, 3))
    for s in range(1, L):
        ocb[s] = rng.normal(0.0, offset_std / 4.0 ** s, size=(K, 3))
        lcb[s] = rng.normal(0.0, 0.1 * l_centre / 4.0 ** s, size=(K, 3))
    og = Group(3, codebook=ocb, idx=rng.integers(0, K, size=(L, na * k), dtype=np.uint8))
    lg = Group(3, codebook=lcb, idx=rng.integers(0, K, size=(L, na), dtype=np.uint8))
    return dataclasses.replace(scene, offsets=None, anchor_l=None, offsets_rvq=og, l_rvq=lg, k_coded=k)


def mask_logits(rng: np.random.Generator, n: int, frac_masked: float) -> np.ndarray:
    """Mask logits with a margin around the 0.5 threshold: the masked
    fraction ~ U[-3,-1], the rest ~ U[1,3]."""
    m = rng.uniform(1.0, 3.0, size=n)
    sel = rng.uniform(size=n) < frac_masked
    m[sel] = rng.uniform(-3.0, -1.0, size=int(sel.sum()))
    return m.astype(np.float32)


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------

def box_scene(seed: int, n: int, half_width: float = 1.0, z_lo: float = 1.0, z_hi: float = 4.0,
              coded: bool = False, L: int = 3, K: int = 64, frac_masked: float = 0.0,
              k: int = 1, offset_std: float = 0.0, logscale_lo=-4.0, logscale_hi=-2.0) -> Scene:
    """Gaussians uniform in a box x,y in [-hw,hw], z in [z_lo,z_hi] in front
    of an identity camera.  ``k`` > 1 groups them under anchors (anchor at a
    uniform point, offsets N(0, offset_std) with l = 1)."""
    rng = np.random.default_rng(seed)
    na = (n + k - 1) // k
    n = na * k
    xyz = np.stack([rng.uniform(-half_width, half_width, na),
                    rng.uniform(-half_width, half_width, na),
                    rng.uniform(z_lo, z_hi, na)], 1).astype(np.float32)
    l = np.ones((na, 3), np.float32)
    off = (rng.normal(0.0, offset_std, size=(na, k, 3)) if offset_std > 0 else np.zeros((na, k, 3))).astype(np.float32)
    if coded:
        groups = coded_groups(rng, n, L, K, logscale_centre=0.5 * (logscale_lo + logscale_hi),
                              logscale_spread=0.25 * (logscale_hi - logscale_lo))
    else:
        groups = raw_groups(rng, n, logscale_lo, logscale_hi)
    mask = mask_logits(rng, n, frac_masked) if frac_masked > 0 else None
    return Scene(xyz, l, off, groups, mask, 0.5)


def tiny_scene(seed: int = 1001, n: int = 2000) -> Scene:
    """Tiny forward render scene: n free Gaussians (one per anchor, O = 0,
    l = 1), x,y ~ U[-1,1], z ~ U[1,4] m, log-scales U[-4,-2], random unit
    quaternions, opacity logit N(0,1), RGB U[0,1]; raw attributes."""
    return box_scene(seed, n)


def tiny_camera() -> Camera:
    return camera(50.0, 50.0, 32.0, 24.0, 64, 48, identity_pose())


def _room_surface_points(rng, room=(4.5, 4.0, 2.6), n_boxes=20, voxel=0.05):
    """Voxel centres (deduplicated) of the room's floor, ceiling, four walls
    and ``n_boxes`` axis-aligned boxes standing on the floor."""
    X, Y, Z = room
    pts = []

    def plane(axis, value, lo, hi):
        # grid points on an axis-aligned rectangle
        a0, a1 = [i for i in range(3) if i != axis]
        g0 = np.arange(lo[0], hi[0] + 1e-9, voxel * 0.5)
        g1 = np.arange(lo[1], hi[1] + 1e-9, voxel * 0.5)
        G0, G1 = np.meshgrid(g0, g1, indexing="ij")
        P = np.zeros((G0.size, 3))
        P[:, axis] = value
        P[:, a0] = G0.ravel()
        P[:, a1] = G1.ravel()
        pts.append(P)

    plane(2, 0.0, (0, 0), (X, Y))
    plane(2, Z, (0, 0), (X, Y))
    plane(0, 0.0, (0, 0), (Y, Z))
    plane(0, X, (0, 0), (Y, Z))
    plane(1, 0.0, (0, 0), (X, Z))
    plane(1, Y, (0, 0), (X, Z))
    for _ in range(n_boxes):
        sx, sy, sz = rng.uniform(0.2, 0.8, size=3)
        x0 = rng.uniform(0.1, X - 0.1 - sx)
        y0 = rng.uniform(0.1, Y - 0.1 - sy)
        plane(2, sz, (x0, y0), (x0 + sx, y0 + sy))
        plane(0, x0, (y0, 0), (y0 + sy, sz))
        plane(0, x0 + sx, (y0, 0), (y0 + sy, sz))
        plane(1, y0, (x0, 0), (x0 + sx, sz))
        plane(1, y0 + sy, (x0, 0), (x0 + sx, sz))
    P = np.concatenate(pts)
    keys = np.unique(np.floor(P / voxel).astype(np.int64), axis=0)
    return (keys.astype(np.float64) + 0.5) * voxel


def room_scene(seed: int = 1002, n_anchors: int = 40000, k: int = 8, L: int = 3, K: int = 64,
               frac_masked: float = 0.2, voxel: float = 0.05) -> Scene:
    """Mapping scene: a 4.5 x 4.0 x 2.6 m room (floor, ceiling, walls) with
    20 boxes on the floor, voxelised at 0.05 m; exactly ``n_anchors``
    anchors (uniform subsample, or padded with jittered duplicates),
    k Gaussians per anchor with offsets O ~ N(0, 0.6^2) and l = 0.05
    (so O*l ~ N(0, 0.03 m)), RVQ-coded attributes (4 groups x L x K),
    ``frac_masked`` of the mask logits below the threshold."""
    rng = np.random.default_rng(seed)
    centres = _room_surface_points(rng, voxel=voxel)
    if centres.shape[0] >= n_anchors:
        sel = np.sort(rng.choice(centres.shape[0], n_anchors, replace=False))
        centres = centres[sel]
    else:
        extra = centres[rng.integers(0, centres.shape[0], n_anchors - centres.shape[0])]
        extra = extra + rng.uniform(-0.5, 0.5, size=extra.shape) * voxel
        centres = np.concatenate([centres, extra])
    xyz = centres.astype(np.float32)
    l = np.full((n_anchors, 3), voxel, np.float32)
    off = rng.normal(0.0, 0.6, size=(n_anchors, k, 3)).astype(np.float32)
    n = n_anchors * k
    groups = coded_groups(rng, n, L, K, logscale_centre=-4.2, logscale_spread=0.25)
    mask = mask_logits(rng, n, frac_masked)
    return Scene(xyz, l, off, groups, mask, 0.5)


def room_camera(width: int = 1200, height: int = 680, f: float = 600.0, pose_seed: Optional[int] = None,
                jitter_deg: float = 0.0, jitter_m: float = 0.0) -> Camera:
    """Camera at (2.25, 2.0, 1.3) in the room looking at the far wall and the
    boxes in front of it; optionally jittered by a random rigid motion."""
    T = look_at((2.25, 2.0, 1.3), (2.25, 4.0, 0.7))
    if pose_seed is not None:
        T = perturb_pose(T, np.random.default_rng(pose_seed), jitter_deg, jitter_m)
    return camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height, T)


def room_trajectory(n_frames: int = 10, width: int = 1200, height: int = 680, f: float = 600.0,
                    step_m: float = 0.01, step_deg: float = 0.25, jitter_deg: float = 0.0, jitter_m: float = 0.0,
                    seed: int = 1006) -> List[Camera]:
    """A handheld-like path through the room: the camera of room_camera()
    slides sideways by step_m and turns by step_deg about the vertical per
    frame, with a small vertical bob, each pose then shaken by a random rigid
    motion (up to jitter_deg / jitter_m)."""
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(n_frames):
        eye = np.array([2.25 - 0.5 * step_m * n_frames + step_m * i, 2.0, 1.3 + 0.01 * math.sin(0.7 * i)])
        a = math.radians(step_deg * (i - 0.5 * n_frames))
        target = eye + np.array([2.0 * math.sin(a), 2.0 * math.cos(a), -0.6])
        T = look_at(eye, target)
        if jitter_deg > 0 or jitter_m > 0:
            T = perturb_pose(T, rng, jitter_deg, jitter_m)
        cams.append(camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height, T))
    return cams


def keyframe_cameras(seed: int = 1003, n_views: int = 8, width: int = 640, height: int = 480,
                     f: float = 500.0, perturbed: bool = True) -> List[Camera]:
    """Keyframes on a smooth arc around the tiny scene (looking at its
    centre, 2.5 m in front of the origin), each optionally perturbed by a
    random rigid motion (rotation up to 2 deg, translation up to 5 cm)."""
    rng = np.random.default_rng(seed)
    cams = []
    for i in range(n_views):
        a = math.radians(-8.0 + 16.0 * i / max(1, n_views - 1))
        eye = (2.5 * math.sin(a) * 0.6, 0.05 * math.sin(3 * a), 2.5 - 2.5 * math.cos(a) * 0.6 - 1.0)
        T = look_at(eye, (0.0, 0.0, 2.5), up=(0.0, -1.0, 0.0))
        if perturbed:
            T = perturb_pose(T, rng, 2.0, 0.05)
        cams.append(camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height, T))
    return cams


def large_scene(seed: int = 1005, n_anchors: int = 375000, k: int = 8, L: int = 3, K: int = 256,
                frac_masked: float = 0.3, logscale_centre: float = math.log(0.05)) -> Scene:
    """Large indoor-outdoor layout over 20 x 20 m: ground plane, 300 boxes
    of heights 0.5-6 m and partial walls; anchors sampled on the surfaces,
    k Gaussians per anchor, RVQ 4 groups x L x K, ``frac_masked`` masked."""
    rng = np.random.default_rng(seed)
    pts = []
    # ground plane (dense near the cameras, sparse far away)
    n_ground = n_anchors // 3
    g = rng.uniform(-10.0, 10.0, size=(n_ground, 2))
    pts.append(np.stack([g[:, 0], g[:, 1], np.zeros(n_ground)], 1))
    # boxes
    n_box_pts = n_anchors // 2
    boxes = []
    for _ in range(300):
        sx, sy = rng.uniform(0.3, 2.0, size=2)
        sz = rng.uniform(0.5, 6.0)
        x0, y0 = rng.uniform(-10.0, 10.0 - sx), rng.uniform(-10.0, 10.0 - sy)
        boxes.append((x0, y0, sx, sy, sz))
    areas = np.array([2 * (b[2] + b[3]) * b[4] + b[2] * b[3] for b in boxes])
    counts = rng.multinomial(n_box_pts, areas / areas.sum())
    for (x0, y0, sx, sy, sz), c in zip(boxes, counts):
        face = rng.integers(0, 5, size=c)      # 0/1: x faces, 2/3: y faces, 4: top
        u, v = rng.uniform(size=c), rng.uniform(size=c)
        P = np.zeros((c, 3))
        P[:, 0] = x0 + u * sx
        P[:, 1] = y0 + u * sy
        P[:, 2] = v * sz
        P[face == 0, 0] = x0
        P[face == 1, 0] = x0 + sx
        P[face == 2, 1] = y0
        P[face == 3, 1] = y0 + sy
        top = face == 4
        P[top, 1] = y0 + v[top] * sy
        P[top, 2] = sz
        pts.append(P)
    # partial walls
    n_wall = n_anchors - n_ground - n_box_pts
    side = rng.integers(0, 4, size=n_wall)
    t = rng.uniform(-10.0, 10.0, size=n_wall)
    h = rng.uniform(0.0, 3.0, size=n_wall)
    P = np.zeros((n_wall, 3))
    P[:, 0] = np.where(side == 0, -10.0, np.where(side == 1, 10.0, t))
    P[:, 1] = np.where(side == 2, -10.0, np.where(side == 3, 10.0, t))
    P[:, 2] = h
    pts.append(P)
    xyz = np.concatenate(pts)[:n_anchors].astype(np.float32)
    l = np.full((n_anchors, 3), 0.1, np.float32)
    off = rng.normal(0.0, 0.5, size=(n_anchors, k, 3)).astype(np.float32)
    n = n_anchors * k
    groups = coded_groups(rng, n, L, K, logscale_centre=logscale_centre, logscale_spread=0.25)
    mask = mask_logits(rng, n, frac_masked)
    return Scene(xyz, l, off, groups, mask, 0.5)


def large_cameras(n_views: int = 4, width: int = 1920, height: int = 1080, f: float = 1000.0) -> List[Camera]:
    """Cameras 1.5 m above the ground near the layout's centre, looking
    outward in four directions."""
    cams = []
    for i in range(n_views):
        a = 2 * math.pi * i / n_views + 0.3
        eye = (0.5 * math.cos(a), 0.5 * math.sin(a), 1.5)
        tgt = (eye[0] + 10 * math.cos(a), eye[1] + 10 * math.sin(a), 1.0)
        cams.append(camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height, look_at(eye, tgt)))
    return cams


def serving_scene(n: int, seed: int) -> Scene:
    """Serving scenes: the tiny-scene recipe (coded attributes, 3 x 64
    codewords) scaled to ``n`` Gaussians, the box half-width growing as
    n^(1/3) so that the density stays that of the tiny scene."""
    a = (n / 2000.0) ** (1.0 / 3.0)
    return box_scene(seed, n, half_width=a, z_lo=1.0, z_hi=1.0 + 3.0 * a, coded=True, L=3, K=64)


def serving_camera(width: int, height: int, pose_seed: Optional[int] = None, max_deg: float = 2.0,
                   max_trans: float = 0.05) -> Camera:
    """A request camera: the tiny camera's field of view (fx = 50 per 64
    pixels of width) at ``width`` x ``height``, at the origin looking down +z,
    optionally moved by a random rigid motion (rotation up to ``max_deg``,
    translation up to ``max_trans`` m)."""
    f = 50.0 * width / 64.0
    T = identity_pose()
    if pose_seed is not None:
        T = perturb_pose(T, np.random.default_rng(pose_seed), max_deg, max_trans)
    return camera(f, f, (width - 1) / 2.0, (height - 1) / 2.0, width, height, T)


def upstream_grads(seed: int, n_pixels_total: int, scale: float = 1.0):
    """Seeded upstream gradient images dL/dC [3*P], dL/dD [P], dL/dS [P]
    (flat, per-view planar blocks), values U[-1,1]*scale/P."""
    rng = np.random.default_rng(seed)
    s = scale / max(1, n_pixels_total)
    dC = (rng.uniform(-1, 1, size=3 * n_pixels_total) * s).astype(np.float32)
    dD = (rng.uniform(-1, 1, size=n_pixels_total) * s).astype(np.float32)
    dS = (rng.uniform(-1, 1, size=n_pixels_total) * s).astype(np.float32)
    return dC, dD, dS


def icp_targets(seed: int, n_views: int, n: int, frac: float = 0.5, noise: float = 0.05,
                centre=(0.0, 0.0, 2.5)):
    """Seeded ICP correspondences: per view and Gaussian a target point
    (camera frame) near ``centre`` and a weight (0 for no correspondence)."""
    rng = np.random.default_rng(seed)
    q = (np.asarray(centre) + rng.normal(0.0, 1.0, size=(n_views, n, 3))).astype(np.float32)
    w = (rng.uniform(size=(n_views, n)) < frac).astype(np.float32) * rng.uniform(0.5, 1.5, size=(n_views, n)).astype(np.float32)
    return q, w
