"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a fact the paper or the mathematics
fixes: closed forms (a single Gaussian on the optical axis), an independent
projection (scipy rotations + a numerically differentiated pinhole),
brute-force per-pixel compositing, invariants (transmittance, occlusion,
permutation, mask == deletion, rigid motion), and central finite
differences for every gradient (scene parameters, codebooks, mask logits
through the straight-through estimator, camera pose, ICP).
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2403_11247_b300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------------------
# helpers (input construction only)
# ---------------------------------------------------------------------------

def raw_scene(mu, logscale, quat, op_logit, rgb, mask=None):
    n = len(mu)
    groups = {
        "logscale": synth.Group(3, raw=np.asarray(logscale, np.float32).reshape(n, 3)),
        "rot": synth.Group(4, raw=np.asarray(quat, np.float32).reshape(n, 4)),
        "opacity": synth.Group(1, raw=np.asarray(op_logit, np.float32).reshape(n, 1)),
        "rgb": synth.Group(3, raw=np.asarray(rgb, np.float32).reshape(n, 3)),
    }
    return synth.Scene(np.asarray(mu, np.float32).reshape(n, 3), np.ones((n, 3), np.float32),
                       np.zeros((n, 1, 3), np.float32), groups,
                       None if mask is None else np.asarray(mask, np.float32), 0.5)


def cam(fx, fy, cx, cy, w, h, T=None):
    return synth.camera(fx, fy, cx, cy, w, h, synth.identity_pose() if T is None else T)


def sigma2d_independent(mu, scales, quat_wxyz, c, dil):
    """Sigma' from an independent route: scipy rotation (x,y,z,w order),
    Sigma as a sum over principal axes, and the Jacobian of the full pinhole
    map x -> pi(W x + t) taken by central differences."""
    q = np.asarray(quat_wxyz, np.float64)
    Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = sum(scales[k] ** 2 * np.outer(Rg[:, k], Rg[:, k]) for k in range(3))
    T = np.asarray(c.T_cw, np.float64)

    def pi(x):
        p = T[:, :3] @ x + T[:, 3]
        return np.array([c.fx * p[0] / p[2] + c.cx, c.fy * p[1] / p[2] + c.cy])

    h = 1e-5
    Jw = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        Jw[:, k] = (pi(mu + e) - pi(mu - e)) / (2 * h)
    return Jw @ Sig @ Jw.T + dil * np.eye(2), pi(mu)


# ---------------------------------------------------------------------------
# Eq. 14 decode
# ---------------------------------------------------------------------------

def test_rvq_single_stage_is_table_lookup():
    rng = np.random.default_rng(0)
    cb = rng.normal(size=(1, 64, 4))
    idx = rng.integers(0, 64, size=(1, 500), dtype=np.uint8)
    out = O.rvq_decode(cb, idx)
    assert np.array_equal(out, cb[0][idx[0]])


def test_rvq_stage_sum_recovers_index_digits():
    # C^s[k] = k * 256^-s: the decoded sum is the index digits in base 256
    L, K = 3, 256
    cb = np.zeros((L, K, 1))
    for s in range(L):
        cb[s, :, 0] = np.arange(K) * 256.0 ** (-s)
    rng = np.random.default_rng(1)
    idx = rng.integers(0, K, size=(L, 1000), dtype=np.uint8)
    v = O.rvq_decode(cb, idx)[:, 0]
    for s in range(L):
        digit = np.floor(v).astype(np.int64)
        assert np.array_equal(digit, idx[s])
        v = (v - digit) * 256.0


def test_rvq_matches_gather_sum():
    rng = np.random.default_rng(2)
    cb = rng.normal(size=(4, 48, 3))
    idx = rng.integers(0, 48, size=(4, 333), dtype=np.uint8)
    ref = sum(cb[s][idx[s]] for s in range(4))
    assert np.allclose(O.rvq_decode(cb, idx), ref, rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# Eq. 2-3 projection
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dil", [0.0, 0.3])
def test_projection_on_axis_closed_form(dil):
    sx, sy, sz, z = 0.11, 0.07, 0.05, 2.5
    sc = raw_scene([[0, 0, z]], [np.log([sx, sy, sz])], [[1, 0, 0, 0]], [0.0], [[0.5, 0.5, 0.5]])
    c = cam(300.0, 250.0, 31.5, 23.5, 64, 48)
    o = O.Oracle(sc, [c], params=dict(dilation=dil))
    proj, b32, _ = o.projection()
    A = (300.0 * sx / z) ** 2 + dil
    Cc = (250.0 * sy / z) ** 2 + dil
    assert proj[0, 10] == 1
    assert np.allclose(proj[0, 3:6], [1 / A, 0.0, 1 / Cc], rtol=1e-6, atol=1e-12)
    assert np.allclose(proj[0, 0:3], [31.5, 23.5, z], rtol=1e-6)
    assert proj[0, 11] == math.ceil(3 * math.sqrt(max(A, Cc)))


def test_projection_rotated_matches_independent_route():
    rng = np.random.default_rng(3)
    n = 40
    q = synth.random_quats(rng, n)
    mu = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(2, 4, n)], 1)
    ls = rng.uniform(-3.5, -2.0, (n, 3))
    sc = raw_scene(mu, ls, q, np.zeros(n), np.full((n, 3), 0.5))
    T = synth.perturb_pose(synth.identity_pose(), rng, 10.0, 0.1).astype(np.float32)
    c = cam(120.0, 110.0, 63.5, 47.5, 128, 96, T)
    o = O.Oracle(sc, [c], params=dict(jacobian_clamp=0, dilation=0.3))
    proj, _, _ = o.projection()
    checked = 0
    for i in range(n):
        if proj[i, 10] != 1:
            continue
        S2, uv = sigma2d_independent(mu[i].astype(np.float32).astype(np.float64), np.exp(ls[i].astype(np.float32).astype(np.float64)),
                                     q[i].astype(np.float32), c, 0.3)
        a, b, cc = proj[i, 3:6]
        conic_inv = np.linalg.inv(np.array([[a, b], [b, cc]]))
        assert np.allclose(conic_inv, S2, rtol=2e-7, atol=1e-9)
        assert np.allclose(proj[i, 0:2], uv, rtol=1e-10)
        checked += 1
    assert checked > 20


def test_fp32_binning_expressions_bit_exact():
    """u32, v32, z32 follow the stated FP32 expression order exactly."""
    sc = synth.room_scene(n_anchors=3000)
    c = synth.room_camera(320, 180, 160.0)
    o = O.Oracle(sc, [c])
    _, b32, _ = o.projection()
    f = np.float32
    a = np.arange(sc.n) // sc.k
    i = np.arange(sc.n) % sc.k
    mu = sc.anchor_xyz[a] + (sc.offsets[a, i] * sc.anchor_l[a])
    T = c.T_cw
    p = [((T[r, 0] * mu[:, 0] + T[r, 1] * mu[:, 1]) + T[r, 2] * mu[:, 2]) + T[r, 3] for r in range(3)]
    z = p[2]
    front = z > f(c.near)
    thr = O.mask_threshold(sc.mask_eps)
    front &= sc.mask_logit > thr
    u = (f(c.fx) * p[0]) / z + f(c.cx)
    v = (f(c.fy) * p[1]) / z + f(c.cy)
    assert u.dtype == np.float32 and front.sum() > 1000
    assert np.array_equal(b32[front, 0].view(np.uint32), u[front].view(np.uint32))
    assert np.array_equal(b32[front, 1].view(np.uint32), v[front].view(np.uint32))
    assert np.array_equal(b32[front, 2].view(np.uint32), z[front].view(np.uint32))


# ---------------------------------------------------------------------------
# Eq. 16-18 compositing
# ---------------------------------------------------------------------------

def test_single_gaussian_closed_form():
    mu = np.array([0.05, -0.03, 2.0])
    ls = np.log([0.08, 0.05, 0.06])
    q = np.array([0.9, 0.2, -0.3, 0.1])
    q /= np.linalg.norm(q)
    ol, rgb = 0.7, np.array([0.2, 0.6, 0.9])
    sc = raw_scene([mu], [ls], [q], [ol], [rgb])
    c = cam(100.0, 100.0, 15.5, 15.5, 32, 32)
    o = O.Oracle(sc, [c], params=dict(jacobian_clamp=0))
    out = o.forward()
    mu32 = mu.astype(np.float32).astype(np.float64)
    S2, uv = sigma2d_independent(mu32, np.exp(ls.astype(np.float32).astype(np.float64)), q.astype(np.float32), c, 0.3)
    conic = np.linalg.inv(S2)
    lam = np.linalg.eigvalsh(S2).max()
    r = math.ceil(3 * math.sqrt(lam))
    _, b32, _ = o.projection()
    u32, v32 = b32[0, 0], b32[0, 1]
    x0, x1 = max(0, math.floor((u32 - np.float32(r)) / 16)), min(2, math.floor((u32 + np.float32(r)) / 16) + 1)
    y0, y1 = max(0, math.floor((v32 - np.float32(r)) / 16)), min(2, math.floor((v32 + np.float32(r)) / 16) + 1)
    opac = 1 / (1 + math.exp(-np.float32(ol)))
    z = (np.asarray(c.T_cw, np.float64)[:, :3] @ mu32 + np.asarray(c.T_cw, np.float64)[:, 3])[2]
    C = out["C"].reshape(3, 32, 32)
    for py in range(32):
        for px in range(32):
            d = np.array([uv[0] - px, uv[1] - py])
            al = min(0.99, opac * math.exp(-0.5 * d @ conic @ d))
            inside = x0 <= px // 16 < x1 and y0 <= py // 16 < y1
            if al < 1 / 255 or not inside:
                al = 0.0
            assert abs(out["S"][py * 32 + px] - al) < 1e-9
            assert abs(out["D"][py * 32 + px] - z * al) < 1e-9
            assert np.allclose(C[:, py, px], rgb.astype(np.float32) * al, atol=1e-9)
    assert out["S"].max() > 0.3


def test_compositing_invariants_tiny_scene():
    sc = synth.tiny_scene()
    c = synth.tiny_camera()
    o = O.Oracle(sc, [c])
    out = o.forward()
    S, T = out["S"], out["T_final"]
    assert S.min() >= 0 and S.max() < 1
    assert np.allclose(S, 1 - T, atol=1e-12)
    rgb_max = sc.groups["rgb"].raw.max(0)
    C = out["C"].reshape(3, -1)
    for ch in range(3):
        assert np.all(C[ch] <= rgb_max[ch] * S + 1e-12)
    proj, _, _ = o.projection()
    zmax = proj[proj[:, 10] == 1, 2].max()
    assert np.all(out["D"] <= zmax * S + 1e-12)
    assert out["evaluated"] == out["n_eval"].sum()
    assert np.all(out["n_contrib"] <= out["n_eval"])


def test_opaque_front_pair_occludes_everything_behind():
    rng = np.random.default_rng(5)
    front_mu = [[0.0, 0.0, 1.0], [0.001, 0.0, 1.05]]
    n_b = 200
    back_mu = np.stack([rng.uniform(-0.3, 0.3, n_b), rng.uniform(-0.3, 0.3, n_b), rng.uniform(2, 4, n_b)], 1)
    mu = np.concatenate([front_mu, back_mu])
    n = len(mu)
    ls = np.concatenate([np.full((2, 3), np.log(1.0)), rng.uniform(-3, -2, (n_b, 3))])
    q = np.concatenate([[[1, 0, 0, 0]] * 2, synth.random_quats(rng, n_b)])
    ol = np.concatenate([[12.0, 12.0], rng.normal(size=n_b)])
    rgb = rng.uniform(size=(n, 3))
    c = cam(50.0, 50.0, 15.5, 15.5, 32, 32)
    full = O.Oracle(raw_scene(mu, ls, q, ol, rgb), [c]).forward()
    front = O.Oracle(raw_scene(mu[:2], ls[:2], q[:2], ol[:2], rgb[:2]), [c]).forward()
    # centre pixels: both front Gaussians at alpha = 0.99, so transmittance
    # reaches 1e-4 and nothing behind may contribute
    for py in range(12, 20):
        for px in range(12, 20):
            i = py * 32 + px
            assert abs(front["S"][i] - 0.9999) < 1e-12
            assert full["S"][i] == front["S"][i] and full["D"][i] == front["D"][i]
    assert np.abs(full["S"] - front["S"]).max() > 1e-4  # away from the centre the back does show


def test_magnitude_sums_are_the_render_of_absolute_colours():
    """C_abs is the sum over blended Gaussians of |c| alpha T: the compositing
    weights do not depend on colour, so it equals the C of the same scene
    with every colour replaced by its absolute value; and it equals |C|
    where the colours share one sign."""
    sc = synth.tiny_scene(seed=13, n=700)
    rgb = sc.groups["rgb"].raw.copy()
    rgb[::2] -= 0.6                                   # mixed signs
    g = dict(sc.groups)
    g["rgb"] = synth.Group(3, raw=rgb)
    mixed = synth.Scene(sc.anchor_xyz, sc.anchor_l, sc.offsets, g)
    g2 = dict(sc.groups)
    g2["rgb"] = synth.Group(3, raw=np.abs(rgb))
    absolute = synth.Scene(sc.anchor_xyz, sc.anchor_l, sc.offsets, g2)
    c = synth.tiny_camera()
    a = O.Oracle(mixed, [c]).forward()
    b = O.Oracle(absolute, [c]).forward()
    assert np.allclose(a["C_abs"], b["C"], rtol=1e-12, atol=1e-15)
    assert np.all(a["C_abs"] >= np.abs(a["C"]) - 1e-15)
    assert (a["C_abs"] > 1.5 * np.abs(a["C"])).any()      # cancellation does occur
    p = O.Oracle(sc, [c]).forward()                        # colours in [0, 1]
    assert np.array_equal(p["C_abs"], p["C"])


def test_flags_mark_decisions_at_their_thresholds():
    """A pixel placed where alpha = alpha_min exactly, and the opaque pair
    whose second Gaussian takes the transmittance exactly to t_min, are
    flagged (bits 0 and 2); pixels far from every threshold are not."""
    # one isotropic Gaussian on the optical axis: sigma^2 = (f s / z)^2 + dil
    f, ls, z, o_logit = 40.0, float(np.float32(math.log(0.05))), 2.0, 1.5
    sig2 = (f * math.exp(ls) / z) ** 2 + 0.3
    o = 1 / (1 + math.exp(-float(np.float32(o_logit))))
    d = math.sqrt(2 * sig2 * math.log(255 * o))          # alpha(d) = 1/255
    c = cam(f, f, 10.0 - d, 15.0, 32, 32)                  # the centre lies d px left of pixel (10, 15)
    sc = raw_scene([[0.0, 0.0, z]], [[ls] * 3], [[1, 0, 0, 0]], [o_logit], [[0.5, 0.5, 0.5]])
    out = O.Oracle(sc, [c]).forward()
    row = 15 * 32 + np.arange(32)
    assert out["flags"][row[10]] & 1
    assert not (out["flags"][row[4]] & 1) and out["margin"][row[4]] > 1   # close to the centre
    assert (out["flags"] != 0).mean() < 0.2
    # the opaque pair of the occlusion pin: T = 0.01 * 0.01 = t_min at the centre
    pair = raw_scene([[0.0, 0.0, 1.0], [0.001, 0.0, 1.05]], [[0.0] * 3] * 2, [[1, 0, 0, 0]] * 2, [12.0, 12.0],
                     [[0.1, 0.2, 0.3]] * 2)
    c2 = cam(50.0, 50.0, 15.5, 15.5, 32, 32)
    op = O.Oracle(pair, [c2]).forward()
    assert all(op["flags"][py * 32 + px] & 4 for py in range(12, 20) for px in range(12, 20))


def test_fp64_rect_count_sees_a_centre_rounding_across_a_tile_edge():
    """u = fx x / z + cx with fx = 3, x = fl32(20/3), z = 1, cx = 0: the FP32
    product 3 x rounds up to 20.0, the exact one is 19.9999995; with radius 4
    the FP32 rect starts at tile floor(16 / 16) = 1, the FP64 one at
    floor(15.9999995 / 16) = 0."""
    x = float(np.float32(20.0 / 3.0))
    assert np.float32(3.0) * np.float32(x) == np.float32(20.0) and 3.0 * x < 20.0
    # flat in z (the Jacobian's x/z^2 column would spread a round one):
    # sigma^2 = 9 s^2 + 0.3 = 1.4025, 3 sigma = 3.55, radius 4
    ls = [math.log(0.35), math.log(0.35), math.log(1e-4)]
    sc = raw_scene([[x, 0.0, 1.0]], [ls], [[1, 0, 0, 0]], [0.0], [[0.5, 0.5, 0.5]])
    o = O.Oracle(sc, [cam(3.0, 3.0, 0.0, 24.0, 64, 48)])
    proj, _, _ = o.projection()
    assert proj[0, 11] == 4 and proj[0, 12] == 1
    assert o.rect_fp64_diff() == (1, 0)
    # the same Gaussian a pixel to the left has both centres inside tile 0 + 4 px
    sc2 = raw_scene([[x - 4.0 / 3.0, 0.0, 1.0]], [ls], [[1, 0, 0, 0]], [0.0], [[0.5] * 3])
    assert O.Oracle(sc2, [cam(3.0, 3.0, 0.0, 24.0, 64, 48)]).rect_fp64_diff() == (0, 0)


@pytest.mark.parametrize("workload", ["mapping", "large view 0"])
def test_fp64_and_fp32_tile_rects_agree(workload):
    """The binning takes tile rects from the FP32 projected centre; the count
    of slots whose rect from the FP64 centre differs is reported and must be
    a negligible share (the radius itself, from FP64 lambda_max, is the same;
    borderline radii are counted apart)."""
    if workload == "mapping":
        o = O.Oracle(synth.room_scene(), [synth.room_camera()])
    else:
        o = O.Oracle(synth.large_scene(), synth.large_cameras()[:1])
    proj, _, _ = o.projection()
    reached = int((proj[:, 11] > 0).sum())
    diff, borderline = o.rect_fp64_diff()
    print(f"{workload}: {diff} of {reached} slots have another FP64 rect; {borderline} borderline radii")
    assert diff <= 1e-3 * reached and borderline <= 1e-2 * reached


def test_permutation_invariance():
    sc = synth.tiny_scene(seed=11, n=600)
    c = synth.tiny_camera()
    perm = np.random.default_rng(6).permutation(sc.n)
    g = {k: synth.Group(v.dim, raw=v.raw[perm]) for k, v in sc.groups.items()}
    sp = synth.Scene(sc.anchor_xyz[perm], sc.anchor_l[perm], sc.offsets[perm], g)
    a = O.Oracle(sc, [c]).forward()
    b = O.Oracle(sp, [c]).forward()
    for k in ("C", "D", "S", "n_eval"):
        assert np.array_equal(a[k], b[k]), k


def test_mask_equals_deletion():
    sc = synth.box_scene(21, 800, frac_masked=0.3)
    c = synth.tiny_camera()
    keep = sc.mask_logit > O.mask_threshold(sc.mask_eps)
    assert 0 < keep.sum() < sc.n
    g = {k: synth.Group(v.dim, raw=v.raw[keep]) for k, v in sc.groups.items()}
    sd = synth.Scene(sc.anchor_xyz[keep], sc.anchor_l[keep], sc.offsets[keep], g)
    a = O.Oracle(sc, [c]).forward()
    b = O.Oracle(sd, [c]).forward()
    for k in ("C", "D", "S"):
        assert np.array_equal(a[k], b[k]), k


def test_rigid_motion_invariance():
    sc = synth.tiny_scene(seed=12, n=500)
    c = synth.tiny_camera()
    Rg = Rotation.from_rotvec([0.3, -0.2, 0.5])
    tg = np.array([0.4, -0.7, 1.1])
    mu2 = Rg.apply(sc.anchor_xyz.astype(np.float64)) + tg
    qr = sc.groups["rot"].raw.astype(np.float64)
    q2 = (Rg * Rotation.from_quat(qr[:, [1, 2, 3, 0]])).as_quat()[:, [3, 0, 1, 2]]
    g = dict(sc.groups)
    g["rot"] = synth.Group(4, raw=q2.astype(np.float32))
    s2 = synth.Scene(mu2.astype(np.float32), sc.anchor_l, sc.offsets, g)
    T = np.asarray(c.T_cw, np.float64)
    Rm = Rg.as_matrix()
    T2 = np.zeros((3, 4))
    T2[:, :3] = T[:, :3] @ Rm.T
    T2[:, 3] = T[:, 3] - T[:, :3] @ Rm.T @ tg
    c2 = synth.camera(c.fx, c.fy, c.cx, c.cy, c.width, c.height, T2)
    # float32 inputs differ by rounding only: compare in FP64 with the moved
    # arrays passed exactly (overrides), flags excluded
    a = O.Oracle(sc, [c]).forward()
    b = O.Oracle(s2, [c2], overrides=dict(anchor_xyz=mu2, raw_rot=q2, T_cw=[T2])).forward()
    ok = (a["flags"] == 0) & (b["flags"] == 0)
    assert ok.mean() > 0.99
    dS = np.abs(a["S"] - b["S"])[ok]
    # membership (FP32 rects) may flip only for a Gaussian exactly at a tile edge
    assert (dS > 1e-7).mean() < 2e-3
    assert np.median(dS) < 1e-12


def test_brute_force_per_pixel_compositing():
    """Per pixel: sort every Gaussian whose rect holds the pixel's tile by
    (FP32 depth, index) and composite directly; no tiles, no lists."""
    rng = np.random.default_rng(7)
    n = 50
    mu = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(1, 3, n)], 1)
    sc = raw_scene(mu, rng.uniform(-3.5, -2.2, (n, 3)), synth.random_quats(rng, n), rng.normal(size=n),
                   rng.uniform(size=(n, 3)))
    c = cam(40.0, 40.0, 15.5, 15.5, 32, 32)
    o = O.Oracle(sc, [c])
    out = o.forward()
    proj, b32, _ = o.projection()
    zbits = b32[:, 2].view(np.uint32)
    for py in range(32):
        for px in range(32):
            tx, ty = px // 16, py // 16
            cand = [i for i in range(n) if proj[i, 10] == 1 and proj[i, 12] <= tx < proj[i, 14]
                    and proj[i, 13] <= ty < proj[i, 15]]
            cand.sort(key=lambda i: (int(zbits[i]), i))
            T, Cacc, D, S = 1.0, np.zeros(3), 0.0, 0.0
            for i in cand:
                dx, dy = proj[i, 0] - px, proj[i, 1] - py
                a, b, cc = proj[i, 3:6]
                pw = -0.5 * (a * dx * dx + cc * dy * dy) - b * dx * dy
                if pw > 0:
                    continue
                al = min(0.99, proj[i, 6] * math.exp(pw))
                if al < 1 / 255:
                    continue
                if T * (1 - al) < 1e-4:
                    break
                Cacc += proj[i, 7:10] * al * T
                D += proj[i, 2] * al * T
                S += al * T
                T *= 1 - al
            k = py * 32 + px
            assert abs(out["S"][k] - S) < 1e-12 and abs(out["D"][k] - D) < 1e-12
            assert np.allclose(out["C"].reshape(3, -1)[:, k], Cacc, atol=1e-12)


def test_bins_are_lexicographic_tile_depth_index():
    sc = synth.tiny_scene()
    c = synth.tiny_camera()
    o = O.Oracle(sc, [c])
    proj, b32, _ = o.projection()
    ts, lst = o.bins()
    zb = b32[:, 2].view(np.uint32).astype(np.int64)
    keys, zs, ns = [], [], []
    for i in np.nonzero(proj[:, 10] == 1)[0]:
        x0, y0, x1, y1 = proj[i, 12:16].astype(int)
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                keys.append(ty * 4 + tx)
                zs.append(zb[i])
                ns.append(i)
    order = np.lexsort((ns, zs, keys))
    assert np.array_equal(np.asarray(ns)[order], lst)
    assert np.array_equal(np.bincount(np.asarray(keys), minlength=12), np.diff(ts))


# ---------------------------------------------------------------------------
# backward: central finite differences in FP64
# ---------------------------------------------------------------------------

def fd_scene(coded: bool, seed: int, with_mask: bool = False):
    rng = np.random.default_rng(seed)
    na, k = 3, 2
    xyz = np.stack([rng.uniform(-0.1, 0.1, na), rng.uniform(-0.1, 0.1, na), [1.6, 2.2, 2.9]], 1).astype(np.float32)
    l = rng.uniform(0.5, 1.5, (na, 3)).astype(np.float32)
    off = rng.normal(0, 0.06, (na, k, 3)).astype(np.float32)
    n = na * k
    if coded:
        L, K = 2, 4
        groups = {}
        for name, d in synth.GROUP_DIMS.items():
            cb = rng.normal(0, 0.3, (L, K, d)).astype(np.float32)
            if name == "logscale":
                cb[0] += -2.4
            if name == "rot":
                cb[0, :, 0] += 1.5
            if name == "rgb":
                cb[0] += 0.5
            groups[name] = synth.Group(d, codebook=cb, idx=rng.integers(0, K, (L, n), dtype=np.uint8))
    else:
        groups = {
            "logscale": synth.Group(3, raw=rng.uniform(-2.6, -2.2, (n, 3)).astype(np.float32)),
            "rot": synth.Group(4, raw=synth.random_quats(rng, n).astype(np.float32)),
            "opacity": synth.Group(1, raw=rng.normal(0, 0.7, (n, 1)).astype(np.float32)),
            "rgb": synth.Group(3, raw=rng.uniform(0, 1, (n, 3)).astype(np.float32)),
        }
    mask = None
    if with_mask:
        mask = rng.uniform(1, 3, n).astype(np.float32)
        mask[1] = -2.0
    return synth.Scene(xyz, l, off, groups, mask, 0.5)


def fd_cams(n_views, off_screen=False):
    cams = []
    rng = np.random.default_rng(40)
    for v in range(n_views):
        T = synth.perturb_pose(synth.identity_pose(), rng, 3.0, 0.03) if v else synth.identity_pose()
        cams.append(cam(40.0, 40.0, 7.5, 7.5, 16, 16, T))
    return cams


def _arrays(scene):
    arr = dict(anchor_xyz=scene.anchor_xyz, anchor_l=scene.anchor_l, offsets=scene.offsets)
    for name, g in scene.groups.items():
        arr[("cb_" if g.coded else "raw_") + name] = g.codebook if g.coded else g.raw
    return {k: np.asarray(v, np.float64) for k, v in arr.items()}


def _objective(scene, cams, ups, overrides):
    o = O.Oracle(scene, cams, overrides=overrides)
    f = o.forward()
    assert not np.any(f["flags"]), "finite differences crossed a threshold"
    return float(ups[0] @ f["C"] + ups[1] @ f["D"] + ups[2] @ f["S"])


def _fd_check(scene, cams, names=None, h=1e-6, rtol=2e-5):
    o = O.Oracle(scene, cams)
    f = o.forward()
    assert f["S"].max() > 0.5 and not np.any(f["flags"])
    ups = synth.upstream_grads(99, o.n_pixels, scale=o.n_pixels)
    ups = [u.astype(np.float64) for u in ups]
    grads = o.backward(*ups)
    base = _arrays(scene)
    key = {"anchor_xyz": "anchor_xyz", "anchor_l": "anchor_l", "offsets": "offsets"}
    for name in (names or base):
        arr = base[name]
        g = grads[key[name]] if name in key else grads[name.split("_", 1)[1]]
        assert g.shape == arr.shape, name
        fd = np.zeros(arr.size)
        for j in range(arr.size):
            hp = h * max(1.0, abs(arr.flat[j]))
            a1 = arr.copy(); a1.flat[j] += hp
            a2 = arr.copy(); a2.flat[j] -= hp
            fd[j] = (_objective(scene, cams, ups, {name: a1}) - _objective(scene, cams, ups, {name: a2})) / (2 * hp)
        scale = max(1e-6, np.abs(fd).max())
        assert np.abs(fd - g.ravel()).max() <= rtol * scale, (name, fd, g.ravel())
    return o, ups, grads


@pytest.mark.parametrize("coded", [False, True])
def test_fd_scene_parameters(coded):
    sc = fd_scene(coded, seed=31 if coded else 30)
    _fd_check(sc, fd_cams(1))


def test_fd_two_views_and_pose():
    sc = fd_scene(False, seed=32)
    cams = fd_cams(2)
    o, ups, grads = _fd_check(sc, cams, names=["anchor_xyz", "raw_rot", "raw_logscale"])
    h = 1e-6
    for v in range(2):
        T0 = np.eye(4)
        T0[:3, :] = np.asarray(cams[v].T_cw, np.float64)
        for k in range(6):
            xi = np.zeros(6)
            xi[k] = h
            Ts = []
            for sgn in (1, -1):
                X = np.zeros((4, 4))
                rho, phi = sgn * xi[:3], sgn * xi[3:]
                X[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
                X[:3, 3] = rho
                Tv = [np.asarray(c.T_cw, np.float64) for c in cams]
                Tv[v] = (expm(X) @ T0)[:3, :]
                Ts.append(_objective(sc, cams, ups, {"T_cw": Tv}))
            fd = (Ts[0] - Ts[1]) / (2 * h)
            assert abs(fd - grads["pose"][v, k]) <= 2e-5 * max(1e-6, np.abs(grads["pose"][v]).max()), (v, k)


def test_fd_jacobian_clamp_branch():
    """A Gaussian whose centre lies off screen beyond the clamp still reaches
    the image; the clamped Jacobian's derivative is exact on that branch."""
    mu = [[-0.45, 0.0, 1.5], [0.02, 0.03, 2.0]]
    sc = raw_scene(mu, [np.log([0.25, 0.2, 0.2]), np.log([0.06, 0.05, 0.07])],
                   [[0.9, 0.1, 0.3, -0.2], [1, 0, 0, 0]], [2.0, 0.3], [[0.9, 0.1, 0.2], [0.1, 0.8, 0.3]])
    cams = [cam(40.0, 40.0, 7.5, 7.5, 16, 16)]
    o = O.Oracle(sc, cams)
    proj, _, _ = o.projection()
    assert proj[0, 10] == 1 and -0.45 / 1.5 < -1.3 * 8 / 40  # clamped in x
    _fd_check(sc, cams, names=["anchor_xyz", "raw_logscale", "raw_rot"])


def test_fd_mask_straight_through():
    """Eq. 11-12: with hat s = M s and hat alpha = M alpha, the estimator is
    dL/dm = dL/dM * sigmoid'(m) at M = 1; dL/dM is checked by differencing a
    continuous multiplier M on s and alpha."""
    sc = fd_scene(False, seed=33, with_mask=True)
    cams = fd_cams(1)
    o = O.Oracle(sc, cams)
    ups = [u.astype(np.float64) for u in synth.upstream_grads(98, o.n_pixels, scale=o.n_pixels)]
    grads = o.backward(*ups)
    base = _arrays(sc)
    h = 1e-6
    keep = sc.mask_logit > O.mask_threshold(0.5)
    assert not keep[1] and grads["mask_logit"][1] == 0.0
    for n in np.nonzero(keep)[0]:
        vals = []
        for M in (1 + h, 1 - h):
            ls = base["raw_logscale"].copy()
            ls[n] += math.log(M)
            op = base["raw_opacity"].copy()
            a = M / (1 + math.exp(-op[n, 0]))
            op[n, 0] = math.log(a / (1 - a))
            vals.append(_objective(sc, cams, ups, {"raw_logscale": ls, "raw_opacity": op}))
        dM = (vals[0] - vals[1]) / (2 * h)
        sm = 1 / (1 + math.exp(-float(sc.mask_logit[n])))
        assert abs(dM * sm * (1 - sm) - grads["mask_logit"][n]) <= 1e-6 * max(1e-3, abs(dM)), n


def test_icp_closed_form_identity_pose():
    rng = np.random.default_rng(8)
    n = 30
    mu = rng.normal(0, 1, (n, 3)) + [0, 0, 3]
    sc = raw_scene(mu, np.full((n, 3), -3.0), [[1, 0, 0, 0]] * n, np.zeros(n), np.full((n, 3), 0.5))
    c = cam(50, 50, 32, 24, 64, 48)
    q, w = synth.icp_targets(9, 1, n)
    loss, dpose = O.Oracle(sc, [c]).icp(q, w)
    m = mu.astype(np.float32).astype(np.float64)
    r = m - q[0]
    assert np.isclose(loss[0], np.sum(w[0][:, None] * r * r), rtol=1e-12)
    g = 2 * w[0][:, None] * r
    assert np.allclose(dpose[0, :3], g.sum(0), rtol=1e-12)
    assert np.allclose(dpose[0, 3:], np.cross(m, g).sum(0), rtol=1e-10, atol=1e-12)


def test_icp_pose_gradient_fd():
    rng = np.random.default_rng(10)
    n = 20
    mu = rng.normal(0, 1, (n, 3)) + [0, 0, 3]
    sc = raw_scene(mu, np.full((n, 3), -3.0), [[1, 0, 0, 0]] * n, np.zeros(n), np.full((n, 3), 0.5))
    T = synth.perturb_pose(synth.identity_pose(), rng, 5.0, 0.1)
    c = cam(50, 50, 32, 24, 64, 48, T)
    q, w = synth.icp_targets(11, 1, n)
    _, dpose = O.Oracle(sc, [c]).icp(q, w)
    T0 = np.eye(4)
    T0[:3] = np.asarray(c.T_cw, np.float64)
    h = 1e-6
    for k in range(6):
        vals = []
        for sgn in (1, -1):
            xi = np.zeros(6)
            xi[k] = sgn * h
            X = np.zeros((4, 4))
            X[:3, :3] = [[0, -xi[5], xi[4]], [xi[5], 0, -xi[3]], [-xi[4], xi[3], 0]]
            X[:3, 3] = xi[:3]
            Tn = (expm(X) @ T0)[:3]
            vals.append(O.Oracle(sc, [c], overrides=dict(T_cw=[Tn])).icp(q, w)[0][0])
        assert abs((vals[0] - vals[1]) / (2 * h) - dpose[0, k]) < 1e-5 * np.abs(dpose).max()


def test_loss_l1_matches_definition():
    rng = np.random.default_rng(12)
    n = 500
    C_, Ct = rng.uniform(size=3 * n), rng.uniform(size=3 * n)
    D_, Dt = rng.uniform(0, 3, n), rng.uniform(0, 3, n)
    Dt[::7] = 0.0
    S_ = rng.uniform(size=n)
    L, dC, dD = O.loss_l1(C_, D_, S_, Ct, Dt, 0.5)
    valid = Dt > 0
    ref = np.abs(C_ - Ct).mean() + 0.5 * np.abs(D_ - Dt)[valid].mean()
    assert np.isclose(L, ref, rtol=1e-13)
    assert np.allclose(dC, np.sign(C_ - Ct) / (3 * n))
    assert np.allclose(dD, np.where(valid, 0.5 * np.sign(D_ - Dt) / valid.sum(), 0))
    Lg, dCg, _ = O.loss_l1(C_, D_, S_, Ct, Dt, 0.5, gate=0.99)
    gate = np.tile(S_ > 0.99, 3)
    assert np.allclose(dCg, np.where(gate, np.sign(C_ - Ct) / (3 * n), 0))


# ---------------------------------------------------------------------------
# exact identities of the reverse mode
# ---------------------------------------------------------------------------

def _decoded_raw_twin(coded_scene):
    """The same scene with every coded group replaced by its decoded values
    (numpy gather-sum, not the oracle's decode)."""
    groups = {}
    for name, g in coded_scene.groups.items():
        if g.coded:
            dec = sum(g.codebook[s][g.idx[s].astype(np.int64)] for s in range(g.codebook.shape[0]))
            groups[name] = synth.Group(g.dim, raw=dec.astype(np.float32))
        else:
            groups[name] = g
    return synth.Scene(coded_scene.anchor_xyz, coded_scene.anchor_l, coded_scene.offsets, groups,
                       coded_scene.mask_logit, coded_scene.mask_eps)


def test_codebook_gradient_is_the_scatter_sum_of_attribute_gradients():
    """dL/dC^s[k] = sum of dL/dattr_n over the Gaussians whose stage-s index
    is k (Eq. 14 is a sum of gathers), checked against the per-Gaussian
    gradients of the decoded twin scene."""
    sc = synth.room_scene(seed=1002, n_anchors=600)
    cams = [synth.room_camera(96, 64, 48.0)]
    ups = synth.upstream_grads(5, 96 * 64, scale=1.0)
    g_coded = O.Oracle(sc, cams).backward(*ups)
    g_raw = O.Oracle(_decoded_raw_twin(sc), cams).backward(*ups)
    for name, g in sc.groups.items():
        per_gauss = np.asarray(g_raw[name], np.float64)
        L, K, d = g.codebook.shape
        want = np.zeros((L, K, d))
        for s in range(L):
            np.add.at(want[s], g.idx[s].astype(np.int64), per_gauss)
        got = np.asarray(g_coded[name], np.float64)
        # the twin's attributes are the FP32 rounding of the FP64 decode
        assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max(), name


def test_translational_pose_gradient_is_the_rotated_sum_of_mean_gradients():
    """d/d rho of L(exp(xi^) T_cw) at 0 = sum_n dL/dp_c,n = R_cw sum_n dL/dmu_n,
    and sum_n dL/dmu_n = sum over anchors of dL/dx_a (Eq. 7)."""
    sc = synth.room_scene(seed=1002, n_anchors=800)
    cams = [synth.room_camera(96, 64, 48.0, pose_seed=3, jitter_deg=5.0, jitter_m=0.1)]
    o = O.Oracle(sc, cams)
    g = o.backward(*synth.upstream_grads(6, 96 * 64, scale=1.0))
    R = np.asarray(cams[0].T_cw, np.float64)[:, :3]
    want = R @ np.asarray(g["anchor_xyz"], np.float64).sum(axis=0)
    got = np.asarray(g["pose"], np.float64)[0][:3]
    # exact up to R R^T = I for the FP32 rotation (~1e-7)
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max(), (got, want)


def test_window_restricts_compositing_to_its_pixels():
    """A window composites exactly the whole-image values inside it and
    nothing outside; its backward equals the whole-image backward of
    upstream gradients that vanish outside it."""
    sc = synth.tiny_scene()
    cams = [synth.tiny_camera()]
    full = O.Oracle(sc, cams)
    f = full.forward()
    o = O.Oracle(sc, cams)
    o.set_window(0, 16, 16, 48, 32)
    w = o.forward()
    W, H = cams[0].width, cams[0].height
    inside = np.zeros((H, W), bool)
    inside[16:32, 16:48] = True
    m = inside.ravel()
    assert np.array_equal(w["S"][m], f["S"][m]) and np.all(w["S"][~m] == 0)
    assert np.array_equal(w["C"][np.tile(m, 3)], f["C"][np.tile(m, 3)])
    ups = synth.upstream_grads(8, W * H, scale=1.0)
    ups_in = [ups[0] * np.tile(m, 3), ups[1] * m, ups[2] * m]
    gw = o.backward(*ups)
    gf = full.backward(*ups_in)
    for k in gf:
        assert np.allclose(np.asarray(gw[k]), np.asarray(gf[k]), rtol=1e-12, atol=1e-15), k


# ---------------------------------------------------------------------------
# Eq. 14 (second line) and Eq. 15: residual quantisation encode and its loss
# ---------------------------------------------------------------------------

def test_rvq_encode_single_stage_is_the_nearest_codeword():
    from oracle.rvq_encode import rvq_encode
    rng = np.random.default_rng(70)
    cb = rng.normal(size=(1, 64, 3)).astype(np.float32)
    x = rng.normal(size=(500, 3)).astype(np.float32)
    d = ((cb[0][None, :, :].astype(np.float64) - x[:, None, :].astype(np.float64)) ** 2).sum(-1)
    srt = np.sort(d, axis=1)
    clear = (srt[:, 1] - srt[:, 0]) > 1e-5 * srt[:, 1]      # no near-tie the FP32 order could flip
    assert clear.mean() > 0.95
    idx = rvq_encode(cb, x)
    assert np.array_equal(idx[0][clear], d.argmin(axis=1)[clear])


def test_rvq_encode_recovers_digits():
    """Codewords k * 16^-(s+1) in every component and vectors sum_s d_s
    16^-(s+1) with digits d_s < 8: the tail after stage s is below half the
    stage's spacing, so the nearest codeword is the digit itself and the
    encoding returns exactly the digits."""
    from oracle.rvq_encode import rvq_encode
    L, K, d = 4, 16, 3
    cb = np.zeros((L, K, d), np.float32)
    for s in range(L):
        cb[s] = (np.arange(K, dtype=np.float64)[:, None] * 16.0 ** -(s + 1)).astype(np.float32)
    rng = np.random.default_rng(71)
    digits = rng.integers(0, K // 2, size=(L, 300))
    x = np.zeros((300, d), np.float64)
    for s in range(L):
        x += (digits[s] * 16.0 ** -(s + 1))[:, None]
    idx = rvq_encode(cb, x.astype(np.float32))
    assert np.array_equal(idx, digits.astype(np.uint8))


def test_rvq_encode_ties_go_to_the_lowest_index_and_error_never_grows():
    from oracle import oracle as Ob
    from oracle.rvq_encode import rvq_encode
    rng = np.random.default_rng(72)
    cb = rng.normal(scale=0.5, size=(3, 32, 4)).astype(np.float32)
    cb[:, 0] = 0.0                      # a zero codeword in every stage: a stage can always keep the residual
    cb[:, 9] = cb[:, 5]                 # duplicates: 9 must never be chosen
    x = rng.normal(size=(400, 4)).astype(np.float32)
    idx = rvq_encode(cb, x)
    assert not np.any(idx == 9)
    err_prev = np.inf
    for s in range(1, 4):
        rec = Ob.rvq_decode(cb[:s], idx[:s])
        err = ((x.astype(np.float64) - rec) ** 2).sum(1)
        assert np.all(err <= np.minimum(err_prev, ((x.astype(np.float64)) ** 2).sum(1)) * (1 + 1e-5) + 1e-9)
        err_prev = err


def test_rvq_loss_matches_definition_and_finite_differences():
    from oracle.rvq_encode import rvq_encode, rvq_loss
    rng = np.random.default_rng(73)
    cb = rng.normal(scale=0.3, size=(3, 8, 2))
    x = rng.normal(size=(50, 2))
    idx = rvq_encode(cb.astype(np.float32), x.astype(np.float32))
    loss, grad = rvq_loss(cb, x, idx)
    # the definition, written as a loop over items and stages
    want = 0.0
    for n in range(50):
        lhat = np.zeros(2)
        for s in range(3):
            e = (x[n] - lhat) - cb[s][idx[s][n]]
            want += e @ e
            lhat += cb[s][idx[s][n]]
    assert abs(loss - want / (50 * 8)) < 1e-12
    # finite differences of the loss with the stop-gradient residuals held
    # fixed (sg: a perturbed codeword moves only its own term)
    h = 1e-6
    R = []
    lhat = np.zeros((50, 2))
    for s in range(3):
        R.append(x - lhat)
        lhat = lhat + cb[s][idx[s].astype(int)]

    def sg_loss(c):
        return sum(float(((R[s] - c[s][idx[s].astype(int)]) ** 2).sum()) for s in range(3)) / (50 * 8)
    for s, k, c in [(0, int(idx[0][0]), 0), (1, int(idx[1][3]), 1), (2, int(idx[2][7]), 0)]:
        cp, cm = cb.copy(), cb.copy()
        cp[s, k, c] += h
        cm[s, k, c] -= h
        fd = (sg_loss(cp) - sg_loss(cm)) / (2 * h)
        assert abs(fd - grad[s, k, c]) <= 1e-6 * max(1.0, abs(fd)), (s, k, c, fd, grad[s, k, c])
    for s in range(3):
        lhat = np.zeros((50, 2))
        for t in range(s):
            lhat += cb[t][idx[t].astype(int)]
        r = x - lhat
        g = np.zeros((8, 2))
        np.add.at(g, idx[s].astype(int), 2 * (cb[s][idx[s].astype(int)] - r))
        assert np.allclose(grad[s], g / (50 * 8), rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------------------
# sliding-window mask: hit counts (Eq. 13), mask loss, removal
# ---------------------------------------------------------------------------

def test_hit_counts_single_gaussian_closed_form():
    """One Gaussian: its hit count is the number of image pixels where
    alpha = o exp(-q/2) reaches 1/255 (it can never trigger the stop)."""
    c = cam(60.0, 60.0, 31.5, 23.5, 64, 48)
    sc = raw_scene([[0.1, -0.05, 2.0]], [[math.log(0.08), math.log(0.05), math.log(0.06)]],
                   [[0.9, 0.1, 0.3, -0.2]], [0.8], [[0.2, 0.5, 0.7]])
    o = O.Oracle(sc, [c])
    hits, seen = o.hit_counts()
    proj, _, _ = o.projection()
    u, v, a, b, cc, op = proj[0, 0], proj[0, 1], proj[0, 3], proj[0, 4], proj[0, 5], proj[0, 6]
    ys, xs = np.mgrid[0:48, 0:64]
    dx, dy = u - xs, v - ys
    alpha = np.minimum(0.99, op * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + cc * dy * dy)))
    # only pixels inside the Gaussian's tile rect are tested
    r0, r1, r2, r3 = (int(t) for t in proj[0, 12:16])
    inrect = (xs >= r0 * 16) & (xs < r2 * 16) & (ys >= r1 * 16) & (ys < r3 * 16)
    want = int(((alpha >= 1 / 255) & inrect).sum())
    assert want > 100 and hits[0] == want and seen[0] == 1


def test_hit_counts_sum_to_blended_pairs_and_views_add():
    sc = synth.tiny_scene()
    cams = [synth.tiny_camera(), synth.tiny_camera()]
    h2, s2 = O.Oracle(sc, cams).hit_counts(threads=4)
    h1, s1 = O.Oracle(sc, cams[:1]).hit_counts(threads=4)
    assert np.array_equal(h2, 2 * h1) and np.array_equal(s2, s1)
    assert h1.sum() > 0 and np.all(h1[s1 == 0] == 0)


def test_mask_loss_and_prune_definitions():
    from oracle.mask import mask_loss, mask_prune, sigmoid
    rng = np.random.default_rng(80)
    m = rng.normal(size=200)
    vis = rng.uniform(size=200) < 0.4
    L, g = mask_loss(m, vis, weight=0.5)
    assert abs(L - 0.5 * np.mean(sigmoid(m[vis]))) < 1e-15
    h = 1e-6
    for j in np.flatnonzero(vis)[:5]:
        mp, mm = m.copy(), m.copy()
        mp[j] += h
        mm[j] -= h
        fd = (mask_loss(mp, vis, 0.5)[0] - mask_loss(mm, vis, 0.5)[0]) / (2 * h)
        assert abs(fd - g[j]) < 1e-8
    assert np.all(g[~vis] == 0)
    hits = rng.integers(0, 5, 200)
    seen = rng.uniform(size=200) < 0.7
    nm, removed = mask_prune(m, hits, seen, 0.5, 2)
    assert np.array_equal(removed, (m <= 0) | (seen & (hits < 2)))
    assert np.all(np.isneginf(nm[removed])) and np.array_equal(nm[~removed], m[~removed])


# ---------------------------------------------------------------------------
# the SSIM term of the bundle-adjustment loss
# ---------------------------------------------------------------------------

def test_ssim_identical_images_and_constant_closed_form():
    from oracle.ssim import C1, ssim_loss
    rng = np.random.default_rng(90)
    x = rng.uniform(size=3 * 24 * 32)
    L, g = ssim_loss(x, x, 1, 32, 24)
    assert abs(L) < 1e-12 and np.abs(g).max() < 1e-12
    # two constant images a, b: away from the border (all window weights
    # inside) the variances vanish and SSIM = (2ab + C1) / (a^2 + b^2 + C1)
    a, b = 0.3, 0.7
    from oracle import ssim as S
    w = S.window()
    xa = np.full((24, 32), a)
    xb = np.full((24, 32), b)
    mx, my = S._filt(xa, w), S._filt(xb, w)
    sxx = S._filt(xa * xa, w) - mx * mx
    syy = S._filt(xb * xb, w) - my * my
    sxy = S._filt(xa * xb, w) - mx * my
    Smap = (2 * mx * my + C1) * (2 * sxy + S.C2) / ((mx * mx + my * my + C1) * (sxx + syy + S.C2))
    assert abs(Smap[12, 16] - (2 * a * b + C1) / (a * a + b * b + C1)) < 1e-12


def test_ssim_window_is_the_normalised_gaussian():
    from oracle.ssim import window
    w = window()
    assert w.shape == (11, 11) and abs(w.sum() - 1) < 1e-15
    assert abs(w[5, 6] / w[5, 5] - math.exp(-1 / (2 * 1.5 ** 2))) < 1e-14


def test_ssim_gradient_matches_finite_differences():
    from oracle.ssim import ssim_loss
    rng = np.random.default_rng(91)
    x = rng.uniform(size=3 * 20 * 18)
    y = np.clip(x + rng.normal(scale=0.1, size=x.size), 0, 1)
    L, g = ssim_loss(x, y, 1, 18, 20)
    h = 1e-6
    for j in rng.choice(x.size, 12, replace=False):
        xp, xm = x.copy(), x.copy()
        xp[j] += h
        xm[j] -= h
        fd = (ssim_loss(xp, y, 1, 18, 20)[0] - ssim_loss(xm, y, 1, 18, 20)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1e-3, abs(fd)), (j, fd, g[j])


# ---------------------------------------------------------------------------
# projective data association for the ICP term
# ---------------------------------------------------------------------------

def test_projective_association_on_a_plane():
    """A fronto-parallel target plane at depth 2.5: every Gaussian within the
    distance gate gets the plane's point on its pixel's ray, which lies on the
    plane and within half a pixel's footprint of the mean's own ray."""
    from oracle.icp_assoc import associate
    rng = np.random.default_rng(95)
    c = cam(80.0, 80.0, 31.5, 23.5, 64, 48)
    mu = np.stack([rng.uniform(-0.8, 0.8, 400), rng.uniform(-0.6, 0.6, 400), rng.uniform(2.4, 2.6, 400)], 1)
    Dt = np.full(64 * 48, 2.5)
    q, w = associate(mu, np.ones(400, bool), [c], Dt, 0.2)
    ok = w[0] > 0
    assert ok.sum() > 300
    assert np.allclose(q[0, ok, 2], 2.5)
    ray = mu[ok] / mu[ok, 2:3] * 2.5          # the mean's own ray at the plane
    assert np.abs(q[0, ok, :2] - ray[:, :2]).max() <= 0.5 * 2.5 / 80.0 + 1e-12
    # gated: a plane 0.5 m behind the means gives no correspondence at max_dist 0.2
    q2, w2 = associate(mu, np.ones(400, bool), [c], np.full(64 * 48, 3.0), 0.2)
    assert w2.sum() == 0


# ---------------------------------------------------------------------------
# anchor growing (Sec. "Sequential Anchor Point Growing", Eq. 10)
# ---------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    """The first three outputs of SplitMix64 seeded with 0, as published
    with the generator (Steele, Lea and Flood 2014; the reference outputs
    used to seed the xoshiro family)."""
    from oracle.grow import GAMMA, MASK64, splitmix64
    got = [splitmix64((i * GAMMA) & MASK64) for i in range(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def _hand_growth_case():
    # (position, gradient sum, count) per Gaussian; eps_g 1, tau_g 0.5, 3 levels
    rows = [((0.3, 0.3, 0.3), 1.2, 2),      # voxel mean 0.6: grows at level 1 only
            ((2.3, 0.1, 0.1), 3.0, 1),      # 3.0: levels 1, 2, 3
            ((2.6, 0.6, 0.6), 5.0, 1),      # same level-1 voxel; its level-2 voxel holds the new level-1 anchor
            ((5.2, 0.2, 0.2), 10.0, 1),     # level-1 voxel holds a scene anchor; levels 2, 3
            ((-0.5, 0.5, 0.5), 0.2, 1),     # level-1 voxel mean (0.2 + 0.9) / 2 = 0.55
            ((-0.7, 0.2, 0.2), 0.9, 1),
            ((-1.5, 0.5, 0.5), 0.9, 3),     # averages 0.3 and 0.3: mean 0.3 (a sum would pass)
            ((-1.2, 0.3, 0.3), 0.3, 1),
            ((-2.1, 0.9, 0.9), 0.3, 3),     # averages 0.1 and 1.0: mean 0.55 (pair-weighted 0.325)
            ((-2.9, 0.1, 0.1), 1.0, 1),     # level 2: 1.0 is not above tau_2 = 1
            ((10.2, 0.2, 0.2), 5.0, 0)]     # never seen
    mu = np.array([r[0] for r in rows], np.float32)
    gs = np.array([r[1] for r in rows], np.float32)
    gc = np.array([r[2] for r in rows], np.int64)
    anchors = np.array([[5.9, 0.9, 0.9]], np.float32)
    expected = {(1, (0.5, 0.5, 0.5)), (1, (2.5, 0.5, 0.5)), (1, (-0.5, 0.5, 0.5)), (1, (-2.5, 0.5, 0.5)),
                (2, (2.375, 0.125, 0.125)), (2, (5.125, 0.125, 0.125)),
                (3, (2.28125, 0.09375, 0.09375)), (3, (2.59375, 0.59375, 0.59375)),
                (3, (5.21875, 0.21875, 0.21875))}
    return mu, gs, gc, anchors, expected


def test_anchor_growing_hand_case():
    """Eq. 10's levels (eps / 4^(m-1), tau * 2^(m-1)), the voxel mean of the
    per-Gaussian averages, strict threshold, occupancy by scene anchors and by
    anchors grown at coarser levels, unseen Gaussians left out: every
    expected centre worked out by hand."""
    from oracle.grow import grow
    mu, gs, gc, anchors, expected = _hand_growth_case()
    out = grow(mu, gs, gc, anchors, 1.0, 0.5, levels=3, p_drop=0.0)
    got = {(m, tuple(float(x) for x in c)) for m, _, c in out}
    assert got == expected
    assert len(out) == len(expected)


def test_anchor_growing_brute_force_voxel_means():
    """Random Gaussians on a small grid: the grown set equals a brute-force
    enumeration of every voxel of every level (pure Python loops over the
    Gaussians per voxel)."""
    from oracle.grow import grow
    rng = np.random.default_rng(21)
    n = 300
    mu = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    gc = rng.integers(0, 4, size=n)
    gs = (gc * rng.uniform(0.0, 2.0, size=n)).astype(np.float32)
    anchors = rng.uniform(-1.0, 1.0, size=(5, 3)).astype(np.float32)
    eps_g, tau_g = 0.5, 0.6
    out = grow(mu, gs, gc, anchors, eps_g, tau_g, levels=2, p_drop=0.0)
    est = [tuple(a) for a in anchors.tolist()]
    want = set()
    for m in (1, 2):
        eps = eps_g / 4 ** (m - 1)
        tau = tau_g * 2 ** (m - 1)
        cells = {}
        for i in range(n):
            if gc[i] == 0:
                continue
            cell = tuple(int(np.floor(np.float32(mu[i][c]) / np.float32(eps))) for c in range(3))
            cells.setdefault(cell, []).append(float(np.float32(gs[i]) / np.float32(gc[i])))
        occ = {tuple(int(np.floor(np.float32(a[c]) / np.float32(eps))) for c in range(3)) for a in est}
        grown = []
        for cell, avgs in cells.items():
            if cell not in occ and sum(avgs) / len(avgs) > tau:
                grown.append(tuple(float(np.float32((cell[c] + 0.5) * eps)) for c in range(3)))
        want |= {(m, g) for g in grown}
        est += grown
    got = {(m, tuple(float(x) for x in c)) for m, _, c in out}
    assert got == want and len(want) > 10


def test_anchor_growing_random_elimination():
    """p_drop 0 keeps every candidate, 1 drops all; the kept sets are nested
    as p_drop grows; the kept fraction is binomial around 1 - p_drop."""
    from oracle.grow import grow
    rng = np.random.default_rng(22)
    n = 4000
    mu = rng.uniform(-10.0, 10.0, size=(n, 3)).astype(np.float32)
    gc = np.ones(n, np.int64)
    gs = np.full(n, 2.0, np.float32)
    anchors = np.zeros((0, 3), np.float32)
    full = {(m, k) for m, k, _ in grow(mu, gs, gc, anchors, 0.05, 1.0, levels=1, p_drop=0.0, seed=7)}
    assert len(full) == n
    assert grow(mu, gs, gc, anchors, 0.05, 1.0, levels=1, p_drop=1.0, seed=7) == []
    k3 = {(m, k) for m, k, _ in grow(mu, gs, gc, anchors, 0.05, 1.0, levels=1, p_drop=0.3, seed=7)}
    k7 = {(m, k) for m, k, _ in grow(mu, gs, gc, anchors, 0.05, 1.0, levels=1, p_drop=0.7, seed=7)}
    assert k7 <= k3 <= full
    for kept, p in ((k3, 0.3), (k7, 0.7)):
        sd = np.sqrt(n * p * (1 - p))
        assert abs(len(kept) - n * (1 - p)) < 5 * sd, (len(kept), p)
    other = {(m, k) for m, k, _ in grow(mu, gs, gc, anchors, 0.05, 1.0, levels=1, p_drop=0.3, seed=8)}
    assert other != k3


def test_anchor_positions_and_prune_definitions():
    """mu = x_a + O l per Gaussian; an anchor seen with mean opacity below
    tau_alpha is removed on all its Gaussians, an unseen one never, the
    threshold itself is kept."""
    from oracle.grow import positions, prune
    xa = np.array([[1.0, 2.0, 3.0]], np.float32)
    l = np.array([[0.5, 2.0, 1.0]], np.float32)
    off = np.array([[[1.0, 1.0, 1.0], [-2.0, 0.0, 0.25]]], np.float32)
    assert np.array_equal(positions(xa, l, off), np.array([[1.5, 4.0, 4.0], [0.0, 2.0, 3.25]], np.float32))
    k = 2
    m0 = np.zeros(8)
    s = np.array([0.05, 0.3, 0.0, 0.2], np.float32)
    c = np.array([1, 2, 0, 2])
    m, removed = prune(m0, s, c, k, 0.1)
    assert removed.tolist() == [True, False, False, False]
    assert np.isneginf(m[:2]).all() and np.all(m[2:] == 0)


def test_growing_statistics_definition():
    """Per pair: |(du, dv)| to its Gaussian, opacity to its anchor, counts;
    views add; invalid slots contribute nothing."""
    from oracle.grow import accumulate
    k, n_views, N = 2, 2, 4
    g2d = np.zeros((n_views * N, 10))
    g2d[0, :2] = (3.0, 4.0)
    g2d[1, :2] = (0.6, 0.8)
    g2d[N + 0, :2] = (5.0, 12.0)
    g2d[N + 3, :2] = (8.0, 6.0)
    valid = np.array([1, 1, 0, 0, 1, 0, 0, 1])
    opa = np.array([0.1, 0.2, 0.9, 0.9, 0.3, 0.9, 0.9, 0.4])
    gs, gc, os_, oc = accumulate(g2d, valid, opa, k, n_views)
    assert np.allclose(gs, [5.0 + 13.0, 1.0, 0.0, 10.0]) and gc.tolist() == [2, 1, 0, 1]
    assert np.allclose(os_, [0.1 + 0.2 + 0.3, 0.4]) and oc.tolist() == [3, 1]


# ---------------------------------------------------------------------------
# random-ray sampling and the loss over the sampled rays (the BA's rays)
# ---------------------------------------------------------------------------

def test_ray_sampler_follows_splitmix64_and_rates():
    from oracle.grow import GAMMA, MASK64, splitmix64
    from oracle.rays import sample_rays, splitmix64_array
    rng = np.random.default_rng(4)
    st = rng.integers(0, 2 ** 63, size=200, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    assert [int(x) for x in splitmix64_array(st)] == [splitmix64(int(x)) for x in st]
    n = 100000
    assert sample_rays(n, 0.0, 3, 0).sum() == 0 and sample_rays(n, 1.0, 3, 0).sum() == n
    a, b = sample_rays(n, 0.1, 3, 0), sample_rays(n, 0.3, 3, 0)
    assert np.all(a <= b)                       # nested as the rate grows
    for m, p in ((a, 0.1), (b, 0.3)):
        assert abs(m.sum() - n * p) < 5 * np.sqrt(n * p * (1 - p))
    assert not np.array_equal(a, sample_rays(n, 0.1, 3, 1))   # a new round draws new rays
    # pixel 5 at round 2 by the rule itself
    key = (3 + 2 * GAMMA) & MASK64
    assert sample_rays(8, 0.5, 3, 2)[5] == int((splitmix64(key ^ 5) >> 11) < 2 ** 52)


def test_masked_loss_hand_case_and_full_mask_reduces_to_the_loss():
    from oracle.rays import loss_l1_masked
    # two views of two pixels; pixel (0, 1) and (1, 0) sampled
    C = np.array([[1.0, 2.0], [0.0, 0.0], [0.5, 0.5], [3.0, 1.0], [1.0, 1.0], [0.0, 2.0]])   # [v][c][p] flattened
    Ct = np.zeros_like(C)
    D = np.array([1.0, 5.0, 2.0, 2.0])
    Dt = np.array([0.5, 6.0, 0.0, 1.0])
    S = np.ones(4)
    mask = np.array([0, 1, 1, 0])
    L, dC, dD = loss_l1_masked(C.ravel(), D, S, Ct.ravel(), Dt, mask, 2, w_depth=0.5)
    # colour: sampled values |2|+|0|+|0.5| (view 0, pixel 1) and |3|+|1|+|0| (view 1, pixel 0) over 3*2
    # depth: only (0, 1) is valid (view 1 pixel 0 has Dt = 0): |5-6| * 0.5 / 1
    assert abs(L - ((2.0 + 0.0 + 0.5 + 3.0 + 1.0 + 0.0) / 6.0 + 0.5)) < 1e-15
    assert np.allclose(dD, [0.0, -0.5, 0.0, 0.0])
    assert np.allclose(dC.reshape(2, 3, 2)[0, :, 0], 0.0) and np.allclose(dC.reshape(2, 3, 2)[1, :, 1], 0.0)
    # every pixel sampled: the bench loss of one view (the C oracle's)
    rng = np.random.default_rng(6)
    P = 97
    Cf, Ctf = rng.uniform(size=3 * P), rng.uniform(size=3 * P)
    Df, Dtf = rng.uniform(1, 3, size=P), np.where(rng.uniform(size=P) < 0.8, rng.uniform(1, 3, size=P), 0.0)
    Sf = rng.uniform(size=P)
    L1, dC1, dD1 = loss_l1_masked(Cf, Df, Sf, Ctf, Dtf, np.ones(P), 1, w_depth=0.5, gate=0.3)
    L2, dC2, dD2 = O.loss_l1(Cf, Df, Sf, Ctf, Dtf, w_depth=0.5, gate=0.3)
    assert abs(L1 - L2) < 1e-12 and np.allclose(dC1, dC2, atol=1e-15) and np.allclose(dD1, dD2, atol=1e-15)


def test_oracle_pixel_mask_composites_only_the_sampled_rays():
    """With a pixel mask the oracle's images equal the full render on the
    sampled pixels and stay zero elsewhere; its backward equals the full
    backward with the upstream gradients of the other pixels zeroed."""
    from oracle.rays import sample_rays
    sc = synth.tiny_scene()
    cams = [synth.tiny_camera(), synth.tiny_camera()]
    o = O.Oracle(sc, cams)
    full = o.forward()
    P = o.n_pixels
    m = sample_rays(P, 0.3, 9, 0)
    om = O.Oracle(sc, cams)
    om.set_pixel_mask(m)
    part = om.forward()
    keep = m.astype(bool)
    assert np.array_equal(part["S"][keep], full["S"][keep]) and not part["S"][~keep].any()
    assert np.array_equal(part["D"][keep], full["D"][keep])
    rng = np.random.default_rng(2)
    dC, dD, dS = rng.normal(size=3 * P), rng.normal(size=P), rng.normal(size=P)
    mC = np.concatenate([np.tile(m[v * (P // 2):(v + 1) * (P // 2)], 3) for v in range(2)])
    gm = om.backward(dC, dD, dS)
    gf = o.backward(dC * mC, dD * m, dS * m)
    for k in ("anchor_xyz", "offsets", "logscale", "rot", "opacity", "rgb"):
        if k in gm and gm[k] is not None:
            assert np.allclose(gm[k], gf[k], rtol=1e-12, atol=1e-15), k
    assert np.allclose(gm["pose"], gf["pose"], rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------------------
# R-VQ coded offsets and scaling factors (the paper's R-VQ targets, Eq. 14)
# ---------------------------------------------------------------------------

def _coded_geometry_fd_scene(seed):
    sc = fd_scene(False, seed=seed)
    rng = np.random.default_rng(seed + 100)
    L, K = 2, 3
    ocb = rng.normal(0, 0.04, (L, K, 3)).astype(np.float32)
    lcb = rng.normal(0, 0.1, (L, K, 3)).astype(np.float32)
    lcb[0] += 1.0
    og = synth.Group(3, codebook=ocb, idx=rng.integers(0, K, (L, sc.n), dtype=np.uint8))
    lg = synth.Group(3, codebook=lcb, idx=rng.integers(0, K, (L, sc.n_anchors), dtype=np.uint8))
    import dataclasses
    return dataclasses.replace(sc, offsets=None, anchor_l=None, offsets_rvq=og, l_rvq=lg, k_coded=sc.k)


def test_coded_geometry_decodes_in_fp32_stage_order_and_renders_as_decoded():
    """A coded scene renders exactly like the raw scene holding the FP32
    stage-order sums of its codewords (numpy float32 adds)."""
    import dataclasses
    sc = _coded_geometry_fd_scene(50)
    og, lg = sc.offsets_rvq, sc.l_rvq
    off = np.zeros((sc.n, 3), np.float32)
    l = np.zeros((sc.n_anchors, 3), np.float32)
    for s in range(2):
        off = off + og.codebook[s][og.idx[s].astype(int)]
        l = l + lg.codebook[s][lg.idx[s].astype(int)]
    raw = dataclasses.replace(sc, offsets=off.reshape(sc.n_anchors, sc.k, 3), anchor_l=l, offsets_rvq=None,
                              l_rvq=None, k_coded=0)
    cams = fd_cams(1)
    a, b = O.Oracle(sc, cams).forward(), O.Oracle(raw, cams).forward()
    for key in ("C", "D", "S"):
        assert np.array_equal(a[key], b[key])


def test_fd_coded_offset_and_scale_codebooks():
    """Central differences of the objective in every codeword entry of the
    offset and scaling-factor codebooks (decoded in FP64 around the point)
    against the scattered analytic gradients."""
    sc = _coded_geometry_fd_scene(51)
    cams = fd_cams(1)
    o = O.Oracle(sc, cams)
    f = o.forward()
    assert f["S"].max() > 0.5 and not np.any(f["flags"])
    ups = [u.astype(np.float64) for u in synth.upstream_grads(99, o.n_pixels, scale=o.n_pixels)]
    grads = o.backward(*ups)
    for key, g, shape in (("offsets", sc.offsets_rvq, (sc.n_anchors, sc.k, 3)), ("anchor_l", sc.l_rvq,
                                                                                  (sc.n_anchors, 3))):
        cb = np.asarray(g.codebook, np.float64)
        ix = np.asarray(g.idx, np.int64)
        fd = np.zeros(cb.size)
        for j in range(cb.size):
            vals = []
            for sgn in (1.0, -1.0):
                c2 = cb.copy()
                c2.flat[j] += sgn * 1e-6
                dec = sum(c2[s][ix[s]] for s in range(cb.shape[0])).reshape(shape)
                vals.append(_objective(sc, cams, ups, {key: dec}))
            fd[j] = (vals[0] - vals[1]) / 2e-6
        an = grads[key].ravel()
        assert an.shape == fd.shape
        assert np.abs(fd - an).max() <= 2e-5 * max(1e-6, np.abs(fd).max()), (key, fd, an)
