"""Oracle of sequential anchor growing and opacity-based anchor removal
(Sec. "Sequential Anchor Point Growing", Eq. 10).  TEST INFRASTRUCTURE ONLY;
plain numpy.

What the method computes, step by step:
1. Statistics, every iteration, over the (view, Gaussian) pairs that survive
   culling in that iteration's render: each Gaussian accumulates the norm of
   the gradient of the loss with respect to its projected 2D mean and a count
   of those pairs; each anchor accumulates the opacities of its visible
   Gaussians and a count of them.
2. Growing, after N iterations, on voxel grids of M levels (the paper: 3):
   level m has voxel size eps_m = eps_g / 4^(m-1) and threshold
   tau_m = tau_g * 2^(m-1) (Eq. 10).  A Gaussian seen in the interval falls in
   the voxel floor(mu / eps_m); the voxel's averaged gradient is the mean,
   over its seen Gaussians, of their per-Gaussian averages (sum / count).  A
   voxel whose average exceeds tau_m and that holds no anchor yet is a
   candidate; candidates go through a random elimination; each survivor gets
   a new anchor at the voxel centre.  Levels run coarse to fine, and the
   anchors grown at a level count as established for the finer ones.
3. Removal: an anchor whose Gaussians' mean opacity over the interval is
   below tau_alpha ("trivial") is removed: the mask logits of its k
   Gaussians become -inf.

Readings where the text is not explicit (each a choice the kernels share):
- The per-Gaussian average is taken in FP32 (sum / count, both FP32) and
  enters the voxel mean as the integer rint(average * 2^32), clamped to
  +-2^52: the voxel sum is then exact and order-free, and "average > tau_m"
  is decided as sum > (tau_m * 2^32) * count in FP64.  A Gaussian whose
  average is not finite is left out.
- Positions mu = x_a + O l and voxel indices floor(mu / eps_m) are FP32 (the
  GPU's rounding), since they decide integers; centres are
  (index + 0.5) * eps_m in FP32.  Voxel indices outside [-2^20, 2^20) are
  skipped.
- Random elimination keeps a candidate voxel iff r >> 11 >= floor(p_drop *
  2^53), r the SplitMix64 output (Steele, Lea and Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014) for the state
  key XOR (seed + m * 0x9E3779B97F4A7C15) mod 2^64, key the packed voxel
  index ((ix + 2^20) << 42 | (iy + 2^20) << 21 | (iz + 2^20)).
- "Trivial" means: seen in the interval (count > 0) and opacity sum below
  tau_alpha * count (FP32 product, FP32 comparison).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
BIAS = 1 << 20


def splitmix64(state: int) -> int:
    """One output of SplitMix64 from `state` (the generator adds the golden
    gamma, then applies its finaliser)."""
    z = (state + GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def positions(anchor_xyz, anchor_l, offsets):
    """mu = x_a + O l per Gaussian, FP32 (product rounded, then the sum)."""
    xa = np.asarray(anchor_xyz, np.float32)
    l = np.asarray(anchor_l, np.float32)
    off = np.asarray(offsets, np.float32).reshape(len(xa), -1, 3)
    return (xa[:, None, :] + off * l[:, None, :]).reshape(-1, 3).astype(np.float32)


def accumulate(g2d, valid, opacity, k, n_views):
    """Step 1 for one iteration.  g2d [slots][>=2] (du, dv first), valid
    [slots] and opacity [slots] per (view, Gaussian) slot = view * N + n.
    Returns (grad_sum [N], grad_cnt [N], opa_sum [A], opa_cnt [A])."""
    g2d = np.asarray(g2d, np.float64)
    valid = np.asarray(valid).astype(bool)
    N = len(valid) // n_views
    norm = np.sqrt(g2d[:, 0] ** 2 + g2d[:, 1] ** 2)
    gs, gc = np.zeros(N), np.zeros(N, np.int64)
    A = N // k
    os_, oc = np.zeros(A), np.zeros(A, np.int64)
    for v in range(n_views):
        sl = slice(v * N, (v + 1) * N)
        ok = valid[sl]
        gs[ok] += norm[sl][ok]
        gc[ok] += 1
        n_ok = np.nonzero(ok)[0]
        np.add.at(os_, n_ok // k, np.asarray(opacity, np.float64)[sl][ok])
        np.add.at(oc, n_ok // k, 1)
    return gs, gc, os_, oc


def voxel_index(p, eps):
    """floor(p / eps) per component, FP32; rows outside the key range -> None mask."""
    q = np.floor(np.asarray(p, np.float32) / np.float32(eps)).astype(np.float64)
    ok = np.all(np.isfinite(q), axis=1) & np.all((q >= -BIAS) & (q < BIAS), axis=1)
    idx = np.zeros(q.shape, np.int64)
    idx[ok] = q[ok].astype(np.int64)
    return idx, ok


def pack(idx):
    i = np.asarray(idx, np.int64) + BIAS
    return (i[:, 0] << 42) | (i[:, 1] << 21) | i[:, 2]


def grow(mu, grad_sum, grad_cnt, anchors, eps_g, tau_g, levels=3, p_drop=0.0, seed=0):
    """Step 2.  mu [N][3] FP32 positions, grad_sum [N] (FP32 values),
    grad_cnt [N], anchors [A][3] existing anchor positions.  Returns a list
    of (level, key, centre[3] FP32) sorted by (level, key)."""
    mu = np.asarray(mu, np.float32)
    gs = np.asarray(grad_sum, np.float32)
    gc = np.asarray(grad_cnt, np.int64)
    seen = gc > 0
    avg = np.zeros(len(gs), np.float32)
    with np.errstate(invalid="ignore", over="ignore"):
        avg[seen] = gs[seen] / gc[seen].astype(np.float32)
    seen &= np.isfinite(avg)
    avg[~seen] = 0
    qv = np.clip(np.rint(avg.astype(np.float64) * 4294967296.0), -2.0 ** 52, 2.0 ** 52).astype(np.int64)
    established = np.asarray(anchors, np.float32).reshape(-1, 3)
    out = []
    threshold = int(float(p_drop) * 2.0 ** 53)
    for m in range(1, levels + 1):
        eps = np.float32(eps_g) / np.float32(4 ** (m - 1))
        tau = np.float32(tau_g) * np.float32(2 ** (m - 1))
        idx, ok = voxel_index(mu, eps)
        use = seen & ok
        keys = pack(idx[use])
        uk, inv = np.unique(keys, return_inverse=True)
        vsum = np.zeros(len(uk), np.int64)
        np.add.at(vsum, inv, qv[use])
        vcnt = np.bincount(inv, minlength=len(uk))
        aidx, aok = voxel_index(established, eps)
        occupied = set(pack(aidx[aok]).tolist())
        seed_m = (int(seed) + m * GAMMA) & MASK64
        grown = []
        for key, s, c in zip(uk.tolist(), vsum.tolist(), vcnt.tolist()):
            if key in occupied:
                continue
            if not float(s) > float(tau) * 4294967296.0 * float(c):
                continue
            if (splitmix64(key ^ seed_m) >> 11) < threshold:
                continue
            ix = ((key >> 42) & ((1 << 21) - 1)) - BIAS
            iy = ((key >> 21) & ((1 << 21) - 1)) - BIAS
            iz = (key & ((1 << 21) - 1)) - BIAS
            centre = ((np.array([ix, iy, iz], np.float64).astype(np.float32) + np.float32(0.5)) * eps).astype(np.float32)
            grown.append((m, key, centre))
        out.extend(grown)
        if grown:
            established = np.concatenate([established, np.stack([g[2] for g in grown])])
    return out


def prune(mask_logit, opa_sum, opa_cnt, k, tau_alpha):
    """Step 3.  Returns (new mask logits [N], removed [A] flags)."""
    m = np.asarray(mask_logit, np.float64).copy()
    s = np.asarray(opa_sum, np.float32)
    c = np.asarray(opa_cnt, np.int64)
    removed = (c > 0) & (s < np.float32(tau_alpha) * c.astype(np.float32))
    m.reshape(-1, k)[removed] = -np.inf
    return m, removed
