"""Oracle of random-ray sampling for the bundle adjustment and of the L1
loss over the sampled rays (Sec. "Tracking and Local-to-Global Bundle
Adjustment": the BA samples rays from the keyframe database).  TEST
INFRASTRUCTURE ONLY; plain numpy.

Readings where the text is not explicit:
- A ray is one pixel of one keyframe.  Each pixel is kept independently with
  probability `rate`, drawn from SplitMix64 (Steele, Lea and Flood, OOPSLA
  2014) as a counter-based generator: pixel p of the flattened keyframes
  (views in order, each row-major) is kept at round r iff
  SplitMix64((seed + r * 0x9E3779B97F4A7C15) ^ p) >> 11 < floor(rate * 2^53).
- The loss over the sampled rays is the bench loss restricted to them: the
  colour mean runs over the sampled pixels, the depth mean over the sampled
  pixels with a valid target (Dt > 0); the silhouette gate (S > gate), when
  on, zeroes terms without changing the normalisers.
"""
from __future__ import annotations

import numpy as np

from oracle.grow import GAMMA, MASK64


def splitmix64_array(states: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for an array of uint64 states (wrapping arithmetic)."""
    z = np.asarray(states, dtype=np.uint64) + np.uint64(GAMMA)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def sample_rays(n: int, rate: float, seed: int, round_: int) -> np.ndarray:
    """uint8 [n]: 1 where pixel p is a sampled ray at this round."""
    key = np.uint64((int(seed) + int(round_) * GAMMA) & MASK64)
    r = splitmix64_array(np.arange(n, dtype=np.uint64) ^ key) >> np.uint64(11)
    return (r < np.uint64(int(float(rate) * 2.0 ** 53))).astype(np.uint8)


def loss_l1_masked(C, D, S, Ct, Dt, mask, n_views, w_depth=0.5, gate=-1.0):
    """L1 colour + w_depth * L1 depth over the sampled pixels of n_views
    views (C, Ct: [n_views][3][P]; D, Dt, S, mask: [n_views][P]).  Returns
    (loss, dC, dD) in FP64."""
    C = np.asarray(C, np.float64).reshape(n_views, 3, -1)
    Ct = np.asarray(Ct, np.float64).reshape(n_views, 3, -1)
    D = np.asarray(D, np.float64).reshape(n_views, -1)
    Dt = np.asarray(Dt, np.float64).reshape(n_views, -1)
    S = np.asarray(S, np.float64).reshape(n_views, -1)
    m = np.asarray(mask).reshape(n_views, -1) != 0
    n_s = int(m.sum())
    valid = m & (Dt > 0)
    n_v = int(valid.sum())
    g = np.ones_like(D) if gate < 0 else (S > gate).astype(np.float64)
    inv_c = 1.0 / (3.0 * n_s) if n_s else 0.0
    inv_d = w_depth / n_v if n_v else 0.0
    rc = C - Ct
    rd = D - Dt
    dC = np.sign(rc) * (m * g)[:, None, :] * inv_c
    dD = np.sign(rd) * (valid * g) * inv_d
    L = float((np.abs(rc) * (m * g)[:, None, :]).sum() * inv_c + (np.abs(rd) * valid * g).sum() * inv_d)
    return L, dC.reshape(-1), dD.reshape(-1)
