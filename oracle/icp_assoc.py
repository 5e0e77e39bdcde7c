"""Oracle of the projective data association behind the ICP term (Eq. 20):
each Gaussian mean's "closest point" q is the target depth map's point on the
ray of the pixel the mean projects to.  TEST INFRASTRUCTURE ONLY; numpy FP64
(decoded means from the C oracle).

For view v and kept Gaussian n with p = T_cw mu in front of the near plane:
pixel (px, py) = nearest integers to (fx x/z + cx, fy y/z + cy); inside the
image, with target depth d > 0 there and |z - d| < max_dist:
q = ((px - cx) d / fx, (py - cy) d / fy, d), w = 1; otherwise q = 0, w = 0.
"""
from __future__ import annotations

import numpy as np


def associate(mu, kept, cams, Dt, max_dist):
    """mu [N][3] world means (FP64), kept [N] bool, Dt flat [views][H][W];
    returns q [views][N][3], w [views][N]."""
    N = mu.shape[0]
    V = len(cams)
    q = np.zeros((V, N, 3))
    w = np.zeros((V, N))
    pb = 0
    for v, c in enumerate(cams):
        T = np.asarray(c.T_cw, np.float64).reshape(3, 4)
        p = mu @ T[:, :3].T + T[:, 3]
        z = p[:, 2]
        front = kept & (z > c.near)
        zs = np.where(front, z, 1.0)
        u = c.fx * p[:, 0] / zs + c.cx
        vv = c.fy * p[:, 1] / zs + c.cy
        px = np.rint(u).astype(np.int64)     # round half to even, as the kernel's conversion
        py = np.rint(vv).astype(np.int64)
        inside = front & (px >= 0) & (px < c.width) & (py >= 0) & (py < c.height)
        d = np.zeros(N)
        idx = np.where(inside, py * c.width + px, 0)
        d[inside] = np.asarray(Dt, np.float64)[pb + idx[inside]]
        ok = inside & (d > 0) & (np.abs(z - d) < max_dist)
        q[v, ok, 0] = (px[ok] - c.cx) * d[ok] / c.fx
        q[v, ok, 1] = (py[ok] - c.cy) * d[ok] / c.fy
        q[v, ok, 2] = d[ok]
        w[v, ok] = 1.0
        pb += c.width * c.height
    return q, w
