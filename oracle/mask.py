"""Oracle of the sliding-window online mask (Sec. "Sliding Window-based
Online Mask", Eq. 13 and the removal at the window bound).  TEST
INFRASTRUCTURE ONLY; plain numpy.

Readings where the text is not explicit:
- The mask loss L_m = (1/N_w) sum_n Sig(m_n) runs over the Gaussians of the
  current viewing frustum (frustum selection: those visible in the frame's
  forward, N_w of them); its gradient w/N_w Sig'(m_n) reaches only them.
- At the window bound a Gaussian is removed when its mask is off
  (Sig(m) <= eps) or when it was visible within the window but hit fewer
  than min_hits rays ("hit frequency in conjunction with the learned mask");
  a removed Gaussian gets the mask logit -inf, i.e. it is never kept again.
"""
from __future__ import annotations

import numpy as np


def sigmoid(m):
    return 1.0 / (1.0 + np.exp(-np.asarray(m, np.float64)))


def mask_loss(mask_logit, visible, weight=1.0):
    """Returns (L_m, dL_m/dm) over the visible Gaussians (FP64)."""
    m = np.asarray(mask_logit, np.float64)
    vis = np.asarray(visible).astype(bool)
    nw = int(vis.sum())
    g = np.zeros_like(m)
    if nw == 0:
        return 0.0, g
    s = sigmoid(m[vis])
    g[vis] = weight * s * (1.0 - s) / nw
    return float(weight * s.sum() / nw), g


def mask_prune(mask_logit, hits, seen, eps, min_hits):
    """Removal at the window bound: returns (new mask logits, removed flags)."""
    m = np.asarray(mask_logit, np.float64).copy()
    off = sigmoid(m) <= eps
    rare = (np.asarray(seen) != 0) & (np.asarray(hits) < min_hits)
    removed = off | rare
    m[removed] = -np.inf
    return m, removed
