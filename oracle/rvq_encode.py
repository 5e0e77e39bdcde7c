"""Oracle of residual-vector-quantisation encoding (Eq. 14, second line) and
of the codebook loss (Eq. 15).  TEST INFRASTRUCTURE ONLY (tests, the smoke
check and the benchmark's CPU legs); plain numpy, no CUDA.

Encoding takes integer decisions (an argmin per stage) from floating point,
so it takes them in FP32 with every rounding spelled out, as the GPU kernel
does: the running reconstruction l_hat is summed in stage order in FP32, the
residual is x - l_hat in FP32, and a codeword's squared distance is the sum
over components, in component order, of the FP32-rounded squares of the
FP32 differences (no fused multiply-add).  Ties go to the lowest index.
The loss and its codebook gradient, given the indices, are FP64.
"""
from __future__ import annotations

import numpy as np


def rvq_encode(codebook: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Eq. 14, second line: for stage s = 1..L, i^s = argmin_k
    || C^s[k] - (x - l_hat^{s-1}) ||^2 with l_hat^{s-1} = sum_{t<s} C^t[i^t].
    codebook [L][K][d], x [n][d] -> idx [L][n] uint8."""
    cb = np.ascontiguousarray(codebook, np.float32)
    xs = np.ascontiguousarray(x, np.float32)
    L, K, d = cb.shape
    n = xs.shape[0]
    idx = np.zeros((L, n), np.uint8)
    lhat = np.zeros((n, d), np.float32)
    for s in range(L):
        r = (xs - lhat).astype(np.float32)                       # [n][d]
        dist = np.zeros((n, K), np.float32)
        for c in range(d):
            diff = (cb[s][None, :, c] - r[:, None, c]).astype(np.float32)
            dist = (dist + (diff * diff).astype(np.float32)).astype(np.float32)
        k = np.argmin(dist, axis=1)                              # first minimum: lowest index
        idx[s] = k.astype(np.uint8)
        lhat = (lhat + cb[s][k]).astype(np.float32)
    return idx


def rvq_loss(codebook: np.ndarray, x: np.ndarray, idx: np.ndarray):
    """Eq. 15: L = 1/(n P) sum_s sum_n || sg[x_n - l_hat_n^{s-1}] - C^s[i_n^s] ||^2
    (P = codewords per stage) and dL/dC^s[k] = 2/(n P) sum_{n: i_n^s = k}
    (C^s[k] - (x_n - l_hat_n^{s-1})); FP64.  Returns (loss, dcodebook)."""
    cb = np.asarray(codebook, np.float64)
    xs = np.asarray(x, np.float64)
    L, K, d = cb.shape
    n = xs.shape[0]
    loss = 0.0
    grad = np.zeros_like(cb)
    lhat = np.zeros((n, d))
    if n == 0:
        return 0.0, grad
    for s in range(L):
        k = idx[s].astype(np.int64)
        r = xs - lhat
        e = cb[s][k] - r
        loss += float((e * e).sum())
        np.add.at(grad[s], k, 2.0 * e)
        lhat = lhat + cb[s][k]
    return loss / (n * K), grad / (n * K)
