"""Residual quantisation encode (Eq. 14, second line) and the codebook loss
(Eq. 15) on the GPU against the oracle: indices bit for bit (both sides take
the argmin in FP32 in the same order), loss and codebook gradient within
FP32 accumulation error; plus the learning use: Adam on the codebooks with
re-encoding lowers the loss."""
import numpy as np
import pytest

from oracle.rvq_encode import rvq_encode, rvq_loss
from paper_2403_11247_b300 import vg as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11247_b300 import build
    build.build()
    return t


def case(seed, L, K, d, n, dup=False):
    rng = np.random.default_rng(seed)
    scale = 0.5 ** np.arange(L)[:, None, None]
    cb = (rng.normal(size=(L, K, d)) * scale).astype(np.float32)
    if dup and K > 3:
        cb[:, 3] = cb[:, 1]
    x = rng.normal(size=(n, d)).astype(np.float32)
    return cb, x


@pytest.mark.parametrize("L,K,d,n", [(1, 64, 3, 1000), (3, 64, 3, 4097), (3, 256, 4, 3000), (6, 64, 3, 777),
                                     (2, 1, 1, 10), (4, 16, 16, 513)])
def test_encode_indices_bit_exact_and_loss(torch, L, K, d, n):
    cb, x = case(L * 100 + K + d, L, K, d, n, dup=True)
    t = lambda a: torch.from_numpy(a).cuda()
    idx, loss, dcb = V.vg_rvq_encode(t(cb), t(x))
    idx = idx.cpu().numpy()
    want = rvq_encode(cb, x)
    assert np.array_equal(idx, want), int((idx != want).sum())
    if K > 3:
        assert not np.any(idx == 3)          # the duplicate of codeword 1 never wins
    ol, og = rvq_loss(cb, x, want)
    assert abs(float(loss.item()) - ol) <= 1e-5 * ol + 1e-12, (float(loss.item()), ol)
    g = dcb.cpu().numpy()
    scale = max(np.abs(og).max(), 1e-12)
    assert np.abs(g - og).max() <= 1e-5 * scale, np.abs(g - og).max() / scale


def test_encode_empty_and_bad_arguments(torch):
    cb = torch.zeros((2, 8, 3), device="cuda")
    x = torch.zeros((0, 3), device="cuda")
    idx, loss, dcb = V.vg_rvq_encode(cb, x)
    assert float(loss.item()) == 0.0 and float(dcb.abs().sum()) == 0.0
    with pytest.raises(V.VgError):
        V.vg_rvq_encode(torch.zeros((2, 300, 3), device="cuda"), torch.zeros((4, 3), device="cuda"))


def test_codebook_learning_lowers_the_loss(torch):
    """Eq. 15 drives the codebooks: alternate encoding and Adam steps on the
    codebooks from their gradient."""
    rng = np.random.default_rng(5)
    centres = rng.normal(size=(16, 3)) * 2
    x = (centres[rng.integers(0, 16, 20000)] + rng.normal(scale=0.1, size=(20000, 3))).astype(np.float32)
    cb = torch.from_numpy((rng.normal(size=(2, 32, 3)) * np.array([1.0, 0.2])[:, None, None]).astype(np.float32)).cuda()
    xs = torch.from_numpy(x).cuda()
    m, v = torch.zeros_like(cb), torch.zeros_like(cb)
    losses = []
    for it in range(1, 101):
        _, loss, dcb = V.vg_rvq_encode(cb, xs)
        losses.append(float(loss.item()))
        V.vg_adam_step([cb], [dcb], [m], [v], 2e-2, step_host=it)
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])
