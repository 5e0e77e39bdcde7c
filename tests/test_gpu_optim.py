"""On-device optimiser steps: vg_adam_step against a plain PyTorch FP32
Adam on the CPU (aligned and unaligned arrays, sizes off multiples of four,
several steps with a device step counter), and vg_pose_step against the
SE(3) matrix exponential from scipy applied to the Adam direction."""
import numpy as np
import pytest

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


def adam_ref(p, g, m, v, lr, b1, b2, eps, step):
    """Adam with the coefficients as the FP32 arguments they are passed as
    (1 - beta computed from the FP32 beta)."""
    f = np.float32
    b1, b2 = f(b1), f(b2)
    m = float(b1) * m + float(f(1) - b1) * g
    v = float(b2) * v + float(f(1) - b2) * g * g
    bc1, bc2 = 1 - float(b1) ** step, 1 - float(b2) ** step
    p = p - (lr / bc1) * m / (v.sqrt() * (1 / np.sqrt(bc2)) + eps)
    return p, m, v


def test_adam_matches_plain_torch(torch):
    rng = np.random.default_rng(0)
    sizes = [1, 3, 4, 1001, 40000 * 3, 7]
    base = [torch.from_numpy(rng.normal(size=n + 1).astype(np.float32)) for n in sizes]
    # the last tensor is a view at an odd offset: not 16-byte aligned
    host_p = [b[:n].clone() for b, n in zip(base, sizes)]
    dev_full = [b.cuda() for b in base]
    dev_p = [d[:n] for d, n in zip(dev_full, sizes)]
    dev_p[-1] = dev_full[-1][1:]
    host_p[-1] = base[-1][1:].clone()
    ms = [torch.zeros_like(p) for p in dev_p]
    vs = [torch.zeros_like(p) for p in dev_p]
    hm = [torch.zeros_like(p) for p in host_p]
    hv = [torch.zeros_like(p) for p in host_p]
    step = torch.ones(1, dtype=torch.int32, device="cuda")
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-15
    for it in range(1, 4):
        gs = [torch.from_numpy(rng.normal(size=p.numel()).astype(np.float32)) for p in host_p]
        V.vg_adam_step(dev_p, [g.cuda() for g in gs], ms, vs, lr, b1, b2, eps, step_dev=step)
        for i in range(len(sizes)):
            host_p[i], hm[i], hv[i] = adam_ref(host_p[i], gs[i], hm[i], hv[i], lr, b1, b2, eps, it)
    torch.cuda.synchronize()
    assert int(step.item()) == 4
    for i in range(len(sizes)):
        assert torch.allclose(dev_p[i].cpu(), host_p[i], rtol=1e-5, atol=1e-6), i
        assert torch.allclose(ms[i].cpu(), hm[i], rtol=1e-5, atol=1e-7), i
        assert torch.allclose(vs[i].cpu(), hv[i], rtol=1e-5, atol=1e-9), i
    # the element in front of the unaligned view is untouched
    assert dev_full[-1][0].item() == base[-1][0].item()


def hat(xi):
    rho, phi = xi[:3], xi[3:]
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    X = np.zeros((4, 4))
    X[:3, :3], X[:3, 3] = K, rho
    return X


@pytest.mark.parametrize("scale", [1e-6, 1e-2, 0.3])
def test_pose_step_is_adam_then_the_se3_exponential(torch, scale):
    from scipy.linalg import expm
    rng = np.random.default_rng(1)
    B = 5
    T = np.zeros((B, 3, 4))
    for b in range(B):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        T[b, :, :3] = q * np.sign(np.linalg.det(q))
        T[b, :, 3] = rng.normal(size=3)
    pose = torch.tensor(T.reshape(B, 12), dtype=torch.float32, device="cuda")
    g = rng.normal(size=(B, 6)) * scale
    m = torch.zeros((B, 6), device="cuda")
    v = torch.zeros((B, 6), device="cuda")
    lr_rot, lr_trans = 0.05, 0.2
    V.vg_pose_step(pose, torch.tensor(g, dtype=torch.float32, device="cuda"), m, v, lr_rot, lr_trans, step_host=1)
    torch.cuda.synchronize()
    out = pose.cpu().numpy().reshape(B, 3, 4)
    gf = g.astype(np.float32).astype(np.float64)
    mm = 0.1 * gf
    vv = 0.001 * gf * gf
    lr = np.array([lr_trans] * 3 + [lr_rot] * 3)
    d = -lr * (mm / 0.1) / (np.sqrt(vv / 0.001) + 1e-15)
    for b in range(B):
        Tb = np.vstack([T[b], [0, 0, 0, 1]])
        ref = (expm(hat(d[b])) @ Tb)[:3]
        assert np.allclose(out[b], ref, atol=3e-6), (b, np.abs(out[b] - ref).max())
        assert np.allclose(m.cpu().numpy()[b], mm[b], rtol=1e-5, atol=1e-12)
