"""The learned proposal's network.

CPU: the reference's gradient formulas against central finite differences
(rounding switched off), and its bf16 rounding against exhaustive float32
cases.  GPU: the library's BF16 tensor-core kernels against the reference
(forward and every gradient tensor), and that training reduces the loss.
"""
import numpy as np
import pytest

import oracle.mlp as R

N_IN = 12


def rand_params(n_in, seed):
    rng = np.random.default_rng(seed)
    H = R.H
    parts = [rng.normal(0, np.sqrt(2.0 / n_in), (n_in, H)), rng.normal(0, 0.1, H),
             rng.normal(0, np.sqrt(2.0 / H), (H, H)), rng.normal(0, 0.1, H),
             rng.normal(0, np.sqrt(2.0 / H), (H, H)), rng.normal(0, 0.1, H),
             rng.normal(0, np.sqrt(1.0 / H), H), rng.normal(0, 0.1, 1)]
    return np.concatenate([np.ravel(x) for x in parts]).astype(np.float32)


def test_reference_gradients_match_finite_differences(monkeypatch):
    monkeypatch.setattr(R, "EXACT", True)
    rng = np.random.default_rng(1)
    p = rand_params(N_IN, 2).astype(np.float64)
    x = rng.normal(size=(7, N_IN))
    t = rng.normal(size=7)
    g, _ = R.gradients(p, x, t)
    idx = rng.choice(len(p), size=60, replace=False)
    idx = np.concatenate([idx, [len(p) - 1, len(p) - 2, 0, N_IN * R.H]])  # b4, w4, W1, b1
    for i in idx:
        e = np.zeros_like(p)
        h = 1e-6 * max(1.0, abs(p[i]))
        e[i] = h
        fd = (R.gradients(p + e, x, t)[1] - R.gradients(p - e, x, t)[1]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_bf16_rounding_nearest_even():
    # exactly representable, halfway (ties to even) and just above halfway
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)
    cases = [(1.0, 1.0), (1.0 + 2.0 ** -8, 1.0), (1.0 + 3 * 2.0 ** -8, 1.0 + 2 * 2.0 ** -7),
             (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7), (-2.5, -2.5), (0.0, 0.0)]
    for x, want in cases:
        assert R.bf16(np.float32(x)) == want, x
    assert one + ulp == np.float32(1.0 + 2.0 ** -7)


@pytest.mark.gpu
def test_gpu_forward_and_gradients_match_reference():
    import torch
    from paper_2202_13511_gb300 import mpdp
    rng = np.random.default_rng(3)
    rows = 300  # not a multiple of the 64-row tiles
    p = rand_params(N_IN, 4)
    x = rng.normal(size=(rows, N_IN)).astype(np.float32)
    t = rng.normal(size=rows).astype(np.float32)
    m = mpdp.Mlp(N_IN)
    m.set_params(p)
    dx = torch.from_numpy(x).cuda()
    dt = torch.from_numpy(t).cuda()
    dy = torch.zeros(rows, dtype=torch.float32, device="cuda")
    m.forward(dx, rows, dy)
    torch.cuda.synchronize()
    y_ref, _ = R.forward(p, x.astype(np.float64))
    y = dy.cpu().numpy()
    scale = np.abs(y_ref).max()
    assert np.max(np.abs(y - y_ref)) <= 2e-2 * scale
    g, loss = m.gradients(dx, dt, rows)
    g_ref, loss_ref = R.gradients(p, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref
    sizes = [N_IN * R.H, R.H, R.H * R.H, R.H, R.H * R.H, R.H, R.H, 1]
    o = 0
    for name, s in zip(["W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"], sizes):
        a, b = g[o:o + s].astype(np.float64), g_ref[o:o + s]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        assert rel < 3e-2 and cos > 0.999, (name, rel, cos)
        o += s
    m.close()


@pytest.mark.gpu
def test_gpu_training_reduces_loss():
    import torch
    from paper_2202_13511_gb300 import mpdp
    rng = np.random.default_rng(5)
    rows = 2048
    x = rng.uniform(-1, 1, size=(rows, N_IN)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2] - 0.5 * x[:, 3] ** 2).astype(np.float32)
    m = mpdp.Mlp(N_IN)
    m.init_params(seed=6)
    dx = torch.from_numpy(x).cuda()
    dt = torch.from_numpy(t).cuda()
    _, l0 = m.gradients(dx, dt, rows)
    for _ in range(300):
        m.train_step(dx, dt, rows, 1e-3)
    _, l1 = m.gradients(dx, dt, rows)
    assert l1 < l0 / 10, (l0, l1)
    m.close()
