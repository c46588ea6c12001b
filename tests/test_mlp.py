"""The learned proposal's network.

CPU: the reference's gradient formulas against central finite differences
(rounding switched off), its bf16 rounding against hand-made float32 cases,
and the exact regime: on dyadic inputs that the reference certifies exact
in float32, a float32 evaluation in any accumulation order equals the
reference bit for bit, while Gaussian inputs are not certified.
GPU: the library's BF16 tensor-core kernels against the reference, element
by element and bit for bit in the exact regime (forward output, loss and
every gradient tensor, on a ragged row count), plus a norm check on
Gaussian inputs, and that training reduces the loss.
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


def exact_regime_inputs(seed, rows=300):
    """Parameters, inputs and targets on small dyadic grids: weights are
    integers / 8 (sparse below the first layer so that sums stay small),
    biases integers / 2^5, 2^8, 2^11, 2^14 (the grids of the layers' sums),
    inputs integers / 4, and targets t = y - rows * q * 2^-14 with q in
    {-1, 0, 1}, so that (y - t) / rows = q * 2^-14 exactly.  y comes from
    the reference's forward pass."""
    rng = np.random.default_rng(seed)
    H = R.H

    def ints(shape, m, dens=1.0):
        v = rng.integers(-m, m + 1, size=shape).astype(np.float64)
        return v * (rng.random(shape) < dens)

    parts = [ints((N_IN, H), 3, 0.5) / 8, ints(H, 4) / 32, ints((H, H), 3, 0.125) / 8, ints(H, 4) / 256,
             ints((H, H), 3, 0.125) / 8, ints(H, 4) / 2048, ints(H, 3) / 8, ints(1, 4) / 16384]
    p = np.concatenate([np.ravel(a) for a in parts]).astype(np.float32)
    x = (ints((rows, N_IN), 3) / 4).astype(np.float32)
    y, _ = R.forward(p, x.astype(np.float64))
    t = (y - rows * rng.integers(-1, 2, size=rows) * 2.0 ** -14).astype(np.float32)
    return p, x, t


def float32_gradients(p, x, t, reverse):
    """The reference's computation in numpy float32 (BLAS accumulation, or
    every sum's terms in reverse order), same rounding points."""
    f = np.float32
    n_in = x.shape[1]
    W1, b1, W2, b2, W3, b3, w4, b4 = [a.astype(f) for a in R.unpack(p, n_in)]
    bf = lambda a: R.bf16(a).astype(f)

    def mm(a, b):
        if not reverse:
            return (a @ b).astype(f)
        out = np.zeros((a.shape[0], b.shape[1]), dtype=f)
        for k in reversed(range(a.shape[1])):
            out = (out + np.outer(a[:, k], b[k, :]).astype(f)).astype(f)
        return out

    Ws, bs = [bf(W1), bf(W2), bf(W3)], [b1, b2, b3]
    hs = [bf(x)]
    for l in range(3):
        hs.append(bf(np.maximum((mm(hs[-1], Ws[l]) + bs[l]).astype(f), f(0))))
    y = (mm(hs[3], w4[:, None])[:, 0] + b4[0]).astype(f)
    rows = x.shape[0]
    d = (y - t.astype(f)).astype(f)
    dy = (d / f(rows)).astype(f)
    dw4 = mm(hs[3].T, dy[:, None])[:, 0]
    db4 = mm(np.ones((1, rows), dtype=f), dy[:, None])[0]
    dz = ((dy[:, None] * w4[None, :]).astype(f) * (hs[3] > 0)).astype(f)
    g = {}
    for l in (3, 2, 1):
        dzb = bf(dz)
        g[f"b{l}"] = mm(np.ones((1, rows), dtype=f), dz)[0]
        g[f"W{l}"] = mm(hs[l - 1].T, dzb)
        if l == 1:
            break
        dz = (mm(dzb, Ws[l - 1].T) * (hs[l - 1] > 0)).astype(f)
    flat = np.concatenate([g["W1"].ravel(), g["b1"], g["W2"].ravel(), g["b2"], g["W3"].ravel(), g["b3"], dw4, db4])
    return y, flat


def test_exact_regime_any_order_equals_reference():
    """In the certified regime float32 in two accumulation orders equals the
    float64 reference bit for bit, bf16 roundings included; the
    certificate is not vacuous (Gaussian inputs fail it, and a bf16 rounding
    actually rounds some values of the third layer)."""
    p, x, t = exact_regime_inputs(11, rows=64)
    x64, t64 = x.astype(np.float64), t.astype(np.float64)
    assert R.exact_regime(p, x64, t64) == []
    y_ref, hs = R.forward(p, x64)
    g_ref, _ = R.gradients(p, x64, t64)
    for reverse in (False, True):
        y, g = float32_gradients(p, x, t, reverse)
        assert np.array_equal(y.astype(np.float64), y_ref)
        assert np.array_equal(g.astype(np.float64), g_ref)
    W1, b1, W2, b2, W3, b3, w4, b4 = R.unpack(p, N_IN)
    v3 = np.maximum(hs[2] @ R.bf16(W3) + b3, 0.0)
    assert np.mean(R.bf16(v3) != v3) > 0.05
    rng = np.random.default_rng(1)
    pg = rand_params(N_IN, 2)
    assert R.exact_regime(pg, rng.normal(size=(64, N_IN)).astype(np.float32).astype(np.float64),
                          rng.normal(size=64).astype(np.float32).astype(np.float64)) != []


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


GRAD_SIZES = [("W1", N_IN * R.H), ("b1", R.H), ("W2", R.H * R.H), ("b2", R.H), ("W3", R.H * R.H), ("b3", R.H),
              ("w4", R.H), ("b4", 1)]


@pytest.mark.gpu
@pytest.mark.parametrize("seed,rows", [(7, 300), (8, 1000)])
def test_gpu_exact_regime_bit_exact(seed, rows):
    """Element by element, bit for bit: in the certified exact regime the
    device's forward output, loss and every gradient tensor equal the
    reference's (row counts not a multiple of the 64-row tiles)."""
    import torch
    from paper_2202_13511_gb300 import mpdp
    p, x, t = exact_regime_inputs(seed, rows)
    x64, t64 = x.astype(np.float64), t.astype(np.float64)
    assert R.exact_regime(p, x64, t64) == []
    y_ref, _ = R.forward(p, x64)
    g_ref, loss_ref = R.gradients(p, x64, t64)
    m = mpdp.Mlp(N_IN)
    m.set_params(p)
    dx = torch.from_numpy(x).cuda()
    dt = torch.from_numpy(t).cuda()
    dy = torch.zeros(rows, dtype=torch.float32, device="cuda")
    m.forward(dx, rows, dy)
    torch.cuda.synchronize()
    y = dy.cpu().numpy().astype(np.float64)
    bad = np.flatnonzero(y != y_ref)
    assert bad.size == 0, ("y", bad[:5], y[bad[:5]], y_ref[bad[:5]])
    g, loss = m.gradients(dx, dt, rows)
    assert loss == loss_ref
    o = 0
    for name, size in GRAD_SIZES:
        a, b = g[o:o + size].astype(np.float64), g_ref[o:o + size]
        bad = np.flatnonzero(a != b)
        assert bad.size == 0, (name, bad.size, bad[:5], a[bad[:5]], b[bad[:5]])
        o += size
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
