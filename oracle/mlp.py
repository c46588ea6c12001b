"""CPU reference of the learned proposal's network, for gradient checks.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy in
float64 with the BF16 rounding points of the GPU kernels made explicit, so
that a wrong layout, transposition or dropped term in the kernels shows as a
difference far above the rounding noise:
  xb = bf16(x); h_l = bf16(relu(h_{l-1} W_l + b_l)) for l = 1..3;
  y = h_3 . w4 + b4;  L = sum (y - t)^2 / (2 rows);
  dz_3 = (dy w4^T) masked by h_3 > 0; dW_l = h_{l-1}^T bf16(dz_l);
  db_l = column sums of dz_l; dh_{l-1} = bf16(dz_l) W_l^T; dz_{l-1} = dh_{l-1}
  masked by h_{l-1} > 0; dw4 = h_3^T dy; db4 = sum dy, with dy = (y - t) / rows.
The weights used in products are bf16(W_l) (the GPU's copies of its f32
masters).  bf16 rounding is round to nearest even on the float32 value.
"""
from __future__ import annotations

import numpy as np

H = 256


EXACT = False  # tests of the formulas themselves switch the rounding off


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest even) through float32, returned as float64."""
    if EXACT:
        return np.asarray(x, dtype=np.float64)
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p: np.ndarray, n_in: int):
    sizes = [n_in * H, H, H * H, H, H * H, H, H, 1]
    out, o = [], 0
    for s in sizes:
        out.append(np.asarray(p[o:o + s], dtype=np.float64))
        o += s
    W1, b1, W2, b2, W3, b3, w4, b4 = out
    return [W1.reshape(n_in, H), b1, W2.reshape(H, H), b2, W3.reshape(H, H), b3, w4, b4]


def forward(p, x):
    n_in = x.shape[1]
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p, n_in)
    h0 = bf16(x)
    h1 = bf16(np.maximum(h0 @ bf16(W1) + b1, 0.0))
    h2 = bf16(np.maximum(h1 @ bf16(W2) + b2, 0.0))
    h3 = bf16(np.maximum(h2 @ bf16(W3) + b3, 0.0))
    y = h3 @ w4 + b4[0]
    return y, (h0, h1, h2, h3)


def gradients(p, x, t):
    """(flat gradient in the parameter layout, loss)."""
    n_in = x.shape[1]
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p, n_in)
    y, (h0, h1, h2, h3) = forward(p, x)
    rows = x.shape[0]
    d = y - t
    loss = float(np.sum(d * d) / (2 * rows))
    dy = d / rows
    dw4 = h3.T @ dy
    db4 = np.array([dy.sum()])
    dz3 = np.outer(dy, w4) * (h3 > 0)
    Ws = [bf16(W1), bf16(W2), bf16(W3)]
    hs = [h0, h1, h2, h3]
    grads = {}
    dz = dz3
    for l in (3, 2, 1):
        dzb = bf16(dz)
        grads[f"b{l}"] = dz.sum(axis=0)
        grads[f"W{l}"] = hs[l - 1].T @ dzb
        if l == 1:
            break
        dh = dzb @ Ws[l - 1].T
        dz = dh * (hs[l - 1] > 0)
    flat = np.concatenate([grads["W1"].ravel(), grads["b1"], grads["W2"].ravel(), grads["b2"],
                           grads["W3"].ravel(), grads["b3"], dw4, db4])
    return flat, loss


# ---------------------------------------------------------------------------
# Exact regime.  When every operand lies on a dyadic grid and every sum is
# small enough on that grid, float32 holds every partial sum of every
# accumulation exactly, in any order and with any alignment of several
# products, and every single float32 operation (bias add, y - t, division by
# the row count, products) is exact as well.  The bf16 rounding points then
# round the same exact values on the device and here.  So a device that
# follows the rounding points above must reproduce forward() and
# gradients() bit for bit, whatever its accumulation order.


def _grid(a) -> int:
    """Smallest g >= 0 with a * 2^g integral everywhere (-1: none up to 2^-200)."""
    a = np.asarray(a, dtype=np.float64)
    for g in range(0, 200):
        s = a * (2.0 ** g)
        if np.all(s == np.floor(s)):
            return g
    return -1


def _sum_exact(a, b) -> bool:
    """Every partial sum of every dot product of a @ b is a float32: the
    products are multiples of 2^-(ga+gb) and their absolute sum stays below
    2^24 such units."""
    ga, gb = _grid(a), _grid(b)
    if ga < 0 or gb < 0:
        return False
    return float(np.max(np.abs(a) @ np.abs(b), initial=0.0)) < 2.0 ** (24 - ga - gb)


def _fits32(v) -> bool:
    v = np.asarray(v, dtype=np.float64)
    return bool(np.all(v.astype(np.float32).astype(np.float64) == v))


def exact_regime(p, x, t) -> list:
    """Steps of forward() and gradients() whose float32 evaluation could
    round (empty: the whole computation is exact in float32)."""
    n_in = x.shape[1]
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p, n_in)
    rows = x.shape[0]
    bad = []
    chk = lambda ok, what: None if ok else bad.append(what)
    chk(_fits32(x) and _fits32(t) and _fits32(p), "inputs are not float32")
    Ws = [bf16(W1), bf16(W2), bf16(W3)]
    chk(all(np.array_equal(Wb, W) for Wb, W in zip(Ws, (W1, W2, W3))), "weights are not bf16")
    bs = [b1, b2, b3]
    hs = [bf16(x)]
    for l in range(3):
        chk(_sum_exact(hs[-1], Ws[l]), f"z{l + 1} accumulation")
        v = hs[-1] @ Ws[l] + bs[l]
        chk(_fits32(v), f"z{l + 1} + b{l + 1}")
        hs.append(bf16(np.maximum(v, 0.0)))
    h3 = hs[3]
    chk(_sum_exact(h3, w4[:, None]) and _fits32(h3 * w4[None, :]), "head sum")
    y = h3 @ w4 + b4[0]
    chk(_fits32(y), "y + b4")
    d = y - t
    chk(_fits32(d) and _fits32(d / rows) and _fits32(d * d), "y - t, (y - t) / rows, (y - t)^2")
    dy = d / rows
    chk(_sum_exact(h3.T, dy[:, None]) and _fits32(dy[:, None] * h3), "dw4")
    chk(_sum_exact(np.ones((1, rows)), dy[:, None]), "db4")
    dz = np.outer(dy, w4) * (h3 > 0)
    chk(_fits32(dz), "dz3")
    for l in (3, 2, 1):
        dzb = bf16(dz)
        chk(_sum_exact(np.ones((1, rows)), dz), f"db{l}")
        chk(_sum_exact(hs[l - 1].T, dzb), f"dW{l}")
        if l == 1:
            break
        chk(_sum_exact(dzb, Ws[l - 1].T), f"dh{l - 1}")
        dz = (dzb @ Ws[l - 1].T) * (hs[l - 1] > 0)
    return bad
