"""FP64 reference of the warm-start network's layers (test infrastructure).

Only tests/ and the benchmark's baselines use this module; the product path
runs the CUDA kernels.  Each function is the plain definition of the
operation, written with numpy:

  conv3d   y[n, co, v] = b[co] + sum_ci sum_t w[co, ci, t] x[n, ci, v + dil * off(t)]
           (conv3d_cl: the same in the channels-last layout of the U-net)
           (zero outside the grid; off(t) = (t//9 - 1, (t//3)%3 - 1, t%3 - 1) in
           (z, y, x)), then max(0, .) when relu
  backward gx = dL/dx, gw = dL/dw, gb = dL/db for dL/dy = gy (ReLU mask from y)
  pool     mean over 2 x 2 x 2 blocks; upsample: nearest neighbour by 2; and
           their adjoints (the gradients)
  mse      L = sum_i m_i (p_i - t_i)^2 / msum,  dL/dp_i = 2 m_i (p_i - t_i) / msum
  adam     Kingma & Ba (2015), bias-corrected moments

Pins: tests/test_oracle_warm.py (identity and shift kernels, finite
differences of the loss through two layers, Adam's first step in closed
form).  bf16_round gives the bfloat16 value (round to nearest even) that the
GPU stores, so that both sides start from the same numbers.
"""
import numpy as np


def tap_offsets(dil):
    """(dz, dy, dx) of the 27 taps, times the dilation."""
    return [((t // 9 - 1) * dil, ((t // 3) % 3 - 1) * dil, (t % 3 - 1) * dil) for t in range(27)]


def _shifted(a, dz, dy, dx):
    """s[..., z, y, x] = a[..., z + dz, y + dy, x + dx], zero outside."""
    out = np.zeros_like(a)
    nz, ny, nx = a.shape[-3:]
    zs, ze = max(0, -dz), min(nz, nz - dz)
    ys, ye = max(0, -dy), min(ny, ny - dy)
    xs, xe = max(0, -dx), min(nx, nx - dx)
    if zs < ze and ys < ye and xs < xe:
        out[..., zs:ze, ys:ye, xs:xe] = a[..., zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv3d(x, w, b, dil, relu):
    """x [n][cin][nz][ny][nx], w [cout][cin][27], b [cout] -> y [n][cout][nz][ny][nx]."""
    x = np.asarray(x, np.float64)
    n, cin = x.shape[:2]
    cout = w.shape[0]
    y = np.zeros((n, cout) + x.shape[2:])
    y += np.asarray(b, np.float64)[None, :, None, None, None]
    for t, (dz, dy, dx) in enumerate(tap_offsets(dil)):
        xs = _shifted(x, dz, dy, dx)  # [n][cin][...]
        y += np.einsum("oc,nczyx->nozyx", w[:, :, t], xs)
    return np.maximum(y, 0.0) if relu else y


def conv3d_backward(x, w, dil, y, relu, gy):
    """Gradients for dL/dy = gy: returns gx, gw, gb."""
    x = np.asarray(x, np.float64)
    g = np.asarray(gy, np.float64)
    if relu:
        g = g * (np.asarray(y) > 0)
    gw = np.zeros(w.shape)
    gx = np.zeros_like(x)
    for t, (dz, dy, dx) in enumerate(tap_offsets(dil)):
        xs = _shifted(x, dz, dy, dx)
        gw[:, :, t] = np.einsum("nozyx,nczyx->oc", g, xs)
        # y[v] gets w x[v + off]: x[u] receives from y[u - off]
        gx += np.einsum("oc,nozyx->nczyx", w[:, :, t], _shifted(g, -dz, -dy, -dx))
    gb = g.sum(axis=(0, 2, 3, 4))
    return gx, gw, gb


def conv3d_cl(x, w, b, relu):
    """Channels-last layer of the U-net: x [n][nz][ny][nx][cin], w [27][cout][cin]
    (tap-major), b [cout] -> y [n][nz][ny][nx][cout]; the same operation as
    conv3d (dilation 1) in another memory layout."""
    xc = np.moveaxis(np.asarray(x, np.float64), -1, 1)
    wc = np.transpose(np.asarray(w, np.float64), (1, 2, 0))
    return np.moveaxis(conv3d(xc, wc, b, 1, relu), 1, -1)


def conv3d_cl_backward(x, w, y, relu, gy):
    """Gradients (gx, gw [27][cout][cin], gb) of conv3d_cl for dL/dy = gy."""
    xc = np.moveaxis(np.asarray(x, np.float64), -1, 1)
    wc = np.transpose(np.asarray(w, np.float64), (1, 2, 0))
    yc = np.moveaxis(np.asarray(y, np.float64), -1, 1)
    gc = np.moveaxis(np.asarray(gy, np.float64), -1, 1)
    gx, gw, gb = conv3d_backward(xc, wc, 1, yc, relu, gc)
    return np.moveaxis(gx, 1, -1), np.transpose(gw, (2, 0, 1)), gb


def avg_pool2(x):
    """Mean over 2 x 2 x 2 blocks of a channels-last [n][nz][ny][nx][c] field."""
    x = np.asarray(x, np.float64)
    n, nz, ny, nx, c = x.shape
    return x.reshape(n, nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(2, 4, 6))


def avg_pool2_backward(gy):
    """Adjoint of avg_pool2: each fine voxel gets 1/8 of its block's gradient."""
    g = np.asarray(gy, np.float64)
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def upsample2(x):
    """Nearest-neighbour upsampling by 2 in z, y and x (channels-last)."""
    x = np.asarray(x, np.float64)
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def upsample2_backward(gy):
    """Adjoint of upsample2: each coarse voxel sums its eight fine ones."""
    g = np.asarray(gy, np.float64)
    n, nz, ny, nx, c = g.shape
    return g.reshape(n, nz // 2, 2, ny // 2, 2, nx // 2, 2, c).sum(axis=(2, 4, 6))


def mse(pred, target, mask=None):
    p = np.asarray(pred, np.float64)
    t = np.asarray(target, np.float64)
    m = np.ones_like(p) if mask is None else np.asarray(mask, np.float64)
    msum = m.sum()
    d = p - t
    return float((m * d * d).sum() / msum), 2.0 * m * d / msum


def adam(w, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; returns (w, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** t)
    vh = m2 / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m1, m2


def bf16_round(a):
    """Nearest bfloat16 value of each float32 (ties to even), as float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
