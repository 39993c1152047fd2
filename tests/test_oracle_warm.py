"""Pins of the warm-start network's FP64 reference (oracle/warm_net.py)
against what the definitions fix: identity and shift kernels, finite
differences through two layers, Adam's first step in closed form, the
bfloat16 rounding rule."""
import numpy as np
import pytest

from oracle import warm_net as W


def rnd(*shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


def test_identity_kernel_reproduces_input():
    x = rnd(2, 3, 5, 4, 6)
    w = np.zeros((3, 3, 27))
    for c in range(3):
        w[c, c, 13] = 1.0  # centre tap
    assert np.allclose(W.conv3d(x, w, np.zeros(3), 1, False), x)


@pytest.mark.parametrize("dil", [1, 2, 3])
def test_single_tap_shifts_by_the_dilation(dil):
    """Tap (dz, dy, dx) = (0, 0, +1) reads the neighbour dil voxels up in x."""
    x = rnd(1, 1, 3, 4, 9, seed=dil)
    w = np.zeros((1, 1, 27))
    w[0, 0, 14] = 2.0
    y = W.conv3d(x, w, np.array([0.5]), dil, False)
    ref = np.full_like(x, 0.5)
    ref[..., :-dil] += 2.0 * x[..., dil:]
    assert np.allclose(y, ref)


def test_relu_and_bias():
    x = rnd(1, 2, 3, 3, 3)
    w = rnd(2, 2, 27, seed=1)
    b = np.array([0.3, -0.2])
    y = W.conv3d(x, w, b, 1, True)
    assert (y >= 0).all()
    assert np.allclose(y, np.maximum(W.conv3d(x, w, b, 1, False), 0))


def two_layer_loss(x, w1, b1, w2, b2, t, mask):
    h = W.conv3d(x, w1, b1, 2, True)
    p = W.conv3d(h, w2, b2, 1, False)
    return W.mse(p, t, mask)[0]


def test_backward_matches_finite_differences():
    """Chain of two layers (ReLU, dilation 2, then linear) and the masked MSE:
    every gradient against central differences."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 2, 4, 3, 5))
    w1, b1 = 0.5 * rng.standard_normal((3, 2, 27)), 0.1 * rng.standard_normal(3)
    w2, b2 = 0.5 * rng.standard_normal((1, 3, 27)), 0.1 * rng.standard_normal(1)
    t = rng.standard_normal((2, 1, 4, 3, 5))
    mask = (rng.random((2, 1, 4, 3, 5)) > 0.3).astype(float)
    h = W.conv3d(x, w1, b1, 2, True)
    p = W.conv3d(h, w2, b2, 1, False)
    _, gp = W.mse(p, t, mask)
    gh, gw2, gb2 = W.conv3d_backward(h, w2, 1, p, False, gp)
    gx, gw1, gb1 = W.conv3d_backward(x, w1, 2, h, True, gh)
    eps = 1e-6

    def fd(arr, idx, f):
        a0 = arr[idx]
        arr[idx] = a0 + eps; lp = f()
        arr[idx] = a0 - eps; lm = f()
        arr[idx] = a0
        return (lp - lm) / (2 * eps)

    f = lambda: two_layer_loss(x, w1, b1, w2, b2, t, mask)
    for idx in [(0, 1, 0), (2, 0, 13), (1, 1, 26)]:
        assert fd(w1, idx, f) == pytest.approx(gw1[idx], rel=1e-5, abs=1e-9)
    for idx in [(0, 2, 5), (0, 0, 13)]:
        assert fd(w2, idx, f) == pytest.approx(gw2[idx], rel=1e-5, abs=1e-9)
    for i in range(3):
        assert fd(b1, (i,), f) == pytest.approx(gb1[i], rel=1e-5, abs=1e-9)
    assert fd(b2, (0,), f) == pytest.approx(gb2[0], rel=1e-5, abs=1e-9)
    for idx in [(0, 0, 1, 1, 2), (1, 1, 3, 2, 4), (0, 1, 0, 0, 0)]:
        assert fd(x, idx, f) == pytest.approx(gx[idx], rel=1e-5, abs=1e-9)


def test_mse_closed_form():
    loss, g = W.mse(np.array([1.0, 2.0, 4.0]), np.array([0.0, 2.0, 1.0]), np.array([1.0, 1.0, 0.0]))
    assert loss == pytest.approx(0.5)
    assert np.allclose(g, [1.0, 0.0, 0.0])


def test_adam_first_step_moves_by_lr():
    """After one step the bias-corrected ratio m/sqrt(v) is g/|g|: each weight
    moves by lr * sign(g) (up to eps)."""
    g = np.array([3.0, -0.01, 1e-3])
    w, m1, m2 = W.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=1e-12)
    assert np.allclose(w, -0.1 * np.sign(g))


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 1e-30], np.float32)
    r = W.bf16_round(vals)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even (1.0); 1 + 3*2^-8 rounds up
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -6
    assert r[3] == -2.5
    assert abs(r[4] - 1e-30) / 1e-30 < 2 ** -8


# ---------------------------------------------------- U-net layers (channels-last)
def test_pool_and_upsample_identities():
    """Pooling an upsampled field returns it exactly; upsampling a constant
    gives the constant; pooling a field linear in z gives the mean of each
    block's two planes."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal((2, 3, 4, 5, 6))
    assert np.allclose(W.avg_pool2(W.upsample2(x)), x, atol=1e-15)
    c = np.full((1, 2, 2, 2, 3), 2.5)
    assert np.array_equal(W.upsample2(c), np.full((1, 4, 4, 4, 3), 2.5))
    z = np.arange(8.0)[None, :, None, None, None] * np.ones((1, 8, 4, 4, 2))
    assert np.allclose(W.avg_pool2(z)[0, :, 0, 0, 0], [0.5, 2.5, 4.5, 6.5])


def test_pool_upsample_backward_are_adjoints():
    """<op(x), g> = <x, op_backward(g)> for both operators (pins the gradients
    to the forward definitions)."""
    rng = np.random.default_rng(8)
    x = rng.standard_normal((2, 4, 6, 8, 3))
    g = rng.standard_normal((2, 2, 3, 4, 3))
    assert np.isclose(np.sum(W.avg_pool2(x) * g), np.sum(x * W.avg_pool2_backward(g)), rtol=1e-13)
    xc = rng.standard_normal((2, 2, 3, 4, 3))
    gf = rng.standard_normal((2, 4, 6, 8, 3))
    assert np.isclose(np.sum(W.upsample2(xc) * gf), np.sum(xc * W.upsample2_backward(gf)), rtol=1e-13)


def test_channels_last_conv_matches_definition_by_finite_differences():
    """conv3d_cl_backward against central differences of a loss through one
    channels-last layer (ReLU on), for an input, a weight and a bias entry."""
    rng = np.random.default_rng(9)
    x = rng.standard_normal((1, 3, 4, 5, 2))
    w = rng.standard_normal((27, 3, 2)) * 0.3
    b = rng.standard_normal(3) * 0.1
    gy = rng.standard_normal((1, 3, 4, 5, 3))

    def L(x_, w_, b_):
        return float(np.sum(W.conv3d_cl(x_, w_, b_, True) * gy))

    y = W.conv3d_cl(x, w, b, True)
    gx, gw, gb = W.conv3d_cl_backward(x, w, y, True, gy)
    h = 1e-6
    for idx in [(0, 1, 2, 3, 1), (0, 0, 0, 0, 0)]:
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        assert np.isclose((L(xp, w, b) - L(xm, w, b)) / (2 * h), gx[idx], rtol=1e-5, atol=1e-8)
    for idx in [(13, 2, 1), (0, 0, 0)]:
        wp = w.copy(); wp[idx] += h
        wm = w.copy(); wm[idx] -= h
        assert np.isclose((L(x, wp, b) - L(x, wm, b)) / (2 * h), gw[idx], rtol=1e-5, atol=1e-8)
    bp = b.copy(); bp[1] += h
    bm = b.copy(); bm[1] -= h
    assert np.isclose((L(x, w, bp) - L(x, w, bm)) / (2 * h), gb[1], rtol=1e-5, atol=1e-8)
