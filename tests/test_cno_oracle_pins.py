"""Pins of the FP64 surrogate-network reference (oracle/cno.py) against things
other than itself: brute-force loops, scipy's 2D correlation, finite
differences of the whole network, adjoint identities and the closed form of
the first Adam steps."""
import itertools

import numpy as np
import pytest

from oracle import cno as C

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_conv3x3_brute_force_loops():
    r = _rng(1)
    x = r.standard_normal((2, 4, 5, 3))
    w = r.standard_normal((4, 9, 3))
    b = r.standard_normal(4)
    y = C.conv3x3(x, w, b)
    n, hh, ww, ci = x.shape
    for nn, h, wc, o in itertools.product(range(n), range(hh), range(ww), range(4)):
        s = b[o]
        for ky in range(3):
            for kx in range(3):
                yy, xx = h + ky - 1, wc + kx - 1
                if 0 <= yy < hh and 0 <= xx < ww:
                    for i in range(ci):
                        s += x[nn, yy, xx, i] * w[o, 3 * ky + kx, i]
        assert abs(y[nn, h, wc, o] - s) < 1e-12


def test_conv3x3_against_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    r = _rng(2)
    x = r.standard_normal((1, 9, 7, 2))
    w = r.standard_normal((3, 9, 2))
    y = C.conv3x3(x, w)
    for o in range(3):
        want = sum(signal.correlate2d(x[0, :, :, i], w[o, :, i].reshape(3, 3), mode="same", boundary="fill")
                   for i in range(2))
        assert np.allclose(y[0, :, :, o], want, atol=1e-12)


def test_conv_backward_adjoint_identities():
    r = _rng(3)
    x = r.standard_normal((2, 6, 5, 3))
    w = r.standard_normal((4, 9, 3))
    dz = r.standard_normal((2, 6, 5, 4))
    dx, dw, db = C.conv3x3_backward(x, w, dz)
    y = C.conv3x3(x, w)
    # <conv(x, w), dz> is bilinear: its partial derivatives are dx and dw
    assert np.isclose((y * dz).sum(), (x * dx).sum(), rtol=1e-12)
    assert np.isclose((y * dz).sum(), (w * dw).sum(), rtol=1e-12)
    assert np.allclose(db, dz.sum(axis=(0, 1, 2)))


def test_conv_backward_finite_differences():
    r = _rng(4)
    x = r.standard_normal((1, 5, 4, 2))
    w = r.standard_normal((3, 9, 2))
    b = r.standard_normal(3)
    dz = r.standard_normal((1, 5, 4, 3))
    dx, dw, db = C.conv3x3_backward(x, w, dz)
    f = lambda xx, ww, bb: (C.conv3x3(xx, ww, bb) * dz).sum()
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 4, 3, 1), (0, 2, 1, 0)]:
        e = np.zeros_like(x); e[idx] = h
        assert abs((f(x + e, w, b) - f(x - e, w, b)) / (2 * h) - dx[idx]) < 1e-7
    for idx in [(0, 0, 0), (2, 8, 1), (1, 4, 0)]:
        e = np.zeros_like(w); e[idx] = h
        assert abs((f(x, w + e, b) - f(x, w - e, b)) / (2 * h) - dw[idx]) < 1e-7
    e = np.zeros_like(b); e[1] = h
    assert abs((f(x, w, b + e) - f(x, w, b - e)) / (2 * h) - db[1]) < 1e-7


def test_pool_up_adjoint_and_inverse():
    r = _rng(5)
    x = r.standard_normal((2, 6, 8, 3))
    y = r.standard_normal((2, 3, 4, 3))
    assert np.isclose((C.pool2(x) * y).sum(), (x * C.up2(y)).sum() / 4.0, rtol=1e-12)
    assert np.allclose(C.pool2(C.up2(y)), y)
    assert np.allclose(C.pool2(np.full((1, 4, 4, 1), 2.5)), 2.5)
    # the four inputs of one output cell
    assert np.isclose(C.pool2(x)[1, 2, 3, 0], x[1, 4:6, 6:8, 0].mean())


def test_lrelu_and_slope():
    z = np.array([-2.0, -1e-30, 0.0, 1e-30, 3.0])
    assert np.array_equal(C.lrelu(z), [-2.0 / 16, -1e-30 / 16, 0.0, 1e-30, 3.0])
    assert np.array_equal(C.lrelu_slope(C.lrelu(z)), [1 / 16, 1 / 16, 1 / 16, 1.0, 1.0])


def _tiny_net(seed=6, cin=2, widths=(2, 3, 4, 4), cout=3):
    r = _rng(seed)
    params = []
    for ci, co, _ in C.layer_table(cin, widths, cout):
        params.append((r.standard_normal((co, 9, ci)) * np.sqrt(2.0 / (9 * ci)), 0.1 * r.standard_normal(co)))
    return params


def test_layer_table_shapes_and_skip_constraint():
    t = C.layer_table(64, (64, 128, 256, 256), 64)
    assert len(t) == 12 and t[0] == (64, 64, True) and t[-1] == (64, 64, False)
    assert [c[1] for c in t] == [64, 64, 128, 128, 256, 256, 256, 256, 128, 64, 64, 64]
    with pytest.raises(ValueError):
        C.layer_table(64, (64, 128, 256, 128), 64)


def test_network_gradient_finite_differences():
    params = _tiny_net()
    r = _rng(7)
    x = r.standard_normal((2, 8, 8, 2))
    target = r.standard_normal((2, 8, 8, 3))
    out, cache = C.forward(params, x)
    loss, dout = C.mse(out, target, nf=2)
    grads = C.backward(params, cache, dout)
    h = 1e-6

    def loss_at(k, which, idx, delta):
        p = [(w.copy(), b.copy()) for w, b in params]
        p[k][which][idx] += delta
        return C.mse(C.forward(p, x)[0], target, nf=2)[0]

    for k in range(12):
        w, b = params[k]
        for idx in [(0, 0, 0), (w.shape[0] - 1, 8, w.shape[2] - 1), (0, 4, 0)]:
            fd = (loss_at(k, 0, idx, h) - loss_at(k, 0, idx, -h)) / (2 * h)
            assert abs(fd - grads[k][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, grads[k][0][idx])
        fd = (loss_at(k, 1, (0,), h) - loss_at(k, 1, (0,), -h)) / (2 * h)
        assert abs(fd - grads[k][1][0]) <= 1e-6 * max(1.0, abs(fd)), (k, "bias")
    # the channels beyond nf carry no loss: the head's gradient there is zero
    assert np.all(grads[11][0][2:] == 0) and np.all(grads[11][1][2:] == 0)


def test_mse_value():
    out = np.zeros((1, 1, 2, 3)); target = np.ones((1, 1, 2, 3))
    loss, dout = C.mse(out, target, nf=2)
    assert loss == 1.0
    assert np.allclose(dout[..., :2], -0.5) and np.all(dout[..., 2] == 0)


def test_adam_first_steps_closed_form():
    g = np.array([0.3, -2.0, 1e-3])
    p0 = np.zeros(3)
    p1, m, v = C.adam(p0, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # after bias correction m_hat = g and v_hat = g^2, so the first step is lr * sign(g) up to eps
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    p2, m, v = C.adam(p1, g, m, v, 2, lr=0.01)
    assert np.allclose(p2 - p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)
