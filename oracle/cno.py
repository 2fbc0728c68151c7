"""FP64 reference of the convolutional neural operator used as the learned
surrogate of the LB step (test infrastructure only).

The surrogate maps the macroscopic fields of the lattice at step n (phi, T,
f_s, C, u_x, u_y, p; normalised, Sec. 2-3 name them) to their change over the
next k steps.  The paper has no network; this module is the plain definition
of the one this project trains, written as the textbook operations so that a
reader can check every line:

* a 3x3 convolution with zero padding (cross-correlation, the convention of
  every deep-learning library): y[n,h,w,o] = b[o] + sum_{t,i} x[n,h+dy_t,w+dx_t,i] W[o,t,i],
  tap t = 3 (dy + 1) + (dx + 1) for dy, dx in {-1, 0, 1}, x = 0 outside the image;
* the leaky rectifier lrelu(z) = z for z > 0, alpha z otherwise, alpha = 1/16,
  whose derivative is taken as alpha at z = 0;
* 2x2 average pooling and nearest-neighbour 2x upsampling;
* a four-level U-shaped network (encoder of two convolutions per level, pooling
  between levels, decoder that upsamples and adds the encoder output of the same
  level before its convolution, and a linear 3x3 head);
* the mean squared error over the first `nf` output channels;
* Adam (Kingma and Ba, 2015, Algorithm 1) with bias correction.

Tensors are NHWC float64 numpy arrays; weights are [out, 9, in].  Backward
passes follow from the chain rule on these definitions and are pinned in the
tests by finite differences, adjoint identities and brute force.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.
"""
from __future__ import annotations

import numpy as np

ALPHA = 1.0 / 16.0
TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]  # tap t = 3 (dy + 1) + (dx + 1)


def layer_table(cin: int, widths, cout: int):
    """(in, out, activation) of the twelve convolutions, in forward order.

    widths = (c0, c1, c2, c3) are the channel counts of the four levels; the
    decoder adds the bottleneck output to the level-2 encoder output, so c3
    must equal c2."""
    c0, c1, c2, c3 = widths
    if c3 != c2:
        raise ValueError("the level-3 width must equal the level-2 width (skip addition)")
    return [(cin, c0, True), (c0, c0, True),      # level 0 encoder
            (c0, c1, True), (c1, c1, True),       # level 1 encoder
            (c1, c2, True), (c2, c2, True),       # level 2 encoder
            (c2, c3, True), (c3, c3, True),       # level 3 (bottleneck)
            (c3, c1, True),                       # level 2 decoder
            (c1, c0, True),                       # level 1 decoder
            (c0, c0, True),                       # level 0 decoder
            (c0, cout, False)]                    # head


def lrelu(z):
    return np.where(z > 0, z, ALPHA * z)


def lrelu_slope(y):
    """Derivative of lrelu at z, from its output y = lrelu(z) (y > 0 iff z > 0)."""
    return np.where(y > 0, 1.0, ALPHA)


def _shifted(x, dy, dx):
    """s[n,h,w,:] = x[n,h+dy,w+dx,:], zero where (h+dy, w+dx) leaves the image."""
    n, hh, ww, c = x.shape
    s = np.zeros_like(x)
    h0, h1 = max(0, -dy), min(hh, hh - dy)
    w0, w1 = max(0, -dx), min(ww, ww - dx)
    if h1 > h0 and w1 > w0:
        s[:, h0:h1, w0:w1, :] = x[:, h0 + dy:h1 + dy, w0 + dx:w1 + dx, :]
    return s


def conv3x3(x, w, b=None):
    """y[n,h,w,o] = b[o] + sum_{t,i} x[n,h+dy_t,w+dx_t,i] W[o,t,i] (zero padding)."""
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (dy, dx) in enumerate(TAPS):
        y += np.einsum("nhwi,oi->nhwo", _shifted(x, dy, dx), w[:, t, :])
    if b is not None:
        y += b
    return y


def conv3x3_backward(x, w, dz):
    """Gradients of sum(dz * conv3x3(x, w, b)) with respect to x, W and b.

    dx[n,h,w,i] = sum_{t,o} dz[n,h-dy_t,w-dx_t,o] W[o,t,i]
    dW[o,t,i]   = sum_{n,h,w} dz[n,h,w,o] x[n,h+dy_t,w+dx_t,i]
    db[o]       = sum_{n,h,w} dz[n,h,w,o]"""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (dy, dxs) in enumerate(TAPS):
        dx += np.einsum("nhwo,oi->nhwi", _shifted(dz, -dy, -dxs), w[:, t, :])
        dw[:, t, :] = np.einsum("nhwo,nhwi->oi", dz, _shifted(x, dy, dxs))
    db = dz.sum(axis=(0, 1, 2))
    return dx, dw, db


def pool2(x):
    """2x2 average pooling (H and W even)."""
    n, hh, ww, c = x.shape
    return x.reshape(n, hh // 2, 2, ww // 2, 2, c).mean(axis=(2, 4))


def up2(x):
    """Nearest-neighbour 2x upsampling."""
    return x.repeat(2, axis=1).repeat(2, axis=2)


def forward(params, x):
    """Network output and the activations the backward pass needs.

    params: list of (W, b) in the order of layer_table.  Returns (out, cache)."""
    a = {}
    def conv(k, inp):
        w, b = params[k]
        z = conv3x3(inp, w, b)
        return lrelu(z)
    a["x0"] = x
    a["a0"] = conv(0, x)
    a["e0"] = conv(1, a["a0"])
    a["p1"] = pool2(a["e0"])
    a["a1"] = conv(2, a["p1"])
    a["e1"] = conv(3, a["a1"])
    a["p2"] = pool2(a["e1"])
    a["a2"] = conv(4, a["p2"])
    a["e2"] = conv(5, a["a2"])
    a["p3"] = pool2(a["e2"])
    a["a3"] = conv(6, a["p3"])
    a["e3"] = conv(7, a["a3"])
    a["u2"] = up2(a["e3"]) + a["e2"]
    a["d2"] = conv(8, a["u2"])
    a["u1"] = up2(a["d2"]) + a["e1"]
    a["d1"] = conv(9, a["u1"])
    a["u0"] = up2(a["d1"]) + a["e0"]
    a["d0"] = conv(10, a["u0"])
    w, b = params[11]
    out = conv3x3(a["d0"], w, b)
    return out, a


def backward(params, a, dout):
    """Gradients [(dW, db)] of sum(dout * out) for every layer, by the chain rule
    through forward()."""
    g = [None] * 12
    def lay(k, inp, dz):
        dx, dw, db = conv3x3_backward(inp, params[k][0], dz)
        g[k] = (dw, db)
        return dx
    d_d0 = lay(11, a["d0"], dout)
    d_u0 = lay(10, a["u0"], d_d0 * lrelu_slope(a["d0"]))
    d_d1 = pool2(d_u0) * 4.0                       # adjoint of up2: sum over the 2x2 block
    d_u1 = lay(9, a["u1"], d_d1 * lrelu_slope(a["d1"]))
    d_d2 = pool2(d_u1) * 4.0
    d_u2 = lay(8, a["u2"], d_d2 * lrelu_slope(a["d2"]))
    d_e3 = pool2(d_u2) * 4.0
    d_a3 = lay(7, a["a3"], d_e3 * lrelu_slope(a["e3"]))
    d_p3 = lay(6, a["p3"], d_a3 * lrelu_slope(a["a3"]))
    d_e2 = d_u2 + up2(d_p3) / 4.0                  # skip path + adjoint of pool2
    d_a2 = lay(5, a["a2"], d_e2 * lrelu_slope(a["e2"]))
    d_p2 = lay(4, a["p2"], d_a2 * lrelu_slope(a["a2"]))
    d_e1 = d_u1 + up2(d_p2) / 4.0
    d_a1 = lay(3, a["a1"], d_e1 * lrelu_slope(a["e1"]))
    d_p1 = lay(2, a["p1"], d_a1 * lrelu_slope(a["a1"]))
    d_e0 = d_u0 + up2(d_p1) / 4.0
    d_a0 = lay(1, a["a0"], d_e0 * lrelu_slope(a["e0"]))
    lay(0, a["x0"], d_a0 * lrelu_slope(a["a0"]))
    return g


def mse(out, target, nf):
    """Mean squared error over the first nf channels and its gradient."""
    diff = out[..., :nf] - target[..., :nf]
    count = diff.size
    dout = np.zeros_like(out)
    dout[..., :nf] = 2.0 * diff / count
    return float((diff * diff).sum() / count), dout


def adam(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1 (Kingma and Ba, Algorithm 1); returns
    (p, m, v) new."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
