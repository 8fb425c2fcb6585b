"""FP64 CPU oracle of the warm-start network (TEST INFRASTRUCTURE ONLY).

A plain numpy restatement of every operation the GPU network runs, written
from the definitions and used only by the tests: 3x3 convolution with zero
padding (NHWC activations, weights [Cout][3][3][Cin]), its input and weight
gradients, ReLU, 2x2 average pooling, nearest 2x upsampling, channel
concatenation, mean-squared error and Adam.  `unet_*` composes them into the
encoder-decoder the library trains:

  level l = 0 .. L-1 (channels C_l):  x -> conv(C_l)+ReLU -> conv(C_l)+ReLU = s_l,
      then (l < L-1) 2x2 average pool -> next level;
  going up, l = L-2 .. 0:  upsample2(current) ++ s_l (channels C_{l+1} + C_l)
      -> conv(C_l)+ReLU -> conv(C_l)+ReLU;
  head: conv(Cout), no activation.  Loss: mean over all outputs of (y - t)^2.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, w, b=None):
    """y[b,h,w,o] = sum_{kh,kw,i} xpad[b,h+kh,w+kw,i] w[o,kh,kw,i] (+ bias[o])."""
    B, H, W, Ci = x.shape
    Co = w.shape[0]
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:H + 1, 1:W + 1] = x
    y = np.zeros((B, H, W, Co))
    for kh in range(3):
        for kw in range(3):
            y += xp[:, kh:kh + H, kw:kw + W, :] @ w[:, kh, kw, :].T
    if b is not None:
        y += b
    return y


def conv3x3_backward(x, w, dy):
    """Gradients (dx, dw, db) of conv3x3 for the upstream gradient dy."""
    B, H, W, Ci = x.shape
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:H + 1, 1:W + 1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for kh in range(3):
        for kw in range(3):
            win = xp[:, kh:kh + H, kw:kw + W, :]
            dw[:, kh, kw, :] = np.einsum("bhwo,bhwi->oi", dy, win)
            dxp[:, kh:kh + H, kw:kw + W, :] += dy @ w[:, kh, kw, :]
    db = dy.sum(axis=(0, 1, 2))
    return dxp[:, 1:H + 1, 1:W + 1], dw, db


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(dy):
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def mse(y, t):
    d = y - t
    return float((d * d).mean()), 2.0 * d / d.size


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def unet_layers(cin, channels, cout):
    """(name, Cin, Cout, relu) of every convolution, in forward order."""
    L = len(channels)
    layers = []
    c = cin
    for l in range(L):
        layers += [(f"e{l}a", c, channels[l], True), (f"e{l}b", channels[l], channels[l], True)]
        c = channels[l]
    for l in range(L - 2, -1, -1):
        layers += [(f"d{l}a", channels[l + 1] + channels[l], channels[l], True),
                   (f"d{l}b", channels[l], channels[l], True)]
    layers.append(("head", channels[0], cout, False))
    return layers


def unet_forward(params, x, channels):
    """Forward pass; params[name] = (w, b).  Returns (y, cache)."""
    L = len(channels)
    cache = {}

    def conv(name, inp, act):
        w, b = params[name]
        z = conv3x3(inp, w, b)
        out = relu(z) if act else z
        cache[name] = (inp, out, act)
        return out

    skips = []
    h = x
    for l in range(L):
        h = conv(f"e{l}a", h, True)
        h = conv(f"e{l}b", h, True)
        skips.append(h)
        if l < L - 1:
            h = avgpool2(h)
    for l in range(L - 2, -1, -1):
        up = upsample2(h)
        cat = np.concatenate([up, skips[l]], axis=-1)
        cache[f"cat{l}"] = up.shape[-1]
        h = conv(f"d{l}a", cat, True)
        h = conv(f"d{l}b", h, True)
    y = conv("head", h, False)
    return y, cache


def unet_grads(params, x, t, channels):
    """Loss and gradients of the U-Net by the chain rule, level by level."""
    L = len(channels)
    y, cache = unet_forward(params, x, channels)
    loss, dy = mse(y, t)
    grads = {}

    def conv_back(name, dout):
        inp, out, act = cache[name]
        w, _ = params[name]
        dz = dout * (out > 0) if act else dout
        dx, dw, db = conv3x3_backward(inp, w, dz)
        grads[name] = (dw, db)
        return dx

    # decoder in reverse forward order (level 0 first): after level l, d is
    # the gradient of the tensor that was upsampled into it, i.e. the output
    # of decoder level l+1, or of the deepest encoder level after l = L-2
    d = conv_back("head", dy)
    dskip = {}
    for l in range(0, L - 1):
        d = conv_back(f"d{l}b", d)
        dcat = conv_back(f"d{l}a", d)
        cu = cache[f"cat{l}"]
        dskip[l] = dcat[..., cu:]
        d = upsample2_backward(dcat[..., :cu])
    # encoder, deepest level first: the gradient of s_l is the pooled path's
    # plus the skip's
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            d = avgpool2_backward(d) + dskip[l]
        d = conv_back(f"e{l}b", d)
        d = conv_back(f"e{l}a", d)
    return loss, grads, y
