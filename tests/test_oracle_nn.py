"""Pins of the network oracle: every gradient against central finite
differences of its own forward definition, and special cases with closed
forms (identity kernels, constant inputs, pooling adjoints)."""
import numpy as np
import pytest

from oracle import nn
import synth


def _rng(seed):
    r = synth.SplitMix64(seed)
    return lambda *shape: np.array([r.uniform() - 0.5 for _ in range(int(np.prod(shape)))]).reshape(shape)


def test_conv_identity_and_shift_kernels():
    R = _rng(1)
    x = R(2, 5, 6, 3)
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, 1, 1, c] = 1.0  # centre tap: identity
    assert np.allclose(nn.conv3x3(x, w), x)
    w = np.zeros((1, 3, 3, 3))
    w[0, 0, 1, 0] = 1.0  # tap (kh=0): y[h] = x[h-1], zero above the top row
    y = nn.conv3x3(x, w)[..., 0]
    assert np.allclose(y[:, 1:], x[:, :-1, :, 0]) and np.allclose(y[:, 0], 0.0)


def test_conv_against_explicit_loops():
    R = _rng(2)
    x, w, b = R(1, 4, 3, 2), R(3, 3, 3, 2), R(3)
    y = nn.conv3x3(x, w, b)
    ref = np.zeros_like(y)
    for h in range(4):
        for ww in range(3):
            for o in range(3):
                s = b[o]
                for kh in range(3):
                    for kw in range(3):
                        hh, xx = h + kh - 1, ww + kw - 1
                        if 0 <= hh < 4 and 0 <= xx < 3:
                            s += np.dot(x[0, hh, xx], w[o, kh, kw])
                ref[0, h, ww, o] = s
    assert np.allclose(y, ref, atol=1e-14)


def _fd(f, arr, idx, h=1e-6):
    old = arr[idx]
    arr[idx] = old + h
    fp = f()
    arr[idx] = old - h
    fm = f()
    arr[idx] = old
    return (fp - fm) / (2 * h)


def test_conv_backward_finite_differences():
    R = _rng(3)
    x, w, b = R(2, 4, 5, 3), R(4, 3, 3, 3), R(4)
    t = R(2, 4, 5, 4)
    loss = lambda: float(((nn.conv3x3(x, w, b) - t) ** 2).sum())
    dy = 2 * (nn.conv3x3(x, w, b) - t)
    dx, dw, db = nn.conv3x3_backward(x, w, dy)
    for idx in [(0, 0, 0, 0), (1, 3, 4, 2), (0, 2, 1, 1)]:
        assert dx[idx] == pytest.approx(_fd(loss, x, idx), rel=1e-6, abs=1e-8)
    for idx in [(0, 0, 0, 0), (3, 2, 1, 2), (1, 1, 2, 0)]:
        assert dw[idx] == pytest.approx(_fd(loss, w, idx), rel=1e-6, abs=1e-8)
    assert db[2] == pytest.approx(_fd(loss, b, (2,)), rel=1e-6)


def test_pool_and_upsample_are_adjoint():
    R = _rng(4)
    a, b = R(2, 6, 4, 3), R(2, 3, 2, 3)
    # <pool(a), b> = <a, pool^T(b)> and <up(b), a> = <b, up^T(a)>
    assert np.dot(nn.avgpool2(a).ravel(), b.ravel()) == pytest.approx(
        np.dot(a.ravel(), nn.avgpool2_backward(b).ravel()))
    assert np.dot(nn.upsample2(b).ravel(), a.ravel()) == pytest.approx(
        np.dot(b.ravel(), nn.upsample2_backward(a).ravel()))
    assert np.allclose(nn.avgpool2(np.ones((1, 4, 4, 1))), 1.0)


def test_adam_first_step_is_sign_step():
    """With bias correction the first Adam step moves by lr * g/|g|."""
    p, g = np.array([1.0, -2.0, 3.0]), np.array([0.5, -4.0, 1e-3])
    p1, _, _ = nn.adam(p, g, np.zeros(3), np.zeros(3), 1, 0.01, eps=0.0)
    assert np.allclose(p1, p - 0.01 * np.sign(g))


def _small_unet(seed, cin=2, channels=(4, 6), cout=2):
    R = _rng(seed)
    params = {}
    for name, ci, co, _ in nn.unet_layers(cin, channels, cout):
        params[name] = (0.5 * R(co, 3, 3, ci), 0.1 * R(co))
    return params


@pytest.mark.parametrize("channels", [(4, 6), (3, 4, 5)])
def test_unet_gradients_finite_differences(channels):
    R = _rng(5)
    params = _small_unet(6, channels=channels)
    x = R(2, 8, 8, 2)
    t = R(2, 8, 8, 2)
    loss, grads, _ = nn.unet_grads(params, x, t, channels)

    def f():
        y, _ = nn.unet_forward(params, x, channels)
        return nn.mse(y, t)[0]

    assert loss == pytest.approx(f())
    names = [n for n, *_ in nn.unet_layers(2, channels, 2)]
    for k, name in enumerate(names):
        w, b = params[name]
        idx = (k % w.shape[0], 1, 2, k % w.shape[3])
        assert grads[name][0][idx] == pytest.approx(_fd(f, w, idx), rel=1e-5, abs=1e-10), name
        assert grads[name][1][0] == pytest.approx(_fd(f, b, (0,)), rel=1e-5, abs=1e-10), name
