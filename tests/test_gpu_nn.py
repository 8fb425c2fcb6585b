"""Tensor-core convolution kernels and the warm-start U-Net against the FP64
network oracle.  Inputs are rounded to BF16 first, so the kernels and the
oracle see the same numbers; the kernels accumulate in FP32 (bound 1e-5
relative for FP32 outputs, 2^-8 for BF16 outputs)."""
import numpy as np
import pytest

from oracle import nn as onn
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_08591_gb300 import _build
    _build.build()


def _bf16(shape, seed, scale=1.0):
    import torch
    r = synth.SplitMix64(seed)
    a = np.array([r.uniform() - 0.5 for _ in range(int(np.prod(shape)))], dtype=np.float32).reshape(shape)
    t = torch.from_numpy(a * scale).to(torch.bfloat16)
    return t.cuda(), t.float().numpy().astype(np.float64)


def _rel(ref, got):
    return float(np.linalg.norm((ref - got).ravel()) / np.linalg.norm(ref.ravel()))


@pytest.fixture(params=["tcgen05-halo", "tcgen05", "mma.sync"])
def kernel(request):
    from paper_2108_08591_gb300 import conv_timeout_flag, set_conv_kernel
    set_conv_kernel(request.param)
    yield request.param
    assert conv_timeout_flag() == 0
    set_conv_kernel("tcgen05-halo")


# shapes: ragged M and N tiles, Cin 8 (halo kernel falls back), Cin 16/32/64/96,
# widths above 64 (several column strips, a narrow last one), 256-wide N tiles
@pytest.mark.parametrize("B,H,W,Cin,Cout", [(2, 10, 7, 16, 40), (1, 8, 8, 96, 32), (3, 5, 9, 8, 16),
                                            (2, 16, 16, 32, 136), (1, 20, 13, 64, 256),
                                            (1, 12, 130, 32, 48), (2, 9, 70, 16, 16), (1, 6, 64, 64, 64)])
def test_conv_forward(kernel, B, H, W, Cin, Cout):
    import torch
    from paper_2108_08591_gb300 import conv3x3_bf16
    x, xn = _bf16((B, H, W, Cin), 1)
    w, wn = _bf16((Cout, 3, 3, Cin), 2)
    bias = torch.linspace(-0.2, 0.3, Cout, device="cuda", dtype=torch.float32)
    ref = onn.conv3x3(xn, wn, bias.cpu().numpy().astype(np.float64))
    got = conv3x3_bf16(x, w, bias).cpu().numpy()
    assert _rel(ref, got) < 1e-5
    got = conv3x3_bf16(x, w, bias, relu=True, out_fp32=False).float().cpu().numpy()
    r = onn.relu(ref)
    assert np.all(np.abs(got - r) <= 2.0 ** -8 * np.abs(r) + 1e-6)


WGRAD_VARIANTS = {  # kernel, channel tile, CTAs per SM, positions per stage
    "tcgen05": ("tcgen05", 0, 0, 0),
    "tcgen05-bn16": ("tcgen05", 16, 1, 0),
    "tcgen05-bn64": ("tcgen05", 64, 1, 0),
    "tcgen05-k64": ("tcgen05", 0, 4, 64),
    "tcgen05-k128": ("tcgen05", 32, 2, 128),
    "mma.sync": ("mma.sync", 0, 0, 0),
}


@pytest.fixture(params=list(WGRAD_VARIANTS))
def wgrad_kernel(request):
    """The weight-gradient kernels; the tcgen05 one also with its 16- and
    64-channel tiles, both pipeline stage lengths and shallow and deep
    pipelines."""
    from paper_2108_08591_gb300 import conv_timeout_flag, set_wgrad_kernel, set_wgrad_tile
    kern, bn, ctas, kc = WGRAD_VARIANTS[request.param]
    set_wgrad_kernel(kern)
    set_wgrad_tile(bn, ctas, kc)
    yield request.param
    assert conv_timeout_flag() == 0
    set_wgrad_kernel("tcgen05")
    set_wgrad_tile(0, 0, 0)


# shapes: ragged channel tiles, Cin 8 (tcgen05 wgrad falls back), several
# column strips, more than 128 output channels (two M tiles), more input
# than output channels (the tcgen05 weight gradient's swapped roles: 96 ->
# 32, and 160 -> 32 with two M tiles of input channels)
@pytest.mark.parametrize("B,H,W,Cin,Cout", [(2, 10, 7, 16, 40), (1, 8, 8, 96, 32), (2, 16, 16, 32, 64),
                                            (1, 5, 66, 32, 16), (3, 5, 9, 8, 16), (1, 12, 130, 32, 48),
                                            (2, 9, 9, 64, 136), (1, 6, 20, 160, 32)])
def test_conv_backward(kernel, wgrad_kernel, B, H, W, Cin, Cout):
    import torch
    from paper_2108_08591_gb300 import conv3x3_bf16_backward, conv3x3_bf16_wgrad
    x, xn = _bf16((B, H, W, Cin), 3)
    w, wn = _bf16((Cout, 3, 3, Cin), 4)
    dz, dzn = _bf16((B, H, W, Cout), 5)
    dx_ref, dw_ref, _ = onn.conv3x3_backward(xn, wn, dzn)
    dx, dw = conv3x3_bf16_backward(x, w, dz)
    assert _rel(dw_ref, dw.cpu().numpy()) < 1e-5
    assert torch.equal(conv3x3_bf16_wgrad(x, dz), dw)  # the same kernel alone
    got = dx.float().cpu().numpy()
    assert np.all(np.abs(got - dx_ref) <= 2.0 ** -8 * np.abs(dx_ref) + 1e-5)


def _oracle_params(flat, cin, channels, cout):
    params, off = {}, 0
    for name, ci, co, _ in onn.unet_layers(cin, channels, cout):
        nw = co * 9 * ci
        w = flat[off:off + nw].reshape(co, 3, 3, ci).astype(np.float64)
        b = flat[off + nw:off + nw + co].astype(np.float64)
        params[name] = (w, b)
        off += nw + co
    assert off == flat.size
    return params


def test_unet_gradients_match_oracle():
    """One training step (lr = 0) of a small U-Net: loss and every parameter
    gradient against the FP64 chain rule of the oracle.  The GPU rounds
    activations and gradients to BF16 between layers, so the error grows
    along the backward chain (measured: 5e-3 at the head, up to ~0.1 for the
    first encoder layer) while the direction stays: cosine >= 0.99 for every
    layer (a wrong flip, transpose or slice would break it), relative error
    <= 2e-2 for the head and the last decoder level, <= 0.15 elsewhere."""
    import torch
    from paper_2108_08591_gb300 import WarmStartNet
    channels, cin, cout, B, H = (16, 32, 48), 16, 16, 2, 16
    net = WarmStartNet(H, H, channels, cin=cin, cout=cout, cout_used=cout, max_batch=B, seed=7)
    xb, xn = _bf16((B, H, H, cin), 11)
    t = torch.from_numpy(np.sin(np.arange(B * H * H * cout) * 0.37).reshape(B, H, H, cout)
                         .astype(np.float32)).cuda()
    loss = net.train_step(xb.float().contiguous(), t, lr=0.0)
    p, g = net.get_params(grads=True)
    params = _oracle_params(p, cin, channels, cout)
    lref, gref, _ = onn.unet_grads(params, xn, t.cpu().numpy().astype(np.float64), channels)
    assert loss == pytest.approx(lref, rel=1e-2)
    got = _oracle_params(g, cin, channels, cout)
    for name in params:
        ew, eb = _rel(gref[name][0], got[name][0]), _rel(gref[name][1], got[name][1])
        cw = float(np.dot(gref[name][0].ravel(), got[name][0].ravel()) /
                   (np.linalg.norm(gref[name][0]) * np.linalg.norm(got[name][0])))
        print(f"GRAD {name} w {ew:.3e} b {eb:.3e} cos {cw:.6f}")
    for name in params:
        bound = 2e-2 if name in ("head", "d0b", "d0a") else 0.15
        assert _rel(gref[name][0], got[name][0]) < bound, name
        assert _rel(gref[name][1], got[name][1]) < bound, name
        cw = float(np.dot(gref[name][0].ravel(), got[name][0].ravel()) /
                   (np.linalg.norm(gref[name][0]) * np.linalg.norm(got[name][0])))
        assert cw > 0.99, name
    net.close()


def test_training_reduces_the_loss():
    import torch
    from paper_2108_08591_gb300 import WarmStartNet
    H, B = 32, 4
    net = WarmStartNet(H, H, (16, 32, 64), cin=16, cout=16, cout_used=3, max_batch=B, seed=3)
    yy, xx = np.meshgrid(np.linspace(0, 1, H), np.linspace(0, 1, H), indexing="ij")
    x = np.zeros((B, H, H, 16), np.float32)
    t = np.zeros((B, H, H, 3), np.float32)
    for b in range(B):
        a = 0.5 + b / B
        x[b, :, :, 0], x[b, :, :, 1], x[b, :, :, 2] = a, xx, yy
        t[b, :, :, 0] = a * np.sin(np.pi * xx) * np.sin(np.pi * yy)
        t[b, :, :, 1] = a * xx * yy
        t[b, :, :, 2] = -a * yy * (1 - yy)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = net.train_step(xd, td, lr=2e-3)
    for _ in range(300):
        last = net.train_step(xd, td, lr=2e-3, want_loss=False)
    last = net.train_step(xd, td, lr=2e-3)
    assert last < 0.05 * first, (first, last)
    net.close()


def test_every_tcgen05_tile_matches_oracle():
    """Every instantiated tile of the two tcgen05 forward kernels, chosen
    through the tuning overrides: halo kernel N tile 16..256 x 1 or 2 M tiles
    x 16- or 32-channel chunks, im2col kernel N tile 16..256 x 3, 4 or 6
    stages (256 x 6 does not fit and is rejected).  A ragged shape with two
    column strips; FP32 output against the FP64 oracle."""
    import torch
    from paper_2108_08591_gb300 import _lib, conv3x3_bf16, conv_timeout_flag, set_conv_kernel
    lib = _lib.load()
    B, H, W, Cin, Cout = 2, 11, 70, 32, 40
    x, xn = _bf16((B, H, W, Cin), 21)
    w, wn = _bf16((Cout, 3, 3, Cin), 22)
    ref = onn.conv3x3(xn, wn, np.zeros(Cout))
    try:
        set_conv_kernel("tcgen05-halo")
        for bn in (16, 32, 64, 128, 256):
            for mt in (1, 2):
                for kc in (16, 32):
                    assert lib.mdf_nn_set_tc_tile(bn, 0) == 0 and lib.mdf_nn_set_halo_tile(mt, kc) == 0
                    got = conv3x3_bf16(x, w).cpu().numpy()
                    assert _rel(ref, got) < 1e-5, ("halo", bn, mt, kc, _rel(ref, got))
        lib.mdf_nn_set_halo_tile(0, 0)
        set_conv_kernel("tcgen05")
        for bn in (16, 32, 64, 128, 256):
            for st in (3, 4, 6):
                rc = lib.mdf_nn_set_tc_tile(bn, st)
                if bn == 256 and st == 6:
                    assert rc != 0
                    continue
                assert rc == 0
                got = conv3x3_bf16(x, w).cpu().numpy()
                assert _rel(ref, got) < 1e-5, ("im2col", bn, st, _rel(ref, got))
        assert conv_timeout_flag() == 0
    finally:
        lib.mdf_nn_set_tc_tile(0, 0)
        lib.mdf_nn_set_halo_tile(0, 0)
        set_conv_kernel("tcgen05-halo")
