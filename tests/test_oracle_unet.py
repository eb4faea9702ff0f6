"""Pins for the CPU oracle of the warm-start network: gradients against
central finite differences, a convolution against a direct loop, and the
closed form of an all-zero network."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet_ref  # noqa: E402


def test_param_count():
    assert unet_ref.num_params(16) == sum(9 * a * b + b for a, b in unet_ref.layer_shapes(16))


def test_zero_weights_give_last_bias():
    base = 16
    theta = np.zeros(unet_ref.num_params(base))
    theta[-16:] = np.arange(16) + 0.5             # bias of the last convolution
    x = np.random.default_rng(0).normal(size=(1, 8, 8, 3))
    _, _, out = unet_ref.loss_and_grad(theta, x, np.zeros((1, 8, 8, 2)), base, torch.float64)
    np.testing.assert_allclose(out[..., 0], 0.5)
    np.testing.assert_allclose(out[..., 1], 1.5)


def test_conv_matches_direct_loop():
    rng = np.random.default_rng(1)
    ci, co, h, w = 16, 16, 5, 6
    wk = rng.normal(size=(9, co, ci))             # the library layout [tap][Cout][Cin]
    b = rng.normal(size=co)
    x = rng.normal(size=(1, ci, h, w))
    theta = np.zeros(unet_ref.num_params(16))      # layer 0 of a base-16 net is 16 -> 16
    theta[:9 * co * ci] = wk.ravel()
    theta[9 * co * ci:9 * co * ci + co] = b
    layer0 = unet_ref.unpack(torch.tensor(theta), 16)[0]
    y = unet_ref.conv(torch.tensor(x), layer0, relu=False).numpy()
    ref = np.zeros((co, h, w))
    for o in range(co):
        for yy in range(h):
            for xx in range(w):
                s = b[o]
                for ky in range(3):
                    for kx in range(3):
                        sy, sx = yy + ky - 1, xx + kx - 1
                        if 0 <= sy < h and 0 <= sx < w:
                            s += wk[3 * ky + kx, o] @ x[0, :, sy, sx]
                ref[o, yy, xx] = s
    np.testing.assert_allclose(y[0], ref, rtol=1e-10, atol=1e-10)


def test_gradient_finite_differences():
    base = 16
    rng = np.random.default_rng(2)
    theta = rng.normal(size=unet_ref.num_params(base)) * 0.2
    x = rng.normal(size=(1, 8, 8, 3))
    t = rng.normal(size=(1, 8, 8, 2))
    _, g, _ = unet_ref.loss_and_grad(theta, x, t, base, torch.float64)
    eps = 1e-6
    for i in rng.choice(theta.size, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        lp = unet_ref.loss_and_grad(tp, x, t, base, torch.float64)[0]
        lm = unet_ref.loss_and_grad(tm, x, t, base, torch.float64)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
