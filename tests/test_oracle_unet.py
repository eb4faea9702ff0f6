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


def _routing_theta(base, spec):
    """Flat parameters from {(conv, out, in, tap): value} and {(conv, out): bias}."""
    shapes = unet_ref.layer_shapes(base)
    theta = np.zeros(unet_ref.num_params(base))
    offs, off = [], 0
    for ci, co in shapes:
        offs.append(off)
        off += 9 * ci * co + co
    for (l, o, i, tap), v in spec["w"].items():
        ci, co = shapes[l]
        theta[offs[l] + (tap * co + o) * ci + i] = v
    for (l, o), v in spec["b"].items():
        ci, co = shapes[l]
        theta[offs[l] + 9 * ci * co + o] = v
    return theta


def _wiring_case():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "unet_wiring.json")))
    base = g["base"]
    C = unet_ref.layer_shapes(base)
    w = {(0, 0, 0, 4): 1.0, (0, 1, 0, 4): -1.0, (0, 2, 1, 4): 1.0,
         (1, 0, 0, 4): 1.0, (1, 0, 1, 4): 1.0, (1, 1, 2, 4): 1.0}
    for l in range(2, 9):
        w[(l, 0, 0, 4)] = 1.0
    w[(9, 0, 0, 4)] = 1.0
    w[(9, 0, C[8][1], 4)] = 10.0                 # skip half starts after conv8's outputs
    w[(10, 0, 0, 4)] = 1.0
    w[(11, 0, 0, 4)] = 1.0
    w[(12, 0, 0, 4)] = 1.0
    w[(12, 0, C[11][1], 4)] = 100.0
    w[(13, 0, 0, 4)] = 1.0
    w[(14, 0, 0, 4)] = 1.0
    w[(15, 0, 0, 4)] = 1.0
    w[(15, 0, C[14][1], 4)] = 1000.0
    w[(15, 1, C[14][1] + 1, 4)] = 1.0
    w[(16, 0, 0, 4)] = 1.0
    w[(16, 1, 1, 4)] = 1.0
    w[(17, 0, 0, 4)] = 1.0
    w[(17, 1, 1, 1)] = -1.0                      # tap 1 = (ky 0, kx 1): the row above
    theta = _routing_theta(base, {"w": w, "b": {(17, 0): -2000.0}})
    x = np.zeros((1, 8, 8, 3))
    x[..., 0] = 1.0
    x[0, 0, 0, 0] = 5.0
    x[..., 1] = (np.arange(8) + 1.0)[None, :, None]
    x[..., 2] = 7.0
    return g, base, theta, x


def test_wiring_matches_hand_derived_golden():
    """Routing weights make the network's output a closed form of block
    means (tests/golden/unet_wiring.json, derived by hand): average (not max)
    pooling, nearest (not bilinear) upsampling, the skip of the matching
    level, [upsampled, skip] concatenation order, a ReLU after inner
    convolutions and none after the last, and the tap orientation."""
    g, base, theta, x = _wiring_case()
    _, _, out = unet_ref.loss_and_grad(theta, x, np.zeros((1, 8, 8, 2)), base, torch.float64)
    want0 = np.array(g["out0"])
    want1 = np.array(g["out1"])
    np.testing.assert_array_equal(out[0, :, :, 0], want0)
    np.testing.assert_array_equal(out[0, :, :, 1], want1)


def test_wiring_pin_catches_planted_mistakes():
    """The golden case fails for each plausible wiring mistake, planted in a
    copy of the oracle's forward pass."""
    import torch.nn.functional as F
    g, base, theta, x = _wiring_case()
    want0 = np.array(g["out0"])
    orig_pool, orig_interp, orig_cat = F.avg_pool2d, F.interpolate, torch.cat
    mistakes = {
        "max pooling": lambda: setattr(F, "avg_pool2d", lambda t, k: F.max_pool2d(t, k)),
        "bilinear upsampling": lambda: setattr(
            F, "interpolate", lambda t, scale_factor, mode: orig_interp(t, scale_factor=scale_factor,
                                                                         mode="bilinear", align_corners=False)),
        "concat order": lambda: setattr(torch, "cat", lambda ts, d: orig_cat(ts[::-1], d)),
    }
    try:
        for name, plant in mistakes.items():
            plant()
            _, _, out = unet_ref.loss_and_grad(theta, x, np.zeros((1, 8, 8, 2)), base, torch.float64)
            F.avg_pool2d, F.interpolate, torch.cat = orig_pool, orig_interp, orig_cat
            assert not np.array_equal(out[0, :, :, 0], want0), name
    finally:
        F.avg_pool2d, F.interpolate, torch.cat = orig_pool, orig_interp, orig_cat


def test_bf16_storage_rounds_within_bf16_steps():
    """The storage emulation moves the FP64 forward pass by BF16 rounding
    only: on a small network the outputs agree to a few BF16 steps of the
    output scale."""
    base = 16
    rng = np.random.default_rng(5)
    theta = np.zeros(unet_ref.num_params(base))
    off = 0
    for ci, co in unet_ref.layer_shapes(base):
        theta[off:off + 9 * ci * co] = rng.normal(size=9 * ci * co) * np.sqrt(2.0 / (9 * ci))
        off += 9 * ci * co + co
    x = rng.normal(size=(1, 16, 16, 3))
    t = np.zeros((1, 16, 16, 2))
    _, g64, o64 = unet_ref.loss_and_grad(theta, x, t, base, torch.float64)
    _, gbf, obf = unet_ref.loss_and_grad(theta, x, t, base, torch.float64, bf16_storage=True)
    scale = np.abs(o64).mean()
    assert 0 < np.abs(obf - o64).max() <= 2 ** -3 * scale
    assert np.linalg.norm(gbf - g64) <= 2 ** -4 * np.linalg.norm(g64)
