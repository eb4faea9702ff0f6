"""Warm-start network kernels against the CPU oracle (oracle/unet_ref.py),
element by element.

Single convolutions: the GPU multiplies BF16 inputs and weights exactly and
accumulates in FP32, then rounds the output to BF16, so every output obeys
|out - ref| <= 2^-8 |ref| + 2^-12 S with S = sum |w||x| + |b| over its taps
(half a BF16 step plus a generous FP32 accumulation term); the weight
gradient (FP32 accumulation, FP32 output) obeys |dW - ref| <= 2^-12 S_w with
S_w = sum |x||g| over its pixels.

The 18-layer network: the oracle with BF16 storage at the library's storage
points (bf16_storage=True) is the reference; the GPU differs from it where
FP32 summation order flips a BF16 rounding, and the flips propagate.  Every
output obeys |out - ref| <= 8 * 2^-8 (|ref| + mean |ref|) (measured at most
4.8), and every parameter gradient of layer l obeys
|g - ref| <= 48 * 2^-8 (|ref| + rms_l(ref)) on 2 x 128 x 128 inputs
(measured at most 23; BF16 activation gradients through 18 layers)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tv():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01563_gb300 import tvcut
    tvcut.lib()
    return tvcut


def bf16_round(x):
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).float().numpy()


def conv_ref_and_scale(x, wk, b):
    """FP64 reference of a 3x3 convolution (NHWC, weights [9][Cout][Cin],
    zero padding) and S = sum |w||x| + |b| per output."""
    from oracle import unet_ref
    co, ci = wk.shape[1], wk.shape[2]
    Wt = torch.tensor(wk, dtype=torch.float64).reshape(3, 3, co, ci).permute(2, 3, 0, 1)
    xt = torch.tensor(x, dtype=torch.float64).permute(0, 3, 1, 2)
    bt = torch.tensor(b, dtype=torch.float64) if b is not None else torch.zeros(co, dtype=torch.float64)
    ref = unet_ref.F.conv2d(xt, Wt, bt, padding=1).permute(0, 2, 3, 1).numpy()
    S = unet_ref.F.conv2d(xt.abs(), Wt.abs(), bt.abs(), padding=1).permute(0, 2, 3, 1).numpy()
    return ref, S


def assert_conv_bound(got, ref, S, relu):
    if relu:
        ref = np.maximum(ref, 0.0)
    d = np.abs(np.asarray(got, np.float64) - ref)
    bound = 2 ** -8 * np.abs(ref) + 2 ** -12 * S
    assert np.all(d <= bound), float((d / np.maximum(bound, 1e-300)).max())


def layer_slices(base):
    from oracle import unet_ref
    off = 0
    for ci, co in unet_ref.layer_shapes(base):
        k = 9 * ci * co + co
        yield slice(off, off + k)
        off += k


def bf16_weights_f32_bias(theta, base):
    """The parameters the GPU forward pass uses: BF16 weights, FP32 biases."""
    from oracle import unet_ref
    th = np.asarray(theta, np.float64).copy()
    off = 0
    for ci, co in unet_ref.layer_shapes(base):
        k = 9 * ci * co
        th[off:off + k] = bf16_round(theta[off:off + k])
        off += k + co
    return th


@pytest.mark.parametrize("shape", [(1, 16, 16, 16, 32), (2, 9, 13, 32, 16), (1, 8, 8, 64, 128)])
def test_conv_forward_and_wgrad(tv, shape):
    n, h, w, ci, co = shape
    rng = np.random.default_rng(sum(shape))
    x = bf16_round(rng.normal(size=(n, h, w, ci)))
    wk = bf16_round(rng.normal(size=(9, co, ci)) * 0.2)
    b = rng.normal(size=co).astype(np.float32)
    xd = torch.tensor(x).to(torch.bfloat16).cuda()
    wd = torch.tensor(wk).to(torch.bfloat16).cuda()
    bd = torch.tensor(b).cuda()
    out = torch.empty((n, h, w, co), dtype=torch.bfloat16, device="cuda")
    tv.lib().tvcut_conv3x3_bf16(xd.data_ptr(), wd.data_ptr(), bd.data_ptr(), out.data_ptr(), n, h, w, ci, co, 1, None)
    torch.cuda.synchronize()
    ref, S = conv_ref_and_scale(x, wk, b)
    assert_conv_bound(out.float().cpu().numpy(), ref, S, relu=True)
    # weight gradient of sum(conv(x) * g) for a random g: dW[t][o][i] = sum_p g[p][o] x[p + tap t][i]
    g = bf16_round(rng.normal(size=(n, h, w, co)))
    xt = torch.tensor(x, dtype=torch.float64).permute(0, 3, 1, 2)
    gt = torch.tensor(g, dtype=torch.float64).permute(0, 3, 1, 2)
    wshape = (co, ci, 3, 3)
    ref_w = torch.nn.grad.conv2d_weight(xt, wshape, gt, padding=1)
    S_w = torch.nn.grad.conv2d_weight(xt.abs(), wshape, gt.abs(), padding=1)
    to_lib = lambda t: t.permute(2, 3, 0, 1).reshape(9, co, ci).numpy()   # [Cout][Cin][ky][kx] -> [tap][Cout][Cin]
    dw = torch.zeros((9, co, ci), dtype=torch.float32, device="cuda")
    gd = torch.tensor(g).to(torch.bfloat16).cuda()
    tv.lib().tvcut_conv3x3_wgrad_bf16(xd.data_ptr(), gd.data_ptr(), dw.data_ptr(), n, h, w, ci, co, None)
    torch.cuda.synchronize()
    d = np.abs(dw.cpu().numpy().astype(np.float64) - to_lib(ref_w))
    assert np.all(d <= 2 ** -12 * to_lib(S_w)), float((d / (2 ** -12 * to_lib(S_w) + 1e-300)).max())


TC_SHAPES = [(1, 16, 128, 16, 32), (2, 16, 64, 32, 16), (1, 8, 256, 64, 128), (1, 4, 128, 128, 256),
             (1, 16, 32, 256, 64), (3, 2, 128, 16, 16), (1, 64, 16, 64, 48),
             # halo strips: heights that are not a multiple of the strip, several images, 64 input channels
             (2, 7, 128, 64, 32), (1, 5, 256, 32, 64), (3, 1, 128, 32, 32)]


@pytest.mark.parametrize("shape", TC_SHAPES)
@pytest.mark.parametrize("relu", [0, 1])
def test_conv_tcgen05(tv, shape, relu):
    """The tcgen05 kernel (engine 2) against the CPU reference and against the
    mma.sync kernel (engine 1): same BF16 inputs, FP32 accumulation in a
    different order, so the BF16 outputs differ by rounding only."""
    n, h, w, ci, co = shape
    rng = np.random.default_rng(sum(shape) + relu)
    x = bf16_round(rng.normal(size=(n, h, w, ci)))
    wk = bf16_round(rng.normal(size=(9, co, ci)) * (0.6 / np.sqrt(ci)))
    b = rng.normal(size=co).astype(np.float32)
    xd = torch.tensor(x).to(torch.bfloat16).cuda()
    wd = torch.tensor(wk).to(torch.bfloat16).cuda()
    bd = torch.tensor(b).cuda()
    outs = []
    for engine in (2, 1, 3, 4):
        out = torch.full((n, h, w, co), 7.0, dtype=torch.bfloat16, device="cuda")
        code = tv.lib().tvcut_conv3x3_bf16_ex(xd.data_ptr(), wd.data_ptr(), bd.data_ptr(), out.data_ptr(),
                                              n, h, w, ci, co, relu, engine, None)
        assert code == tv.OK
        torch.cuda.synchronize()
        outs.append(out.float().cpu().numpy())
    assert tv.lib().tvcut_conv_tc_error() == 0
    # the persistent (halo or not) and the one-tile-per-CTA forms run the same
    # MMAs in the same order
    np.testing.assert_array_equal(outs[0], outs[2])
    np.testing.assert_array_equal(outs[3], outs[2])
    ref, S = conv_ref_and_scale(x, wk, b)
    assert_conv_bound(outs[0], ref, S, relu=bool(relu))
    assert_conv_bound(outs[1], ref, S, relu=bool(relu))
    # rounding only: no output differs by more than a few BF16 steps of its magnitude
    assert np.all(np.abs(outs[0] - outs[1]) <= 2 ** -6 * np.maximum(np.abs(outs[1]), 1.0))


@pytest.mark.parametrize("shape", [(1, 512, 512, 16, 32), (2, 256, 256, 64, 256), (4, 64, 128, 32, 64),
                                   (1, 1024, 64, 128, 128), (3, 96, 256, 256, 16), (1, 256, 256, 64, 32),
                                   (2, 64, 384, 32, 48), (1, 128, 128, 16, 16),
                                   (2, 131, 256, 64, 32), (3, 37, 384, 32, 32), (1, 258, 128, 16, 32),
                                   (2, 2, 512, 32, 16)])
def test_conv_tcgen05_persistent_many_tiles(tv, shape):
    """Shapes with several tiles per persistent CTA, so that both tensor-memory
    accumulator buffers and the stage or halo ring are reused many times: the
    persistent forms (engine 2, with the halo-loaded operand where the shape
    allows; engine 4 without it) equal the one-tile-per-CTA form (engine 3)
    bit for bit and the mma.sync kernel (engine 1) up to rounding."""
    n, h, w, ci, co = shape
    g = torch.Generator(device="cuda").manual_seed(sum(shape))
    xd = torch.randn((n, h, w, ci), generator=g, device="cuda").to(torch.bfloat16)
    wd = (torch.randn((9, co, ci), generator=g, device="cuda") * (0.6 / ci ** 0.5)).to(torch.bfloat16)
    bd = torch.randn((co,), generator=g, device="cuda")
    outs = []
    for engine in (2, 3, 1, 4):
        out = torch.full((n, h, w, co), 7.0, dtype=torch.bfloat16, device="cuda")
        code = tv.lib().tvcut_conv3x3_bf16_ex(xd.data_ptr(), wd.data_ptr(), bd.data_ptr(), out.data_ptr(),
                                              n, h, w, ci, co, 1, engine, None)
        assert code == tv.OK
        torch.cuda.synchronize()
        outs.append(out.float())
    assert tv.lib().tvcut_conv_tc_error() == 0
    assert torch.equal(outs[0], outs[1])
    assert torch.equal(outs[3], outs[1])
    d = (outs[0] - outs[2]).abs()
    assert bool((d <= 2 ** -6 * torch.clamp(outs[2].abs(), min=1.0)).all())


@pytest.mark.parametrize("engine,shape", [(2, (1, 16, 128, 16, 32)), (4, (1, 16, 128, 16, 32)),
                                          (3, (1, 16, 128, 16, 32)), (2, (1, 8, 256, 64, 128))])
def test_conv_tcgen05_bounded_wait_gives_up(tv, engine, shape):
    """The stall hook makes CTA 0 skip its first operand load: the MMA
    issuer's bounded wait gives up (2 s), the launch ends by itself, the
    error flag reads 1 once and is cleared, and the context stays usable:
    the next launch without the hook is complete and correct."""
    n, h, w, ci, co = shape
    g = torch.Generator(device="cuda").manual_seed(11)
    xd = torch.randn((n, h, w, ci), generator=g, device="cuda").to(torch.bfloat16)
    wd = (torch.randn((9, co, ci), generator=g, device="cuda") * 0.2).to(torch.bfloat16)
    out = torch.zeros((n, h, w, co), dtype=torch.bfloat16, device="cuda")
    ref = torch.zeros_like(out)
    assert tv.lib().tvcut_conv3x3_bf16_ex(xd.data_ptr(), wd.data_ptr(), None, ref.data_ptr(), n, h, w, ci, co, 0, 1,
                                          None) == tv.OK
    assert tv.lib().tvcut_conv_tc_error() == 0
    try:
        assert tv.lib().tvcut_conv_tc_stall(1) == tv.OK
        assert tv.lib().tvcut_conv3x3_bf16_ex(xd.data_ptr(), wd.data_ptr(), None, out.data_ptr(), n, h, w, ci, co, 0,
                                              engine, None) == tv.OK
        torch.cuda.synchronize()
        assert tv.lib().tvcut_conv_tc_error() == 1
        assert tv.lib().tvcut_conv_tc_error() == 0
    finally:
        assert tv.lib().tvcut_conv_tc_stall(0) == tv.OK
    out.zero_()
    assert tv.lib().tvcut_conv3x3_bf16_ex(xd.data_ptr(), wd.data_ptr(), None, out.data_ptr(), n, h, w, ci, co, 0,
                                          engine, None) == tv.OK
    torch.cuda.synchronize()
    assert tv.lib().tvcut_conv_tc_error() == 0
    d = (out.float() - ref.float()).abs()
    assert bool((d <= 2 ** -6 * torch.clamp(ref.float().abs(), min=1.0)).all())


def test_conv_tcgen05_rejects_other_shapes(tv):
    x = torch.zeros((2, 9, 13, 32), dtype=torch.bfloat16, device="cuda")
    wk = torch.zeros((9, 16, 32), dtype=torch.bfloat16, device="cuda")
    out = torch.zeros((2, 9, 13, 16), dtype=torch.bfloat16, device="cuda")
    code = tv.lib().tvcut_conv3x3_bf16_ex(x.data_ptr(), wk.data_ptr(), None, out.data_ptr(), 2, 9, 13, 32, 16, 0, 2,
                                          None)
    assert code == tv.ERR_INVALID
    # engine 0 takes the mma.sync kernel for it
    code = tv.lib().tvcut_conv3x3_bf16_ex(x.data_ptr(), wk.data_ptr(), None, out.data_ptr(), 2, 9, 13, 32, 16, 0, 0,
                                          None)
    assert code == tv.OK


def net_vs_oracle(tv, net, base, x, t, engine):
    """GPU forward output, loss and parameter gradient of one engine, with
    the BF16-storage oracle's on the GPU's own parameters."""
    from oracle import unet_ref
    net.set_engine(engine)
    out = net.forward(torch.tensor(x).cuda()).cpu().numpy()
    loss = net.backward(torch.tensor(t).cuda())
    grad = net.params(which=1)
    th = bf16_weights_f32_bias(net.params(), base)
    ref_loss, ref_grad, ref_out = unet_ref.loss_and_grad(th, bf16_round(x), t, base, torch.float64, bf16_storage=True)
    return out, loss, grad, ref_out, ref_loss, ref_grad


def assert_forward_bound(out, ref_out):
    scale = np.abs(ref_out).mean()
    r = np.abs(out - ref_out) / (2 ** -8 * (np.abs(ref_out) + scale))
    assert r.max() <= 8.0, float(r.max())


def assert_gradient_bound(grad, ref_grad, base):
    for li, sl in enumerate(layer_slices(base)):
        g, ref = grad[sl], ref_grad[sl]
        rms = np.sqrt(np.mean(ref ** 2))
        r = np.abs(g - ref) / (2 ** -8 * (np.abs(ref) + rms))
        assert r.max() <= 48.0, (li, float(r.max()))


def test_network_engines_agree(tv):
    """128 x 128 images: every layer's shape goes to the tcgen05 kernel
    (engine 0); the one-tile-per-CTA tcgen05 form (engine 3) gives the same
    forward pass bit for bit, and every engine (also the mma.sync kernels,
    engine 1) meets the element-wise bounds against the oracle."""
    base, n, h, w = 32, 2, 128, 128
    net = tv.UNet(base=base, batch=n, H=h, W=w, seed=5)
    rng = np.random.default_rng(6)
    x = rng.normal(size=(n, h, w, 3)).astype(np.float32)
    t = rng.normal(size=(n, h, w, 2)).astype(np.float32)
    res = {}
    for engine in (0, 1, 3):
        out, loss, grad, ref_out, ref_loss, ref_grad = net_vs_oracle(tv, net, base, x, t, engine)
        res[engine] = out
        assert_forward_bound(out, ref_out)
        assert abs(loss - ref_loss) <= 1e-3 * ref_loss
        assert_gradient_bound(grad, ref_grad, base)
    assert tv.lib().tvcut_conv_tc_error() == 0
    np.testing.assert_array_equal(res[0], res[3])
    net.close()


def test_network_forward_backward(tv):
    """A small, non-square image (levels down to 4 x 3 pixels): forward pass
    and loss element by element; gradients of layers this small are sums
    over a handful of pixels, so only their direction is compared here (the
    element-wise gradient bounds are checked on 128 x 128 inputs above)."""
    from oracle import unet_ref
    base, n, h, w = 32, 2, 32, 24
    net = tv.UNet(base=base, batch=n, H=h, W=w, seed=7)
    assert net.params().size == unet_ref.num_params(base)
    rng = np.random.default_rng(3)
    x = rng.normal(size=(n, h, w, 3)).astype(np.float32)
    t = rng.normal(size=(n, h, w, 2)).astype(np.float32)
    out, loss, grad, ref_out, ref_loss, ref_grad = net_vs_oracle(tv, net, base, x, t, 0)
    assert_forward_bound(out, ref_out)
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    for li, sl in enumerate(layer_slices(base)):
        gl, rl = grad[sl], ref_grad[sl]
        cos = float(gl @ rl / (np.linalg.norm(gl) * np.linalg.norm(rl) + 1e-30))
        assert cos > 0.98, (li, cos)
    net.close()


def test_backward_and_training_are_deterministic(tv):
    """Equal inputs give equal gradients bit for bit (the reductions sum
    their partials in a fixed order), and a few Adam steps from the same seed
    give equal parameters, at a shape whose layers split the weight gradient
    into many pixel chunks."""
    rng = np.random.default_rng(9)
    x = torch.tensor(rng.normal(size=(4, 64, 64, 3)).astype(np.float32)).cuda()
    t = torch.tensor(rng.normal(size=(4, 64, 64, 2)).astype(np.float32)).cuda()
    runs = []
    for rep in range(2):
        net = tv.UNet(base=32, batch=4, H=64, W=64, seed=13)
        losses = []
        for step in range(3):
            net.forward(x)
            losses.append(net.backward(t))
            if step == 0:
                g0 = net.params(which=1)
            net.adam(lr=1e-3)
        runs.append((g0, losses, net.params()))
        net.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1]
    np.testing.assert_array_equal(runs[0][2], runs[1][2])


def test_training_reduces_loss(tv):
    net = tv.UNet(base=32, batch=4, H=32, W=32, seed=11)
    rng = np.random.default_rng(4)
    x = torch.tensor(rng.normal(size=(4, 32, 32, 3)).astype(np.float32)).cuda()
    # a smooth, learnable target: local averages of the input channels
    xt = x.permute(0, 3, 1, 2)
    t = torch.nn.functional.avg_pool2d(xt[:, :2], 3, stride=1, padding=1).permute(0, 2, 3, 1).contiguous()
    losses = []
    for _ in range(150):
        net.forward(x)
        losses.append(net.backward(t))
        net.adam(lr=2e-3)
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])
    net.close()


def test_params_roundtrip(tv):
    net = tv.UNet(base=16, batch=1, H=16, W=16, seed=1)
    p = net.params()
    net.set_params(p * 0.5)
    np.testing.assert_array_equal(net.params(), (p * 0.5).astype(np.float32))
    net.close()
