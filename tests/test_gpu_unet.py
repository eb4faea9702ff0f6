"""Warm-start network kernels against the CPU oracle (oracle/unet_ref.py,
PyTorch CPU FP32).  The GPU computes with BF16 weights and activations and
FP32 accumulation, so results are compared by relative L2 error: 2e-2 for a
single convolution, 5e-2 for the 18-layer forward pass, 1e-1 for parameter
gradients (BF16 activation gradients through 18 layers)."""
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


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def bf16_round(x):
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("shape", [(1, 16, 16, 16, 32), (2, 9, 13, 32, 16), (1, 8, 8, 64, 128)])
def test_conv_forward_and_wgrad(tv, shape):
    from oracle import unet_ref
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
    W = torch.tensor(wk, requires_grad=True)
    Wt = W.reshape(3, 3, co, ci).permute(2, 3, 0, 1)
    xt = torch.tensor(x).permute(0, 3, 1, 2)
    ref = torch.relu(unet_ref.F.conv2d(xt, Wt, torch.tensor(b), padding=1)).permute(0, 2, 3, 1)
    assert rel(out.float().cpu().numpy(), ref.detach().numpy()) < 2e-2
    # weight gradient of sum(ref * g) for a random g (before the ReLU: use the linear conv)
    g = bf16_round(rng.normal(size=(n, h, w, co)))
    lin = unet_ref.F.conv2d(xt, Wt, None, padding=1).permute(0, 2, 3, 1)
    (lin * torch.tensor(g)).sum().backward()
    dw = torch.zeros((9, co, ci), dtype=torch.float32, device="cuda")
    gd = torch.tensor(g).to(torch.bfloat16).cuda()
    tv.lib().tvcut_conv3x3_wgrad_bf16(xd.data_ptr(), gd.data_ptr(), dw.data_ptr(), n, h, w, ci, co, None)
    torch.cuda.synchronize()
    assert rel(dw.cpu().numpy(), W.grad.numpy()) < 2e-2


TC_SHAPES = [(1, 16, 128, 16, 32), (2, 16, 64, 32, 16), (1, 8, 256, 64, 128), (1, 4, 128, 128, 256),
             (1, 16, 32, 256, 64), (3, 2, 128, 16, 16), (1, 64, 16, 64, 48)]


@pytest.mark.parametrize("shape", TC_SHAPES)
@pytest.mark.parametrize("relu", [0, 1])
def test_conv_tcgen05(tv, shape, relu):
    """The tcgen05 kernel (engine 2) against the CPU reference and against the
    mma.sync kernel (engine 1): same BF16 inputs, FP32 accumulation in a
    different order, so the BF16 outputs differ by rounding only."""
    from oracle import unet_ref
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
    Wt = torch.tensor(wk).reshape(3, 3, co, ci).permute(2, 3, 0, 1)
    xt = torch.tensor(x).permute(0, 3, 1, 2)
    ref = unet_ref.F.conv2d(xt, Wt, torch.tensor(b), padding=1).permute(0, 2, 3, 1)
    if relu:
        ref = torch.relu(ref)
    ref = ref.numpy()
    assert rel(outs[0], ref) < 1e-2
    assert rel(outs[0], outs[1]) < 1e-2
    # rounding only: no output differs by more than a few BF16 steps of its magnitude
    assert np.all(np.abs(outs[0] - outs[1]) <= 2 ** -6 * np.maximum(np.abs(outs[1]), 1.0))


@pytest.mark.parametrize("shape", [(1, 512, 512, 16, 32), (2, 256, 256, 64, 256), (4, 64, 128, 32, 64),
                                   (1, 1024, 64, 128, 128), (3, 96, 256, 256, 16), (1, 256, 256, 64, 32),
                                   (2, 64, 384, 32, 48), (1, 128, 128, 16, 16)])
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


def test_network_engines_agree(tv):
    """128 x 128 images: every layer's shape goes to the tcgen05 kernel
    (engine 0); the same network on the mma.sync kernels (engine 1) and the
    CPU oracle agree with it."""
    from oracle import unet_ref
    base, n, h, w = 32, 2, 128, 128
    net = tv.UNet(base=base, batch=n, H=h, W=w, seed=5)
    rng = np.random.default_rng(6)
    x = torch.tensor(rng.normal(size=(n, h, w, 3)).astype(np.float32)).cuda()
    t = torch.tensor(rng.normal(size=(n, h, w, 2)).astype(np.float32)).cuda()
    res = []
    for engine in (0, 1, 3):
        net.set_engine(engine)
        out = net.forward(x).cpu().numpy()
        loss = net.backward(t)
        res.append((out, loss, net.params(which=1)))
    assert tv.lib().tvcut_conv_tc_error() == 0
    np.testing.assert_array_equal(res[0][0], res[2][0])
    # the weight gradient's kernel accumulates with atomics: equal up to summation order
    assert rel(res[0][2], res[2][2]) < 1e-5
    assert rel(res[0][0], res[1][0]) < 1e-2
    assert abs(res[0][1] - res[1][1]) < 1e-2 * res[1][1]
    assert rel(res[0][2], res[1][2]) < 5e-2
    theta_bf = bf16_round(net.params())
    ref_loss, _, ref_out = unet_ref.loss_and_grad(theta_bf, bf16_round(x.cpu().numpy()), t.cpu().numpy(), base)
    assert rel(res[0][0], ref_out) < 5e-2
    net.close()


def test_network_forward_backward(tv):
    from oracle import unet_ref
    base, n, h, w = 32, 2, 32, 24
    net = tv.UNet(base=base, batch=n, H=h, W=w, seed=7)
    theta = net.params()
    assert theta.size == unet_ref.num_params(base)
    rng = np.random.default_rng(3)
    x = rng.normal(size=(n, h, w, 3)).astype(np.float32)
    t = rng.normal(size=(n, h, w, 2)).astype(np.float32)
    out = net.forward(torch.tensor(x).cuda())
    loss = net.backward(torch.tensor(t).cuda())
    grad = net.params(which=1)
    theta_bf = bf16_round(theta)                 # the forward pass uses BF16 weights
    ref_loss, ref_grad, ref_out = unet_ref.loss_and_grad(theta_bf, bf16_round(x), t, base)
    assert rel(out.cpu().numpy(), ref_out) < 5e-2
    assert abs(loss - ref_loss) < 5e-2 * ref_loss
    assert rel(grad, ref_grad) < 1e-1
    # per-layer gradient direction
    off = 0
    for ci, co in unet_ref.layer_shapes(base):
        k = 9 * ci * co + co
        gl, rl = grad[off:off + k], ref_grad[off:off + k]
        cos = float(gl @ rl / (np.linalg.norm(gl) * np.linalg.norm(rl) + 1e-30))
        assert cos > 0.98, (ci, co, cos)
        off += k
    net.close()


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
