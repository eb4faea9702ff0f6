"""What the learned warm start gains: a U-Net trained on the GPU for a few
seconds on solver-generated problems predicts the per-block duals of a
held-out problem; the solver started there reaches the oracle's exact
min-cut in fewer iterations than the cold-started method (Sec. 4.4 warm
starts reuse dual variables; here they are predicted)."""
import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tv():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01563_gb300 import tvcut
    tvcut.lib()
    return tvcut


def iters_to_cut(tv, s, e_star, net=None, cap=3000):
    if net is None:
        s.reset()
    else:
        net.predict_state(s)
    for k in range(1, cap + 1):
        _, st = s.iterate(1)
        if st.energy_i64 == e_star:
            return k
    return cap + 1


def test_targets_are_block_duals(tv, orc):
    """The training targets are the shadow y_k of a (nearly) converged state:
    y_0 + y_1 = w - x* (Sec. 2.3) with x* the TV solution."""
    from paper_1503_01563_gb300 import learn
    probs = [inputs.uniform_grid((24, 32), 5)]
    y = learn.solve_targets(probs, 2000, dtype=tv.F64)[0].cpu().numpy()
    w, a = probs[0]
    _, x = orc.iterate(0, w, a, orc.cold_state(0, w), 3000)
    np.testing.assert_allclose(y.sum(0), w - x, atol=1e-6)


def test_learned_warm_start_saves_iterations(tv, orc):
    from paper_1503_01563_gb300 import learn
    X, Y = learn.make_training_set(1024, 64, 64, seed=21, iters=600)
    net = tv.UNet(base=32, batch=16, H=64, W=64, seed=5)
    hist = learn.train(net, X, Y, steps=500, batch=16)
    assert np.mean(hist[-20:]) < 0.5 * hist[0]
    w, a = inputs.uniform_grid((256, 256), 777)           # held out
    e_star = orc.maxflow(w, a)[1]
    s = tv.Solver((256, 256), dtype=tv.F32, check_every=1)
    s.set_problem(torch.from_numpy(w).cuda(), [torch.from_numpy(x).cuda() for x in a])
    cold = iters_to_cut(tv, s, e_star)
    warm = iters_to_cut(tv, s, e_star, net)
    print(f"iterations to the exact min-cut: cold {cold}, learned warm start {warm}")
    assert warm <= 0.85 * cold, (cold, warm)
    lab, st = s.cut()
    assert st.energy_i64 == e_star and orc.energy(w, a, lab) == e_star
    net.close()
    s.close()


@pytest.mark.parametrize("dims,algo", [((64, 96), 0), ((128, 40), 3), ((48, 48), 2)])
def test_device_prediction_equals_host_features_path(tv, dims, algo):
    """tvcut_unet_predict_state (features from the solver's device inputs,
    forward pass, rescaling into the state's layouts) equals, bit for bit,
    the same steps taken outside the library: host features, the FP32-input
    forward pass, the FP32 rescaling and tvcut_set_state."""
    from paper_1503_01563_gb300 import learn
    w, a = inputs.uniform_grid(dims, 31)
    net = tv.UNet(base=32, batch=1, H=dims[0], W=dims[1], seed=9)
    s = tv.Solver(dims, algo=algo, dtype=tv.F32)
    s.set_problem(torch.from_numpy(w).cuda(), [torch.from_numpy(x).cuda() for x in a])
    net.predict_state(s)
    got = s.state()
    f, sc = learn.features(w, a)
    out = net.forward(torch.from_numpy(f[None]).cuda())
    want = (out[0].permute(2, 0, 1) * sc).contiguous().cpu().numpy()
    np.testing.assert_array_equal(got, want)
    assert np.abs(want).max() > 0
    # a handle on another stream: the prediction is ordered after its inputs
    st = torch.cuda.Stream()
    s2 = tv.Solver(dims, algo=algo, dtype=tv.F32, stream=st.cuda_stream)
    s2.set_problem(torch.from_numpy(w).cuda(), [torch.from_numpy(x).cuda() for x in a])
    net.predict_state(s2)
    np.testing.assert_array_equal(s2.state(), want)
    s.close()
    s2.close()
    net.close()


def test_device_prediction_fp64_handle(tv):
    """An FP64 solver gets the same prediction as an FP32 one, widened: the
    features are the same FP32 values and the rescaled output is an FP32
    product in both."""
    w, a = inputs.uniform_grid((64, 40), 33)
    net = tv.UNet(base=32, batch=1, H=64, W=40, seed=4)
    got = []
    for dt in (tv.F32, tv.F64):
        s = tv.Solver((64, 40), dtype=dt)
        s.set_problem(w, a)
        net.predict_state(s)
        got.append(s.state())
        s.close()
    np.testing.assert_array_equal(got[0].astype(np.float64), got[1])
    net.close()


def test_predict_state_rejects_other_grids(tv):
    net = tv.UNet(base=16, batch=1, H=16, W=16, seed=1)
    s3 = tv.Solver((8, 8, 8), dtype=tv.F32)
    w, a = inputs.uniform_grid((8, 8, 8), 1)
    s3.set_problem(w, a)
    with pytest.raises(tv.TvcutError) as e:
        net.predict_state(s3)
    assert e.value.code == tv.ERR_INVALID
    s2 = tv.Solver((12, 16), dtype=tv.F32)
    with pytest.raises(tv.TvcutError) as e:
        net.predict_state(s2)                            # inputs not set
    assert e.value.code == tv.ERR_STATE
    w, a = inputs.uniform_grid((12, 16), 1)
    s2.set_problem(w, a)
    with pytest.raises(tv.TvcutError) as e:
        net.predict_state(s2)                            # 12 is not a multiple of 8
    assert e.value.code == tv.ERR_INVALID
    s2.close()
    s3.close()
    net.close()
