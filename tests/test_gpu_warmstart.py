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


def iters_to_cut(tv, s, e_star, z0=None, cap=3000):
    if z0 is None:
        s.reset()
    else:
        tv.tvcut_set_state(s.h, z0)
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
    warm = iters_to_cut(tv, s, e_star, learn.predict_state(net, w, a))
    print(f"iterations to the exact min-cut: cold {cold}, learned warm start {warm}")
    assert warm <= 0.85 * cold, (cold, warm)
    lab, st = s.cut()
    assert st.energy_i64 == e_star and orc.energy(w, a, lab) == e_star
    net.close()
    s.close()
