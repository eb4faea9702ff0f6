"""Warm start across a sequence of similar problems (Sec. 4.4: reuse the
dual variables of the previous problem; Fig. 3b: frames of a video), and
host-side failure handling that faults nothing on the device."""
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


def frames(n, dims=(256, 256), seed=3):
    """A drifting blob image: frame t is the base image shifted by t pixels
    plus fresh small noise; segmentation energies scaled to integers."""
    g = np.random.default_rng(seed)
    base = inputs.blob_image((dims[0], dims[1] + n), seed, noise=0.0)
    out = []
    for t in range(n):
        img = np.clip(base[:, t:t + dims[1]] + g.normal(0, 0.03, size=dims), 0, 1)
        w, a = inputs.segmentation_terms(img)
        out.append(inputs.to_integer(w, a))
    return out


def iters_to(tv, s, e_star, cap=4000):
    for k in range(1, cap + 1):
        _, st = s.iterate(1)
        if st.energy_i64 == e_star:
            return k
    return cap + 1


def test_sequence_warm_start(tv, orc):
    seq = frames(4)
    s = tv.Solver(seq[0][0].shape, dtype=tv.F32, check_every=1)
    prev = None
    cold_total = warm_total = 0
    for t, (w, a) in enumerate(seq):
        e_star = orc.maxflow(w, a)[1]
        s.set_problem(w, a)                      # resets to a cold start
        cold = iters_to(tv, s, e_star)
        if prev is not None:
            s.set_state(prev)                    # start from the previous frame's dual variables
            warm = iters_to(tv, s, e_star)
            cold_total += cold
            warm_total += warm
            lab, st = s.cut()
            assert st.energy_i64 == e_star and orc.energy(w, a, lab) == e_star
        prev = s.dual()
    print(f"frames 1-3: cold {cold_total} iterations, warm from previous frame {warm_total}")
    assert warm_total < cold_total


def test_dual_is_shadow(tv, orc):
    """get_dual = per-block projection of the state (oracle project_block)."""
    for dims in [(20, 24), (9, 10, 11)]:
        w, a = inputs.uniform_grid(dims, 3)
        s = tv.Solver(dims, dtype=tv.F64, check_every=1000)
        s.set_problem(w, a)
        s.iterate(7)
        z, y = s.state(), s.dual()
        for k in range(len(dims)):
            np.testing.assert_allclose(y[k], orc.project_block(z[k], a[k], k), atol=1e-9 * max(1, np.abs(z).max()))
        s.close()


def test_allocation_failure_is_reported(tv):
    with pytest.raises(tv.TvcutError) as e:
        tv.Solver((1 << 20, 1 << 19))            # 2^39 vertices: the allocation fails
    assert e.value.code in (tv.ERR_OOM, tv.ERR_CUDA)
    s = tv.Solver((8, 8))                        # the context is still usable
    w, a = inputs.uniform_grid((8, 8), 1)
    s.set_problem(w, a)
    s.iterate(3)
    s.close()
