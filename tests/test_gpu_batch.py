"""Batched grids (tvcut_batch_*): every grid of a batch of uneven 2D grids
must evolve exactly like the same grid solved alone, agree with the FP64
oracle, and reach its exact min-cut (problem (D), Sec. 2.3)."""
import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS = [(37, 53), (64, 64), (5, 40), (1, 17), (23, 1), (2, 2), (130, 70), (64, 300)]


@pytest.fixture(scope="module")
def tv():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01563_gb300 import tvcut
    tvcut.lib()
    return tvcut


def problems(seed0=100):
    return [inputs.uniform_grid(d, seed0 + i) for i, d in enumerate(DIMS)]


@pytest.mark.parametrize("algo", [0, 1, 3])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_matches_single_grid_and_oracle(tv, orc, algo, dtype):
    code = tv.F64 if dtype == "f64" else tv.F32
    probs = problems()
    b = tv.Batch(DIMS, algo=algo, dtype=code)
    for g, (w, a) in enumerate(probs):
        b.set_problem(g, w, a)
    b.reset()
    b.iterate(9)
    b.iterate(8)                  # graph for another count; state carries over
    for g, (w, a) in enumerate(probs):
        s = tv.Solver(DIMS[g], algo=algo, dtype=code, check_every=10 ** 6)
        s.set_problem(w, a)
        s.iterate(17)
        np.testing.assert_array_equal(b.state(g), s.state())       # same kernels, same arithmetic
        ref, _ = orc.iterate(algo, w, a, orc.cold_state(algo, w), 17)
        tol = 1e-9 if dtype == "f64" else 1e-4
        assert np.abs(b.state(g) - ref).max() <= tol * max(1.0, np.abs(ref).max())
        s.close()
    b.close()


@pytest.mark.parametrize("algo", [0, 3])
def test_batch_exact_cuts(tv, orc, algo):
    probs = problems(200)
    b = tv.Batch(DIMS, algo=algo, dtype=tv.F64)
    for g, (w, a) in enumerate(probs):
        b.set_problem(g, w, a)
    b.reset()
    code, stats = b.iterate(1500)
    for g, (w, a) in enumerate(probs):
        e_star = orc.maxflow(w, a)[1]
        lab, st = b.cut(g)
        assert st.energy_i64 == e_star, g
        assert orc.energy(w, a, lab) == e_star
    assert code == tv.OK
    b.close()


@pytest.mark.parametrize("algo", [0, 3])
def test_batch_graph_replay_deterministic(tv, orc, algo):
    """Replays of one captured graph (3 x 4 iterations) give identical results
    run to run; for FISTA, 3 x 3 iterations (an odd count alternates the roles
    of the two iterate buffers between calls) match the oracle's 9 steps."""
    probs = problems(300)
    runs = []
    for _ in range(2):
        b = tv.Batch(DIMS, algo=algo, dtype=tv.F32)
        for g, (w, a) in enumerate(probs):
            b.set_problem(g, w, a)
        b.reset()
        for _ in range(3):
            code, st = b.iterate(4)    # replays one captured graph
        runs.append(([b.state(g) for g in range(len(DIMS))], [s.energy_i64 for s in st]))
        b.close()
    for s1, s2 in zip(runs[0][0], runs[1][0]):
        np.testing.assert_array_equal(s1, s2)
    assert runs[0][1] == runs[1][1]
    if algo == 3:
        b = tv.Batch(DIMS, algo=algo, dtype=tv.F32)
        for g, (w, a) in enumerate(probs):
            b.set_problem(g, w, a)
        b.reset()
        for _ in range(3):
            b.iterate(3)
        for g, (w, a) in enumerate(probs):
            ref, _ = orc.iterate(3, w, a, orc.cold_state(3, w), 9)
            assert np.abs(b.state(g) - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())
        b.close()


def test_batch_autotune_keeps_results(tv):
    probs = problems(400)
    b = tv.Batch(DIMS, dtype=tv.F32)
    for g, (w, a) in enumerate(probs):
        b.set_problem(g, w, a)
    b.reset()
    b.iterate(5)
    before = [b.state(g) for g in range(len(DIMS))]
    threads, per_sm, pred = b.autotune()
    assert threads in (64, 128, 256) and per_sm in (4, 8, 16) and pred in (0, 1, 2)
    b.reset()
    b.iterate(5)
    for g in range(len(DIMS)):
        np.testing.assert_array_equal(b.state(g), before[g])


@pytest.mark.parametrize("algo", [0, 1, 3])
def test_batch_step_forms_agree(tv, orc, algo):
    """The three forms of the scan step (branchy, predicated, padded weights
    loaded a step ahead) give bit-identical iterates, within 1e-4 of the
    FP64 oracle, for AAR, AP and FISTA (whose projection scan takes the
    branchy step for form 2)."""
    probs = problems(401)
    out = []
    for step in (0, 1, 2):
        b = tv.Batch(DIMS, algo=algo, dtype=tv.F32)
        for g, (w, a) in enumerate(probs):
            b.set_problem(g, w, a)
        b.set_launch(128, 8, step)
        b.reset()
        b.iterate(7)
        out.append([b.state(g) for g in range(len(DIMS))])
        b.close()
    for g in range(len(DIMS)):
        np.testing.assert_array_equal(out[1][g], out[0][g])
        np.testing.assert_array_equal(out[2][g], out[0][g])
    for g in (0, len(DIMS) - 1):
        w, a = probs[g]
        ref, _ = orc.iterate(algo, w, a, orc.cold_state(algo, w), 7)
        assert np.abs(out[2][g] - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


def test_batch_set_launch_rejects(tv):
    b = tv.Batch([(4, 4), (3, 5)])
    for bad in ((96, 8, 0), (128, 0, 0), (128, 33, 0), (128, 8, 3), (128, 8, -1)):
        with pytest.raises(tv.TvcutError):
            b.set_launch(*bad)
    b.close()


def test_batch_errors(tv):
    with pytest.raises(tv.TvcutError):
        tv.Batch([(0, 5)])
    with pytest.raises(tv.TvcutError):
        tv.Batch([(4, 4)], algo=2)                # BCD is single-grid only
    b = tv.Batch([(4, 4), (3, 5)])
    w, a = inputs.uniform_grid((4, 4), 1)
    b.set_problem(0, w, a)
    with pytest.raises(tv.TvcutError) as e:
        b.iterate(2)
    assert e.value.code == tv.ERR_STATE
    bad = [x.copy() for x in inputs.uniform_grid((3, 5), 2)[1]]
    bad[1][0, 0] = -3
    with pytest.raises(tv.TvcutError) as e:
        b.set_problem(1, inputs.uniform_grid((3, 5), 2)[0], bad)
    assert e.value.code == tv.ERR_INVALID
    b.close()
