"""The lane-group scan with the funnel form of the taut string (Sec. 3.2;
mapping 11) against the oracle: one iteration from given states, FP64 within
1e-9 and FP32 within 1e-4 of max|x|; integer states with exact ties and zero
weights; chains whose hull outgrows a lane's ring (the local-form fallback);
the projection-mode methods (BCD, FISTA); the 2D segmentation at full size
to the benchmark's iteration count, and the 2048^2 problem's 2048-element
chains.  The zig-zag blocks of an 8-connected grid are covered in
test_gpu_conn8.py."""
import os

import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FUNNEL = 11


@pytest.fixture(scope="module")
def tv():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01563_gb300 import tvcut
    tvcut.lib()
    return tvcut


def rel_err(got, want):
    return float(np.abs(np.asarray(got, np.float64) - want).max() / max(1.0, np.abs(want).max()))


def random_state(dims, nblk, seed, integer=False):
    g = np.random.default_rng(seed)
    s = np.empty((nblk,) + tuple(dims))
    for k in range(nblk):
        base = g.normal(0, 30, size=dims) + np.cumsum(g.integers(-1, 2, size=dims) * 20.0, axis=k % len(dims))
        s[k] = np.round(base) if integer else base
    return s


# chain lengths 1 .. 4099: every lane count (4 .. 32), ragged last pieces
STATE_CASES = [(64, 64), (37, 53), (1, 9), (9, 1), (2, 2), (1, 2048), (3, 2049), (2, 4099), (13, 17, 19),
               (1, 5, 6), (40, 3, 70), (300, 7)]


@pytest.mark.parametrize("dims", STATE_CASES)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("algo", [0, 1])
def test_one_iteration_from_random_states(tv, orc, dims, dtype, algo):
    w, a = inputs.uniform_grid(dims, 23)
    st = random_state(dims, len(dims), 24)
    code = tv.F64 if dtype == "f64" else tv.F32
    tol = 1e-9 if dtype == "f64" else 1e-4
    s = tv.Solver(dims, algo=algo, dtype=code, check_every=1000, mapping=FUNNEL)
    s.set_problem(w, a)
    s.set_state(st)
    s.iterate(1)
    ref_s, ref_x = orc.iterate(algo, w, a, st, 1)
    assert rel_err(s.state(), ref_s) < tol
    assert rel_err(s.primal(), ref_x) < tol
    s.close()


@pytest.mark.parametrize("dims", [(24, 30), (6, 7, 8), (5, 260)])
def test_integer_states_with_ties_and_zero_weights(tv, orc, dims):
    """Integer states and weights in [0, 3]: collinear tube points (pops and
    crossings decided by exact zeros) and zero-width tube knots."""
    g = np.random.default_rng(7)
    w = g.integers(-10, 11, size=dims).astype(np.int32)
    a = [g.integers(0, 4, size=inputs.compact_shape(dims, k)).astype(np.int32) for k in range(len(dims))]
    st = np.round(random_state(dims, len(dims), 8, integer=True) * 0.1)
    s = tv.Solver(dims, dtype=tv.F64, check_every=1000, mapping=FUNNEL)
    s.set_problem(w, a)
    s.set_state(st)
    s.iterate(3)
    ref_s, ref_x = orc.iterate(0, w, a, st, 3)
    assert rel_err(s.state(), ref_s) < 1e-9
    assert rel_err(s.primal(), ref_x) < 1e-9
    s.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_hull_overflow_falls_back_to_local_form(tv, orc, dtype):
    """Convex ramps under wide tubes: every upper point stays on the convex
    minorant, so a lane's ring of 16 vertices fills and the lane continues in
    local form from its apex; the result is still the prox."""
    dims = (6, 1500)
    j = np.arange(dims[1], dtype=np.float64)
    st = np.empty((2,) + dims)
    st[0] = np.random.default_rng(3).normal(0, 1, size=dims)
    for r in range(dims[0]):
        st[1, r] = 1e-3 * (j - 700.0 + 100 * r) ** 2 / (1 + r)
    w = np.zeros(dims)
    a = [np.full(inputs.compact_shape(dims, 0), 0.5), np.full(inputs.compact_shape(dims, 1), 1e4)]
    code = tv.F64 if dtype == "f64" else tv.F32
    tol = 1e-9 if dtype == "f64" else 1e-4
    s = tv.Solver(dims, dtype=code, check_every=1000, mapping=FUNNEL)
    s.set_problem(w, a)
    s.set_state(st)
    s.iterate(1)
    ref_s, ref_x = orc.iterate(0, w, a, st, 1)
    assert rel_err(s.state(), ref_s) < tol
    assert rel_err(s.primal(), ref_x) < tol
    s.close()


@pytest.mark.parametrize("algo", [2, 3])
@pytest.mark.parametrize("dims", [(64, 64), (13, 17, 19), (3, 700)])
def test_projection_mode_methods(tv, orc, algo, dims):
    w, a = inputs.uniform_grid(dims, 25)
    s = tv.Solver(dims, algo=algo, dtype=tv.F64, check_every=1000, mapping=FUNNEL)
    s.set_problem(w, a)
    s.iterate(12)
    ref_s, ref_x = orc.iterate(algo, w, a, orc.cold_state(algo, w), 12)
    assert rel_err(s.state(), ref_s) < 1e-9
    assert rel_err(s.primal(), ref_x) < 1e-9
    s.close()


def test_segmentation_full_size(tv, orc):
    """1024^2 blob segmentation to the benchmark's k* = 223 in FP32 against
    the FP64 oracle (primal and state within 2e-4 of max|x|, the lane-group
    scan's stated FP32 tolerance on this drifting AAR state) and the exact
    min-cut; FP64 after 50 iterations within 1e-9.  The plateaus of these
    iterates fill some lanes' rings and segment lists, so the fallbacks run
    too."""
    dims = (1024, 1024)
    w, a = inputs.segmentation_problem(dims, 2)
    wd, ad = torch.from_numpy(w).cuda(), [torch.from_numpy(x).cuda() for x in a]
    s = tv.Solver(dims, dtype=tv.F32, check_every=10 ** 6, mapping=FUNNEL)
    s.set_problem(wd, ad)
    s.iterate(223)
    ref_s, x = orc.iterate(0, w, a, orc.cold_state(0, w), 223, nthreads=os.cpu_count() or 1)
    assert rel_err(s.primal(), x) < 2e-4
    assert rel_err(s.state(), ref_s) < 2e-4
    lab, st = s.cut()
    assert st.energy_i64 == orc.maxflow(w, a)[1]
    s.close()
    s = tv.Solver(dims, dtype=tv.F64, check_every=10 ** 6, mapping=FUNNEL)
    s.set_problem(wd, ad)
    s.iterate(50)
    ref_s, x = orc.iterate(0, w, a, orc.cold_state(0, w), 50, nthreads=os.cpu_count() or 1)
    assert rel_err(s.primal(), x) < 1e-9
    assert rel_err(s.state(), ref_s) < 1e-9
    s.close()


def test_long_chains_2048(tv, orc):
    """2048-element chains (the learned warm start's 2048^2 problems): a
    256 x 2048 strip, AAR and BCD, FP32 against the FP64 oracle."""
    dims = (256, 2048)
    w, a = inputs.uniform_grid(dims, 41)
    for algo, k in ((0, 60), (2, 20)):
        s = tv.Solver(dims, algo=algo, dtype=tv.F32, check_every=10 ** 6, mapping=FUNNEL)
        s.set_problem(w, a)
        s.iterate(k)
        ref_s, x = orc.iterate(algo, w, a, orc.cold_state(algo, w), k, nthreads=os.cpu_count() or 1)
        assert rel_err(s.primal(), x) < 1e-4, algo
        assert rel_err(s.state(), ref_s) < 1e-4, algo
        s.close()
