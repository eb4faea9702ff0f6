"""FISTA on the smooth dual (Sec. 4.1) on the GPU against the CPU oracle.

One step: v = Pi_L(y + beta (y - y_prev)) for all blocks, then y <- Pi_K(v)
by the chain scan in projection mode; beta = (t_{k-1} - 1)/t_k.  The oracle
runs the same steps from the same start in one call (its momentum restarts
at every call, like the library's after tvcut_set_state).  Tolerances as in
the AAR/AP parity tests: FP64 to 1e-9 relative, FP32 to 1e-4 of max|x|; cut
energies on integer data exactly.
"""
import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FISTA = 3
CASES = [(64, 64), (37, 53), (1, 9), (9, 1), (2, 2), (13, 17, 19), (1, 5, 6), (7, 1, 3), (40, 1000)]


@pytest.fixture(scope="module")
def tv():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01563_gb300 import tvcut
    tvcut.lib()
    return tvcut


def rel_err(got, want):
    return float(np.abs(np.asarray(got, np.float64) - want).max() / max(1.0, np.abs(want).max()))


@pytest.mark.parametrize("dims", CASES)
@pytest.mark.parametrize("mapping", [-1, 5, 6, 8, 9, 11])
def test_fista_iterations_f64(tv, orc, dims, mapping):
    w, a = inputs.uniform_grid(dims, 31)
    s = tv.Solver(dims, algo=FISTA, dtype=tv.F64, check_every=1000, mapping=mapping)
    s.set_problem(w, a)
    done = 0
    for k in (1, 2, 3, 6, 17):
        s.iterate(k - done)                       # the momentum carries across calls
        done = k
        st, x = orc.iterate(FISTA, w, a, orc.cold_state(FISTA, w), k)
        assert rel_err(s.state(), st) < 1e-9, k
        assert rel_err(s.primal(), x) < 1e-9, k
        np.testing.assert_array_equal(s.dual(), s.state())    # the FISTA state is y
    s.close()


@pytest.mark.parametrize("dims", [(64, 64), (37, 53), (13, 17, 19)])
def test_fista_iterations_f32(tv, orc, dims):
    w, a = inputs.uniform_grid(dims, 32)
    s = tv.Solver(dims, algo=FISTA, dtype=tv.F32, check_every=1000)
    s.set_problem(w, a)
    done = 0
    for k in (1, 10, 50):
        s.iterate(k - done)
        done = k
        st, x = orc.iterate(FISTA, w, a, orc.cold_state(FISTA, w), k)
        assert rel_err(s.primal(), x) < 1e-4, k
        assert rel_err(s.state(), st) < 1e-4, k
    s.close()


@pytest.mark.parametrize("dims", [(64, 64), (12, 14, 16)])
def test_fista_exact_cut(tv, orc, dims):
    w, a = inputs.uniform_grid(dims, 4)
    e_star = orc.maxflow(w, a)[1]
    s = tv.Solver(dims, algo=FISTA, dtype=tv.F64, check_every=5, threshold=0.5 / w.size)
    s.set_problem(w, a)
    code, st = s.iterate(20000)
    assert code == tv.OK and st.certified
    lab, st = s.cut()
    assert st.energy_i64 == e_star
    assert orc.energy(w, a, lab) == e_star
    s.close()


def test_fista_set_state_restarts_momentum(tv, orc):
    """After tvcut_set_state the steps are those of a fresh FISTA run from
    that state (previous iterate = state, t = 1)."""
    dims = (30, 20, 9)
    w, a = inputs.uniform_grid(dims, 7)
    s = tv.Solver(dims, algo=FISTA, dtype=tv.F64, check_every=1000)
    s.set_problem(w, a)
    s.iterate(6)
    mid = s.state()
    s2 = tv.Solver(dims, algo=FISTA, dtype=tv.F64, check_every=1000)
    s2.set_problem(w, a)
    s2.set_state(mid)
    s2.iterate(7)
    want, x = orc.iterate(FISTA, w, a, mid, 7)
    assert rel_err(s2.state(), want) < 1e-9
    assert rel_err(s2.primal(), x) < 1e-9
    s.close()
    s2.close()


def test_fista_rejected_with_fused_sweeps(tv):
    with pytest.raises(tv.TvcutError) as e:
        tv.Solver((8, 8), algo=FISTA, mapping=3)
    assert e.value.code == tv.ERR_INVALID
