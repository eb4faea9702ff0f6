"""Block coordinate descent (Sec. 4.1) on the GPU against the CPU oracle.

One BCD cycle updates the blocks in turn, y_k <- Pi_{K_k}(w - sum_{j != k} y_j),
each through the same chain scan as AAR/AP.  Tolerances as in the AAR/AP
parity tests: FP64 to 1e-9 relative, FP32 to 1e-4 of max|x|; cut energies on
integer data exactly.
"""
import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BCD = 2
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
def test_bcd_iterations_f64(tv, orc, dims, mapping):
    w, a = inputs.uniform_grid(dims, 21)
    s = tv.Solver(dims, algo=BCD, dtype=tv.F64, check_every=1000, mapping=mapping)
    s.set_problem(w, a)
    st = orc.cold_state(BCD, w)
    done = 0
    for k in (1, 6, 17):
        s.iterate(k - done)
        st, x = orc.iterate(BCD, w, a, st, k - done)
        done = k
        assert rel_err(s.state(), st) < 1e-9, k
        assert rel_err(s.primal(), x) < 1e-9, k
        np.testing.assert_array_equal(s.dual(), s.state())    # the BCD state is y
    s.close()


@pytest.mark.parametrize("dims", [(64, 64), (37, 53), (13, 17, 19)])
def test_bcd_iterations_f32(tv, orc, dims):
    w, a = inputs.uniform_grid(dims, 22)
    s = tv.Solver(dims, algo=BCD, dtype=tv.F32, check_every=1000)
    s.set_problem(w, a)
    st = orc.cold_state(BCD, w)
    done = 0
    for k in (1, 10, 50):
        s.iterate(k - done)
        st, x = orc.iterate(BCD, w, a, st, k - done)
        done = k
        assert rel_err(s.primal(), x) < 1e-4, k
        assert rel_err(s.state(), st) < 1e-4, k
    s.close()


@pytest.mark.parametrize("dims", [(64, 64), (12, 14, 16)])
def test_bcd_exact_cut(tv, orc, dims):
    w, a = inputs.uniform_grid(dims, 4)
    e_star = orc.maxflow(w, a)[1]
    s = tv.Solver(dims, algo=BCD, dtype=tv.F64, check_every=5, threshold=0.5 / w.size)
    s.set_problem(w, a)
    code, st = s.iterate(20000)
    assert code == tv.OK and st.certified
    lab, st = s.cut()
    assert st.energy_i64 == e_star
    assert orc.energy(w, a, lab) == e_star
    s.close()


def test_bcd_dual_objective_monotone(tv, orc):
    """Each BCD step minimises the dual exactly over one block, so
    1/2 |w - sum_k y_k|^2 = 1/2 |x|^2 never increases (Sec. 4.1)."""
    dims = (48, 40)
    w, a = inputs.uniform_grid(dims, 6)
    s = tv.Solver(dims, algo=BCD, dtype=tv.F64, check_every=1000)
    s.set_problem(w, a)
    prev = np.inf
    for _ in range(30):
        s.iterate(1)
        d = 0.5 * float((s.primal() ** 2).sum())
        assert d <= prev * (1 + 1e-12) + 1e-9
        prev = d
    s.close()


def test_bcd_set_state_resume(tv, orc):
    """Checkpoint/resume of the BCD state through get/set_state."""
    dims = (30, 20, 9)
    w, a = inputs.uniform_grid(dims, 7)
    s = tv.Solver(dims, algo=BCD, dtype=tv.F64, check_every=1000)
    s.set_problem(w, a)
    s.iterate(5)
    mid = s.state()
    s.iterate(5)
    s2 = tv.Solver(dims, algo=BCD, dtype=tv.F64, check_every=1000)
    s2.set_problem(w, a)
    s2.set_state(mid)
    s2.iterate(5)
    np.testing.assert_array_equal(s2.state(), s.state())
    s.close()
    s2.close()


def test_bcd_rejected_where_not_built(tv):
    with pytest.raises(tv.TvcutError) as e:
        tv.Solver((8, 8), algo=BCD, mapping=2)
    assert e.value.code == tv.ERR_INVALID
    with pytest.raises(tv.TvcutError) as e:
        tv.Batch([(8, 8)], algo=BCD)
    assert e.value.code == tv.ERR_INVALID
