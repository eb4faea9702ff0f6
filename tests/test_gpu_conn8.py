"""2D 8-connected grids on the GPU (four blocks: columns, rows and the two
blocks of zig-zag paths of Sec. 3.1, Fig. 2 middle) against the 8-connected
oracle (oracle/conn8.py).  Tolerances as in the 4-connected parity tests:
FP64 iterates to 1e-9 relative, FP32 to 1e-4 of max|x|; cut energies on
integer data exactly."""
import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(64, 64), (37, 53), (2, 2), (1, 9), (9, 1), (33, 65), (5, 128), (3, 2)]


@pytest.fixture(scope="module")
def tv():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01563_gb300 import tvcut
    tvcut.lib()
    return tvcut


@pytest.fixture(scope="module")
def c8(orc):
    from oracle import conn8
    return conn8


def rel_err(got, want):
    return float(np.abs(np.asarray(got, np.float64) - want).max() / max(1.0, np.abs(want).max()))


@pytest.mark.parametrize("dims", CASES)
@pytest.mark.parametrize("algo", [0, 1, 2, 3])
@pytest.mark.parametrize("mapping", [-1, 5, 6, 8, 11])
def test_conn8_iterations_f64(tv, c8, dims, algo, mapping):
    w, a = inputs.uniform_grid8(dims, 41)
    s = tv.Solver(dims, algo=algo, dtype=tv.F64, check_every=1000, mapping=mapping, connectivity=8)
    s.set_problem(w, a)
    st = c8.cold_state(algo, w)
    done = 0
    for k in (1, 6, 17):
        s.iterate(k - done)
        if algo == 3:                  # FISTA: the oracle's momentum restarts per call, so run it from cold
            st, x = c8.iterate(algo, w, a, c8.cold_state(algo, w), k)
        else:
            st, x = c8.iterate(algo, w, a, st, k - done)
        done = k
        assert rel_err(s.state(), st) < 1e-9, k
        assert rel_err(s.primal(), x) < 1e-9, k
        if algo >= 2:
            np.testing.assert_array_equal(s.dual(), s.state())
    s.close()


@pytest.mark.parametrize("dims", [(64, 64), (37, 53)])
@pytest.mark.parametrize("algo", [0, 1, 2, 3])
def test_conn8_iterations_f32(tv, c8, dims, algo):
    w, a = inputs.uniform_grid8(dims, 42)
    s = tv.Solver(dims, algo=algo, dtype=tv.F32, check_every=1000, connectivity=8)
    s.set_problem(w, a)
    st = c8.cold_state(algo, w)
    done = 0
    for k in (1, 10, 50):
        s.iterate(k - done)
        if algo == 3:
            st, x = c8.iterate(algo, w, a, c8.cold_state(algo, w), k)
        else:
            st, x = c8.iterate(algo, w, a, st, k - done)
        done = k
        assert rel_err(s.primal(), x) < 1e-4, k
        assert rel_err(s.state(), st) < 1e-4, k
    s.close()


@pytest.mark.parametrize("dims", [(48, 40), (33, 17)])
@pytest.mark.parametrize("algo", [0, 2, 3])
def test_conn8_exact_cut(tv, c8, dims, algo):
    w, a = inputs.uniform_grid8(dims, 4)
    e_star = c8.maxflow(w, a)[1]
    s = tv.Solver(dims, algo=algo, dtype=tv.F64, check_every=5, threshold=0.5 / w.size, connectivity=8)
    s.set_problem(w, a)
    code, st = s.iterate(20000)
    assert code == tv.OK and st.certified
    lab, st = s.cut()
    assert st.energy_i64 == e_star
    assert c8.energy(w, a, lab) == e_star
    s.close()


def test_conn8_check_statistics(tv, c8):
    dims = (29, 31)
    w, a = inputs.uniform_grid8(dims, 5)
    s = tv.Solver(dims, dtype=tv.F64, check_every=1, level_sets=0, connectivity=8)
    s.set_problem(w, a)
    for k in (1, 7, 40):
        _, st = s.iterate(k)
        lab, _ = s.cut()
        x = s.primal()
        assert np.array_equal(lab, (x > 0).astype(np.uint8))
        assert st.energy_i64 == c8.energy(w, a, lab)
        f = c8.tv_value(a, x)
        assert abs(st.tv_value - f) < 1e-8 * max(1, f)
        y = w - x
        assert abs(st.tv_gap - (f - (y * x).sum())) < 1e-6 * max(1, f)
    s.close()


def test_conn8_state_roundtrip_and_dual(tv, c8):
    dims = (20, 27)
    w, a = inputs.uniform_grid8(dims, 6)
    s = tv.Solver(dims, dtype=tv.F64, check_every=1000, connectivity=8)
    s.set_problem(w, a)
    s.iterate(9)
    st = s.state()
    assert st.shape == (4,) + dims
    np.testing.assert_allclose(s.dual(), c8.project_K(st, a), atol=1e-9 * max(1, np.abs(st).max()))
    s2 = tv.Solver(dims, dtype=tv.F64, check_every=1000, connectivity=8)
    s2.set_problem(w, a)
    s2.set_state(st)
    np.testing.assert_array_equal(s2.state(), st)
    s.iterate(5)
    s2.iterate(5)
    np.testing.assert_array_equal(s2.state(), s.state())
    s.close()
    s2.close()


def test_conn8_errors(tv):
    for kw in (dict(mapping=2), dict(mapping=4)):
        with pytest.raises(tv.TvcutError) as e:
            tv.Solver((8, 8), connectivity=8, **kw)
        assert e.value.code == tv.ERR_INVALID
    with pytest.raises(tv.TvcutError) as e:
        tv.Solver((4, 4, 4), connectivity=8)
    assert e.value.code == tv.ERR_INVALID
    import ctypes
    p = tv.tvcut_default_params()
    p.connectivity = 8
    flat = (ctypes.c_int64 * 2)(8, 8)
    hb = ctypes.c_void_p()
    assert tv.lib().tvcut_batch_create(1, flat, ctypes.byref(p), None, ctypes.byref(hb)) == tv.ERR_INVALID
    s = tv.Solver((6, 7), connectivity=8)
    w, a = inputs.uniform_grid8((6, 7), 1)
    s.set_problem(w, a[:3])
    with pytest.raises(tv.TvcutError) as e:
        s.iterate(1)                                # anti-diagonal weights missing
    assert e.value.code == tv.ERR_STATE
    with pytest.raises(tv.TvcutError) as e:
        tv.tvcut_set_weights(s.h, 4, a[3])
    assert e.value.code == tv.ERR_INVALID
    s.close()
