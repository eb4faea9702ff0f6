"""tvcut_iterate_noalloc: iterations for callers that cannot let the library
allocate device memory (a framework allocator that owns the GPU's memory, or
a latency-critical loop where a cudaMalloc is not acceptable).  Its only
scratch is a fixed array inside the library image; this checks that its
results match the CPU oracle's iterations (FP64) and the handle-based entry
point (tvcut_iterate) within the tolerance used by the other GPU tests
(FP32 1e-4, FP64 1e-9 of max|x|), on two calls in a row that share that
array, and that oversized grids are refused."""
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


def via_handle(tv, w, a, algo, dtype, iters):
    s = tv.Solver(w.shape, algo=algo, dtype=dtype, check_every=10 ** 6)
    s.set_problem(w, a)
    s.iterate(iters)
    st, x = s.state(), s.primal()
    s.close()
    return st.astype(np.float64), x


def rel_err(got, want):
    return float(np.abs(np.asarray(got, np.float64) - want).max() / max(1.0, np.abs(want).max()))


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_noalloc_matches_oracle_and_handle_two_calls(tv, orc, algo, dtype):
    tdt = torch.float32 if dtype == "f32" else torch.float64
    code = tv.F32 if dtype == "f32" else tv.F64
    tol = 1e-4 if dtype == "f32" else 1e-9
    problems = [inputs.uniform_grid((96, 130), 21), inputs.uniform_grid((20, 24, 28), 22)]
    for call, (w, a) in enumerate(problems):          # two calls in a row share the scratch
        iters = 13 + call
        want_state, want_x = via_handle(tv, w, a, algo, code, iters)
        ref_state, ref_x = orc.iterate(algo, w, a, orc.cold_state(algo, w), iters)
        r = w.ndim
        wd = torch.from_numpy(w).to("cuda", tdt)
        ad = [torch.from_numpy(x).to("cuda", tdt) for x in a]
        if algo == tv.AAR:
            state = torch.zeros((r,) + w.shape, dtype=tdt, device="cuda")
        else:
            state = (wd / r).unsqueeze(0).repeat((r,) + (1,) * w.ndim).contiguous()
        x = torch.empty_like(wd)
        tv.tvcut_iterate_noalloc(w.shape, algo, wd, ad, state, x, iters)
        torch.cuda.synchronize()
        got_state, got_x = state.cpu().numpy(), x.cpu().numpy()
        assert rel_err(got_state, ref_state) < tol, call
        assert rel_err(got_x, ref_x) < tol, call
        assert rel_err(got_state, want_state) < tol, call
        assert rel_err(got_x, want_x) < tol, call


def test_noalloc_rejects_oversized_grid(tv):
    dims = (2049, 1024)                                # 2^21 + 1024 vertices > the FP32 limit
    w = torch.zeros(dims, dtype=torch.float32, device="cuda")
    a = [torch.zeros((2048, 1024), device="cuda"), torch.zeros((2049, 1023), device="cuda")]
    state = torch.zeros((2,) + dims, device="cuda")
    with pytest.raises(tv.TvcutError) as e:
        tv.tvcut_iterate_noalloc(dims, tv.AAR, w, a, state, None, 1)
    assert e.value.code == tv.ERR_INVALID
    assert "at most" in str(e.value)
