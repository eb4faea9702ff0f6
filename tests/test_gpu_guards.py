"""Guard regions around every caller-owned output buffer: each API call that
writes results (states, duals, primal, labels, batched states and labels,
convolution outputs) writes exactly its own range, in device and host
memory, and leaves poison-filled guards before and after it untouched.  A
stand-in for a sanitizer run on the caller-visible side of the boundary."""
import ctypes

import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

G = 1024          # guard elements on each side


@pytest.fixture(scope="module")
def tv():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01563_gb300 import tvcut
    tvcut.lib()
    return tvcut


def guarded(n, dtype, device):
    """(whole buffer, the middle n elements); the guards hold a bit pattern
    no result can have (0xA5 bytes)."""
    nbytes = (n + 2 * G) * torch.empty((), dtype=dtype).element_size()
    raw = torch.full((nbytes,), 0xA5, dtype=torch.uint8, device=device)
    if device == "cpu":
        raw = raw.pin_memory()
    buf = raw.view(dtype)
    return raw, buf[G:G + n]


def guards_intact(raw, n, dtype):
    es = torch.empty((), dtype=dtype).element_size()
    b = raw.cpu().numpy()
    return bool((b[:G * es] == 0xA5).all() and (b[(G + n) * es:] == 0xA5).all())


@pytest.mark.parametrize("dims,dtype,conn", [((37, 53), "f32", 0), ((5, 7, 9), "f64", 0), ((19, 23), "f32", 8)])
@pytest.mark.parametrize("device", ["cuda", "cpu"])
def test_solver_outputs_stay_in_range(tv, dims, dtype, conn, device):
    if conn == 8:
        w, a = inputs.uniform_grid8(dims, 3)
    else:
        w, a = inputs.uniform_grid(dims, 3)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    s = tv.Solver(dims, algo=tv.AAR, dtype=tv.F64 if dtype == "f64" else tv.F32, check_every=1000,
                  connectivity=conn)
    s.set_problem(w, a)
    s.iterate(7)
    n = int(np.prod(dims))
    nb = s.nblk
    raw, mid = guarded(nb * n, tdt, device)
    tv.tvcut_get_state(s.h, mid.view((nb,) + dims))
    assert guards_intact(raw, nb * n, tdt)
    assert torch.isfinite(mid).all()
    raw, mid = guarded(nb * n, tdt, device)
    code = tv.lib().tvcut_get_dual(s.h, ctypes.c_void_p(mid.data_ptr()), tv.DEVICE if device == "cuda" else tv.HOST)
    assert code == tv.OK
    torch.cuda.synchronize()
    assert guards_intact(raw, nb * n, tdt)
    raw, mid = guarded(n, tdt, device)
    tv.tvcut_get_primal(s.h, mid.view(dims))
    assert guards_intact(raw, n, tdt)
    raw, mid = guarded(n, torch.uint8, device)
    tv.tvcut_cut(s.h, mid.view(dims))
    torch.cuda.synchronize()
    assert guards_intact(raw, n, torch.uint8)
    assert int(mid.max()) <= 1
    s.close()


@pytest.mark.parametrize("device", ["cuda", "cpu"])
def test_batch_outputs_stay_in_range(tv, device):
    dims = [(37, 53), (5, 40), (1, 17), (64, 300)]
    b = tv.Batch(dims, dtype=tv.F32)
    for g, d in enumerate(dims):
        b.set_problem(g, *inputs.uniform_grid(d, 50 + g))
    b.reset()
    b.iterate(6)
    for g, d in enumerate(dims):
        n = d[0] * d[1]
        raw, mid = guarded(2 * n, torch.float32, device)
        code = tv.lib().tvcut_batch_get_state(b.h, g, ctypes.c_void_p(mid.data_ptr()),
                                              tv.DEVICE if device == "cuda" else tv.HOST)
        assert code >= 0
        torch.cuda.synchronize()
        assert guards_intact(raw, 2 * n, torch.float32)
        raw, mid = guarded(n, torch.uint8, device)
        st = tv.Stats()
        code = tv.lib().tvcut_batch_cut(b.h, g, ctypes.c_void_p(mid.data_ptr()),
                                        tv.DEVICE if device == "cuda" else tv.HOST, ctypes.byref(st))
        assert code >= 0
        torch.cuda.synchronize()
        assert guards_intact(raw, n, torch.uint8)
    b.close()


@pytest.mark.parametrize("engine,shape", [(0, (1, 16, 128, 16, 32)), (0, (2, 8, 256, 64, 128)), (3, (1, 8, 128, 32, 48)),
                                          (1, (1, 9, 13, 32, 16))])
def test_conv_output_stays_in_range(tv, engine, shape):
    n, h, w, ci, co = shape
    g = torch.Generator(device="cuda").manual_seed(5)
    xd = torch.randn((n, h, w, ci), generator=g, device="cuda").to(torch.bfloat16)
    wd = (torch.randn((9, co, ci), generator=g, device="cuda") * 0.2).to(torch.bfloat16)
    bd = torch.randn((co,), generator=g, device="cuda")
    m = n * h * w * co
    raw, mid = guarded(m, torch.bfloat16, "cuda")
    code = tv.lib().tvcut_conv3x3_bf16_ex(xd.data_ptr(), wd.data_ptr(), bd.data_ptr(), mid.data_ptr(), n, h, w, ci, co,
                                          1, engine, None)
    assert code == tv.OK
    torch.cuda.synchronize()
    assert tv.lib().tvcut_conv_tc_error() == 0
    assert guards_intact(raw, m, torch.bfloat16)
