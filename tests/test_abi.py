"""The C-ABI library loads and exports every function declared in
include/tvcut.h (no GPU needed: nothing is called that touches the device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(tvcut_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_1503_01563_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    names = declared_functions()
    assert "tvcut_create" in names and "tvcut_iterate" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols(built):
    from paper_1503_01563_gb300 import tvcut
    assert set(declared_functions()) <= set(tvcut.EXPORTED)
    tvcut.load(built)


def test_host_only_calls(built):
    """Calls that need no device: defaults and argument validation."""
    from paper_1503_01563_gb300 import tvcut
    p = tvcut.tvcut_default_params()
    assert p.algo == tvcut.AAR and p.iterate_dtype == tvcut.F32 and p.check_every == 10
    lib = tvcut.load(built)
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 2)(4, 4)
    assert lib.tvcut_create(1, dims, None, None, ctypes.byref(h)) == tvcut.ERR_INVALID
    assert b"ndim" in lib.tvcut_last_error(None)
    bad = (ctypes.c_int64 * 2)(0, 4)
    assert lib.tvcut_create(2, bad, None, None, ctypes.byref(h)) == tvcut.ERR_INVALID
    p.check_every = 0
    assert lib.tvcut_create(2, dims, ctypes.byref(p), None, ctypes.byref(h)) == tvcut.ERR_INVALID
    assert lib.tvcut_iterate(None, 1, None) == tvcut.ERR_INVALID
    for field, bad in (("certify", 3), ("certify", -1), ("stop_on_approx", 2), ("mapping", 12)):
        q = tvcut.tvcut_default_params()
        setattr(q, field, bad)
        assert lib.tvcut_create(2, dims, ctypes.byref(q), None, ctypes.byref(h)) == tvcut.ERR_INVALID, field
        assert field.encode() in lib.tvcut_last_error(None)
    assert lib.tvcut_mp_fallbacks(None, 0) == tvcut.ERR_INVALID
    assert lib.tvcut_unet_predict_state(None, None) == tvcut.ERR_INVALID


def test_no_oracle_in_product_path():
    """The product package neither imports nor links the oracle."""
    pkg = os.path.join(ROOT, "paper_1503_01563_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "oracle.h" not in src and "liboracle" not in src, f


def _noalloc_args(dims=(6, 5), dt="float32"):
    import numpy as np
    w = np.zeros(dims, dt)
    a = [np.zeros(tuple(d - 1 if j == k else d for j, d in enumerate(dims)), dt) for k in range(len(dims))]
    state = np.zeros((len(dims),) + dims, dt)
    x = np.zeros(dims, dt)
    return dims, w, a, state, x


@pytest.mark.parametrize("case", ["state_dtype", "a_dtype", "x_dtype", "state_shape", "w_shape", "a_shape",
                                  "a_count", "x_shape", "host_buffers"])
def test_noalloc_wrapper_rejects_mismatched_buffers(case):
    """tvcut_iterate_noalloc's binding checks every buffer's dtype and shape
    before a pointer reaches the library (no GPU needed: nothing is called)."""
    import numpy as np
    from paper_1503_01563_gb300 import tvcut
    dims, w, a, state, x = _noalloc_args()
    if case == "state_dtype":
        state = state.astype(np.float64)
    elif case == "a_dtype":
        a[1] = a[1].astype(np.float64)
    elif case == "x_dtype":
        x = x.astype(np.float64)
    elif case == "state_shape":
        state = state[:1]
    elif case == "w_shape":
        w = w[:-1]
    elif case == "a_shape":
        a[0] = np.zeros(dims, np.float32)
    elif case == "a_count":
        a = a[:1]
    elif case == "x_shape":
        x = x.ravel()
    with pytest.raises(ValueError) as e:
        tvcut.tvcut_iterate_noalloc(dims, tvcut.AAR, w, a, state, x, 1)
    if case == "host_buffers":
        assert "device tensors" in str(e.value)
