"""Python binding of the tvcut C-ABI (include/tvcut.h).

Argument marshalling only: every step of the solver runs in libtvcut.so's
CUDA kernels.  Functions carry the C names (``tvcut_create`` ...); ``Solver``
wraps a handle for convenience.  Arrays may be numpy arrays (host memory) or
CUDA torch tensors (device memory); the binding passes their pointers and the
matching ``space`` flag.  There is no fallback: if libtvcut.so is missing the
import-time load raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtvcut.so")

OK, NOT_CONVERGED = 0, 1
ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_STATE, ERR_TIMEOUT = -1, -2, -3, -4, -5
I32, F32, F64 = 0, 1, 2
HOST, DEVICE = 0, 1
AAR, AP, BCD, FISTA = 0, 1, 2, 3

EXPORTED = [
    "tvcut_default_params", "tvcut_create", "tvcut_destroy", "tvcut_last_error",
    "tvcut_set_unary", "tvcut_set_weights", "tvcut_reset", "tvcut_iterate", "tvcut_cut",
    "tvcut_get_primal", "tvcut_get_state", "tvcut_set_state", "tvcut_warmstart_primal",
    "tvcut_project_chains", "tvcut_profile", "tvcut_profile_read", "tvcut_iterate_noalloc", "tvcut_get_dual",
    "tvcut_batch_create", "tvcut_batch_destroy", "tvcut_batch_last_error", "tvcut_batch_set_unary",
    "tvcut_batch_set_weights", "tvcut_batch_reset", "tvcut_batch_iterate", "tvcut_batch_cut",
    "tvcut_batch_get_state", "tvcut_batch_autotune", "tvcut_batch_set_launch",
    "tvcut_unet_create", "tvcut_unet_destroy", "tvcut_unet_last_error", "tvcut_unet_resize",
    "tvcut_unet_forward", "tvcut_unet_backward", "tvcut_unet_adam", "tvcut_unet_num_params",
    "tvcut_unet_get_params", "tvcut_unet_set_params", "tvcut_conv3x3_bf16", "tvcut_conv3x3_wgrad_bf16",
    "tvcut_conv3x3_bf16_ex", "tvcut_conv_tc_error", "tvcut_unet_set_engine", "tvcut_conv_tc_stall",
    "tvcut_unet_predict_state", "tvcut_mp_fallbacks",
]
K_PROX, K_UPDATE, K_CHECK, K_OTHER, NKINDS = 0, 1, 2, 3, 4


class Params(ctypes.Structure):
    _fields_ = [
        ("algo", ctypes.c_int),
        ("iterate_dtype", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("mapping", ctypes.c_int),
        ("gap_tol", ctypes.c_double),
        ("threshold", ctypes.c_double),
        ("level_sets", ctypes.c_int),
        ("connectivity", ctypes.c_int),
        ("certify", ctypes.c_int),
        ("stop_on_approx", ctypes.c_int),
        ("reserved", ctypes.c_int * 4),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int64),
        ("energy", ctypes.c_double),
        ("energy_i64", ctypes.c_int64),
        ("energy_exact", ctypes.c_int),
        ("certified", ctypes.c_int),
        ("discrete_lb", ctypes.c_double),
        ("tv_value", ctypes.c_double),
        ("tv_gap", ctypes.c_double),
        ("x_absmax", ctypes.c_double),
        ("n_label1", ctypes.c_int64),
        ("threshold", ctypes.c_double),
        ("certified_lb", ctypes.c_double),
        ("reserved", ctypes.c_int64 * 2),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class TvcutError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tvcut error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libtvcut.so not built ({path}); run paper_1503_01563_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    c_int = ctypes.c_int
    st = ctypes.c_int
    sig = {
        "tvcut_default_params": (None, [ctypes.POINTER(Params)]),
        "tvcut_create": (st, [c_int, P, ctypes.POINTER(Params), P, ctypes.POINTER(P)]),
        "tvcut_destroy": (None, [P]),
        "tvcut_last_error": (ctypes.c_char_p, [P]),
        "tvcut_set_unary": (st, [P, P, c_int, c_int]),
        "tvcut_set_weights": (st, [P, c_int, P, c_int, c_int]),
        "tvcut_reset": (st, [P]),
        "tvcut_iterate": (st, [P, i64, ctypes.POINTER(Stats)]),
        "tvcut_cut": (st, [P, P, c_int, ctypes.POINTER(Stats)]),
        "tvcut_get_primal": (st, [P, P, c_int, c_int]),
        "tvcut_get_state": (st, [P, P, c_int]),
        "tvcut_set_state": (st, [P, P, c_int]),
        "tvcut_get_dual": (st, [P, P, c_int]),
        "tvcut_warmstart_primal": (st, [P, P, ctypes.c_float, c_int]),
        "tvcut_project_chains": (st, [c_int, P, c_int, P, P, P, c_int, c_int, P]),
        "tvcut_profile": (st, [P, c_int]),
        "tvcut_profile_read": (st, [P, P, P]),
        "tvcut_iterate_noalloc": (st, [c_int, P, c_int, c_int, P, P, P, P, i64, P]),
        "tvcut_batch_create": (st, [c_int, P, ctypes.POINTER(Params), P, ctypes.POINTER(P)]),
        "tvcut_batch_destroy": (None, [P]),
        "tvcut_batch_last_error": (ctypes.c_char_p, [P]),
        "tvcut_batch_set_unary": (st, [P, c_int, P, c_int, c_int]),
        "tvcut_batch_set_weights": (st, [P, c_int, c_int, P, c_int, c_int]),
        "tvcut_batch_reset": (st, [P]),
        "tvcut_batch_iterate": (st, [P, i64, P]),
        "tvcut_batch_cut": (st, [P, c_int, P, c_int, ctypes.POINTER(Stats)]),
        "tvcut_batch_get_state": (st, [P, c_int, P, c_int]),
        "tvcut_batch_autotune": (st, [P, P]),
        "tvcut_batch_set_launch": (st, [P, c_int, c_int, c_int]),
        "tvcut_unet_create": (st, [c_int, c_int, c_int, c_int, ctypes.c_uint64, P, ctypes.POINTER(P)]),
        "tvcut_unet_destroy": (None, [P]),
        "tvcut_unet_last_error": (ctypes.c_char_p, [P]),
        "tvcut_unet_resize": (st, [P, c_int, c_int, c_int]),
        "tvcut_unet_forward": (st, [P, P, P]),
        "tvcut_unet_backward": (st, [P, P, ctypes.POINTER(ctypes.c_float)]),
        "tvcut_unet_adam": (st, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
        "tvcut_unet_num_params": (st, [P, ctypes.POINTER(i64)]),
        "tvcut_unet_get_params": (st, [P, P, c_int]),
        "tvcut_unet_set_params": (st, [P, P]),
        "tvcut_conv3x3_bf16": (st, [P, P, P, P, c_int, c_int, c_int, c_int, c_int, c_int, P]),
        "tvcut_conv3x3_wgrad_bf16": (st, [P, P, P, c_int, c_int, c_int, c_int, c_int, P]),
        "tvcut_conv3x3_bf16_ex": (st, [P, P, P, P, c_int, c_int, c_int, c_int, c_int, c_int, c_int, P]),
        "tvcut_conv_tc_error": (c_int, []),
        "tvcut_conv_tc_stall": (st, [c_int]),
        "tvcut_unet_set_engine": (st, [P, c_int]),
        "tvcut_unet_predict_state": (st, [P, P]),
        "tvcut_mp_fallbacks": (st, [ctypes.POINTER(ctypes.c_ulonglong), c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


# ---- marshalling helpers ----------------------------------------------------

def _dtype_code(dt) -> int:
    dt = str(dt)
    if dt.endswith("int32"):
        return I32
    if dt.endswith("float32"):
        return F32
    if dt.endswith("float64"):
        return F64
    raise TypeError(f"unsupported dtype {dt}")


def _buf(arr):
    """(pointer, space, dtype code, keepalive) of a numpy array or torch tensor."""
    if isinstance(arr, np.ndarray):
        arr = np.ascontiguousarray(arr)
        return ctypes.c_void_p(arr.ctypes.data), HOST, _dtype_code(arr.dtype), arr
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(arr, torch.Tensor):
        if not arr.is_contiguous():
            raise ValueError("tensor must be contiguous")
        space = DEVICE if arr.is_cuda else HOST
        return ctypes.c_void_p(arr.data_ptr()), space, _dtype_code(arr.dtype), arr
    arr = np.ascontiguousarray(np.asarray(arr))
    return ctypes.c_void_p(arr.ctypes.data), HOST, _dtype_code(arr.dtype), arr


def _check(code, h=None):
    if code < 0:
        msg = lib().tvcut_last_error(h)
        raise TvcutError(code, msg.decode() if msg else "")
    return code


def tvcut_default_params() -> Params:
    p = Params()
    lib().tvcut_default_params(ctypes.byref(p))
    return p


def tvcut_create(dims, params: Params | None = None, stream=None):
    dims_arr = (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])
    h = ctypes.c_void_p()
    s = ctypes.c_void_p(int(stream) if stream else 0)
    _check(lib().tvcut_create(len(dims), dims_arr, ctypes.byref(params) if params else None, s, ctypes.byref(h)))
    return h


def tvcut_destroy(h):
    lib().tvcut_destroy(h)


def tvcut_set_unary(h, w):
    p, space, dt, keep = _buf(w)
    return _check(lib().tvcut_set_unary(h, p, dt, space), h)


def tvcut_set_weights(h, axis, a):
    p, space, dt, keep = _buf(a)
    return _check(lib().tvcut_set_weights(h, int(axis), p, dt, space), h)


def tvcut_reset(h):
    return _check(lib().tvcut_reset(h), h)


def tvcut_iterate(h, max_iters):
    st = Stats()
    code = _check(lib().tvcut_iterate(h, int(max_iters), ctypes.byref(st)), h)
    return code, st


def tvcut_cut(h, labels=None):
    """labels: None, a uint8 numpy array (host) or a uint8 CUDA tensor."""
    st = Stats()
    if labels is None:
        _check(lib().tvcut_cut(h, None, HOST, ctypes.byref(st)), h)
    elif isinstance(labels, np.ndarray):
        assert labels.dtype == np.uint8 and labels.flags.c_contiguous
        _check(lib().tvcut_cut(h, ctypes.c_void_p(labels.ctypes.data), HOST, ctypes.byref(st)), h)
    else:
        _check(lib().tvcut_cut(h, ctypes.c_void_p(labels.data_ptr()), DEVICE if labels.is_cuda else HOST,
                               ctypes.byref(st)), h)
    return st


def tvcut_get_primal(h, out):
    p, space, dt, keep = _buf(out)
    return _check(lib().tvcut_get_primal(h, p, dt, space), h)


def tvcut_get_state(h, out):
    p, space, dt, keep = _buf(out)
    return _check(lib().tvcut_get_state(h, p, space), h)


def tvcut_set_state(h, s):
    p, space, dt, keep = _buf(s)
    return _check(lib().tvcut_set_state(h, p, space), h)


def tvcut_warmstart_primal(h, xhat, tau: float):
    p, space, dt, keep = _buf(xhat)
    if dt != F32:
        raise TypeError("xhat must be float32")
    return _check(lib().tvcut_warmstart_primal(h, p, ctypes.c_float(tau), space), h)


def tvcut_project_chains(dims, axis, v, a, out, what=0, stream=None):
    """Device tensors only (float32 or float64)."""
    dims_arr = (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])
    pv, sv, dv, _ = _buf(v)
    pa, sa, da, _ = _buf(a)
    po, so, do, _ = _buf(out)
    if not (sv == sa == so == DEVICE):
        raise ValueError("tvcut_project_chains takes device tensors")
    s = ctypes.c_void_p(int(stream) if stream else 0)
    return _check(lib().tvcut_project_chains(len(dims), dims_arr, int(axis), pv, pa, po, dv, int(what), s))


def tvcut_mp_fallbacks(reset=False):
    """Chains of the message-passing prox (mapping 10) recomputed by the taut
    string since the last reset."""
    n = ctypes.c_ulonglong()
    _check(lib().tvcut_mp_fallbacks(ctypes.byref(n), 1 if reset else 0))
    return int(n.value)


def tvcut_profile(h, enable: bool):
    return _check(lib().tvcut_profile(h, 1 if enable else 0), h)


def tvcut_profile_read(h):
    """Returns (ms per kernel kind, launches per kernel kind) as numpy arrays."""
    ms = np.zeros(NKINDS, dtype=np.float64)
    n = np.zeros(NKINDS, dtype=np.int64)
    _check(lib().tvcut_profile_read(h, ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(n.ctypes.data)), h)
    return ms, n


def _noalloc_check(dims, w, a, state, x):
    """Shape and dtype checks of tvcut_iterate_noalloc's buffers, made before
    any pointer reaches the library: the C side trusts the sizes it derives
    from ``dims``, so a short or mistyped buffer would be read or written past
    its end on the device."""
    dims = tuple(int(d) for d in dims)
    if len(dims) not in (2, 3):
        raise ValueError("dims must have 2 or 3 entries")

    def meta(t, name):
        if t is None:
            raise ValueError(f"{name} is required")
        return tuple(int(d) for d in t.shape), str(t.dtype)

    wshape, wdt = meta(w, "w")
    if wshape != dims:
        raise ValueError(f"w must have shape {dims}, got {wshape}")
    if not (wdt.endswith("float32") or wdt.endswith("float64")):
        raise ValueError(f"w must be float32 or float64, got {wdt}")
    if len(a) != len(dims):
        raise ValueError(f"need {len(dims)} weight arrays (one per axis), got {len(a)}")
    for k, ak in enumerate(a):
        want = tuple(d - 1 if j == k else d for j, d in enumerate(dims))
        shp, dt = meta(ak, f"a[{k}]")
        if shp != want:
            raise ValueError(f"a[{k}] must have shape {want}, got {shp}")
        if dt != wdt:
            raise ValueError(f"a[{k}] has dtype {dt}; every buffer must have w's dtype {wdt}")
    shp, dt = meta(state, "state")
    if shp != (len(dims),) + dims:
        raise ValueError(f"state must have shape {(len(dims),) + dims}, got {shp}")
    if dt != wdt:
        raise ValueError(f"state has dtype {dt}; every buffer must have w's dtype {wdt}")
    if x is not None:
        shp, dt = meta(x, "x")
        if shp != dims:
            raise ValueError(f"x must have shape {dims}, got {shp}")
        if dt != wdt:
            raise ValueError(f"x has dtype {dt}; every buffer must have w's dtype {wdt}")
    return dims


def tvcut_iterate_noalloc(dims, algo, w, a, state, x=None, iters=1, stream=None):
    """Iterations on caller-owned device tensors, with no device allocation
    inside the library (see include/tvcut.h).  w, a[k], state, x: contiguous
    CUDA tensors of one float dtype; a[k] has the grid's shape with dims[k]-1
    along axis k; state has shape (ndim,) + dims.  With iters == 0 nothing
    runs and x is left as it is."""
    dims = _noalloc_check(dims, w, a, state, x)
    dims_arr = (ctypes.c_int64 * len(dims))(*dims)
    pw, sw, dt, _ = _buf(w)
    bufs = [_buf(ak) for ak in a]
    ps, ss, dts, _ = _buf(state)
    xb = _buf(x) if x is not None else None
    if (sw != DEVICE or ss != DEVICE or any(b[1] != DEVICE for b in bufs)
            or (xb is not None and xb[1] != DEVICE)):
        raise ValueError("tvcut_iterate_noalloc takes device tensors")
    arr = (ctypes.c_void_p * len(bufs))(*[b[0].value for b in bufs])
    s = ctypes.c_void_p(int(stream) if stream else 0)
    px = xb[0] if xb is not None else None
    return _check(lib().tvcut_iterate_noalloc(len(dims), dims_arr, int(algo), dt, pw, arr, ps, px, int(iters), s))


class Solver:
    """One grid: ``Solver(dims, algo=AAR, dtype=F32)``; ``set_problem(w, a)``;
    ``iterate(k)``; ``cut()``.  ``connectivity=8``: a 2D grid with diagonal
    edges; ``a`` then holds four arrays (vertical, horizontal, diagonal,
    anti-diagonal) and states have four blocks."""

    def __init__(self, dims, algo=AAR, dtype=F32, check_every=10, gap_tol=0.0, threshold=0.0,
                 stream=None, level_sets=None, mapping=-1, connectivity=0, certify=0, stop_on_approx=0):
        p = tvcut_default_params()
        p.certify = certify
        p.stop_on_approx = stop_on_approx
        p.mapping = mapping
        p.connectivity = connectivity
        if level_sets is not None:
            p.level_sets = level_sets
        p.algo = algo
        p.iterate_dtype = dtype
        p.check_every = check_every
        p.gap_tol = gap_tol
        p.threshold = threshold
        self.dims = tuple(int(d) for d in dims)
        self.n = int(np.prod(self.dims))
        self.dtype = dtype
        self.nblk = 4 if connectivity == 8 else len(self.dims)
        self.h = tvcut_create(self.dims, p, stream)

    def close(self):
        if self.h:
            tvcut_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_problem(self, w, a):
        tvcut_set_unary(self.h, w)
        for k, ak in enumerate(a):
            tvcut_set_weights(self.h, k, ak)

    def reset(self):
        tvcut_reset(self.h)

    def iterate(self, max_iters):
        return tvcut_iterate(self.h, max_iters)

    def cut(self, labels=True):
        if labels:
            lab = np.empty(self.dims, dtype=np.uint8)
            st = tvcut_cut(self.h, lab)
            return lab, st
        return None, tvcut_cut(self.h, None)

    def primal(self, dtype=np.float64):
        x = np.empty(self.dims, dtype=dtype)
        tvcut_get_primal(self.h, x)
        return x

    def state(self):
        s = np.empty((self.nblk,) + self.dims, dtype=np.float64 if self.dtype == F64 else np.float32)
        tvcut_get_state(self.h, s)
        return s

    def dual(self):
        """Shadow duals y_k of the current state, shape (ndim,) + dims."""
        y = np.empty((self.nblk,) + self.dims, dtype=np.float64 if self.dtype == F64 else np.float32)
        _check(lib().tvcut_get_dual(self.h, ctypes.c_void_p(y.ctypes.data), HOST), self.h)
        return y

    def set_state(self, s):
        want = np.float64 if self.dtype == F64 else np.float32
        tvcut_set_state(self.h, np.ascontiguousarray(s, dtype=want))


def _bcheck(code, b):
    if code < 0:
        msg = lib().tvcut_batch_last_error(b)
        raise TvcutError(code, msg.decode() if msg else "")
    return code


class Batch:
    """Many independent 2D grids iterated together (tvcut_batch_*)."""

    def __init__(self, dims_list, algo=AAR, dtype=F32, threshold=0.0, level_sets=None, stream=None):
        p = tvcut_default_params()
        p.algo = algo
        p.iterate_dtype = dtype
        p.threshold = threshold
        if level_sets is not None:
            p.level_sets = level_sets
        self.dims = [(int(h), int(w)) for h, w in dims_list]
        self.G = len(self.dims)
        self.dtype = dtype
        flat = (ctypes.c_int64 * (2 * self.G))(*[v for hw in self.dims for v in hw])
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(int(stream) if stream else 0)
        _bcheck(lib().tvcut_batch_create(self.G, flat, ctypes.byref(p), s, ctypes.byref(h)), None)
        self.h = h

    def close(self):
        if self.h:
            lib().tvcut_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_problem(self, g, w, a):
        pw, sw, dw, kw = _buf(w)
        _bcheck(lib().tvcut_batch_set_unary(self.h, int(g), pw, dw, sw), self.h)
        for k, ak in enumerate(a):
            pa, sa, da, ka = _buf(ak)
            _bcheck(lib().tvcut_batch_set_weights(self.h, int(g), k, pa, da, sa), self.h)

    def reset(self):
        _bcheck(lib().tvcut_batch_reset(self.h), self.h)

    def iterate(self, iters):
        out = (Stats * self.G)()
        code = _bcheck(lib().tvcut_batch_iterate(self.h, int(iters), out), self.h)
        return code, list(out)

    def cut(self, g):
        lab = np.empty(self.dims[g], dtype=np.uint8)
        st = Stats()
        _bcheck(lib().tvcut_batch_cut(self.h, int(g), ctypes.c_void_p(lab.ctypes.data), HOST, ctypes.byref(st)),
                self.h)
        return lab, st

    def state(self, g):
        s = np.empty((2,) + self.dims[g], dtype=np.float64 if self.dtype == F64 else np.float32)
        _bcheck(lib().tvcut_batch_get_state(self.h, int(g), ctypes.c_void_p(s.ctypes.data), HOST), self.h)
        return s

    def autotune(self):
        ch = (ctypes.c_int * 3)()
        _bcheck(lib().tvcut_batch_autotune(self.h, ch), self.h)
        return int(ch[0]), int(ch[1]), int(ch[2])

    def set_launch(self, threads, ctas_per_sm, step):
        """Chain-prox launch shape and step form (0 branchy, 1 predicated,
        2 padded weights), e.g. a saved autotune result."""
        _bcheck(lib().tvcut_batch_set_launch(self.h, int(threads), int(ctas_per_sm), int(step)), self.h)


def _ucheck(code, u):
    if code < 0:
        msg = lib().tvcut_unet_last_error(u)
        raise TvcutError(code, msg.decode() if msg else "")
    return code


class UNet:
    """The warm-start network (tvcut_unet_*).  Tensors are CUDA float32."""

    def __init__(self, base=32, batch=1, H=64, W=64, seed=0, stream=None):
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(int(stream) if stream else 0)
        _ucheck(lib().tvcut_unet_create(int(base), int(batch), int(H), int(W), ctypes.c_uint64(seed), s,
                                        ctypes.byref(h)), None)
        self.h = h
        self.shape = (batch, H, W)
        n = ctypes.c_int64()
        _ucheck(lib().tvcut_unet_num_params(self.h, ctypes.byref(n)), self.h)
        self.nparams = int(n.value)

    def close(self):
        if self.h:
            lib().tvcut_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def resize(self, batch, H, W):
        _ucheck(lib().tvcut_unet_resize(self.h, int(batch), int(H), int(W)), self.h)
        self.shape = (batch, H, W)

    def forward(self, x, out=None):
        """x: (batch, H, W, 3) float32 CUDA tensor; returns (batch, H, W, 2)."""
        import torch
        if out is None:
            out = torch.empty(self.shape + (2,), dtype=torch.float32, device=x.device)
        _ucheck(lib().tvcut_unet_forward(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr())),
                self.h)
        return out

    def backward(self, target):
        loss = ctypes.c_float()
        _ucheck(lib().tvcut_unet_backward(self.h, ctypes.c_void_p(target.data_ptr()), ctypes.byref(loss)), self.h)
        return float(loss.value)

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _ucheck(lib().tvcut_unet_adam(self.h, lr, beta1, beta2, eps), self.h)

    def params(self, which=0):
        out = np.empty(self.nparams, dtype=np.float32)
        _ucheck(lib().tvcut_unet_get_params(self.h, ctypes.c_void_p(out.ctypes.data), int(which)), self.h)
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        _ucheck(lib().tvcut_unet_set_params(self.h, ctypes.c_void_p(p.ctypes.data)), self.h)

    def predict_state(self, solver):
        """Warm-start `solver` (a 2D 4-connected Solver) from the network's
        predicted block duals, computed on the device from its problem."""
        _ucheck(lib().tvcut_unet_predict_state(self.h, solver.h), self.h)

    def set_engine(self, engine):
        """0: tcgen05 convolutions where the shape allows (default), 1: mma.sync."""
        _ucheck(lib().tvcut_unet_set_engine(self.h, int(engine)), self.h)
