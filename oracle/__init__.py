"""CPU oracle for the min-cut-by-TV-denoising method (FP64, plain C).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1503_01563_gb300``; the two meet only through
the seeded input generators, which hold none of the method's arithmetic.

Functions and the passages of "Convex Optimization for Parallel Energy
Minimization" they follow:

- ``tv1d_prox``         exact weighted 1D-TV prox by the taut string (Sec. 3.2)
- ``tv1d_certificate``  Lagrangian certificate of a chain prox (Sec. 3.2, 2.3)
- ``project_block``     Pi_{K_k} = I - prox on every chain of one block
                        (Sec. 3.1, Sec. 4.2)
- ``iterate``           AAR (Eq. 3), AP (Sec. 4.2), BCD and FISTA (Sec. 4.1)
- ``cold_state``        z = 0 (AAR), lambda = Pi_L(0) (AP), y = 0 (BCD, FISTA)
- ``tv_value``          f(x) = sum_e a_e |x_i - x_j| (Eq. 2)
- ``energy``            E(l) = f(l) - w^T l (problem (D))
- ``bruteforce``        min over all 2^n labellings (problem (D))
- ``maxflow``           s-t max-flow / min-cut of the energy (Eq. 2 as a cut)
- ``conn8``             the same for 2D 8-connected grids: edge list, the
                        zig-zag decomposition (Sec. 3.1, Fig. 2), the four
                        methods with four blocks, energy, TV, max-flow on an
                        edge list, brute force

Arrays are numpy; weights are passed per axis in compact layout (the grid's
shape with dims[k]-1 along axis k).  Parity is pinned for every function by
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["tv1d.c", "dr.c", "maxflow.c"]
_lib = None

AAR, AP, BCD, FISTA = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP over chains, like the paper's
    implementation in Sec. 5.1).  Returns the library path."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(_HERE, "oracle.h")])
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.oracle_tv1d_prox.argtypes = [i64, P, P, P]
    lib.oracle_tv1d_prox.restype = ctypes.c_int
    lib.oracle_tv1d_certificate.argtypes = [i64, P, P, P, P]
    lib.oracle_tv1d_certificate.restype = None
    lib.oracle_project_block.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P, ctypes.c_int]
    lib.oracle_project_block.restype = None
    lib.oracle_iterate.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, i64, P, ctypes.c_int]
    lib.oracle_iterate.restype = ctypes.c_int
    lib.oracle_cold_state.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
    lib.oracle_cold_state.restype = None
    lib.oracle_tv_value.argtypes = [ctypes.c_int, P, P, P]
    lib.oracle_tv_value.restype = ctypes.c_double
    lib.oracle_energy.argtypes = [ctypes.c_int, P, P, P, P]
    lib.oracle_energy.restype = ctypes.c_double
    lib.oracle_bruteforce.argtypes = [ctypes.c_int, P, P, P, P, P, P, P]
    lib.oracle_bruteforce.restype = ctypes.c_int
    lib.oracle_maxflow.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
    lib.oracle_maxflow.restype = ctypes.c_int
    lib.oracle_maxflow_edges.argtypes = [ctypes.c_int, i64, P, i64, P, P, P, P, P, P]
    lib.oracle_maxflow_edges.restype = ctypes.c_int
    _lib = lib
    return lib


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class _Weights:
    """Keeps compact per-axis FP64 weight arrays alive and exposes a double**."""

    def __init__(self, dims, a):
        if len(a) != len(dims):
            raise ValueError("need one weight array per axis")
        self.arrs = []
        for k, ak in enumerate(a):
            ak = _f64(ak)
            want = tuple(d - 1 if j == k else d for j, d in enumerate(dims))
            if ak.shape != want:
                raise ValueError(f"axis {k} weights must have shape {want}, got {ak.shape}")
            self.arrs.append(ak)
        self.pp = (ctypes.c_void_p * len(dims))(*[a.ctypes.data for a in self.arrs])


def _dims(shape):
    d = np.ascontiguousarray(np.asarray(shape, dtype=np.int64))
    return d, len(shape)


def tv1d_prox(v, a) -> np.ndarray:
    v = _f64(v).ravel()
    a = _f64(a).ravel()
    m = v.size
    if a.size != max(m - 1, 0):
        raise ValueError("a must have m-1 entries")
    x = np.empty(m, dtype=np.float64)
    if m and _load().oracle_tv1d_prox(m, _ptr(v), _ptr(a if a.size else np.zeros(1)), _ptr(x)) != 0:
        raise RuntimeError("oracle_tv1d_prox failed")
    return x


def tv1d_certificate(v, a, x) -> np.ndarray:
    v, a, x = _f64(v).ravel(), _f64(a).ravel(), _f64(x).ravel()
    out = np.zeros(3, dtype=np.float64)
    _load().oracle_tv1d_certificate(v.size, _ptr(v), _ptr(a if a.size else np.zeros(1)), _ptr(x), _ptr(out))
    return out


def project_block(v, a_axis, axis: int, nthreads: int = 1) -> np.ndarray:
    v = _f64(v)
    dims, nd = _dims(v.shape)
    a_axis = _f64(a_axis)
    y = np.empty_like(v)
    _load().oracle_project_block(nd, _ptr(dims), axis, _ptr(v), _ptr(a_axis), _ptr(y), nthreads)
    return y


def cold_state(algo: int, w) -> np.ndarray:
    w = _f64(w)
    dims, nd = _dims(w.shape)
    s = np.empty((nd,) + w.shape, dtype=np.float64)
    _load().oracle_cold_state(algo, nd, _ptr(dims), _ptr(w), _ptr(s))
    return s


def iterate(algo: int, w, a, state, iters: int, nthreads: int = 1):
    """Run `iters` iterations; returns (new_state, x) with x = w - sum_k y_k
    of the last shadow.  `state` has shape (ndim,) + grid shape.  FISTA's
    momentum starts afresh at every call, so run it in one call."""
    w = _f64(w)
    dims, nd = _dims(w.shape)
    wt = _Weights(w.shape, a)
    s = np.array(state, dtype=np.float64, copy=True, order="C")
    if s.shape != (nd,) + w.shape:
        raise ValueError("bad state shape")
    x = np.empty_like(w)
    rc = _load().oracle_iterate(algo, nd, _ptr(dims), _ptr(w), wt.pp, _ptr(s), int(iters), _ptr(x), nthreads)
    if rc != 0:
        raise RuntimeError("oracle_iterate failed")
    return s, x


def tv_value(a, x) -> float:
    x = _f64(x)
    dims, nd = _dims(x.shape)
    wt = _Weights(x.shape, a)
    return float(_load().oracle_tv_value(nd, _ptr(dims), wt.pp, _ptr(x)))


def energy(w, a, labels) -> float:
    w = _f64(w)
    dims, nd = _dims(w.shape)
    wt = _Weights(w.shape, a)
    lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8))
    return float(_load().oracle_energy(nd, _ptr(dims), _ptr(w), wt.pp, _ptr(lab)))


def bruteforce(w, a):
    """Returns (E*, number of minimisers, S_min, S_max) over all 2^n labellings."""
    w = _f64(w)
    dims, nd = _dims(w.shape)
    wt = _Weights(w.shape, a)
    emin = np.zeros(1, dtype=np.float64)
    cnt = np.zeros(1, dtype=np.int64)
    smin = np.zeros(w.shape, dtype=np.uint8)
    smax = np.zeros(w.shape, dtype=np.uint8)
    rc = _load().oracle_bruteforce(nd, _ptr(dims), _ptr(w), wt.pp, _ptr(emin), _ptr(cnt), _ptr(smin), _ptr(smax))
    if rc != 0:
        raise ValueError("bruteforce needs 1 <= n <= 26")
    return float(emin[0]), int(cnt[0]), smin, smax


def maxflow(w, a, method: int = 1):
    """Returns (flow, E*, S_max) for integral data; method 0 = Edmonds-Karp,
    1 = FIFO push-relabel."""
    w = _f64(w)
    dims, nd = _dims(w.shape)
    wt = _Weights(w.shape, a)
    flow = np.zeros(1, dtype=np.int64)
    emin = np.zeros(1, dtype=np.int64)
    smax = np.zeros(w.shape, dtype=np.uint8)
    rc = _load().oracle_maxflow(method, nd, _ptr(dims), _ptr(w), wt.pp, _ptr(flow), _ptr(emin), _ptr(smax))
    if rc != 0:
        raise ValueError("maxflow needs integral w and integral a >= 0")
    return int(flow[0]), int(emin[0]), smax


def min_cut(w, a, method: int = 1):
    """E* with both the minimal and the maximal minimising labellings.  The
    minimal one is the complement of the maximal minimiser of the mirrored
    energy E_{-w} (E_w(1 - l) = E_{-w}(l) - sum w)."""
    _, e, smax = maxflow(w, a, method)
    _, _, smax_neg = maxflow(-_f64(w), a, method)
    smin = (1 - smax_neg).astype(np.uint8)
    return e, smin, smax


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
