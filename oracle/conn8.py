"""Oracle for 2D 8-connected grids (FP64).  TEST INFRASTRUCTURE ONLY: only
``tests/`` may import it; it shares no code with the CUDA library.

Sec. 3.1 splits the 2D 8-connected grid into vertical lines, horizontal lines
and zig-zag paths (Fig. 2, middle).  Weights come as four arrays:

- ``a[0]`` (H-1, W): vertical edges (r, c)-(r+1, c);
- ``a[1]`` (H, W-1): horizontal edges (r, c)-(r, c+1);
- ``a[2]`` (H-1, W-1): diagonal edges (r, c)-(r+1, c+1);
- ``a[3]`` (H-1, W-1): anti-diagonal edges (r, c+1)-(r+1, c).

The four blocks: 0 = columns, 1 = rows, 2 = zig-zag paths between rows
(2p, 2p+1), 3 = zig-zag paths between rows (2p+1, 2p+2).  Between two rows
(t, t+1) the path that starts at (t, 0) visits row t in even columns and
row t+1 in odd ones, and the path that starts at (t+1, 0) does the opposite;
consecutive vertices of either path are joined by a diagonal or an
anti-diagonal edge, and the two paths together hold each such edge between
the two rows exactly once.  A row with no partner in a block (row 0 in block
3, the last row in one of the two) forms paths without edges there.

Path q of block 2 or 3 starts at (q, 0); its vertex in column c is
(row(q, c), c).  Each block's projection gathers its paths into a (W, H)
array with path q as column q and runs the C chain projection on it.  The
methods of Sec. 4 then follow the same steps as ``dr.c``: Pi_K blockwise,
Pi_L(u)_k = u_k + (w - sum u)/r with r = 4.
"""
from __future__ import annotations

import numpy as np

from . import _load, _ptr, _f64, project_block, tv1d_prox  # noqa: F401

AAR, AP, BCD, FISTA = 0, 1, 2, 3
R = 4


def weight_shapes(H: int, W: int):
    return [(H - 1, W), (H, W - 1), (H - 1, W - 1), (H - 1, W - 1)]


def edges(dims, a):
    """Undirected edges (i, j, a_e) of the 8-connected grid, each once."""
    H, W = dims
    idx = np.arange(H * W).reshape(H, W)
    I = [idx[:-1, :].ravel(), idx[:, :-1].ravel(), idx[:-1, :-1].ravel(), idx[:-1, 1:].ravel()]
    J = [idx[1:, :].ravel(), idx[:, 1:].ravel(), idx[1:, 1:].ravel(), idx[1:, :-1].ravel()]
    A = [np.asarray(x, dtype=np.float64).ravel() for x in a]
    return np.concatenate(I), np.concatenate(J), np.concatenate(A)


def path_rows(H: int, W: int, block: int) -> np.ndarray:
    """rows[c, q] = row(q, c): the row of path q's vertex in column c, for
    block 2 (pairs starting at even rows) or 3 (at odd rows)."""
    b = block - 2
    q = np.arange(H)
    top = ((q - b) % 2 == 0) & (q + 1 <= H - 1) & (q >= b)
    bottom = ((q - b) % 2 == 1) & (q - 1 >= b)
    partner = np.where(top, q + 1, np.where(bottom, q - 1, q))
    c = np.arange(W)[:, None]
    return np.where(c % 2 == 0, q[None, :], partner[None, :])


def path_weights(a, H: int, W: int, block: int) -> np.ndarray:
    """wz[c, q]: weight of the edge between path q's vertices in columns c and
    c+1 (diagonal if the path steps down, anti-diagonal if up, 0 if it stays)."""
    rows = path_rows(H, W, block)
    r0, r1 = rows[:-1], rows[1:]
    c = np.arange(W - 1)[:, None] + np.zeros((1, H), dtype=int)
    ad, aa = np.asarray(a[2], np.float64), np.asarray(a[3], np.float64)
    wz = np.zeros((W - 1, H))
    down = r1 == r0 + 1
    up = r1 == r0 - 1
    wz[down] = ad[r0[down], c[down]]
    wz[up] = aa[r1[up], c[up]]
    return wz


def project(v, a, block: int, nthreads: int = 1) -> np.ndarray:
    """Pi_{K_k}(v) = v - prox_{f_k}(v) for one block (chains independent)."""
    v = _f64(v)
    H, W = v.shape
    if block in (0, 1):
        return project_block(v, a[block], block, nthreads)
    if W == 1:
        return np.zeros_like(v)
    rows = path_rows(H, W, block)
    cols = np.arange(W)[:, None] + np.zeros((1, H), dtype=int)
    z = v[rows, cols]                                   # (W, H): path q down column q
    yz = project_block(z, path_weights(a, H, W, block), 0, nthreads)
    y = np.empty_like(v)
    y[rows, cols] = yz
    return y


def project_K(s, a, nthreads: int = 1) -> np.ndarray:
    return np.stack([project(s[k], a, k, nthreads) for k in range(R)])


def project_L(w, u) -> np.ndarray:
    """Pi_L(u)_k = u_k + (w - sum_j u_j) / r (Eq. dualA)."""
    return u + (_f64(w) - u.sum(0)) / R


def cold_state(algo: int, w) -> np.ndarray:
    w = _f64(w)
    s = np.zeros((R,) + w.shape)
    return project_L(w, s) if algo == AP else s


def iterate(algo: int, w, a, state, iters: int, nthreads: int = 1):
    """`iters` iterations of AAR (Eq. 3), AP (Sec. 4.2), BCD or FISTA
    (Sec. 4.1) with the four blocks; returns (state, x), x = w - sum_k y_k of
    the last dual iterate.  FISTA's momentum starts afresh at every call."""
    w = _f64(w)
    s = np.array(state, dtype=np.float64, copy=True)
    y = s.copy() if algo in (BCD, FISTA) else None
    u, t = s.copy(), 1.0
    for _ in range(iters):
        if algo == AAR:
            y = project_K(s, a, nthreads)
            rk = 2 * y - s                                  # R_K z
            rl = 2 * project_L(w, rk) - rk                  # R_L R_K z
            s = 0.5 * (rl + s)
        elif algo == AP:
            y = project_K(s, a, nthreads)
            s = project_L(w, y)
        elif algo == BCD:
            for k in range(R):
                v = w - (s.sum(0) - s[k])
                s[k] = project(v, a, k, nthreads)
            y = s.copy()
        else:
            yn = project_K(project_L(w, u), a, nthreads)
            tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            u = yn + ((t - 1.0) / tn) * (yn - s)
            s, t = yn, tn
            y = s.copy()
    if y is None:
        y = s.copy() if algo in (BCD, FISTA) else project_K(s, a, nthreads)
    return s, w - y.sum(0)


def tv_value(a, x) -> float:
    x = _f64(x)
    I, J, A = edges(x.shape, a)
    x = x.ravel()
    return float((A * np.abs(x[I] - x[J])).sum())


def energy(w, a, labels) -> int | float:
    """E(l) = sum_e a_e [l_i != l_j] - w^T l (problem (D)) over all 8-connected edges."""
    w = _f64(w)
    I, J, A = edges(w.shape, a)
    l = np.asarray(labels).ravel().astype(np.int64)
    e = float((A * (l[I] != l[J])).sum() - (w.ravel() * l).sum())
    return int(round(e)) if float(e).is_integer() else e


def maxflow(w, a, method: int = 1):
    """(flow, E*, S_max) by max-flow on the 8-connected graph (integral data)."""
    w = _f64(w)
    I, J, A = edges(w.shape, a)
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    A = np.ascontiguousarray(A, dtype=np.float64)
    flow = np.zeros(1, dtype=np.int64)
    emin = np.zeros(1, dtype=np.int64)
    smax = np.zeros(w.shape, dtype=np.uint8)
    rc = _load().oracle_maxflow_edges(method, np.int64(w.size), _ptr(w), np.int64(I.size), _ptr(I), _ptr(J),
                                      _ptr(A), _ptr(flow), _ptr(emin), _ptr(smax))
    if rc != 0:
        raise ValueError("maxflow needs integral w and integral a >= 0")
    return int(flow[0]), int(emin[0]), smax


def min_cut(w, a, method: int = 1):
    """E* with the minimal and maximal minimisers (as oracle.min_cut)."""
    _, e, smax = maxflow(w, a, method)
    _, _, smax_neg = maxflow(-_f64(w), a, method)
    return e, (1 - smax_neg).astype(np.uint8), smax


def bruteforce(w, a):
    """min over all 2^n labellings (n <= 20): (E*, number of minimisers)."""
    w = _f64(w)
    n = w.size
    I, J, A = edges(w.shape, a)
    L = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int8)
    E = (A[None, :] * (L[:, I] != L[:, J])).sum(1) - L @ w.ravel()
    best = E.min()
    return int(round(best)), int((E == best).sum())
