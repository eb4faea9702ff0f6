"""Pins for the 8-connected oracle (oracle/conn8.py): the zig-zag
decomposition of Sec. 3.1 (Fig. 2, middle) holds every edge once and every
vertex once per block; max-flow on the edge list against brute force and
against the 4-connected oracle when the diagonals are 0; the limits of the
four methods against a graph-TV solver over all edges; thresholding at zero
against the min-cut (Sec. 2.3)."""
import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs


@pytest.fixture(scope="module")
def c8(orc):
    from oracle import conn8
    return conn8


def grid8(dims, seed, w_range=(-50, 50), a_range=(1, 20)):
    return inputs.uniform_grid8(dims, seed, w_range=w_range, a_range=a_range)


def graph_tv_prox(w, I, J, A, iters=60000):
    """argmin_x 1/2||x - w||^2 + sum_e a_e |x_i - x_j| by accelerated projected
    gradient on the edge duals (|p_e| <= a_e), x = w - B^T p; no chains."""
    wf = w.astype(np.float64).ravel()
    deg = np.bincount(np.concatenate([I, J]), minlength=wf.size).max()
    step = 1.0 / (2.0 * deg)
    p = np.zeros(A.size)
    q = p.copy()
    t = 1.0

    def primal(p):
        bt = np.zeros_like(wf)
        np.add.at(bt, I, p)
        np.add.at(bt, J, -p)
        return wf - bt

    for _ in range(iters):
        x = primal(q)
        pn = np.clip(q + step * (x[I] - x[J]), -A, A)
        tn = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        q = pn + ((t - 1) / tn) * (pn - p)
        p, t = pn, tn
    return primal(p).reshape(w.shape)


@pytest.mark.parametrize("dims", [(5, 6), (6, 5), (2, 7), (7, 2), (1, 4), (4, 1), (3, 3)])
def test_paths_hold_each_diagonal_edge_and_vertex_once(c8, dims):
    H, W = dims
    diag = set()
    for b in (2, 3):
        rows = c8.path_rows(H, W, b)
        # every vertex once per block
        seen = np.zeros((H, W), int)
        for q in range(H):
            for c in range(W):
                seen[rows[c, q], c] += 1
        assert np.all(seen == 1)
        for q in range(H):
            for c in range(W - 1):
                r0, r1 = rows[c, q], rows[c + 1, q]
                assert abs(r0 - r1) <= 1
                if r0 != r1:
                    e = ((r0, c), (r1, c + 1))
                    assert e not in diag
                    diag.add(e)
    want = {((r, c), (r + 1, c + 1)) for r in range(H - 1) for c in range(W - 1)}
    want |= {((r + 1, c), (r, c + 1)) for r in range(H - 1) for c in range(W - 1)}
    assert diag == want


def test_path_weights_follow_the_edges(c8):
    H, W = 6, 7
    w, a = grid8((H, W), 3)
    for b in (2, 3):
        rows, wz = c8.path_rows(H, W, b), c8.path_weights(a, H, W, b)
        for q in range(H):
            for c in range(W - 1):
                r0, r1 = rows[c, q], rows[c + 1, q]
                want = a[2][r0, c] if r1 == r0 + 1 else (a[3][r1, c] if r1 == r0 - 1 else 0.0)
                assert wz[c, q] == want


@pytest.mark.parametrize("dims", [(3, 4), (4, 4), (2, 6)])
def test_maxflow_against_bruteforce(c8, dims):
    for seed in range(15):
        w, a = grid8(dims, seed, w_range=(-12, 12), a_range=(0, 6))
        e, nmin = c8.bruteforce(w, a)
        for method in (0, 1):
            _, emf, smax = c8.maxflow(w, a, method)
            assert emf == e
            assert c8.energy(w, a, smax) == e
        e2, smin, smax = c8.min_cut(w, a)
        assert e2 == e and c8.energy(w, a, smin) == e
        assert np.all(smin <= smax)


def test_zero_diagonals_reduce_to_four_connected(c8, orc):
    w, a = grid8((9, 11), 4)
    a = [a[0], a[1], np.zeros_like(a[2]), np.zeros_like(a[3])]
    assert c8.maxflow(w, a)[1] == orc.maxflow(w, a[:2])[1]
    lab = (np.random.default_rng(1).random(w.shape) > 0.5).astype(np.uint8)
    assert c8.energy(w, a, lab) == orc.energy(w, a[:2], lab)
    x = np.random.default_rng(2).normal(size=w.shape)
    assert abs(c8.tv_value(a, x) - orc.tv_value(a[:2], x)) < 1e-9
    _, x4 = orc.iterate(0, w, a[:2], orc.cold_state(0, w), 3000)
    _, x8 = c8.iterate(0, w, a, c8.cold_state(0, w), 3000)
    np.testing.assert_allclose(x8, x4, atol=1e-6)


@pytest.mark.parametrize("dims", [(5, 6), (4, 7)])
def test_limits_agree_with_graph_tv(c8, dims):
    w, a = grid8(dims, 21, w_range=(-6, 6), a_range=(1, 3))
    I, J, A = c8.edges(dims, a)
    ref = graph_tv_prox(w, I, J, A)
    for algo in (0, 1, 2, 3):
        _, x = c8.iterate(algo, w, a, c8.cold_state(algo, w), 3000)
        np.testing.assert_allclose(x, ref, atol=2e-6, err_msg=f"algo {algo}")


def test_threshold_gives_min_cut(c8):
    w, a = grid8((14, 12), 5)
    E, smin, smax = c8.min_cut(w, a)
    _, x = c8.iterate(0, w, a, c8.cold_state(0, w), 4000)
    assert c8.energy(w, a, (x > 1e-7).astype(np.uint8)) == E
    assert np.array_equal((x > 1e-7).astype(np.uint8), smin)
    assert np.array_equal((x >= -1e-7).astype(np.uint8), smax)


def test_fista_starts_as_ap(c8):
    w, a = grid8((7, 9), 8)
    for k in (1, 2):
        _, xf = c8.iterate(3, w, a, c8.cold_state(3, w), k)
        _, xa = c8.iterate(1, w, a, c8.cold_state(1, w), k)
        np.testing.assert_allclose(xf, xa, atol=1e-12)
