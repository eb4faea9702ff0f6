"""Pins for the oracle's chain prox (Sec. 3.2) and block projection (Sec. 3.1).

Nothing here re-calls the oracle's own construction: each check compares it
with something the mathematics fixes independently -- hand-derived cases,
closed forms, symmetries of the prox, a projected-gradient solver of the dual
box QP written here in numpy, and the Lagrangian certificate (itself pinned by
planted mistakes).
"""
import json
import os

import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def objective(v, a, x):
    return 0.5 * np.sum((x - v) ** 2) + np.sum(a * np.abs(np.diff(x)))


def dual_box_qp(v, a, iters=200000):
    """min_u 1/2 ||v - D^T u||^2 s.t. |u| <= a by accelerated projected
    gradient; x = v - D^T u with (D^T u)_i = u_{i-1} - u_i."""
    m = v.size
    if m == 1:
        return v.copy()
    u = np.zeros(m - 1)
    yk = u.copy()
    t = 1.0
    step = 0.25                      # 1/L, L = ||D D^T|| <= 4

    def primal(u):
        dtu = np.zeros(m)
        dtu[1:] += u
        dtu[:-1] -= u
        return v - dtu

    for _ in range(iters):
        x = primal(yk)
        grad = -(x[1:] - x[:-1])     # d/du of 1/2||v - D^T u||^2 = -D x
        un = np.clip(yk - step * grad, -a, a)
        tn = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        yk = un + ((t - 1) / tn) * (un - u)
        u, t = un, tn
    return primal(u)


def test_hand_cases(orc):
    for c in json.load(open(GOLDEN))["tv1d"]:
        x = orc.tv1d_prox(c["v"], c["a"])
        np.testing.assert_allclose(x, c["x"], atol=1e-12, err_msg=c["why"])


@pytest.mark.parametrize("m", [1, 2, 3, 5, 31, 33, 100, 257])
def test_certificate_zero_on_random_chains(orc, m):
    for seed in range(20):
        v, a = inputs.random_chain(m, seed)
        if seed % 4 == 1:
            a[::3] = 0.0              # some zero weights
        if seed % 4 == 2:
            v = np.round(v)            # ties
        x = orc.tv1d_prox(v, a)
        cert = orc.tv1d_certificate(v, a, x)
        scale = 1.0 + np.abs(v).sum()
        assert cert[0] <= 1e-9 * scale
        assert cert[1] <= 1e-9 * scale
        assert abs(cert[2]) <= 1e-8 * scale


def test_certificate_catches_planted_mistakes(orc):
    v, a = inputs.random_chain(40, 3)
    x = orc.tv1d_prox(v, a)
    assert np.all(np.abs(orc.tv1d_certificate(v, a, x)) < 1e-8)
    # shifted solution: the end multiplier is no longer zero
    assert orc.tv1d_certificate(v, a, x + 0.1)[0] > 1e-3
    # one element perturbed inside a flat run: feasibility or complementarity breaks
    bad = x.copy()
    bad[20] += 0.5
    c = orc.tv1d_certificate(v, a, bad)
    assert c[0] > 1e-3 or c[1] > 1e-3 or abs(c[2]) > 1e-3
    # the prox for weights 2a is not the prox for a
    x2 = orc.tv1d_prox(v, 2 * a)
    c = orc.tv1d_certificate(v, a, x2)
    assert c[1] > 1e-3 or abs(c[2]) > 1e-3
    # sign flip of the jumps (solution of the wrong sign convention)
    flip = np.mean(x) - (x - np.mean(x))
    c = orc.tv1d_certificate(v, a, flip)
    assert max(c[0], c[1], abs(c[2])) > 1e-3


@pytest.mark.parametrize("m", [2, 3, 7, 20, 40])
def test_matches_dual_projected_gradient(orc, m):
    for seed in range(6):
        v, a = inputs.random_chain(m, 100 + seed, scale=3.0, a_scale=2.0)
        x = orc.tv1d_prox(v, a)
        xq = dual_box_qp(v, a, iters=20000 if m <= 7 else 120000)
        np.testing.assert_allclose(x, xq, atol=1e-7)


def test_closed_forms(orc):
    g = np.random.default_rng(5)
    for _ in range(50):
        v1, v2 = g.normal(size=2) * 5
        a = g.uniform(0, 4)
        d = min(a, abs(v1 - v2) / 2)
        s = np.sign(v1 - v2)
        np.testing.assert_allclose(orc.tv1d_prox([v1, v2], [a]), [v1 - s * d, v2 + s * d], atol=1e-12)
    v = g.normal(size=30)
    np.testing.assert_allclose(orc.tv1d_prox(v, np.zeros(29)), v, atol=0)
    big = np.full(29, np.abs(v).sum() + 1)
    np.testing.assert_allclose(orc.tv1d_prox(v, big), np.full(30, v.mean()), atol=1e-12)


def test_symmetries(orc):
    for seed in range(10):
        v, a = inputs.random_chain(50, 200 + seed)
        x = orc.tv1d_prox(v, a)
        np.testing.assert_allclose(orc.tv1d_prox(v + 3.25, a), x + 3.25, atol=1e-9)
        np.testing.assert_allclose(orc.tv1d_prox(-v, a), -x, atol=1e-9)
        np.testing.assert_allclose(orc.tv1d_prox(v[::-1], a[::-1]), x[::-1], atol=1e-9)
        np.testing.assert_allclose(orc.tv1d_prox(2.5 * v, 2.5 * a), 2.5 * x, atol=1e-9)


def test_prox_is_a_minimiser(orc):
    g = np.random.default_rng(9)
    for seed in range(10):
        v, a = inputs.random_chain(25, 300 + seed)
        x = orc.tv1d_prox(v, a)
        f0 = objective(v, a, x)
        for _ in range(200):
            p = x + g.normal(size=x.size) * 10 ** g.uniform(-4, 0)
            assert objective(v, a, p) >= f0 - 1e-9


def test_block_projection_is_in_K(orc):
    """y = Pi_{K_k}(v) lies in K_k: on every chain y = D^T u with |u| <= a,
    i.e. the chain sums of y vanish and |running sum| <= a (Sec. 2.2, 3.1)."""
    for dims, axis in [((7, 9), 0), ((7, 9), 1), ((4, 5, 6), 0), ((4, 5, 6), 1), ((4, 5, 6), 2)]:
        w, a = inputs.uniform_grid(dims, 11 + axis)
        v = w.astype(np.float64) * 0.7
        y = orc.project_block(v, a[axis], axis)
        ym = np.moveaxis(y, axis, -1)
        am = np.moveaxis(a[axis].astype(np.float64), axis, -1)
        cs = np.cumsum(ym, axis=-1)
        np.testing.assert_allclose(cs[..., -1], 0, atol=1e-9)
        # with u_k = -(y_0 + ... + y_k) the bound is |u_k| <= a_k
        assert np.all(np.abs(cs[..., :-1]) <= am + 1e-9)
        # and each chain is the prox of its own slice
        vm = np.moveaxis(v, axis, -1).reshape(-1, dims[axis])
        for c in range(0, vm.shape[0], 5):
            xc = orc.tv1d_prox(vm[c], am.reshape(-1, dims[axis] - 1)[c])
            np.testing.assert_allclose(ym.reshape(-1, dims[axis])[c], vm[c] - xc, atol=1e-12)


def test_projection_idempotent_and_nonexpansive(orc):
    w, a = inputs.uniform_grid((6, 11), 4)
    v = w.astype(np.float64)
    y = orc.project_block(v, a[1], 1)
    np.testing.assert_allclose(orc.project_block(y, a[1], 1), y, atol=1e-9)
    v2 = v + np.random.default_rng(0).normal(size=v.shape)
    y2 = orc.project_block(v2, a[1], 1)
    assert np.linalg.norm(y2 - y) <= np.linalg.norm(v2 - v) + 1e-9
