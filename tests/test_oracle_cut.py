"""Pins for the oracle's exact min-cut: brute force, Edmonds-Karp and
push-relabel against each other, hand-derived cases, closed forms and a
Viterbi dynamic programme on chains written here (problem (D), Eq. 2)."""
import json
import os

import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def _weights(dims, a):
    return [np.asarray(x, dtype=np.float64).reshape(inputs.compact_shape(dims, k)) for k, x in enumerate(a)]


def test_hand_cases(orc):
    for c in json.load(open(GOLDEN))["energy"]:
        dims = tuple(c["dims"])
        w = np.asarray(c["w"], dtype=np.float64)
        a = _weights(dims, c["a"])
        lab = np.asarray(c["labels"], dtype=np.uint8)
        assert orc.energy(w, a, lab) == c["emin"], c["why"]
        e, _, smin, _ = orc.bruteforce(w, a)
        assert e == c["emin"], c["why"]
        assert np.array_equal(smin, lab), c["why"]
        assert orc.maxflow(w, a, 0)[1] == c["emin"]
        assert orc.maxflow(w, a, 1)[1] == c["emin"]


def test_energy_closed_forms(orc):
    w, a = inputs.uniform_grid((5, 6), 1)
    zero = np.zeros(w.shape, np.uint8)
    one = np.ones(w.shape, np.uint8)
    assert orc.energy(w, a, zero) == 0
    assert orc.energy(w, a, one) == -w.sum()
    cb = (np.indices(w.shape).sum(0) % 2).astype(np.uint8)
    # a checkerboard cuts every edge
    assert orc.energy(w, a, cb) == sum(x.sum() for x in a) - (w * cb).sum()
    x = np.arange(30, dtype=np.float64).reshape(5, 6)
    assert orc.tv_value(a, np.full((5, 6), 2.0)) == 0
    # f(x) for x = 6 h + col: horizontal steps 1, vertical steps 6
    assert orc.tv_value(a, x) == a[1].sum() * 1 + a[0].sum() * 6


def test_zero_weights_closed_form(orc):
    """a = 0: E* = -sum max(w, 0), minimal minimiser {w > 0}, maximal {w >= 0}."""
    w, a = inputs.uniform_grid((4, 4), 3, w_range=(-3, 3))
    a = [np.zeros_like(x) for x in a]
    e, cnt, smin, smax = orc.bruteforce(w, a)
    assert e == -np.maximum(w, 0).sum()
    assert np.array_equal(smin, (w > 0).astype(np.uint8))
    assert np.array_equal(smax, (w >= 0).astype(np.uint8))
    assert cnt == 2 ** int((w == 0).sum())
    E, mn, mx = orc.min_cut(w, a)
    assert E == e and np.array_equal(mn, smin) and np.array_equal(mx, smax)


def chain_dp(w, a):
    """Viterbi over l_i in {0,1} on a chain: min sum a_k [l_k != l_{k+1}] - w.l"""
    best = np.array([0.0, -w[0]])
    for i in range(1, w.size):
        nb = np.empty(2)
        for l in (0, 1):
            nb[l] = min(best[l], best[1 - l] + a[i - 1]) - (w[i] if l else 0.0)
        best = nb
    return best.min()


def test_chain_dp(orc):
    for seed in range(40):
        w, a = inputs.uniform_grid((1, 37), seed)
        e = chain_dp(w[0].astype(float), a[1][0].astype(float))
        assert orc.maxflow(w, a, 1)[1] == e
        assert orc.maxflow(w, a, 0)[1] == e


@pytest.mark.parametrize("dims", [(4, 4), (3, 5), (3, 3, 2), (2, 2, 4), (1, 16)])
def test_bruteforce_vs_maxflow(orc, dims):
    for seed in range(60):
        w, a = inputs.uniform_grid(dims, seed)
        e, cnt, smin, smax = orc.bruteforce(w, a)
        f0, e0, sm0 = orc.maxflow(w, a, 0)
        f1, e1, sm1 = orc.maxflow(w, a, 1)
        assert e == e0 == e1
        assert f0 == f1 == e + np.maximum(w, 0).sum()
        assert np.array_equal(sm0, smax) and np.array_equal(sm1, smax)
        E, mn, mx = orc.min_cut(w, a)
        assert np.array_equal(mn, smin) and np.array_equal(mx, smax)
        assert orc.energy(w, a, smin) == e and orc.energy(w, a, smax) == e


def test_bruteforce_catches_planted_mistake(orc):
    """A labelling one flip away from the optimum costs more (brute force is
    the minimum, not just some labelling)."""
    w, a = inputs.uniform_grid((4, 4), 7)
    e, _, smin, _ = orc.bruteforce(w, a)
    for i in range(16):
        lab = smin.copy().ravel()
        lab[i] ^= 1
        assert orc.energy(w, a, lab.reshape(4, 4)) >= e


def test_push_relabel_vs_edmonds_karp_mid(orc):
    for seed in range(3):
        w, a = inputs.uniform_grid((24, 31), seed)
        assert orc.maxflow(w, a, 0)[1] == orc.maxflow(w, a, 1)[1]
        w, a = inputs.uniform_grid((6, 7, 8), seed)
        r0, r1 = orc.maxflow(w, a, 0), orc.maxflow(w, a, 1)
        assert r0[1] == r1[1] and np.array_equal(r0[2], r1[2])


def test_maxflow_rejects_bad_input(orc):
    w, a = inputs.uniform_grid((3, 3), 0)
    with pytest.raises(ValueError):
        orc.maxflow(w.astype(float) + 0.5, a)
    a2 = [x.astype(float) for x in a]
    a2[0][0, 0] = -1
    with pytest.raises(ValueError):
        orc.maxflow(w, a2)
