"""Pins for the oracle's chain prox by a sequence of chain min-cuts
(oracle/parametric.py, Sec. 3.2 "Message passing"): the hand-derived chain
cases, the closed forms, the taut-string oracle on random chains, brute-force
min-marginals of the message passing, exact ties at an interval's mean, the
bound on the number of min-cuts, and planted mistakes that the pins catch."""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import parametric as par

HERE = os.path.dirname(os.path.abspath(__file__))


def golden_chains():
    return json.load(open(os.path.join(HERE, "golden", "hand_cases.json")))["tv1d"]


@pytest.mark.parametrize("case", golden_chains(), ids=lambda c: str(c["v"]))
def test_hand_derived_cases_exact(case):
    x, _ = par.tv1d_prox_parametric(case["v"], case["a"])
    assert [Fraction(t) for t in case["x"]] == x


def test_closed_forms():
    rng = np.random.default_rng(1)
    v = rng.integers(-20, 21, size=9)
    x, _ = par.tv1d_prox_parametric(v, [0] * 8)                     # a = 0: identity
    assert x == [Fraction(int(t)) for t in v]
    x, cuts = par.tv1d_prox_parametric(v, [10 ** 6] * 8)            # a >= sum |v|: the mean
    assert x == [Fraction(int(v.sum()), 9)] * 9 and cuts == 1
    assert par.tv1d_prox_parametric([Fraction(7, 3)], [])[0] == [Fraction(7, 3)]
    for v1, v2, a in [(5, -5, 2), (5, -5, 7), (-3, 4, 1), (2, 2, 3)]:   # m = 2 closed form
        d = min(Fraction(a), Fraction(abs(v1 - v2), 2))
        s = 1 if v1 > v2 else -1
        x, _ = par.tv1d_prox_parametric([v1, v2], [a])
        assert x == [v1 - s * d, v2 + s * d]


def test_matches_taut_string_oracle(orc):
    """Random chains with plateaus and zero weights: the exact parametric
    solution agrees with the FP64 taut string to rounding."""
    rng = np.random.default_rng(2)
    for trial in range(60):
        m = int(rng.integers(1, 40))
        v = np.round(rng.normal(0, 8, size=m) + np.cumsum(rng.integers(-1, 2, size=m) * 6.0), 3)
        a = np.round(rng.uniform(0, 5, size=m - 1), 3)
        a[rng.random(a.shape) < 0.15] = 0.0
        x, _ = par.tv1d_prox_parametric(v, a)
        ref = orc.tv1d_prox(v, a)
        np.testing.assert_allclose([float(t) for t in x], ref, rtol=0, atol=1e-9 * max(1.0, np.abs(v).max()))


def test_integer_chains_with_ties_at_the_mean(orc):
    """Integer data makes a level of x* equal an interval's mean often; those
    elements are fixed exactly (M_i(1) = M_i(0)).  Checked against the taut
    string and the Lagrangian certificate."""
    rng = np.random.default_rng(3)
    ties = 0
    for trial in range(200):
        m = int(rng.integers(2, 14))
        v = rng.integers(-6, 7, size=m)
        a = rng.integers(0, 4, size=m - 1)
        x, _ = par.tv1d_prox_parametric(v, a)
        xf = np.array([float(t) for t in x])
        np.testing.assert_allclose(xf, orc.tv1d_prox(v, a), atol=1e-9)
        cert = orc.tv1d_certificate(v, a, xf)
        assert cert[0] < 1e-9 and cert[1] < 1e-9
        vp = [Fraction(int(t)) for t in v]
        alpha = sum(vp) / m
        mm = par.chain_min_cut_min_marginals(vp, [Fraction(int(t)) for t in a], alpha)
        ties += sum(1 for m0, m1 in mm if m0 == m1) > 0 and any(m0 != m1 for m0, m1 in mm)
    assert ties > 0                                   # partial ties do occur in this set


def test_message_passing_min_marginals_brute_force():
    """M_i(b) equals the minimum of E_alpha over all labellings with l_i = b,
    and thresholding M gives the minimal and maximal minimisers."""
    rng = np.random.default_rng(4)
    for trial in range(40):
        m = int(rng.integers(1, 10))
        vp = [Fraction(int(t)) for t in rng.integers(-9, 10, size=m)]
        a = [Fraction(int(t)) for t in rng.integers(0, 5, size=m - 1)]
        alpha = Fraction(int(rng.integers(-4, 5)), int(rng.integers(1, 4)))
        mm = par.chain_min_cut_min_marginals(vp, a, alpha)
        labs = list(itertools.product((0, 1), repeat=m))
        energies = {l: par.chain_min_cut_energy(vp, a, alpha, l) for l in labs}
        emin = min(energies.values())
        minimisers = [l for l, e in energies.items() if e == emin]
        for i in range(m):
            for b in (0, 1):
                assert mm[i][b] == min(e for l, e in energies.items() if l[i] == b)
            assert (mm[i][1] < mm[i][0]) == all(l[i] for l in minimisers)
            assert (mm[i][1] <= mm[i][0]) == any(l[i] for l in minimisers)


def test_number_of_min_cuts_is_bounded():
    rng = np.random.default_rng(5)
    for trial in range(30):
        m = int(rng.integers(1, 30))
        v = rng.integers(-20, 21, size=m)
        a = rng.integers(0, 6, size=m - 1)
        x, cuts = par.tv1d_prox_parametric(v, a)
        runs = 1 + sum(1 for i in range(m - 1) if x[i] != x[i + 1])
        assert 1 <= cuts <= 2 * runs - 1


def test_pins_catch_planted_mistakes(orc, monkeypatch):
    """A wrong sign in the boundary modification, or the maximal minimiser in
    place of the minimal one without the tie class, fails the comparison."""
    rng = np.random.default_rng(6)
    cases = [(rng.integers(-9, 10, size=12), rng.integers(1, 5, size=11)) for _ in range(20)]

    def differs():
        for v, a in cases:
            try:
                x, _ = par.tv1d_prox_parametric(v, a)
            except ArithmeticError:
                return True
            if np.abs(np.array([float(t) for t in x]) - orc.tv1d_prox(v, a)).max() > 1e-6:
                return True
        return False

    assert not differs()
    good = par.chain_min_cut_min_marginals
    monkeypatch.setattr(par, "chain_min_cut_min_marginals",
                        lambda vp, a, al: [(m1, m0) for m0, m1 in good(vp, a, al)])   # labels swapped
    assert differs()
    monkeypatch.setattr(par, "chain_min_cut_min_marginals",
                        lambda vp, a, al: [(m0, m1 + (1 if m0 == m1 else 0)) for m0, m1 in good(vp, a, al)])
    assert differs()
