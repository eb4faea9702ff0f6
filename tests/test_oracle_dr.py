"""Pins for the oracle's product-space methods (Sec. 4): AAR (Eq. 3), AP
(Sec. 4.2), BCD and FISTA (Sec. 4.1).  Their limits are checked against a TV
denoiser over all grid edges written here (dual projected gradient, no chain
decomposition), against exact min-cuts (thresholding at zero, Sec. 2.3), and
against properties the paper states or implies: dual feasibility, the duality
gaps of Sec. 2.2-2.3, the divergence of the AAR iterates at the rate of the
gap vector (Sec. 4.3), monotone BCD, and for FISTA its reduction to AP while
the momentum is zero and the O(1/k^2) bound of accelerated gradient methods."""
import numpy as np
import pytest

from paper_1503_01563_gb300 import inputs

AAR, AP, BCD, FISTA = 0, 1, 2, 3


def edges(dims, a):
    """Undirected grid edges (i, j, a_e) built from compact weights."""
    idx = np.arange(int(np.prod(dims))).reshape(dims)
    I, J, A = [], [], []
    for k in range(len(dims)):
        sl0 = [slice(None)] * len(dims)
        sl1 = [slice(None)] * len(dims)
        sl0[k] = slice(0, dims[k] - 1)
        sl1[k] = slice(1, dims[k])
        I.append(idx[tuple(sl0)].ravel())
        J.append(idx[tuple(sl1)].ravel())
        A.append(np.asarray(a[k], dtype=np.float64).ravel())
    return np.concatenate(I), np.concatenate(J), np.concatenate(A)


def graph_tv_prox(w, a, iters=60000):
    """argmin_x 1/2||x - w||^2 + sum_e a_e |x_i - x_j| via accelerated
    projected gradient on the dual p (|p_e| <= a_e), x = w - B^T p."""
    dims = w.shape
    I, J, A = edges(dims, a)
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
    return primal(p).reshape(dims)


def run(orc, algo, w, a, iters):
    s = orc.cold_state(algo, w)
    return orc.iterate(algo, w, a, s, iters)


def test_zero_weights_give_identity(orc):
    w, a = inputs.uniform_grid((5, 7), 2)
    a = [np.zeros_like(x) for x in a]
    for algo in (AAR, AP, BCD, FISTA):
        _, x = run(orc, algo, w, a, 1)
        np.testing.assert_allclose(x, w, atol=1e-12)


def test_separable_case(orc):
    """Only horizontal edges: the TV problem splits into independent row
    chains, so x* is the row-wise chain prox of w."""
    w, a = inputs.uniform_grid((6, 9), 3)
    a = [np.zeros_like(a[0]), a[1]]
    want = np.stack([orc.tv1d_prox(w[h].astype(float), a[1][h].astype(float)) for h in range(6)])
    for algo in (AAR, AP, BCD, FISTA):
        _, x = run(orc, algo, w, a, 400)
        np.testing.assert_allclose(x, want, atol=1e-8)


@pytest.mark.parametrize("dims", [(5, 6), (3, 4, 3)])
def test_limits_agree_with_graph_tv(orc, dims):
    w, a = inputs.uniform_grid(dims, 21, w_range=(-6, 6), a_range=(1, 3))
    ref = graph_tv_prox(w, a)
    for algo in (AAR, AP, BCD, FISTA):
        _, x = run(orc, algo, w, a, 3000)
        np.testing.assert_allclose(x, ref, atol=2e-6, err_msg=f"algo {algo}")


def test_threshold_gives_min_cut_bruteforce(orc):
    """Sec. 2.3: thresholding the TV solution at zero solves (D); the strict
    threshold gives the minimal minimiser and the non-strict one the maximal."""
    for dims in [(4, 4), (3, 3, 2)]:
        for seed in range(12):
            w, a = inputs.uniform_grid(dims, seed, w_range=(-10, 10), a_range=(1, 6))
            e, _, smin, smax = orc.bruteforce(w, a)
            _, x = run(orc, AAR, w, a, 3000)
            assert np.array_equal((x > 1e-7).astype(np.uint8), smin)
            assert np.array_equal((x >= -1e-7).astype(np.uint8), smax)
            assert orc.energy(w, a, (x > 1e-7).astype(np.uint8)) == e


def test_threshold_gives_min_cut_maxflow(orc):
    w, a = inputs.uniform_grid((24, 20), 5)
    E, smin, smax = orc.min_cut(w, a)
    for algo in (AAR, AP, BCD, FISTA):
        _, x = run(orc, algo, w, a, 2500)
        assert orc.energy(w, a, (x > 1e-7).astype(np.uint8)) == E
        assert np.array_equal((x > 1e-7).astype(np.uint8), smin)
        assert np.array_equal((x >= -1e-7).astype(np.uint8), smax)


def shadow(orc, s, a):
    return np.stack([orc.project_block(s[k], a[k], k) for k in range(s.shape[0])])


def test_gaps_along_aar(orc):
    """For y in K the discrete lower bound sum min(y_i - w_i, 0) (dual of (C))
    never exceeds E*, and the TV duality gap f(x) - y^T x (x = w - y) is >= 0
    and tends to 0."""
    w, a = inputs.uniform_grid((12, 10), 8)
    E = orc.maxflow(w, a)[1]
    s = orc.cold_state(AAR, w)
    gaps = []
    for _ in range(40):
        s, x = orc.iterate(AAR, w, a, s, 10)
        y = w - x                                  # = sum_k y_k of the shadow
        lb = np.minimum(y - w, 0).sum()
        lab = (x > 0).astype(np.uint8)
        assert lb <= E + 1e-7 <= orc.energy(w, a, lab) + 1e-7
        gap = orc.tv_value(a, x) - (y * x).sum()
        assert gap >= -1e-7
        gaps.append(gap)
    assert gaps[-1] < 1e-6 * max(1.0, gaps[0])
    assert E - lb < 1e-6


def test_aar_diverges_at_gap_vector_rate(orc):
    """Sec. 4.3: the AAR sequence z diverges while its shadow converges; the
    step z^{k+1} - z^k tends to the gap vector between K and L, which is x*/r
    in every block (x* the TV solution)."""
    for dims in [(8, 9), (4, 5, 3)]:
        w, a = inputs.uniform_grid(dims, 4)
        r = len(dims)
        s, x = run(orc, AAR, w, a, 3000)
        s2, _ = orc.iterate(AAR, w, a, s, 1)
        for k in range(r):
            np.testing.assert_allclose(s2[k] - s[k], x / r, atol=1e-7)


def test_ap_fixed_point(orc):
    """At the AP limit lambda = Pi_L(Pi_K(lambda)) and lambda_k - y_k = x*/r."""
    w, a = inputs.uniform_grid((7, 8), 6)
    s, x = run(orc, AP, w, a, 3000)
    y = shadow(orc, s, a)
    for k in range(2):
        np.testing.assert_allclose(s[k] - y[k], x / 2, atol=1e-7)
    np.testing.assert_allclose(w - y.sum(0), x, atol=1e-9)


def test_aar_firmly_nonexpansive(orc):
    """T = 1/2 (R_L R_K + I) is firmly nonexpansive: ||Tz - Tz'||^2 +
    ||(I-T)z - (I-T)z'||^2 <= ||z - z'||^2 (a dropped 1/2 or a wrong
    reflection breaks this)."""
    w, a = inputs.uniform_grid((6, 6), 9)
    g = np.random.default_rng(1)
    for _ in range(10):
        z = g.normal(size=(2, 6, 6)) * 20
        z2 = z + g.normal(size=z.shape) * 5
        t1, _ = orc.iterate(AAR, w, a, z, 1)
        t2, _ = orc.iterate(AAR, w, a, z2, 1)
        lhs = np.sum((t1 - t2) ** 2) + np.sum(((z - t1) - (z2 - t2)) ** 2)
        assert lhs <= np.sum((z - z2) ** 2) * (1 + 1e-12) + 1e-9


def test_bcd_monotone(orc):
    """Cyclic projections minimise 1/2 ||sum_k y_k - w||^2 (Eq. dualdec2)
    exactly over one block at a time, so the objective never increases."""
    w, a = inputs.uniform_grid((9, 9), 10)
    s = orc.cold_state(BCD, w)
    prev = np.inf
    for _ in range(30):
        s, _ = orc.iterate(BCD, w, a, s, 1)
        obj = 0.5 * np.sum((s.sum(0) - w) ** 2)
        assert obj <= prev + 1e-9
        prev = obj


def test_cold_states(orc):
    w, _ = inputs.uniform_grid((3, 4, 5), 1)
    assert np.all(orc.cold_state(AAR, w) == 0)
    assert np.all(orc.cold_state(BCD, w) == 0)
    assert np.all(orc.cold_state(FISTA, w) == 0)
    lam = orc.cold_state(AP, w)
    np.testing.assert_allclose(lam.sum(0), w)
    np.testing.assert_allclose(lam[0], lam[2])


def test_fista_starts_as_ap(orc):
    """FISTA's extrapolation weight (t_k - 1)/t_{k+1} is 0 for k = 1 (t_1 = 1),
    so from y = 0 its first two iterates are projected gradient steps
    y <- Pi_K(Pi_L(u)), which are AP's from lambda = Pi_L(0); the third
    already differs (a dropped or misplaced momentum term fails here)."""
    for dims in [(9, 11), (4, 5, 6)]:
        w, a = inputs.uniform_grid(dims, 13)
        for k in (1, 2):
            _, xf = run(orc, FISTA, w, a, k)
            _, xa = run(orc, AP, w, a, k)
            np.testing.assert_allclose(xf, xa, atol=1e-12, err_msg=f"iterate {k}")
        _, xf = run(orc, FISTA, w, a, 3)
        _, xa = run(orc, AP, w, a, 3)
        assert np.abs(xf - xa).max() > 1e-6


def test_fista_rate_bound(orc):
    """Beck and Teboulle's bound for FISTA with constant step 1/L:
    g(y_k) - g* <= 2 L ||y_0 - y*||^2 / (k + 1)^2 for every minimiser y*, here
    g(y) = 1/2 ||sum_k y_k - w||^2 = 1/2 ||x||^2, L = r (Sec. 4.1), y_0 = 0 and
    y* the limit of cyclic projections."""
    for dims in [(10, 12), (5, 4, 6)]:
        w, a = inputs.uniform_grid(dims, 17)
        r = len(dims)
        ystar, xstar = run(orc, BCD, w, a, 4000)
        gstar = 0.5 * np.sum(xstar ** 2)
        D = np.sum(ystar ** 2)
        for k in (1, 2, 3, 5, 8, 13, 21, 34, 55):
            _, x = run(orc, FISTA, w, a, k)
            assert 0.5 * np.sum(x ** 2) - gstar <= 2 * r * D / (k + 1) ** 2 + 1e-9, k


def test_fista_faster_than_ap(orc):
    """The momentum pays on these problems, as the paper's Table 1 reports
    (FISTA needs fewer iterations than AP on every dataset listed)."""
    w, a = inputs.uniform_grid((24, 20), 5)
    _, xstar = run(orc, BCD, w, a, 4000)
    gstar = 0.5 * np.sum(xstar ** 2)
    _, xf = run(orc, FISTA, w, a, 150)
    _, xa = run(orc, AP, w, a, 150)
    assert 0.5 * np.sum(xf ** 2) - gstar < 0.1 * (0.5 * np.sum(xa ** 2) - gstar)
