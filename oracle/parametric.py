"""Chain prox by a sequence of chain min-cuts (Sec. 3.2, "Message passing").

TEST INFRASTRUCTURE ONLY: only ``tests/`` may import it; it shares no code
with the CUDA library.

Sec. 3.2 names message passing as an alternative to the taut string: message
passing solves the min-cut problem on a chain, and the exact TV solution
follows from a sequence of at most n such min-cuts.  This module states that
method plainly, in exact rational arithmetic (``fractions.Fraction``), so that
every set it forms is exact; it is meant for small chains.

The chain prox  min_x 1/2 sum_i (x_i - v_i)^2 + sum_k a_k |x_{k+1} - x_k|  is
solved on intervals of the chain, starting from the whole chain:

1. On an interval I with unary v' (the input, modified at the ends of I as in
   step 4), the solution on I has mean alpha = mean(v' over I): the edge
   terms inside I cancel in the sum of the optimality conditions.
2. The cut energy  E_alpha(l) = sum_{edges k in I} a_k |l_{k+1} - l_k|
   - sum_{i in I} (v'_i - alpha) l_i  over l in {0, 1}^I is minimised by
   min-sum message passing: forward messages F_i(l), backward messages
   B_i(l) and min-marginals M_i(l) = F_i(l) + B_i(l) (F includes the unary
   of i, B does not).
3. The minimal minimiser {i : M_i(1) < M_i(0)} is {x* > alpha} and the
   maximal one {M_i(1) <= M_i(0)} is {x* >= alpha} (Sec. 2.3: thresholding
   the TV solution gives the minimal / maximal minimisers of the cut
   energy, here of the interval's problem).  Elements with
   M_i(1) = M_i(0) have x*_i = alpha and are final.
4. For each edge k in I whose ends fall in different classes (above alpha,
   at alpha, below alpha), the sign of x_{k+1} - x_k is known, so the edge
   term is linear on each side: the end with the larger value gets
   v' -= a_k and the other v' += a_k.  Each maximal run of elements above
   (or below) alpha is then a new interval whose solution is the prox of
   its own modified unary.

An interval is always a union of whole constant runs of x*, and every
min-cut either fixes at least one run at its final value or splits its
interval into two or more intervals, so a chain whose solution has S maximal
constant runs takes at most 2 S - 1 min-cuts.
"""
from __future__ import annotations

from fractions import Fraction


def chain_min_cut_min_marginals(vp, a, alpha):
    """Min-marginals (M_i(0), M_i(1)) of E_alpha on one chain by min-sum
    message passing (exact, two states per element)."""
    m = len(vp)
    unary = [(Fraction(0), alpha - vp[i]) for i in range(m)]     # cost of label 0, of label 1
    fwd = [None] * m
    fwd[0] = unary[0]
    for i in range(1, m):
        ak = a[i - 1]
        fwd[i] = tuple(unary[i][l] + min(fwd[i - 1][lp] + (ak if lp != l else 0) for lp in (0, 1))
                       for l in (0, 1))
    bwd = [None] * m
    bwd[m - 1] = (Fraction(0), Fraction(0))
    for i in range(m - 2, -1, -1):
        ak = a[i]
        bwd[i] = tuple(min(unary[i + 1][ln] + bwd[i + 1][ln] + (ak if ln != l else 0) for ln in (0, 1))
                       for l in (0, 1))
    return [(fwd[i][0] + bwd[i][0], fwd[i][1] + bwd[i][1]) for i in range(m)]


def chain_min_cut_energy(vp, a, alpha, labels):
    """E_alpha(labels) on one chain (for checking the message passing)."""
    e = Fraction(0)
    for k in range(len(vp) - 1):
        if labels[k] != labels[k + 1]:
            e += a[k]
    for i, l in enumerate(labels):
        if l:
            e -= vp[i] - alpha
    return e


def tv1d_prox_parametric(v, a):
    """Exact prox of a weighted chain (x as Fractions) and the number of
    min-cuts solved.  v: m values, a: m-1 weights >= 0 (floats, ints or
    Fractions; floats are taken at their exact binary value)."""
    v = [Fraction(x) for x in v]
    a = [Fraction(x) for x in a]
    m = len(v)
    if len(a) != max(m - 1, 0):
        raise ValueError("a must have m-1 entries")
    x = [None] * m
    vp = list(v)
    todo = [(0, m)] if m else []
    cuts = 0
    while todo:
        lo, hi = todo.pop()
        alpha = sum(vp[lo:hi]) / (hi - lo)
        mm = chain_min_cut_min_marginals(vp[lo:hi], a[lo:hi - 1], alpha)
        cuts += 1
        cls = [1 if m1 < m0 else (-1 if m1 > m0 else 0) for m0, m1 in mm]
        if cls[0] != 0 and all(c == cls[0] for c in cls):
            # the mean of x* on I is alpha, so x* cannot lie on one side of it
            raise ArithmeticError("a min-cut put the whole interval on one side of its mean")
        for i, c in enumerate(cls):
            if c == 0:
                x[lo + i] = alpha
        for k in range(lo, hi - 1):
            ck, cn = cls[k - lo], cls[k + 1 - lo]
            if ck > cn:                        # x_k > x_{k+1}
                vp[k] -= a[k]
                vp[k + 1] += a[k]
            elif ck < cn:                      # x_k < x_{k+1}
                vp[k] += a[k]
                vp[k + 1] -= a[k]
        i = lo
        while i < hi:
            j = i
            while j + 1 < hi and cls[j + 1 - lo] == cls[i - lo]:
                j += 1
            if cls[i - lo] != 0:
                todo.append((i, j + 1))
            i = j + 1
    return x, cuts
