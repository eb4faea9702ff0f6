/*
 * Oracle: exact weighted 1D total-variation prox on a chain (Sec. 3.2 of
 * "Convex Optimization for Parallel Energy Minimization").  TEST
 * INFRASTRUCTURE ONLY: never called by the product path.
 *
 * The paper solves each chain with a taut-string method that allows a weight
 * per edge.  The fact used here is the classical taut-string characterisation
 * of the 1D-TV prox: with running sums V_0 = 0, V_k = v_1 + ... + v_k, the
 * minimiser x has running sums S_k = x_1 + ... + x_k that form the shortest
 * ("taut") polygonal string from (0, 0) to (m, V_m) that passes through every
 * gate [V_k - a_k, V_k + a_k] at abscissa k (k = 1..m-1).  The string is
 * built gate by gate from an anchor point: the set of slopes that reach all
 * gates seen so far is an interval [lo, hi]; when a new gate leaves that
 * interval empty, the string must bend at the gate point that fixed the
 * violated end of the interval, which becomes the new anchor, and the scan
 * restarts there.  Slopes of the string are the prox values x.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>

int oracle_tv1d_prox(int64_t m, const double* v, const double* a, double* x)
{
    if (m <= 0) return m == 0 ? 0 : -1;
    double* V = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    if (!V) return -1;
    V[0] = 0.0;
    for (int64_t k = 1; k <= m; ++k) V[k] = V[k - 1] + v[k - 1];

    /* gate k (1 <= k <= m): [V_k - r_k, V_k + r_k], radius a_{k} between
     * element k and k+1 (0-based a[k-1]); the end point is pinned. */
#define GATE_R(k) ((k) == m ? 0.0 : a[(k) - 1])

    int64_t k0 = 0;     /* anchor abscissa */
    double s0 = 0.0;    /* anchor ordinate S_{k0} */
    while (k0 < m) {
        double hi = INFINITY, lo = -INFINITY;
        int64_t khi = -1, klo = -1;
        int64_t bend = -1;
        double bend_s = 0.0, slope = 0.0;
        for (int64_t k = k0 + 1; k <= m; ++k) {
            double up = V[k] + GATE_R(k), dn = V[k] - GATE_R(k);
            double su = (up - s0) / (double)(k - k0);
            double sl = (dn - s0) / (double)(k - k0);
            if (sl > hi) {          /* gate k lies above every feasible ray:
                                       the string turns up at the upper gate
                                       point khi */
                bend = khi; slope = hi; bend_s = V[khi] + GATE_R(khi);
                break;
            }
            if (su < lo) {          /* gate k lies below every feasible ray:
                                       the string turns down at klo */
                bend = klo; slope = lo; bend_s = V[klo] - GATE_R(klo);
                break;
            }
            if (su < hi) { hi = su; khi = k; }
            if (sl > lo) { lo = sl; klo = k; }
        }
        if (bend < 0) {             /* the end point was reached in a line */
            slope = (V[m] - s0) / (double)(m - k0);
            bend = m; bend_s = V[m];
        }
        for (int64_t i = k0; i < bend; ++i) x[i] = slope;
        k0 = bend;
        s0 = bend_s;
    }
#undef GATE_R
    free(V);
    return 0;
}

void oracle_tv1d_certificate(int64_t m, const double* v, const double* a,
                             const double* x, double* out)
{
    /* Stationarity of 1/2||x - v||^2 + sum_k u_k (x_{k+1} - x_k) in x_i:
     * x_i - v_i + u_{i-1} - u_i = 0 with u_{-1} = 0, so u_i is the running
     * sum of (x - v); the chain end forces u_{m-1} = 0. */
    double u = 0.0, feas = 0.0, comp = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        u += x[i] - v[i];
        if (i < m - 1) {
            double d = x[i + 1] - x[i];
            double over = fabs(u) - a[i];
            if (over > feas) feas = over;
            comp += a[i] * fabs(d) - u * d;
        }
    }
    out[0] = fabs(u);
    out[1] = feas;
    out[2] = comp;
}
