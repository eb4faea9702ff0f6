/*
 * CPU oracle for the min-cut-by-TV-denoising method of "Convex Optimization
 * for Parallel Energy Minimization" (Kumar, Barbero, Jegelka, Sra, Bach).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain, FP64 statement
 * of what the GPU path must compute.  It shares no code, header, table or
 * helper with the CUDA library; only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  The product path never calls it.
 *
 * Conventions shared by every function below (all plain C, FP64):
 *   - A grid has ndim (2 or 3) axes with sizes dims[0..ndim-1], row-major,
 *     last axis fastest (numpy order).  n = prod(dims).
 *   - Unary w (n values): the energy is E(x) = f(x) - w^T x (Sec. 2, Eq. 1-2,
 *     problem (D)); label 1 is favoured where w_i > 0.
 *   - Edge weights along axis k are given in "compact" layout: an array with
 *     the grid's shape except dims[k]-1 along axis k; entry (.., i_k, ..) is the
 *     weight a_e >= 0 of the undirected edge between (.., i_k, ..) and
 *     (.., i_k+1, ..).  Each undirected edge is counted once in f.
 *   - Decomposition (Sec. 3.1, Fig. 1): block k of the product space holds all
 *     chains along axis k; r = ndim blocks.  Block states are stored as r
 *     consecutive n-arrays, block k at offset k*n.
 */
#ifndef TVCUT_ORACLE_H
#define TVCUT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exact weighted 1D-TV prox on one chain (Sec. 3.2):
 *   x = argmin 1/2 sum_i (x_i - v_i)^2 + sum_{k<m-1} a_k |x_{k+1} - x_k|,
 * computed as the taut string through the tube of half-width a around the
 * running sums of v.  O(m^2) worst case.  Returns 0, or -1 on bad input. */
int oracle_tv1d_prox(int64_t m, const double* v, const double* a, double* x);

/* Lagrangian certificate for a candidate chain prox x: with u_i = sum_{j<=i}
 * (x_j - v_j) (the multiplier of the edge (i, i+1) from stationarity),
 * writes out[0] = |u_{m-1}| (must be 0), out[1] = max_k max(|u_k| - a_k, 0)
 * (dual feasibility), out[2] = sum_k (a_k |x_{k+1}-x_k| - u_k (x_{k+1}-x_k))
 * (complementarity = duality gap of the chain problem). */
void oracle_tv1d_certificate(int64_t m, const double* v, const double* a,
                             const double* x, double* out);

/* Projection onto the base polytope K_k of block k (all chains along axis k):
 * y = v - prox_{f_k}(v) (Sec. 2.2-2.3 and Sec. 3.3: Pi_K = I - prox).
 * a_compact is block k's weights in compact layout.  nthreads <= 0: default. */
void oracle_project_block(int ndim, const int64_t* dims, int axis,
                          const double* v, const double* a_compact, double* y,
                          int nthreads);

/* Run `iters` iterations of a product-space method (Sec. 4) from state `s`
 * (r*n doubles, updated in place).  algo 0: averaged alternating reflections
 * (Eq. 3, state z); 1: alternating projections (Sec. 4.2, state lambda);
 * 2: cyclic projections / block coordinate descent (Sec. 4.1, state y);
 * 3: FISTA on the smooth dual of Sec. 4.1 (state y; the momentum starts
 * afresh at every call: t = 1, extrapolated point = s).
 * a[k] points at axis k's compact weights.  x_out (n, may be NULL) receives
 * the primal x = w - sum_k y_k of the last shadow y computed (Eq. dualA and
 * the relation x = w - y of Sec. 2.3).  Returns 0, -1 on bad input. */
int oracle_iterate(int algo, int ndim, const int64_t* dims, const double* w,
                   const double* const* a, double* s, int64_t iters,
                   double* x_out, int nthreads);

/* Cold-start state of each method: AAR z = 0; AP lambda_k = w / r (the
 * projection of 0 onto L); BCD and FISTA y = 0.  Writes r*n doubles. */
void oracle_cold_state(int algo, int ndim, const int64_t* dims,
                       const double* w, double* s);

/* Total variation f(x) = sum over undirected edges a_e |x_i - x_j| (Eq. 2). */
double oracle_tv_value(int ndim, const int64_t* dims, const double* const* a,
                       const double* x);

/* Discrete energy E(l) = f(l) - w^T l of a 0/1 labelling (problem (D)). */
double oracle_energy(int ndim, const int64_t* dims, const double* w,
                     const double* const* a, const uint8_t* labels);

/* Brute force over all 2^n labellings (n <= 26).  Writes the minimum energy,
 * the number of minimisers, and the intersection / union of all minimisers
 * (the minimal and maximal minimisers). Returns 0, or -1 if n is too large. */
int oracle_bruteforce(int ndim, const int64_t* dims, const double* w,
                      const double* const* a, double* emin, int64_t* count,
                      uint8_t* s_min, uint8_t* s_max);

/* Max-flow on the s-t graph of the energy (Eq. 2 as a cut function):
 * arcs s->i with capacity max(w_i,0), i->t with max(-w_i,0), and both
 * directions of every grid edge with capacity a_e.  Inputs must be integral.
 * method 0: Edmonds-Karp (tiny graphs); 1: FIFO push-relabel with global
 * relabelling.  Writes the flow value, E* = flow - sum_i max(w_i,0), and the
 * maximal minimising labelling (vertices that cannot reach t in the residual
 * graph).  Returns 0, or -1 on bad (non-integral or negative) input. */
/* The same for an explicit list of undirected edges (ei[e], ej[e]) with
 * weights ae[e] (integers >= 0) over n vertices, e.g. a grid with its
 * diagonals (8-connected).  Returns 0, -1 on bad input. */
int oracle_maxflow_edges(int method, int64_t n, const double* w, int64_t nedges,
                         const int64_t* ei, const int64_t* ej, const double* ae,
                         int64_t* flow, int64_t* emin, uint8_t* s_max);

int oracle_maxflow(int method, int ndim, const int64_t* dims, const double* w,
                   const double* const* a, int64_t* flow, int64_t* emin,
                   uint8_t* s_max);

#ifdef __cplusplus
}
#endif
#endif
