/*
 * Oracle: block projections and the product-space methods of Sec. 4 of
 * "Convex Optimization for Parallel Energy Minimization", in FP64.
 * TEST INFRASTRUCTURE ONLY: never called by the product path.
 *
 * Every step is written in the paper's own form, without fusion:
 *   Pi_K   : blockwise projection, Pi_{K_k}(v) = v - prox_{f_k}(v), every
 *            chain of block k independently (Sec. 3.1, Sec. 4.2).
 *   Pi_L   : lambda_k = u_k + (w - sum_j u_j) / r   (Eq. dualA).
 *   R      : 2 Pi - I                               (Eq. 2 of Sec. 4.3).
 *   AAR    : z <- 1/2 (R_L R_K + I) z, shadow y = Pi_K(z)   (Eq. 3).
 *   AP     : y <- Pi_K(lambda), lambda <- Pi_L(y)           (Sec. 4.2).
 *   BCD    : y_k <- Pi_{K_k}(w - sum_{j != k} y_j), k = 0..r-1 in turn
 *            (Sec. 4.1, reading the printed inner sum over y_i as y_j).
 *   FISTA  : accelerated projected gradient on the smooth dual
 *            g(y) = 1/2 ||sum_k y_k - w||^2 over K_1 x ... x K_r (Sec. 4.1,
 *            problem dualdec2).  grad_k g(u) = sum_j u_j - w for every block,
 *            Lipschitz constant r, so the gradient step from u is
 *            u - grad g(u) / r = Pi_L(u) and y <- Pi_K(Pi_L(u)); then
 *            t+ = (1 + sqrt(1 + 4 t^2)) / 2 and u <- y + ((t - 1) / t+)(y - y_prev)
 *            (Beck and Teboulle's FISTA with constant step; t = 1 and u = y
 *            at the start of every call, so the momentum restarts per call).
 *   primal : x = w - sum_k y_k                      (Sec. 2.3, x = w - y).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int64_t grid_size(int ndim, const int64_t* dims)
{
    int64_t n = 1;
    for (int d = 0; d < ndim; ++d) n *= dims[d];
    return n;
}

/* outer = prod(dims[:axis]), inner = prod(dims[axis+1:]) */
static void axis_split(int ndim, const int64_t* dims, int axis,
                       int64_t* outer, int64_t* inner)
{
    *outer = 1; *inner = 1;
    for (int d = 0; d < axis; ++d) *outer *= dims[d];
    for (int d = axis + 1; d < ndim; ++d) *inner *= dims[d];
}

void oracle_project_block(int ndim, const int64_t* dims, int axis,
                          const double* v, const double* a_compact, double* y,
                          int nthreads)
{
    int64_t outer, inner, m = dims[axis];
    axis_split(ndim, dims, axis, &outer, &inner);
    int64_t nchains = outer * inner;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double* cv = (double*)malloc(sizeof(double) * (size_t)m);
        double* ca = (double*)malloc(sizeof(double) * (size_t)(m > 1 ? m - 1 : 1));
        double* cx = (double*)malloc(sizeof(double) * (size_t)m);
#pragma omp for schedule(static)
        for (int64_t c = 0; c < nchains; ++c) {
            int64_t o = c / inner, q = c % inner;
            int64_t base = o * m * inner + q;
            int64_t abase = o * (m - 1) * inner + q;
            for (int64_t j = 0; j < m; ++j) cv[j] = v[base + j * inner];
            for (int64_t j = 0; j + 1 < m; ++j) ca[j] = a_compact[abase + j * inner];
            oracle_tv1d_prox(m, cv, ca, cx);
            for (int64_t j = 0; j < m; ++j) y[base + j * inner] = cv[j] - cx[j];
        }
        free(cv); free(ca); free(cx);
    }
}

static void project_K(int ndim, const int64_t* dims, const double* const* a,
                      const double* s, double* y, int64_t n, int nthreads)
{
    for (int k = 0; k < ndim; ++k)
        oracle_project_block(ndim, dims, k, s + k * n, a[k], y + k * n, nthreads);
}

/* Pi_L of Eq. dualA: per vertex, add the common correction (w - sum u)/r. */
static void project_L(int r, int64_t n, const double* w, const double* u,
                      double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = 0; k < r; ++k) s += u[k * n + i];
        double c = (w[i] - s) / (double)r;
        for (int k = 0; k < r; ++k) out[k * n + i] = u[k * n + i] + c;
    }
}

static void primal_from_y(int r, int64_t n, const double* w, const double* y,
                          double* x)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = 0; k < r; ++k) s += y[k * n + i];
        x[i] = w[i] - s;
    }
}

void oracle_cold_state(int algo, int ndim, const int64_t* dims,
                       const double* w, double* s)
{
    int64_t n = grid_size(ndim, dims);
    int r = ndim;
    memset(s, 0, sizeof(double) * (size_t)(r * n));
    if (algo == 1) {               /* lambda^0 = Pi_L(0) */
        double* zero = (double*)calloc((size_t)(r * n), sizeof(double));
        project_L(r, n, w, zero, s);
        free(zero);
    }
}

int oracle_iterate(int algo, int ndim, const int64_t* dims, const double* w,
                   const double* const* a, double* s, int64_t iters,
                   double* x_out, int nthreads)
{
    if (ndim < 1 || ndim > 3 || iters < 0 || algo < 0 || algo > 3) return -1;
    int64_t n = grid_size(ndim, dims);
    int r = ndim;
    double* y = (double*)malloc(sizeof(double) * (size_t)(r * n));
    double* t1 = (double*)malloc(sizeof(double) * (size_t)(r * n));
    double* t2 = (double*)malloc(sizeof(double) * (size_t)(r * n));
    double* v = (double*)malloc(sizeof(double) * (size_t)n);
    if (!y || !t1 || !t2 || !v) { free(y); free(t1); free(t2); free(v); return -1; }
    int have_y = 0;
    double tk = 1.0;                        /* FISTA: t_1 = 1, u_1 = y_prev = s */
    if (algo == 3) {
        memcpy(t2, s, sizeof(double) * (size_t)(r * n));      /* u      */
        memcpy(y, s, sizeof(double) * (size_t)(r * n));       /* y_prev */
    }
    for (int64_t it = 0; it < iters; ++it) {
        if (algo == 0) {
            /* AAR (Eq. 3): z <- 1/2 (R_L R_K z + z); shadow y = Pi_K(z). */
            project_K(ndim, dims, a, s, y, n, nthreads);
            for (int64_t i = 0; i < r * n; ++i) t1[i] = 2.0 * y[i] - s[i];   /* R_K z */
            project_L(r, n, w, t1, t2);                                      /* Pi_L  */
            for (int64_t i = 0; i < r * n; ++i) {
                double rl = 2.0 * t2[i] - t1[i];                             /* R_L   */
                s[i] = 0.5 * (rl + s[i]);
            }
        } else if (algo == 1) {
            /* AP (Sec. 4.2): y = Pi_K(lambda); lambda = Pi_L(y). */
            project_K(ndim, dims, a, s, y, n, nthreads);
            project_L(r, n, w, y, s);
        } else if (algo == 2) {
            /* BCD (Sec. 4.1): y_k <- Pi_{K_k}(w - sum_{j != k} y_j). */
            for (int k = 0; k < r; ++k) {
                for (int64_t i = 0; i < n; ++i) {
                    double o = 0.0;
                    for (int j = 0; j < r; ++j)
                        if (j != k) o += s[j * n + i];
                    v[i] = w[i] - o;
                }
                oracle_project_block(ndim, dims, k, v, a[k], s + k * n, nthreads);
            }
            memcpy(y, s, sizeof(double) * (size_t)(r * n));
        } else {
            /* FISTA: y = Pi_K(u - grad g(u) / r) = Pi_K(Pi_L(u)); momentum. */
            project_L(r, n, w, t2, t1);
            project_K(ndim, dims, a, t1, s, n, nthreads);
            double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
            double beta = (tk - 1.0) / tn;
            for (int64_t i = 0; i < r * n; ++i) {
                t2[i] = s[i] + beta * (s[i] - y[i]);
                y[i] = s[i];
            }
            tk = tn;
        }
        have_y = 1;
    }
    if (x_out) {
        if (!have_y) {
            if (algo >= 2) memcpy(y, s, sizeof(double) * (size_t)(r * n));
            else project_K(ndim, dims, a, s, y, n, nthreads);
        }
        primal_from_y(r, n, w, y, x_out);
    }
    free(y); free(t1); free(t2); free(v);
    return 0;
}

/* Visit every undirected grid edge (i, j) once with its weight. */
#define FOR_EACH_EDGE(ndim, dims, a, BODY)                                     \
    do {                                                                       \
        for (int k_ = 0; k_ < (ndim); ++k_) {                                  \
            int64_t outer_, inner_, m_ = (dims)[k_];                           \
            axis_split((ndim), (dims), k_, &outer_, &inner_);                  \
            for (int64_t o_ = 0; o_ < outer_; ++o_)                            \
                for (int64_t j_ = 0; j_ + 1 < m_; ++j_)                        \
                    for (int64_t q_ = 0; q_ < inner_; ++q_) {                  \
                        int64_t ei = o_ * m_ * inner_ + j_ * inner_ + q_;      \
                        int64_t ej = ei + inner_;                              \
                        double ae = (a)[k_][o_ * (m_ - 1) * inner_ + j_ * inner_ + q_]; \
                        BODY                                                   \
                    }                                                          \
        }                                                                      \
    } while (0)

double oracle_tv_value(int ndim, const int64_t* dims, const double* const* a,
                       const double* x)
{
    double f = 0.0;
    FOR_EACH_EDGE(ndim, dims, a, { f += ae * fabs(x[ei] - x[ej]); });
    return f;
}

double oracle_energy(int ndim, const int64_t* dims, const double* w,
                     const double* const* a, const uint8_t* labels)
{
    int64_t n = grid_size(ndim, dims);
    double e = 0.0;
    FOR_EACH_EDGE(ndim, dims, a, { if (labels[ei] != labels[ej]) e += ae; });
    for (int64_t i = 0; i < n; ++i)
        if (labels[i]) e -= w[i];
    return e;
}

int oracle_bruteforce(int ndim, const int64_t* dims, const double* w,
                      const double* const* a, double* emin, int64_t* count,
                      uint8_t* s_min, uint8_t* s_max)
{
    int64_t n = grid_size(ndim, dims);
    if (n < 1 || n > 26) return -1;
    uint8_t* lab = (uint8_t*)malloc((size_t)n);
    double best = INFINITY;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) { s_min[i] = 1; s_max[i] = 0; }
    for (uint64_t mask = 0; mask < (1ull << n); ++mask) {
        for (int64_t i = 0; i < n; ++i) lab[i] = (uint8_t)((mask >> i) & 1u);
        double e = oracle_energy(ndim, dims, w, a, lab);
        if (cnt == 0 || e < best - 1e-9 * (1.0 + fabs(best))) {
            best = e; cnt = 0;
            for (int64_t i = 0; i < n; ++i) { s_min[i] = 1; s_max[i] = 0; }
        }
        if (fabs(e - best) <= 1e-9 * (1.0 + fabs(best))) {
            ++cnt;
            for (int64_t i = 0; i < n; ++i) {
                s_min[i] &= lab[i];
                s_max[i] |= lab[i];
            }
        }
    }
    free(lab);
    *emin = best;
    *count = cnt;
    return 0;
}
