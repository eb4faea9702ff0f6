/*
 * Oracle: exact min-cut of the grid energy by max-flow.  TEST
 * INFRASTRUCTURE ONLY: never called by the product path.
 *
 * Problem (D) of Sec. 2: minimise E(l) = sum_e a_e [l_i != l_j] - w^T l over
 * l in {0,1}^n with a_e >= 0 (Eq. 2, each undirected edge once).  With source
 * side S = {i : l_i = 1}, the s-t cut of the graph with arcs s->i (capacity
 * max(w_i,0)), i->t (max(-w_i,0)) and i<->j (a_e each way) costs
 *   sum_{i not in S} w_i^+ + sum_{i in S} w_i^- + sum_{e across} a_e
 *   = sum_i w_i^+ + E(1_S),
 * so E* = maxflow - sum_i w_i^+.  Two independent algorithms are provided:
 * Edmonds-Karp (shortest augmenting paths) and FIFO push-relabel with global
 * relabelling.  Capacities are exact 64-bit integers.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t nn, na;
    int64_t* first;   /* nn + 1 */
    int64_t* head;
    int64_t* cap;     /* residual capacity */
    int64_t* rev;     /* index of the reverse arc */
} graph_t;

static int is_integral(double v)
{
    return isfinite(v) && floor(v) == v && fabs(v) < 9.0e15;
}

static void axis_split2(int ndim, const int64_t* dims, int axis,
                        int64_t* outer, int64_t* inner)
{
    *outer = 1; *inner = 1;
    for (int d = 0; d < axis; ++d) *outer *= dims[d];
    for (int d = axis + 1; d < ndim; ++d) *inner *= dims[d];
}

/* Build the residual graph; returns 0 or -1 on bad input / no memory. */
static int build_graph(int ndim, const int64_t* dims, const double* w,
                       const double* const* a, graph_t* g, int64_t* wplus)
{
    memset(g, 0, sizeof(*g));
    int64_t n = 1;
    for (int d = 0; d < ndim; ++d) n *= dims[d];
    int64_t nedges = 0;
    for (int k = 0; k < ndim; ++k) nedges += n / dims[k] * (dims[k] - 1);
    int64_t npairs = 2 * n + nedges;           /* s-arc, t-arc, grid edges */
    g->nn = n + 2;
    g->na = 2 * npairs;
    int64_t* tail = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    int64_t* hd = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    int64_t* cp = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    g->first = (int64_t*)calloc((size_t)(g->nn + 1), sizeof(int64_t));
    g->head = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    g->cap = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    g->rev = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    if (!tail || !hd || !cp || !g->first || !g->head || !g->cap || !g->rev) {
        free(tail); free(hd); free(cp);
        return -1;
    }
    int64_t s = n, t = n + 1, na = 0, wp = 0;
    int bad = 0;
#define ADD_PAIR(u, v, cuv, cvu) do { tail[na] = (u); hd[na] = (v); cp[na] = (cuv); ++na; \
                                      tail[na] = (v); hd[na] = (u); cp[na] = (cvu); ++na; } while (0)
    for (int64_t i = 0; i < n; ++i) {
        if (!is_integral(w[i])) bad = 1;
        int64_t wi = (int64_t)w[i];
        if (wi > 0) wp += wi;
        ADD_PAIR(s, i, wi > 0 ? wi : 0, 0);
        ADD_PAIR(i, t, wi < 0 ? -wi : 0, 0);
    }
    for (int k = 0; k < ndim; ++k) {
        int64_t outer, inner, m = dims[k];
        axis_split2(ndim, dims, k, &outer, &inner);
        for (int64_t o = 0; o < outer; ++o)
            for (int64_t j = 0; j + 1 < m; ++j)
                for (int64_t q = 0; q < inner; ++q) {
                    int64_t ei = o * m * inner + j * inner + q;
                    double ae = a[k][o * (m - 1) * inner + j * inner + q];
                    if (!is_integral(ae) || ae < 0) bad = 1;
                    ADD_PAIR(ei, ei + inner, (int64_t)ae, (int64_t)ae);
                }
    }
#undef ADD_PAIR
    /* counting sort of arcs by tail; arcs 2p and 2p+1 are mutual reverses */
    for (int64_t e = 0; e < na; ++e) g->first[tail[e] + 1]++;
    for (int64_t u = 0; u < g->nn; ++u) g->first[u + 1] += g->first[u];
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->nn);
    int64_t* where = (int64_t*)malloc(sizeof(int64_t) * (size_t)na);
    memcpy(pos, g->first, sizeof(int64_t) * (size_t)g->nn);
    for (int64_t e = 0; e < na; ++e) {
        int64_t p = pos[tail[e]]++;
        where[e] = p;
        g->head[p] = hd[e];
        g->cap[p] = cp[e];
    }
    for (int64_t e = 0; e < na; ++e) g->rev[where[e]] = where[e ^ 1];
    free(pos); free(where); free(tail); free(hd); free(cp);
    *wplus = wp;
    return bad ? -1 : 0;
}

static void free_graph(graph_t* g)
{
    free(g->first); free(g->head); free(g->cap); free(g->rev);
}

/* Shortest augmenting paths (Edmonds-Karp). */
static int64_t edmonds_karp(graph_t* g, int64_t s, int64_t t)
{
    int64_t* pred = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->nn);
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->nn);
    int64_t flow = 0;
    for (;;) {
        for (int64_t u = 0; u < g->nn; ++u) pred[u] = -1;
        int64_t qh = 0, qt = 0;
        queue[qt++] = s;
        pred[s] = -2;
        while (qh < qt && pred[t] == -1) {
            int64_t u = queue[qh++];
            for (int64_t e = g->first[u]; e < g->first[u + 1]; ++e) {
                int64_t v = g->head[e];
                if (g->cap[e] > 0 && pred[v] == -1) {
                    pred[v] = e;
                    queue[qt++] = v;
                }
            }
        }
        if (pred[t] == -1) break;
        int64_t b = INT64_MAX;
        for (int64_t v = t; v != s; v = g->head[g->rev[pred[v]]])
            if (g->cap[pred[v]] < b) b = g->cap[pred[v]];
        for (int64_t v = t; v != s; v = g->head[g->rev[pred[v]]]) {
            g->cap[pred[v]] -= b;
            g->cap[g->rev[pred[v]]] += b;
        }
        flow += b;
    }
    free(pred); free(queue);
    return flow;
}

/* Exact distances to t in the residual graph (BFS over reverse arcs);
 * unreachable vertices get label nn. */
static void distances_to_sink(graph_t* g, int64_t t, int64_t* d, int64_t* queue)
{
    for (int64_t u = 0; u < g->nn; ++u) d[u] = g->nn;
    int64_t qh = 0, qt = 0;
    d[t] = 0;
    queue[qt++] = t;
    while (qh < qt) {
        int64_t v = queue[qh++];
        for (int64_t e = g->first[v]; e < g->first[v + 1]; ++e) {
            int64_t u = g->head[e];
            /* u -> v is residual iff the reverse of e has capacity */
            if (d[u] == g->nn && g->cap[g->rev[e]] > 0) {
                d[u] = d[v] + 1;
                queue[qt++] = u;
            }
        }
    }
}

/* FIFO push-relabel, first phase (maximum preflow); returns the flow value. */
static int64_t push_relabel(graph_t* g, int64_t s, int64_t t)
{
    int64_t nn = g->nn;
    int64_t* h = (int64_t*)malloc(sizeof(int64_t) * (size_t)nn);
    int64_t* ex = (int64_t*)calloc((size_t)nn, sizeof(int64_t));
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)nn);
    int64_t* fifo = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nn + 1));
    int64_t* bfsq = (int64_t*)malloc(sizeof(int64_t) * (size_t)nn);
    uint8_t* inq = (uint8_t*)calloc((size_t)nn, 1);
    int64_t qh = 0, qt = 0, qn = 0;
#define ENQ(u) do { fifo[qt] = (u); qt = (qt + 1) % (nn + 1); ++qn; inq[u] = 1; } while (0)

    for (int64_t e = g->first[s]; e < g->first[s + 1]; ++e) {
        int64_t c = g->cap[e];
        if (c > 0) {
            g->cap[e] = 0;
            g->cap[g->rev[e]] += c;
            ex[g->head[e]] += c;
        }
    }
    distances_to_sink(g, t, h, bfsq);
    h[s] = nn;
    for (int64_t u = 0; u < nn; ++u) {
        cur[u] = g->first[u];
        if (u != s && u != t && ex[u] > 0 && h[u] < nn) ENQ(u);
    }
    int64_t work = 0, relabel_budget = 6 * nn + (g->na / 2);
    while (qn > 0) {
        int64_t u = fifo[qh]; qh = (qh + 1) % (nn + 1); --qn; inq[u] = 0;
        while (ex[u] > 0 && h[u] < nn) {
            int64_t e = cur[u];
            if (e == g->first[u + 1]) {                 /* relabel */
                int64_t best = 2 * nn;
                for (int64_t f = g->first[u]; f < g->first[u + 1]; ++f)
                    if (g->cap[f] > 0 && h[g->head[f]] + 1 < best) best = h[g->head[f]] + 1;
                h[u] = best < nn ? best : nn;
                cur[u] = g->first[u];
                work += 12 + (g->first[u + 1] - g->first[u]);
                continue;
            }
            int64_t v = g->head[e];
            if (g->cap[e] > 0 && h[u] == h[v] + 1) {     /* push */
                int64_t d = ex[u] < g->cap[e] ? ex[u] : g->cap[e];
                g->cap[e] -= d;
                g->cap[g->rev[e]] += d;
                ex[u] -= d;
                ex[v] += d;
                if (v != s && v != t && !inq[v]) ENQ(v);
            } else {
                ++cur[u];
            }
        }
        if (work > relabel_budget) {                     /* global relabel */
            work = 0;
            distances_to_sink(g, t, h, bfsq);
            h[s] = nn;
            qh = qt = qn = 0;
            for (int64_t x = 0; x < nn; ++x) {
                inq[x] = 0;
                cur[x] = g->first[x];
            }
            for (int64_t x = 0; x < nn; ++x)
                if (x != s && x != t && ex[x] > 0 && h[x] < nn) ENQ(x);
        }
    }
#undef ENQ
    int64_t flow = ex[t];
    free(h); free(ex); free(cur); free(fifo); free(bfsq); free(inq);
    return flow;
}

/* The same graph for an explicit list of undirected edges (i, j, a_e),
 * e.g. the grid with diagonals; returns 0 or -1. */
static int build_graph_edges(int64_t n, const double* w, int64_t nedges,
                             const int64_t* ei, const int64_t* ej, const double* ae,
                             graph_t* g, int64_t* wplus)
{
    memset(g, 0, sizeof(*g));
    int64_t npairs = 2 * n + nedges;
    g->nn = n + 2;
    g->na = 2 * npairs;
    int64_t* tail = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    int64_t* hd = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    int64_t* cp = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    g->first = (int64_t*)calloc((size_t)(g->nn + 1), sizeof(int64_t));
    g->head = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    g->cap = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    g->rev = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->na);
    if (!tail || !hd || !cp || !g->first || !g->head || !g->cap || !g->rev) {
        free(tail); free(hd); free(cp);
        return -1;
    }
    int64_t s = n, t = n + 1, na = 0, wp = 0;
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!is_integral(w[i])) bad = 1;
        int64_t wi = (int64_t)w[i];
        if (wi > 0) wp += wi;
        tail[na] = s; hd[na] = i; cp[na] = wi > 0 ? wi : 0; ++na;
        tail[na] = i; hd[na] = s; cp[na] = 0; ++na;
        tail[na] = i; hd[na] = t; cp[na] = wi < 0 ? -wi : 0; ++na;
        tail[na] = t; hd[na] = i; cp[na] = 0; ++na;
    }
    for (int64_t e = 0; e < nedges; ++e) {
        if (!is_integral(ae[e]) || ae[e] < 0 || ei[e] < 0 || ei[e] >= n || ej[e] < 0 || ej[e] >= n) bad = 1;
        int64_t c = (int64_t)ae[e];
        tail[na] = ei[e]; hd[na] = ej[e]; cp[na] = c; ++na;
        tail[na] = ej[e]; hd[na] = ei[e]; cp[na] = c; ++na;
    }
    if (bad) {
        free(tail); free(hd); free(cp);
        return -1;
    }
    for (int64_t e = 0; e < na; ++e) g->first[tail[e] + 1]++;
    for (int64_t u = 0; u < g->nn; ++u) g->first[u + 1] += g->first[u];
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->nn);
    int64_t* where = (int64_t*)malloc(sizeof(int64_t) * (size_t)na);
    memcpy(pos, g->first, sizeof(int64_t) * (size_t)g->nn);
    for (int64_t e = 0; e < na; ++e) {
        int64_t p = pos[tail[e]]++;
        where[e] = p;
        g->head[p] = hd[e];
        g->cap[p] = cp[e];
    }
    for (int64_t e = 0; e < na; ++e) g->rev[where[e]] = where[e ^ 1];
    free(pos); free(where); free(tail); free(hd); free(cp);
    *wplus = wp;
    return 0;
}

static void finish_maxflow(graph_t* g, int method, int64_t* flow, int64_t* emin,
                           uint8_t* s_max, int64_t wplus);

int oracle_maxflow_edges(int method, int64_t n, const double* w, int64_t nedges,
                         const int64_t* ei, const int64_t* ej, const double* ae,
                         int64_t* flow, int64_t* emin, uint8_t* s_max)
{
    if (n < 1 || nedges < 0 || (method != 0 && method != 1)) return -1;
    graph_t g;
    int64_t wplus = 0;
    if (build_graph_edges(n, w, nedges, ei, ej, ae, &g, &wplus) != 0) {
        free_graph(&g);
        return -1;
    }
    finish_maxflow(&g, method, flow, emin, s_max, wplus);
    free_graph(&g);
    return 0;
}

static void finish_maxflow(graph_t* g, int method, int64_t* flow, int64_t* emin,
                           uint8_t* s_max, int64_t wplus)
{
    int64_t n = g->nn - 2, s = n, t = n + 1;
    int64_t f = method == 0 ? edmonds_karp(g, s, t) : push_relabel(g, s, t);
    if (s_max) {
        int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->nn);
        int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (size_t)g->nn);
        distances_to_sink(g, t, d, q);
        for (int64_t i = 0; i < n; ++i) s_max[i] = (uint8_t)(d[i] >= g->nn);
        free(d); free(q);
    }
    *flow = f;
    *emin = f - wplus;
}

int oracle_maxflow(int method, int ndim, const int64_t* dims, const double* w,
                   const double* const* a, int64_t* flow, int64_t* emin,
                   uint8_t* s_max)
{
    if (ndim < 1 || ndim > 3 || (method != 0 && method != 1)) return -1;
    for (int d = 0; d < ndim; ++d) if (dims[d] < 1) return -1;
    graph_t g;
    int64_t wplus = 0;
    if (build_graph(ndim, dims, w, a, &g, &wplus) != 0) {
        free_graph(&g);
        return -1;
    }
    int64_t n = g.nn - 2, s = n, t = n + 1;
    int64_t f = method == 0 ? edmonds_karp(&g, s, t) : push_relabel(&g, s, t);
    if (s_max) {
        /* vertices that reach t in the residual graph form the minimal sink
         * side; the rest is the maximal minimising source set */
        int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)g.nn);
        int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (size_t)g.nn);
        distances_to_sink(&g, t, d, q);
        for (int64_t i = 0; i < n; ++i) s_max[i] = (uint8_t)(d[i] >= g.nn);
        free(d); free(q);
    }
    *flow = f;
    *emin = f - wplus;
    free_graph(&g);
    return 0;
}
