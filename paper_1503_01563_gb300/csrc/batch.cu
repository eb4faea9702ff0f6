// Batched solves: many independent 2D grids of different sizes iterated
// together (the product-space method of Sec. 4 on each grid; the grids share
// nothing).  All grids live in packed device arrays, and one iteration of
// every grid is two launches:
//   scan   -- the chain prox of every chain of every grid (Sec. 3.2): a
//             persistent grid of CTAs pulls work items (128 chains of one
//             grid and axis, longest chains first) from an atomic counter;
//   update -- the AAR/AP update of every vertex of every grid (Eq. 3 with
//             Eq. dualA, or Sec. 4.2) over 32x32 tiles, grid-stride.
// FISTA (Sec. 4.1, smooth dual) runs the extrapolation and gradient step
// first (tiles), then the scan in projection mode, which writes the new
// iterate over the previous one; the two buffers swap roles every iteration
// and the momentum sequence t lives in device memory, so a captured graph
// replays correctly.
// A whole call (its iterations and the closing check) is captured once into
// a CUDA graph per iteration count and replayed.  Per grid, the check sums
// row-chunk partials in a fixed order (reproducible) and picks the best of
// the level sets around the threshold (Sec. 2.1), like the single-grid path.
// Layout per grid g (H x W, vertices at offset off_g): unary, primal, labels
// and the block of axis 0 in natural layout; the block of axis 1 (rows) and
// its weights transposed (element (r, c) at c*H + r), so that every chain's
// consecutive elements are one chain apart.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "taut_string.cuh"
#include "tvcut_internal.cuh"

using namespace tvcut;

namespace {

struct GridDesc {
    int64_t off;      // vertex offset
    int64_t aoff0;    // offset of axis-0 weights ((H-1) x W, natural)
    int64_t aoff1;    // offset of axis-1 weights ((W-1) x H, transposed)
    int H, W;
};

struct ScanItem {     // chains [c0, c0 + count) of one axis of one grid
    int g, axis, c0, count;
};

struct Tile {         // rows [r0, r0+32) x cols [c0, c0+32) of grid g
    int g, r0, c0, pad;
};

struct RowItem {      // rows [r0, r1) of grid g, for the check
    int g, r0, r1, pad;
};

template <typename T>
struct BatchArgs {
    const GridDesc* grids;
    const ScanItem* items;
    int nitems;
    const Tile* tiles;
    int ntiles;
    const RowItem* rows;
    int nrows;
    int G;
    T* s0;            // axis-0 block states (natural)
    T* s1;            // axis-1 block states (transposed)
    T* x0;            // axis-0 prox outputs (FISTA: the points v to project)
    T* x1;
    T* p0;            // FISTA: previous iterate (natural / transposed)
    T* p1;
    double* mom;      // FISTA: t_{k-1}, t_k
    const T* w;
    const T* a0;
    const T* a1;
    const T* ap0;     // a0 / a1 padded to the state layouts (0 at each chain's end)
    const T* ap1;
    T* xout;
    uint8_t* labels;
    int* counter;     // work-item counter of the scan
    int check;
    T threshold;
    const T* levels;  // G x nlevels
    int nlevels;
    CheckPartial* partials;   // per row item
    LevelPartial* lpartials;  // per row item
    CheckPartial* gsum;       // per grid
    LevelPartial* glev;       // per grid
    const T* best_level;      // per grid (labels pass)
};

// VAR: the chain scan's step: 0 branchy (scan_chain), 1 predicated
// (scan_chain_predicated), 2 branchy on padded weights with each element
// loaded a step ahead (scan_chain_padded; prox output only).
template <typename T, int VAR, bool SHADOW>
__global__ void __launch_bounds__(256) batch_scan_kernel(BatchArgs<T> A)
{
    __shared__ int item_s;
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(A.counter, 1);
        __syncthreads();
        const int it = item_s;
        __syncthreads();
        if (it >= A.nitems) return;
        const ScanItem I = A.items[it];
        for (int t = threadIdx.x; t < I.count; t += blockDim.x) {
            const GridDesc D = A.grids[I.g];
            const int c = I.c0 + t;
            const int64_t b = D.off + c;
            // prox of s into x, or (SHADOW, FISTA) projection of v = x into p
            const T* in = SHADOW ? (I.axis == 0 ? A.x0 : A.x1) : (I.axis == 0 ? A.s0 : A.s1);
            T* out = SHADOW ? (I.axis == 0 ? A.p0 : A.p1) : (I.axis == 0 ? A.x0 : A.x1);
            if (I.axis == 0) {        // column c: H elements, stride W (natural)
                if constexpr (VAR == 2) scan_chain_padded<T, SHADOW>(D.H, in + b, A.ap0 + b, out + b, D.W);
                else if constexpr (VAR == 1) scan_chain_predicated<T, SHADOW>(D.H, in + b, A.a0 + D.aoff0 + c, out + b, D.W);
                else scan_chain<T, SHADOW>(D.H, in + b, A.a0 + D.aoff0 + c, out + b, D.W);
            } else {                  // row c: W elements, stride H (transposed)
                if constexpr (VAR == 2) scan_chain_padded<T, SHADOW>(D.W, in + b, A.ap1 + b, out + b, D.H);
                else if constexpr (VAR == 1) scan_chain_predicated<T, SHADOW>(D.W, in + b, A.a1 + D.aoff1 + c, out + b, D.H);
                else scan_chain<T, SHADOW>(D.W, in + b, A.a1 + D.aoff1 + c, out + b, D.H);
            }
        }
    }
}

// FISTA step on every vertex of every grid: u_k = y_k + beta (y_k - p_k),
// v_k = u_k + (w - u_0 - u_1) / 2 into x_k (the block of axis 1 transposed);
// beta = (t_{k-1} - 1) / t_k from device memory.  EVAL instead writes the
// primal x = w - y_0 - y_1 for the check.
template <typename T, bool EVAL>
__global__ void __launch_bounds__(256) batch_fista_kernel(BatchArgs<T> A)
{
    __shared__ T sy[32][33];
    __shared__ T sp[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const T beta = EVAL ? T(0) : (T)((A.mom[0] - 1.0) / A.mom[1]);
    for (int ti = blockIdx.x; ti < A.ntiles; ti += gridDim.x) {
        const Tile tile = A.tiles[ti];
        const GridDesc D = A.grids[tile.g];
        const int64_t H = D.H, W = D.W;
        __syncthreads();
#pragma unroll
        for (int cc = ty; cc < 32; cc += 8) {
            const int64_t c = tile.c0 + cc, r = tile.r0 + tx;
            if (c < W && r < H) {
                sy[cc][tx] = A.s1[D.off + c * H + r];
                if (!EVAL) sp[cc][tx] = A.p1[D.off + c * H + r];
            }
        }
        __syncthreads();
#pragma unroll
        for (int rr = ty; rr < 32; rr += 8) {
            const int64_t r = tile.r0 + rr, c = tile.c0 + tx;
            if (r >= H || c >= W) continue;
            const int64_t g = D.off + r * W + c;
            const T wg = A.w[g];
            const T y0 = A.s0[g], y1 = sy[tx][rr];
            if (EVAL) {
                A.xout[g] = (wg - y0) - y1;           // as the single-grid path
                continue;
            }
            const T u0 = y0 + beta * (y0 - A.p0[g]);
            const T u1 = y1 + beta * (y1 - sp[tx][rr]);
            const T corr = (wg - (u0 + u1)) / T(2);
            A.x0[g] = u0 + corr;
            sy[tx][rr] = u1 + corr;
        }
        if (EVAL) continue;
        __syncthreads();
#pragma unroll
        for (int cc = ty; cc < 32; cc += 8) {
            const int64_t c = tile.c0 + cc, r = tile.r0 + tx;
            if (c < W && r < H) A.x1[D.off + c * H + r] = sy[cc][tx];
        }
    }
}

// t_{k-1} <- t_k, t_k <- (1 + sqrt(1 + 4 t_k^2)) / 2 (one thread)
__global__ void batch_momentum_kernel(double* mom)
{
    const double t = mom[1];
    mom[0] = t;
    mom[1] = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) batch_update_kernel(BatchArgs<T> A)
{
    __shared__ T sz[32][33];
    __shared__ T sx[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int ti = blockIdx.x; ti < A.ntiles; ti += gridDim.x) {
        const Tile tile = A.tiles[ti];
        const GridDesc D = A.grids[tile.g];
        const int64_t H = D.H, W = D.W;
        __syncthreads();
#pragma unroll
        for (int cc = ty; cc < 32; cc += 8) {
            const int64_t c = tile.c0 + cc, r = tile.r0 + tx;
            if (c < W && r < H) {
                sz[cc][tx] = A.s1[D.off + c * H + r];
                sx[cc][tx] = A.x1[D.off + c * H + r];
            }
        }
        __syncthreads();
#pragma unroll
        for (int rr = ty; rr < 32; rr += 8) {
            const int64_t r = tile.r0 + rr, c = tile.c0 + tx;
            if (r >= H || c >= W) continue;
            const int64_t g = D.off + r * W + c;
            const T wg = A.w[g];
            const T z0 = A.s0[g], z1 = sz[tx][rr];
            const T y0 = z0 - A.x0[g], y1 = z1 - sx[tx][rr];
            const T ysum = y0 + y1;
            if (A.check) A.xout[g] = wg - ysum;
            T cc;
            if constexpr (MODE == UPD_AAR) cc = (wg - T(2) * ysum + (z0 + z1)) / T(2);
            else cc = (wg - ysum) / T(2);
            A.s0[g] = y0 + cc;
            sz[tx][rr] = y1 + cc;
        }
        __syncthreads();
#pragma unroll
        for (int cc = ty; cc < 32; cc += 8) {
            const int64_t c = tile.c0 + cc, r = tile.r0 + tx;
            if (c < W && r < H) A.s1[D.off + c * H + r] = sz[cc][tx];
        }
    }
}

// Check of one row item: labels at the threshold, FP64 sums and level-set
// energies (exact int64 for integer problems).
template <typename T, bool EXACT>
__global__ void __launch_bounds__(256) batch_check_kernel(BatchArgs<T> A)
{
    using Acc = typename std::conditional<EXACT, long long, double>::type;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int ri = blockIdx.x; ri < A.nrows; ri += gridDim.x) {
        const RowItem R = A.rows[ri];
        const GridDesc D = A.grids[R.g];
        const int64_t H = D.H, W = D.W;
        const T* lev = A.levels + (int64_t)R.g * A.nlevels;
        const int L = A.nlevels;
        CheckPartial acc{0, 0, 0, 0, 0, 0, 0, 0};
        Acc el[kMaxLevels];
        int n1l[kMaxLevels];
#pragma unroll
        for (int j = 0; j < kMaxLevels; ++j) { el[j] = 0; n1l[j] = 0; }
        auto mask_of = [&](T xv) {
            unsigned mk = 0;
#pragma unroll
            for (int j = 0; j < kMaxLevels; ++j)
                if (j < L && xv > lev[j]) mk |= 1u << j;
            return mk;
        };
        const T thr = A.threshold;
        for (int64_t r = R.r0 + wid; r < R.r1; r += 8) {
            for (int64_t c = lane; c < W; c += 32) {
                const int64_t g = D.off + r * W + c;
                const T xg = A.xout[g];
                const bool l = xg > thr;
                A.labels[g] = (uint8_t)l;
                const double wg = (double)A.w[g], xd = (double)xg;
                acc.lb -= fmax(xd, 0.0);
                acc.ytx += (wg - xd) * xd;
                acc.xabs = fmax(acc.xabs, fabs(xd));
                if (l) { acc.energy -= wg; acc.energy_i -= llrint(wg); acc.n1 += 1; }
                const unsigned mk = mask_of(xg);
                const Acc wv = EXACT ? (Acc)llrint(wg) : (Acc)wg;
#pragma unroll
                for (int j = 0; j < kMaxLevels; ++j)
                    if ((mk >> j) & 1u) { el[j] -= wv; n1l[j] += 1; }
                auto edge = [&](T x2, double ae) {
                    acc.tv += ae * fabs(xd - (double)x2);
                    if (l != (x2 > thr)) { acc.energy += ae; acc.energy_i += llrint(ae); }
                    const unsigned diff = mk ^ mask_of(x2);
                    const Acc av = EXACT ? (Acc)llrint(ae) : (Acc)ae;
#pragma unroll
                    for (int j = 0; j < kMaxLevels; ++j)
                        if ((diff >> j) & 1u) el[j] += av;
                };
                if (c + 1 < W) edge(A.xout[g + 1], (double)A.a1[D.aoff1 + c * H + r]);
                if (r + 1 < H) edge(A.xout[g + W], (double)A.a0[D.aoff0 + r * W + c]);
            }
        }
        // block reduction in a fixed order
        __shared__ CheckPartial ws[8];
        __shared__ double se[8];
        __shared__ long long sei[8];
        __shared__ long long sn[8];
        for (int d = 16; d > 0; d >>= 1) {
            acc.energy += __shfl_down_sync(0xffffffffu, acc.energy, d);
            acc.lb += __shfl_down_sync(0xffffffffu, acc.lb, d);
            acc.tv += __shfl_down_sync(0xffffffffu, acc.tv, d);
            acc.ytx += __shfl_down_sync(0xffffffffu, acc.ytx, d);
            acc.xabs = fmax(acc.xabs, __shfl_down_sync(0xffffffffu, acc.xabs, d));
            acc.energy_i += __shfl_down_sync(0xffffffffu, acc.energy_i, d);
            acc.n1 += __shfl_down_sync(0xffffffffu, acc.n1, d);
        }
        __syncthreads();
        if (lane == 0) ws[wid] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            CheckPartial t{0, 0, 0, 0, 0, 0, 0, 0};
            for (int w = 0; w < 8; ++w) {
                t.energy += ws[w].energy; t.lb += ws[w].lb; t.tv += ws[w].tv; t.ytx += ws[w].ytx;
                t.xabs = fmax(t.xabs, ws[w].xabs); t.energy_i += ws[w].energy_i; t.n1 += ws[w].n1;
            }
            A.partials[ri] = t;
        }
        for (int j = 0; j < L; ++j) {
            Acc a = el[j];
            long long c = n1l[j];
            for (int d = 16; d > 0; d >>= 1) {
                a += __shfl_down_sync(0xffffffffu, a, d);
                c += __shfl_down_sync(0xffffffffu, c, d);
            }
            __syncthreads();
            if (lane == 0) {
                if (EXACT) sei[wid] = (long long)a;
                else se[wid] = (double)a;
                sn[wid] = c;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double ta = 0.0;
                long long tb = 0, tc = 0;
                for (int w = 0; w < 8; ++w) {
                    if (EXACT) tb += sei[w];
                    else ta += se[w];
                    tc += sn[w];
                }
                if (EXACT) ta = (double)tb;
                A.lpartials[ri].energy[j] = ta;
                A.lpartials[ri].energy_i[j] = tb;
                A.lpartials[ri].n1[j] = tc;
            }
        }
    }
}

// One CTA per grid: sum that grid's row-item partials in order.
__global__ void __launch_bounds__(32) batch_finalize_kernel(const RowItem* rows, int nrows, const int* first_row,
                                                            const CheckPartial* partials, const LevelPartial* lpart,
                                                            int L, CheckPartial* gsum, LevelPartial* glev)
{
    const int g = blockIdx.x;
    const int r0 = first_row[g], r1 = first_row[g + 1];
    if (threadIdx.x == 0) {
        CheckPartial t{0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = r0; i < r1; ++i) {
            const CheckPartial& p = partials[i];
            t.energy += p.energy; t.lb += p.lb; t.tv += p.tv; t.ytx += p.ytx;
            t.xabs = fmax(t.xabs, p.xabs); t.energy_i += p.energy_i; t.n1 += p.n1;
        }
        gsum[g] = t;
    }
    const int j = threadIdx.x;
    if (j < L) {
        double a = 0.0;
        long long b = 0, c = 0;
        for (int i = r0; i < r1; ++i) {
            a += lpart[i].energy[j];
            b += lpart[i].energy_i[j];
            c += lpart[i].n1[j];
        }
        glev[g].energy[j] = a;
        glev[g].energy_i[j] = b;
        glev[g].n1[j] = c;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) batch_labels_kernel(BatchArgs<T> A)
{
    for (int ri = blockIdx.x; ri < A.nrows; ri += gridDim.x) {
        const RowItem R = A.rows[ri];
        const GridDesc D = A.grids[R.g];
        const T thr = A.best_level[R.g];
        const int64_t b = D.off + (int64_t)R.r0 * D.W, e = D.off + (int64_t)R.r1 * D.W;
        for (int64_t g = b + threadIdx.x; g < e; g += blockDim.x) A.labels[g] = (uint8_t)(A.xout[g] > thr);
    }
}

template <typename T>
__global__ void batch_cold_ap_kernel(BatchArgs<T> A)
{
    // lambda_k = w / 2 on every vertex of every grid (the row block transposed)
    for (int ti = blockIdx.x; ti < A.ntiles; ti += gridDim.x) {
        const Tile tile = A.tiles[ti];
        const GridDesc D = A.grids[tile.g];
        for (int k = threadIdx.x; k < 1024; k += blockDim.x) {
            const int64_t r = tile.r0 + (k >> 5), c = tile.c0 + (k & 31);
            if (r >= D.H || c >= D.W) continue;
            const T v = A.w[D.off + r * D.W + c] / T(2);
            A.s0[D.off + r * D.W + c] = v;
            A.s1[D.off + c * D.H + r] = v;
        }
    }
}

}  // namespace

// ------------------------------------------------------------------------------------
// host side

struct tvcut_batch_ctx {
    int G = 0;
    tvcut_params p;
    cudaStream_t stream = nullptr;
    int esize = 4;
    std::vector<GridDesc> grids;
    int64_t n = 0, na0 = 0, na1 = 0;
    // device
    GridDesc* d_grids = nullptr;
    ScanItem* d_items = nullptr;
    Tile* d_tiles = nullptr;
    RowItem* d_rows = nullptr;
    int* d_first_row = nullptr;
    int* d_counter = nullptr;
    void *s0 = nullptr, *s1 = nullptr, *x0 = nullptr, *x1 = nullptr, *w = nullptr, *a0 = nullptr, *a1 = nullptr;
    void *ap0 = nullptr, *ap1 = nullptr;  // a0 / a1 padded to the state layouts
    void *p0 = nullptr, *p1 = nullptr;   // FISTA: the other iterate buffers
    double* mom = nullptr;               // FISTA: t_{k-1}, t_k
    bool flip = false;                   // FISTA: the current iterate is in p0/p1
    void* xout = nullptr;
    void* stage = nullptr;            // staging of one grid's host input (max grid bytes x 8)
    uint8_t* labels = nullptr;
    void* levels = nullptr;           // G x kMaxLevels
    void* best = nullptr;             // G
    CheckPartial* partials = nullptr;
    LevelPartial* lpartials = nullptr;
    CheckPartial* gsum = nullptr;
    LevelPartial* glev = nullptr;
    int* d_flags = nullptr;
    unsigned* d_absmax = nullptr;
    int nitems = 0, ntiles = 0, nrows = 0;
    std::vector<double> wmax;
    std::vector<char> have_w, have_a0, have_a1, int_w, int_a0, int_a1;
    std::vector<double> host_levels;  // G x L
    int L = 0;
    // host mirrors of the per-grid check results
    std::vector<CheckPartial> h_gsum;
    std::vector<LevelPartial> h_glev;
    std::vector<tvcut_stats> stats;
    int64_t iters = 0;
    bool checked = false;
    // launch configuration (autotuned)
    int scan_threads = 128;
    int scan_ctas_per_sm = 8;
    int scan_step = 1;                // form of the chain scan step (VAR of batch_scan_kernel)
    int sms = 152;
    // graph cache
    cudaGraphExec_t graph = nullptr;
    int64_t graph_iters = -1;
    bool graph_flip = false;
    std::string err;
};

static thread_local std::string g_berr;

static tvcut_status bfail(tvcut_batch_t b, tvcut_status st, const std::string& m)
{
    if (b) b->err = m;
    else g_berr = m;
    return st;
}

static tvcut_status bcuda(tvcut_batch_t b, cudaError_t e, const char* where)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? TVCUT_ERR_OOM : TVCUT_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define BCK(b, expr, where)                                    \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return bcuda(b, e_, where);     \
    } while (0)

extern "C" const char* tvcut_batch_last_error(tvcut_batch_t b)
{
    return b ? b->err.c_str() : g_berr.c_str();
}

extern "C" void tvcut_batch_destroy(tvcut_batch_t b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    void* ptrs[] = {b->d_grids, b->d_items, b->d_tiles, b->d_rows, b->d_first_row, b->d_counter, b->s0, b->s1,
                    b->x0, b->x1, b->w, b->a0, b->a1, b->ap0, b->ap1, b->xout, b->stage, b->labels, b->levels, b->best,
                    b->partials, b->lpartials, b->gsum, b->glev, b->d_flags, b->d_absmax, b->p0, b->p1, b->mom};
    for (void* q : ptrs) cudaFree(q);
    delete b;
}

extern "C" tvcut_status tvcut_batch_create(int G, const int64_t* dims, const tvcut_params* p, void* stream,
                                           tvcut_batch_t* out)
{
    if (!out) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_create: out is NULL");
    *out = nullptr;
    if (G < 1 || !dims) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_create: need G >= 1 grids");
    tvcut_params prm;
    tvcut_default_params(&prm);
    if (p) prm = *p;
    if ((prm.algo != TVCUT_AAR && prm.algo != TVCUT_AP && prm.algo != TVCUT_FISTA) || (prm.iterate_dtype != TVCUT_F32 && prm.iterate_dtype != TVCUT_F64) ||
        prm.level_sets < 0 || 2 * prm.level_sets + 1 > kMaxLevels || prm.threshold != prm.threshold ||
        (prm.connectivity != 0 && prm.connectivity != 4))
        return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_create: bad params");
    tvcut_batch_t b = new tvcut_batch_ctx();
    b->G = G;
    b->p = prm;
    b->stream = (cudaStream_t)stream;
    b->esize = prm.iterate_dtype == TVCUT_F64 ? 8 : 4;
    b->grids.resize(G);
    int64_t maxn = 0;
    std::vector<ScanItem> items;
    std::vector<Tile> tiles;
    std::vector<RowItem> rows;
    std::vector<int> first_row(G + 1, 0);
    for (int g = 0; g < G; ++g) {
        const int64_t H = dims[2 * g], W = dims[2 * g + 1];
        if (H < 1 || W < 1 || H > (1 << 20) || W > (1 << 20)) {
            delete b;
            return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_create: every grid needs 1 <= H, W <= 2^20");
        }
        GridDesc& D = b->grids[g];
        D.H = (int)H;
        D.W = (int)W;
        D.off = b->n;
        D.aoff0 = b->na0;
        D.aoff1 = b->na1;
        b->n += H * W;
        b->na0 += (H - 1) * W;
        b->na1 += H * (W - 1);
        maxn = std::max(maxn, H * W);
        for (int c = 0; c < W; c += 128) items.push_back({g, 0, c, (int)std::min<int64_t>(128, W - c)});
        for (int c = 0; c < H; c += 128) items.push_back({g, 1, c, (int)std::min<int64_t>(128, H - c)});
        for (int r = 0; r < H; r += 32)
            for (int c = 0; c < W; c += 32) tiles.push_back({g, r, c, 0});
        first_row[g] = (int)rows.size();
        for (int r = 0; r < H; r += 32) rows.push_back({g, r, (int)std::min<int64_t>(H, r + 32), 0});
    }
    first_row[G] = (int)rows.size();
    // longest chains first: better balance for the dynamically fetched items
    std::stable_sort(items.begin(), items.end(), [&](const ScanItem& x, const ScanItem& y) {
        const int lx = x.axis == 0 ? b->grids[x.g].H : b->grids[x.g].W;
        const int ly = y.axis == 0 ? b->grids[y.g].H : b->grids[y.g].W;
        return lx > ly;
    });
    b->nitems = (int)items.size();
    b->ntiles = (int)tiles.size();
    b->nrows = (int)rows.size();
    const size_t es = (size_t)b->esize;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
    };
    A((void**)&b->d_grids, sizeof(GridDesc) * G);
    A((void**)&b->d_items, sizeof(ScanItem) * items.size());
    A((void**)&b->d_tiles, sizeof(Tile) * tiles.size());
    A((void**)&b->d_rows, sizeof(RowItem) * rows.size());
    A((void**)&b->d_first_row, sizeof(int) * (G + 1));
    A((void**)&b->d_counter, sizeof(int) * 4);
    A(&b->s0, es * b->n);
    A(&b->s1, es * b->n);
    A(&b->x0, es * b->n);
    A(&b->x1, es * b->n);
    A(&b->w, es * b->n);
    A(&b->a0, es * b->na0);
    A(&b->a1, es * b->na1);
    A(&b->ap0, es * b->n);
    A(&b->ap1, es * b->n);
    A(&b->xout, es * b->n);
    if (prm.algo == TVCUT_FISTA) {
        A(&b->p0, es * b->n);
        A(&b->p1, es * b->n);
        A((void**)&b->mom, 2 * sizeof(double));
    }
    A(&b->stage, 8 * (size_t)maxn);
    A((void**)&b->labels, (size_t)b->n);
    A(&b->levels, es * (size_t)G * kMaxLevels);
    A(&b->best, es * (size_t)G);
    A((void**)&b->partials, sizeof(CheckPartial) * rows.size());
    A((void**)&b->lpartials, sizeof(LevelPartial) * rows.size());
    A((void**)&b->gsum, sizeof(CheckPartial) * G);
    A((void**)&b->glev, sizeof(LevelPartial) * G);
    A((void**)&b->d_flags, sizeof(int) * 2);
    A((void**)&b->d_absmax, sizeof(unsigned) * 2);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_grids, b->grids.data(), sizeof(GridDesc) * G, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), sizeof(ScanItem) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_rows, rows.data(), sizeof(RowItem) * rows.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_first_row, first_row.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        tvcut_status st = bcuda(nullptr, e, "tvcut_batch_create");
        tvcut_batch_destroy(b);
        cudaGetLastError();            // clear the runtime's last error
        return st;
    }
    b->wmax.assign(G, 0.0);
    b->have_w.assign(G, 0);
    b->have_a0.assign(G, 0);
    b->have_a1.assign(G, 0);
    b->int_w.assign(G, 0);
    b->int_a0.assign(G, 0);
    b->int_a1.assign(G, 0);
    b->h_gsum.resize(G);
    b->h_glev.resize(G);
    b->stats.resize(G);
    *out = b;
    return TVCUT_OK;
}

template <typename T>
static BatchArgs<T> args_of(tvcut_batch_t b)
{
    BatchArgs<T> A;
    memset(&A, 0, sizeof(A));
    A.grids = b->d_grids;
    A.items = b->d_items;
    A.nitems = b->nitems;
    A.tiles = b->d_tiles;
    A.ntiles = b->ntiles;
    A.rows = b->d_rows;
    A.nrows = b->nrows;
    A.G = b->G;
    A.s0 = (T*)b->s0;
    A.s1 = (T*)b->s1;
    A.x0 = (T*)b->x0;
    A.x1 = (T*)b->x1;
    A.p0 = (T*)b->p0;
    A.p1 = (T*)b->p1;
    A.mom = b->mom;
    if (b->flip) {                       // FISTA: the current iterate is in p
        std::swap(A.s0, A.p0);
        std::swap(A.s1, A.p1);
    }
    A.w = (const T*)b->w;
    A.a0 = (const T*)b->a0;
    A.a1 = (const T*)b->a1;
    A.ap0 = (const T*)b->ap0;
    A.ap1 = (const T*)b->ap1;
    A.xout = (T*)b->xout;
    A.labels = b->labels;
    A.counter = b->d_counter;
    A.threshold = (T)b->p.threshold;
    A.levels = (const T*)b->levels;
    A.nlevels = b->L;
    A.partials = b->partials;
    A.lpartials = b->lpartials;
    A.gsum = b->gsum;
    A.glev = b->glev;
    A.best_level = (const T*)b->best;
    return A;
}

// Copy one grid's array (host or device, any element type) into dst through
// the conversion kernel; `transpose`: dst receives the (rows x cols) array
// transposed.
template <typename T>
static tvcut_status batch_ingest(tvcut_batch_t b, const void* src, int dtype, int space, int64_t rows,
                                 int64_t cols, bool nonneg, bool transpose, T* dst, double* absmax, const char* what)
{
    if (dtype != TVCUT_I32 && dtype != TVCUT_F32 && dtype != TVCUT_F64)
        return bfail(b, TVCUT_ERR_INVALID, std::string(what) + ": bad dtype");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE) return bfail(b, TVCUT_ERR_INVALID, std::string(what) + ": bad space");
    const int64_t count = rows * cols;
    if (count > 0 && !src) return bfail(b, TVCUT_ERR_INVALID, std::string(what) + ": NULL data");
    if (count == 0) return TVCUT_OK;
    const size_t isz = dtype == TVCUT_F64 ? 8 : 4;
    const void* d = src;
    if (space == TVCUT_HOST) {              // raw caller bytes -> staging area (8 x largest grid)
        BCK(b, cudaMemcpyAsync(b->stage, src, isz * (size_t)count, cudaMemcpyHostToDevice, b->stream), what);
        d = b->stage;
    }
    BCK(b, cudaMemsetAsync(b->d_flags, 0, sizeof(int) * 2, b->stream), what);
    BCK(b, cudaMemsetAsync(b->d_absmax, 0, sizeof(unsigned) * 2, b->stream), what);
    T* conv = transpose ? (T*)b->x0 : dst;  // the prox-output array is free outside iterations
    BCK(b, launch_convert<T>(d, dtype, conv, count, nonneg, b->d_flags, b->d_absmax, b->stream), what);
    if (transpose) BCK(b, launch_transpose<T>(conv, dst, rows, cols, b->stream), what);
    int flags = 0;
    unsigned amax = 0;
    BCK(b, cudaMemcpyAsync(&flags, b->d_flags, sizeof(int), cudaMemcpyDeviceToHost, b->stream), what);
    BCK(b, cudaMemcpyAsync(&amax, b->d_absmax, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream), what);
    BCK(b, cudaStreamSynchronize(b->stream), what);
    if (flags & FLAG_NONFINITE) return bfail(b, TVCUT_ERR_INVALID, std::string(what) + ": non-finite value");
    if (flags & FLAG_NEGATIVE) return bfail(b, TVCUT_ERR_INVALID, std::string(what) + ": negative edge weight");
    if (flags & FLAG_INEXACT) return bfail(b, TVCUT_ERR_INVALID, std::string(what) + ": integer not exact in the iterate type");
    if (absmax) {
        float f;
        memcpy(&f, &amax, sizeof(f));
        *absmax = f;
    }
    return TVCUT_OK;
}

// The captured graph bakes in launch parameters that depend on the inputs
// (integer or not); it is rebuilt after any input changes.
static void drop_graph(tvcut_batch_t b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_iters = -1;
}

#define BDISPATCH(b, FN, ...) ((b)->esize == 8 ? FN<double>(__VA_ARGS__) : FN<float>(__VA_ARGS__))

template <typename T>
static tvcut_status bset_unary(tvcut_batch_t b, int g, const void* w, int dtype, int space)
{
    const GridDesc& D = b->grids[g];
    double amax = 0;
    tvcut_status st = batch_ingest<T>(b, w, dtype, space, D.H, D.W, false, false, (T*)b->w + D.off, &amax,
                                      "tvcut_batch_set_unary");
    b->have_w[g] = st == TVCUT_OK;
    if (st != TVCUT_OK) return st;
    b->int_w[g] = dtype == TVCUT_I32;
    b->wmax[g] = amax;
    b->checked = false;
    drop_graph(b);
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_batch_set_unary(tvcut_batch_t b, int g, const void* w, int dtype, int space)
{
    if (!b) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_set_unary: NULL handle");
    if (g < 0 || g >= b->G) return bfail(b, TVCUT_ERR_INVALID, "tvcut_batch_set_unary: grid index out of range");
    return BDISPATCH(b, bset_unary, b, g, w, dtype, space);
}

template <typename T>
static tvcut_status bset_weights(tvcut_batch_t b, int g, int axis, const void* a, int dtype, int space)
{
    const GridDesc& D = b->grids[g];
    tvcut_status st;
    if (axis == 0) {
        st = batch_ingest<T>(b, a, dtype, space, D.H - 1, D.W, true, false, (T*)b->a0 + D.aoff0, nullptr,
                             "tvcut_batch_set_weights");
        b->have_a0[g] = st == TVCUT_OK;
        b->int_a0[g] = dtype == TVCUT_I32;
        if (st == TVCUT_OK) {             // columns: chain c's element j at j W + c, both layouts
            ScanAxis<T> X;
            memset(&X, 0, sizeof(X));
            X.nchains = D.W;
            X.inner = D.W;
            X.m = D.H;
            X.a = (const T*)b->a0 + D.aoff0;
            BCK(b, launch_pad_weights<T>(X, (T*)b->ap0 + D.off, b->stream), "tvcut_batch_set_weights");
        }
    } else {
        st = batch_ingest<T>(b, a, dtype, space, D.H, D.W - 1, true, true, (T*)b->a1 + D.aoff1, nullptr,
                             "tvcut_batch_set_weights");
        b->have_a1[g] = st == TVCUT_OK;
        b->int_a1[g] = dtype == TVCUT_I32;
        if (st == TVCUT_OK) {             // rows: element j of row c at j H + c, both layouts
            ScanAxis<T> X;
            memset(&X, 0, sizeof(X));
            X.nchains = D.H;
            X.inner = 1;
            X.m = D.W;
            X.transposed = 1;
            X.a = (const T*)b->a1 + D.aoff1;
            BCK(b, launch_pad_weights<T>(X, (T*)b->ap1 + D.off, b->stream), "tvcut_batch_set_weights");
        }
    }
    b->checked = false;
    drop_graph(b);
    return st;
}

extern "C" tvcut_status tvcut_batch_set_weights(tvcut_batch_t b, int g, int axis, const void* a, int dtype, int space)
{
    if (!b) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_set_weights: NULL handle");
    if (g < 0 || g >= b->G) return bfail(b, TVCUT_ERR_INVALID, "tvcut_batch_set_weights: grid index out of range");
    if (axis != 0 && axis != 1) return bfail(b, TVCUT_ERR_INVALID, "tvcut_batch_set_weights: axis must be 0 or 1");
    return BDISPATCH(b, bset_weights, b, g, axis, a, dtype, space);
}

static bool batch_ready(tvcut_batch_t b)
{
    for (int g = 0; g < b->G; ++g)
        if (!b->have_w[g] || !b->have_a0[g] || !b->have_a1[g]) return false;
    return true;
}

template <typename T>
static tvcut_status breset(tvcut_batch_t b)
{
    if (b->p.algo == TVCUT_AP) {
        BatchArgs<T> A = args_of<T>(b);
        batch_cold_ap_kernel<T><<<b->sms * 8, 256, 0, b->stream>>>(A);
        BCK(b, cudaGetLastError(), "tvcut_batch_reset");
    } else {
        BCK(b, cudaMemsetAsync(b->s0, 0, (size_t)b->esize * b->n, b->stream), "tvcut_batch_reset");
        BCK(b, cudaMemsetAsync(b->s1, 0, (size_t)b->esize * b->n, b->stream), "tvcut_batch_reset");
    }
    if (b->p.algo == TVCUT_FISTA) {      // y_prev = y = 0, t_0 = t_1 = 1
        static const double one[2] = {1.0, 1.0};
        BCK(b, cudaMemsetAsync(b->p0, 0, (size_t)b->esize * b->n, b->stream), "tvcut_batch_reset");
        BCK(b, cudaMemsetAsync(b->p1, 0, (size_t)b->esize * b->n, b->stream), "tvcut_batch_reset");
        BCK(b, cudaMemcpyAsync(b->mom, one, sizeof(one), cudaMemcpyHostToDevice, b->stream), "tvcut_batch_reset");
        BCK(b, cudaStreamSynchronize(b->stream), "tvcut_batch_reset");
        b->flip = false;
    }
    b->iters = 0;
    b->checked = false;
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_batch_reset(tvcut_batch_t b)
{
    if (!b) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_reset: NULL handle");
    if (!batch_ready(b)) return bfail(b, TVCUT_ERR_STATE, "tvcut_batch_reset: unary and weights of every grid must be set");
    return BDISPATCH(b, breset, b);
}

// Enqueue `iters` iterations and the check (no host synchronisation).
template <typename T>
static cudaError_t enqueue(tvcut_batch_t b, int64_t iters)
{
    BatchArgs<T> A = args_of<T>(b);
    const bool aar = b->p.algo == TVCUT_AAR;
    const bool fista = b->p.algo == TVCUT_FISTA;
    const unsigned scan_grid = (unsigned)(b->sms * b->scan_ctas_per_sm);
    for (int64_t it = 0; it < iters; ++it) {
        A.check = it == iters - 1;
        cudaError_t e = cudaSuccess;
        if (fista) {
            batch_fista_kernel<T, false><<<b->sms * 16, 256, 0, b->stream>>>(A);
            e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream);
            if (e != cudaSuccess) return e;
            if (b->scan_step == 1) batch_scan_kernel<T, 1, true><<<scan_grid, b->scan_threads, 0, b->stream>>>(A);
            else batch_scan_kernel<T, 0, true><<<scan_grid, b->scan_threads, 0, b->stream>>>(A);
            batch_momentum_kernel<<<1, 1, 0, b->stream>>>(b->mom);
            std::swap(A.s0, A.p0);                // the new iterate is where the scan wrote
            std::swap(A.s1, A.p1);
            if (A.check) batch_fista_kernel<T, true><<<b->sms * 16, 256, 0, b->stream>>>(A);
        } else {
            e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream);
            if (e != cudaSuccess) return e;
            if (b->scan_step == 2) batch_scan_kernel<T, 2, false><<<scan_grid, b->scan_threads, 0, b->stream>>>(A);
            else if (b->scan_step == 1) batch_scan_kernel<T, 1, false><<<scan_grid, b->scan_threads, 0, b->stream>>>(A);
            else batch_scan_kernel<T, 0, false><<<scan_grid, b->scan_threads, 0, b->stream>>>(A);
            if (aar) batch_update_kernel<T, UPD_AAR><<<b->sms * 16, 256, 0, b->stream>>>(A);
            else batch_update_kernel<T, UPD_AP><<<b->sms * 16, 256, 0, b->stream>>>(A);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    bool exact = true;
    for (int g = 0; g < b->G; ++g) exact = exact && b->int_w[g] && b->int_a0[g] && b->int_a1[g];
    if (exact) batch_check_kernel<T, true><<<b->sms * 4, 256, 0, b->stream>>>(A);
    else batch_check_kernel<T, false><<<b->sms * 4, 256, 0, b->stream>>>(A);
    batch_finalize_kernel<<<b->G, 32, 0, b->stream>>>(b->d_rows, b->nrows, b->d_first_row, b->partials, b->lpartials,
                                                      b->L, b->gsum, b->glev);
    return cudaGetLastError();
}

template <typename T>
static tvcut_status prepare_levels(tvcut_batch_t b)
{
    b->L = b->p.level_sets > 0 ? 2 * b->p.level_sets + 1 : 0;
    if (b->L == 0) return TVCUT_OK;
    std::vector<T> lv((size_t)b->G * kMaxLevels, T(0));
    b->host_levels.assign((size_t)b->G * b->L, 0.0);
    for (int g = 0; g < b->G; ++g) {
        double* hl = &b->host_levels[(size_t)g * b->L];
        int L = 0;
        hl[L++] = b->p.threshold;
        for (int j = 0; j < b->p.level_sets; ++j) {
            const double d = b->wmax[g] * pow(10.0, -(double)(j + 2));
            hl[L++] = b->p.threshold + d;
            hl[L++] = b->p.threshold - d;
        }
        for (int j = 0; j < b->L; ++j) lv[(size_t)g * b->L + j] = (T)hl[j];
    }
    BCK(b, cudaMemcpyAsync(b->levels, lv.data(), sizeof(T) * (size_t)b->G * b->L, cudaMemcpyHostToDevice, b->stream),
        "levels");
    return TVCUT_OK;
}

template <typename T>
static tvcut_status biterate(tvcut_batch_t b, int64_t iters, tvcut_stats* out)
{
    tvcut_status st = prepare_levels<T>(b);
    if (st != TVCUT_OK) return st;
    if (b->graph_iters != iters || b->graph_flip != b->flip || !b->graph) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaStream_t cs = b->stream;
        bool own = false;
        if (!cs) {                              // capture needs a non-default stream
            BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "tvcut_batch_iterate");
            own = true;
        }
        cudaStream_t saved = b->stream;
        b->stream = cs;
        if (own) BCK(b, cudaStreamSynchronize(saved), "tvcut_batch_iterate");
        cudaGraph_t graph;
        BCK(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "graph capture");
        cudaError_t e = enqueue<T>(b, iters);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        b->stream = saved;
        if (own) cudaStreamDestroy(cs);
        if (e != cudaSuccess) return bcuda(b, e, "graph capture");
        if (e2 != cudaSuccess) return bcuda(b, e2, "graph capture");
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
        b->graph_iters = iters;
        b->graph_flip = b->flip;
    }
    BCK(b, cudaGraphLaunch(b->graph, b->stream), "tvcut_batch_iterate");
    b->iters += iters;
    if (b->p.algo == TVCUT_FISTA && (iters & 1)) b->flip = !b->flip;
    BCK(b, cudaMemcpyAsync(b->h_gsum.data(), b->gsum, sizeof(CheckPartial) * b->G, cudaMemcpyDeviceToHost, b->stream),
        "tvcut_batch_iterate");
    if (b->L > 0)
        BCK(b, cudaMemcpyAsync(b->h_glev.data(), b->glev, sizeof(LevelPartial) * b->G, cudaMemcpyDeviceToHost, b->stream),
            "tvcut_batch_iterate");
    BCK(b, cudaStreamSynchronize(b->stream), "tvcut_batch_iterate");
    // best level per grid, then relabel the grids whose best level is not the threshold
    std::vector<T> bestv(b->G);
    bool relabel = false, all_cert = true;
    for (int g = 0; g < b->G; ++g) {
        const CheckPartial& s = b->h_gsum[g];
        const bool exact = b->int_w[g] && b->int_a0[g] && b->int_a1[g];
        tvcut_stats& o = b->stats[g];
        memset(&o, 0, sizeof(o));
        o.iters = b->iters;
        o.energy = s.energy;
        o.energy_i64 = s.energy_i;
        o.n_label1 = s.n1;
        o.threshold = b->p.threshold;
        int best = 0;
        const LevelPartial& lp = b->h_glev[g];
        for (int j = 1; j < b->L; ++j) {
            const bool lower = exact ? lp.energy_i[j] < lp.energy_i[best] : lp.energy[j] < lp.energy[best];
            if (lower) best = j;
        }
        bestv[g] = (T)(b->L > 0 ? b->host_levels[(size_t)g * b->L + best] : b->p.threshold);
        if (best > 0) {
            o.energy = lp.energy[best];
            o.energy_i64 = lp.energy_i[best];
            o.n_label1 = lp.n1[best];
            o.threshold = b->host_levels[(size_t)g * b->L + best];
            relabel = true;
        }
        o.energy_exact = exact ? 1 : 0;
        o.discrete_lb = s.lb;
        o.tv_value = s.tv;
        o.tv_gap = s.tv - s.ytx;
        o.x_absmax = s.xabs;
        o.certified = (exact && (double)o.energy_i64 - s.lb < 1.0) ? 1 : 0;   // approximate bound only
        o.certified_lb = -INFINITY;
        all_cert = all_cert && o.certified;
    }
    if (relabel) {
        BCK(b, cudaMemcpyAsync(b->best, bestv.data(), sizeof(T) * b->G, cudaMemcpyHostToDevice, b->stream),
            "tvcut_batch_iterate");
        BatchArgs<T> A = args_of<T>(b);
        batch_labels_kernel<T><<<b->sms * 4, 256, 0, b->stream>>>(A);
        BCK(b, cudaGetLastError(), "tvcut_batch_iterate");
        BCK(b, cudaStreamSynchronize(b->stream), "tvcut_batch_iterate");
    }
    b->checked = true;
    if (out) memcpy(out, b->stats.data(), sizeof(tvcut_stats) * b->G);
    return all_cert ? TVCUT_OK : TVCUT_NOT_CONVERGED;
}

extern "C" tvcut_status tvcut_batch_iterate(tvcut_batch_t b, int64_t iters, tvcut_stats* out)
{
    if (!b) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_iterate: NULL handle");
    if (iters < 1) return bfail(b, TVCUT_ERR_INVALID, "tvcut_batch_iterate: iters must be >= 1");
    if (!batch_ready(b)) return bfail(b, TVCUT_ERR_STATE, "tvcut_batch_iterate: unary and weights of every grid must be set");
    return BDISPATCH(b, biterate, b, iters, out);
}

extern "C" tvcut_status tvcut_batch_cut(tvcut_batch_t b, int g, uint8_t* labels, int space, tvcut_stats* out)
{
    if (!b) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_cut: NULL handle");
    if (g < 0 || g >= b->G) return bfail(b, TVCUT_ERR_INVALID, "tvcut_batch_cut: grid index out of range");
    if (!b->checked) return bfail(b, TVCUT_ERR_STATE, "tvcut_batch_cut: run tvcut_batch_iterate first");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE) return bfail(b, TVCUT_ERR_INVALID, "tvcut_batch_cut: bad space");
    const GridDesc& D = b->grids[g];
    if (labels) {
        BCK(b, cudaMemcpyAsync(labels, b->labels + D.off, (size_t)D.H * D.W,
                               space == TVCUT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, b->stream),
            "tvcut_batch_cut");
        BCK(b, cudaStreamSynchronize(b->stream), "tvcut_batch_cut");
    }
    if (out) *out = b->stats[g];
    return TVCUT_OK;
}

template <typename T>
static tvcut_status bget_state(tvcut_batch_t b, int g, void* s, int space)
{
    const GridDesc& D = b->grids[g];
    const int64_t n = (int64_t)D.H * D.W;
    const cudaMemcpyKind k = space == TVCUT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const BatchArgs<T> A = args_of<T>(b);            // the current iterate (FISTA: either buffer)
    BCK(b, cudaMemcpyAsync(s, A.s0 + D.off, sizeof(T) * n, k, b->stream), "tvcut_batch_get_state");
    BCK(b, launch_transpose<T>(A.s1 + D.off, (T*)b->stage, D.W, D.H, b->stream), "tvcut_batch_get_state");
    BCK(b, cudaMemcpyAsync((T*)s + n, b->stage, sizeof(T) * n, k, b->stream), "tvcut_batch_get_state");
    BCK(b, cudaStreamSynchronize(b->stream), "tvcut_batch_get_state");
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_batch_get_state(tvcut_batch_t b, int g, void* s, int space)
{
    if (!b) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_get_state: NULL handle");
    if (g < 0 || g >= b->G || !s) return bfail(b, TVCUT_ERR_INVALID, "tvcut_batch_get_state: bad grid or NULL output");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE) return bfail(b, TVCUT_ERR_INVALID, "tvcut_batch_get_state: bad space");
    return BDISPATCH(b, bget_state, b, g, s, space);
}

// Autotuner: time the scan launch (it writes only the prox outputs, so the
// state is untouched) for each CTA size and CTA count per SM, keep the fastest.
template <typename T>
static tvcut_status bautotune(tvcut_batch_t b, int* chosen)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_iters = -1;
    }
    BatchArgs<T> A = args_of<T>(b);
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0), "autotune");
    BCK(b, cudaEventCreate(&e1), "autotune");
    const int threads[] = {64, 128, 256};
    const int per_sm[] = {4, 8, 16};
    float best = 1e30f;
    int bt = b->scan_threads, bp = b->scan_ctas_per_sm, bv = b->scan_step;
    for (int pv = 0; pv < 3; ++pv)
        for (int t : threads)
            for (int q : per_sm) {
                float tot = 0.f;
                for (int rep = 0; rep < 3; ++rep) {
                    BCK(b, cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream), "autotune");
                    BCK(b, cudaEventRecord(e0, b->stream), "autotune");
                    if (pv == 2) batch_scan_kernel<T, 2, false><<<b->sms * q, t, 0, b->stream>>>(A);
                    else if (pv == 1) batch_scan_kernel<T, 1, false><<<b->sms * q, t, 0, b->stream>>>(A);
                    else batch_scan_kernel<T, 0, false><<<b->sms * q, t, 0, b->stream>>>(A);
                    BCK(b, cudaGetLastError(), "autotune");
                    BCK(b, cudaEventRecord(e1, b->stream), "autotune");
                    BCK(b, cudaEventSynchronize(e1), "autotune");
                    float ms = 0.f;
                    BCK(b, cudaEventElapsedTime(&ms, e0, e1), "autotune");
                    if (rep > 0) tot += ms;
                }
                if (tot < best) {
                    best = tot;
                    bt = t;
                    bp = q;
                    bv = pv;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->scan_threads = bt;
    b->scan_ctas_per_sm = bp;
    b->scan_step = bv;
    if (chosen) {
        chosen[0] = bt;
        chosen[1] = bp;
        chosen[2] = bv;
    }
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_batch_set_launch(tvcut_batch_t b, int threads, int ctas_per_sm, int step)
{
    if (!b) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_set_launch: NULL handle");
    if ((threads != 64 && threads != 128 && threads != 256) || ctas_per_sm < 1 || ctas_per_sm > 32 || step < 0 ||
        step > 2)
        return bfail(b, TVCUT_ERR_INVALID, "tvcut_batch_set_launch: threads 64/128/256, ctas_per_sm 1..32, step 0..2");
    b->scan_threads = threads;
    b->scan_ctas_per_sm = ctas_per_sm;
    b->scan_step = step;
    drop_graph(b);
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_batch_autotune(tvcut_batch_t b, int* chosen)
{
    if (!b) return bfail(nullptr, TVCUT_ERR_INVALID, "tvcut_batch_autotune: NULL handle");
    if (!batch_ready(b)) return bfail(b, TVCUT_ERR_STATE, "tvcut_batch_autotune: set every grid first");
    return BDISPATCH(b, bautotune, b, chosen);
}
