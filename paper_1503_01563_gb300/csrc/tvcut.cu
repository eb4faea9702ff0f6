// C-ABI of tvcut (declared in include/tvcut.h): handle, device buffers and
// the iteration driver of the methods of Sec. 4 (AAR, AP, BCD, FISTA).
//
// With r blocks (one per axis, or four on an 8-connected 2D grid), AAR
// (Eq. 3 and Eq. dualA) is
//   z_k <- y_k + (w - 2 sum_j y_j + sum_j z_j) / r ,   y = Pi_K(z),
// and AP (Sec. 4.2) lambda_k <- y_k + (w - sum_j y_j) / r.  The default (scan)
// schedule runs one scan launch over all blocks and one update launch
// (scan.cu); the fused schedules (mapping 1-4, sweep.cu) run one sweep per
// block, the last one updating every block state.  BCD and FISTA keep the
// duals y and alternate a preparation pass with the scan in projection mode.
// On check iterations the primal x = w - sum_k y_k is written for the check
// kernels (aux.cu) to threshold and evaluate.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "tvcut_internal.cuh"

using namespace tvcut;

struct tvcut_ctx {
    int ndim = 0;
    int nblk = 0;                  // blocks: ndim, or 4 for an 8-connected 2D grid
    bool conn8 = false;
    int64_t dims[3] = {1, 1, 1};
    int64_t n = 0;
    tvcut_params p;
    cudaStream_t stream = nullptr;
    int esize = 4;                 // bytes of the iterate type
    void* state = nullptr;         // ndim * n
    void* w = nullptr;             // n
    void* a[4] = {nullptr, nullptr, nullptr, nullptr};   // per block, in the block's layout
    int64_t a_len[4] = {0, 0, 0, 0};                      // input length per weight axis
    void* ap[4] = {nullptr, nullptr, nullptr, nullptr};  // the same weights padded to the state's layout
    void* adiag = nullptr;         // 8-connected: diagonal / anti-diagonal weights, (H-1) x (W-1) row-major
    void* aanti = nullptr;
    void* scratch = nullptr;       // 2n: P | x  (also the staging area of host inputs)
    void* xk = nullptr;            // ndim * n: per-block prox outputs of the scan schedule
    void* yprev = nullptr;         // FISTA: ndim * n, the previous iterate (swaps with state)
    double fista_tprev = 1.0;      // FISTA momentum sequence: t_{k-1} and t_k of the next step
    double fista_t = 1.0;
    bool tlast = true;             // scan schedule: block ndim-1 (state, weights) stored transposed
    uint8_t* labels = nullptr;     // n
    double* ycert = nullptr;       // n, FP64: the exactly feasible dual of the rigorous bound (on first use)
    double* y64 = nullptr;         // FP32 iterates: nblk * n FP64 block duals for the bound (on first use)
    double* a64 = nullptr;         // nblk * n: the blocks' weights in FP64
    double* w64 = nullptr;         // n: the unary in FP64
    double* t64 = nullptr;         // n: FP64 scratch
    double* lbpart = nullptr;      // 2 * kCheckBlocks partial sums of that bound
    CheckPartial* partials = nullptr;
    LevelPartial* level_partials = nullptr;
    double wmax = 0.0;             // max |w|: scale of the level-set ladder
    double amax[4] = {0, 0, 0, 0}; // max a per weight axis (scale of the learned warm start's features)
    DevStatus* dstatus = nullptr;
    DevStatus* hstatus = nullptr;  // pinned
    bool have_w = false, have_a[4] = {false, false, false, false};
    bool int_w = false, int_a[4] = {false, false, false, false};
    bool x_valid = false, labels_valid = false;
    int64_t iters = 0;
    tvcut_stats last;
    std::string err;
    // tracing: launch counts per kernel kind, and (when enabled) device time
    // from CUDA events recorded around each launch on the handle's stream
    bool prof = false;
    double prof_ms[TVCUT_NKINDS] = {0, 0, 0, 0};
    int64_t launches[TVCUT_NKINDS] = {0, 0, 0, 0};
    struct Pending { int kind; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool;
};

static thread_local std::string g_err;

namespace tvcut {
// Record a failure of a call without a handle (read by tvcut_last_error(NULL)).
void set_thread_error(const std::string& msg) { g_err = msg; }
}  // namespace tvcut

static tvcut_status fail(tvcut_t h, tvcut_status st, const std::string& msg)
{
    if (h) h->err = msg;
    else g_err = msg;
    return st;
}

static tvcut_status cuda_fail(tvcut_t h, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? TVCUT_ERR_OOM : TVCUT_ERR_CUDA, m);
}

#define CK(h, expr, where)                                  \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
    } while (0)

extern "C" void tvcut_default_params(tvcut_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->algo = TVCUT_AAR;
    p->iterate_dtype = TVCUT_F32;
    p->check_every = 10;
    p->mapping = -1;
    p->gap_tol = 0.0;
    p->threshold = 0.0;
    p->level_sets = 8;
}

extern "C" const char* tvcut_last_error(tvcut_t h)
{
    return h ? h->err.c_str() : g_err.c_str();
}

extern "C" void tvcut_destroy(tvcut_t h)
{
    if (!h) return;
    cudaFree(h->state);
    cudaFree(h->w);
    for (int k = 0; k < 4; ++k) cudaFree(h->a[k]);
    for (int k = 0; k < 4; ++k) cudaFree(h->ap[k]);
    cudaFree(h->adiag);
    cudaFree(h->aanti);
    cudaFree(h->scratch);
    cudaFree(h->xk);
    cudaFree(h->yprev);
    cudaFree(h->labels);
    cudaFree(h->ycert);
    cudaFree(h->lbpart);
    cudaFree(h->y64);
    cudaFree(h->a64);
    cudaFree(h->w64);
    cudaFree(h->t64);
    cudaFree(h->partials);
    cudaFree(h->level_partials);
    cudaFree(h->dstatus);
    cudaFreeHost(h->hstatus);
    for (auto& p : h->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    delete h;
}

static bool valid_params(const tvcut_params* p, std::string& why)
{
    if (p->algo != TVCUT_AAR && p->algo != TVCUT_AP && p->algo != TVCUT_BCD && p->algo != TVCUT_FISTA) {
        why = "params.algo must be TVCUT_AAR, TVCUT_AP, TVCUT_BCD or TVCUT_FISTA";
        return false;
    }
    if ((p->algo == TVCUT_BCD || p->algo == TVCUT_FISTA) && p->mapping >= 1 && p->mapping <= 4) {
        why = "TVCUT_BCD and TVCUT_FISTA run on the scan schedule (mapping -1, 0 or 5..9)";
        return false;
    }
    if (p->iterate_dtype != TVCUT_F32 && p->iterate_dtype != TVCUT_F64) { why = "params.iterate_dtype must be TVCUT_F32 or TVCUT_F64"; return false; }
    if (p->check_every < 1) { why = "params.check_every must be >= 1"; return false; }
    if (p->mapping < -1 || p->mapping > 11) { why = "params.mapping must be -1 (auto) or 0..11"; return false; }
    if (!(p->gap_tol >= 0.0)) { why = "params.gap_tol must be >= 0"; return false; }
    if (p->threshold != p->threshold) { why = "params.threshold is NaN"; return false; }
    if (p->level_sets < 0 || 2 * p->level_sets + 1 > kMaxLevels) { why = "params.level_sets must be in [0, 8]"; return false; }
    if (p->certify < 0 || p->certify > 2) { why = "params.certify must be 0, 1 or 2"; return false; }
    if (p->stop_on_approx != 0 && p->stop_on_approx != 1) { why = "params.stop_on_approx must be 0 or 1"; return false; }
    for (int i = 0; i < 4; ++i) if (p->reserved[i]) { why = "params.reserved must be zero"; return false; }
    if (p->connectivity != 0 && p->connectivity != 4 && p->connectivity != 6 && p->connectivity != 8) {
        why = "params.connectivity must be 0, 4, 6 or 8";
        return false;
    }
    if (p->connectivity == 8 && p->mapping >= 1 && p->mapping <= 4) {
        why = "connectivity 8 runs on the scan schedule (mapping -1, 0 or 5..9)";
        return false;
    }
    return true;
}

extern "C" tvcut_status tvcut_create(int ndim, const int64_t* dims, const tvcut_params* p,
                                     void* cuda_stream, tvcut_t* out)
{
    if (!out) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_create: out is NULL");
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_create: ndim must be 2 or 3");
    if (!dims) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_create: dims is NULL");
    int64_t n = 1;
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 1 || dims[k] > (int64_t)1 << 30)
            return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_create: every dims[k] must be in [1, 2^30]");
        n *= dims[k];
        if (n > ((int64_t)1 << 40)) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_create: grid too large");
    }
    tvcut_params prm;
    tvcut_default_params(&prm);
    if (p) prm = *p;
    std::string why;
    if (!valid_params(&prm, why)) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_create: " + why);

    if ((prm.connectivity == 8 && ndim != 2) || (prm.connectivity == 4 && ndim != 2) ||
        (prm.connectivity == 6 && ndim != 3))
        return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_create: connectivity 4 and 8 need ndim 2, 6 needs ndim 3");
    tvcut_t h = new tvcut_ctx();
    h->ndim = ndim;
    h->conn8 = prm.connectivity == 8;
    h->nblk = h->conn8 ? 4 : ndim;
    for (int k = 0; k < ndim; ++k) h->dims[k] = dims[k];
    h->n = n;
    h->p = prm;
    h->stream = (cudaStream_t)cuda_stream;
    h->esize = prm.iterate_dtype == TVCUT_F64 ? 8 : 4;
    h->tlast = prm.mapping <= 0 || prm.mapping >= 5;
    memset(&h->last, 0, sizeof(h->last));
    const size_t es = (size_t)h->esize;
    cudaError_t e = cudaSuccess;
    const int nb = h->nblk;
    if (e == cudaSuccess) e = cudaMalloc(&h->state, es * (size_t)(nb * n));
    if (e == cudaSuccess) e = cudaMalloc(&h->w, es * (size_t)n);
    for (int k = 0; k < ndim && e == cudaSuccess; ++k) {
        h->a_len[k] = n / dims[k] * (dims[k] - 1);
        e = cudaMalloc(&h->a[k], es * (size_t)(h->a_len[k] > 0 ? h->a_len[k] : 1));
    }
    if (h->conn8) {                // path weights of blocks 2, 3 ((W-1) x H) and the diagonal inputs
        const int64_t nd = (dims[0] - 1) * (dims[1] - 1), nz = (dims[1] - 1) * dims[0];
        h->a_len[2] = h->a_len[3] = nd;
        for (int k = 2; k < 4 && e == cudaSuccess; ++k) e = cudaMalloc(&h->a[k], es * (size_t)(nz > 0 ? nz : 1));
        if (e == cudaSuccess) e = cudaMalloc(&h->adiag, es * (size_t)(nd > 0 ? nd : 1));
        if (e == cudaSuccess) e = cudaMalloc(&h->aanti, es * (size_t)(nd > 0 ? nd : 1));
    }
    // padded copies for the thread scan (the block-transposed schedule only)
    for (int k = 0; k < nb && e == cudaSuccess && h->tlast; ++k) e = cudaMalloc(&h->ap[k], es * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&h->scratch, es * (size_t)(2 * n));
    if (e == cudaSuccess) e = cudaMalloc(&h->xk, es * (size_t)(nb * n));
    if (e == cudaSuccess && prm.algo == TVCUT_FISTA) e = cudaMalloc(&h->yprev, es * (size_t)(nb * n));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->labels, (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->partials, sizeof(CheckPartial) * kCheckBlocks);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->level_partials, sizeof(LevelPartial) * kCheckBlocks);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->dstatus, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->hstatus, sizeof(DevStatus));
    if (e != cudaSuccess) {
        tvcut_status st = cuda_fail(nullptr, e, "tvcut_create: allocation");
        tvcut_destroy(h);
        cudaGetLastError();            // clear the runtime's last error: later calls must not see it
        return st;
    }
    *out = h;
    return TVCUT_OK;
}

// ---- typed helpers --------------------------------------------------------

template <typename T>
static T* P_of(tvcut_t h) { return (T*)h->scratch; }
template <typename T>
static T* X_of(tvcut_t h) { return (T*)h->scratch + h->n; }
template <typename T>
static T* S_of(tvcut_t h, int k) { return (T*)h->state + (int64_t)k * h->n; }
template <typename T>
static T* XK_of(tvcut_t h, int k) { return (T*)h->xk + (int64_t)k * h->n; }
static int64_t cols_of(tvcut_t h) { return h->dims[h->ndim - 1]; }
// mapping 5: thread per chain; 6, 7, 8, 9: 32, 16, 8, 4 lanes per chain; 10:
// the message-passing chain prox (mpprox.cu), a CTA per chain
static int scan_force(int mapping) { return mapping >= 5 ? mapping - 4 : 0; }
static int64_t rows_of(tvcut_t h) { return h->n / h->dims[h->ndim - 1]; }

// In-place layout change of an (rows x cols) array through the xk area
// (free outside iterations): natural -> transposed (forward) or back.
template <typename T>
static cudaError_t relayout(tvcut_t h, T* arr, int64_t rows, int64_t cols, bool forward)
{
    if (rows * cols <= 0) return cudaSuccess;
    T* tmp = XK_of<T>(h, 0);
    cudaError_t e = forward ? launch_transpose<T>(arr, tmp, rows, cols, h->stream)
                            : launch_transpose<T>(arr, tmp, cols, rows, h->stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(arr, tmp, sizeof(T) * (size_t)(rows * cols), cudaMemcpyDeviceToDevice, h->stream);
}

// Layout of block k's state and weights in the scan schedule: 0 natural, 1
// transposed (the last axis' block), 2 / 3 the zig-zag path layouts of an
// 8-connected grid.
static int block_layout(tvcut_t h, int k)
{
    if (h->conn8 && k >= 2) return k;
    return (h->tlast && k == h->ndim - 1) ? 1 : 0;
}

// Scan geometry of block k (chains of the axis, or the H zig-zag paths of length W).
template <typename T>
static ScanAxis<T> block_axis(tvcut_t h, int k, const T* v, T* x)
{
    ScanAxis<T> X;
    memset(&X, 0, sizeof(X));
    if (block_layout(h, k) >= 2) {
        X.nchains = h->dims[0];
        X.inner = 1;
        X.m = (int)h->dims[1];
        X.transposed = 1;
    } else {
        ChainGeom g = chain_geom(h->ndim, h->dims, k);
        X.nchains = g.nchains;
        X.inner = g.inner;
        X.m = g.m;
        X.transposed = block_layout(h, k) == 1 ? 1 : 0;
    }
    X.v = v;
    X.a = (const T*)h->a[k];
    X.ap = (const T*)h->ap[k];
    X.x = x;
    return X;
}

// Block k of a state from grid layout to its own, in place (through the xk area).
template <typename T>
static cudaError_t to_internal(tvcut_t h, int k, T* arr)
{
    const int L = block_layout(h, k);
    if (L == 0) return cudaSuccess;
    if (L == 1) return relayout<T>(h, arr, rows_of(h), cols_of(h), true);
    T* tmp = XK_of<T>(h, 0);
    cudaError_t e = launch_zz_relayout<T>(arr, tmp, (int)h->dims[0], (int)h->dims[1], L, true, h->stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(arr, tmp, sizeof(T) * (size_t)h->n, cudaMemcpyDeviceToDevice, h->stream);
}

// Block k of a state from its own layout to grid layout, out of place.
template <typename T>
static cudaError_t to_natural(tvcut_t h, int k, const T* arr, T* out)
{
    const int L = block_layout(h, k);
    if (L == 0) return cudaMemcpyAsync(out, arr, sizeof(T) * (size_t)h->n, cudaMemcpyDeviceToDevice, h->stream);
    if (L == 1) return launch_transpose<T>(arr, out, cols_of(h), rows_of(h), h->stream);
    return launch_zz_relayout<T>(arr, out, (int)h->dims[0], (int)h->dims[1], L, false, h->stream);
}

// ---- tracing ----------------------------------------------------------------

static cudaError_t take_event(tvcut_t h, cudaEvent_t* e)
{
    if (!h->ev_pool.empty()) {
        *e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

// Launch `nk` kernels through `fn` as one traced group of kind `kind`.
template <class F>
static cudaError_t traced(tvcut_t h, int kind, int nk, F&& fn)
{
    h->launches[kind] += nk;
    if (!h->prof) return fn();
    cudaEvent_t a, b;
    cudaError_t e = take_event(h, &a);
    if (e == cudaSuccess) e = take_event(h, &b);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(a, h->stream);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(b, h->stream);
    h->pending.push_back({kind, a, b});
    return e;
}

// Accumulate the pending event pairs; call only after the stream synchronised.
static cudaError_t flush_trace(tvcut_t h)
{
    cudaError_t err = cudaSuccess;
    for (auto& p : h->pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e == cudaSuccess) h->prof_ms[p.kind] += ms;
        else if (err == cudaSuccess) err = e;
        h->ev_pool.push_back(p.a);
        h->ev_pool.push_back(p.b);
    }
    h->pending.clear();
    return err;
}

static size_t dtype_size(int dt)
{
    return dt == TVCUT_F64 ? 8 : 4;
}

// Bring a caller array (host or device) into `dst` (iterate type), validating.
template <typename T>
static tvcut_status ingest(tvcut_t h, const void* src, int dtype, int space, int64_t count,
                           bool nonneg, T* dst, const char* what)
{
    if (dtype != TVCUT_I32 && dtype != TVCUT_F32 && dtype != TVCUT_F64)
        return fail(h, TVCUT_ERR_INVALID, std::string(what) + ": dtype must be TVCUT_I32, TVCUT_F32 or TVCUT_F64");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE)
        return fail(h, TVCUT_ERR_INVALID, std::string(what) + ": space must be TVCUT_HOST or TVCUT_DEVICE");
    if (count > 0 && !src) return fail(h, TVCUT_ERR_INVALID, std::string(what) + ": NULL data");
    const void* dsrc = src;
    if (space == TVCUT_HOST && count > 0) {
        // staging in the scratch area (2n iterate values >= count * 8 bytes)
        CK(h, cudaMemcpyAsync(h->scratch, src, dtype_size(dtype) * (size_t)count, cudaMemcpyHostToDevice, h->stream), what);
        dsrc = h->scratch;
    }
    int* dflags = &h->dstatus->flags;       // flags and absmax_bits are adjacent
    CK(h, cudaMemsetAsync(dflags, 0, 2 * sizeof(int), h->stream), what);
    if (count > 0)
        CK(h, traced(h, TVCUT_K_OTHER, 1, [&] {
               return launch_convert<T>(dsrc, dtype, dst, count, nonneg, dflags, &h->dstatus->absmax_bits, h->stream);
           }), what);
    CK(h, cudaMemcpyAsync(&h->hstatus->flags, dflags, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream), what);
    CK(h, cudaStreamSynchronize(h->stream), what);
    CK(h, flush_trace(h), what);
    const int f = h->hstatus->flags;
    if (f & FLAG_NONFINITE) return fail(h, TVCUT_ERR_INVALID, std::string(what) + ": non-finite value");
    if (f & FLAG_NEGATIVE) return fail(h, TVCUT_ERR_INVALID, std::string(what) + ": negative edge weight (energy not submodular)");
    if (f & FLAG_INEXACT) return fail(h, TVCUT_ERR_INVALID, std::string(what) + ": integer too large to be exact in the iterate type (|v| <= 2^24 for FP32)");
    return TVCUT_OK;
}

// FISTA: start the momentum afresh from the current state (previous iterate =
// current, t = 1), as at a cold start; a no-op for the other methods.
static cudaError_t restart_momentum(tvcut_t h)
{
    h->fista_tprev = h->fista_t = 1.0;
    if (h->p.algo != TVCUT_FISTA) return cudaSuccess;
    return cudaMemcpyAsync(h->yprev, h->state, (size_t)h->esize * (size_t)(h->nblk * h->n),
                           cudaMemcpyDeviceToDevice, h->stream);
}

template <typename T>
static tvcut_status cold_start(tvcut_t h)
{
    if (h->p.algo == TVCUT_AP) {
        CK(h, traced(h, TVCUT_K_OTHER, 1, [&] { return launch_cold_ap<T>((const T*)h->w, (T*)h->state, h->nblk, h->n, h->stream); }),
           "cold start");
        for (int k = 0; k < h->nblk; ++k)
            CK(h, traced(h, TVCUT_K_OTHER, 1, [&] { return to_internal<T>(h, k, S_of<T>(h, k)); }), "cold start");
    } else {
        CK(h, cudaMemsetAsync(h->state, 0, (size_t)h->esize * (size_t)(h->nblk * h->n), h->stream), "cold start");
    }
    CK(h, restart_momentum(h), "cold start");
    h->iters = 0;
    h->x_valid = h->labels_valid = false;
    return TVCUT_OK;
}

static bool inputs_ready(tvcut_t h)
{
    if (!h->have_w) return false;
    for (int k = 0; k < h->nblk; ++k) if (!h->have_a[k]) return false;
    return true;
}

// One pass over the blocks.  mode_first/mid/last select the epilogues.
template <typename T>
static cudaError_t run_sweeps(tvcut_t h, int first, int mid, int last, int check)
{
    const int r = h->ndim;
    for (int k = 0; k < r; ++k) {
        SweepArgs<T> A;
        memset(&A, 0, sizeof(A));
        A.g = chain_geom(h->ndim, h->dims, k);
        A.v = S_of<T>(h, k);
        A.a = (const T*)h->a[k];
        A.out = S_of<T>(h, k);
        A.P = P_of<T>(h);
        A.w = (const T*)h->w;
        for (int j = 0; j < r; ++j) A.Z[j] = S_of<T>(h, j);
        A.x = X_of<T>(h);
        A.r = r;
        A.check = check;
        A.mapping = h->p.mapping == 4 ? 0 : h->p.mapping;
        const int mode = k == 0 ? first : (k == r - 1 ? last : mid);
        const int kind = k == r - 1 ? TVCUT_K_UPDATE : TVCUT_K_PROX;
        cudaError_t e = traced(h, kind, 1, [&] { return launch_sweep<T>(mode, A, h->stream); });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One iteration (or, with mode UPD_EVAL, only the primal of the current
// state).  Scan schedule: one scan launch for all blocks + one update launch;
// fused schedule (mapping 1..4): one sweep per block, the last one updating.
template <typename T>
static Prep8Args<T> prep8_args(tvcut_t h)
{
    Prep8Args<T> A;
    memset(&A, 0, sizeof(A));
    A.rows = h->dims[0];
    A.cols = h->dims[1];
    for (int j = 0; j < 4; ++j) A.y[j] = S_of<T>(h, j);
    A.w = (const T*)h->w;
    A.xout = X_of<T>(h);
    return A;
}

// x = w - sum_k y_k of a state that holds the block duals (BCD, FISTA).
template <typename T>
static cudaError_t primal_of_duals(tvcut_t h)
{
    if (h->conn8) {
        const Prep8Args<T> A = prep8_args<T>(h);
        return traced(h, TVCUT_K_UPDATE, 1, [&] { return launch_prep8<T>(PREP8_PRIMAL, A, h->stream); });
    }
    UpdateArgs<T> U;
    memset(&U, 0, sizeof(U));
    U.rows = rows_of(h);
    U.cols = cols_of(h);
    U.r = h->ndim;
    for (int k = 0; k < h->ndim; ++k) U.s[k] = S_of<T>(h, k);
    U.w = (const T*)h->w;
    U.xout = X_of<T>(h);
    return traced(h, TVCUT_K_UPDATE, 1, [&] { return launch_bcd_prepare<T>(U, -1, h->stream); });
}

// One cycle of block coordinate descent (Sec. 4.1, cyclic projections): for
// k = 0..r-1, v = w - sum_{j != k} y_j, y_k = v - prox_{f_k}(v).  The state
// holds the y_k; on check iterations the primal w - sum_k y_k goes to x.
template <typename T>
static cudaError_t run_bcd(tvcut_t h, int check)
{
    if (h->conn8) {                // four blocks; v_k in block k's own layout
        for (int k = 0; k < 4; ++k) {
            Prep8Args<T> A = prep8_args<T>(h);
            A.k = k;
            A.out[k] = P_of<T>(h);
            cudaError_t e = traced(h, TVCUT_K_UPDATE, 1, [&] { return launch_prep8<T>(PREP8_BCD, A, h->stream); });
            if (e != cudaSuccess) return e;
            ScanArgs<T> S;
            memset(&S, 0, sizeof(S));
            S.naxes = 1;
            S.force = scan_force(h->p.mapping);
            S.shadow = 1;
            S.ax[0] = block_axis<T>(h, k, P_of<T>(h), S_of<T>(h, k));
            e = traced(h, TVCUT_K_PROX, 1, [&] { return launch_scan<T>(S, h->stream); });
            if (e != cudaSuccess) return e;
        }
        return check ? primal_of_duals<T>(h) : cudaSuccess;
    }
    const int r = h->ndim;
    UpdateArgs<T> U;
    memset(&U, 0, sizeof(U));
    U.rows = rows_of(h);
    U.cols = cols_of(h);
    U.r = r;
    for (int k = 0; k < r; ++k) U.s[k] = S_of<T>(h, k);
    U.w = (const T*)h->w;
    U.xout = P_of<T>(h);                                  // v_k, in block k's layout
    for (int k = 0; k < r; ++k) {
        cudaError_t e = traced(h, TVCUT_K_UPDATE, 1, [&] { return launch_bcd_prepare<T>(U, k, h->stream); });
        if (e != cudaSuccess) return e;
        ScanArgs<T> S;
        memset(&S, 0, sizeof(S));
        S.naxes = 1;
        S.force = scan_force(h->p.mapping);
        ChainGeom g = chain_geom(h->ndim, h->dims, k);
        S.ax[0].nchains = g.nchains;
        S.ax[0].inner = g.inner;
        S.ax[0].m = g.m;
        S.ax[0].transposed = k == r - 1 ? 1 : 0;
        S.ax[0].v = P_of<T>(h);
        S.ax[0].a = (const T*)h->a[k];
        if (S.ax[0].transposed == (block_layout(h, k) == 1 ? 1 : 0)) S.ax[0].ap = (const T*)h->ap[k];
        S.ax[0].x = S_of<T>(h, k);
        S.shadow = 1;                                     // y_k = v_k - prox(v_k)
        e = traced(h, TVCUT_K_PROX, 1, [&] { return launch_scan<T>(S, h->stream); });
        if (e != cudaSuccess) return e;
    }
    if (check) {
        U.xout = X_of<T>(h);
        return traced(h, TVCUT_K_UPDATE, 1, [&] { return launch_bcd_prepare<T>(U, -1, h->stream); });
    }
    return cudaSuccess;
}

// One FISTA step on the smooth dual (Sec. 4.1): v = Pi_L(y + beta (y - y_prev))
// for all blocks, then y_prev <- Pi_K(v) by the scan (all blocks in one
// launch, projection mode), then the two buffers swap so that the state holds
// the new iterate.  beta = (t_{k-1} - 1) / t_k with t_0 = t_1 = 1.
template <typename T>
static cudaError_t run_fista(tvcut_t h, int check)
{
    const int r = h->nblk;
    const T beta = (T)((h->fista_tprev - 1.0) / h->fista_t);
    cudaError_t e;
    if (h->conn8) {
        Prep8Args<T> A = prep8_args<T>(h);
        A.beta = beta;
        for (int k = 0; k < 4; ++k) {
            A.p[k] = (const T*)h->yprev + (int64_t)k * h->n;
            A.out[k] = XK_of<T>(h, k);
        }
        e = traced(h, TVCUT_K_UPDATE, 1, [&] { return launch_prep8<T>(PREP8_FISTA, A, h->stream); });
    } else {
        FistaArgs<T> F;
        memset(&F, 0, sizeof(F));
        F.rows = rows_of(h);
        F.cols = cols_of(h);
        F.r = r;
        F.beta = beta;
        for (int k = 0; k < r; ++k) {
            F.y[k] = S_of<T>(h, k);
            F.p[k] = (const T*)h->yprev + (int64_t)k * h->n;
            F.v[k] = XK_of<T>(h, k);
        }
        F.w = (const T*)h->w;
        e = traced(h, TVCUT_K_UPDATE, 1, [&] { return launch_fista_prepare<T>(F, h->stream); });
    }
    if (e != cudaSuccess) return e;
    ScanArgs<T> S;
    memset(&S, 0, sizeof(S));
    S.naxes = r;
    S.force = scan_force(h->p.mapping);
    S.shadow = 1;
    for (int k = 0; k < r; ++k) S.ax[k] = block_axis<T>(h, k, XK_of<T>(h, k), (T*)h->yprev + (int64_t)k * h->n);
    e = traced(h, TVCUT_K_PROX, 1, [&] { return launch_scan<T>(S, h->stream); });
    if (e != cudaSuccess) return e;
    std::swap(h->state, h->yprev);
    h->fista_tprev = h->fista_t;
    h->fista_t = 0.5 * (1.0 + sqrt(1.0 + 4.0 * h->fista_t * h->fista_t));
    return check ? primal_of_duals<T>(h) : cudaSuccess;
}

template <typename T>
static cudaError_t run_iteration(tvcut_t h, int mode, int check)
{
    if (h->p.algo == TVCUT_FISTA) {
        if (mode == UPD_EVAL) return primal_of_duals<T>(h);
        return run_fista<T>(h, check);
    }
    if (h->p.algo == TVCUT_BCD) {
        if (mode == UPD_EVAL) return primal_of_duals<T>(h);     // primal of the current duals
        return run_bcd<T>(h, check);
    }
    if (!h->tlast) {
        if (mode == UPD_EVAL) return run_sweeps<T>(h, MODE_EVAL_FIRST, MODE_EVAL_MID, MODE_EVAL_LAST, 1);
        if (mode == UPD_AAR) return run_sweeps<T>(h, MODE_AAR_FIRST, MODE_AAR_MID, MODE_AAR_LAST, check);
        return run_sweeps<T>(h, MODE_AP_FIRST, MODE_AP_MID, MODE_AP_LAST, check);
    }
    const int r = h->ndim;
    ScanArgs<T> S;
    memset(&S, 0, sizeof(S));
    S.naxes = h->nblk;
    S.force = scan_force(h->p.mapping);
    for (int k = 0; k < h->nblk; ++k) S.ax[k] = block_axis<T>(h, k, S_of<T>(h, k), XK_of<T>(h, k));
    cudaError_t e = traced(h, TVCUT_K_PROX, 1, [&] { return launch_scan<T>(S, h->stream); });
    if (e != cudaSuccess) return e;
    if (h->conn8) {                // four blocks: rows, columns and the two path blocks
        Update8Args<T> U8;
        memset(&U8, 0, sizeof(U8));
        U8.rows = h->dims[0];
        U8.cols = h->dims[1];
        U8.check = check;
        for (int k = 0; k < 4; ++k) {
            U8.s[k] = S_of<T>(h, k);
            U8.x[k] = XK_of<T>(h, k);
        }
        U8.w = (const T*)h->w;
        U8.xout = X_of<T>(h);
        return traced(h, TVCUT_K_UPDATE, 1, [&] { return launch_update8<T>(mode, U8, h->stream); });
    }
    UpdateArgs<T> U;
    memset(&U, 0, sizeof(U));
    U.rows = rows_of(h);
    U.cols = cols_of(h);
    U.r = r;
    U.check = check;
    for (int k = 0; k < r; ++k) {
        U.s[k] = S_of<T>(h, k);
        U.x[k] = XK_of<T>(h, k);
    }
    U.w = (const T*)h->w;
    U.xout = X_of<T>(h);
    return traced(h, TVCUT_K_UPDATE, 1, [&] { return launch_update<T>(mode, U, h->stream); });
}

// Block k's chain geometry over FP64 arrays (v, a compact, x), as block_axis.
template <typename T>
static ScanAxis<double> axis64(tvcut_t h, int k, const double* v, const double* a, double* x)
{
    const ScanAxis<T> G = block_axis<T>(h, k, nullptr, nullptr);
    ScanAxis<double> X;
    memset(&X, 0, sizeof(X));
    X.nchains = G.nchains;
    X.inner = G.inner;
    X.m = G.m;
    X.transposed = G.transposed;
    X.v = v;
    X.a = a;
    X.ap = nullptr;
    X.x = x;
    return X;
}

// FP64 block duals of an FP32 handle's current state, for the rigorous bound.
// The FP32 state is an exact input, but duals computed from it in FP32 carry
// the chain prox's rounding at the state's magnitude (about eps |z| per
// element), which the bound sums over the grid: on 256^3 it leaves the bound
// ~10^3 below the energy.  So the duals are recomputed in FP64: for AAR and
// AP the FP64 chain projections of the state blocks, for BCD and FISTA one
// FP64 sweep of block coordinate descent (y_k <- Pi_{K_k}(w - sum_{j != k}
// y_j), blocks in turn) from their FP32 duals.  Fills h->y64 and h->a64.
template <typename T>
static cudaError_t fp64_duals(tvcut_t h, int* nlaunch)
{
    const size_t nb = (size_t)h->nblk * (size_t)h->n;
    cudaError_t e = cudaSuccess;
    if (!h->y64) {                                        // all four or none
        double *y = nullptr, *a = nullptr, *w = nullptr, *t = nullptr;
        e = cudaMalloc(&y, sizeof(double) * nb);
        if (e == cudaSuccess) e = cudaMalloc(&a, sizeof(double) * nb);
        if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(double) * (size_t)h->n);
        if (e == cudaSuccess) e = cudaMalloc(&t, sizeof(double) * (size_t)h->n);
        if (e != cudaSuccess) {
            cudaFree(y);
            cudaFree(a);
            cudaFree(w);
            cudaFree(t);
            return e;
        }
        h->y64 = y;
        h->a64 = a;
        h->w64 = w;
        h->t64 = t;
    }
    // the conversions' validation flags and max|v| land in the status record's
    // fields, which only input validation reads (after clearing them)
    int* flags = &h->dstatus->flags;
    unsigned* amax = &h->dstatus->absmax_bits;
    int nl = 0;
    for (int k = 0; k < h->nblk && e == cudaSuccess; ++k) {
        const ScanAxis<T> G = block_axis<T>(h, k, nullptr, nullptr);
        const int64_t cnt = G.nchains * (int64_t)(G.m - 1);
        if (cnt > 0) {
            e = launch_convert<double>(h->a[k], TVCUT_F32, h->a64 + (size_t)k * h->n, cnt, false, flags, amax, h->stream);
            ++nl;
        }
    }
    const bool shadow_of_state = h->p.algo == TVCUT_AAR || h->p.algo == TVCUT_AP;
    if (shadow_of_state) {
        for (int k = 0; k < h->nblk && e == cudaSuccess; ++k) {
            e = launch_convert<double>(S_of<T>(h, k), TVCUT_F32, h->t64, h->n, false, flags, amax, h->stream);
            ScanArgs<double> S;
            memset(&S, 0, sizeof(S));
            S.naxes = 1;
            S.shadow = 1;
            S.ax[0] = axis64<T>(h, k, h->t64, h->a64 + (size_t)k * h->n, h->y64 + (size_t)k * h->n);
            if (e == cudaSuccess) e = launch_scan<double>(S, h->stream);
            nl += 2;
        }
    } else {
        for (int k = 0; k < h->nblk && e == cudaSuccess; ++k) {
            e = launch_convert<double>(S_of<T>(h, k), TVCUT_F32, h->y64 + (size_t)k * h->n, h->n, false, flags, amax,
                                       h->stream);
            ++nl;
        }
        if (e == cudaSuccess) e = launch_convert<double>(h->w, TVCUT_F32, h->w64, h->n, false, flags, amax, h->stream);
        ++nl;
        for (int k = 0; k < h->nblk && e == cudaSuccess; ++k) {
            if (h->conn8) {
                Prep8Args<double> A;
                memset(&A, 0, sizeof(A));
                A.rows = h->dims[0];
                A.cols = h->dims[1];
                for (int j = 0; j < 4; ++j) A.y[j] = h->y64 + (size_t)j * h->n;
                A.w = h->w64;
                A.k = k;
                A.out[k] = h->t64;
                e = launch_prep8<double>(PREP8_BCD, A, h->stream);
            } else {
                UpdateArgs<double> U;
                memset(&U, 0, sizeof(U));
                U.rows = rows_of(h);
                U.cols = cols_of(h);
                U.r = h->ndim;
                for (int j = 0; j < h->ndim; ++j) U.s[j] = h->y64 + (size_t)j * h->n;
                U.w = h->w64;
                U.xout = h->t64;                          // v_k, in block k's layout
                e = launch_bcd_prepare<double>(U, k, h->stream);
            }
            ScanArgs<double> S;
            memset(&S, 0, sizeof(S));
            S.naxes = 1;
            S.shadow = 1;                                 // y_k = v_k - prox(v_k)
            S.ax[0] = axis64<T>(h, k, h->t64, h->a64 + (size_t)k * h->n, h->y64 + (size_t)k * h->n);
            if (e == cudaSuccess) e = launch_scan<double>(S, h->stream);
            nl += 2;
        }
    }
    *nlaunch = nl;
    return e;
}

// Rigorous discrete lower bound (Sec. 2.2): the block duals of the current
// state (the state itself for BCD and FISTA, its chain projections
// Pi_{K_k}(s_k) for AAR and AP) made exactly feasible chain by chain in FP64,
// summed, and bounded by sum_i min(y_i - w_i, 0); the FP64 rounding of that
// sum is covered by subtracting 2^-36 of the sum of the magnitudes.
template <typename T>
static tvcut_status rigorous_lb(tvcut_t h, double* lb_out)
{
    if (!h->ycert) {                                      // both or neither
        double *y = nullptr, *p = nullptr;
        cudaError_t e = cudaMalloc(&y, sizeof(double) * (size_t)h->n);
        if (e == cudaSuccess) e = cudaMalloc(&p, sizeof(double) * 2 * kCheckBlocks);
        if (e != cudaSuccess) {
            cudaFree(y);
            cudaFree(p);
            return cuda_fail(h, e, "certify: allocation");
        }
        h->ycert = y;
        h->lbpart = p;
    }
    const bool shadow = h->p.algo == TVCUT_AAR || h->p.algo == TVCUT_AP;
    if (sizeof(T) == 4) {                                 // FP32 iterates: the duals in FP64
        int nl = 0;
        CK(h, fp64_duals<T>(h, &nl), "certify: FP64 duals");
        h->launches[TVCUT_K_CHECK] += nl;
        CK(h, traced(h, TVCUT_K_CHECK, h->nblk + 1, [&] {
               cudaError_t e = cudaSuccess;
               for (int k = 0; k < h->nblk && e == cudaSuccess; ++k) {
                   CertifyArgs<double> A;
                   memset(&A, 0, sizeof(A));
                   A.X = axis64<T>(h, k, h->y64 + (size_t)k * h->n, h->a64 + (size_t)k * h->n, nullptr);
                   A.layout = block_layout(h, k);
                   A.first = k == 0 ? 1 : 0;
                   A.H = h->dims[0];
                   A.W = h->ndim == 2 ? h->dims[1] : 1;
                   A.Y = h->ycert;
                   e = launch_certify_block<double>(A, h->stream);
               }
               if (e == cudaSuccess) e = launch_certify_lb<T>(h->ycert, (const T*)h->w, h->n, h->lbpart, h->stream);
               return e;
           }), "certify");
    } else {
    const T* yk[4];
    for (int k = 0; k < h->nblk; ++k) yk[k] = shadow ? XK_of<T>(h, k) : S_of<T>(h, k);
    const int nk = (shadow ? 1 : 0) + h->nblk + 1;
    CK(h, traced(h, TVCUT_K_CHECK, nk, [&] {
           cudaError_t e = cudaSuccess;
           if (shadow) {
               ScanArgs<T> S;
               memset(&S, 0, sizeof(S));
               S.naxes = h->nblk;
               for (int k = 0; k < h->nblk; ++k) S.ax[k] = block_axis<T>(h, k, S_of<T>(h, k), XK_of<T>(h, k));
               S.shadow = 1;
               e = launch_scan<T>(S, h->stream);
           }
           for (int k = 0; k < h->nblk && e == cudaSuccess; ++k) {
               CertifyArgs<T> A;
               memset(&A, 0, sizeof(A));
               A.X = block_axis<T>(h, k, yk[k], nullptr);
               A.layout = block_layout(h, k);
               A.first = k == 0 ? 1 : 0;
               A.H = h->dims[0];
               A.W = h->ndim == 2 ? h->dims[1] : 1;
               A.Y = h->ycert;
               e = launch_certify_block<T>(A, h->stream);
           }
           if (e == cudaSuccess) e = launch_certify_lb<T>(h->ycert, (const T*)h->w, h->n, h->lbpart, h->stream);
           return e;
       }), "certify");
    }
    std::vector<double> part(2 * kCheckBlocks);
    CK(h, cudaMemcpyAsync(part.data(), h->lbpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, h->stream),
       "certify");
    CK(h, cudaStreamSynchronize(h->stream), "certify");
    CK(h, flush_trace(h), "certify");
    double lb = 0.0, mag = 0.0;
    for (int b = 0; b < kCheckBlocks; ++b) {
        lb += part[2 * b];
        mag += part[2 * b + 1];
    }
    *lb_out = lb - mag * ldexp(1.0, -36);
    return TVCUT_OK;
}

template <typename T>
static tvcut_status run_check(tvcut_t h)
{
    CheckArgs<T> C;
    memset(&C, 0, sizeof(C));
    C.ndim = h->ndim;
    C.n = h->n;
    for (int k = 0; k < h->ndim; ++k) {
        C.dims[k] = h->dims[k];
        ChainGeom g = chain_geom(h->ndim, h->dims, k);
        C.inner[k] = g.inner;
        C.a[k] = (const T*)h->a[k];
    }
    C.x = X_of<T>(h);
    C.w = (const T*)h->w;
    C.labels = h->labels;
    if (h->conn8) {
        C.adiag = (const T*)h->adiag;
        C.aanti = (const T*)h->aanti;
    }
    C.threshold = (T)h->p.threshold;
    C.last_transposed = h->tlast ? 1 : 0;
    C.partials = h->partials;
    // level-set ladder: threshold, then threshold +- S 10^-j, j = 2, 3, ...;
    // the kernel takes it in ascending order of the iterate-type values
    double lv[kMaxLevels];
    int L = 0;
    lv[L++] = h->p.threshold;
    if (h->p.level_sets > 0 && h->wmax > 0.0) {
        for (int j = 0; j < h->p.level_sets; ++j) {
            const double d = h->wmax * pow(10.0, -(double)(j + 2));
            lv[L++] = h->p.threshold + d;
            lv[L++] = h->p.threshold - d;
        }
    }
    int order[kMaxLevels], pos[kMaxLevels];
    for (int j = 0; j < L; ++j) order[j] = j;
    for (int i = 1; i < L; ++i)                          // stable insertion sort
        for (int j = i; j > 0 && (T)lv[order[j - 1]] > (T)lv[order[j]]; --j) std::swap(order[j - 1], order[j]);
    for (int q = 0; q < L; ++q) pos[order[q]] = q;
    C.nlevels = L;
    for (int q = 0; q < L; ++q) C.levels[q] = (T)lv[order[q]];
    C.level_partials = h->level_partials;
    bool exact_data = h->int_w;
    for (int k = 0; k < h->nblk; ++k) exact_data = exact_data && h->int_a[k];
    CK(h, traced(h, TVCUT_K_CHECK, 3, [&] { return launch_check<T>(C, exact_data, h->dstatus, h->stream); }),
       "check");
    CK(h, cudaMemcpyAsync(h->hstatus, h->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream), "check");
    CK(h, cudaStreamSynchronize(h->stream), "check");
    CK(h, flush_trace(h), "check");
    const CheckPartial& s = h->hstatus->sum;
    tvcut_stats& st = h->last;
    memset(&st, 0, sizeof(st));
    bool exact = h->int_w;
    for (int k = 0; k < h->nblk; ++k) exact = exact && h->int_a[k];
    st.iters = h->iters;
    // keep the lowest-energy level set; ties go to the earlier ladder entry
    // (the plain threshold first)
    const LevelPartial& lp = h->hstatus->levels;
    int best = 0;
    for (int j = 1; j < L; ++j) {
        const int qj = pos[j], qb = pos[best];
        const bool lower = exact ? lp.energy_i[qj] < lp.energy_i[qb] : lp.energy[qj] < lp.energy[qb];
        if (lower) best = j;
    }
    st.energy = lp.energy[pos[best]];
    st.energy_i64 = lp.energy_i[pos[best]];
    st.n_label1 = lp.n1[pos[best]];
    st.threshold = lv[best];
    if (best > 0)
        CK(h, traced(h, TVCUT_K_CHECK, 1, [&] { return launch_labels<T>(X_of<T>(h), (T)lv[best], h->labels, h->n, h->stream); }),
           "check");
    st.energy_exact = exact ? 1 : 0;
    st.discrete_lb = s.lb;
    st.tv_value = s.tv;
    st.tv_gap = s.tv - s.ytx;
    st.x_absmax = s.xabs;
    // certified only against the rigorous bound; it is evaluated at every
    // check (certify 1), or when the approximate bound is within 1 + 1e-7 |E|
    // of the energy and FP64 duals can bring it within 1 (their rounding
    // floor n * 2^-53 * max|x| summed over the grid stays below 1/2): by
    // default for FP64 iterates, with certify 2 also for FP32 ones, whose
    // duals are then recomputed in FP64 (about one FP64 iteration)
    st.certified = 0;
    st.certified_lb = -INFINITY;
    h->labels_valid = true;
    if (exact) {
        const double E = (double)st.energy_i64;
        const bool reachable = (double)h->n * ldexp(1.0, -53) * std::max(s.xabs, 1.0) < 0.5;   // FP64 duals
        const bool close = reachable && E - s.lb < 1.0 + 1e-7 * fabs(E);
        const bool when_close = h->p.certify == 2 || (h->p.certify == 0 && sizeof(T) == 8);
        if (h->p.certify == 1 || (when_close && close)) {
            double lb = 0.0;
            tvcut_status cs = rigorous_lb<T>(h, &lb);
            if (cs != TVCUT_OK) return cs;
            st.certified_lb = lb;
            st.certified = E - lb < 1.0 ? 1 : 0;
        }
    }
    return TVCUT_OK;
}

template <typename T>
static tvcut_status ensure_primal(tvcut_t h)
{
    if (h->x_valid) return TVCUT_OK;
    CK(h, run_iteration<T>(h, UPD_EVAL, 1), "evaluate primal");
    h->x_valid = true;
    h->labels_valid = false;
    return TVCUT_OK;
}

template <typename T>
static tvcut_status iterate_impl(tvcut_t h, int64_t max_iters, tvcut_stats* out)
{
    const int mode = h->p.algo == TVCUT_AAR ? UPD_AAR : UPD_AP;
    tvcut_status ret = TVCUT_NOT_CONVERGED;
    for (int64_t it = 0; it < max_iters; ++it) {
        const bool check = ((h->iters + 1) % h->p.check_every == 0) || it == max_iters - 1;
        CK(h, run_iteration<T>(h, mode, check ? 1 : 0), "iterate");
        h->iters += 1;
        h->x_valid = false;
        h->labels_valid = false;
        if (check) {
            h->x_valid = true;
            tvcut_status st = run_check<T>(h);
            if (st != TVCUT_OK) return st;
            const tvcut_stats& s = h->last;
            const bool approx = h->p.stop_on_approx && s.energy_exact && (double)s.energy_i64 - s.discrete_lb < 1.0;
            if (s.certified || approx || (h->p.gap_tol > 0.0 && s.tv_gap <= h->p.gap_tol)) {
                ret = TVCUT_OK;
                break;
            }
        }
    }
    if (out) *out = h->last;
    return ret;
}

// ---- C-ABI entry points ----------------------------------------------------

#define DISPATCH(h, FN, ...) ((h)->esize == 8 ? FN<double>(__VA_ARGS__) : FN<float>(__VA_ARGS__))

template <typename T>
static tvcut_status set_unary_impl(tvcut_t h, const void* w, int dtype, int space)
{
    tvcut_status st = ingest<T>(h, w, dtype, space, h->n, false, (T*)h->w, "tvcut_set_unary");
    if (st != TVCUT_OK) { h->have_w = false; return st; }
    h->have_w = true;
    h->int_w = dtype == TVCUT_I32;
    {
        float m;
        const unsigned bits = h->hstatus->absmax_bits;
        memcpy(&m, &bits, sizeof(m));
        h->wmax = (double)m;
    }
    return cold_start<T>(h);
}

extern "C" tvcut_status tvcut_set_unary(tvcut_t h, const void* w, int dtype, int space)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_set_unary: NULL handle");
    return DISPATCH(h, set_unary_impl, h, w, dtype, space);
}

template <typename T>
static tvcut_status set_weights_impl(tvcut_t h, int axis, const void* a, int dtype, int space)
{
    // 8-connected: axes 2, 3 are the diagonal inputs, kept in grid layout for
    // the check; the two path blocks' weights are built from both of them
    const bool diag = h->conn8 && axis >= 2;
    T* dst = diag ? (T*)(axis == 2 ? h->adiag : h->aanti) : (T*)h->a[axis];
    tvcut_status st = ingest<T>(h, a, dtype, space, h->a_len[axis], true, dst, "tvcut_set_weights");
    if (st != TVCUT_OK) { h->have_a[axis] = false; return st; }
    {
        float m;
        const unsigned bits = h->hstatus->absmax_bits;
        memcpy(&m, &bits, sizeof(m));
        h->amax[axis] = h->a_len[axis] > 0 ? (double)m : 0.0;
    }
    if (h->tlast && axis == h->ndim - 1)
        CK(h, relayout<T>(h, (T*)h->a[axis], rows_of(h), cols_of(h) - 1, true), "tvcut_set_weights");
    if (!diag && h->ap[axis])
        CK(h, launch_pad_weights<T>(block_axis<T>(h, axis, nullptr, nullptr), (T*)h->ap[axis], h->stream),
           "tvcut_set_weights");
    if (diag && (h->have_a[5 - axis] || h->a_len[axis] == 0)) {
        for (int b = 2; b < 4; ++b) {
            CK(h, launch_zz_weights<T>((const T*)h->adiag, (const T*)h->aanti, (T*)h->a[b], (int)h->dims[0],
                                       (int)h->dims[1], b, h->stream),
               "tvcut_set_weights");
            if (h->ap[b])
                CK(h, launch_pad_weights<T>(block_axis<T>(h, b, nullptr, nullptr), (T*)h->ap[b], h->stream),
                   "tvcut_set_weights");
        }
    }
    h->have_a[axis] = true;
    h->int_a[axis] = dtype == TVCUT_I32;
    if (h->have_w) return cold_start<T>(h);
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_set_weights(tvcut_t h, int axis, const void* a, int dtype, int space)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_set_weights: NULL handle");
    if (axis < 0 || axis >= h->nblk) return fail(h, TVCUT_ERR_INVALID, "tvcut_set_weights: axis out of range");
    return DISPATCH(h, set_weights_impl, h, axis, a, dtype, space);
}

extern "C" tvcut_status tvcut_reset(tvcut_t h)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_reset: NULL handle");
    if (!h->have_w) return fail(h, TVCUT_ERR_STATE, "tvcut_reset: unary not set");
    return DISPATCH(h, cold_start, h);
}

extern "C" tvcut_status tvcut_iterate(tvcut_t h, int64_t max_iters, tvcut_stats* out)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_iterate: NULL handle");
    if (max_iters < 1) return fail(h, TVCUT_ERR_INVALID, "tvcut_iterate: max_iters must be >= 1");
    if (!inputs_ready(h)) return fail(h, TVCUT_ERR_STATE, "tvcut_iterate: unary and all edge weights must be set first");
    return DISPATCH(h, iterate_impl, h, max_iters, out);
}

template <typename T>
static tvcut_status cut_impl(tvcut_t h, uint8_t* labels, int space, tvcut_stats* out)
{
    if (!h->labels_valid) {
        tvcut_status st = ensure_primal<T>(h);
        if (st != TVCUT_OK) return st;
        st = run_check<T>(h);
        if (st != TVCUT_OK) return st;
    }
    if (labels) {
        CK(h, cudaMemcpyAsync(labels, h->labels, (size_t)h->n,
                              space == TVCUT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream),
           "tvcut_cut");
        CK(h, cudaStreamSynchronize(h->stream), "tvcut_cut");
    }
    if (out) *out = h->last;
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_cut(tvcut_t h, uint8_t* labels, int space, tvcut_stats* out)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_cut: NULL handle");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE) return fail(h, TVCUT_ERR_INVALID, "tvcut_cut: bad space");
    if (!inputs_ready(h)) return fail(h, TVCUT_ERR_STATE, "tvcut_cut: unary and all edge weights must be set first");
    return DISPATCH(h, cut_impl, h, labels, space, out);
}

template <typename T>
static tvcut_status get_primal_impl(tvcut_t h, void* x, int dtype, int space)
{
    tvcut_status st = ensure_primal<T>(h);
    if (st != TVCUT_OK) return st;
    const size_t bytes = dtype_size(dtype) * (size_t)h->n;
    if (space == TVCUT_DEVICE) {
        CK(h, launch_convert_out<T>(X_of<T>(h), x, dtype, h->n, h->stream), "tvcut_get_primal");
        CK(h, cudaStreamSynchronize(h->stream), "tvcut_get_primal");
        return TVCUT_OK;
    }
    if ((size_t)dtype_size(dtype) == sizeof(T)) {
        CK(h, cudaMemcpyAsync(x, X_of<T>(h), bytes, cudaMemcpyDeviceToHost, h->stream), "tvcut_get_primal");
        CK(h, cudaStreamSynchronize(h->stream), "tvcut_get_primal");
        return TVCUT_OK;
    }
    // other element type: copy out in the iterate type, then widen/narrow
    std::vector<T> tmp((size_t)h->n);
    CK(h, cudaMemcpyAsync(tmp.data(), X_of<T>(h), sizeof(T) * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream),
       "tvcut_get_primal");
    CK(h, cudaStreamSynchronize(h->stream), "tvcut_get_primal");
    if (dtype == TVCUT_F64) for (int64_t i = 0; i < h->n; ++i) ((double*)x)[i] = (double)tmp[(size_t)i];
    else for (int64_t i = 0; i < h->n; ++i) ((float*)x)[i] = (float)tmp[(size_t)i];
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_get_primal(tvcut_t h, void* x, int dtype, int space)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_get_primal: NULL handle");
    if (!x) return fail(h, TVCUT_ERR_INVALID, "tvcut_get_primal: NULL output");
    if (dtype != TVCUT_F32 && dtype != TVCUT_F64) return fail(h, TVCUT_ERR_INVALID, "tvcut_get_primal: dtype must be F32 or F64");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE) return fail(h, TVCUT_ERR_INVALID, "tvcut_get_primal: bad space");
    if (!inputs_ready(h)) return fail(h, TVCUT_ERR_STATE, "tvcut_get_primal: unary and all edge weights must be set first");
    return DISPATCH(h, get_primal_impl, h, x, dtype, space);
}

template <typename T>
static tvcut_status get_state_impl(tvcut_t h, void* s, int space)
{
    const cudaMemcpyKind kind = space == TVCUT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int k = 0; k < h->nblk; ++k) {
        const T* src = S_of<T>(h, k);
        if (block_layout(h, k) != 0) {         // back to grid layout through the xk area
            T* tmp = XK_of<T>(h, 0);
            CK(h, to_natural<T>(h, k, src, tmp), "tvcut_get_state");
            src = tmp;
        }
        CK(h, cudaMemcpyAsync((T*)s + (int64_t)k * h->n, src, sizeof(T) * (size_t)h->n, kind, h->stream),
           "tvcut_get_state");
    }
    CK(h, cudaStreamSynchronize(h->stream), "tvcut_get_state");
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_get_state(tvcut_t h, void* s, int space)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_get_state: NULL handle");
    if (!s) return fail(h, TVCUT_ERR_INVALID, "tvcut_get_state: NULL output");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE) return fail(h, TVCUT_ERR_INVALID, "tvcut_get_state: bad space");
    return DISPATCH(h, get_state_impl, h, s, space);
}

// Shadow duals y_k = Pi_{K_k}(s_k) = s_k - prox(s_k) of the current state,
// every block through the scan launch, out in grid layout.
template <typename T>
static tvcut_status get_dual_impl(tvcut_t h, void* out, int space)
{
    ScanArgs<T> S;
    memset(&S, 0, sizeof(S));
    S.naxes = h->nblk;
    for (int k = 0; k < h->nblk; ++k) S.ax[k] = block_axis<T>(h, k, S_of<T>(h, k), XK_of<T>(h, k));
    S.shadow = 1;                                         // y_k = s_k - prox(s_k)
    CK(h, traced(h, TVCUT_K_PROX, 1, [&] { return launch_scan<T>(S, h->stream); }), "tvcut_get_dual");
    const cudaMemcpyKind kind = space == TVCUT_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int k = 0; k < h->nblk; ++k) {
        const T* src = XK_of<T>(h, k);
        if (block_layout(h, k) != 0) {         // back to grid layout through the P|x scratch (2n values)
            T* tmp = P_of<T>(h);
            CK(h, to_natural<T>(h, k, src, tmp), "tvcut_get_dual");
            src = tmp;
            h->x_valid = h->labels_valid = false;    // the scratch held the primal
        }
        CK(h, cudaMemcpyAsync((T*)out + (int64_t)k * h->n, src, sizeof(T) * (size_t)h->n, kind, h->stream),
           "tvcut_get_dual");
    }
    CK(h, cudaStreamSynchronize(h->stream), "tvcut_get_dual");
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_get_dual(tvcut_t h, void* y, int space)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_get_dual: NULL handle");
    if (!y) return fail(h, TVCUT_ERR_INVALID, "tvcut_get_dual: NULL output");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE) return fail(h, TVCUT_ERR_INVALID, "tvcut_get_dual: bad space");
    if (!inputs_ready(h)) return fail(h, TVCUT_ERR_STATE, "tvcut_get_dual: unary and all edge weights must be set first");
    if (h->p.algo == TVCUT_BCD || h->p.algo == TVCUT_FISTA)
        return DISPATCH(h, get_state_impl, h, y, space);     // the BCD and FISTA states are y itself
    return DISPATCH(h, get_dual_impl, h, y, space);
}

namespace tvcut {

tvcut_status problem_view(tvcut_t h, ProblemView* v, std::string* why)
{
    if (h->ndim != 2 || h->conn8) {
        *why = "the learned warm start takes 2D 4-connected grids";
        return TVCUT_ERR_INVALID;
    }
    if (!inputs_ready(h)) {
        *why = "unary and all edge weights must be set first";
        return TVCUT_ERR_STATE;
    }
    v->esize = h->esize;
    v->H = h->dims[0];
    v->W = h->dims[1];
    v->w = h->w;
    v->a0 = h->a[0];
    v->a1 = h->a[1];
    v->a1_transposed = h->tlast ? 1 : 0;
    v->s0 = (char*)h->state;
    v->s1 = (char*)h->state + (size_t)h->esize * (size_t)h->n;
    v->s1_transposed = block_layout(h, 1) == 1 ? 1 : 0;
    v->scale = std::max(std::max(h->wmax, std::max(h->amax[0], h->amax[1])), 1e-12);
    v->stream = h->stream;
    return TVCUT_OK;
}

tvcut_status state_written(tvcut_t h)
{
    CK(h, restart_momentum(h), "tvcut_unet_predict_state");
    h->x_valid = h->labels_valid = false;
    return TVCUT_OK;
}

}  // namespace tvcut

template <typename T>
static tvcut_status set_state_impl(tvcut_t h, const void* s, int space)
{
    CK(h, cudaMemcpyAsync(h->state, s, sizeof(T) * (size_t)(h->nblk * h->n),
                          space == TVCUT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream),
       "tvcut_set_state");
    for (int k = 0; k < h->nblk; ++k) CK(h, to_internal<T>(h, k, S_of<T>(h, k)), "tvcut_set_state");
    CK(h, restart_momentum(h), "tvcut_set_state");
    CK(h, cudaStreamSynchronize(h->stream), "tvcut_set_state");
    h->x_valid = h->labels_valid = false;
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_set_state(tvcut_t h, const void* s, int space)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_set_state: NULL handle");
    if (!s) return fail(h, TVCUT_ERR_INVALID, "tvcut_set_state: NULL input");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE) return fail(h, TVCUT_ERR_INVALID, "tvcut_set_state: bad space");
    return DISPATCH(h, set_state_impl, h, s, space);
}

template <typename T>
static tvcut_status warmstart_impl(tvcut_t h, const float* xhat, float tau, int space)
{
    const float* d = xhat;
    if (space == TVCUT_HOST) {
        CK(h, cudaMemcpyAsync(h->scratch, xhat, sizeof(float) * (size_t)h->n, cudaMemcpyHostToDevice, h->stream),
           "tvcut_warmstart_primal");
        d = (const float*)h->scratch;
    }
    // the kernel reads xhat[i] before writing state; state and scratch are disjoint
    CK(h, traced(h, TVCUT_K_OTHER, 1, [&] { return launch_warmstart<T>((const T*)h->w, d, tau, (T*)h->state, h->nblk, h->n, h->stream); }),
       "tvcut_warmstart_primal");
    for (int k = 0; k < h->nblk; ++k) CK(h, to_internal<T>(h, k, S_of<T>(h, k)), "tvcut_warmstart_primal");
    CK(h, restart_momentum(h), "tvcut_warmstart_primal");
    CK(h, cudaStreamSynchronize(h->stream), "tvcut_warmstart_primal");
    h->x_valid = h->labels_valid = false;
    h->iters = 0;
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_warmstart_primal(tvcut_t h, const float* xhat, float tau, int space)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_warmstart_primal: NULL handle");
    if (!xhat) return fail(h, TVCUT_ERR_INVALID, "tvcut_warmstart_primal: NULL xhat");
    if (space != TVCUT_HOST && space != TVCUT_DEVICE) return fail(h, TVCUT_ERR_INVALID, "tvcut_warmstart_primal: bad space");
    if (!(tau == tau)) return fail(h, TVCUT_ERR_INVALID, "tvcut_warmstart_primal: tau is NaN");
    if (!h->have_w) return fail(h, TVCUT_ERR_STATE, "tvcut_warmstart_primal: unary not set");
    return DISPATCH(h, warmstart_impl, h, xhat, tau, space);
}

template <typename T>
static tvcut_status project_impl(int ndim, const int64_t* dims, int axis, const void* v, const void* a,
                                 void* out, int what, cudaStream_t s)
{
    SweepArgs<T> A;
    memset(&A, 0, sizeof(A));
    A.g = chain_geom(ndim, dims, axis);
    A.v = (const T*)v;
    A.a = (const T*)a;
    A.out = (T*)out;
    A.mapping = -1;
    cudaError_t e = launch_sweep<T>(what == 1 ? MODE_PROX : MODE_PROJ, A, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "tvcut_project_chains");
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_project_chains(int ndim, const int64_t* dims, int axis, const void* v,
                                             const void* a, void* out, int dtype, int what,
                                             void* cuda_stream)
{
    if (ndim < 1 || ndim > 3 || !dims) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_project_chains: ndim must be 1..3");
    if (axis < 0 || axis >= ndim) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_project_chains: axis out of range");
    if (what != 0 && what != 1) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_project_chains: what must be 0 or 1");
    int64_t n = 1;
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 1 || dims[k] > (int64_t)1 << 30) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_project_chains: bad dims");
        n *= dims[k];
    }
    if (!v || !out || (!a && dims[axis] > 1)) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_project_chains: NULL pointer");
    if (dtype == TVCUT_F32) return project_impl<float>(ndim, dims, axis, v, a, out, what, (cudaStream_t)cuda_stream);
    if (dtype == TVCUT_F64) return project_impl<double>(ndim, dims, axis, v, a, out, what, (cudaStream_t)cuda_stream);
    return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_project_chains: dtype must be TVCUT_F32 or TVCUT_F64");
}

extern "C" tvcut_status tvcut_profile(tvcut_t h, int enable)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_profile: NULL handle");
    CK(h, cudaStreamSynchronize(h->stream), "tvcut_profile");
    CK(h, flush_trace(h), "tvcut_profile");
    h->prof = enable != 0;
    for (int k = 0; k < TVCUT_NKINDS; ++k) {
        h->prof_ms[k] = 0.0;
        h->launches[k] = 0;
    }
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_profile_read(tvcut_t h, double* ms, int64_t* launches)
{
    if (!h) return fail(nullptr, TVCUT_ERR_INVALID, "tvcut_profile_read: NULL handle");
    CK(h, cudaStreamSynchronize(h->stream), "tvcut_profile_read");
    CK(h, flush_trace(h), "tvcut_profile_read");
    for (int k = 0; k < TVCUT_NKINDS; ++k) {
        if (ms) ms[k] = h->prof_ms[k];
        if (launches) launches[k] = h->launches[k];
    }
    return TVCUT_OK;
}
