// Chain prox by a sequence of chain min-cuts solved by message passing
// (Sec. 3.2, "Message passing": message passing solves the min-cut problem on
// a chain, and the exact TV solution follows from a sequence of min-cuts).
//
// One CTA owns one chain (m <= kMpMaxLen), held in shared memory.  The chain
// is cut into intervals; at first the whole chain is one.  A round treats
// every open interval at once:
//
//   1. alpha = mean of the modified unary v' over the interval (the solution
//      on an interval has the mean of its v': the edge terms inside cancel);
//   2. the cut energy sum a_k |l_{k+1} - l_k| - sum (v'_i - alpha) l_i is
//      solved by min-sum message passing in difference form: the forward
//      message delta_i = F_i(1) - F_i(0) obeys
//          delta_i = clamp(delta_{i-1}, -a_{i-1}, a_{i-1}) + (alpha - v'_i),
//      the backward one beta_i = B_i(1) - B_i(0) obeys
//          beta_i = clamp(beta_{i+1} + (alpha - v'_{i+1}), -a_i, a_i),
//      and the min-marginal difference M_i(1) - M_i(0) = delta_i + beta_i.
//      Both recurrences compose maps x -> min(max(x, L), H) + C, which stay in
//      that family, so they run as segmented block scans;
//   3. M_i(1) - M_i(0) < 0 means x*_i > alpha, > 0 means x*_i < alpha, and 0
//      means x*_i = alpha (final); numerically a band of width tol around 0
//      is the tie class.  Where the class changes inside an interval the
//      edge's sign is known, and its term moves into v' of both ends (the
//      larger end v' -= a, the smaller v' += a); each run of one class is a
//      new interval.  An interval that neither splits nor ties (possible
//      only through rounding on an interval of equal values) is final at its
//      mean.
//
// The message differences stay bounded by a + |v' - alpha|, so the rounding
// does not grow with the chain length, unlike accumulated min-sum costs.
// When no interval is left the result is checked against the optimality
// conditions of the chain prox in FP64 (running sums u_j of v - x within
// [-a_j, a_j], at -a_j / +a_j where x rises / falls, 0 at the chain end);
// a chain that fails them is recomputed by the taut string.  The number of
// such chains is counted (tvcut_mp_fallbacks).
#include "tvcut_internal.cuh"
#include "taut_string.cuh"

namespace tvcut {

namespace {

constexpr int kMpThreads = 256;
constexpr int kMpWarps = kMpThreads / 32;

__device__ unsigned long long g_mp_fallbacks = 0;

template <typename T>
__device__ __forceinline__ T clamp_to(T x, T lo, T hi) { return x < lo ? lo : (x > hi ? hi : x); }

// x -> min(max(x, L), H) + C; a constant c is (c, c, 0).
template <typename T>
struct ClampMap {
    T L, H, C;
};

// g applied after f.  clamp(clamp(x, L1, H1) + C1, L2, H2) + C2
//   = clamp(x, clamp(L1, L2 - C1, H2 - C1), clamp(H1, L2 - C1, H2 - C1)) + C1 + C2
template <typename T>
struct ComposeOp {
    __device__ __forceinline__ ClampMap<T> operator()(const ClampMap<T>& f, const ClampMap<T>& g) const
    {
        const T lo = g.L - f.C, hi = g.H - f.C;
        return {clamp_to(f.L, lo, hi), clamp_to(f.H, lo, hi), f.C + g.C};
    }
};

template <typename T>
struct SumCount {
    T s;
    int n;
};

template <typename T>
struct SumOp {
    __device__ __forceinline__ SumCount<T> operator()(const SumCount<T>& a, const SumCount<T>& b) const
    {
        return {a.s + b.s, a.n + b.n};
    }
};

struct KeepFirst {                               // the segment's first element's value
    __device__ __forceinline__ int operator()(int a, int) const { return a; }
};

struct PlusD {
    __device__ __forceinline__ double operator()(double a, double b) const { return a + b; }
};

template <typename T>
__device__ __forceinline__ T shfl_up_any(T v, int d)
{
    return __shfl_up_sync(0xffffffffu, v, d);
}
template <typename T>
__device__ __forceinline__ ClampMap<T> shfl_up_any(const ClampMap<T>& v, int d)
{
    return {__shfl_up_sync(0xffffffffu, v.L, d), __shfl_up_sync(0xffffffffu, v.H, d),
            __shfl_up_sync(0xffffffffu, v.C, d)};
}
template <typename T>
__device__ __forceinline__ SumCount<T> shfl_up_any(const SumCount<T>& v, int d)
{
    return {__shfl_up_sync(0xffffffffu, v.s, d), __shfl_up_sync(0xffffffffu, v.n, d)};
}

// A partial fold of a segmented scan: `e` no element, `f` a segment starts
// inside (the fold then holds only the part after the last start).
template <typename V>
struct Part {
    V v;
    int e, f;
};

template <typename V, class Op>
__device__ __forceinline__ Part<V> join(const Part<V>& a, const Part<V>& b, Op op)
{
    if (a.e) return b;
    if (b.e) return a;
    if (b.f) return b;
    return {op(a.v, b.v), 0, a.f};
}

template <typename V>
__device__ __forceinline__ Part<V> shfl_part(const Part<V>& p, int d)
{
    return {shfl_up_any(p.v, d), __shfl_up_sync(0xffffffffu, p.e, d), __shfl_up_sync(0xffffffffu, p.f, d)};
}

// Segmented inclusive scan over the chain's m elements in shared memory, in
// index order (REV = false) or in reverse index order (REV = true): on return
// val[i] is the op-fold from the nearest segment start at or before i (in
// scan order) through i.  head[i] != 0 marks segment starts in scan order;
// the first element in scan order must be one.  Thread t owns the E
// consecutive elements [t E, t E + E).  `scratch` holds kMpThreads + kMpWarps
// Parts of V.
template <typename V, class Op, bool REV>
__device__ void block_seg_scan(V* val, const unsigned char* head, int m, int E, Op op, void* scratch)
{
    Part<V>* slot = (Part<V>*)scratch;                     // one per rank in scan order
    Part<V>* wpart = slot + kMpThreads;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int lo = t * E, hi = min(m, lo + E);
    Part<V> mine;                                          // this thread's fold, in scan order
    mine.e = 1;
    mine.f = 0;
    for (int q = 0; q < hi - lo; ++q) {
        const int i = REV ? hi - 1 - q : lo + q;
        const Part<V> p = {val[i], 0, head[i] ? 1 : 0};
        mine = join(mine, p, op);
    }
    const int rank = REV ? kMpThreads - 1 - t : t;         // position of this thread's fold in scan order
    slot[rank] = mine;
    __syncthreads();
    Part<V> cur = slot[t];                                 // thread t scans rank slot t
    for (int d = 1; d < 32; d <<= 1) {
        const Part<V> o = shfl_part(cur, d);
        if (lane >= d) cur = join(o, cur, op);
    }
    if (lane == 31) wpart[warp] = cur;
    __syncthreads();
    if (t == 0)
        for (int w = 1; w < kMpWarps; ++w) wpart[w] = join(wpart[w - 1], wpart[w], op);
    __syncthreads();
    if (warp > 0) cur = join(wpart[warp - 1], cur, op);    // inclusive fold of ranks 0 .. t
    slot[t] = cur;
    __syncthreads();
    Part<V> run;                                           // exclusive fold of this thread's rank
    run.e = 1;
    run.f = 0;
    if (rank > 0) run = slot[rank - 1];
    for (int q = 0; q < hi - lo; ++q) {
        const int i = REV ? hi - 1 - q : lo + q;
        const Part<V> p = {val[i], 0, head[i] ? 1 : 0};
        run = join(run, p, op);
        val[i] = run.v;
    }
    __syncthreads();
}

// Shared-memory layout of one chain of up to M elements.  The modified unary
// is kept as the input v plus an offset (the edge terms moved in so far,
// sums of +-a), so the output is formed from the input itself.
template <typename T>
struct MpLayout {
    unsigned char* fw;      // scan buffer: forward maps, interval sums, verification sums
    unsigned char* bw;      // scan buffer: backward maps, head indices
    T* v;                   // the chain's input
    T* off;                 // v' - v
    T* av;                  // a_i (edge i, i+1), 0 at the chain end
    T* xo;                  // final values
    T* sH;                  // per interval (indexed by its head): mean of v'
    int* hid;               // head index of each element's interval
    int* chg;               // per interval: splits + ties found in the current pass
    unsigned char *act, *head, *hd, *tl;
    signed char* cls;
    void* scratch;
};

template <typename T>
constexpr size_t mp_slot()                  // bytes per element of a scan buffer (maps, sums, FP64 check)
{
    return sizeof(ClampMap<T>) > sizeof(double) ? sizeof(ClampMap<T>) : sizeof(double);
}

template <typename T>
constexpr size_t mp_part()                  // bytes of one scan Part (the largest value type)
{
    return sizeof(Part<ClampMap<T>>) > sizeof(Part<double>) ? sizeof(Part<ClampMap<T>>) : sizeof(Part<double>);
}

// Byte offsets of the layout's sections, each rounded up to 16 bytes (the
// scans keep doubles and 16-byte structs in them).  off[14] is the total.
__host__ __device__ constexpr size_t mp_align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename T>
__host__ __device__ inline void mp_offsets(int M, size_t* off)
{
    const size_t sz[14] = {(size_t)M * mp_slot<T>(), (size_t)M * mp_slot<T>(), (size_t)M * sizeof(T),
                           (size_t)(kMpThreads + kMpWarps) * mp_part<T>(), (size_t)M * sizeof(T),
                           (size_t)M * sizeof(T), (size_t)M * sizeof(T), (size_t)M * sizeof(T),
                           (size_t)M * sizeof(int), (size_t)M * sizeof(int), (size_t)M, (size_t)M, (size_t)M,
                           (size_t)M};
    size_t o = 0;
    for (int j = 0; j < 14; ++j) {
        off[j] = o;
        o = mp_align16(o + sz[j]);
    }
    off[14] = o + (size_t)M;                        // the class bytes last
}

template <typename T>
inline size_t mp_smem_bytes(int M)
{
    size_t off[15];
    mp_offsets<T>(M, off);
    return off[14];
}

template <typename T>
__device__ MpLayout<T> mp_layout(unsigned char* base, int M)
{
    size_t off[15];
    mp_offsets<T>(M, off);
    MpLayout<T> L;
    L.fw = base + off[0];
    L.bw = base + off[1];
    L.sH = (T*)(base + off[2]);
    L.scratch = base + off[3];
    L.v = (T*)(base + off[4]);
    L.off = (T*)(base + off[5]);
    L.av = (T*)(base + off[6]);
    L.xo = (T*)(base + off[7]);
    L.hid = (int*)(base + off[8]);
    L.chg = (int*)(base + off[9]);
    L.act = base + off[10];
    L.head = base + off[11];
    L.hd = base + off[12];
    L.tl = base + off[13];
    L.cls = (signed char*)(base + off[14] - (size_t)M);
    return L;
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T* red)
{
    for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T r = red[0];
    for (int w = 1; w < kMpWarps; ++w) r = max(r, red[w]);
    __syncthreads();
    return r;
}

// One CTA per chain; M = the longest chain of the launch (shared memory).
template <typename T, bool SHADOW>
__global__ void __launch_bounds__(kMpThreads) mp_prox_kernel(ScanArgs<T> A, int M)
{
    extern __shared__ __align__(16) unsigned char mp_smem[];
    int k = 0;
    while (k + 1 < A.naxes && blockIdx.x >= A.ax[k + 1].block_begin) ++k;
    const ScanAxis<T>& X = A.ax[k];
    const int64_t c = (int64_t)blockIdx.x - X.block_begin;
    if (c >= X.nchains) return;
    int64_t base, abase, stride;
    if (X.transposed) {
        base = c;
        abase = c;
        stride = X.nchains;
    } else {
        const int64_t o = c / X.inner;
        const int64_t q = c - o * X.inner;
        base = o * (int64_t)X.m * X.inner + q;
        abase = o * (int64_t)(X.m - 1) * X.inner + q;
        stride = X.inner;
    }
    const int m = X.m, t = threadIdx.x;
    const int E = (m + kMpThreads - 1) / kMpThreads;
    MpLayout<T> L = mp_layout<T>(mp_smem, M);
    __shared__ T red[kMpWarps];
    ClampMap<T>* fw = (ClampMap<T>*)L.fw;
    ClampMap<T>* bw = (ClampMap<T>*)L.bw;
    T vmax = T(0), amax = T(0);
    for (int i = t; i < m; i += kMpThreads) {
        const T vi = X.v[base + (int64_t)i * stride];
        const T ai = i < m - 1 ? X.a[abase + (int64_t)i * stride] : T(0);
        L.v[i] = vi;
        L.off[i] = T(0);
        L.av[i] = ai;
        L.act[i] = 1;
        L.head[i] = i == 0;
        vmax = max(vmax, fabs(vi));
        amax = max(amax, ai);
    }
    vmax = block_max<T>(vmax, red);
    amax = block_max<T>(amax, red);
    const T eps = sizeof(T) == 4 ? T(5.9604644775390625e-08) : T(1.1102230246251565e-16);
    const T tol = T(16) * eps * (vmax + T(2) * amax);      // width of the tie band
    bool failed = false;
    for (int round = 0;; ++round) {
        // intervals: runs of active elements between heads
        bool any = false;
        for (int i = t; i < m; i += kMpThreads) {
            const bool a = L.act[i];
            any = any || a;
            L.hd[i] = !a || L.head[i] || i == 0 || !L.act[i - 1];
            L.tl[i] = !a || i == m - 1 || !L.act[i + 1] || L.head[i + 1];
            ((int*)L.bw)[i] = i;
            const SumCount<T> sc = {a ? L.v[i] + L.off[i] : T(0), a ? 1 : 0};
            ((SumCount<T>*)L.fw)[i] = sc;
        }
        if (!__syncthreads_or(any)) break;
        if (round > m + 2) {                                // cannot happen in exact arithmetic
            failed = true;
            break;
        }
        block_seg_scan<int, KeepFirst, false>((int*)L.bw, L.hd, m, E, KeepFirst(), L.scratch);
        block_seg_scan<SumCount<T>, SumOp<T>, false>((SumCount<T>*)L.fw, L.hd, m, E, SumOp<T>(), L.scratch);
        for (int i = t; i < m; i += kMpThreads) {
            const int h = ((int*)L.bw)[i];
            L.hid[i] = h;
            if (L.act[i] && L.tl[i]) {
                const SumCount<T> sc = ((SumCount<T>*)L.fw)[i];
                L.sH[h] = sc.s / (T)sc.n;                   // the interval's mean
            }
        }
        __syncthreads();
        // message maps: forward delta_i, backward beta_i (constants at the interval ends)
        for (int i = t; i < m; i += kMpThreads) {
            ClampMap<T> f = {T(0), T(0), T(0)}, g = {T(0), T(0), T(0)};
            if (L.act[i]) {
                const T alpha = L.sH[L.hid[i]];
                const T ci = alpha - (L.v[i] + L.off[i]);
                if (L.hd[i]) f = {ci, ci, T(0)};
                else f = {-L.av[i - 1], L.av[i - 1], ci};
                if (!L.tl[i]) {
                    const T cn = alpha - (L.v[i + 1] + L.off[i + 1]);
                    g = {-L.av[i] - cn, L.av[i] - cn, cn};
                }
            }
            fw[i] = f;
            bw[i] = g;
        }
        __syncthreads();
        block_seg_scan<ClampMap<T>, ComposeOp<T>, false>(fw, L.hd, m, E, ComposeOp<T>(), L.scratch);
        block_seg_scan<ClampMap<T>, ComposeOp<T>, true>(bw, L.tl, m, E, ComposeOp<T>(), L.scratch);
        for (int i = t; i < m; i += kMpThreads) {
            signed char cl = 0;
            if (L.act[i]) {
                const T mm = (fw[i].L + fw[i].C) + (bw[i].L + bw[i].C);
                cl = mm < -tol ? 1 : (mm > tol ? -1 : 0);
                if (L.hd[i]) L.chg[i] = 0;
            }
            L.cls[i] = cl;
        }
        __syncthreads();
        for (int i = t; i < m; i += kMpThreads)
            if (L.act[i] && (L.cls[i] == 0 || (!L.hd[i] && L.cls[i] != L.cls[i - 1]))) atomicAdd(&L.chg[L.hid[i]], 1);
        __syncthreads();
        for (int i = t; i < m; i += kMpThreads) {
            if (!L.act[i]) continue;
            const int h = L.hid[i];
            const signed char ci = L.cls[i];
            if (L.chg[h] == 0 || ci == 0) {                 // tie, or an interval of equal values
                L.xo[i] = (T)L.sH[h];
                L.act[i] = 0;
                continue;
            }
            T d = T(0);
            bool newhead = L.hd[i];
            if (!L.hd[i] && L.cls[i - 1] != ci) {            // edge (i-1, i) inside the interval
                d += L.cls[i - 1] > ci ? L.av[i - 1] : -L.av[i - 1];
                newhead = true;
            }
            if (!L.tl[i] && L.cls[i + 1] != ci) d += ci > L.cls[i + 1] ? -L.av[i] : L.av[i];   // edge (i, i+1)
            L.off[i] += d;
            L.head[i] = newhead;
        }
        __syncthreads();
    }
    // optimality of the chain prox, in FP64: u_j = sum_{i <= j} (v_i - x_i) lies in
    // [-a_j, a_j], at -a_j where x rises, at +a_j where it falls, and is 0 at the end.
    // Tolerance: the rounding of x to the iterate type, summed along the chain, plus
    // the tie band's width per element.
    double* u = (double*)L.fw;
    for (int i = t; i < m; i += kMpThreads) {
        u[i] = (double)L.v[i] - (double)L.xo[i];
        L.hd[i] = i == 0;
    }
    __syncthreads();
    block_seg_scan<double, PlusD, false>(u, L.hd, m, E, PlusD(), L.scratch);
    const double tolu = (double)m * (double)eps * ((double)vmax + 32.0 * (double)amax);
    const double tolx = 2.0 * (double)eps * ((double)vmax + 2.0 * (double)amax);
    bool bad = false;
    for (int i = t; i < m; i += kMpThreads) {
        const double ui = u[i];
        if (i == m - 1) {
            bad = bad || fabs(ui) > tolu;
        } else {
            const double ai = (double)L.av[i];
            const double dx = (double)L.xo[i + 1] - (double)L.xo[i];
            bad = bad || fabs(ui) > ai + tolu;
            if (dx > tolx) bad = bad || ui > -ai + tolu;
            if (dx < -tolx) bad = bad || ui < ai - tolu;
        }
    }
    failed = __syncthreads_or(bad || failed);
    if (failed) {                                           // recompute by the taut string
        if (t == 0) {
            atomicAdd(&g_mp_fallbacks, 1ull);
            scan_chain<T, SHADOW>(m, X.v + base, X.a + abase, X.x + base, stride);
        }
        return;
    }
    for (int i = t; i < m; i += kMpThreads) {
        const int64_t e = base + (int64_t)i * stride;
        X.x[e] = SHADOW ? L.v[i] - L.xo[i] : L.xo[i];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_mp_prox(const ScanArgs<T>& A, cudaStream_t s)
{
    if (A.naxes == 0) return cudaSuccess;
    ScanArgs<T> B = A;
    int M = 1;
    int64_t blocks = 0;
    for (int k = 0; k < B.naxes; ++k) {
        B.ax[k].block_begin = blocks;
        blocks += B.ax[k].nchains;
        M = max(M, B.ax[k].m);
    }
    if (blocks == 0) return cudaSuccess;
    const size_t bytes = mp_smem_bytes<T>(M);
    cudaError_t e;
    if (A.shadow) {
        e = cudaFuncSetAttribute(mp_prox_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e == cudaSuccess) mp_prox_kernel<T, true><<<(unsigned)blocks, kMpThreads, bytes, s>>>(B, M);
    } else {
        e = cudaFuncSetAttribute(mp_prox_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e == cudaSuccess) mp_prox_kernel<T, false><<<(unsigned)blocks, kMpThreads, bytes, s>>>(B, M);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template cudaError_t launch_mp_prox<float>(const ScanArgs<float>&, cudaStream_t);
template cudaError_t launch_mp_prox<double>(const ScanArgs<double>&, cudaStream_t);

}  // namespace tvcut

extern "C" tvcut_status tvcut_mp_fallbacks(unsigned long long* count, int reset)
{
    if (!count) return TVCUT_ERR_INVALID;
    if (cudaMemcpyFromSymbol(count, tvcut::g_mp_fallbacks, sizeof(*count)) != cudaSuccess) return TVCUT_ERR_CUDA;
    if (reset) {
        const unsigned long long zero = 0;
        if (cudaMemcpyToSymbol(tvcut::g_mp_fallbacks, &zero, sizeof(zero)) != cudaSuccess) return TVCUT_ERR_CUDA;
    }
    return TVCUT_OK;
}

