// The lane-group chain prox (Sec. 3.2) for launches with few, long chains:
// G lanes (4 .. 32) share a chain in speculative pieces, with the taut string
// in local form (wscan_kernel) or in funnel form (fscan_kernel, mapping 11),
// and the launch plans that size them.  scan.cu dispatches here.
#include <mutex>

#include "tvcut_internal.cuh"
#include "taut_string.cuh"
#include "funnel.cuh"

namespace tvcut {

__device__ __forceinline__ void scan_cp_async(void* smem, const void* gmem, int bytes)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
template <typename T>
__device__ __forceinline__ void scan_cp_elem(T* smem, const T* gmem) { scan_cp_async(smem, gmem, (int)sizeof(T)); }
__device__ __forceinline__ void scan_cp_wait()
{
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---- lane-group (speculative pieces) scan -------------------------------------
//
// For few, long chains (a 2D grid has only H + W of them) one thread per chain
// leaves the GPU idle, so G lanes (4 .. 32, the kernel's template parameter)
// share one chain: lane L scans piece L of G from a guessed state (a segment
// starts at the piece start with multiplier 0; exact for lane 0) and records
// every bend it finds (position e and
// direction).  After a bend at e the scan state is fixed (the next segment
// starts at e+1 with multiplier +-a_e), so a lane's trajectory is the true one
// from the first bend it shares with the true scan.  Lane L then continues
// from its own piece end into piece L+1 until it produces a bend that lane
// L+1 (or any later lane) recorded; that lane's results after the bend are
// then exact, and lane L rewrites every position before it.  Lane 0 is
// exact, so following merges from lane 0 reaches the chain end through
// verified lanes only; lanes not on that path are overwritten.  A launch
// lasts as long as its slowest chain's critical path (piece, continuation,
// rewrite); in the form with lists (LIST), each lane keeps its
// continuation's segments so that the rewrite only stores them (the same
// values: the same scan from the same state).  The launch plan below picks
// the lane count and the form.

// Advance one lane's scan through positions st.i .. stop-1 (data in shared
// memory, skewed).  on_bend(s, e, d, t) is called for every finished segment
// [s, e] with value t (d = 1: the string bends up at e, 2: down, 0: chain end)
// and returns true to stop.  Returns 0 at stop, 1 when stopped by on_bend,
// 2 at the chain end.
template <typename T, class OnBend>
__device__ __forceinline__ int lane_scan(LaneState<T>& st, int m, int stop, const T* sv, const T* sa, OnBend on_bend)
{
    for (;;) {
        if (st.i >= stop) return 0;
        const int i = st.i;
        const T vi = sv[skew32(i)];
        const T Ai = (i < m - 1) ? sa[skew32(i)] : T(0);
        bool init = (i == st.s);
        if (!init) {
            st.uh += st.th - vi;
            st.ul += st.tl - vi;
            const bool bhi = st.uh < -Ai;
            const bool blo = !bhi && st.ul > Ai;
            if (bhi || blo) {
                const int e = bhi ? st.ih : st.il;
                const T t = bhi ? st.th : st.tl;
                st.u0 = bhi ? st.ah : -st.al;
                const int s_old = st.s;
                st.s = e + 1;
                if (on_bend(s_old, e, bhi ? 1 : 2, t)) {
                    st.i = st.s;
                    return 1;
                }
                if (st.s < i) {
                    st.i = st.s;
                    continue;
                }
                init = true;
            } else {
                const int len = i - st.s + 1;
                if (st.uh > Ai) {
                    st.th -= div_len<T>(st.uh - Ai, len);
                    st.uh = Ai;
                    st.ih = i;
                    st.ah = Ai;
                }
                if (st.ul < -Ai) {
                    st.tl += div_len<T>(-Ai - st.ul, len);
                    st.ul = -Ai;
                    st.il = i;
                    st.al = Ai;
                }
            }
        }
        if (init) {
            st.th = vi + Ai - st.u0;
            st.tl = vi - Ai - st.u0;
            st.uh = Ai;
            st.ul = -Ai;
            st.ih = st.il = i;
            st.ah = st.al = Ai;
        }
        if (i == m - 1) {
            on_bend(st.s, m - 1, 0, st.th);
            st.i = m;
            return 2;
        }
        st.i = i + 1;
    }
}


// A continuation's finished segments (end, value), kept by phase 2 so that
// phase 3 writes them instead of scanning the continuation again; a lane
// whose continuation has more than kContSegs segments scans it again.
constexpr int kContSegs = 16;

template <typename T>
struct ContSeg {
    int e;
    T t;
};

// G lanes share a chain (G = 4 .. 32, a warp holds 32/G chains); a CTA holds
// nc chains, nc * G threads.  With few chains G = 32 spreads each chain over a
// whole warp; with many, a smaller G does less speculative work per chain.
template <typename T, bool SHADOW, int G, bool LIST>
__global__ void __launch_bounds__(256) wscan_kernel(ScanArgs<T> A, int nc)
{
    extern __shared__ __align__(16) unsigned char wsm[];
    constexpr int KS = LIST ? kContSegs : 0;
    int k = 0;
    while (k + 1 < A.naxes && blockIdx.x >= A.ax[k + 1].block_begin) ++k;
    const ScanAxis<T>& X = A.ax[k];
    const int m = X.m;
    const int pitch = skew32(m) + 1;
    ContSeg<T>* sg = (ContSeg<T>*)wsm;                        // KS per lane
    T* sv = (T*)(sg + (size_t)nc * G * KS);
    T* sa = sv + (size_t)nc * pitch;
    uint8_t* code = (uint8_t*)(sa + (size_t)nc * pitch);
    const int64_t c0 = (int64_t)(blockIdx.x - X.block_begin) * nc;
    const int nvalid = (int)min((int64_t)nc, X.nchains - c0);

    auto gbase = [&](int64_t c, int64_t& vb, int64_t& ab, int64_t& st) {
        if (X.transposed) { vb = c; ab = c; st = X.nchains; }
        else {
            const int64_t o = c / X.inner, q = c - o * X.inner;
            vb = o * (int64_t)m * X.inner + q;
            ab = o * (int64_t)(m - 1) * X.inner + q;
            st = X.inner;
        }
    };
    // stage the CTA's chains (chain index fastest: consecutive chains are
    // consecutive in global memory) and clear the bend codes
    for (int idx = threadIdx.x; idx < nc * m; idx += blockDim.x) {
        const int c = idx % nc, j = idx / nc;
        code[c * m + j] = 0;
        if (c >= nvalid) continue;
        int64_t vb, ab, st;
        gbase(c0 + c, vb, ab, st);
        scan_cp_elem(sv + c * pitch + skew32(j), X.v + vb + (int64_t)j * st);
        if (j < m - 1) scan_cp_elem(sa + c * pitch + skew32(j), X.a + ab + (int64_t)j * st);
    }
    scan_cp_wait();
    __syncthreads();

    // lanes of chains past the end stay (inactive) for the group shuffles
    const int ch = threadIdx.x / G, gl = threadIdx.x % G;
    const int glane0 = (threadIdx.x & 31) & ~(G - 1);     // first warp lane of the group
    const bool valid = ch < nvalid;
    int64_t vb = 0, ab = 0, gst = 0;
    if (valid) gbase(c0 + ch, vb, ab, gst);
    T* gx = X.x + vb;
    const T* cv = sv + ch * pitch;
    const T* ca = sa + ch * pitch;
    uint8_t* cc = code + ch * m;
    const int lp = (m + G - 1) / G;               // piece length
    const int npieces = valid ? (m + lp - 1) / lp : 0;
    const int p0 = gl * lp;
    const int p1 = min(m, p0 + lp);
    const bool active = gl < npieces;
    const bool lastp = gl == npieces - 1;
    auto write_seg = [&](int from, int to, T t) {
        for (int j = from; j <= to; ++j) gx[(int64_t)j * gst] = SHADOW ? cv[skew32(j)] - t : t;
    };

    // phase 1: every piece from a guessed state
    LaneState<T> st{p0, p0, p0, p0, T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    if (active) {
        lane_scan<T>(st, m, lastp ? m : p1, cv, ca, [&](int s0, int e, int d, T t) {
            if (d) cc[e] = (uint8_t)d;
            write_seg(s0, e, t);
            return false;
        });
    }
    __syncwarp();
    // phase 2: continue until a bend recorded by a later piece (or the end),
    // keeping the segments passed
    int merge = m - 1, nseg = 0;
    ContSeg<T>* seg = sg + (size_t)threadIdx.x * KS;
    if (active && !lastp) {
        LaneState<T> s2 = st;
        lane_scan<T>(s2, m, m, cv, ca, [&](int, int e, int d, T t) {
            if constexpr (LIST) {
                if (nseg < KS) seg[nseg] = ContSeg<T>{e, t};
            }
            ++nseg;
            if (d && e >= p1 && cc[e] == (uint8_t)d) {
                merge = e;
                return true;
            }
            return false;
        });
    }
    // verified pieces: lane 0, then the piece holding each verified lane's
    // merge bend (pieces skipped over are rewritten by that continuation);
    // G steps for every group, so that the whole warp shuffles together
    const int target = (active && !lastp && merge < m - 1) ? merge / lp : npieces;
    unsigned verified = 0;
    int v = 0;
#pragma unroll 1
    for (int it = 0; it < G; ++it) {
        const bool live = v < npieces;
        if (live) verified |= 1u << v;
        const int nv = __shfl_sync(0xffffffffu, target, glane0 + (live ? v : 0));
        if (live) v = nv;
    }
    // phase 3: verified lanes write their continuation up to the merge bend
    // (the same segments phase 2 passed, from the same state)
    if (((verified >> gl) & 1u) && active && !lastp) {
        if (LIST && nseg <= KS) {
            int s0 = st.s;
            for (int q = 0; q < nseg; ++q) {
                const ContSeg<T> sq = seg[q];
                write_seg(s0, sq.e, sq.t);
                s0 = sq.e + 1;
            }
        } else {
            lane_scan<T>(st, m, m, cv, ca, [&](int s0, int e, int, T t) {
                write_seg(s0, e, t);
                return e >= merge;
            });
        }
    }
}

// ---- lane-group scan with the funnel (no rescans) --------------------------
//
// The phases of wscan_kernel with the funnel form of the taut string
// (funnel.cuh) in place of the local form: a lane's cost is then linear in
// the elements it passes, where the local form restarts behind every bend
// and is quadratic on the long plateaus of segmentation iterates.  Phase 2
// keeps the segments of its continuation (up to kFunnelSegs), so that phase 3
// writes them instead of scanning again.  A lane whose hull chain fills
// (kFunnelQ vertices), or whose continuation has more segments, falls back to
// the local form from its apex.

constexpr int kFunnelQ = 16;
constexpr int kFunnelSegs = 16;

template <typename T>
struct FSeg {
    int e;
    T t;
};

template <typename T, int G>
__host__ __device__ __forceinline__ size_t fscan_lane_bytes()
{
    return (size_t)G * (2 * kFunnelQ * sizeof(FVert<T>) + kFunnelSegs * sizeof(FSeg<T>));
}

template <typename T, bool SHADOW, int G>
__global__ void __launch_bounds__(256) fscan_kernel(ScanArgs<T> A, int nc)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    int k = 0;
    while (k + 1 < A.naxes && blockIdx.x >= A.ax[k + 1].block_begin) ++k;
    const ScanAxis<T>& X = A.ax[k];
    const int m = X.m;
    const int pitch = skew32(m) + 1;
    FVert<T>* dq = (FVert<T>*)fsm;                                    // 2 rings per lane
    FSeg<T>* sg = (FSeg<T>*)(dq + (size_t)nc * G * 2 * kFunnelQ);   // continuation segments per lane
    T* sv = (T*)(sg + (size_t)nc * G * kFunnelSegs);
    T* sa = sv + (size_t)nc * pitch;
    uint8_t* code = (uint8_t*)(sa + (size_t)nc * pitch);
    const int64_t c0 = (int64_t)(blockIdx.x - X.block_begin) * nc;
    const int nvalid = (int)min((int64_t)nc, X.nchains - c0);

    auto gbase = [&](int64_t c, int64_t& vb, int64_t& ab, int64_t& st) {
        if (X.transposed) { vb = c; ab = c; st = X.nchains; }
        else {
            const int64_t o = c / X.inner, q = c - o * X.inner;
            vb = o * (int64_t)m * X.inner + q;
            ab = o * (int64_t)(m - 1) * X.inner + q;
            st = X.inner;
        }
    };
    for (int idx = threadIdx.x; idx < nc * m; idx += blockDim.x) {
        const int c = idx % nc, j = idx / nc;
        code[c * m + j] = 0;
        if (c >= nvalid) continue;
        int64_t vb, ab, st;
        gbase(c0 + c, vb, ab, st);
        scan_cp_elem(sv + c * pitch + skew32(j), X.v + vb + (int64_t)j * st);
        if (j < m - 1) scan_cp_elem(sa + c * pitch + skew32(j), X.a + ab + (int64_t)j * st);
    }
    scan_cp_wait();
    __syncthreads();

    const int ch = threadIdx.x / G, gl = threadIdx.x % G;
    const int glane0 = (threadIdx.x & 31) & ~(G - 1);
    const bool valid = ch < nvalid;
    int64_t vb = 0, ab = 0, gst = 0;
    if (valid) gbase(c0 + ch, vb, ab, gst);
    T* gx = X.x + vb;
    const T* cv = sv + ch * pitch;
    const T* ca = sa + ch * pitch;
    uint8_t* cc = code + ch * m;
    FVert<T>* U = dq + (size_t)threadIdx.x * 2 * kFunnelQ;
    FVert<T>* L = U + kFunnelQ;
    FSeg<T>* seg = sg + (size_t)threadIdx.x * kFunnelSegs;
    const int lp = (m + G - 1) / G;
    const int npieces = valid ? (m + lp - 1) / lp : 0;
    const int p0 = gl * lp;
    const int p1 = min(m, p0 + lp);
    const bool active = gl < npieces;
    const bool lastp = gl == npieces - 1;
    auto write_seg = [&](int from, int to, T t) {
        for (int j = from; j <= to; ++j) gx[(int64_t)j * gst] = SHADOW ? cv[skew32(j)] - t : t;
    };

    // phase 1: every piece from a guessed state (a segment starting at the
    // piece start with multiplier 0; exact for piece 0)
    FunnelState<T> f = funnel_start<T>(p0);
    LaneState<T> st{};
    bool loc = false;                 // the lane runs the local form from here on
    LaneState<T> open{};              // restart state of the open segment at the piece end
    if (active) {
        auto rec = [&](int s0, int e, int d, T t) {
            if (d) cc[e] = (uint8_t)d;
            write_seg(s0, e, t);
            return false;
        };
        const int stop = lastp ? m : p1;
        if (funnel_scan<T, kFunnelQ>(f, m, stop, cv, ca, U, L, rec) == 3) {
            st = funnel_to_local<T>(f, ca);
            loc = true;
            lane_scan<T>(st, m, stop, cv, ca, rec);
        }
        if (loc) open = LaneState<T>{st.s, st.s, st.s, st.s, st.u0, T(0), T(0), T(0), T(0), T(0), T(0)};
        else open = funnel_to_local<T>(f, ca);
    }
    __syncwarp();
    // phase 2: continue until a bend recorded by a later piece (or the end),
    // keeping the segments passed
    int merge = m - 1, nseg = 0;
    if (active && !lastp) {
        auto keep = [&](int, int e, int d, T t) {
            if (nseg < kFunnelSegs) seg[nseg] = FSeg<T>{e, t};
            ++nseg;
            if (d && e >= p1 && cc[e] == (uint8_t)d) {
                merge = e;
                return true;
            }
            return false;
        };
        if (!loc && funnel_scan<T, kFunnelQ>(f, m, m, cv, ca, U, L, keep) == 3) {
            st = funnel_to_local<T>(f, ca);
            loc = true;
        }
        if (loc) lane_scan<T>(st, m, m, cv, ca, keep);
    }
    const int target = (active && !lastp && merge < m - 1) ? merge / lp : npieces;
    unsigned verified = 0;
    int v = 0;
#pragma unroll 1
    for (int it = 0; it < G; ++it) {
        const bool live = v < npieces;
        if (live) verified |= 1u << v;
        const int nv = __shfl_sync(0xffffffffu, target, glane0 + (live ? v : 0));
        if (live) v = nv;
    }
    // phase 3: verified lanes write their continuation up to the merge bend
    if (((verified >> gl) & 1u) && active && !lastp) {
        if (nseg <= kFunnelSegs) {
            int s0 = open.s;
            for (int q = 0; q < nseg; ++q) {
                const FSeg<T> sq = seg[q];
                write_seg(s0, sq.e, sq.t);
                s0 = sq.e + 1;
            }
        } else {
            lane_scan<T>(open, m, m, cv, ca, [&](int s0, int e, int, T t) {
                write_seg(s0, e, t);
                return e >= merge;
            });
        }
    }
}

template <typename T, int G>
static size_t fscan_smem(int m, int nc)
{
    return (size_t)nc * (fscan_lane_bytes<T, G>() + 2 * (size_t)(skew32(m) + 1) * sizeof(T) + (size_t)m);
}

// Chains per CTA for the funnel scan: whole warps, at most 256 threads, and
// as many chains per SM as the shared memory allows (227 KB per SM).
template <typename T, int G>
static int fscan_chains(int m)
{
    const int per_warp = 32 / G;
    int best = 0, best_per_sm = 0;
    for (int nc = per_warp; nc * G <= 256; nc += per_warp) {
        const size_t b = fscan_smem<T, G>(m, nc);
        if (b > 227 * 1024) break;
        const int per_sm = (int)((227 * 1024) / b) * nc;
        if (per_sm > best_per_sm) { best = nc; best_per_sm = per_sm; }
    }
    return best;
}

template <typename T, bool SHADOW, int G>
static cudaError_t launch_fscan_g(const ScanArgs<T>& wrp, int mmax, cudaStream_t s)
{
    const int nc = fscan_chains<T, G>(mmax);
    if (nc == 0) return cudaErrorInvalidValue;
    ScanArgs<T> a = wrp;
    int64_t blocks = 0;
    for (int k = 0; k < a.naxes; ++k) {
        a.ax[k].block_begin = blocks;
        blocks += (a.ax[k].nchains + nc - 1) / nc;
    }
    if (blocks == 0) return cudaSuccess;
    const size_t smem = fscan_smem<T, G>(mmax, nc);
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(fscan_kernel<T, SHADOW, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    fscan_kernel<T, SHADOW, G><<<(unsigned)blocks, nc * G, smem, s>>>(a, nc);
    return cudaGetLastError();
}

// Lanes per chain for the funnel scan: pieces of at least 16 elements, 4 to
// 32 lanes, and fewer lanes when a chain's staging does not fit.
template <typename T>
static int fscan_lanes(int mmax)
{
    int G = 32;
    while (G > 4 && mmax < 16 * G) G >>= 1;
    auto fits = [&](int g) {
        return g == 32 ? fscan_chains<T, 32>(mmax) > 0 : g == 16 ? fscan_chains<T, 16>(mmax) > 0
             : g == 8 ? fscan_chains<T, 8>(mmax) > 0 : fscan_chains<T, 4>(mmax) > 0;
    };
    while (G > 4 && !fits(G)) G >>= 1;
    return fits(G) ? G : 0;
}

template <typename T, bool SHADOW>
static cudaError_t launch_fscan(const ScanArgs<T>& wrp, int G, int mmax, cudaStream_t s)
{
    switch (G) {
    case 32: return launch_fscan_g<T, SHADOW, 32>(wrp, mmax, s);
    case 16: return launch_fscan_g<T, SHADOW, 16>(wrp, mmax, s);
    case 8: return launch_fscan_g<T, SHADOW, 8>(wrp, mmax, s);
    default: return launch_fscan_g<T, SHADOW, 4>(wrp, mmax, s);
    }
}

template <typename T>
static size_t wscan_smem(int m, int nc, int G, bool list)
{
    return (size_t)nc * ((size_t)G * (list ? kContSegs : 0) * sizeof(ContSeg<T>) +
                         2 * (size_t)(skew32(m) + 1) * sizeof(T) + (size_t)m);
}

// Chains per CTA for G lanes per chain: at most 256 threads, whole warps, and
// shared memory within 100 KB (two CTAs per SM); 0 if a warp's chains do not fit.
template <typename T>
static int wscan_chains(int m, int G, bool list)
{
    const int per_warp = 32 / G;
    int nc = 256 / G;
    while (nc > per_warp && wscan_smem<T>(m, nc, G, list) > 100 * 1024) nc -= per_warp;
    return wscan_smem<T>(m, nc, G, list) <= 200 * 1024 ? nc : 0;
}

template <typename T, bool SHADOW, bool LIST>
static void (*wscan_fn(int G))(ScanArgs<T>, int)
{
    return G == 32 ? wscan_kernel<T, SHADOW, 32, LIST>
         : G == 16 ? wscan_kernel<T, SHADOW, 16, LIST>
         : G == 8 ? wscan_kernel<T, SHADOW, 8, LIST>
                  : wscan_kernel<T, SHADOW, 4, LIST>;
}

// Launch plan of the lane-group scan.  A launch shape has up to four forms:
// G or G/2 lanes per chain (G from the automatic rule; a forced lane count
// keeps one) and, for each, with or without the continuation lists (they
// spare phase 3 a second scan of every verified continuation but take shared
// memory).  All forms give the same results, and which is fastest depends on
// the iterates, not only on the shape: per launch, on the 1024^2 blob
// segmentation's AAR iterates 16 lanes took 180 us against 204 us for 32,
// while its FISTA and BCD iterates ran 9% and 5% faster with 32; lists
// against plain, that AAR 203 against 238 us and FISTA 393 against 583 us,
// the 8-connected 1024^2 AAR 7% slower with them and its FISTA 2% faster,
// uniform 2048^2 BCD 10% faster and its FISTA 14% slower.  So the forms are timed: per launch shape, from the third launch
// on, the first NF launches in every kTunePeriod run one form each between
// CUDA events on the caller's stream (the iterates change along a solve, so
// the trials recur); a form whose mean is at least 10% above the fastest
// one's over 2 kTuneMin trials each is tried only once in kTuneSlowPeriod
// launches, since a trial costs its gap to the fastest form; the events are read
// without blocking at later launches, and the other launches take the form
// with the lowest mean trial time once every form has kTuneMin trials.
// Until then, and when the stream is being captured into a graph or an event
// fails, G lanes with the lists if they add no wave work (their CTAs fit the
// GPU at once, or they need no more fractional waves than the plain form).
// Occupancy comes from the runtime (the kernels' registers and shared
// memory).  Plans are cached per shape.
struct WscanPlan {
    int G;
    bool list;
    int nc;
    int64_t blocks;
    size_t smem;
};

constexpr int kTuneSkip = 2;
constexpr int kTunePeriod = 16;
constexpr int kTuneSlowPeriod = 128;
constexpr int kTuneMin = 3;
constexpr int kTuneSlots = 8;          // event pairs in flight
constexpr int kMaxForms = 4;

struct WscanEntry {
    int dev, G, mmax, naxes, force;
    int64_t nchains;
    WscanPlan form[kMaxForms];
    int nf;
    int rule;                          // form taken until every form has kTuneMin trials
    bool timing;                       // false: no timing (one form only, or an event failed)
    int launches, trials;
    cudaEvent_t ev0[kTuneSlots], ev1[kTuneSlots];
    bool pending[kTuneSlots];
    int var[kTuneSlots];
    double sum[kMaxForms];
    int cnt[kMaxForms];
};

static void wscan_entry_release(WscanEntry& E)
{
    for (int t = 0; t < kTuneSlots; ++t) {
        if (E.ev0[t]) cudaEventDestroy(E.ev0[t]);
        if (E.ev1[t]) cudaEventDestroy(E.ev1[t]);
        E.ev0[t] = E.ev1[t] = nullptr;
        E.pending[t] = false;
    }
}

// Reads the trials that have finished.  On an event error the timing stops
// and the rule's form is kept.
static void wscan_entry_poll(WscanEntry& E)
{
    if (!E.timing) return;
    for (int t = 0; t < kTuneSlots; ++t) {
        if (!E.pending[t]) continue;
        const cudaError_t q = cudaEventQuery(E.ev1[t]);
        if (q == cudaErrorNotReady) continue;
        float ms = 0.f;
        if (q != cudaSuccess || cudaEventElapsedTime(&ms, E.ev0[t], E.ev1[t]) != cudaSuccess) {
            cudaGetLastError();
            E.timing = false;
            wscan_entry_release(E);
            return;
        }
        E.pending[t] = false;
        E.sum[E.var[t]] += ms;
        E.cnt[E.var[t]] += 1;
    }
}

// The form for launches that are not trials (-1 when some form has too few
// trials: the rule's form then).
static int wscan_entry_best(const WscanEntry& E)
{
    if (!E.timing) return -1;
    int best = -1;
    for (int f = 0; f < E.nf; ++f) {
        if (E.cnt[f] < kTuneMin) return -1;
        if (best < 0 || E.sum[f] / E.cnt[f] < E.sum[best] / E.cnt[best]) best = f;
    }
    return best;
}

// Whether form f trails the fastest form far enough to be tried rarely.
static bool wscan_entry_far(const WscanEntry& E, int best, int f)
{
    return best >= 0 && f != best && E.cnt[f] >= 2 * kTuneMin && E.cnt[best] >= 2 * kTuneMin &&
           E.sum[f] / E.cnt[f] >= 1.1 * (E.sum[best] / E.cnt[best]);
}

template <typename T, bool SHADOW>
static cudaError_t wscan_entry_make(const ScanArgs<T>& wrp, int G, bool halve, int mmax, int dev, WscanEntry& E)
{
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    static bool attr_set[64][4][2] = {};
    E.nf = 0;
    double waves_g[2] = {-1.0, -1.0};  // G lanes: plain, lists
    int idx_g[2] = {-1, -1};
    for (int gv = 0; gv < (halve && G > 4 ? 2 : 1); ++gv) {
        const int g = gv ? G / 2 : G;
        const int gi = g == 32 ? 0 : g == 16 ? 1 : g == 8 ? 2 : 3;
        for (int li = 0; li < 2; ++li) {
            const bool list = li == 1;
            const int nc = wscan_chains<T>(mmax, g, list);
            if (nc == 0) continue;
            int64_t blocks = 0;
            for (int k = 0; k < wrp.naxes; ++k) blocks += (wrp.ax[k].nchains + nc - 1) / nc;
            const size_t smem = wscan_smem<T>(mmax, nc, g, list);
            void (*fn)(ScanArgs<T>, int) = list ? wscan_fn<T, SHADOW, true>(g) : wscan_fn<T, SHADOW, false>(g);
            if (dev < 0 || dev >= 64 || !attr_set[dev][gi][li]) {
                e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                if (e != cudaSuccess) return e;
                if (dev >= 0 && dev < 64) attr_set[dev][gi][li] = true;
            }
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nc * g, smem);
            if (e != cudaSuccess) return e;
            if (per_sm < 1) continue;
            if (gv == 0) {
                waves_g[li] = (double)blocks / ((double)per_sm * sms);
                idx_g[li] = E.nf;
            }
            E.form[E.nf++] = WscanPlan{g, list, nc, blocks, smem};
        }
    }
    if (E.nf == 0) return cudaErrorInvalidConfiguration;
    const double allow = waves_g[0] > 1.0 ? waves_g[0] : 1.0;
    if (idx_g[1] >= 0 && (idx_g[0] < 0 || waves_g[1] <= allow)) E.rule = idx_g[1];
    else if (idx_g[0] >= 0) E.rule = idx_g[0];
    else E.rule = 0;
    E.timing = E.nf > 1;
    E.launches = E.trials = 0;
    for (int t = 0; t < kTuneSlots; ++t) {
        E.ev0[t] = E.ev1[t] = nullptr;
        E.pending[t] = false;
        E.var[t] = 0;
    }
    for (int f = 0; f < kMaxForms; ++f) {
        E.sum[f] = 0.0;
        E.cnt[f] = 0;
    }
    return cudaSuccess;
}

// Plans (and, on trial launches, times) one lane-group scan launch and
// issues it.  G: lanes per chain of the automatic rule or the forced count;
// halve: G/2 lanes are a candidate too.
template <typename T, bool SHADOW>
static cudaError_t wscan_run(ScanArgs<T> wrp, int G, bool halve, int mmax, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int64_t nchains = 0;
    for (int k = 0; k < wrp.naxes; ++k) nchains += wrp.ax[k].nchains;
    static WscanEntry cache[8];
    static int nkeys = 0, next = 0;
    static std::mutex mu;                  // handles on other host threads share the cache
    std::lock_guard<std::mutex> lock(mu);
    WscanEntry* E = nullptr;
    const int fkey = halve ? 1 : 0;
    for (int i = 0; i < nkeys; ++i) {
        WscanEntry& c = cache[i];
        if (c.dev == dev && c.G == G && c.force == fkey && c.mmax == mmax && c.naxes == wrp.naxes &&
            c.nchains == nchains)
            E = &c;
    }
    if (!E) {
        WscanEntry& c = cache[next];
        if (next < nkeys) wscan_entry_release(c);
        c.dev = dev;
        c.G = G;
        c.force = fkey;
        c.mmax = mmax;
        c.naxes = wrp.naxes;
        c.nchains = nchains;
        e = wscan_entry_make<T, SHADOW>(wrp, G, halve, mmax, dev, c);
        if (e != cudaSuccess) return e;
        E = &c;
        next = (next + 1) % 8;
        if (nkeys < 8) ++nkeys;
    }
    {
        // event queries are not allowed in a thread with a global-mode
        // capture in progress; relaxed mode permits them and leaves it intact
        cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
        const bool swapped = cudaThreadExchangeStreamCaptureMode(&mode) == cudaSuccess;
        wscan_entry_poll(*E);
        if (swapped) cudaThreadExchangeStreamCaptureMode(&mode);
        cudaGetLastError();
    }
    const int best = wscan_entry_best(*E);
    int form = best >= 0 ? best : E->rule;
    int slot = -1;
    const int64_t since = E->launches - kTuneSkip;
    const int phase = (int)(since % kTunePeriod);
    if (E->timing && since >= 0 && phase < E->nf &&
        (!wscan_entry_far(*E, best, phase) || since % kTuneSlowPeriod < kTunePeriod)) {
        const int t = E->trials % kTuneSlots;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (!E->pending[t] && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            slot = t;
            form = phase;
        }
        cudaGetLastError();
    }
    ++E->launches;
    const WscanPlan P = E->form[form];
    int64_t blocks = 0;
    for (int k = 0; k < wrp.naxes; ++k) {
        wrp.ax[k].block_begin = blocks;
        blocks += (wrp.ax[k].nchains + P.nc - 1) / P.nc;
    }
    if (blocks == 0) return cudaSuccess;
    if (slot >= 0) {
        if ((E->ev0[slot] || cudaEventCreate(&E->ev0[slot]) == cudaSuccess) &&
            (E->ev1[slot] || cudaEventCreate(&E->ev1[slot]) == cudaSuccess) &&
            cudaEventRecord(E->ev0[slot], s) == cudaSuccess) {
            E->pending[slot] = true;
            E->var[slot] = form;
            ++E->trials;
        } else {                           // no timing: keep the rule's form
            cudaGetLastError();
            E->timing = false;
            wscan_entry_release(*E);
            slot = -1;
        }
    }
    void (*fn)(ScanArgs<T>, int) = P.list ? wscan_fn<T, SHADOW, true>(P.G) : wscan_fn<T, SHADOW, false>(P.G);
    fn<<<(unsigned)P.blocks, P.nc * P.G, P.smem, s>>>(wrp, P.nc);
    e = cudaGetLastError();
    if (slot >= 0 && E->pending[slot] && cudaEventRecord(E->ev1[slot], s) != cudaSuccess) {
        cudaGetLastError();
        E->timing = false;
        wscan_entry_release(*E);
    }
    return e;
}


// ---- entry points for the dispatch in scan.cu ---------------------------------

// Whether one chain of m elements can be staged for the lane-group scan.
template <typename T>
bool lane_scan_fits(int m)
{
    return wscan_smem<T>(m, 1, 32, false) <= 200 * 1024;
}

// Lane-group scan of every chain of wrp's axes: lanes per chain from
// wrp.force (0 automatic: pieces of about 16 elements, measured on 256^3 and
// 128^3 grids and 1024^2 images: fewer pieces per chain do less speculative
// work, shorter ones keep more lanes busy; 2..5: 32, 16, 8 or 4 lanes).
template <typename T>
cudaError_t launch_lane_scan(ScanArgs<T> wrp, cudaStream_t s)
{
    int mmax = 0;
    for (int k = 0; k < wrp.naxes; ++k) mmax = max(mmax, wrp.ax[k].m);
    int G = 32;
    if (wrp.force == 0) while (G > 4 && mmax < 16 * G) G >>= 1;
    else G = wrp.force == 3 ? 16 : wrp.force == 4 ? 8 : wrp.force == 5 ? 4 : 32;
    if (wscan_chains<T>(mmax, G, false) == 0) G = 32;   // long chains: whole warps
    const bool halve = wrp.force == 0;                 // automatic: G / 2 lanes are a candidate too
    return wrp.shadow ? wscan_run<T, true>(wrp, G, halve, mmax, s) : wscan_run<T, false>(wrp, G, halve, mmax, s);
}

// Whether a chain of m elements fits the funnel lane-group scan.
template <typename T>
bool funnel_scan_fits(int m)
{
    return fscan_lanes<T>(m) > 0;
}

// Funnel lane-group scan of every chain of fun's axes (mapping 11).
template <typename T>
cudaError_t launch_funnel_scan(ScanArgs<T> fun, cudaStream_t s)
{
    int mmax = 0;
    for (int k = 0; k < fun.naxes; ++k) mmax = max(mmax, fun.ax[k].m);
    const int G = fscan_lanes<T>(mmax);
    return fun.shadow ? launch_fscan<T, true>(fun, G, mmax, s) : launch_fscan<T, false>(fun, G, mmax, s);
}

template bool lane_scan_fits<float>(int);
template bool lane_scan_fits<double>(int);
template cudaError_t launch_lane_scan<float>(ScanArgs<float>, cudaStream_t);
template cudaError_t launch_lane_scan<double>(ScanArgs<double>, cudaStream_t);
template bool funnel_scan_fits<float>(int);
template bool funnel_scan_fits<double>(int);
template cudaError_t launch_funnel_scan<float>(ScanArgs<float>, cudaStream_t);
template cudaError_t launch_funnel_scan<double>(ScanArgs<double>, cudaStream_t);

}  // namespace tvcut
