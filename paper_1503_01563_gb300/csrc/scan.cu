// Iteration kernels of the methods of Sec. 4.
//
// AAR and AP: one iteration = one scan launch + one update launch:
//
//   scan:   x_k = prox_{f_k}(s_k) on every chain of every block k at once.
//           The blocks' projections are independent in the product space
//           (Sec. 4.2: Pi_K splits into the Pi_{K_k}), so all axes share one
//           launch; a thread (reading weights padded to the state layout, so
//           that each element is loaded one step ahead), or a group of 4-32
//           lanes, owns one chain.  The prox is the taut string of Sec. 3.2
//           in local form (see scan_chain).  Each block's state is stored so
//           that consecutive chains are consecutive in memory ("chain-major"):
//           the natural row-major layout already is for every axis but the
//           last, the last axis' block (rows) is kept transposed, and the
//           zig-zag path blocks of an 8-connected grid use the transposed
//           layout with rows swapped within pairs.  A warp's loads of one
//           step are thus one 128-byte line.
//
//   update: per vertex, y_k = s_k - x_k and
//             AAR (Eq. 3 with Eq. dualA): s_k <- y_k + (w - 2 sum y + sum s)/r
//             AP  (Sec. 4.2):             s_k <- y_k + (w - sum y)/r
//           and, on check iterations, the primal x = w - sum_k y_k (Sec. 2.3).
//           Elementwise and coalesced (16-byte accesses in FP32); the
//           transposed blocks go through shared-memory tiles.
//
// BCD and FISTA (Sec. 4.1) hold the duals y_k; their passes form the point to
// project (bcd_prepare_kernel, fista_prepare_kernel, prep8_kernel) and the
// scan writes the projection v - prox(v) directly (SHADOW).
#include <mutex>

#include "tvcut_internal.cuh"
#include "taut_string.cuh"
#include "funnel.cuh"

namespace tvcut {

constexpr int kScanThreads = 128;

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

// PADDED: every axis carries its weights in the state's layout (ap), so the
// scan loads each element one step ahead (scan_chain_padded).  Used for the
// prox output only: the projection-mode padded scan needs 48 registers, and
// at 48 a 256^3 launch (196,608 chains, 10 CTAs of 128 per SM) no longer
// fits the GPU in one wave; the compact scan needs 40.
template <typename T, bool SHADOW, bool PADDED>
__global__ void __launch_bounds__(kScanThreads) scan_kernel(ScanArgs<T> A)
{
    int k = 0;
    while (k + 1 < A.naxes && blockIdx.x >= A.ax[k + 1].block_begin) ++k;
    const ScanAxis<T>& X = A.ax[k];
    const int64_t c = (int64_t)(blockIdx.x - X.block_begin) * kScanThreads + threadIdx.x;
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
    if constexpr (PADDED) scan_chain_padded<T, SHADOW>(X.m, X.v + base, X.ap + base, X.x + base, stride);
    else scan_chain<T, SHADOW>(X.m, X.v + base, X.a + abase, X.x + base, stride);
}

template <typename T>
__global__ void pad_weights_kernel(const T* __restrict__ a, T* __restrict__ ap, int64_t n, int64_t nchains,
                                   int64_t inner, int m, int transposed)
{
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t j, src;
        if (transposed) {                        // element j of chain c at j * nchains + c, both layouts
            j = idx / nchains;
            src = idx;
        } else {                                 // chain (o, q): o * m * inner + j * inner + q, compact (m - 1)
            const int64_t o = idx / ((int64_t)m * inner);
            j = idx / inner - o * m;
            src = idx - o * inner;
        }
        ap[idx] = j < m - 1 ? a[src] : T(0);
    }
}

template <typename T>
cudaError_t launch_pad_weights(const ScanAxis<T>& X, T* ap, cudaStream_t s)
{
    const int64_t n = X.nchains * (int64_t)X.m;
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    pad_weights_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(X.a, ap, n, X.nchains, X.inner, X.m, X.transposed);
    return cudaGetLastError();
}

// ---- lane-group (speculative pieces) scan -------------------------------------
//
// For few, long chains (a 2D grid has only H + W of them) one thread per chain
// leaves the GPU idle, so G lanes (4 .. 32, the kernel's template parameter)
// share one chain: lane L scans piece L of G from a guessed state (a segment starts at the piece start with multiplier
// 0; exact for lane 0) and records every bend it finds (position e and
// direction).  After a bend at e the scan state is fixed (the next segment
// starts at e+1 with multiplier +-a_e), so a lane's trajectory is the true one
// from the first bend it shares with the true scan.  Lane L then continues
// from its own piece end into piece L+1 until it produces a bend that lane
// L+1 (or any later lane) recorded; that lane's results after the bend are
// then exact, and lane L rewrites every position before it.  Lane 0 is
// exact, so following merges from lane 0 reaches the chain end through
// verified lanes only; lanes not on that path are overwritten.  A launch
// lasts as long as its slowest chain's critical path (piece, continuation,
// rewrite); where shared memory allows it without another wave of CTAs,
// each lane keeps its continuation's segments so that the rewrite only
// stores them (the same values: the same scan from the same state).

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

// Launch plan of the lane-group scan for G lanes per chain: with or without
// the continuation lists (they spare phase 3 a second scan of every verified
// continuation but take shared memory), whichever needs fewer waves of CTAs
// over the GPU (the lists on a tie).  Occupancy comes from the runtime (the
// kernels' registers and shared memory); plans are cached per shape.
struct WscanPlan {
    bool list;
    int nc;
    int64_t blocks;
    size_t smem;
};

template <typename T, bool SHADOW>
static cudaError_t wscan_plan(const ScanArgs<T>& wrp, int G, int mmax, WscanPlan& P)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int64_t nchains = 0;
    for (int k = 0; k < wrp.naxes; ++k) nchains += wrp.ax[k].nchains;
    struct Key {
        int dev, G, mmax, naxes;
        int64_t nchains;
    };
    static Key keys[8];
    static WscanPlan plans[8];
    static int nkeys = 0, next = 0;
    static std::mutex mu;                  // handles on other host threads share the cache
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < nkeys; ++i)
        if (keys[i].dev == dev && keys[i].G == G && keys[i].mmax == mmax && keys[i].naxes == wrp.naxes &&
            keys[i].nchains == nchains) {
            P = plans[i];
            return cudaSuccess;
        }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    static bool attr_set[64][4][2] = {};
    const int gi = G == 32 ? 0 : G == 16 ? 1 : G == 8 ? 2 : 3;
    int64_t waves[2] = {-1, -1};
    WscanPlan cand[2];
    for (int li = 0; li < 2; ++li) {
        const bool list = li == 1;
        const int nc = wscan_chains<T>(mmax, G, list);
        if (nc == 0) continue;
        int64_t blocks = 0;
        for (int k = 0; k < wrp.naxes; ++k) blocks += (wrp.ax[k].nchains + nc - 1) / nc;
        const size_t smem = wscan_smem<T>(mmax, nc, G, list);
        void (*fn)(ScanArgs<T>, int) = list ? wscan_fn<T, SHADOW, true>(G) : wscan_fn<T, SHADOW, false>(G);
        if (dev < 0 || dev >= 64 || !attr_set[dev][gi][li]) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) attr_set[dev][gi][li] = true;
        }
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nc * G, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) continue;
        waves[li] = (blocks + (int64_t)per_sm * sms - 1) / ((int64_t)per_sm * sms);
        cand[li] = WscanPlan{list, nc, blocks, smem};
    }
    if (waves[1] >= 0 && (waves[0] < 0 || waves[1] <= waves[0])) P = cand[1];
    else if (waves[0] >= 0) P = cand[0];
    else return cudaErrorInvalidConfiguration;
    keys[next] = Key{dev, G, mmax, wrp.naxes, nchains};
    plans[next] = P;
    next = (next + 1) % 8;
    if (nkeys < 8) ++nkeys;
    return cudaSuccess;
}

template <typename T, bool SHADOW>
static cudaError_t launch_wscan(const ScanArgs<T>& wrp, int G, const WscanPlan& P, cudaStream_t s)
{
    void (*fn)(ScanArgs<T>, int) = P.list ? wscan_fn<T, SHADOW, true>(G) : wscan_fn<T, SHADOW, false>(G);
    fn<<<(unsigned)P.blocks, P.nc * G, P.smem, s>>>(wrp, P.nc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scan(ScanArgs<T> A, cudaStream_t s)
{
    // one thread per chain unless the launch has too few chains to fill the
    // GPU, in which case long chains go to the lane-group scan (measured
    // on 256^3: 65,536 chains of 256 run faster as warps, 196,608 as threads)
    if (A.force == 6) {            // message passing for the chains that fit, one thread per chain for the rest
        ScanArgs<T> mp = A, rest = A;
        mp.naxes = rest.naxes = 0;
        rest.force = 1;
        for (int k = 0; k < A.naxes; ++k) {
            if (A.ax[k].m <= kMpMaxLen) mp.ax[mp.naxes++] = A.ax[k];
            else rest.ax[rest.naxes++] = A.ax[k];
        }
        cudaError_t e = launch_mp_prox<T>(mp, s);
        if (e != cudaSuccess || rest.naxes == 0) return e;
        return launch_scan<T>(rest, s);
    }
    if (A.force == 7) {            // funnel lane groups for the chains whose staging fits, one thread per chain for the rest
        ScanArgs<T> fun = A, rest = A;
        fun.naxes = rest.naxes = 0;
        rest.force = 1;
        int mmax = 0;
        for (int k = 0; k < A.naxes; ++k) {
            if (A.ax[k].m >= 2 && fscan_lanes<T>(A.ax[k].m) > 0) {
                fun.ax[fun.naxes++] = A.ax[k];
                mmax = max(mmax, A.ax[k].m);
            } else {
                rest.ax[rest.naxes++] = A.ax[k];
            }
        }
        if (fun.naxes) {
            const int G = fscan_lanes<T>(mmax);
            cudaError_t e = A.shadow ? launch_fscan<T, true>(fun, G, mmax, s) : launch_fscan<T, false>(fun, G, mmax, s);
            if (e != cudaSuccess) return e;
        }
        return rest.naxes ? launch_scan<T>(rest, s) : cudaSuccess;
    }
    int64_t total = 0;
    for (int k = 0; k < A.naxes; ++k) total += A.ax[k].nchains;
    ScanArgs<T> thr, wrp;
    thr.naxes = wrp.naxes = 0;
    thr.force = wrp.force = A.force;
    thr.shadow = wrp.shadow = A.shadow;
    for (int k = 0; k < A.naxes; ++k) {
        const ScanAxis<T>& X = A.ax[k];
        bool warp = X.m >= 64 && total <= 98304 && wscan_smem<T>(X.m, 1, 32, false) <= 200 * 1024;
        if (A.force == 1) warp = false;
        if (A.force >= 2) warp = X.m >= 2 && wscan_smem<T>(X.m, 1, 32, false) <= 200 * 1024;
        if (warp) wrp.ax[wrp.naxes++] = X;
        else thr.ax[thr.naxes++] = X;
    }
    if (thr.naxes) {
        int64_t blocks = 0;
        for (int k = 0; k < thr.naxes; ++k) {
            thr.ax[k].block_begin = blocks;
            blocks += (thr.ax[k].nchains + kScanThreads - 1) / kScanThreads;
        }
        bool padded = !A.shadow;
        for (int k = 0; k < thr.naxes; ++k) padded = padded && thr.ax[k].ap != nullptr;
        if (blocks > 0) {
            const dim3 g((unsigned)blocks), b(kScanThreads);
            if (padded) {
                scan_kernel<T, false, true><<<g, b, 0, s>>>(thr);
            } else {
                if (A.shadow) scan_kernel<T, true, false><<<g, b, 0, s>>>(thr);
                else scan_kernel<T, false, false><<<g, b, 0, s>>>(thr);
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    if (wrp.naxes) {
        int mmax = 0;
        for (int k = 0; k < wrp.naxes; ++k) mmax = max(mmax, wrp.ax[k].m);
        // automatic: pieces of about 16 elements (measured on 256^3 and 128^3
        // grids and 1024^2 images: fewer pieces per chain do less speculative
        // work, shorter ones keep more lanes busy)
        int G = 32;
        if (A.force == 0) while (G > 4 && mmax < 16 * G) G >>= 1;
        else G = A.force == 3 ? 16 : A.force == 4 ? 8 : A.force == 5 ? 4 : 32;
        if (wscan_chains<T>(mmax, G, false) == 0) G = 32;   // long chains: whole warps
        WscanPlan P;
        cudaError_t e = A.shadow ? wscan_plan<T, true>(wrp, G, mmax, P) : wscan_plan<T, false>(wrp, G, mmax, P);
        if (e != cudaSuccess) return e;
        int64_t blocks = 0;
        for (int k = 0; k < wrp.naxes; ++k) {
            wrp.ax[k].block_begin = blocks;
            blocks += (wrp.ax[k].nchains + P.nc - 1) / P.nc;
        }
        if (blocks > 0)
            return A.shadow ? launch_wscan<T, true>(wrp, G, P, s) : launch_wscan<T, false>(wrp, G, P, s);
    }
    return cudaSuccess;
}

// ---- update -----------------------------------------------------------------
//
// The grid is viewed as R rows of W = dims[last] columns.  Natural arrays hold
// (r, c) at r*W + c; the last block's state and prox output are transposed,
// (r, c) at c*R + r.  A CTA owns a 32x32 tile; the transposed arrays are
// staged through shared memory.

constexpr int kTile = 32;
constexpr int kUpdThreads = 256;

template <typename T, int MODE, int R_>
__global__ void __launch_bounds__(kUpdThreads) update_kernel(UpdateArgs<T> A)
{
    __shared__ T sz[kTile][kTile + 1];
    __shared__ T sx[kTile][kTile + 1];
    const int64_t R = A.rows, W = A.cols;
    const int64_t tiles_c = (W + kTile - 1) / kTile;
    const int64_t r0 = (blockIdx.x / tiles_c) * kTile;
    const int64_t c0 = (blockIdx.x % tiles_c) * kTile;
    constexpr int last = R_ - 1;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;    // 32 x 8

    // stage the transposed block: element (r0+rr, c0+cc) at (c0+cc)*R + r0+rr
#pragma unroll
    for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
        const int64_t c = c0 + cc, r = r0 + tx;
        if (c < W && r < R) {
            sz[cc][tx] = A.s[last][c * R + r];
            sx[cc][tx] = A.x[last][c * R + r];
        }
    }
    __syncthreads();
#pragma unroll
    for (int rr = ty; rr < kTile; rr += kUpdThreads / kTile) {
        const int64_t r = r0 + rr, c = c0 + tx;
        if (r >= R || c >= W) continue;
        const int64_t g = r * W + c;
        const T wg = A.w[g];
        T yk[R_];
        T ysum = T(0), ssum = T(0);
#pragma unroll
        for (int k = 0; k < R_; ++k) {
            const T sv = (k == last) ? sz[tx][rr] : A.s[k][g];
            const T xv = (k == last) ? sx[tx][rr] : A.x[k][g];
            yk[k] = sv - xv;
            ysum += yk[k];
            ssum += sv;
        }
        if (A.check) A.xout[g] = wg - ysum;
        if constexpr (MODE != UPD_EVAL) {
            T c;
            if constexpr (MODE == UPD_AAR) c = (wg - T(2) * ysum + ssum) / T(R_);
            else c = (wg - ysum) / T(R_);
#pragma unroll
            for (int k = 0; k < R_; ++k) {
                const T nv = yk[k] + c;
                if (k == last) sz[tx][rr] = nv;
                else A.s[k][g] = nv;
            }
        }
    }
    if constexpr (MODE != UPD_EVAL) {
        __syncthreads();
#pragma unroll
        for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
            const int64_t c = c0 + cc, r = r0 + tx;
            if (c < W && r < R) A.s[last][c * R + r] = sz[cc][tx];
        }
    }
}

// FP32 form with 16-byte accesses (rows and columns multiples of 4): a thread
// owns row rr and four consecutive columns of the 32 x 32 tile, the
// transposed block is staged four rows at a time; the arithmetic and its
// order are those of update_kernel.
template <int MODE, int R_>
__global__ void __launch_bounds__(kUpdThreads) update_kernel_v4(UpdateArgs<float> A)
{
    __shared__ float sz[kTile][kTile + 1];
    __shared__ float sx[kTile][kTile + 1];
    const int64_t R = A.rows, W = A.cols;
    const int64_t tiles_c = (W + kTile - 1) / kTile;
    const int64_t r0 = (blockIdx.x / tiles_c) * kTile;
    const int64_t c0 = (blockIdx.x % tiles_c) * kTile;
    constexpr int last = R_ - 1;
    const int q4 = threadIdx.x & 7, rr = threadIdx.x >> 3;          // 8 quads x 32 rows
    {   // stage the transposed block: element (r0+i, c0+cc) at (c0+cc)*R + r0+i
        const int cc = rr;
        const int64_t c = c0 + cc, r = r0 + 4 * q4;
        if (c < W && r < R) {
            const float4 zv = *(const float4*)(A.s[last] + c * R + r);
            const float4 xv = *(const float4*)(A.x[last] + c * R + r);
            sz[cc][4 * q4 + 0] = zv.x; sz[cc][4 * q4 + 1] = zv.y; sz[cc][4 * q4 + 2] = zv.z; sz[cc][4 * q4 + 3] = zv.w;
            sx[cc][4 * q4 + 0] = xv.x; sx[cc][4 * q4 + 1] = xv.y; sx[cc][4 * q4 + 2] = xv.z; sx[cc][4 * q4 + 3] = xv.w;
        }
    }
    __syncthreads();
    const int64_t r = r0 + rr, c = c0 + 4 * q4;
    if (r < R && c < W) {
        const int64_t g = r * W + c;
        const float4 w4 = *(const float4*)(A.w + g);
        float4 sv4[R_], xv4[R_];
#pragma unroll
        for (int k = 0; k < R_; ++k) {
            if (k == last) {
                sv4[k] = make_float4(sz[4 * q4 + 0][rr], sz[4 * q4 + 1][rr], sz[4 * q4 + 2][rr], sz[4 * q4 + 3][rr]);
                xv4[k] = make_float4(sx[4 * q4 + 0][rr], sx[4 * q4 + 1][rr], sx[4 * q4 + 2][rr], sx[4 * q4 + 3][rr]);
            } else {
                sv4[k] = *(const float4*)(A.s[k] + g);
                xv4[k] = *(const float4*)(A.x[k] + g);
            }
        }
        float out[R_][4];
        float xo[4];
        const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float yk[R_];
            float ysum = 0.f, ssum = 0.f;
#pragma unroll
            for (int k = 0; k < R_; ++k) {
                const float sv = j == 0 ? sv4[k].x : j == 1 ? sv4[k].y : j == 2 ? sv4[k].z : sv4[k].w;
                const float xv = j == 0 ? xv4[k].x : j == 1 ? xv4[k].y : j == 2 ? xv4[k].z : xv4[k].w;
                yk[k] = sv - xv;
                ysum += yk[k];
                ssum += sv;
            }
            xo[j] = wv[j] - ysum;
            float cc;
            if constexpr (MODE == UPD_AAR) cc = (wv[j] - 2.f * ysum + ssum) / float(R_);
            else cc = (wv[j] - ysum) / float(R_);
#pragma unroll
            for (int k = 0; k < R_; ++k) out[k][j] = yk[k] + cc;
        }
        if (A.check) *(float4*)(A.xout + g) = make_float4(xo[0], xo[1], xo[2], xo[3]);
        if constexpr (MODE != UPD_EVAL) {
#pragma unroll
            for (int k = 0; k < R_; ++k) {
                if (k == last) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) sz[4 * q4 + j][rr] = out[k][j];
                } else {
                    *(float4*)(A.s[k] + g) = make_float4(out[k][0], out[k][1], out[k][2], out[k][3]);
                }
            }
        }
    }
    if constexpr (MODE != UPD_EVAL) {
        __syncthreads();
        const int cc = rr;
        const int64_t c2 = c0 + cc, r2 = r0 + 4 * q4;
        if (c2 < W && r2 < R)
            *(float4*)(A.s[last] + c2 * R + r2) =
                make_float4(sz[cc][4 * q4 + 0], sz[cc][4 * q4 + 1], sz[cc][4 * q4 + 2], sz[cc][4 * q4 + 3]);
    }
}

template <typename T>
static bool update_v4_ok(const UpdateArgs<T>& A)
{
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
        if (A.rows % 4 || A.cols % 4) return false;
        uintptr_t m = (uintptr_t)A.w | (uintptr_t)A.xout;
        for (int k = 0; k < A.r; ++k) m |= (uintptr_t)A.s[k] | (uintptr_t)A.x[k];
        return (m & 15) == 0;
    }
}

template <typename T>
cudaError_t launch_update(int mode, const UpdateArgs<T>& A, cudaStream_t s)
{
    const int64_t tiles = ((A.rows + kTile - 1) / kTile) * ((A.cols + kTile - 1) / kTile);
    if (tiles == 0) return cudaSuccess;
    if (A.r != 2 && A.r != 3) return cudaErrorInvalidValue;
    if constexpr (sizeof(T) == 4) {
        if (update_v4_ok(A)) {
            const UpdateArgs<float>& F = reinterpret_cast<const UpdateArgs<float>&>(A);
#define TVCUT_UPD4(M)                                                                      \
    (A.r == 3 ? (update_kernel_v4<M, 3><<<(unsigned)tiles, kUpdThreads, 0, s>>>(F), 0)      \
              : (update_kernel_v4<M, 2><<<(unsigned)tiles, kUpdThreads, 0, s>>>(F), 0))
            switch (mode) {
            case UPD_AAR: TVCUT_UPD4(UPD_AAR); break;
            case UPD_AP: TVCUT_UPD4(UPD_AP); break;
            case UPD_EVAL: TVCUT_UPD4(UPD_EVAL); break;
            default: return cudaErrorInvalidValue;
            }
#undef TVCUT_UPD4
            return cudaGetLastError();
        }
    }
#define TVCUT_UPD(M)                                                                       \
    (A.r == 3 ? (update_kernel<T, M, 3><<<(unsigned)tiles, kUpdThreads, 0, s>>>(A), 0)      \
              : (update_kernel<T, M, 2><<<(unsigned)tiles, kUpdThreads, 0, s>>>(A), 0))
    switch (mode) {
    case UPD_AAR: TVCUT_UPD(UPD_AAR); break;
    case UPD_AP: TVCUT_UPD(UPD_AP); break;
    case UPD_EVAL: TVCUT_UPD(UPD_EVAL); break;
    default: return cudaErrorInvalidValue;
    }
#undef TVCUT_UPD
    return cudaGetLastError();
}

// ---- layout conversion of one block: natural (R x W) <-> transposed (W x R) ----

template <typename T>
__global__ void __launch_bounds__(kUpdThreads) transpose_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                                int64_t R, int64_t W)
{
    __shared__ T t[kTile][kTile + 1];
    const int64_t tiles_c = (W + kTile - 1) / kTile;
    const int64_t r0 = (blockIdx.x / tiles_c) * kTile;
    const int64_t c0 = (blockIdx.x % tiles_c) * kTile;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    for (int rr = ty; rr < kTile; rr += kUpdThreads / kTile) {
        const int64_t r = r0 + rr, c = c0 + tx;
        if (r < R && c < W) t[rr][tx] = in[r * W + c];
    }
    __syncthreads();
    for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
        const int64_t c = c0 + cc, r = r0 + tx;
        if (r < R && c < W) out[c * R + r] = t[tx][cc];
    }
}

template <typename T>
cudaError_t launch_transpose(const T* in, T* out, int64_t R, int64_t W, cudaStream_t s)
{
    const int64_t tiles = ((R + kTile - 1) / kTile) * ((W + kTile - 1) / kTile);
    if (tiles == 0) return cudaSuccess;
    transpose_kernel<T><<<(unsigned)tiles, kUpdThreads, 0, s>>>(in, out, R, W);
    return cudaGetLastError();
}

// BCD (Sec. 4.1): out = w - sum_{j != skip} y_j for every vertex, written in
// the layout of block `skip` (transposed when skip is the last block; natural
// when skip < 0 or another block).  Tile-based like the update: the last
// block's duals are transposed through shared memory.
template <typename T, int R_>
__global__ void __launch_bounds__(kUpdThreads) bcd_prepare_kernel(UpdateArgs<T> A, int skip)
{
    __shared__ T sy[kTile][kTile + 1];
    const int64_t R = A.rows, W = A.cols;
    const int64_t tiles_c = (W + kTile - 1) / kTile;
    const int64_t r0 = (blockIdx.x / tiles_c) * kTile;
    const int64_t c0 = (blockIdx.x % tiles_c) * kTile;
    constexpr int last = R_ - 1;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    if (skip != last) {
#pragma unroll
        for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
            const int64_t c = c0 + cc, r = r0 + tx;
            if (c < W && r < R) sy[cc][tx] = A.s[last][c * R + r];
        }
    }
    __syncthreads();
#pragma unroll
    for (int rr = ty; rr < kTile; rr += kUpdThreads / kTile) {
        const int64_t r = r0 + rr, c = c0 + tx;
        if (r >= R || c >= W) continue;
        const int64_t g = r * W + c;
        T v = A.w[g];
#pragma unroll
        for (int k = 0; k < R_; ++k) {
            if (k == skip) continue;
            v -= (k == last) ? sy[tx][rr] : A.s[k][g];
        }
        if (skip == last) sy[tx][rr] = v;
        else A.xout[g] = v;
    }
    if (skip == last) {
        __syncthreads();
#pragma unroll
        for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
            const int64_t c = c0 + cc, r = r0 + tx;
            if (c < W && r < R) A.xout[c * R + r] = sy[cc][tx];
        }
    }
}

template <typename T>
cudaError_t launch_bcd_prepare(const UpdateArgs<T>& A, int skip, cudaStream_t s)
{
    const int64_t tiles = ((A.rows + kTile - 1) / kTile) * ((A.cols + kTile - 1) / kTile);
    if (tiles == 0) return cudaSuccess;
    if (A.r == 3) bcd_prepare_kernel<T, 3><<<(unsigned)tiles, kUpdThreads, 0, s>>>(A, skip);
    else if (A.r == 2) bcd_prepare_kernel<T, 2><<<(unsigned)tiles, kUpdThreads, 0, s>>>(A, skip);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// FISTA on the smooth dual (Sec. 4.1): g(y) = 1/2 ||sum_k y_k - w||^2 has the
// same gradient sum_j u_j - w in every block and Lipschitz constant r, so the
// gradient step from the extrapolated point u is Pi_L(u).  Per vertex, for all
// blocks: u_k = y_k + beta (y_k - p_k), v_k = u_k + (w - sum_j u_j) / r.  The
// scan then writes Pi_{K_k}(v_k) over p (the buffers swap roles afterwards).
template <typename T, int R_>
__global__ void __launch_bounds__(kUpdThreads) fista_prepare_kernel(FistaArgs<T> A)
{
    __shared__ T sy[kTile][kTile + 1];
    __shared__ T sp[kTile][kTile + 1];
    const int64_t R = A.rows, W = A.cols;
    const int64_t tiles_c = (W + kTile - 1) / kTile;
    const int64_t r0 = (blockIdx.x / tiles_c) * kTile;
    const int64_t c0 = (blockIdx.x % tiles_c) * kTile;
    constexpr int last = R_ - 1;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
#pragma unroll
    for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
        const int64_t c = c0 + cc, r = r0 + tx;
        if (c < W && r < R) {
            sy[cc][tx] = A.y[last][c * R + r];
            sp[cc][tx] = A.p[last][c * R + r];
        }
    }
    __syncthreads();
#pragma unroll
    for (int rr = ty; rr < kTile; rr += kUpdThreads / kTile) {
        const int64_t r = r0 + rr, c = c0 + tx;
        if (r >= R || c >= W) continue;
        const int64_t g = r * W + c;
        T u[R_];
        T usum = T(0);
#pragma unroll
        for (int k = 0; k < R_; ++k) {
            const T yv = (k == last) ? sy[tx][rr] : A.y[k][g];
            const T pv = (k == last) ? sp[tx][rr] : A.p[k][g];
            u[k] = yv + A.beta * (yv - pv);
            usum += u[k];
        }
        const T corr = (A.w[g] - usum) / T(R_);
#pragma unroll
        for (int k = 0; k < R_; ++k) {
            const T vv = u[k] + corr;
            if (k == last) sy[tx][rr] = vv;
            else A.v[k][g] = vv;
        }
    }
    __syncthreads();
#pragma unroll
    for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
        const int64_t c = c0 + cc, r = r0 + tx;
        if (c < W && r < R) A.v[last][c * R + r] = sy[cc][tx];
    }
}

template <typename T>
cudaError_t launch_fista_prepare(const FistaArgs<T>& A, cudaStream_t s)
{
    const int64_t tiles = ((A.rows + kTile - 1) / kTile) * ((A.cols + kTile - 1) / kTile);
    if (tiles == 0) return cudaSuccess;
    if (A.r == 3) fista_prepare_kernel<T, 3><<<(unsigned)tiles, kUpdThreads, 0, s>>>(A);
    else if (A.r == 2) fista_prepare_kernel<T, 2><<<(unsigned)tiles, kUpdThreads, 0, s>>>(A);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---- 8-connected 2D grids ------------------------------------------------------

template <typename T>
__global__ void zz_weights_kernel(const T* __restrict__ ad, const T* __restrict__ aa, T* __restrict__ wz, int H,
                                  int W, int block)
{
    const int64_t total = (int64_t)(W - 1) * H;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / H), q = (int)(i - (int64_t)c * H);
        const int r0 = zz_row(q, c, H, block), r1 = zz_row(q, c + 1, H, block);
        T v = T(0);
        if (r1 == r0 + 1) v = ad[(int64_t)r0 * (W - 1) + c];          // diagonal (r0, c)-(r0+1, c+1)
        else if (r1 == r0 - 1) v = aa[(int64_t)r1 * (W - 1) + c];     // anti-diagonal (r1, c+1)-(r1+1, c)
        wz[i] = v;
    }
}

template <typename T>
cudaError_t launch_zz_weights(const T* ad, const T* aa, T* wz, int H, int W, int block, cudaStream_t s)
{
    const int64_t total = (int64_t)(W - 1) * H;
    if (total <= 0) return cudaSuccess;
    const int blocks = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
    zz_weights_kernel<T><<<blocks, 256, 0, s>>>(ad, aa, wz, H, W, block);
    return cudaGetLastError();
}

template <typename T>
__global__ void zz_relayout_kernel(const T* __restrict__ in, T* __restrict__ out, int H, int W, int block,
                                   int to_paths)
{
    const int64_t total = (int64_t)H * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        if (to_paths) {          // out[c * H + q] = vertex (zz_row(q, c), c)
            const int c = (int)(i / H), q = (int)(i - (int64_t)c * H);
            out[i] = in[(int64_t)zz_row(q, c, H, block) * W + c];
        } else {                 // out[r * W + c] = position c * H + zz_row(r, c)
            const int r = (int)(i / W), c = (int)(i - (int64_t)r * W);
            out[i] = in[(int64_t)c * H + zz_row(r, c, H, block)];
        }
    }
}

template <typename T>
cudaError_t launch_zz_relayout(const T* in, T* out, int H, int W, int block, bool to_paths, cudaStream_t s)
{
    const int64_t total = (int64_t)H * W;
    if (total <= 0) return cudaSuccess;
    const int blocks = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
    zz_relayout_kernel<T><<<blocks, 256, 0, s>>>(in, out, H, W, block, to_paths ? 1 : 0);
    return cudaGetLastError();
}

// AAR / AP update (or the primal only) of an 8-connected 2D grid, four
// blocks.  A CTA owns 32 x 32 vertices.  The row block (transposed) is
// staged like in update_kernel; the two path blocks are staged over the path
// positions q in [r0 - 1, r0 + 33) of the tile's columns, which hold every
// position of the tile's vertices (a path leaves its row by at most one), and
// only the positions whose vertex lies in the tile are written back.
constexpr int kZzWin = kTile + 2;
template <typename T, int MODE>
__global__ void __launch_bounds__(kUpdThreads) update8_kernel(Update8Args<T> A)
{
    extern __shared__ __align__(16) unsigned char u8sm[];
    typedef T Tile1[kTile + 1];
    typedef T TileZ[kZzWin + 1];
    Tile1* sz1 = (Tile1*)u8sm;                       // [col][row]
    Tile1* sx1 = sz1 + kTile;
    TileZ* sz2 = (TileZ*)(sx1 + kTile);              // [col][q - (r0 - 1)]
    TileZ* sx2 = sz2 + kTile;
    TileZ* sz3 = sx2 + kTile;
    TileZ* sx3 = sz3 + kTile;
    const int64_t R = A.rows, W = A.cols;
    const int H = (int)R;
    const int64_t tiles_c = (W + kTile - 1) / kTile;
    const int64_t r0 = (blockIdx.x / tiles_c) * kTile;
    const int64_t c0 = (blockIdx.x % tiles_c) * kTile;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
#pragma unroll
    for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
        const int64_t c = c0 + cc, r = r0 + tx;
        if (c < W && r < R) {
            sz1[cc][tx] = A.s[1][c * R + r];
            sx1[cc][tx] = A.x[1][c * R + r];
        }
    }
    for (int idx = threadIdx.x; idx < kTile * kZzWin; idx += kUpdThreads) {
        const int cc = idx / kZzWin, qq = idx - cc * kZzWin;
        const int64_t c = c0 + cc, q = r0 - 1 + qq;
        if (c < W && q >= 0 && q < R) {
            sz2[cc][qq] = A.s[2][c * R + q];
            sx2[cc][qq] = A.x[2][c * R + q];
            sz3[cc][qq] = A.s[3][c * R + q];
            sx3[cc][qq] = A.x[3][c * R + q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int rr = ty; rr < kTile; rr += kUpdThreads / kTile) {
        const int64_t r = r0 + rr, c = c0 + tx;
        if (r >= R || c >= W) continue;
        const int64_t g = r * W + c;
        const int q2 = zz_row((int)r, (int)c, H, 2) - (int)(r0 - 1);
        const int q3 = zz_row((int)r, (int)c, H, 3) - (int)(r0 - 1);
        const T wg = A.w[g];
        const T sv[4] = {A.s[0][g], sz1[tx][rr], sz2[tx][q2], sz3[tx][q3]};
        const T xv[4] = {A.x[0][g], sx1[tx][rr], sx2[tx][q2], sx3[tx][q3]};
        T yk[4];
        T ysum = T(0), ssum = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            yk[k] = sv[k] - xv[k];
            ysum += yk[k];
            ssum += sv[k];
        }
        if (A.check) A.xout[g] = wg - ysum;
        if constexpr (MODE != UPD_EVAL) {
            T cc;
            if constexpr (MODE == UPD_AAR) cc = (wg - T(2) * ysum + ssum) / T(4);
            else cc = (wg - ysum) / T(4);
            A.s[0][g] = yk[0] + cc;
            sz1[tx][rr] = yk[1] + cc;
            sz2[tx][q2] = yk[2] + cc;
            sz3[tx][q3] = yk[3] + cc;
        }
    }
    if constexpr (MODE != UPD_EVAL) {
        __syncthreads();
#pragma unroll
        for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
            const int64_t c = c0 + cc, r = r0 + tx;
            if (c < W && r < R) A.s[1][c * R + r] = sz1[cc][tx];
        }
        for (int idx = threadIdx.x; idx < kTile * kZzWin; idx += kUpdThreads) {
            const int cc = idx / kZzWin, qq = idx - cc * kZzWin;
            const int64_t c = c0 + cc, q = r0 - 1 + qq;
            if (c >= W || q < 0 || q >= R) continue;
            const int64_t v2 = zz_row((int)q, (int)c, H, 2), v3 = zz_row((int)q, (int)c, H, 3);
            if (v2 >= r0 && v2 < r0 + kTile) A.s[2][c * R + q] = sz2[cc][qq];
            if (v3 >= r0 && v3 < r0 + kTile) A.s[3][c * R + q] = sz3[cc][qq];
        }
    }
}

template <typename T>
static size_t update8_smem()
{
    return sizeof(T) * (2 * (size_t)kTile * (kTile + 1) + 4 * (size_t)kTile * (kZzWin + 1));
}

template <typename T>
cudaError_t launch_update8(int mode, const Update8Args<T>& A, cudaStream_t s)
{
    const int64_t tiles = ((A.rows + kTile - 1) / kTile) * ((A.cols + kTile - 1) / kTile);
    if (tiles == 0) return cudaSuccess;
    const size_t smem = update8_smem<T>();
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(update8_kernel<T, UPD_AAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(update8_kernel<T, UPD_AP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(update8_kernel<T, UPD_EVAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    if (mode == UPD_AAR) update8_kernel<T, UPD_AAR><<<(unsigned)tiles, kUpdThreads, smem, s>>>(A);
    else if (mode == UPD_AP) update8_kernel<T, UPD_AP><<<(unsigned)tiles, kUpdThreads, smem, s>>>(A);
    else update8_kernel<T, UPD_EVAL><<<(unsigned)tiles, kUpdThreads, smem, s>>>(A);
    return cudaGetLastError();
}

// The dual-iterate passes of an 8-connected grid (BCD, FISTA, primal), staged
// like update8_kernel: the row block over the tile's rows, the two path blocks
// over the windows [r0 - 1, r0 + 33) of path positions; outputs in the path
// layouts go back only at positions whose vertex lies in the tile.
template <typename T, int KIND>
__global__ void __launch_bounds__(kUpdThreads) prep8_kernel(Prep8Args<T> A)
{
    extern __shared__ __align__(16) unsigned char p8sm[];
    typedef T Tile1[kTile + 1];
    typedef T TileZ[kZzWin + 1];
    Tile1* sy1 = (Tile1*)p8sm;
    Tile1* sp1 = sy1 + kTile;
    TileZ* sy2 = (TileZ*)(sp1 + kTile);
    TileZ* sp2 = sy2 + kTile;
    TileZ* sy3 = sp2 + kTile;
    TileZ* sp3 = sy3 + kTile;
    const int64_t R = A.rows, W = A.cols;
    const int H = (int)R;
    const int64_t tiles_c = (W + kTile - 1) / kTile;
    const int64_t r0 = (blockIdx.x / tiles_c) * kTile;
    const int64_t c0 = (blockIdx.x % tiles_c) * kTile;
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    constexpr bool PREV = KIND == PREP8_FISTA;
#pragma unroll
    for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
        const int64_t c = c0 + cc, r = r0 + tx;
        if (c < W && r < R) {
            sy1[cc][tx] = A.y[1][c * R + r];
            if (PREV) sp1[cc][tx] = A.p[1][c * R + r];
        }
    }
    for (int idx = threadIdx.x; idx < kTile * kZzWin; idx += kUpdThreads) {
        const int cc = idx / kZzWin, qq = idx - cc * kZzWin;
        const int64_t c = c0 + cc, q = r0 - 1 + qq;
        if (c < W && q >= 0 && q < R) {
            sy2[cc][qq] = A.y[2][c * R + q];
            sy3[cc][qq] = A.y[3][c * R + q];
            if (PREV) {
                sp2[cc][qq] = A.p[2][c * R + q];
                sp3[cc][qq] = A.p[3][c * R + q];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int rr = ty; rr < kTile; rr += kUpdThreads / kTile) {
        const int64_t r = r0 + rr, c = c0 + tx;
        if (r >= R || c >= W) continue;
        const int64_t g = r * W + c;
        const int q2 = zz_row((int)r, (int)c, H, 2) - (int)(r0 - 1);
        const int q3 = zz_row((int)r, (int)c, H, 3) - (int)(r0 - 1);
        const T yv[4] = {A.y[0][g], sy1[tx][rr], sy2[tx][q2], sy3[tx][q3]};
        const T wg = A.w[g];
        if constexpr (KIND == PREP8_PRIMAL) {
            T v = wg;
#pragma unroll
            for (int j = 0; j < 4; ++j) v -= yv[j];
            A.xout[g] = v;
        } else if constexpr (KIND == PREP8_BCD) {
            T v = wg;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j != A.k) v -= yv[j];
            // the result goes to block k's layout: staged in that block's buffer
            if (A.k == 0) A.out[0][g] = v;
            else if (A.k == 1) sp1[tx][rr] = v;
            else if (A.k == 2) sp2[tx][q2] = v;
            else sp3[tx][q3] = v;
        } else {
            const T pv[4] = {A.p[0][g], sp1[tx][rr], sp2[tx][q2], sp3[tx][q3]};
            T u[4];
            T usum = T(0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                u[j] = yv[j] + A.beta * (yv[j] - pv[j]);
                usum += u[j];
            }
            const T corr = (wg - usum) / T(4);
            A.out[0][g] = u[0] + corr;
            sp1[tx][rr] = u[1] + corr;         // every thread has read its own p values above
            sp2[tx][q2] = u[2] + corr;
            sp3[tx][q3] = u[3] + corr;
        }
    }
    if constexpr (KIND != PREP8_PRIMAL) {
        __syncthreads();
        const bool all = KIND == PREP8_FISTA;
        if (all || A.k == 1) {
#pragma unroll
            for (int cc = ty; cc < kTile; cc += kUpdThreads / kTile) {
                const int64_t c = c0 + cc, r = r0 + tx;
                if (c < W && r < R) A.out[1][c * R + r] = sp1[cc][tx];
            }
        }
        if (all || A.k >= 2) {
            for (int idx = threadIdx.x; idx < kTile * kZzWin; idx += kUpdThreads) {
                const int cc = idx / kZzWin, qq = idx - cc * kZzWin;
                const int64_t c = c0 + cc, q = r0 - 1 + qq;
                if (c >= W || q < 0 || q >= R) continue;
                const int64_t v2 = zz_row((int)q, (int)c, H, 2), v3 = zz_row((int)q, (int)c, H, 3);
                if ((all || A.k == 2) && v2 >= r0 && v2 < r0 + kTile) A.out[2][c * R + q] = sp2[cc][qq];
                if ((all || A.k == 3) && v3 >= r0 && v3 < r0 + kTile) A.out[3][c * R + q] = sp3[cc][qq];
            }
        }
    }
}

template <typename T>
cudaError_t launch_prep8(int kind, const Prep8Args<T>& A, cudaStream_t s)
{
    const int64_t tiles = ((A.rows + kTile - 1) / kTile) * ((A.cols + kTile - 1) / kTile);
    if (tiles == 0) return cudaSuccess;
    const size_t smem = update8_smem<T>();
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(prep8_kernel<T, PREP8_BCD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(prep8_kernel<T, PREP8_PRIMAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(prep8_kernel<T, PREP8_FISTA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    if (kind == PREP8_BCD) prep8_kernel<T, PREP8_BCD><<<(unsigned)tiles, kUpdThreads, smem, s>>>(A);
    else if (kind == PREP8_PRIMAL) prep8_kernel<T, PREP8_PRIMAL><<<(unsigned)tiles, kUpdThreads, smem, s>>>(A);
    else prep8_kernel<T, PREP8_FISTA><<<(unsigned)tiles, kUpdThreads, smem, s>>>(A);
    return cudaGetLastError();
}

#define TVCUT_SCAN_INST(T)                                                                  \
    template cudaError_t launch_prep8<T>(int, const Prep8Args<T>&, cudaStream_t);           \
    template cudaError_t launch_update8<T>(int, const Update8Args<T>&, cudaStream_t);       \
    template cudaError_t launch_zz_weights<T>(const T*, const T*, T*, int, int, int, cudaStream_t); \
    template cudaError_t launch_zz_relayout<T>(const T*, T*, int, int, int, bool, cudaStream_t); \
    template cudaError_t launch_fista_prepare<T>(const FistaArgs<T>&, cudaStream_t);        \
    template cudaError_t launch_bcd_prepare<T>(const UpdateArgs<T>&, int, cudaStream_t);    \
    template cudaError_t launch_scan<T>(ScanArgs<T>, cudaStream_t);                         \
    template cudaError_t launch_pad_weights<T>(const ScanAxis<T>&, T*, cudaStream_t);        \
    template cudaError_t launch_update<T>(int, const UpdateArgs<T>&, cudaStream_t);         \
    template cudaError_t launch_transpose<T>(const T*, T*, int64_t, int64_t, cudaStream_t);
TVCUT_SCAN_INST(float)
TVCUT_SCAN_INST(double)

}  // namespace tvcut
