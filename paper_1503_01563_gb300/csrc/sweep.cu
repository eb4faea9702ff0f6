// Chain sweeps: the exact weighted 1D-TV prox of every chain of one grid axis
// (Sec. 3.2), with the per-vertex update of the product-space method fused
// into the pass that produces each chain's result (Sec. 4.2-4.3, Eq. dualA).
//
// One thread owns one chain.  The prox is the taut string through the tube
// of half-width a around the running sums of v, written in local form so that
// no running sum of the (possibly large, drifting) input is ever formed:
// from a segment start s with incoming multiplier u0 (u_{s-1}), a common value
// t for x_s..x_i gives the multiplier u_i = u0 + sum_{j=s..i} (t - v_j), which
// must stay in [-a_i, a_i] (and reach 0 at the chain end).  The thread keeps
// the largest (th) and smallest (tl) feasible t together with u_i for both;
// when th is too small for the lower bound at i, the string has to bend up at
// the point ih that last limited th -- the segment [s, ih] is final with value
// th and the multiplier there is +a_ih; symmetrically for tl.  The scan then
// restarts after the bend.  Each finished segment is emitted element by
// element through the sweep's epilogue.
#include "tvcut_internal.cuh"

namespace tvcut {

ChainGeom chain_geom(int ndim, const int64_t* dims, int axis)
{
    ChainGeom g;
    g.outer = 1;
    g.inner = 1;
    for (int d = 0; d < axis; ++d) g.outer *= dims[d];
    for (int d = axis + 1; d < ndim; ++d) g.inner *= dims[d];
    g.m = (int)dims[axis];
    g.nchains = g.outer * g.inner;
    return g;
}

template <typename T, int MODE>
__device__ __forceinline__ void epilogue(const SweepArgs<T>& A, int64_t g, T v, T t)
{
    const T y = v - t;
    if constexpr (MODE == MODE_PROJ) {
        A.out[g] = y;
    } else if constexpr (MODE == MODE_PROX) {
        A.out[g] = t;
    } else if constexpr (MODE == MODE_AAR_FIRST) {
        A.P[g] = A.w[g] + v - T(2) * y;
        A.out[g] = y;
    } else if constexpr (MODE == MODE_AAR_MID) {
        A.P[g] = A.P[g] + v - T(2) * y;
        A.out[g] = y;
    } else if constexpr (MODE == MODE_AAR_LAST) {
        // z_k <- y_k + (w - 2 sum_j y_j + sum_j z_j)/r  (Eq. 3 with Eq. dualA)
        const T c = (A.P[g] + v - T(2) * y) / T(A.r);
        T ysum = y;
        for (int k = 0; k < A.r - 1; ++k) {
            const T yk = A.Z[k][g];
            ysum += yk;
            A.Z[k][g] = yk + c;
        }
        A.Z[A.r - 1][g] = y + c;
        if (A.check) A.x[g] = A.w[g] - ysum;
    } else if constexpr (MODE == MODE_AP_FIRST) {
        A.P[g] = A.w[g] - y;
        A.out[g] = y;
    } else if constexpr (MODE == MODE_AP_MID) {
        A.P[g] = A.P[g] - y;
        A.out[g] = y;
    } else if constexpr (MODE == MODE_AP_LAST) {
        // lambda_k <- y_k + (w - sum_j y_j)/r  (Pi_L, Eq. dualA)
        const T xg = A.P[g] - y;
        const T c = xg / T(A.r);
        for (int k = 0; k < A.r - 1; ++k) A.Z[k][g] = A.Z[k][g] + c;
        A.Z[A.r - 1][g] = y + c;
        if (A.check) A.x[g] = xg;
    } else if constexpr (MODE == MODE_EVAL_FIRST) {
        A.P[g] = A.w[g] - y;
    } else if constexpr (MODE == MODE_EVAL_MID) {
        A.P[g] = A.P[g] - y;
    } else if constexpr (MODE == MODE_EVAL_LAST) {
        A.x[g] = A.P[g] - y;
    }
}

// Thread-per-chain sweep reading the chain straight from global memory
// (consecutive threads own consecutive chains, so for every axis but the
// last the warp's loads of one step are contiguous).  The in-place modes
// write a position only once its segment is final; the scan never reads a
// position again after that, so v may alias the outputs.
template <typename T, int MODE>
__global__ void __launch_bounds__(128) sweep_global_kernel(SweepArgs<T> A)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= A.g.nchains) return;
    const int64_t inner = A.g.inner;
    const int m = A.g.m;
    const int64_t o = c / inner;
    const int64_t q = c - o * inner;
    const int64_t base = o * (int64_t)m * inner + q;
    const T* v = A.v + base;
    const T* a = A.a + (o * (int64_t)(m - 1) * inner + q);

    auto emit = [&](int from, int to, T t) {
        for (int j = from; j <= to; ++j) {
            const int64_t off = (int64_t)j * inner;
            epilogue<T, MODE>(A, base + off, v[off], t);
        }
    };

    int s = 0, i = 0, ih = 0, il = 0;
    T u0 = T(0), th = T(0), tl = T(0), uh = T(0), ul = T(0), ah = T(0), al = T(0);
    for (;;) {
        const T vi = v[(int64_t)i * inner];
        const T Ai = (i < m - 1) ? a[(int64_t)i * inner] : T(0);
        if (i == s) {
            th = vi + Ai - u0;
            tl = vi - Ai - u0;
            uh = Ai;
            ul = -Ai;
            ih = il = i;
            ah = al = Ai;
        } else {
            uh += th - vi;
            ul += tl - vi;
            if (uh < -Ai) {            // bend up at ih
                emit(s, ih, th);
                u0 = ah;
                s = i = ih + 1;
                continue;
            }
            if (ul > Ai) {             // bend down at il
                emit(s, il, tl);
                u0 = -al;
                s = i = il + 1;
                continue;
            }
            const T len = T(i - s + 1);
            if (uh > Ai) {
                th -= (uh - Ai) / len;
                uh = Ai;
                ih = i;
                ah = Ai;
            }
            if (ul < -Ai) {
                tl += (-Ai - ul) / len;
                ul = -Ai;
                il = i;
                al = Ai;
            }
        }
        if (i == m - 1) {
            emit(s, m - 1, th);
            break;
        }
        ++i;
    }
}

// ---- tiled sweep ------------------------------------------------------------
//
// One CTA owns NC chains of one axis (a "tile") and stages them whole into
// shared memory, element-major ([j][lane], padded pitch NC+1 so that both the
// transposing loads of row chains and the per-lane scan are bank-conflict
// free).  Three phases separated by barriers:
//   L: all threads issue asynchronous 4/8-byte copies (cp.async) of the chain
//      inputs v and the weights a, coalesced along whichever index is
//      contiguous in global memory, with every copy in flight at once;
//   S: warp 0 runs the taut-string scan of its lane's chain out of shared
//      memory; each final segment value is written over the weights of the
//      same positions, which the scan never reads again;
//   E: all threads apply the sweep's epilogue element by element from
//      shared memory (y = v - x), coalesced like phase L.
// Several CTAs per SM overlap their phases.

constexpr int kTileThreads = 256;

__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem)
{
    if constexpr (sizeof(T) == 8) cp_async_8(smem, gmem);
    else cp_async_4(smem, gmem);
}

// Taut-string scan of one chain held in shared memory at sv[j*LD], sa[j*LD];
// final segment values overwrite sa.
template <typename T, int LD>
__device__ __forceinline__ void scan_smem(int m, const T* sv, T* sa)
{
    int s = 0, i = 0, ih = 0, il = 0;
    T u0 = T(0), th = T(0), tl = T(0), uh = T(0), ul = T(0), ah = T(0), al = T(0);
    for (;;) {
        const T vi = sv[i * LD];
        const T Ai = (i < m - 1) ? sa[i * LD] : T(0);
        if (i == s) {
            th = vi + Ai - u0;
            tl = vi - Ai - u0;
            uh = Ai;
            ul = -Ai;
            ih = il = i;
            ah = al = Ai;
        } else {
            uh += th - vi;
            ul += tl - vi;
            if (uh < -Ai) {
                for (int j = s; j <= ih; ++j) sa[j * LD] = th;
                u0 = ah;
                s = i = ih + 1;
                continue;
            }
            if (ul > Ai) {
                for (int j = s; j <= il; ++j) sa[j * LD] = tl;
                u0 = -al;
                s = i = il + 1;
                continue;
            }
            const T len = T(i - s + 1);
            if (uh > Ai) {
                th -= (uh - Ai) / len;
                uh = Ai;
                ih = i;
                ah = Ai;
            }
            if (ul < -Ai) {
                tl += (-Ai - ul) / len;
                ul = -Ai;
                il = i;
                al = Ai;
            }
        }
        if (i == m - 1) {
            for (int j = s; j <= m - 1; ++j) sa[j * LD] = th;
            break;
        }
        ++i;
    }
}

template <typename T, int MODE, int NC, bool ROWS>
__global__ void __launch_bounds__(kTileThreads) sweep_tile_kernel(SweepArgs<T> A)
{
    constexpr int LD = NC + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sv = (T*)smem_raw;
    const int m = A.g.m;
    T* sa = sv + (size_t)m * LD;
    const int64_t inner = A.g.inner;

    // tile -> first chain; lanes beyond `nvalid` are padding
    int64_t vbase, abase;     // global offsets of (lane 0, j = 0)
    int nvalid;
    if constexpr (ROWS) {
        const int64_t c0 = (int64_t)blockIdx.x * NC;
        nvalid = (int)min((int64_t)NC, A.g.nchains - c0);
        vbase = c0 * m;
        abase = c0 * (m - 1);
    } else {
        const int64_t tiles_per_o = (inner + NC - 1) / NC;
        const int64_t o = blockIdx.x / tiles_per_o;
        const int64_t q0 = (blockIdx.x - o * tiles_per_o) * NC;
        nvalid = (int)min((int64_t)NC, inner - q0);
        vbase = o * (int64_t)m * inner + q0;
        abase = o * (int64_t)(m - 1) * inner + q0;
    }
    const int total = m * NC;

    // ---- L: stage v and a ----
    for (int idx = threadIdx.x; idx < total; idx += kTileThreads) {
        int j, lane;
        if constexpr (ROWS) { lane = idx / m; j = idx - lane * m; }
        else { j = idx / NC; lane = idx - j * NC; }
        T* dv = sv + j * LD + lane;
        T* da = sa + j * LD + lane;
        if (lane < nvalid) {
            const int64_t gv = ROWS ? vbase + (int64_t)lane * m + j : vbase + (int64_t)j * inner + lane;
            cp_async_elem(dv, A.v + gv);
            if (j < m - 1) {
                const int64_t ga = ROWS ? abase + (int64_t)lane * (m - 1) + j : abase + (int64_t)j * inner + lane;
                cp_async_elem(da, A.a + ga);
            }
        } else {
            *dv = T(0);
            *da = T(0);
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // ---- S: one lane per chain ----
    if (threadIdx.x < NC && (int)threadIdx.x < nvalid) scan_smem<T, LD>(m, sv + threadIdx.x, sa + threadIdx.x);
    __syncthreads();

    // ---- E: fused epilogue ----
#pragma unroll 4
    for (int idx = threadIdx.x; idx < total; idx += kTileThreads) {
        int j, lane;
        if constexpr (ROWS) { lane = idx / m; j = idx - lane * m; }
        else { j = idx / NC; lane = idx - j * NC; }
        if (lane >= nvalid) continue;
        const int64_t g = ROWS ? vbase + (int64_t)lane * m + j : vbase + (int64_t)j * inner + lane;
        epilogue<T, MODE>(A, g, sv[j * LD + lane], sa[j * LD + lane]);
    }
}

template <typename T>
static size_t tile_smem_bytes(int m, int nc)
{
    return (size_t)2 * (size_t)m * (size_t)(nc + 1) * sizeof(T);
}

constexpr size_t kTileSmemLimit = 200 * 1024;

template <typename T, int MODE, int NC, bool ROWS>
static cudaError_t launch_tile(const SweepArgs<T>& A, cudaStream_t s)
{
    const size_t smem = tile_smem_bytes<T>(A.g.m, NC);
    static bool attr_set[64] = {};        // per instantiation and device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(sweep_tile_kernel<T, MODE, NC, ROWS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemLimit);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    int64_t tiles;
    if (ROWS) tiles = (A.g.nchains + NC - 1) / NC;
    else tiles = A.g.outer * ((A.g.inner + NC - 1) / NC);
    sweep_tile_kernel<T, MODE, NC, ROWS><<<(unsigned)tiles, kTileThreads, smem, s>>>(A);
    return cudaGetLastError();
}

template <typename T, int MODE, int NC>
static cudaError_t launch_tile_nc(const SweepArgs<T>& A, cudaStream_t s)
{
    if (A.g.inner == 1) return launch_tile<T, MODE, NC, true>(A, s);
    return launch_tile<T, MODE, NC, false>(A, s);
}

template <typename T, int MODE>
static cudaError_t launch_mode(const SweepArgs<T>& A, cudaStream_t s)
{
    if (A.g.nchains <= 0 || A.g.m <= 0) return cudaSuccess;
    const int mp = A.mapping;
    if (mp == 3 && tile_smem_bytes<T>(A.g.m, 32) <= kTileSmemLimit) return launch_tile_nc<T, MODE, 32>(A, s);
    if (mp == 2 && tile_smem_bytes<T>(A.g.m, 16) <= kTileSmemLimit) return launch_tile_nc<T, MODE, 16>(A, s);
    if (mp == 1 && tile_smem_bytes<T>(A.g.m, 8) <= kTileSmemLimit) return launch_tile_nc<T, MODE, 8>(A, s);
    if (mp < 0) {
        // widest tile that fits the shared-memory budget; the thread-per-chain
        // global-memory kernel takes chains too long for any tile
        if (tile_smem_bytes<T>(A.g.m, 32) <= kTileSmemLimit / 2 && A.g.nchains >= 32 * 152)
            return launch_tile_nc<T, MODE, 32>(A, s);
        if (tile_smem_bytes<T>(A.g.m, 16) <= kTileSmemLimit)
            return launch_tile_nc<T, MODE, 16>(A, s);
        if (tile_smem_bytes<T>(A.g.m, 8) <= kTileSmemLimit)
            return launch_tile_nc<T, MODE, 8>(A, s);
    }
    const int threads = 128;
    const int64_t blocks = (A.g.nchains + threads - 1) / threads;
    sweep_global_kernel<T, MODE><<<(unsigned)blocks, threads, 0, s>>>(A);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep(int mode, const SweepArgs<T>& A, cudaStream_t s)
{
    switch (mode) {
    case MODE_PROJ: return launch_mode<T, MODE_PROJ>(A, s);
    case MODE_PROX: return launch_mode<T, MODE_PROX>(A, s);
    case MODE_AAR_FIRST: return launch_mode<T, MODE_AAR_FIRST>(A, s);
    case MODE_AAR_MID: return launch_mode<T, MODE_AAR_MID>(A, s);
    case MODE_AAR_LAST: return launch_mode<T, MODE_AAR_LAST>(A, s);
    case MODE_AP_FIRST: return launch_mode<T, MODE_AP_FIRST>(A, s);
    case MODE_AP_MID: return launch_mode<T, MODE_AP_MID>(A, s);
    case MODE_AP_LAST: return launch_mode<T, MODE_AP_LAST>(A, s);
    case MODE_EVAL_FIRST: return launch_mode<T, MODE_EVAL_FIRST>(A, s);
    case MODE_EVAL_MID: return launch_mode<T, MODE_EVAL_MID>(A, s);
    case MODE_EVAL_LAST: return launch_mode<T, MODE_EVAL_LAST>(A, s);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_sweep<float>(int, const SweepArgs<float>&, cudaStream_t);
template cudaError_t launch_sweep<double>(int, const SweepArgs<double>&, cudaStream_t);

}  // namespace tvcut
