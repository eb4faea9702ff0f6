// Iteration kernels of the product-space methods (Sec. 4.2-4.3).
//
// One iteration = one scan launch + one update launch:
//
//   scan:   x_k = prox_{f_k}(s_k) on every chain of every block k at once.
//           The blocks' projections are independent in the product space
//           (Sec. 4.2: Pi_K splits into the Pi_{K_k}), so all axes share one
//           launch; one thread owns one chain.  The prox is the taut string of
//           Sec. 3.2 in local form (see scan_chain).  Each block's state is
//           stored so that consecutive chains are consecutive in memory
//           ("chain-major"): the natural row-major layout already is for
//           every axis but the last, and the last axis' block (rows) is kept
//           transposed.  A warp's loads of one step are thus one 128-byte
//           line.
//
//   update: per vertex, y_k = s_k - x_k and
//             AAR (Eq. 3 with Eq. dualA): s_k <- y_k + (w - 2 sum y + sum s)/r
//             AP  (Sec. 4.2):             s_k <- y_k + (w - sum y)/r
//           and, on check iterations, the primal x = w - sum_k y_k (Sec. 2.3).
//           Elementwise and coalesced; the transposed row block goes through
//           32x32 shared-memory tiles.
#include "tvcut_internal.cuh"

namespace tvcut {

constexpr int kScanThreads = 128;

// Taut-string scan of one chain: element j of v at v[j*stride], weight of
// edge (j, j+1) at a[j*stride]; writes x[j*stride] = prox value.  From a
// segment start s with incoming multiplier u0, a common value t on s..i gives
// u_i = u0 + sum_{j=s..i} (t - v_j), which must stay in [-a_i, a_i] (and be 0
// at the chain end).  th/tl are the largest/smallest feasible t and uh/ul the
// matching u_i; when the feasible set empties, the segment ends at the point
// that last limited the violated bound (the string bends there) and the scan
// resumes after it.  Pointers advance by `stride` per element; only a rescan
// recomputes them.
template <typename T>
__device__ __forceinline__ T div_len(T num, int len)
{
    if constexpr (sizeof(T) == 4) return num * __frcp_rn((float)len);   // 1/len correctly rounded
    else return num / (T)len;
}

template <typename T>
__device__ __forceinline__ void scan_chain(int m, const T* __restrict__ v, const T* __restrict__ a,
                                           T* __restrict__ x, int64_t stride)
{
    int s = 0, i = 0, ih = 0, il = 0;
    T u0 = T(0), th = T(0), tl = T(0), uh = T(0), ul = T(0), ah = T(0), al = T(0);
    const T* pv = v;
    const T* pa = a;
    T* px = x;                                   // next element to write
    for (;;) {
        const T vi = *pv;
        const T Ai = (i < m - 1) ? *pa : T(0);
        bool init = (i == s);
        if (!init) {
            uh += th - vi;
            ul += tl - vi;
            const bool bhi = uh < -Ai;
            const bool blo = !bhi && ul > Ai;
            if (bhi || blo) {                        // the string bends at e
                const int e = bhi ? ih : il;
                const T t = bhi ? th : tl;
                u0 = bhi ? ah : -al;
                for (int j = s; j <= e; ++j, px += stride) *px = t;
                s = e + 1;
                if (s < i) {                         // rescan from the bend
                    i = s;
                    pv = v + (int64_t)s * stride;
                    pa = a + (int64_t)s * stride;
                    continue;
                }
                init = true;                         // the new segment starts at i
            } else {
                const int len = i - s + 1;
                if (uh > Ai) {
                    th -= div_len<T>(uh - Ai, len);
                    uh = Ai;
                    ih = i;
                    ah = Ai;
                }
                if (ul < -Ai) {
                    tl += div_len<T>(-Ai - ul, len);
                    ul = -Ai;
                    il = i;
                    al = Ai;
                }
            }
        }
        if (init) {
            th = vi + Ai - u0;
            tl = vi - Ai - u0;
            uh = Ai;
            ul = -Ai;
            ih = il = i;
            ah = al = Ai;
        }
        if (i == m - 1) {
            for (int j = s; j <= m - 1; ++j, px += stride) *px = th;
            break;
        }
        ++i;
        pv += stride;
        pa += stride;
    }
}

template <typename T>
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
    scan_chain<T>(X.m, X.v + base, X.a + abase, X.x + base, stride);
}

template <typename T>
cudaError_t launch_scan(ScanArgs<T> A, cudaStream_t s)
{
    int64_t blocks = 0;
    for (int k = 0; k < A.naxes; ++k) {
        A.ax[k].block_begin = (unsigned)blocks;
        blocks += (A.ax[k].nchains + kScanThreads - 1) / kScanThreads;
    }
    if (blocks == 0) return cudaSuccess;
    scan_kernel<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(A);
    return cudaGetLastError();
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

template <typename T>
cudaError_t launch_update(int mode, const UpdateArgs<T>& A, cudaStream_t s)
{
    const int64_t tiles = ((A.rows + kTile - 1) / kTile) * ((A.cols + kTile - 1) / kTile);
    if (tiles == 0) return cudaSuccess;
#define TVCUT_UPD(M)                                                                       \
    (A.r == 3 ? (update_kernel<T, M, 3><<<(unsigned)tiles, kUpdThreads, 0, s>>>(A), 0)      \
              : (update_kernel<T, M, 2><<<(unsigned)tiles, kUpdThreads, 0, s>>>(A), 0))
    if (A.r != 2 && A.r != 3) return cudaErrorInvalidValue;
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

#define TVCUT_SCAN_INST(T)                                                                  \
    template cudaError_t launch_scan<T>(ScanArgs<T>, cudaStream_t);                         \
    template cudaError_t launch_update<T>(int, const UpdateArgs<T>&, cudaStream_t);         \
    template cudaError_t launch_transpose<T>(const T*, T*, int64_t, int64_t, cudaStream_t);
TVCUT_SCAN_INST(float)
TVCUT_SCAN_INST(double)

}  // namespace tvcut
