// Iteration kernels of the methods of Sec. 4.
//
// AAR and AP: one iteration = one scan launch + one update launch:
//
//   scan:   x_k = prox_{f_k}(s_k) on every chain of every block k at once.
//           The blocks' projections are independent in the product space
//           (Sec. 4.2: Pi_K splits into the Pi_{K_k}), so all axes share one
//           launch; a thread (reading weights padded to the state layout, so
//           that each element is loaded one step ahead), or a group of 4-32
//           lanes (lanescan.cu), owns one chain.  The prox is the taut string of Sec. 3.2
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
#include "tvcut_internal.cuh"
#include "taut_string.cuh"

namespace tvcut {

constexpr int kScanThreads = 128;

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
        for (int k = 0; k < A.naxes; ++k) {
            if (A.ax[k].m >= 2 && funnel_scan_fits<T>(A.ax[k].m)) fun.ax[fun.naxes++] = A.ax[k];
            else rest.ax[rest.naxes++] = A.ax[k];
        }
        if (fun.naxes) {
            cudaError_t e = launch_funnel_scan<T>(fun, s);
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
        bool warp = X.m >= 64 && total <= 98304 && lane_scan_fits<T>(X.m);
        if (A.force == 1) warp = false;
        if (A.force >= 2) warp = X.m >= 2 && lane_scan_fits<T>(X.m);
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
    if (wrp.naxes) return launch_lane_scan<T>(wrp, s);
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
