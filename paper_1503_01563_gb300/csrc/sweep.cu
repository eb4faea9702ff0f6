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

template <typename T, int MODE>
static cudaError_t launch_mode(const SweepArgs<T>& A, cudaStream_t s)
{
    if (A.g.nchains <= 0 || A.g.m <= 0) return cudaSuccess;
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
