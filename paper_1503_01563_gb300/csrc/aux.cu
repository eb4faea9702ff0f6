// Per-check evaluation of the primal x (Sec. 2.2-2.3): labels l = [x > alpha],
// the cut energy E(l) of problem (D) (FP64 and exact int64), the discrete
// lower bound sum_i min(y_i - w_i, 0) with y = w - x, the total variation
// f(x) and y^T x for the TV duality gap.  Sums run in FP64/int64 with a fixed
// grid and a fixed two-level reduction order, so results are reproducible
// bit for bit.  Also: input conversion/validation, cold and warm starts.
#include "tvcut_internal.cuh"

#include <math.h>

#include <type_traits>

namespace tvcut {

__device__ __forceinline__ void partial_add(CheckPartial& a, const CheckPartial& b)
{
    a.energy += b.energy;
    a.lb += b.lb;
    a.tv += b.tv;
    a.ytx += b.ytx;
    a.xabs = fmax(a.xabs, b.xabs);
    a.energy_i += b.energy_i;
    a.n1 += b.n1;
}

__device__ __forceinline__ CheckPartial partial_shfl_down(const CheckPartial& p, int d)
{
    CheckPartial q;
    q.energy = __shfl_down_sync(0xffffffffu, p.energy, d);
    q.lb = __shfl_down_sync(0xffffffffu, p.lb, d);
    q.tv = __shfl_down_sync(0xffffffffu, p.tv, d);
    q.ytx = __shfl_down_sync(0xffffffffu, p.ytx, d);
    q.xabs = __shfl_down_sync(0xffffffffu, p.xabs, d);
    q.energy_i = __shfl_down_sync(0xffffffffu, p.energy_i, d);
    q.n1 = __shfl_down_sync(0xffffffffu, p.n1, d);
    q.pad = 0;
    return q;
}

// Block-wide reduction in a fixed order; result valid in thread 0.
template <int THREADS>
__device__ CheckPartial block_reduce(CheckPartial p)
{
    __shared__ CheckPartial warp_sums[THREADS / 32];
    for (int d = 16; d > 0; d >>= 1) partial_add(p, partial_shfl_down(p, d));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_sums[wid] = p;
    __syncthreads();
    if (wid == 0) {
        CheckPartial q = lane < THREADS / 32 ? warp_sums[lane] : CheckPartial{0, 0, 0, 0, 0, 0, 0, 0};
        for (int d = 16; d > 0; d >>= 1) partial_add(q, partial_shfl_down(q, d));
        p = q;
    }
    return p;
}

// One pass over the grid: labels at the plain threshold, the FP64 sums of the
// check (discrete lower bound, y^T x, f(x), max |x|) and the energies of the
// level sets [x > levels[q]] (Sec. 2.1: every level set of a solution of the
// relaxation solves (D)) for an ascending ladder that contains the plain
// threshold.  The level index q(v) = #{levels below v} gives a value's labels
// at every level at once ([v > level_j] = [j < q(v)]), so an edge's ends
// differ exactly on the levels in [min q, max q) and a vertex is labelled 1 on
// the levels below its q.  Both are intervals, kept as per-thread difference
// arrays: entry 0, the common case, lives in a register, and the other
// entries are touched only by values inside the ladder's range.  Each warp
// walks whole rows of the last axis, so a vertex's neighbours along every
// axis are at fixed offsets (+1 from the next lane, +W, +H*W).  Integer
// problems accumulate level energies in exact int64, others in FP64; every
// sum has a fixed order.
template <typename T, bool EXACT>
__global__ void __launch_bounds__(kCheckThreads) check_kernel(CheckArgs<T> A)
{
    using Acc = typename std::conditional<EXACT, long long, double>::type;
    CheckPartial acc{0, 0, 0, 0, 0, 0, 0, 0};
    Acc dE[kMaxLevels + 1];
    int dN[kMaxLevels + 1];
    for (int q = 0; q <= kMaxLevels; ++q) { dE[q] = 0; dN[q] = 0; }
    Acc e0 = 0;
    long long n0 = 0;
    T xabs = T(0);
    const int L = A.nlevels;
    const int nd = A.ndim;
    const int64_t W = A.dims[nd - 1];
    const int64_t R = A.n / W;
    const int64_t Hm = nd >= 2 ? A.dims[nd - 2] : 1;          // axis nd-2 extent
    const int64_t D0 = nd == 3 ? A.dims[0] : 1;
    const T thr = A.threshold;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * kCheckThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kCheckThreads) >> 5;
    auto level_of = [&](T v) {
        int q = 0;
#pragma unroll
        for (int j = 0; j < kMaxLevels; ++j) q += (j < L && v > A.levels[j]) ? 1 : 0;
        return q;
    };
    auto to_acc = [](T v) -> Acc {
        if constexpr (!EXACT) return (Acc)v;
        else if constexpr (sizeof(T) == 4) return (Acc)__float2int_rn((float)v);   // |v| <= 2^24
        else return (Acc)llrint((double)v);
    };
    auto add_edge = [&](double xd, T x2, int q1, int q2, T ae) {
        acc.tv += (double)ae * fabs(xd - (double)x2);
        const int lo = min(q1, q2), hi = max(q1, q2);
        if (lo != hi) {
            const Acc av = to_acc(ae);
            if (lo == 0) e0 += av;
            else dE[lo] += av;
            if (hi < L) dE[hi] -= av;
        }
    };
    for (int64_t r = warp; r < R; r += nwarps) {
        const int64_t h = r % Hm;                 // coordinate along axis nd-2
        const int64_t d = r / Hm;                 // coordinate along axis 0 (3D)
        for (int64_t cb = 0; cb < W; cb += 32) {  // uniform in the warp (shuffles)
            const int64_t c = cb + lane;
            const bool in = c < W;
            const int64_t g = r * W + c;
            const T xg = in ? A.x[g] : T(0);
            const int qg = level_of(xg);
            T xr = __shfl_down_sync(0xffffffffu, xg, 1);
            int qr = __shfl_down_sync(0xffffffffu, qg, 1);
            if (!in) continue;
            if (lane == 31 && c + 1 < W) {
                xr = A.x[g + 1];
                qr = level_of(xr);
            }
            A.labels[g] = (uint8_t)(xg > thr);
            const T wt = A.w[g];
            const double wg = (double)wt;
            const double xd = (double)xg;
            acc.lb -= fmax(xd, 0.0);
            acc.ytx += (wg - xd) * xd;
            xabs = fmax(xabs, fabs(xg));
            if (qg > 0) {
                const Acc wv = to_acc(wt);
                e0 -= wv;
                n0 += 1;
                if (qg < L) {
                    dE[qg] += wv;
                    dN[qg] -= 1;
                }
            }
            // last axis: edge (c, c+1) of row r
            if (c + 1 < W) {
                const int64_t ai = A.last_transposed ? c * R + r : r * (W - 1) + c;
                add_edge(xd, xr, qg, qr, A.a[nd - 1][ai]);
            }
            // axis nd-2: edge (h, h+1); compact index ((d*(Hm-1) + h) * W + c)
            if (h + 1 < Hm) {
                const T x2 = A.x[g + W];
                add_edge(xd, x2, qg, level_of(x2), A.a[nd - 2][(d * (Hm - 1) + h) * W + c]);
            }
            // axis 0 of a 3D grid: edge (d, d+1); compact index = g
            if (nd == 3 && d + 1 < D0) {
                const T x2 = A.x[g + Hm * W];
                add_edge(xd, x2, qg, level_of(x2), A.a[0][g]);
            }
            // 8-connected 2D grid: edges to (h+1, c+1) and (h+1, c-1)
            if (A.adiag && h + 1 < Hm) {
                if (c + 1 < W) {
                    const T x2 = A.x[g + W + 1];
                    add_edge(xd, x2, qg, level_of(x2), A.adiag[h * (W - 1) + c]);
                }
                if (c >= 1) {
                    const T x2 = A.x[g + W - 1];
                    add_edge(xd, x2, qg, level_of(x2), A.aanti[h * (W - 1) + c - 1]);
                }
            }
        }
    }
    acc.xabs = (double)xabs;
    CheckPartial rsum = block_reduce<kCheckThreads>(acc);
    if (threadIdx.x == 0) A.partials[blockIdx.x] = rsum;
    // level partials: prefix sums of the difference arrays, one level at a
    // time, each summed over the block in a fixed order
    __shared__ double se[kCheckThreads / 32];
    __shared__ long long sei[kCheckThreads / 32];
    __shared__ long long sn[kCheckThreads / 32];
    const int wid = threadIdx.x >> 5;
    Acc run = e0;
    long long rn = n0;
    for (int q = 0; q < L; ++q) {
        if (q > 0) {
            run += dE[q];
            rn += dN[q];
        }
        Acc a = run;
        long long c = rn;
        for (int dd = 16; dd > 0; dd >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, dd);
            c += __shfl_down_sync(0xffffffffu, c, dd);
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
            for (int w = 0; w < kCheckThreads / 32; ++w) {
                if (EXACT) tb += sei[w];
                else ta += se[w];
                tc += sn[w];
            }
            if (EXACT) ta = (double)tb;
            A.level_partials[blockIdx.x].energy[q] = ta;
            A.level_partials[blockIdx.x].energy_i[q] = tb;
            A.level_partials[blockIdx.x].n1[q] = tc;
        }
    }
}

__global__ void __launch_bounds__(256) finalize_kernel(const CheckPartial* partials, int count,
                                                       DevStatus* status)
{
    CheckPartial acc{0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < count; i += blockDim.x) partial_add(acc, partials[i]);
    CheckPartial r = block_reduce<256>(acc);
    if (threadIdx.x == 0) status->sum = r;
}

__global__ void __launch_bounds__(32) level_finalize_kernel(const LevelPartial* partials, int count, int L,
                                                            DevStatus* status)
{
    const int j = threadIdx.x;
    if (j >= L) return;
    double a = 0.0;
    long long b = 0, c = 0;
    for (int i = 0; i < count; ++i) {
        a += partials[i].energy[j];
        b += partials[i].energy_i[j];
        c += partials[i].n1[j];
    }
    status->levels.energy[j] = a;
    status->levels.energy_i[j] = b;
    status->levels.n1[j] = c;
}

template <typename T>
cudaError_t launch_check(const CheckArgs<T>& A, bool exact, DevStatus* status, cudaStream_t s)
{
    if (exact) check_kernel<T, true><<<kCheckBlocks, kCheckThreads, 0, s>>>(A);
    else check_kernel<T, false><<<kCheckBlocks, kCheckThreads, 0, s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finalize_kernel<<<1, 256, 0, s>>>(A.partials, kCheckBlocks, status);
    e = cudaGetLastError();
    if (e != cudaSuccess || A.nlevels <= 0) return e;
    level_finalize_kernel<<<1, 32, 0, s>>>(A.level_partials, kCheckBlocks, A.nlevels, status);
    return cudaGetLastError();
}

template <typename T>
__global__ void labels_kernel(const T* x, T thr, uint8_t* labels, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        labels[i] = (uint8_t)(x[i] > thr);
}

template <typename T>
cudaError_t launch_labels(const T* x, T threshold, uint8_t* labels, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    labels_kernel<T><<<kCheckBlocks, kCheckThreads, 0, s>>>(x, threshold, labels, n);
    return cudaGetLastError();
}

// ---- conversion of caller inputs into the iterate type, with validation ----

template <typename S, typename T>
__global__ void convert_kernel(const S* src, T* dst, int64_t n, bool nonneg, int* flags, unsigned* absmax_bits)
{
    int f = 0;
    float amax = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const S v = src[i];
        const double d = (double)v;
        if (!isfinite(d)) f |= FLAG_NONFINITE;
        if (nonneg && d < 0.0) f |= FLAG_NEGATIVE;
        const T t = (T)v;
        if constexpr (std::is_integral<S>::value) {
            if ((double)t != d) f |= FLAG_INEXACT;  // integer input not exact in T
        }
        dst[i] = t;
        amax = fmaxf(amax, fabsf((float)d));
    }
    if (f) atomicOr(flags, f);
    if (isfinite(amax) && amax > 0.f) atomicMax(absmax_bits, __float_as_uint(amax));   // order-preserving for >= 0
}

template <typename T>
cudaError_t launch_convert(const void* src, int src_dtype, T* dst, int64_t n, bool nonneg,
                           int* flags, unsigned* absmax_bits, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
    switch (src_dtype) {
    case TVCUT_I32: convert_kernel<int32_t, T><<<blocks, threads, 0, s>>>((const int32_t*)src, dst, n, nonneg, flags, absmax_bits); break;
    case TVCUT_F32: convert_kernel<float, T><<<blocks, threads, 0, s>>>((const float*)src, dst, n, nonneg, flags, absmax_bits); break;
    case TVCUT_F64: convert_kernel<double, T><<<blocks, threads, 0, s>>>((const double*)src, dst, n, nonneg, flags, absmax_bits); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S, typename D>
__global__ void copy_convert_kernel(const S* src, D* dst, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = (D)src[i];
}

template <typename T>
cudaError_t launch_convert_out(const T* src, void* dst, int dst_dtype, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
    switch (dst_dtype) {
    case TVCUT_F32: copy_convert_kernel<T, float><<<blocks, threads, 0, s>>>(src, (float*)dst, n); break;
    case TVCUT_F64: copy_convert_kernel<T, double><<<blocks, threads, 0, s>>>(src, (double*)dst, n); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// AP cold start: lambda_k = w / r, the projection of 0 onto L (Eq. dualA).
template <typename T>
__global__ void cold_ap_kernel(const T* w, T* state, int r, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T c = w[i] / T(r);
        for (int k = 0; k < r; ++k) state[k * n + i] = c;
    }
}

template <typename T>
cudaError_t launch_cold_ap(const T* w, T* state, int r, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
    cold_ap_kernel<T><<<blocks, threads, 0, s>>>(w, state, r, n);
    return cudaGetLastError();
}

// Warm start from a predicted primal: s_k = (w - xhat)/r + tau * xhat.
template <typename T>
__global__ void warmstart_kernel(const T* w, const float* xhat, float tau, T* state, int r, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T xh = (T)xhat[i];
        const T c = (w[i] - xh) / T(r) + T(tau) * xh;
        for (int k = 0; k < r; ++k) state[k * n + i] = c;
    }
}

template <typename T>
cudaError_t launch_warmstart(const T* w, const float* xhat, float tau, T* state, int r, int64_t n,
                             cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
    warmstart_kernel<T><<<blocks, threads, 0, s>>>(w, xhat, tau, state, r, n);
    return cudaGetLastError();
}


// ---- rigorous discrete lower bound (Sec. 2.2) --------------------------------
//
// Any y in K gives E* >= sum_i min(y_i - w_i, 0).  A block dual y_k computed
// in the iterate's precision is only close to K_k, so the bound is taken from
// a point that is exactly in it: along each chain the edge multipliers are
// the running sums u_j = y_0 + ... + y_j of the block dual (the string
// offsets of the taut string, Sec. 3.2), clamped to [-a_j, a_j], with
// u = 0 after the chain's last element; the chain's contribution to vertex j
// is then u_j - u_{j-1}, which lies in K_k by construction.  Sums run in
// FP64, the blocks are added one launch at a time into an FP64 vertex array
// (each vertex lies on one chain of every block), and the bound is reduced
// per CTA in a fixed order.

template <typename T>
__global__ void __launch_bounds__(256) certify_block_kernel(CertifyArgs<T> A)
{
    const ScanAxis<T>& X = A.X;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < X.nchains;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = X.transposed ? 0 : c / X.inner, q = X.transposed ? 0 : c - o * X.inner;
        double run = 0.0, uprev = 0.0;
        for (int j = 0; j < X.m; ++j) {
            const int64_t e = X.transposed ? (int64_t)j * X.nchains + c : o * X.m * X.inner + q + (int64_t)j * X.inner;
            run += (double)X.v[e];
            double u = 0.0;
            if (j < X.m - 1) {
                const int64_t wi = X.transposed ? e : o * (X.m - 1) * X.inner + q + (int64_t)j * X.inner;
                const double a = (double)X.a[wi];
                u = run < -a ? -a : (run > a ? a : run);
            }
            const double yh = u - uprev;
            uprev = u;
            int64_t nat = e;
            if (A.layout == 1) nat = c * X.m + j;
            else if (A.layout >= 2) nat = (int64_t)zz_row((int)c, j, (int)A.H, A.layout) * A.W + j;
            A.Y[nat] = A.first ? yh : A.Y[nat] + yh;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kCheckThreads) certify_lb_kernel(const double* __restrict__ Y, const T* __restrict__ w,
                                                                  int64_t n, double* __restrict__ part)
{
    double s = 0.0, mag = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double y = Y[i];
        const double d = y - (double)w[i];
        const double m = d < 0.0 ? d : 0.0;
        s += m;
        mag += fabs(m) + fabs(y);
    }
    __shared__ double sh[2][kCheckThreads];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = mag;
    __syncthreads();
    for (int h = kCheckThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + h];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sh[0][0];
        part[2 * blockIdx.x + 1] = sh[1][0];
    }
}

template <typename T>
cudaError_t launch_certify_block(const CertifyArgs<T>& A, cudaStream_t s)
{
    if (A.X.nchains <= 0 || A.X.m <= 0) return cudaSuccess;
    const int64_t want = (A.X.nchains + 255) / 256;
    const int blocks = (int)(want < 8192 ? want : 8192);
    certify_block_kernel<T><<<blocks, 256, 0, s>>>(A);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_certify_lb(const double* Y, const T* w, int64_t n, double* part, cudaStream_t s)
{
    certify_lb_kernel<T><<<kCheckBlocks, kCheckThreads, 0, s>>>(Y, w, n, part);
    return cudaGetLastError();
}

#define TVCUT_INST(T)                                                                          \
    template cudaError_t launch_check<T>(const CheckArgs<T>&, bool, DevStatus*, cudaStream_t);  \
    template cudaError_t launch_convert<T>(const void*, int, T*, int64_t, bool, int*, unsigned*, cudaStream_t); \
    template cudaError_t launch_labels<T>(const T*, T, uint8_t*, int64_t, cudaStream_t);         \
    template cudaError_t launch_convert_out<T>(const T*, void*, int, int64_t, cudaStream_t);    \
    template cudaError_t launch_cold_ap<T>(const T*, T*, int, int64_t, cudaStream_t);           \
    template cudaError_t launch_warmstart<T>(const T*, const float*, float, T*, int, int64_t, cudaStream_t); \
    template cudaError_t launch_certify_block<T>(const CertifyArgs<T>&, cudaStream_t);             \
    template cudaError_t launch_certify_lb<T>(const double*, const T*, int64_t, double*, cudaStream_t);
TVCUT_INST(float)
TVCUT_INST(double)

}  // namespace tvcut
