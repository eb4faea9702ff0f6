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

template <typename T>
__global__ void __launch_bounds__(kCheckThreads) check_kernel(CheckArgs<T> A)
{
    CheckPartial acc{0, 0, 0, 0, 0, 0, 0, 0};
    const T thr = A.threshold;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < A.n; g += stride) {
        const T xg = A.x[g];
        const bool l = xg > thr;
        A.labels[g] = (uint8_t)l;
        const double wg = (double)A.w[g];
        const double xd = (double)xg;
        acc.lb -= fmax(xd, 0.0);
        acc.ytx += (wg - xd) * xd;
        acc.xabs = fmax(acc.xabs, fabs(xd));
        if (l) {
            acc.energy -= wg;
            acc.energy_i -= llrint(wg);
            acc.n1 += 1;
        }
        for (int k = 0; k < A.ndim; ++k) {
            const int64_t inner = A.inner[k];
            const int64_t mk = A.dims[k];
            const int64_t o = g / (mk * inner);
            const int64_t j = (g - o * mk * inner) / inner;
            if (j + 1 < mk) {
                const T x2 = A.x[g + inner];
                // compact index; the last axis' weights may be stored transposed
                const int64_t ai = (A.last_transposed && k == A.ndim - 1) ? j * (A.n / mk) + o : g - o * inner;
                const double ae = (double)A.a[k][ai];
                acc.tv += ae * fabs(xd - (double)x2);
                if (l != (x2 > thr)) {
                    acc.energy += ae;
                    acc.energy_i += llrint(ae);
                }
            }
        }
    }
    CheckPartial r = block_reduce<kCheckThreads>(acc);
    if (threadIdx.x == 0) A.partials[blockIdx.x] = r;
}

__global__ void __launch_bounds__(256) finalize_kernel(const CheckPartial* partials, int count,
                                                       DevStatus* status)
{
    CheckPartial acc{0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < count; i += blockDim.x) partial_add(acc, partials[i]);
    CheckPartial r = block_reduce<256>(acc);
    if (threadIdx.x == 0) status->sum = r;
}

// Energies of the level sets [x > levels[j]] (Sec. 2.1: every level set of a
// solution of the relaxation solves (D)), FP64 and exact int64.
template <typename T>
__global__ void __launch_bounds__(kCheckThreads) level_kernel(CheckArgs<T> A)
{
    double e[kMaxLevels];
    long long ei[kMaxLevels];
    int n1[kMaxLevels];
#pragma unroll
    for (int j = 0; j < kMaxLevels; ++j) { e[j] = 0.0; ei[j] = 0; n1[j] = 0; }
    const int L = A.nlevels;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < A.n; g += stride) {
        const T xg = A.x[g];
        const double wg = (double)A.w[g];
        const long long wi = llrint(wg);
#pragma unroll
        for (int j = 0; j < kMaxLevels; ++j)
            if (j < L && xg > A.levels[j]) { e[j] -= wg; ei[j] -= wi; n1[j] += 1; }
        for (int k = 0; k < A.ndim; ++k) {
            const int64_t inner = A.inner[k];
            const int64_t mk = A.dims[k];
            const int64_t o = g / (mk * inner);
            const int64_t jj = (g - o * mk * inner) / inner;
            if (jj + 1 < mk) {
                const T x2 = A.x[g + inner];
                const int64_t ai = (A.last_transposed && k == A.ndim - 1) ? jj * (A.n / mk) + o : g - o * inner;
                const double ae = (double)A.a[k][ai];
                const long long aei = llrint(ae);
#pragma unroll
                for (int j = 0; j < kMaxLevels; ++j)
                    if (j < L && ((xg > A.levels[j]) != (x2 > A.levels[j]))) { e[j] += ae; ei[j] += aei; }
            }
        }
    }
    // block reduction, one level at a time, fixed order
    __shared__ double se[kCheckThreads / 32];
    __shared__ long long sei[kCheckThreads / 32];
    __shared__ long long sn[kCheckThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMaxLevels; ++j) {
        if (j >= L) break;
        double a = e[j];
        long long b = ei[j];
        long long c = n1[j];
        for (int d = 16; d > 0; d >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, d);
            b += __shfl_down_sync(0xffffffffu, b, d);
            c += __shfl_down_sync(0xffffffffu, c, d);
        }
        if (lane == 0) { se[wid] = a; sei[wid] = b; sn[wid] = c; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double ta = 0.0;
            long long tb = 0, tc = 0;
            for (int w = 0; w < kCheckThreads / 32; ++w) { ta += se[w]; tb += sei[w]; tc += sn[w]; }
            A.level_partials[blockIdx.x].energy[j] = ta;
            A.level_partials[blockIdx.x].energy_i[j] = tb;
            A.level_partials[blockIdx.x].n1[j] = tc;
        }
        __syncthreads();
    }
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
cudaError_t launch_check(const CheckArgs<T>& A, DevStatus* status, cudaStream_t s)
{
    check_kernel<T><<<kCheckBlocks, kCheckThreads, 0, s>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    finalize_kernel<<<1, 256, 0, s>>>(A.partials, kCheckBlocks, status);
    e = cudaGetLastError();
    if (e != cudaSuccess || A.nlevels <= 0) return e;
    level_kernel<T><<<kCheckBlocks, kCheckThreads, 0, s>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
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

#define TVCUT_INST(T)                                                                          \
    template cudaError_t launch_check<T>(const CheckArgs<T>&, DevStatus*, cudaStream_t);        \
    template cudaError_t launch_convert<T>(const void*, int, T*, int64_t, bool, int*, unsigned*, cudaStream_t); \
    template cudaError_t launch_labels<T>(const T*, T, uint8_t*, int64_t, cudaStream_t);         \
    template cudaError_t launch_convert_out<T>(const T*, void*, int, int64_t, cudaStream_t);    \
    template cudaError_t launch_cold_ap<T>(const T*, T*, int, int64_t, cudaStream_t);           \
    template cudaError_t launch_warmstart<T>(const T*, const float*, float, T*, int, int64_t, cudaStream_t);
TVCUT_INST(float)
TVCUT_INST(double)

}  // namespace tvcut
