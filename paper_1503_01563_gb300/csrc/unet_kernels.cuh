// Kernels of the learned warm start: a U-Net with BF16 weights and
// activations and FP32 accumulation.  Convolutions are implicit GEMMs on the
// tensor cores (mma.sync m16n8k16, BF16 inputs, FP32 accumulators); the rest
// (pooling, upsampling, concatenation, loss, Adam) is elementwise.
//
// Layouts: activations NHWC BF16 with the channel count a multiple of 16;
// a 3x3 convolution's weights are [9][Cout][Cin] (tap k = 3*ky + kx, input
// pixel (y + ky - 1, x + kx - 1), zero outside the image).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "conv_args.cuh"

namespace tvcut {
namespace nn {

constexpr int BM = 64;      // pixels per CTA tile
constexpr int BN = 64;      // output channels per CTA tile
constexpr int BK = 16;      // reduction slice (one tap x 16 channels)
constexpr int SROW = 24;    // padded smem row (BF16) of a 16-wide slice: conflict-free fragments

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp's 16 x 64 block of the CTA tile: rows [16w, 16w+16) of As (pixels
// x k) against all 64 columns of Bs (channels x k).
__device__ __forceinline__ void warp_tile_mma(const __nv_bfloat16 (*As)[SROW], const __nv_bfloat16 (*Bs)[SROW],
                                              float acc[8][4], int warp, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const int r0 = warp * 16 + g;
    uint32_t a[4];
    a[0] = *(const uint32_t*)&As[r0][2 * t];
    a[1] = *(const uint32_t*)&As[r0 + 8][2 * t];
    a[2] = *(const uint32_t*)&As[r0][2 * t + 8];
    a[3] = *(const uint32_t*)&As[r0 + 8][2 * t + 8];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        uint32_t b[2];
        b[0] = *(const uint32_t*)&Bs[nt * 8 + g][2 * t];
        b[1] = *(const uint32_t*)&Bs[nt * 8 + g][2 * t + 8];
        mma_bf16(acc[nt], a, b);
    }
}



// out[p][co] = act(bias[co] + sum_k sum_ci in[p + off_k][ci] * wt[k][co][ci])
//
// CTA tile: 128 pixels x 64 output channels, 8 warps (16 pixels x 64 channels
// each).  The reduction runs over "slices" (one tap, 16 input channels); two
// slices form a stage, staged into shared memory by 16-byte cp.async copies
// (zero-filled outside the image) in a two-deep pipeline, so the next stage
// loads while the tensor cores work on the current one.
constexpr int FBM = 128;
constexpr int FTHREADS = 256;

__device__ __forceinline__ void cp16(void* smem, const void* gmem, bool valid)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;                  // 0 bytes read: zero fill
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(FTHREADS) conv3x3_fwd_kernel(ConvArgs A)
{
    __shared__ __align__(16) __nv_bfloat16 As[2][2][FBM][SROW];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][2][BN][SROW];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t P = (int64_t)A.N * A.H * A.W;
    const int64_t p0 = (int64_t)blockIdx.x * FBM;
    const int n0 = blockIdx.y * BN;
    const int cslices = A.Cin / BK;
    const int nslices = 9 * cslices;
    const int nstages = (nslices + 1) / 2;
    // A loads: 128 pixels x 2 slices x 2 halves = 512 16-byte copies, 2 per thread
    int apix[2], ay[2], ax[2];
    int64_t an[2];
    bool aval[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int idx = tid + r * FTHREADS;
        apix[r] = idx >> 2;
        const int64_t p = p0 + apix[r];
        aval[r] = p < P;
        const int64_t pp = aval[r] ? p : 0;
        ax[r] = (int)(pp % A.W);
        const int64_t q = pp / A.W;
        ay[r] = (int)(q % A.H);
        an[r] = q / A.H;
    }
    auto load_stage = [&](int t, int buf) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * FTHREADS;
            const int j = (idx >> 1) & 1, h = idx & 1;
            const int sl = 2 * t + j;
            const int k = sl / cslices, c0 = (sl - k * cslices) * BK;
            const int yy = ay[r] + k / 3 - 1, xx = ax[r] + k % 3 - 1;
            const bool ok = aval[r] && sl < nslices && yy >= 0 && yy < A.H && xx >= 0 && xx < A.W;
            const __nv_bfloat16* src = ok ? A.in + ((an[r] * A.H + yy) * A.W + xx) * A.Cin + c0 + 8 * h : A.in;
            cp16(&As[buf][j][apix[r]][8 * h], src, ok);
        }
        {   // B: 64 channels x 2 slices x 2 halves = 256 copies, 1 per thread
            const int co = tid >> 2, j = (tid >> 1) & 1, h = tid & 1;
            const int sl = 2 * t + j;
            const int k = sl / cslices, c0 = (sl - k * cslices) * BK;
            const bool ok = sl < nslices && n0 + co < A.Cout;
            const __nv_bfloat16* src = ok ? A.wt + ((int64_t)k * A.Cout + n0 + co) * A.Cin + c0 + 8 * h : A.wt;
            cp16(&Bs[buf][j][co][8 * h], src, ok);
        }
        cp_commit();
    };
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    load_stage(0, 0);
    for (int t = 0; t < nstages; ++t) {
        const int buf = t & 1;
        if (t + 1 < nstages) {
            load_stage(t + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        warp_tile_mma(As[buf][0], Bs[buf][0], acc, warp, lane);
        if (2 * t + 1 < nslices) warp_tile_mma(As[buf][1], Bs[buf][1], acc, warp, lane);
        __syncthreads();
    }
    // epilogue: rows warp*16 + g (+8), columns nt*8 + 2t (+1)
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int64_t p = p0 + warp * 16 + g + 8 * half;
        if (p >= P) continue;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int co = n0 + nt * 8 + 2 * tq + j;
                if (co >= A.Cout) continue;
                float v = acc[nt][2 * half + j];
                if (A.bias) v += A.bias[co];
                if (A.relu) v = fmaxf(v, 0.f);
                const int64_t o = p * A.CoutStride + co;
                if (A.mask && !(__bfloat162float(A.mask[o]) > 0.f)) v = 0.f;
                A.out[o] = __float2bfloat16(v);
                if (A.out_f32) A.out_f32[p * A.Cout + co] = v;
            }
        }
    }
}

struct WgradArgs {
    const __nv_bfloat16* in;     // N x H x W x Cin   (layer input)
    const __nv_bfloat16* dout;   // N x H x W x Cout  (gradient of the layer output, after the ReLU mask)
    float* dw;                   // 9 x Cout x Cin, accumulated
    float* part;                 // nullptr: add into dw atomically; else one 9 x Cout x Cin slice per pixel
                                 // chunk (written, not added), summed in chunk order afterwards
    int N, H, W, Cin, Cout;
    int64_t pix_per_cta;
};

// dw[k][co][ci] += sum_p dout[p][co] * in[p + off_k][ci]: a GEMM with the
// pixels as the reduction, split across CTAs (blockIdx.z = tap x pixel chunk).
__global__ void __launch_bounds__(128) conv3x3_wgrad_kernel(WgradArgs A)
{
    __shared__ __align__(16) __nv_bfloat16 As[BM][SROW];   // [co][p]
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][SROW];   // [ci][p]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t P = (int64_t)A.N * A.H * A.W;
    const int co0 = blockIdx.x * BM, ci0 = blockIdx.y * BN;
    const int nchunks = (int)((P + A.pix_per_cta - 1) / A.pix_per_cta);
    const int k = blockIdx.z / nchunks;
    const int64_t pbeg = (int64_t)(blockIdx.z % nchunks) * A.pix_per_cta;
    const int64_t pend = min(P, pbeg + A.pix_per_cta);
    const int dy = k / 3 - 1, dx = k % 3 - 1;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    // loads: 16 pixels x 64 channels per operand; thread -> (pixel tid>>3, 8 channels)
    const int lp = tid >> 3, lc = (tid & 7) * 8;
    for (int64_t pb = pbeg; pb < pend; pb += BK) {
        const int64_t p = pb + lp;
        __nv_bfloat16 va[8], vb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) va[j] = vb[j] = __float2bfloat16(0.f);
        if (p < pend) {
            if (co0 + lc < A.Cout) *(uint4*)va = *(const uint4*)(A.dout + p * A.Cout + co0 + lc);
            const int x = (int)(p % A.W);
            const int64_t q = p / A.W;
            const int y = (int)(q % A.H);
            const int64_t n = q / A.H;
            const int yy = y + dy, xx = x + dx;
            if (yy >= 0 && yy < A.H && xx >= 0 && xx < A.W && ci0 + lc < A.Cin)
                *(uint4*)vb = *(const uint4*)(A.in + ((n * A.H + yy) * A.W + xx) * A.Cin + ci0 + lc);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            As[lc + j][lp] = va[j];
            Bs[lc + j][lp] = vb[j];
        }
        __syncthreads();
        warp_tile_mma(As, Bs, acc, warp, lane);
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int co = co0 + warp * 16 + g + 8 * half;
        if (co >= A.Cout) continue;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int ci = ci0 + nt * 8 + 2 * t + j;
                if (ci >= A.Cin) continue;
                const int64_t idx = ((int64_t)k * A.Cout + co) * A.Cin + ci;
                if (!A.part) atomicAdd(&A.dw[idx], acc[nt][2 * half + j]);
                else if (nchunks == 1) A.dw[idx] += acc[nt][2 * half + j];      // the only writer of idx
                else A.part[(int64_t)(blockIdx.z % nchunks) * 9 * A.Cout * A.Cin + idx] = acc[nt][2 * half + j];
            }
    }
}

}  // namespace nn
}  // namespace tvcut
