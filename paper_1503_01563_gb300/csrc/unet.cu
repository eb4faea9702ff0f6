// Learned warm start: a U-Net that maps a grid problem (unary, vertical and
// horizontal edge weights) to the per-block dual variables y_k of the
// product-space iteration (Sec. 4), used as its starting point (Sec. 4.4:
// warm starts reuse the dual variables).  BF16 weights and activations, FP32
// accumulation and FP32 master weights; forward, backward and Adam run in
// the kernels of unet_kernels.cuh and below.
//
// Architecture (base channels C, 4 levels; every conv 3x3 + ReLU unless noted):
//   e1 = conv(conv(x; 16->C); C->C)            x = input padded to 16 channels
//   e2 = conv(conv(pool(e1); C->2C); 2C->2C)   pool = 2x2 average
//   e3 = conv(conv(pool(e2); 2C->4C); 4C->4C)
//   e4 = conv(conv(pool(e3); 4C->8C); 8C->8C)
//   d3 = conv(conv([conv(up(e4); 8C->4C), e3]; 8C->4C); 4C->4C)   up = nearest 2x
//   d2 = conv(conv([conv(up(d3); 4C->2C), e2]; 4C->2C); 2C->2C)
//   d1 = conv(conv([conv(up(d2); 2C->C), e1]; 2C->C); C->C)
//   out = conv(d1; C->16) without ReLU; channels 0 and 1 are the prediction.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tvcut.h"
#include "tvcut_internal.cuh"
#include "unet_kernels.cuh"

using namespace tvcut::nn;
typedef __nv_bfloat16 bf16;

namespace {

// Elementwise kernels work on 8 channels (16 bytes) per thread: every
// channel count is a multiple of 16 and every tensor is its own allocation.
__device__ __forceinline__ void unpack8(const uint4& u, float* f)
{
    const __nv_bfloat162* h = (const __nv_bfloat162*)&u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 t = __bfloat1622float2(h[k]);
        f[2 * k] = t.x;
        f[2 * k + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 pack8(const float* f)
{
    uint4 u;
    __nv_bfloat162* h = (__nv_bfloat162*)&u;
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    return u;
}

#define GRID_STRIDE(i, n) \
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// x[p] = [in[p][0..2], 0 x 13] (one pixel per thread)
__global__ void input_pack_kernel(const float* in, bf16* x, int64_t P)
{
    GRID_STRIDE(p, P) {
        float f[8] = {in[p * 3], in[p * 3 + 1], in[p * 3 + 2], 0.f, 0.f, 0.f, 0.f, 0.f};
        const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        uint4* o = (uint4*)(x + p * 16);
        o[0] = pack8(f);
        o[1] = pack8(z);
    }
}

// The network's input straight from a handle's device problem: pixel (r, c)
// gets [w, a_down, a_right] / s, then zeros to 16 channels, in BF16 (a_down =
// the vertical edge (r, c)-(r+1, c), a_right = the horizontal edge
// (r, c)-(r, c+1), 0 on the last row / column).  Each feature is rounded
// from FP64 to FP32 and then to BF16, the path of an FP32 feature array.
template <typename T>
__global__ void features_pack_kernel(const T* __restrict__ w, const T* __restrict__ a0, const T* __restrict__ a1,
                                     int a1_transposed, int H, int W, double s, bf16* __restrict__ x)
{
    GRID_STRIDE(p, (int64_t)H * W) {
        const int r = (int)(p / W), c = (int)(p - (int64_t)r * W);
        float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        f[0] = (float)((double)w[p] / s);
        if (r < H - 1) f[1] = (float)((double)a0[p] / s);
        if (c < W - 1)
            f[2] = (float)((double)(a1_transposed ? a1[(int64_t)c * H + r] : a1[(int64_t)r * (W - 1) + c]) / s);
        uint4* o = (uint4*)(x + p * 16);
        o[0] = pack8(f);
        o[1] = pack8(z);
    }
}

// Predicted block duals y_k = output channel k times s (an FP32 product),
// written into a handle's state blocks in their own layouts.
template <typename T>
__global__ void state_from_output_kernel(const float* __restrict__ o16, int H, int W, float s, T* __restrict__ s0,
                                         T* __restrict__ s1, int s1_transposed)
{
    GRID_STRIDE(p, (int64_t)H * W) {
        const int r = (int)(p / W), c = (int)(p - (int64_t)r * W);
        s0[p] = (T)(o16[p * 16] * s);
        s1[s1_transposed ? (int64_t)c * H + r : p] = (T)(o16[p * 16 + 1] * s);
    }
}

// 2x2 average: out (H/2 x W/2, C channels) from in (H x W, pixel stride Cs); one
// 8-channel group per thread
__global__ void pool_fwd_kernel(const bf16* in, bf16* out, int N, int H, int W, int C, int Cs)
{
    const int Ho = H / 2, Wo = W / 2, C8 = C / 8;
    const int64_t total = (int64_t)N * Ho * Wo * C8;
    GRID_STRIDE(i, total) {
        const int g = (int)(i % C8);
        const int64_t po = i / C8;
        const int x = (int)(po % Wo);
        const int64_t q = po / Wo;
        const int y = (int)(q % Ho);
        const int64_t n = q / Ho;
        const int64_t b = ((n * H + 2 * y) * W + 2 * x) * Cs + 8 * g;
        const int64_t rs = (int64_t)W * Cs;
        float f0[8], f1[8], f2[8], f3[8], r[8];
        unpack8(*(const uint4*)(in + b), f0);
        unpack8(*(const uint4*)(in + b + Cs), f1);
        unpack8(*(const uint4*)(in + b + rs), f2);
        unpack8(*(const uint4*)(in + b + rs + Cs), f3);
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = 0.25f * (f0[k] + f1[k] + f2[k] + f3[k]);
        *(uint4*)(out + po * C + 8 * g) = pack8(r);
    }
}

// g_in (H x W) += g_out (H/2 x W/2) / 4 spread over each 2x2 block
__global__ void pool_bwd_kernel(const bf16* gout, bf16* gin, int N, int H, int W, int C)
{
    const int C8 = C / 8;
    const int64_t total = (int64_t)N * H * W * C8;
    GRID_STRIDE(i, total) {
        const int g = (int)(i % C8);
        const int64_t p = i / C8;
        const int x = (int)(p % W);
        const int64_t q = p / W;
        const int y = (int)(q % H);
        const int64_t n = q / H;
        float a[8], b[8];
        unpack8(*(const uint4*)(gout + ((n * (H / 2) + y / 2) * (W / 2) + x / 2) * C + 8 * g), b);
        bf16* d = gin + p * C + 8 * g;
        unpack8(*(const uint4*)d, a);
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = a[k] + 0.25f * b[k];
        *(uint4*)d = pack8(a);
    }
}

__global__ void up_fwd_kernel(const bf16* in, bf16* out, int N, int H, int W, int C)   // H, W: output size
{
    const int C8 = C / 8;
    const int64_t total = (int64_t)N * H * W * C8;
    GRID_STRIDE(i, total) {
        const int g = (int)(i % C8);
        const int64_t p = i / C8;
        const int x = (int)(p % W);
        const int64_t q = p / W;
        const int y = (int)(q % H);
        const int64_t n = q / H;
        *(uint4*)(out + p * C + 8 * g) =
            *(const uint4*)(in + ((n * (H / 2) + y / 2) * (W / 2) + x / 2) * C + 8 * g);
    }
}

__global__ void up_bwd_kernel(const bf16* gout, bf16* gin, int N, int H, int W, int C)  // H, W: input (coarse) size
{
    const int C8 = C / 8;
    const int64_t total = (int64_t)N * H * W * C8;
    GRID_STRIDE(i, total) {
        const int g = (int)(i % C8);
        const int64_t p = i / C8;
        const int x = (int)(p % W);
        const int64_t q = p / W;
        const int y = (int)(q % H);
        const int64_t n = q / H;
        const int64_t b = ((n * 2 * H + 2 * y) * 2 * W + 2 * x) * C + 8 * g;
        const int64_t rs = (int64_t)2 * W * C;
        float f0[8], f1[8], f2[8], f3[8], r[8];
        unpack8(*(const uint4*)(gout + b), f0);
        unpack8(*(const uint4*)(gout + b + C), f1);
        unpack8(*(const uint4*)(gout + b + rs), f2);
        unpack8(*(const uint4*)(gout + b + rs + C), f3);
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = f0[k] + f1[k] + f2[k] + f3[k];
        *(uint4*)(gin + p * C + 8 * g) = pack8(r);
    }
}


// ga = g[:, :Ca] (overwrite); gb += g[:, Ca:]
__global__ void concat_bwd_kernel(const bf16* g, bf16* ga, bf16* gb, int64_t P, int Ca, int Cb)
{
    const int C8 = (Ca + Cb) / 8, A8 = Ca / 8;
    GRID_STRIDE(i, P * C8) {
        const int64_t p = i / C8;
        const int q = (int)(i - p * C8);
        const uint4 v = *(const uint4*)(g + 8 * i);
        if (q < A8) {
            *(uint4*)(ga + p * Ca + 8 * q) = v;
        } else {
            bf16* d = gb + p * Cb + 8 * (q - A8);
            float x[8], y[8];
            unpack8(*(const uint4*)d, x);
            unpack8(v, y);
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = x[k] + y[k];
            *(uint4*)d = pack8(x);
        }
    }
}

// g *= (y > 0): gradient at a ReLU output -> gradient at its input (n % 8 == 0)
// g (C channels per pixel) is zeroed where y (the activation, pixel stride Cs) is not positive
__global__ void relu_mask_kernel(bf16* g, const bf16* y, int64_t n, int C, int Cs)
{
    GRID_STRIDE(i, n / 8) {
        float gv[8], yv[8];
        const int64_t e = 8 * i, p = e / C;
        unpack8(*(const uint4*)(g + e), gv);
        unpack8(*(const uint4*)(y + p * Cs + (e - p * C)), yv);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (!(yv[k] > 0.f)) gv[k] = 0.f;
        *(uint4*)(g + 8 * i) = pack8(gv);
    }
}

// part[block][c] = block's share of sum_p g[p][c]
__global__ void bias_grad_kernel(const bf16* g, float* part, int64_t P, int C)
{
    __shared__ float s[256];
    const int c = threadIdx.x % C;
    const int lanes = blockDim.x / C;          // blockDim is a multiple of C (C <= 256)
    const int lane = threadIdx.x / C;
    float acc = 0.f;
    for (int64_t p = (int64_t)blockIdx.x * lanes + lane; p < P; p += (int64_t)gridDim.x * lanes)
        acc += __bfloat162float(g[p * C + c]);
    s[threadIdx.x] = acc;
    __syncthreads();
    if (lane == 0) {
        float t = 0.f;
        for (int l = 0; l < lanes; ++l) t += s[l * C + c];
        part[(int64_t)blockIdx.x * C + c] = t;           // summed over the blocks in order afterwards
    }
}

// out[j] += sum_{c < nparts} part[c * n + j], in order of c (the deterministic
// second stage of the gradient and loss reductions)
__global__ void parts_reduce_kernel(const float* part, float* out, int64_t n, int nparts)
{
    GRID_STRIDE(j, n) {
        float t = 0.f;
        for (int c = 0; c < nparts; ++c) t += part[(int64_t)c * n + j];
        out[j] += t;
    }
}

// MSE over the first `used` of `C` output channels: loss partial per block (loss_acc[block]),
// gradient 2 (o - t) / count
__global__ void mse_kernel(const float* out, const float* target, bf16* gout, float* loss_acc, int64_t P, int C, int used,
                           float inv_count)
{
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P * C; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = i / C;
        const int c = (int)(i % C);
        float g = 0.f;
        if (c < used) {
            const float d = out[p * C + c] - target[p * used + c];
            acc += d * d;
            g = 2.f * d * inv_count;
        }
        gout[i] = __float2bfloat16(g);
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    __shared__ float ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {                              // this block's share, summed in order afterwards
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        loss_acc[blockIdx.x] = t * inv_count;
    }
}

__global__ void output_unpack_kernel(const float* o16, float* out, int64_t P, int C, int used)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P * used; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = o16[(i / used) * C + i % used];
}

__global__ void adam_kernel(float* w, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// bf16 weights for the forward ([9][Cout][Cin]) and the input-gradient
// convolution ([9][Cin][Cout], taps mirrored: tap k' uses k = 8 - k')
__global__ void weight_cast_kernel(const float* w, bf16* wf, bf16* wd, int Cin, int Cout)
{
    const int64_t n = (int64_t)9 * Cin * Cout;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(i % Cin);
        const int64_t q = i / Cin;
        const int co = (int)(q % Cout);
        const int k = (int)(q / Cout);
        const bf16 b = __float2bfloat16(w[i]);
        wf[i] = b;
        wd[((int64_t)(8 - k) * Cin + ci) * Cout + co] = b;
    }
}

inline int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

struct Conv {
    int cin, cout, relu;
    int64_t woff, boff;     // offsets into the parameter vector
};

struct Act {                // one activation tensor (and its gradient)
    int c, level;           // channels, resolution level (0 = full)
    bf16* y = nullptr;
    bf16* g = nullptr;
    int ys = 0;             // channels between consecutive pixels of y (0: c)
    int vof = -1;           // >= 0: y is the channel slice [voff, voff + c) of act vof's y (not owned)
    int voff = 0;
};

}  // namespace

struct tvcut_unet_ctx {
    int base = 32;
    int N = 0, H = 0, W = 0;
    cudaStream_t stream = nullptr;
    std::vector<Conv> convs;
    int64_t nparams = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wf = nullptr, *wd = nullptr;          // per-conv bf16 weights (same offsets as params)
    int64_t adam_t = 0;
    std::vector<Act> acts;
    float* out16 = nullptr;                      // N x H x W x 16 FP32 output
    float* loss = nullptr;
    float* gpart = nullptr;                      // partial sums of the gradient and loss reductions
    int64_t gpart_cap = 0;                       // its size in floats (grown at a backward pass)
    int engine = 0;                              // convolutions: 0 tcgen05 where supported, 1 mma.sync
    std::string err;
};

static thread_local std::string g_uerr;

static tvcut_status ufail(tvcut_unet_t u, tvcut_status st, const std::string& m)
{
    if (u) u->err = m;
    else g_uerr = m;
    return st;
}

#define UCK(u, expr, where)                                                                           \
    do {                                                                                              \
        cudaError_t e_ = (expr);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return ufail(u, e_ == cudaErrorMemoryAllocation ? TVCUT_ERR_OOM : TVCUT_ERR_CUDA,         \
                         std::string(where) + ": " + cudaGetErrorString(e_));                         \
    } while (0)

// activation indices in the order of the forward pass
enum {
    A_X, A_E1A, A_E1, A_P1, A_E2A, A_E2, A_P2, A_E3A, A_E3, A_P3, A_E4A, A_E4,
    A_U3A, A_U3, A_C3, A_D3A, A_D3, A_U2A, A_U2, A_C2, A_D2A, A_D2, A_U1A, A_U1, A_C1, A_D1A, A_D1, A_OUT, A_COUNT
};

static void define_net(tvcut_unet_t u)
{
    const int C = u->base;
    auto conv = [&](int cin, int cout, int relu) {
        Conv c{cin, cout, relu, u->nparams, 0};
        u->nparams += (int64_t)9 * cin * cout;
        c.boff = u->nparams;
        u->nparams += cout;
        u->convs.push_back(c);
    };
    // conv order = forward order
    conv(16, C, 1); conv(C, C, 1);
    conv(C, 2 * C, 1); conv(2 * C, 2 * C, 1);
    conv(2 * C, 4 * C, 1); conv(4 * C, 4 * C, 1);
    conv(4 * C, 8 * C, 1); conv(8 * C, 8 * C, 1);
    conv(8 * C, 4 * C, 1); conv(8 * C, 4 * C, 1); conv(4 * C, 4 * C, 1);
    conv(4 * C, 2 * C, 1); conv(4 * C, 2 * C, 1); conv(2 * C, 2 * C, 1);
    conv(2 * C, C, 1); conv(2 * C, C, 1); conv(C, C, 1);
    conv(C, 16, 0);
    const int ch[A_COUNT] = {16, C, C, C, 2 * C, 2 * C, 2 * C, 4 * C, 4 * C, 4 * C, 8 * C, 8 * C,
                             8 * C, 4 * C, 8 * C, 4 * C, 4 * C, 4 * C, 2 * C, 4 * C, 2 * C, 2 * C, 2 * C, C, 2 * C, C, C, 16};
    const int lv[A_COUNT] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0};
    u->acts.resize(A_COUNT);
    for (int i = 0; i < A_COUNT; ++i) {
        u->acts[i].c = ch[i];
        u->acts[i].level = lv[i];
    }
    // the decoder's concatenations [upsampled branch, skip] are not copied: both
    // producing convolutions write into their channel slices of the buffer
    const int views[6][3] = {{A_U3, A_C3, 0}, {A_E3, A_C3, 4 * C}, {A_U2, A_C2, 0},
                             {A_E2, A_C2, 2 * C}, {A_U1, A_C1, 0}, {A_E1, A_C1, C}};
    for (const auto& v : views) {
        u->acts[v[0]].vof = v[1];
        u->acts[v[0]].voff = v[2];
    }
}

static void free_acts(tvcut_unet_t u)
{
    for (auto& a : u->acts) {
        if (a.vof < 0) cudaFree(a.y);
        cudaFree(a.g);
        a.y = a.g = nullptr;
    }
    cudaFree(u->out16);
    u->out16 = nullptr;
}

static tvcut_status alloc_acts(tvcut_unet_t u, int N, int H, int W)
{
    if (N < 1 || H < 8 || W < 8 || H % 8 || W % 8)
        return ufail(u, TVCUT_ERR_INVALID, "tvcut_unet: batch >= 1 and H, W multiples of 8 (>= 8) required");
    free_acts(u);
    u->N = N;
    u->H = H;
    u->W = W;
    for (auto& a : u->acts) {
        const int64_t P = (int64_t)N * (H >> a.level) * (W >> a.level);
        if (a.vof < 0) UCK(u, cudaMalloc(&a.y, sizeof(bf16) * P * a.c), "tvcut_unet activations");
        UCK(u, cudaMalloc(&a.g, sizeof(bf16) * P * a.c), "tvcut_unet activations");
    }
    for (auto& a : u->acts) {
        if (a.vof < 0) continue;
        a.y = u->acts[a.vof].y + a.voff;
        a.ys = u->acts[a.vof].c;
    }
    UCK(u, cudaMalloc(&u->out16, sizeof(float) * (int64_t)N * H * W * 16), "tvcut_unet activations");
    return TVCUT_OK;
}

static uint64_t splitmix64(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" const char* tvcut_unet_last_error(tvcut_unet_t u) { return u ? u->err.c_str() : g_uerr.c_str(); }

extern "C" void tvcut_unet_destroy(tvcut_unet_t u)
{
    if (!u) return;
    free_acts(u);
    cudaFree(u->params);
    cudaFree(u->grads);
    cudaFree(u->m);
    cudaFree(u->v);
    cudaFree(u->wf);
    cudaFree(u->wd);
    cudaFree(u->loss);
    cudaFree(u->gpart);
    delete u;
}

static tvcut_status refresh_bf16(tvcut_unet_t u)
{
    for (const Conv& c : u->convs) {
        const int64_t n = (int64_t)9 * c.cin * c.cout;
        weight_cast_kernel<<<blocks_for(n), 256, 0, u->stream>>>(u->params + c.woff, u->wf + c.woff, u->wd + c.woff,
                                                                  c.cin, c.cout);
    }
    UCK(u, cudaGetLastError(), "tvcut_unet weights");
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_unet_create(int base, int N, int H, int W, uint64_t seed, void* stream,
                                          tvcut_unet_t* out)
{
    if (!out) return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_unet_create: out is NULL");
    *out = nullptr;
    if (base < 16 || base % 16 || base > 64)
        return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_unet_create: base channels must be 16, 32, 48 or 64");
    tvcut_unet_t u = new tvcut_unet_ctx();
    u->base = base;
    u->stream = (cudaStream_t)stream;
    define_net(u);
    const size_t pb = sizeof(float) * (size_t)u->nparams;
    cudaError_t e = cudaMalloc(&u->params, pb);
    if (e == cudaSuccess) e = cudaMalloc(&u->grads, pb);
    if (e == cudaSuccess) e = cudaMalloc(&u->m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&u->v, pb);
    if (e == cudaSuccess) e = cudaMalloc(&u->wf, sizeof(bf16) * (size_t)u->nparams);
    if (e == cudaSuccess) e = cudaMalloc(&u->wd, sizeof(bf16) * (size_t)u->nparams);
    if (e == cudaSuccess) e = cudaMalloc(&u->loss, sizeof(float) * 4);
    if (e == cudaSuccess) e = cudaMemset(u->m, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(u->v, 0, pb);
    if (e != cudaSuccess) {
        tvcut_unet_destroy(u);
        cudaGetLastError();            // clear the runtime's last error
        return ufail(nullptr, TVCUT_ERR_OOM, "tvcut_unet_create: allocation");
    }
    // He-normal weights (Box-Muller on splitmix64), zero biases
    std::vector<float> h((size_t)u->nparams, 0.f);
    uint64_t s = seed;
    for (const Conv& c : u->convs) {
        const float sd = sqrtf(2.f / (9.f * c.cin));
        for (int64_t i = 0; i < (int64_t)9 * c.cin * c.cout; ++i) {
            const double u1 = ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            const double u2 = ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            h[(size_t)(c.woff + i)] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
        }
    }
    e = cudaMemcpy(u->params, h.data(), pb, cudaMemcpyHostToDevice);
    tvcut_status st = e == cudaSuccess ? alloc_acts(u, N, H, W) : TVCUT_ERR_CUDA;
    if (st == TVCUT_OK) st = refresh_bf16(u);
    if (st != TVCUT_OK) {
        std::string m = u->err;
        tvcut_unet_destroy(u);
        cudaGetLastError();
        return ufail(nullptr, st, m.empty() ? "tvcut_unet_create failed" : m);
    }
    *out = u;
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_unet_resize(tvcut_unet_t u, int N, int H, int W)
{
    if (!u) return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_unet_resize: NULL handle");
    return alloc_acts(u, N, H, W);
}

// A 3x3 convolution: the tcgen05 kernel when the shape allows it (engine 0:
// its persistent forms; 3: one tile per CTA; 4: persistent without the halo
// form), else the mma.sync kernel.
static cudaError_t launch_conv(const ConvArgs& A, int engine, cudaStream_t s)
{
    if (engine != 1 && conv_tc_supported(A))
        return launch_conv3x3_tc(A, s, engine == 3 ? 1 : engine == 4 ? 2 : 0);
    const int64_t P = (int64_t)A.N * A.H * A.W;
    dim3 grid((unsigned)((P + FBM - 1) / FBM), (unsigned)((A.Cout + BN - 1) / BN));
    conv3x3_fwd_kernel<<<grid, FTHREADS, 0, s>>>(A);
    return cudaGetLastError();
}

static tvcut_status run_conv(tvcut_unet_t u, int ci, const Act& in, Act& out, const bf16* wt, bool bias)
{
    const Conv& c = u->convs[ci];
    ConvArgs A;
    A.in = in.y;
    A.wt = wt + c.woff;
    A.bias = bias ? u->params + c.boff : nullptr;
    A.out = out.y;                           // a channel slice of a concatenation for the skip and upsampled branches
    A.out_f32 = (ci == (int)u->convs.size() - 1) ? u->out16 : nullptr;
    A.mask = nullptr;
    A.N = u->N;
    A.H = u->H >> in.level;
    A.W = u->W >> in.level;
    A.Cin = c.cin;
    A.Cout = c.cout;
    A.CoutStride = out.ys ? out.ys : c.cout;
    A.relu = c.relu;
    UCK(u, launch_conv(A, u->engine, u->stream), "conv forward");
    return TVCUT_OK;
}

#define UST(x) do { tvcut_status s_ = (x); if (s_ != TVCUT_OK) return s_; } while (0)

static tvcut_status forward(tvcut_unet_t u, const float* in)
{
    auto& a = u->acts;
    const int N = u->N, H = u->H, W = u->W;
    const int64_t P0 = (int64_t)N * H * W;
    if (in) input_pack_kernel<<<blocks_for(P0), 256, 0, u->stream>>>(in, a[A_X].y, P0);   // else packed already
    const bf16* wf = u->wf;
    auto pool = [&](int i, int o) {
        const int lv = a[i].level;
        const int64_t n = (int64_t)N * (H >> (lv + 1)) * (W >> (lv + 1)) * a[i].c;
        pool_fwd_kernel<<<blocks_for(n / 8), 256, 0, u->stream>>>(a[i].y, a[o].y, N, H >> lv, W >> lv, a[i].c,
                                                                  a[i].ys ? a[i].ys : a[i].c);
    };
    auto up = [&](int i, int o) {
        const int lv = a[o].level;
        const int64_t n = (int64_t)N * (H >> lv) * (W >> lv) * a[i].c;
        up_fwd_kernel<<<blocks_for(n / 8), 256, 0, u->stream>>>(a[i].y, a[o].y, N, H >> lv, W >> lv, a[i].c);
    };

    UST(run_conv(u, 0, a[A_X], a[A_E1A], wf, true));
    UST(run_conv(u, 1, a[A_E1A], a[A_E1], wf, true));
    pool(A_E1, A_P1);
    UST(run_conv(u, 2, a[A_P1], a[A_E2A], wf, true));
    UST(run_conv(u, 3, a[A_E2A], a[A_E2], wf, true));
    pool(A_E2, A_P2);
    UST(run_conv(u, 4, a[A_P2], a[A_E3A], wf, true));
    UST(run_conv(u, 5, a[A_E3A], a[A_E3], wf, true));
    pool(A_E3, A_P3);
    UST(run_conv(u, 6, a[A_P3], a[A_E4A], wf, true));
    UST(run_conv(u, 7, a[A_E4A], a[A_E4], wf, true));
    up(A_E4, A_U3A);
    UST(run_conv(u, 8, a[A_U3A], a[A_U3], wf, true));
    UST(run_conv(u, 9, a[A_C3], a[A_D3A], wf, true));
    UST(run_conv(u, 10, a[A_D3A], a[A_D3], wf, true));
    up(A_D3, A_U2A);
    UST(run_conv(u, 11, a[A_U2A], a[A_U2], wf, true));
    UST(run_conv(u, 12, a[A_C2], a[A_D2A], wf, true));
    UST(run_conv(u, 13, a[A_D2A], a[A_D2], wf, true));
    up(A_D2, A_U1A);
    UST(run_conv(u, 14, a[A_U1A], a[A_U1], wf, true));
    UST(run_conv(u, 15, a[A_C1], a[A_D1A], wf, true));
    UST(run_conv(u, 16, a[A_D1A], a[A_D1], wf, true));
    UST(run_conv(u, 17, a[A_D1], a[A_OUT], wf, true));
    UCK(u, cudaGetLastError(), "tvcut_unet_forward");
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_unet_forward(tvcut_unet_t u, const float* in, float* out)
{
    if (!u) return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_unet_forward: NULL handle");
    if (!in) return ufail(u, TVCUT_ERR_INVALID, "tvcut_unet_forward: NULL input");
    UST(forward(u, in));
    if (out) {
        const int64_t P = (int64_t)u->N * u->H * u->W;
        output_unpack_kernel<<<blocks_for(P * 2), 256, 0, u->stream>>>(u->out16, out, P, 16, 2);
        UCK(u, cudaGetLastError(), "tvcut_unet_forward");
    }
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_unet_predict_state(tvcut_unet_t u, tvcut_t h)
{
    if (!u) return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_unet_predict_state: NULL network");
    if (!h) return ufail(u, TVCUT_ERR_INVALID, "tvcut_unet_predict_state: NULL solver handle");
    tvcut::ProblemView v;
    std::string why;
    tvcut_status st = tvcut::problem_view(h, &v, &why);
    if (st != TVCUT_OK) return ufail(u, st, "tvcut_unet_predict_state: " + why);
    if (v.H < 8 || v.W < 8 || v.H % 8 || v.W % 8 || v.H > (1 << 16) || v.W > (1 << 16))
        return ufail(u, TVCUT_ERR_INVALID, "tvcut_unet_predict_state: H and W must be multiples of 8 in [8, 65536]");
    if (u->N != 1 || u->H != (int)v.H || u->W != (int)v.W) UST(alloc_acts(u, 1, (int)v.H, (int)v.W));
    const int H = (int)v.H, W = (int)v.W;
    const int64_t P = (int64_t)H * W;
    struct EventGuard {                          // destroyed on every return path
        cudaEvent_t e = nullptr;
        ~EventGuard() { if (e) cudaEventDestroy(e); }
    } guard;
    cudaEvent_t ev = nullptr;
    if (u->stream != v.stream) {                 // the network's stream runs after the handle's
        UCK(u, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "tvcut_unet_predict_state");
        guard.e = ev;
        UCK(u, cudaEventRecord(ev, v.stream), "tvcut_unet_predict_state");
        UCK(u, cudaStreamWaitEvent(u->stream, ev, 0), "tvcut_unet_predict_state");
    }
    if (v.esize == 8)
        features_pack_kernel<double><<<blocks_for(P), 256, 0, u->stream>>>(
            (const double*)v.w, (const double*)v.a0, (const double*)v.a1, v.a1_transposed, H, W, v.scale,
            u->acts[A_X].y);
    else
        features_pack_kernel<float><<<blocks_for(P), 256, 0, u->stream>>>(
            (const float*)v.w, (const float*)v.a0, (const float*)v.a1, v.a1_transposed, H, W, v.scale,
            u->acts[A_X].y);
    UCK(u, cudaGetLastError(), "tvcut_unet_predict_state");
    UST(forward(u, nullptr));
    if (v.esize == 8)
        state_from_output_kernel<double><<<blocks_for(P), 256, 0, u->stream>>>(
            u->out16, H, W, (float)v.scale, (double*)v.s0, (double*)v.s1, v.s1_transposed);
    else
        state_from_output_kernel<float><<<blocks_for(P), 256, 0, u->stream>>>(
            u->out16, H, W, (float)v.scale, (float*)v.s0, (float*)v.s1, v.s1_transposed);
    UCK(u, cudaGetLastError(), "tvcut_unet_predict_state");
    if (ev) {                                    // and the handle's stream after the network's
        UCK(u, cudaEventRecord(ev, u->stream), "tvcut_unet_predict_state");
        UCK(u, cudaStreamWaitEvent(v.stream, ev, 0), "tvcut_unet_predict_state");
    }
    st = tvcut::state_written(h);
    if (st != TVCUT_OK) return ufail(u, st, "tvcut_unet_predict_state: " + std::string(tvcut_last_error(h)));
    return TVCUT_OK;
}

// resolution level of each convolution's input, in forward order
static const int kConvLevel[18] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0, 0};
constexpr int64_t kWgradPixels = 4096;           // pixels per weight-gradient CTA
constexpr int kBiasBlocks = 256;

// Floats of partial sums the backward pass needs at the current shape: the
// weight gradient's per-chunk slices of the largest layer, the bias
// gradient's per-block rows, the loss's per-block values.
static int64_t gpart_floats(tvcut_unet_t u)
{
    int64_t need = (int64_t)blocks_for((int64_t)u->N * u->H * u->W * 16);
    for (size_t ci = 0; ci < u->convs.size(); ++ci) {
        const Conv& c = u->convs[ci];
        const int lv = kConvLevel[ci];
        const int64_t P = (int64_t)u->N * (u->H >> lv) * (u->W >> lv);
        const int64_t nch = (P + kWgradPixels - 1) / kWgradPixels;
        if (nch > 1) need = std::max<int64_t>(need, nch * 9 * c.cin * c.cout);
        need = std::max<int64_t>(need, (int64_t)kBiasBlocks * c.cout);
    }
    return need;
}

// gradient of conv ci: g_out is the gradient at its output (after the ReLU
// mask); accumulates dW, db and writes the gradient of its input into gin
// (overwrite) when gin != nullptr.
static tvcut_status conv_backward(tvcut_unet_t u, int ci, const Act& in, const Act& out, bf16* gin)
{
    const Conv& c = u->convs[ci];
    const int Hl = u->H >> in.level, Wl = u->W >> in.level;
    const int64_t P = (int64_t)u->N * Hl * Wl;
    WgradArgs G;
    G.in = in.y;
    G.dout = out.g;
    G.dw = u->grads + c.woff;
    G.N = u->N;
    G.H = Hl;
    G.W = Wl;
    G.Cin = c.cin;
    G.Cout = c.cout;
    G.part = u->gpart;
    G.pix_per_cta = kWgradPixels;
    const int nch = (int)((P + G.pix_per_cta - 1) / G.pix_per_cta);
    dim3 gw((unsigned)((c.cout + BM - 1) / BM), (unsigned)((c.cin + BN - 1) / BN), (unsigned)(9 * nch));
    conv3x3_wgrad_kernel<<<gw, 128, 0, u->stream>>>(G);
    const int64_t nw = (int64_t)9 * c.cout * c.cin;
    if (nch > 1) parts_reduce_kernel<<<blocks_for(nw), 256, 0, u->stream>>>(u->gpart, G.dw, nw, nch);
    const int lanes = 256 / c.cout > 0 ? 256 / c.cout : 1;
    bias_grad_kernel<<<kBiasBlocks, lanes * c.cout, 0, u->stream>>>(out.g, u->gpart, P, c.cout);
    parts_reduce_kernel<<<blocks_for(c.cout), 256, 0, u->stream>>>(u->gpart, u->grads + c.boff, c.cout, kBiasBlocks);
    if (gin) {
        ConvArgs A;
        A.in = out.g;
        A.wt = u->wd + c.woff;
        A.bias = nullptr;
        A.out = gin;
        A.out_f32 = nullptr;
        A.mask = nullptr;
        A.N = u->N;
        A.H = Hl;
        A.W = Wl;
        A.Cin = c.cout;
        A.Cout = c.cin;
        A.CoutStride = c.cin;
        A.relu = 0;
        UCK(u, launch_conv(A, u->engine, u->stream), "conv backward");
    }
    UCK(u, cudaGetLastError(), "conv backward");
    return TVCUT_OK;
}

static void mask(tvcut_unet_t u, Act& a)
{
    const int64_t n = (int64_t)u->N * (u->H >> a.level) * (u->W >> a.level) * a.c;
    relu_mask_kernel<<<blocks_for(n / 8), 256, 0, u->stream>>>(a.g, a.y, n, a.c, a.ys ? a.ys : a.c);
}

extern "C" tvcut_status tvcut_unet_backward(tvcut_unet_t u, const float* target, float* loss_out)
{
    if (!u) return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_unet_backward: NULL handle");
    if (!target) return ufail(u, TVCUT_ERR_INVALID, "tvcut_unet_backward: NULL target");
    auto& a = u->acts;
    const int N = u->N, H = u->H, W = u->W;
    const int64_t P0 = (int64_t)N * H * W;
    UCK(u, cudaMemsetAsync(u->grads, 0, sizeof(float) * (size_t)u->nparams, u->stream), "tvcut_unet_backward");
    UCK(u, cudaMemsetAsync(u->loss, 0, sizeof(float), u->stream), "tvcut_unet_backward");
    const int64_t need = gpart_floats(u);
    if (u->gpart_cap < need) {
        UCK(u, cudaStreamSynchronize(u->stream), "tvcut_unet_backward");
        cudaFree(u->gpart);
        u->gpart = nullptr;
        u->gpart_cap = 0;
        UCK(u, cudaMalloc(&u->gpart, sizeof(float) * (size_t)need), "tvcut_unet_backward: partial sums");
        u->gpart_cap = need;
    }
    const int mblocks = blocks_for(P0 * 16);
    mse_kernel<<<mblocks, 256, 0, u->stream>>>(u->out16, target, a[A_OUT].g, u->gpart, P0, 16, 2,
                                               1.f / (float)(P0 * 2));
    parts_reduce_kernel<<<1, 32, 0, u->stream>>>(u->gpart, u->loss, 1, mblocks);
    auto pool_b = [&](int o, int i) {       // a[i].g += pool'(a[o].g)
        const int lv = a[i].level;
        const int64_t n = (int64_t)N * (H >> lv) * (W >> lv) * a[i].c;
        pool_bwd_kernel<<<blocks_for(n / 8), 256, 0, u->stream>>>(a[o].g, a[i].g, N, H >> lv, W >> lv, a[i].c);
    };
    auto up_b = [&](int o, int i) {         // a[i].g = up'(a[o].g)
        const int lv = a[i].level;
        const int64_t n = (int64_t)N * (H >> lv) * (W >> lv) * a[i].c;
        up_bwd_kernel<<<blocks_for(n / 8), 256, 0, u->stream>>>(a[o].g, a[i].g, N, H >> lv, W >> lv, a[i].c);
    };
    auto cat_b = [&](int o, int x, int s) { // a[x].g = g[:Cx]; a[s].g += g[Cx:]
        const int lv = a[o].level;
        const int64_t P = (int64_t)N * (H >> lv) * (W >> lv);
        concat_bwd_kernel<<<blocks_for(P * a[o].c / 8), 256, 0, u->stream>>>(a[o].g, a[x].g, a[s].g, P, a[x].c, a[s].c);
    };
    // skip tensors receive gradient from the decoder first: clear them
    for (int i : {A_E1, A_E2, A_E3})
        UCK(u, cudaMemsetAsync(a[i].g, 0, sizeof(bf16) * (size_t)N * (H >> a[i].level) * (W >> a[i].level) * a[i].c,
                               u->stream), "tvcut_unet_backward");
    UST(conv_backward(u, 17, a[A_D1], a[A_OUT], a[A_D1].g));
    mask(u, a[A_D1]);
    UST(conv_backward(u, 16, a[A_D1A], a[A_D1], a[A_D1A].g));
    mask(u, a[A_D1A]);
    UST(conv_backward(u, 15, a[A_C1], a[A_D1A], a[A_C1].g));
    cat_b(A_C1, A_U1, A_E1);
    mask(u, a[A_U1]);
    UST(conv_backward(u, 14, a[A_U1A], a[A_U1], a[A_U1A].g));
    up_b(A_U1A, A_D2);
    mask(u, a[A_D2]);
    UST(conv_backward(u, 13, a[A_D2A], a[A_D2], a[A_D2A].g));
    mask(u, a[A_D2A]);
    UST(conv_backward(u, 12, a[A_C2], a[A_D2A], a[A_C2].g));
    cat_b(A_C2, A_U2, A_E2);
    mask(u, a[A_U2]);
    UST(conv_backward(u, 11, a[A_U2A], a[A_U2], a[A_U2A].g));
    up_b(A_U2A, A_D3);
    mask(u, a[A_D3]);
    UST(conv_backward(u, 10, a[A_D3A], a[A_D3], a[A_D3A].g));
    mask(u, a[A_D3A]);
    UST(conv_backward(u, 9, a[A_C3], a[A_D3A], a[A_C3].g));
    cat_b(A_C3, A_U3, A_E3);
    mask(u, a[A_U3]);
    UST(conv_backward(u, 8, a[A_U3A], a[A_U3], a[A_U3A].g));
    up_b(A_U3A, A_E4);
    mask(u, a[A_E4]);
    UST(conv_backward(u, 7, a[A_E4A], a[A_E4], a[A_E4A].g));
    mask(u, a[A_E4A]);
    UST(conv_backward(u, 6, a[A_P3], a[A_E4A], a[A_P3].g));
    pool_b(A_P3, A_E3);
    mask(u, a[A_E3]);
    UST(conv_backward(u, 5, a[A_E3A], a[A_E3], a[A_E3A].g));
    mask(u, a[A_E3A]);
    UST(conv_backward(u, 4, a[A_P2], a[A_E3A], a[A_P2].g));
    pool_b(A_P2, A_E2);
    mask(u, a[A_E2]);
    UST(conv_backward(u, 3, a[A_E2A], a[A_E2], a[A_E2A].g));
    mask(u, a[A_E2A]);
    UST(conv_backward(u, 2, a[A_P1], a[A_E2A], a[A_P1].g));
    pool_b(A_P1, A_E1);
    mask(u, a[A_E1]);
    UST(conv_backward(u, 1, a[A_E1A], a[A_E1], a[A_E1A].g));
    mask(u, a[A_E1A]);
    UST(conv_backward(u, 0, a[A_X], a[A_E1A], nullptr));
    UCK(u, cudaGetLastError(), "tvcut_unet_backward");
    if (loss_out) {
        UCK(u, cudaMemcpyAsync(loss_out, u->loss, sizeof(float), cudaMemcpyDeviceToHost, u->stream), "tvcut_unet_backward");
        UCK(u, cudaStreamSynchronize(u->stream), "tvcut_unet_backward");
    }
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_unet_adam(tvcut_unet_t u, float lr, float beta1, float beta2, float eps)
{
    if (!u) return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_unet_adam: NULL handle");
    u->adam_t += 1;
    const float c1 = 1.f - powf(beta1, (float)u->adam_t), c2 = 1.f - powf(beta2, (float)u->adam_t);
    adam_kernel<<<blocks_for(u->nparams), 256, 0, u->stream>>>(u->params, u->grads, u->m, u->v, u->nparams, lr, beta1,
                                                               beta2, eps, c1, c2);
    UCK(u, cudaGetLastError(), "tvcut_unet_adam");
    return refresh_bf16(u);
}

extern "C" tvcut_status tvcut_unet_num_params(tvcut_unet_t u, int64_t* count)
{
    if (!u || !count) return ufail(u, TVCUT_ERR_INVALID, "tvcut_unet_num_params: NULL argument");
    *count = u->nparams;
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_unet_get_params(tvcut_unet_t u, float* dst, int which)
{
    if (!u || !dst) return ufail(u, TVCUT_ERR_INVALID, "tvcut_unet_get_params: NULL argument");
    const float* src = which == 1 ? u->grads : u->params;
    UCK(u, cudaMemcpyAsync(dst, src, sizeof(float) * (size_t)u->nparams, cudaMemcpyDeviceToHost, u->stream),
        "tvcut_unet_get_params");
    UCK(u, cudaStreamSynchronize(u->stream), "tvcut_unet_get_params");
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_unet_set_params(tvcut_unet_t u, const float* src)
{
    if (!u || !src) return ufail(u, TVCUT_ERR_INVALID, "tvcut_unet_set_params: NULL argument");
    UCK(u, cudaMemcpyAsync(u->params, src, sizeof(float) * (size_t)u->nparams, cudaMemcpyHostToDevice, u->stream),
        "tvcut_unet_set_params");
    UST(refresh_bf16(u));
    UCK(u, cudaStreamSynchronize(u->stream), "tvcut_unet_set_params");
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_conv3x3_bf16(const void* in, const void* wt, const float* bias, void* out, int N, int H,
                                           int W, int Cin, int Cout, int relu, void* stream)
{
    return tvcut_conv3x3_bf16_ex(in, wt, bias, out, N, H, W, Cin, Cout, relu, 0, stream);
}

extern "C" tvcut_status tvcut_conv3x3_bf16_ex(const void* in, const void* wt, const float* bias, void* out, int N,
                                              int H, int W, int Cin, int Cout, int relu, int engine, void* stream)
{
    if (!in || !wt || !out || N < 1 || H < 1 || W < 1 || Cin % 16 || Cout % 16 || Cin < 16 || Cout < 16)
        return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_conv3x3_bf16: bad arguments (channels multiples of 16)");
    if (engine < 0 || engine > 4) return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_conv3x3_bf16_ex: engine must be 0..4");
    ConvArgs A;
    A.in = (const bf16*)in;
    A.wt = (const bf16*)wt;
    A.bias = bias;
    A.out = (bf16*)out;
    A.out_f32 = nullptr;
    A.mask = nullptr;
    A.N = N;
    A.H = H;
    A.W = W;
    A.Cin = Cin;
    A.Cout = Cout;
    A.CoutStride = Cout;
    A.relu = relu;
    if (engine >= 2 && !conv_tc_supported(A))
        return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_conv3x3_bf16_ex: shape not supported by the tcgen05 kernel");
    cudaError_t e = launch_conv(A, engine == 2 ? 0 : engine, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ufail(nullptr, TVCUT_ERR_CUDA, cudaGetErrorString(e));
    }
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_conv3x3_wgrad_bf16(const void* in, const void* dout, float* dw, int N, int H, int W,
                                                 int Cin, int Cout, void* stream)
{
    if (!in || !dout || !dw || N < 1 || H < 1 || W < 1 || Cin % 16 || Cout % 16 || Cin < 16 || Cout < 16)
        return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_conv3x3_wgrad_bf16: bad arguments (channels multiples of 16)");
    WgradArgs G;
    G.in = (const bf16*)in;
    G.dout = (const bf16*)dout;
    G.dw = dw;
    G.part = nullptr;                            // added atomically (summation order varies)
    G.N = N;
    G.H = H;
    G.W = W;
    G.Cin = Cin;
    G.Cout = Cout;
    G.pix_per_cta = 4096;
    const int64_t P = (int64_t)N * H * W;
    const int nch = (int)((P + G.pix_per_cta - 1) / G.pix_per_cta);
    dim3 gw((unsigned)((Cout + BM - 1) / BM), (unsigned)((Cin + BN - 1) / BN), (unsigned)(9 * nch));
    conv3x3_wgrad_kernel<<<gw, 128, 0, (cudaStream_t)stream>>>(G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ufail(nullptr, TVCUT_ERR_CUDA, cudaGetErrorString(e));
    return TVCUT_OK;
}

extern "C" tvcut_status tvcut_unet_set_engine(tvcut_unet_t u, int engine)
{
    if (!u) return ufail(nullptr, TVCUT_ERR_INVALID, "tvcut_unet_set_engine: NULL handle");
    if (engine != 0 && engine != 1 && engine != 3 && engine != 4)
        return ufail(u, TVCUT_ERR_INVALID, "tvcut_unet_set_engine: engine must be 0, 1, 3 or 4");
    u->engine = engine;
    return TVCUT_OK;
}

extern "C" int tvcut_conv_tc_error(void)
{
    return conv_tc_take_error();
}

extern "C" tvcut_status tvcut_conv_tc_stall(int on)
{
    if (conv_tc_set_stall(on ? 1 : 0) != 0) return ufail(nullptr, TVCUT_ERR_CUDA, "tvcut_conv_tc_stall: cudaMemcpyToSymbol");
    return TVCUT_OK;
}
