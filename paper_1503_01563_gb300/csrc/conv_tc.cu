// 3x3 convolution (BF16 in, FP32 accumulate) on the 5th-generation tensor
// cores: an implicit GEMM with M = 128 output pixels per CTA, N = Cout and
// K = 9 taps x Cin.
//
//   A (pixels x K): for tap (ky, kx) and a channel chunk, the 128 pixels of
//      the tile shifted by (ky - 1, kx - 1) are one TMA box of the NHWC
//      activation tensor (zero fill outside the image = the conv's padding),
//      written to shared memory in the K-major swizzled layout tcgen05.mma
//      reads.  The tile is 128 consecutive pixels of one image row (W a
//      multiple of 128) or 128/W whole rows (W < 128).
//   B (Cout x K): the weights [9][Cout][Cin] of the same tap and chunk, one
//      TMA box.
//   D: FP32 accumulators in tensor memory (128 lanes x Cout columns).
//
// Three forms share these pieces:
//   conv3x3_tc_kernel   one 128-pixel tile per CTA: one thread issues the TMA
//                       loads into a ring of stages (mbarriers count the
//                       bytes), one thread issues the MMAs and frees each
//                       stage with tcgen05.commit; then all four warps read
//                       their 32 accumulator rows with tcgen05.ld, add bias,
//                       apply ReLU / mask, and store BF16 (and FP32);
//   conv3x3_tcp_kernel  persistent CTAs with the producer, the MMA issuer and
//                       eight epilogue warps in separate warps and two
//                       tensor-memory accumulator buffers, so that one tile's
//                       epilogue overlaps the next tiles' loads and MMAs;
//   conv3x3_tch_kernel  the persistent form for 16-64 input channels with the
//                       tile's three input rows loaded once per 8 channels
//                       (the nine taps are descriptor offsets into them) and
//                       the weights resident in shared memory.
// The three issue the same MMAs in the same order, so their outputs are
// identical.  Every wait is bounded by a 2 s clock; a wait that gives up
// raises an error flag the host reads back, every role stops at its next
// tile, and each CTA still releases its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "conv_args.cuh"

namespace tvcut {
namespace nn {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 128;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

__device__ int g_conv_tc_error;
// Test hook (tvcut_conv_tc_stall): while set, CTA 0 of every launch skips its
// first operand load, so that its MMA issuer's bounded wait gives up.
__device__ int g_conv_tc_stall;

struct TcShape {
    int cblk;       // channels per K block (16, 32 or 64): one swizzle row
    int chunks;     // K blocks per tap (Cin / cblk)
    int kblocks;    // 9 * chunks
    int stages;
    int a_bytes;    // 128 x cblk x 2
    int b_bytes;    // Cout x cblk x 2
    int swz;        // shared-memory descriptor layout code (6: 32 B, 4: 64 B, 2: 128 B swizzle)
    int ncols;      // tensor-memory columns allocated (power of two >= 32, >= Cout)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait for the phase with the given parity to complete; false after 2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    const unsigned long long t0 = clock_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock_ns() - t0 > TC_WAIT_NS) {
            atomicExch(&g_conv_tc_error, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile: rows of
// `row_bytes` (the swizzle width), groups of 8 rows `8 * row_bytes` apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t row_bytes, uint32_t layout)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);                 // start address
    d |= (uint64_t)1 << 16;                                   // leading byte offset (unused when swizzled)
    d |= (uint64_t)(((8u * row_bytes) & 0x3FFFFu) >> 4) << 32; // stride byte offset: 8-row groups
    d |= (uint64_t)1 << 46;                                   // descriptor version
    d |= (uint64_t)layout << 61;                              // swizzle mode
    return d;
}

__device__ __forceinline__ void mma_bf16_ss(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Epilogue of one accumulator row (output pixel p, tensor-memory row trow)
// for the 16-column chunks c0, c0 + cstep, ...: bias, ReLU, mask, BF16 (and
// optional FP32) stores.  Every lane of the warp calls it (tcgen05.ld is
// .sync.aligned).
__device__ __forceinline__ void epilogue_row(const ConvArgs& A, int64_t p, uint32_t trow, int c0, int cstep)
{
    const bool vbias = A.bias && ((uintptr_t)A.bias & 15) == 0;
    for (int c = c0; c < A.Cout; c += cstep) {
        uint32_t r[16];
        tmem_ld16(trow + (uint32_t)c, r);
        const int64_t o = p * A.CoutStride + c;
        __align__(16) __nv_bfloat16 ob[16];
        __align__(16) __nv_bfloat16 mk[16];
        __align__(16) float bs[16];
        if (A.mask) {
            *(uint4*)&mk[0] = *(const uint4*)(A.mask + o);
            *(uint4*)&mk[8] = *(const uint4*)(A.mask + o + 8);
        }
        if (vbias) {
#pragma unroll
            for (int j = 0; j < 16; j += 4) *(float4*)&bs[j] = *(const float4*)(A.bias + c + j);
        } else if (A.bias) {
#pragma unroll
            for (int j = 0; j < 16; ++j) bs[j] = A.bias[c + j];
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float v = __uint_as_float(r[j]);
            if (A.bias) v += bs[j];
            if (A.relu) v = fmaxf(v, 0.f);
            if (A.mask && !(__bfloat162float(mk[j]) > 0.f)) v = 0.f;
            ob[j] = __float2bfloat16(v);
            if (A.out_f32) A.out_f32[p * A.Cout + c + j] = v;
        }
        *(uint4*)(A.out + o) = *(const uint4*)&ob[0];
        *(uint4*)(A.out + o + 8) = *(const uint4*)&ob[8];
    }
}

__global__ void __launch_bounds__(TC_THREADS, 10) conv3x3_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB, ConvArgs A,
                                                                TcShape S)
{
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);   // swizzle atoms: 1 KB aligned
    const int stage_bytes = S.a_bytes + S.b_bytes;
    uint64_t* full = (uint64_t*)(sm + (size_t)S.stages * stage_bytes);
    uint64_t* empty = full + S.stages;
    uint64_t* done = empty + S.stages;
    uint32_t* tslot = (uint32_t*)(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // the tile: 128 consecutive pixels (never across images: H*W % 128 == 0)
    const int64_t HW = (int64_t)A.H * A.W;
    const int64_t p0 = (int64_t)blockIdx.x * TC_M;
    const int img = (int)(p0 / HW);
    const int64_t rem = p0 - (int64_t)img * HW;
    const int y0 = (int)(rem / A.W), x0 = (int)(rem - (int64_t)(rem / A.W) * A.W);

    if (tid == 0) {
        for (int s = 0; s < S.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(S.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // producer: TMA loads of A and B for every K block into the stage ring
        for (int kb = 0; kb < S.kblocks; ++kb) {
            const int s = kb % S.stages, use = kb / S.stages;
            if (use > 0 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1))) break;
            const int tap = kb / S.chunks, c0 = (kb - tap * S.chunks) * S.cblk;
            const int ky = tap / 3, kx = tap - 3 * ky;
            uint8_t* sa = sm + (size_t)s * stage_bytes;
            mbar_expect_tx(&full[s], (uint32_t)stage_bytes);
            if (kb == 0 && blockIdx.x == 0 && *(volatile int*)&g_conv_tc_stall) continue;
            tma_load_4d(sa, &tmA, c0, x0 + kx - 1, y0 + ky - 1, img, &full[s]);
            tma_load_3d(sa + S.a_bytes, &tmB, c0, 0, tap, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: M = 128, N = Cout, BF16 x BF16 -> FP32, both K-major
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(A.Cout >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);
        const uint32_t row_bytes = (uint32_t)S.cblk * 2u;
        bool ok = true;
        for (int kb = 0; kb < S.kblocks && ok; ++kb) {
            const int s = kb % S.stages, use = kb / S.stages;
            ok = mbar_wait(&full[s], (uint32_t)(use & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(sm + (size_t)s * stage_bytes);
            const uint64_t ad = smem_desc(sa, row_bytes, (uint32_t)S.swz);
            const uint64_t bd = smem_desc(sa + (uint32_t)S.a_bytes, row_bytes, (uint32_t)S.swz);
            for (int k = 0; k < S.cblk / 16; ++k)           // 16 channels = 32 bytes per MMA
                mma_bf16_ss(tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, (kb | k) ? 1u : 0u);
            mma_commit(&empty[s]);                          // stage free once these MMAs are done
        }
        if (ok) mma_commit(done);
        else mbar_arrive(done);
    }
    __syncwarp();

    // epilogue: warp w owns accumulator rows (pixels) 32w .. 32w+31
    const bool have = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();
    if (__all_sync(0xffffffffu, have && !*(volatile int*)&g_conv_tc_error))
        epilogue_row(A, p0 + warp * 32 + lane, tmem + ((uint32_t)(warp * 32) << 16), 0, 16);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S.ncols) : "memory");
    }
}

// Persistent form: a CTA loops over tiles blockIdx.x, blockIdx.x + gridDim.x,
// ... with its roles in separate warps, so that the loads and MMAs of the
// next tile run while the epilogue drains the last one.
//   warp 8 (one lane): TMA producer, one continuous stream of K blocks over
//                      all of the CTA's tiles into the stage ring;
//   warp 9 (one lane): MMA issuer, accumulating tile i into tensor-memory
//                      buffer i % 2 (two buffers of ncols columns), then
//                      committing to tfull[i % 2];
//   warps 0-7:         epilogue of tile i from buffer i % 2: warp w reads
//                      accumulator lanes 32 (w % 4) .. + 31 (the lane
//                      quarter a warp may access) and the 16-column chunks
//                      w / 4, w / 4 + 2, ...; then one arrival per warp on
//                      tempty[i % 2] frees the buffer.
// Every wait is bounded as in conv3x3_tc_kernel; after a give-up every role
// stops at its next tile, and the CTA still frees its tensor memory.
constexpr int TCP_EPI_WARPS = 8;
constexpr int TCP_THREADS = 32 * (TCP_EPI_WARPS + 2);
constexpr int TCP_MAX_CTAS = 3;

__device__ __forceinline__ bool tc_failed() { return *(volatile int*)&g_conv_tc_error != 0; }

__device__ __forceinline__ void tile_origin(const ConvArgs& A, int64_t t, int64_t& p0, int& img, int& y0, int& x0)
{
    const int64_t HW = (int64_t)A.H * A.W;
    p0 = t * TC_M;
    img = (int)(p0 / HW);
    const int64_t rem = p0 - (int64_t)img * HW;
    y0 = (int)(rem / A.W);
    x0 = (int)(rem - (int64_t)y0 * A.W);
}

__global__ void __launch_bounds__(TCP_THREADS, TCP_MAX_CTAS) conv3x3_tcp_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                  const __grid_constant__ CUtensorMap tmB,
                                                                  ConvArgs A, TcShape S, int64_t tiles)
{
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int stage_bytes = S.a_bytes + S.b_bytes;
    uint64_t* full = (uint64_t*)(sm + (size_t)S.stages * stage_bytes);
    uint64_t* empty = full + S.stages;
    uint64_t* tfull = empty + S.stages;      // [2]
    uint64_t* tempty = tfull + 2;            // [2]
    uint32_t* tslot = (uint32_t*)(tempty + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < S.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], TCP_EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(2 * S.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == TCP_EPI_WARPS) {
        if (lane == 0) {
            int64_t kbg = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < tiles && ok && !tc_failed(); t += gridDim.x) {
                int64_t p0;
                int img, y0, x0;
                tile_origin(A, t, p0, img, y0, x0);
                for (int kb = 0; kb < S.kblocks; ++kb, ++kbg) {
                    const int s = (int)(kbg % S.stages);
                    const int64_t use = kbg / S.stages;
                    if (use > 0 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    const int tap = kb / S.chunks, c0 = (kb - tap * S.chunks) * S.cblk;
                    const int ky = tap / 3, kx = tap - 3 * ky;
                    uint8_t* sa = sm + (size_t)s * stage_bytes;
                    mbar_expect_tx(&full[s], (uint32_t)stage_bytes);
                    if (kbg == 0 && blockIdx.x == 0 && *(volatile int*)&g_conv_tc_stall) continue;
                    tma_load_4d(sa, &tmA, c0, x0 + kx - 1, y0 + ky - 1, img, &full[s]);
                    tma_load_3d(sa + S.a_bytes, &tmB, c0, 0, tap, &full[s]);
                }
            }
        }
    } else if (warp == TCP_EPI_WARPS + 1) {
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(A.Cout >> 3) << 17) |
                                   ((uint32_t)(TC_M >> 4) << 24);
            const uint32_t row_bytes = (uint32_t)S.cblk * 2u;
            int64_t kbg = 0;
            int it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < tiles && ok && !tc_failed(); t += gridDim.x, ++it) {
                const int buf = it & 1, ubuf = it >> 1;
                if (ubuf > 0 && !mbar_wait(&tempty[buf], (uint32_t)((ubuf - 1) & 1))) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * S.ncols);
                for (int kb = 0; kb < S.kblocks; ++kb, ++kbg) {
                    const int s = (int)(kbg % S.stages);
                    const int64_t use = kbg / S.stages;
                    if (!mbar_wait(&full[s], (uint32_t)(use & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_u32(sm + (size_t)s * stage_bytes);
                    const uint64_t ad = smem_desc(sa, row_bytes, (uint32_t)S.swz);
                    const uint64_t bd = smem_desc(sa + (uint32_t)S.a_bytes, row_bytes, (uint32_t)S.swz);
                    for (int k = 0; k < S.cblk / 16; ++k)
                        mma_bf16_ss(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, (kb | k) ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(&tfull[buf]);
            }
        }
    } else {
        int it = 0;
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
            const int buf = it & 1, ubuf = it >> 1;
            const bool have = mbar_wait(&tfull[buf], (uint32_t)(ubuf & 1));
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!__all_sync(0xffffffffu, have && !tc_failed())) break;   // warp-uniform: tcgen05.ld is .aligned
            int64_t p0;
            int img, y0, x0;
            tile_origin(A, t, p0, img, y0, x0);
            const int q = warp & 3;
            const int m = q * 32 + lane;
            const int64_t p = p0 + m;
            const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * S.ncols);
            epilogue_row(A, p, trow, (warp >> 2) * 16, 16 * (TCP_EPI_WARPS / 4));
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * S.ncols)
                     : "memory");
    }
}

// Halo form (Cin 16, 32 or 64, tiles inside one image row): per tile one
// TMA box per 8-channel chunk brings the three input rows the tile's taps
// read, 130 pixels wide (the tile and one pixel on each side; zero fill at
// the image border), in the canonical K-major layout without swizzle:
// [chunk][row][pixel][8 channels].  The A operand of tap (ky, kx) is then
// the same buffer started ky rows and kx pixels further (16-byte steps of
// the descriptor's start address), so the nine taps need no further loads.
// The weights of all nine taps stay resident in shared memory for the CTA's
// life ([tap][chunk][cout][8]).  Roles and bounded waits are those of
// conv3x3_tcp_kernel; where tensor memory holds four accumulator buffers
// per CTA, the eight epilogue warps form two groups of four that drain
// alternate tiles (buffers i % 4), so that two tiles' epilogues overlap.
constexpr int HALO_W = TC_M + 2;

struct HaloShape {
    int kch;         // Cin / 8
    int kstride;     // bytes of one chunk's three halo rows (128-byte multiple)
    int slot_bytes;  // kch * kstride
    int slots;
    int w_bytes;     // 9 * kch * Cout * 16
    int ncols;
    int groups;      // epilogue groups (1 or 2): group g drains tiles i with i % groups == g
    int nbuf;        // tensor-memory accumulator buffers: 2 per group
};

__device__ __forceinline__ uint64_t smem_desc_plain(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;   // next 8-element group along K
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;   // next 8 rows
    d |= (uint64_t)1 << 46;                          // descriptor version; layout 0: no swizzle
    return d;
}

__global__ void __launch_bounds__(TCP_THREADS, TCP_MAX_CTAS) conv3x3_tch_kernel(const __grid_constant__ CUtensorMap tmH,
                                                                               const __grid_constant__ CUtensorMap tmW,
                                                                               ConvArgs A, HaloShape S, int64_t tiles)
{
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t* wsm = sm;                                   // resident weights
    uint8_t* hsm = sm + S.w_bytes;                       // halo slots
    uint64_t* wbar = (uint64_t*)(hsm + (size_t)S.slots * S.slot_bytes);
    uint64_t* full = wbar + 1;
    uint64_t* empty = full + S.slots;
    uint64_t* tfull = empty + S.slots;                   // [nbuf]
    uint64_t* tempty = tfull + S.nbuf;                   // [nbuf]
    uint32_t* tslot = (uint32_t*)(tempty + S.nbuf);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gw = TCP_EPI_WARPS / S.groups;             // warps per epilogue group

    if (tid == 0) {
        mbar_init(wbar, 1);
        for (int s = 0; s < S.slots; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < S.nbuf; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], (uint32_t)gw);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(S.nbuf * S.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const int wchunk = A.Cout * 16;                      // bytes of one (tap, chunk) weight box

    if (warp == TCP_EPI_WARPS) {
        if (lane == 0) {
            mbar_expect_tx(wbar, (uint32_t)S.w_bytes);
            for (int t = 0; t < 9; ++t)
                for (int kc = 0; kc < S.kch; ++kc)
                    tma_load_3d(wsm + (size_t)(t * S.kch + kc) * wchunk, &tmW, 8 * kc, 0, t, wbar);
            int64_t it = 0;
            for (int64_t t = blockIdx.x; t < tiles && !tc_failed(); t += gridDim.x, ++it) {
                const int s = (int)(it % S.slots);
                const int64_t use = it / S.slots;
                if (use > 0 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1))) break;
                int64_t p0;
                int img, y0, x0;
                tile_origin(A, t, p0, img, y0, x0);
                uint8_t* slot = hsm + (size_t)s * S.slot_bytes;
                mbar_expect_tx(&full[s], (uint32_t)(S.kch * 3 * HALO_W * 16));
                if (it == 0 && blockIdx.x == 0 && *(volatile int*)&g_conv_tc_stall) continue;
                for (int kc = 0; kc < S.kch; ++kc)
                    tma_load_4d(slot + (size_t)kc * S.kstride, &tmH, 8 * kc, x0 - 1, y0 - 1, img, &full[s]);
            }
        }
    } else if (warp == TCP_EPI_WARPS + 1) {
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(A.Cout >> 3) << 17) |
                                   ((uint32_t)(TC_M >> 4) << 24);
            bool ok = mbar_wait(wbar, 0);
            const uint32_t wbase = smem_u32(wsm);
            int64_t it = 0;
            for (int64_t t = blockIdx.x; t < tiles && ok && !tc_failed(); t += gridDim.x, ++it) {
                const int buf = (int)(it % S.nbuf);
                const int64_t ubuf = it / S.nbuf;
                if (ubuf > 0 && !mbar_wait(&tempty[buf], (uint32_t)((ubuf - 1) & 1))) break;
                const int s = (int)(it % S.slots);
                const int64_t use = it / S.slots;
                if (!mbar_wait(&full[s], (uint32_t)(use & 1))) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * S.ncols);
                const uint32_t hbase = smem_u32(hsm + (size_t)s * S.slot_bytes);
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * ky;
                    for (int h = 0; h < S.kch / 2; ++h) {
                        const uint32_t sa = hbase + (uint32_t)(2 * h * S.kstride) + (uint32_t)((ky * HALO_W + kx) * 16);
                        const uint32_t sb = wbase + (uint32_t)((tap * S.kch + 2 * h) * wchunk);
                        mma_bf16_ss(d, smem_desc_plain(sa, (uint32_t)S.kstride, 128u),
                                    smem_desc_plain(sb, (uint32_t)wchunk, 128u), idesc, (tap | h) ? 1u : 0u);
                    }
                }
                mma_commit(&empty[s]);
                mma_commit(&tfull[buf]);
            }
        }
    } else {
        const int g = warp / gw, wi = warp - g * gw;
        const int q = wi & 3;                            // lane quarter (warp % 4 == wi % 4)
        for (int64_t it = g; blockIdx.x + it * gridDim.x < tiles; it += S.groups) {
            const int64_t t = blockIdx.x + it * gridDim.x;
            const int buf = (int)(it % S.nbuf);
            const int64_t ubuf = it / S.nbuf;
            const bool have = mbar_wait(&tfull[buf], (uint32_t)(ubuf & 1));
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!__all_sync(0xffffffffu, have && !tc_failed())) break;
            int64_t p0;
            int img, y0, x0;
            tile_origin(A, t, p0, img, y0, x0);
            const int64_t p = p0 + q * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * S.ncols);
            epilogue_row(A, p, trow, (wi >> 2) * 16, 16 * (gw / 4));
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S.nbuf * S.ncols)
                     : "memory");
    }
}

// ---- host ---------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    }
    return fn;
}

// Shapes the tensor-core kernel takes: Cin 16, 32 or a multiple of 64,
// Cout a multiple of 16 up to 256, tiles of 128 pixels within image rows,
// 16-byte aligned tensors.
bool conv_tc_supported(const ConvArgs& A)
{
    if (!(A.Cin == 16 || A.Cin == 32 || (A.Cin % 64 == 0 && A.Cin <= 1024))) return false;
    if (A.Cout < 16 || A.Cout > 256 || A.Cout % 16 || A.CoutStride % 16) return false;
    if (A.W >= TC_M ? (A.W % TC_M) != 0 : (TC_M % A.W) != 0) return false;
    if (((int64_t)A.H * A.W) % TC_M) return false;
    if (((uintptr_t)A.in | (uintptr_t)A.wt | (uintptr_t)A.out) & 15) return false;
    if (A.mask && ((uintptr_t)A.mask & 15)) return false;
    return encode_fn() != nullptr;
}

static TcShape tc_shape(const ConvArgs& A)
{
    TcShape S;
    S.cblk = A.Cin < 64 ? A.Cin : 64;
    S.chunks = A.Cin / S.cblk;
    S.kblocks = 9 * S.chunks;
    S.a_bytes = TC_M * S.cblk * 2;
    S.b_bytes = A.Cout * S.cblk * 2;
    S.swz = S.cblk == 16 ? 6 : S.cblk == 32 ? 4 : 2;
    int nc = 32;
    while (nc < A.Cout) nc <<= 1;
    S.ncols = nc;
    // a short ring (about 24 KB) so that many CTAs share an SM: on the U-Net's
    // layers at 256^2 .. 2048^2 that beat deeper pipelines (2.8 ms for the
    // 15 inference layers against 4.7 ms with a 96 KB ring)
    const int stage = S.a_bytes + S.b_bytes;
    int st = (24 * 1024) / stage;
    if (st < 2) st = 2;
    if (st > S.kblocks) st = S.kblocks;
    if (st > 8) st = 8;
    S.stages = st;
    return S;
}

static size_t tc_smem(const TcShape& S)
{
    return 1024 + (size_t)S.stages * (S.a_bytes + S.b_bytes) + (size_t)(2 * S.stages + 4) * 8 + 16;
}

// Persistent form: CTAs per SM as tensor memory allows (two accumulator
// buffers of ncols columns each, 512 columns per SM), at most 3, sharing a
// stage ring budget of 192 KB per SM, deep enough to keep the few-channel
// layers' loads streaming across tiles.
static int tcp_ctas_per_sm(const TcShape& S)
{
    const int c = 512 / (2 * S.ncols);
    return c < TCP_MAX_CTAS ? c : TCP_MAX_CTAS;
}

static TcShape tcp_shape(const ConvArgs& A)
{
    TcShape S = tc_shape(A);
    const int stage = S.a_bytes + S.b_bytes;
    const int ring = 192 * 1024 / tcp_ctas_per_sm(S);
    int st = ring / stage;
    if (st < 2) st = 2;
    if (st > 32) st = 32;
    S.stages = st;
    return S;
}

static int sm_count()
{
    static int dev_cached = -1, n = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev != dev_cached) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 0;
        dev_cached = dev;
    }
    return n;
}

// Halo form: Cin 16, 32 or 64, tiles inside one image row, the nine taps'
// weights at most 48 KB, and at least two CTAs per SM with at least two halo
// slots each (at most 6) within tensor memory and a 216 KB shared-memory
// budget.  With one CTA per SM the form was slower than the others
// (2048^2, 64 -> 32 channels: 619 us against 357-390 us).
static bool tch_shape(const ConvArgs& A, HaloShape& S, int& cps)
{
    if (!(A.Cin == 16 || A.Cin == 32 || A.Cin == 64) || A.W % TC_M) return false;
    S.kch = A.Cin / 8;
    S.kstride = ((3 * HALO_W * 16 + 127) / 128) * 128;
    S.slot_bytes = S.kch * S.kstride;
    S.w_bytes = 9 * S.kch * A.Cout * 16;
    if (S.w_bytes > 48 * 1024) return false;
    int nc = 32;
    while (nc < A.Cout) nc <<= 1;
    S.ncols = nc;
    cps = 512 / (2 * nc);
    if (cps > TCP_MAX_CTAS) cps = TCP_MAX_CTAS;
    for (; cps >= 2; --cps) {
        const int budget = 216 * 1024 / cps - 1024 - 256 - S.w_bytes;
        int sl = budget / S.slot_bytes;
        if (sl > 6) sl = 6;
        if (sl >= 2) {
            S.slots = sl;
            // two epilogue groups of four warps, each draining its own pair
            // of accumulator buffers, where tensor memory holds four per CTA
            S.groups = cps * 4 * nc <= 512 ? 2 : 1;
            S.nbuf = 2 * S.groups;
            return true;
        }
    }
    return false;
}

static size_t tch_smem(const HaloShape& S)
{
    return 1024 + (size_t)S.w_bytes + (size_t)S.slots * S.slot_bytes + (size_t)(1 + 2 * S.slots + 2 * S.nbuf) * 8 +
           16;
}

static cudaError_t launch_tch(const ConvArgs& A, const HaloShape& S, int cps, cudaStream_t s)
{
    EncodeTiledFn enc = encode_fn();
    alignas(64) CUtensorMap tmH, tmW;
    {   // activations (C, W, H, N); box: 8 channels x 130 pixels x 3 rows
        const cuuint64_t dims[4] = {(cuuint64_t)A.Cin, (cuuint64_t)A.W, (cuuint64_t)A.H, (cuuint64_t)A.N};
        const cuuint64_t strides[3] = {(cuuint64_t)A.Cin * 2, (cuuint64_t)A.W * A.Cin * 2,
                                       (cuuint64_t)A.H * A.W * A.Cin * 2};
        const cuuint32_t box[4] = {8, (cuuint32_t)HALO_W, 3, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&tmH, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)A.in, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {   // weights [9][Cout][Cin]: dims (Cin, Cout, 9); box: 8 channels x Cout
        const cuuint64_t dims[3] = {(cuuint64_t)A.Cin, (cuuint64_t)A.Cout, 9};
        const cuuint64_t strides[2] = {(cuuint64_t)A.Cin * 2, (cuuint64_t)A.Cout * A.Cin * 2};
        const cuuint32_t box[3] = {8, (cuuint32_t)A.Cout, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        if (enc(&tmW, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)A.wt, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    static int attr_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_dev != dev) {
        e = cudaFuncSetAttribute(conv3x3_tch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const int sms = sm_count();
    if (sms <= 0) return cudaErrorInvalidDevice;
    const int64_t tiles = (int64_t)A.N * A.H * A.W / TC_M;
    int64_t grid = (int64_t)sms * cps;
    if (grid > tiles) grid = tiles;
    conv3x3_tch_kernel<<<(unsigned)grid, TCP_THREADS, tch_smem(S), s>>>(tmH, tmW, A, S, tiles);
    return cudaGetLastError();
}

cudaError_t launch_conv3x3_tc(const ConvArgs& A, cudaStream_t s, int form)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc || !conv_tc_supported(A)) return cudaErrorNotSupported;
    bool persistent = form == 0 || form == 2;
    if (form == 0) {
        HaloShape H;
        int cps = 0;
        if (tch_shape(A, H, cps)) return launch_tch(A, H, cps, s);
        // without the halo form, few output channels favour one tile per CTA
        // (2048^2, 64 -> 32 channels: 357 us against 390 us persistent)
        if (A.Cout <= 32) persistent = false;
    }
    const TcShape S = persistent ? tcp_shape(A) : tc_shape(A);
    const CUtensorMapSwizzle swz = S.cblk == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                   : S.cblk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                  : CU_TENSOR_MAP_SWIZZLE_128B;
    alignas(64) CUtensorMap tmA, tmB;
    {   // activations: dims (C, W, H, N); box (cblk, bw, bh, 1) = 128 pixels
        const int bw = A.W >= TC_M ? TC_M : A.W;
        const int bh = TC_M / bw;
        const cuuint64_t dims[4] = {(cuuint64_t)A.Cin, (cuuint64_t)A.W, (cuuint64_t)A.H, (cuuint64_t)A.N};
        const cuuint64_t strides[3] = {(cuuint64_t)A.Cin * 2, (cuuint64_t)A.W * A.Cin * 2,
                                       (cuuint64_t)A.H * A.W * A.Cin * 2};
        const cuuint32_t box[4] = {(cuuint32_t)S.cblk, (cuuint32_t)bw, (cuuint32_t)bh, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)A.in, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {   // weights [9][Cout][Cin]: dims (Cin, Cout, 9); box (cblk, Cout, 1)
        const cuuint64_t dims[3] = {(cuuint64_t)A.Cin, (cuuint64_t)A.Cout, 9};
        const cuuint64_t strides[2] = {(cuuint64_t)A.Cin * 2, (cuuint64_t)A.Cout * A.Cin * 2};
        const cuuint32_t box[3] = {(cuuint32_t)S.cblk, (cuuint32_t)A.Cout, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        if (enc(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)A.wt, dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const size_t smem = tc_smem(S);
    static int attr_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_dev != dev) {
        e = cudaFuncSetAttribute(conv3x3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv3x3_tcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const int64_t tiles = (int64_t)A.N * A.H * A.W / TC_M;
    if (persistent) {
        const int sms = sm_count();
        if (sms <= 0) return cudaErrorInvalidDevice;
        int64_t grid = (int64_t)sms * tcp_ctas_per_sm(S);
        if (grid > tiles) grid = tiles;
        conv3x3_tcp_kernel<<<(unsigned)grid, TCP_THREADS, smem, s>>>(tmA, tmB, A, S, tiles);
    } else {
        conv3x3_tc_kernel<<<(unsigned)tiles, TC_THREADS, smem, s>>>(tmA, tmB, A, S);
    }
    return cudaGetLastError();
}

// Sets the stall test hook (see g_conv_tc_stall); < 0 on a CUDA error.
int conv_tc_set_stall(int on)
{
    return cudaMemcpyToSymbol(g_conv_tc_stall, &on, sizeof(int)) == cudaSuccess ? 0 : -1;
}

// 1 if a tensor-core convolution gave up waiting since the last call (and
// clears the flag), 0 if not, < 0 on a CUDA error.  Synchronises the device.
int conv_tc_take_error()
{
    int v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_conv_tc_error, sizeof(int)) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(g_conv_tc_error, &z, sizeof(int)) != cudaSuccess) return -1;
    return v;
}

}  // namespace nn
}  // namespace tvcut
