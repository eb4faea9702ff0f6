// Arguments of a 3x3 convolution layer (NHWC BF16 activations, weights
// [9][Cout][Cin]), shared by the mma.sync kernels (unet_kernels.cuh) and the
// tcgen05 kernel (conv_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tvcut {
namespace nn {

struct ConvArgs {
    const __nv_bfloat16* in;    // N x H x W x Cin
    const __nv_bfloat16* wt;    // 9 x Cout x Cin
    const float* bias;          // Cout or nullptr
    __nv_bfloat16* out;         // N x H x W x CoutStride (channels >= Cout untouched)
    float* out_f32;             // optional FP32 copy (N x H x W x Cout) or nullptr
    const __nv_bfloat16* mask;  // optional: out *= (mask > 0), same layout as out
    int N, H, W, Cin, Cout, CoutStride;
    int relu;
};

// tcgen05 implicit-GEMM convolution (conv_tc.cu): the shapes it takes, its
// launch (cudaErrorNotSupported otherwise), and its give-up flag.
bool conv_tc_supported(const ConvArgs& A);
// form 0: persistent, warp-specialised, halo-loaded A operand where the
// shape allows (default); 1: one 128-pixel tile per CTA; 2: persistent
// without the halo form
cudaError_t launch_conv3x3_tc(const ConvArgs& A, cudaStream_t s, int form = 0);
int conv_tc_take_error();
int conv_tc_set_stall(int on);

}  // namespace nn
}  // namespace tvcut
