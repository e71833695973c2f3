// Learned warm-start network: shared declarations of the tensor-core
// convolution and the element-wise kernels (unet.cu) used by the network
// driver (unet_net.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace purify {

using bf16 = __nv_bfloat16;

struct ConvArgs {
    const bf16* in;          // NHWC, channel stride in_cs, first channel in_co
    int B, H, W, Cin, in_cs, in_co;
    const bf16* w;           // [Npad][k][k][Cinp], zero padded
    int k, Cinp, Npad;
    const float* bias;       // [Cout] or null
    int Cout, relu;
    bf16* out;               // NHWC BF16 (channel stride out_cs, offset out_co) or null
    int out_cs, out_co;
    float* out_f32;          // NHWC FP32 [pixels][Cout] or null
    const float* residual;   // added to out_f32 when not null ([pixels][Cout])
    int* err;                // set to 1 when a bounded wait gives up
    int up;                  // 1: the input is the (H/2, W/2) image read through a x2 nearest upsampling
};

void conv_tc_launch(const ConvArgs& a, cudaStream_t st);
int round16(int v);
__global__ void k_f32_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, int64_t n);
__global__ void k_pack_weights(const float* __restrict__ w, bf16* __restrict__ wp, int Cout, int k, int Cin, int Npad,
                               int Cinp);

}  // namespace purify
