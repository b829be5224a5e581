// Correction network on tcgen05 tensor cores (BF16 operands, FP32 accumulation
// in tensor memory).  Work in progress: only the weight conversion exists yet.
#include <cuda_bf16.h>

#include "pl_device.cuh"
#include "pl_kernels.h"

namespace pl {

size_t bf16_weight_elems() { return 128 * 64 + 128 * 128 + 64 * 128; }

__global__ void k_convert_weights_bf16(const float* __restrict__ w32, uint16_t* __restrict__ wb) {
    // W2 [128x64], W3 [128x128], W4 [64x128] copied in blob order, rounded to nearest even.
    const int off_w2 = 64 * 2 + 64;
    const int off_w3 = off_w2 + 128 * 64 + 128;
    const int off_w4 = off_w3 + 128 * 128 + 128;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 32768; k += gridDim.x * blockDim.x) {
        float v;
        if (k < 8192) v = w32[off_w2 + k];
        else if (k < 8192 + 16384) v = w32[off_w3 + (k - 8192)];
        else v = w32[off_w4 + (k - 8192 - 16384)];
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        wb[k] = *reinterpret_cast<uint16_t*>(&b);
    }
}

cudaError_t launch_convert_weights_bf16(const float* w32, uint16_t* wbf16, cudaStream_t s) {
    k_convert_weights_bf16<<<32, 256, 0, s>>>(w32, wbf16);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_tc(const LatticeView& v, cudaStream_t s) {
    (void)v;
    (void)s;
    return cudaErrorNotSupported;
}

}  // namespace pl
