// 3x3 convolution on the tcgen05 tensor cores (implicit GEMM, BF16 operands, FP32
// accumulation in tensor memory); see umma.cu.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace tt {
// Whether the tensor-core convolution handles these channel counts.
bool conv3x3_umma_ok(int Cin, int Cout);
size_t conv3x3_umma_smem(int Cout);
// out[b][o][p] = act(bias[o] + sum W[o][c][tap] X[b][c][p + tap]) (zero padding),
// gated by (gate > 0) when gate is given, pre-activation into zout when given.
void conv3x3_umma(tt_ctx* c, int B, int Cin, int Cout, int nx, int ny, const float* X, const __nv_bfloat16* W,
                  const float* bias, int relu, const float* gate, float* zout, float* out);
}  // namespace tt
