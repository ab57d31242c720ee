// Internal interface of the tcgen05 BF16 GEMM (mlp.cu) for other kernels.
#pragma once
#include "common.cuh"

namespace drgb {

// partials[z][M][N] (FP32) = A[M x K] B[N x K]^T restricted to the z-th of
// the K splits, A and B row-major BF16 with K contiguous (device); M a
// multiple of 128, N of 64, K of 64.  *splits_used receives the number of
// K splits launched (at most `splits`).
int tc_gemm_nt_f32(Ctx* c, const void* A, const void* B, int M, int N, int K, int splits, float* partials,
                   int* splits_used, cudaStream_t st);

}  // namespace drgb
