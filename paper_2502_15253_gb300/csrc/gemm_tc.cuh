// Tensor-core GEMM on sm_103a: D = A B^T with A [M x K] and B [N x K] row-major (K-major),
// bf16 (kind::f16) or FP32 read as TF32 (kind::tf32) operands, FP32 accumulation in tensor
// memory, and a fused epilogue. Used by the warm-start MLP (bf16) and the batched response
// fold (TF32 / split 3xTF32).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace fitcore {

enum GemmEpi : int {
    EPI_F32 = 0,        // C = D                                   (fp32)
    EPI_BIAS_F32 = 1,   // C = D + bias[n]                         (fp32)
    EPI_BIAS_GELU = 2,  // C = D + bias[n] (fp32, pre-activation), Y = gelu(C) (bf16)
    EPI_DGELU = 3,      // Y = D * gelu'(aux[m][n])                (bf16)
    EPI_F32_ADD = 4,    // C += D                                  (fp32)
};

struct GemmOut {
    int epi = EPI_F32;
    float *C = nullptr;
    int ldc = 0;
    __nv_bfloat16 *Y = nullptr;
    int ldy = 0;
    const float *bias = nullptr;
    const float *aux = nullptr;
    int ldaux = 0;
    // optional transposed copy of Y (EPI_BIAS_GELU, EPI_DGELU): Yt[n * ldyt + m] = Y[m][n], so
    // that a later product over the batch (a weight gradient) reads it K-major without a
    // separate transpose
    __nv_bfloat16 *Yt = nullptr;
    int ldyt = 0;
    int vec = 0;   // set by tc_gemm: bit 0 C, 1 Y, 2 aux, 3 Yt rows 16-byte aligned; bit 4 bias aligned
    // never split K over CTAs (the split adds partial tiles with atomics, so its FP32 sums
    // depend on their order): results identical from call to call
    bool deterministic = false;
};

// Returns 0, or a negative FIT_ERR_* code (message through the library's error string).
// A: M x K, lda elements per row; B: N x K, ldb per row; element type bf16 (tf32 = false) or
// float (tf32 = true). Rows of A and B must start 16-byte aligned. err: device int that the
// kernel ORs with 1/2/4 if a pipeline wait timed out (nullptr = library scratch).
int tc_gemm(bool tf32, int M, int N, int K, const void *A, int lda, const void *B, int ldb, const GemmOut &out,
            cudaStream_t stream, int *err_dev);

// Reads and clears the pipeline-timeout flag of tc_gemm launches that used the library's own
// flag (synchronises the device): 0 = no timeout.
int tc_gemm_take_error();

}  // namespace fitcore
