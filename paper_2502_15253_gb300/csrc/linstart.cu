// Start points from the linearised best fit (see fit_linear_start in capi.cu): the residuals of
// each pseudo-experiment against the nominal expectation, their product with the model's
// rows K on the tensor cores (per dataset subset the split-TF32 product Rh Kh^T + Rh Kl^T +
// Rl Kh^T, which keeps FP32 accuracy: the rows of strongly correlated nuisances cancel), and
// the start theta0 + delta in double.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/fitcore.h"
#include "gemm_tc.cuh"

int fitcore_fail(int code, const std::string &msg);
void fitcore_count_launch();

namespace {

// nearest value with a 10-bit mantissa (a TF32 operand read exactly by the tensor cores)
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// r = data[b][j] - mu0[j] for j < D (0 in the padding columns up to Dp), split into its TF32
// part Rh and the rest Rl
__global__ void lin_residual_kernel(int B, int D, int Dp, const float *__restrict__ data,
                                    const float *__restrict__ mu0, float *__restrict__ Rh, float *__restrict__ Rl) {
    const int64_t total = (int64_t)B * Dp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / Dp), j = (int)(e % Dp);
        const float r = j < D ? data[(int64_t)b * D + j] - mu0[j] : 0.f;
        const float h = tf32_round(r);
        Rh[e] = h;
        Rl[e] = r - h;
    }
}

// theta[b][i] = theta0[i] + delta_{sel[b]}[b][i]; delta of subset v at [(v * B + b) * Pp + i]
__global__ void lin_combine_kernel(int B, int P, int Pp, const double *__restrict__ theta0,
                                   const float *__restrict__ delta, const int *__restrict__ sel,
                                   double *__restrict__ theta) {
    const int64_t total = (int64_t)B * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / P), i = (int)(e % P);
        theta[e] = theta0[i] + (double)delta[((int64_t)sel[b] * B + b) * Pp + i];
    }
}

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

namespace fitcore {

// theta_out [B x P] (device) = theta0 + K_{v(b)} (data_b - mu0) with K_v (device, one per
// dataset subset v, theta space: [P x Dp] TF32 part then [P x Dp] rest), sel [B] (device) the
// subset of each instance. Asynchronous on s; the scratch comes from the stream-ordered pool.
int linear_start_apply(int B, int P, int D, const double *theta0_dev, const float *mu0_dev, const float *data,
                       const float *const *K, int n_var, const int *sel_dev, double *theta_out, cudaStream_t s) {
    const int Dp = (D + 3) & ~3, Pp = (P + 3) & ~3;
    float *R = nullptr, *delta = nullptr;
    if (cudaMallocAsync(&R, sizeof(float) * 2 * (size_t)B * Dp, s) != cudaSuccess ||
        cudaMallocAsync(&delta, sizeof(float) * (size_t)n_var * B * Pp, s) != cudaSuccess) {
        cudaGetLastError();
        if (R) cudaFreeAsync(R, s);
        return fitcore_fail(FIT_ERR_OOM, "fit_linear_start: workspace");
    }
    float *Rh = R, *Rl = R + (size_t)B * Dp;
    lin_residual_kernel<<<grid_for((int64_t)B * Dp), 256, 0, s>>>(B, D, Dp, data, mu0_dev, Rh, Rl);
    fitcore_count_launch();
    int rc = FIT_OK;
    for (int v = 0; v < n_var && rc == FIT_OK; ++v) {
        const float *Kh = K[v], *Kl = K[v] + (size_t)P * Dp;
        GemmOut o;
        o.C = delta + (size_t)v * B * Pp;
        o.ldc = Pp;
        o.deterministic = true;   // the same data give the same start on every call
        o.epi = EPI_F32;
        rc = tc_gemm(true, B, P, D, Rh, Dp, Kh, Dp, o, s, nullptr);
        o.epi = EPI_F32_ADD;
        if (rc == FIT_OK) rc = tc_gemm(true, B, P, D, Rh, Dp, Kl, Dp, o, s, nullptr);
        if (rc == FIT_OK) rc = tc_gemm(true, B, P, D, Rl, Dp, Kh, Dp, o, s, nullptr);
    }
    if (rc == FIT_OK) {
        lin_combine_kernel<<<grid_for((int64_t)B * P), 256, 0, s>>>(B, P, Pp, theta0_dev, delta, sel_dev, theta_out);
        fitcore_count_launch();
        if (cudaGetLastError() != cudaSuccess) rc = fitcore_fail(FIT_ERR_CUDA, "fit_linear_start: launch");
    }
    cudaFreeAsync(R, s);
    cudaFreeAsync(delta, s);
    return rc;
}

}  // namespace fitcore
