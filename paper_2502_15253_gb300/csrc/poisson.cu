// Poisson pseudo-data on the device: n_i ~ Poisson(mu_i) for every element of a batch of
// expectations (the training set of the warm-start network is drawn this way).
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), a counter-based generator:
// element i of call (seed, offset) uses counters (i + offset, draw, 0, 0), so every element's
// stream is independent of the launch shape and reproducible. Sampling: the multiplication
// method (Knuth) for mu < 10, Hormann's transformed rejection with squeeze (PTRS, 1993) above.
#include <algorithm>
#include <cstdint>
#include <string>

#include "../../include/fitcore.h"
#include "philox.cuh"

int fitcore_fail(int code, const std::string &msg);
void fitcore_count_launch();

namespace fitcore {

namespace {

using rng::philox4x32_10;
using rng::u01;

constexpr float kMuMax = 4194304.f;   // 2^22: above, the float steps of PTRS lose integers

struct Stream {
    uint32_t c0, c1, k0, k1, draw;
    uint32_t buf[4];
    int left;
    __device__ float next() {
        if (left == 0) {
            uint32_t c[4] = {c0, c1, draw++, 0u};
            philox4x32_10(c, k0, k1);
            buf[0] = c[0];
            buf[1] = c[1];
            buf[2] = c[2];
            buf[3] = c[3];
            left = 4;
        }
        return u01(buf[4 - left--]);
    }
};

// Every float operation that decides the returned integer is written with explicit rounding
// (no contraction), so that a host implementation of the same steps in IEEE single and
// double precision takes the same decisions.
__device__ float poisson_draw(float mu, Stream &st) {
    if (!(mu > 0.f)) return mu == 0.f ? 0.f : NAN;
    if (!(mu < kMuMax)) return NAN;
    if (mu < 10.f) {
        // multiplication method: smallest k with u_0 u_1 ... u_k <= exp(-mu)
        const float L = (float)exp(-(double)mu);
        float p = 1.f;
        for (int k = 0; k < 1000; ++k) {
            p = __fmul_rn(p, st.next());
            if (p <= L) return (float)k;
        }
        return 1000.f;
    }
    // PTRS: transformed rejection with squeeze
    const float smu = sqrtf(mu);
    const float b = __fmaf_rn(2.53f, smu, 0.931f);
    const float a = __fmaf_rn(0.02483f, b, -0.059f);
    const float inv_alpha = __fadd_rn(1.1239f, __fdiv_rn(1.1328f, __fsub_rn(b, 3.4f)));
    const float vr = __fsub_rn(0.9277f, __fdiv_rn(3.6224f, __fsub_rn(b, 2.f)));
    const double lmu = log((double)mu);
    for (int it = 0; it < 1000; ++it) {
        const float U = __fsub_rn(st.next(), 0.5f);
        const float V = st.next();
        const float us = __fsub_rn(0.5f, fabsf(U));
        const float t = __fadd_rn(__fdiv_rn(__fmul_rn(2.f, a), us), b);
        const float k = floorf(__fadd_rn(__fadd_rn(__fmul_rn(t, U), mu), 0.43f));
        if (us >= 0.07f && V <= vr) return k;
        if (k < 0.f || (us < 0.013f && V > us)) continue;
        const double lhs = __dsub_rn(__dadd_rn(log((double)V), log((double)inv_alpha)),
                                     log(__dadd_rn(__ddiv_rn((double)a, __dmul_rn((double)us, (double)us)), (double)b)));
        const double rhs = __dsub_rn(__dadd_rn(-(double)mu, __dmul_rn((double)k, lmu)), lgamma((double)k + 1.0));
        if (lhs <= rhs) return k;
    }
    return rintf(mu);
}

__global__ void poisson_kernel(const float *__restrict__ mu, int64_t n, uint64_t seed, uint64_t offset,
                               float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ctr = (uint64_t)i + offset;
        Stream st{(uint32_t)ctr, (uint32_t)(ctr >> 32), (uint32_t)seed, (uint32_t)(seed >> 32), 0u, {0, 0, 0, 0}, 0};
        out[i] = poisson_draw(mu[i], st);
    }
}

}  // namespace

int poisson_sample(int64_t n, const float *mu, uint64_t seed, uint64_t offset, float *out, cudaStream_t s) {
    if (n <= 0) return FIT_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    poisson_kernel<<<grid, 256, 0, s>>>(mu, n, seed, offset, out);
    fitcore_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, std::string("fit_poisson_sample: ") + cudaGetErrorString(e));
    return FIT_OK;
}

}  // namespace fitcore
