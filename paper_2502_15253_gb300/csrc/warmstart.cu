// Training samples of the warm-start network, drawn on the device: parameter vectors theta
// (nuisances from their priors, the parameters of interest uniform in a window), a dataset
// mask per sample, and the standardised regression targets. The expected spectra, the Poisson
// pseudo-data and the log-normalised inputs come from batched.cu, poisson.cu and mlp.cu.
//
// Random numbers: Philox4x32-10 under key = seed; parameter i of sample b uses the counter
// (b + offset, i, 0x0D8A0001, 0) and its four words give a normal deviate (Box-Muller on words
// 0 and 1), a uniform (word 2) and, for i = 0, the mask choice (word 3).
#include <algorithm>
#include <cmath>
#include <string>

#include "dev_model.cuh"
#include "kernels.cuh"
#include "philox.cuh"

int fitcore_fail(int code, const std::string &msg);
void fitcore_count_launch();

namespace fitcore {

namespace {

constexpr uint32_t kDrawTag = 0x0D8A0001u;

// One block per sample. Individually constrained (or free) parameters: theta0 + zscale z;
// parameters of a covariance block: theta0 + L z over the block (L the Cholesky factor);
// listed parameters: theta0 + h (2u - 1), replacing the prior draw.
__global__ void __launch_bounds__(128) draw_kernel(const DevModel *__restrict__ gm, int B, uint64_t seed,
                                                   uint64_t offset, int n_uni, const int *__restrict__ uidx,
                                                   const double *__restrict__ uhalf, int n_masks,
                                                   const uint32_t *__restrict__ choices, double *__restrict__ theta,
                                                   uint32_t *__restrict__ masks, float *__restrict__ z_out) {
    extern __shared__ double z[];
    const DevModel &m = *gm;
    const int b = blockIdx.x, P = m.P;
    const uint64_t ctr = (uint64_t)b + offset;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    double *th = theta + (int64_t)b * P;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        uint32_t c[4] = {(uint32_t)ctr, (uint32_t)(ctr >> 32), (uint32_t)i, kDrawTag};
        rng::philox4x32_10(c, k0, k1);
        const double u1 = rng::u01(c[0]), u2 = rng::u01(c[1]);
        z[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
        const float zs = m.zscale[i];
        double v = m.theta0[i] + (double)zs * z[i];
        for (int t = 0; t < n_uni; ++t)
            if (uidx[t] == i) v = m.theta0[i] + uhalf[t] * (2.0 * (double)rng::u01(c[2]) - 1.0);
        th[i] = v;   // block rows are overwritten below
        if (i == 0 && masks) {
            uint32_t mk = 0xFFFFFFFFu;
            if (n_masks > 0) {
                int q = (int)(rng::u01(c[3]) * (float)n_masks);
                mk = choices[min(q, n_masks - 1)];
            }
            masks[b] = mk;
        }
    }
    __syncthreads();
    // covariance blocks: row r of the block = theta0 + sum_{c <= r} L[r][c] z[idx[c]]
    for (int k = 0; k < m.n_blocks; ++k) {
        const int n = m.blk_size[k];
        const int *idx = m.blk_idx + m.blk_idx_off[k];
        const double *L = m.blk_L64 + m.blk_mat_off[k];
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            const int p = idx[r];
            bool listed = false;
            for (int t = 0; t < n_uni; ++t) listed |= (uidx[t] == p);
            if (listed) continue;
            double acc = 0.0;
            for (int c = 0; c <= r; ++c) acc = fma(L[(int64_t)r * n + c], z[idx[c]], acc);
            th[p] = m.theta0[p] + acc;
        }
    }
    // whitened coordinates of the drawn point: the normal deviate inside a block, the
    // scaled offset elsewhere (a listed parameter's uniform draw included)
    if (z_out) {
        __syncthreads();
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const float zs = m.zscale[i];
            z_out[(int64_t)b * P + i] = zs > 0.f ? (float)((th[i] - m.theta0[i]) / (double)zs) : (float)z[i];
        }
    }
}

// Regression targets at the linearised maximum-likelihood point of each sample. For the drawn
// point z_t with expectation mu_t and counts n, one Gauss-Newton step on -2lnL with the
// expected Hessian at the nominal point, (J^T W J + Lambda) delta = J^T W (n - mu_t) -
// Lambda z_t, moves the point to where a fit would end (to first order); target t is
// y = (theta_p - theta0_p) / scale_t + zf_t delta_p, with delta_p = K1_t (n - mu_t) - K2_t z_t
// (rows of the solved system for the target's coordinate p, one pair per dataset-mask variant).
// One block per sample, one warp per target.
__global__ void mle_targets_kernel(int B, int P, int D, const double *__restrict__ theta,
                                   const double *__restrict__ theta0, const float *__restrict__ z,
                                   const float *__restrict__ cnt, const float *__restrict__ mu, int n_t,
                                   const int *__restrict__ idx, const double *__restrict__ scale,
                                   const float *__restrict__ K1, const float *__restrict__ K2,
                                   const float *__restrict__ zf, int n_var, const uint32_t *__restrict__ choices,
                                   const uint32_t *__restrict__ masks, int n_out, const int *__restrict__ status,
                                   float *__restrict__ y) {
    const int b = blockIdx.x, lane = threadIdx.x & 31, t = threadIdx.x >> 5;
    if (t >= n_out) return;
    float v = 0.f;
    if (t < n_t && !(status && status[b])) {
        int var = 0;
        if (n_var > 1 && masks)
            for (int q = 0; q < n_var; ++q)
                if (choices[q] == masks[b]) var = q;
        const float *k1 = K1 + ((int64_t)var * n_t + t) * D, *k2 = K2 + ((int64_t)var * n_t + t) * P;
        const float *nb = cnt + (int64_t)b * D, *mb = mu + (int64_t)b * D, *zb = z + (int64_t)b * P;
        float acc = 0.f;
        for (int j = lane; j < D; j += 32) acc = fmaf(k1[j], nb[j] - mb[j], acc);
        for (int i = lane; i < P; i += 32) acc = fmaf(-k2[i], zb[i], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        const int p = idx[t];
        v = (float)((theta[(int64_t)b * P + p] - theta0[p]) / scale[t]) + zf[var * n_t + t] * acc;
    }
    if (lane == 0) y[(int64_t)b * n_out + t] = v;
}

// y[b][t] -= sum_j Kt[var][t][j] (cnt[b][j] - mu0[j]): the target minus the linearised best
// fit from the nominal point (standardised rows Kt of the sample's dataset subset), so that the
// network learns the correction to the linearised start; a warp per (sample, target)
__global__ void lin_residual_targets_kernel(int D, int n_t, const float *__restrict__ Kt, const float *__restrict__ mu0,
                                            const float *__restrict__ cnt, int n_var,
                                            const uint32_t *__restrict__ choices, const uint32_t *__restrict__ masks,
                                            int n_out, const int *__restrict__ status, float *__restrict__ y) {
    const int b = blockIdx.x, lane = threadIdx.x & 31, t = threadIdx.x >> 5;
    if (t >= n_t || (status && status[b])) return;
    int var = 0;
    if (n_var > 1 && masks)
        for (int q = 0; q < n_var; ++q)
            if (choices[q] == masks[b]) var = q;
    const float *k = Kt + ((int64_t)var * n_t + t) * D, *nb = cnt + (int64_t)b * D;
    float acc = 0.f;
    for (int j = lane; j < D; j += 32) acc = fmaf(k[j], nb[j] - mu0[j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[(int64_t)b * n_out + t] -= acc;
}

// y[b][t] = (theta[b][idx_t] - theta0[idx_t]) / scale_t for t < n_t, 0 for n_t <= t < n_out
// and for samples whose expectation failed (status != 0)
__global__ void targets_kernel(int B, int P, const double *__restrict__ theta, const double *__restrict__ theta0,
                               int n_t, const int *__restrict__ idx, const double *__restrict__ scale, int n_out,
                               const int *__restrict__ status, float *__restrict__ y) {
    const int64_t total = (int64_t)B * n_out;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / n_out), t = (int)(e % n_out);
        float v = 0.f;
        if (t < n_t && !(status && status[b])) {
            const int p = idx[t];
            v = (float)((theta[(int64_t)b * P + p] - theta0[p]) / scale[t]);
        }
        y[e] = v;
    }
}

}  // namespace

int draw_theta(const DevModel &h, const DevModel *dev, int B, uint64_t seed, uint64_t offset, int n_uni,
               const int *uidx, const double *uhalf, int n_masks, const uint32_t *choices, double *theta,
               uint32_t *masks, cudaStream_t s, float *z_out) {
    const size_t smem = sizeof(double) * (size_t)h.P;
    if (smem > 48 * 1024) return fitcore_fail(FIT_ERR_INVALID_ARG, "warm-start draw: too many parameters");
    draw_kernel<<<B, 128, smem, s>>>(dev, B, seed, offset, n_uni, uidx, uhalf, n_masks, choices, theta, masks,
                                     z_out);
    fitcore_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, std::string("warm-start draw: ") + cudaGetErrorString(e));
    return FIT_OK;
}

int targets(int B, int P, const double *theta, const double *theta0, int n_t, const int *idx, const double *scale,
            int n_out, const int *status, float *y, cudaStream_t s) {
    const int64_t n = (int64_t)B * n_out;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
    targets_kernel<<<grid, 256, 0, s>>>(B, P, theta, theta0, n_t, idx, scale, n_out, status, y);
    fitcore_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, std::string("warm-start targets: ") + cudaGetErrorString(e));
    return FIT_OK;
}

int mle_targets(int B, int P, int D, const double *theta, const double *theta0, const float *z, const float *cnt,
                const float *mu, int n_t, const int *idx, const double *scale, const float *K1, const float *K2,
                const float *zf, int n_var, const uint32_t *choices, const uint32_t *masks, int n_out,
                const int *status, float *y, cudaStream_t s) {
    if (n_out > 32) return fitcore_fail(FIT_ERR_INVALID_ARG, "warm-start targets: more than 32 outputs");
    mle_targets_kernel<<<B, 32 * n_out, 0, s>>>(B, P, D, theta, theta0, z, cnt, mu, n_t, idx, scale, K1, K2, zf,
                                                n_var, choices, masks, n_out, status, y);
    fitcore_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, std::string("warm-start targets: ") + cudaGetErrorString(e));
    return FIT_OK;
}

int lin_residual_targets(int B, int D, int n_t, const float *Kt, const float *mu0, const float *cnt, int n_var,
                         const uint32_t *choices, const uint32_t *masks, int n_out, const int *status, float *y,
                         cudaStream_t s) {
    if (B == 0) return FIT_OK;
    lin_residual_targets_kernel<<<B, 32 * n_t, 0, s>>>(D, n_t, Kt, mu0, cnt, n_var, choices, masks, n_out, status, y);
    fitcore_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, std::string("warm-start residual targets: ") + cudaGetErrorString(e));
    return FIT_OK;
}

namespace {

// theta of the 2k perturbed points of each sample: row b 2k + 2q + s is theta_b with parameter
// o_param[q] moved by +h_q (s = 0) or -h_q (s = 1), h_q = hz zscale (a step of hz in z)
__global__ void perturb_kernel(int B, int P, int k, const double *__restrict__ theta, const int *__restrict__ o_param,
                               const float *__restrict__ zscale, double hz, double *__restrict__ out) {
    const int64_t total = (int64_t)B * 2 * k * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / P;
        const int i = (int)(e % P), b = (int)(row / (2 * k)), qs = (int)(row % (2 * k)), q = qs / 2;
        double v = theta[(int64_t)b * P + i];
        if (i == o_param[q]) v += (qs & 1 ? -hz : hz) * (double)zscale[i];
        out[e] = v;
    }
}

constexpr int kRefMaxK = 3;      // refreshed columns (mass splittings) at most

// Targets at the refreshed linearised best fit (see linear_mle_rows): one block per sample.
// Shared memory: r, J_o (k rows), y, Gp J_o (k rows) over the D bins, z_n over P_n.
__global__ void __launch_bounds__(256) refresh_targets_kernel(
    int B, int P, int D, int k, int Pn, int n_rows, const double *__restrict__ theta,
    const double *__restrict__ theta0, const float *__restrict__ z, const float *__restrict__ cnt,
    const float *__restrict__ mu, const float *__restrict__ mup, const int *__restrict__ st_p,
    const int *__restrict__ o_param, const int *__restrict__ n_param, const int *__restrict__ tkind,
    const float *__restrict__ lam_o, const float *__restrict__ bufs, int64_t var_floats, float inv2hz, int n_t,
    const int *__restrict__ idx, const double *__restrict__ scale, const float *__restrict__ zf, int n_var,
    const uint32_t *__restrict__ choices, const uint32_t *__restrict__ masks, int n_out,
    const int *__restrict__ status, float *__restrict__ y) {
    extern __shared__ float sh[];
    float *r = sh, *Jo = r + D, *yv = Jo + k * D, *GJ = yv + D, *zn = GJ + k * D;
    __shared__ float red[8][kRefMaxK * kRefMaxK + kRefMaxK];
    __shared__ float dlt[kRefMaxK];
    __shared__ int bad;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        int st = status ? status[b] : 0;
        for (int q = 0; q < 2 * k; ++q) st |= st_p[(int64_t)b * 2 * k + q];
        bad = st;
    }
    __syncthreads();
    if (bad) {
        for (int t = tid; t < n_out; t += blockDim.x) y[(int64_t)b * n_out + t] = 0.f;
        return;
    }
    int var = 0;
    if (n_var > 1 && masks)
        for (int q = 0; q < n_var; ++q)
            if (choices[q] == masks[b]) var = q;
    const float *Gp = bufs + (int64_t)var * var_floats, *Ht = Gp + (int64_t)D * D, *R1 = Ht + (int64_t)Pn * D,
                *R2 = R1 + (int64_t)n_rows * D;
    const float *zb = z + (int64_t)b * P;
    for (int j = tid; j < D; j += blockDim.x) {
        r[j] = cnt[(int64_t)b * D + j] - mu[(int64_t)b * D + j];
        for (int q = 0; q < k; ++q)
            Jo[q * D + j] = (mup[((int64_t)b * 2 * k + 2 * q) * D + j] - mup[((int64_t)b * 2 * k + 2 * q + 1) * D + j]) *
                            inv2hz;
    }
    for (int c = tid; c < Pn; c += blockDim.x) zn[c] = zb[n_param[c]];
    __syncthreads();
    // y = Gp r + H z_n and Gp J_o (Gp symmetric: column j read across the threads)
    for (int j = tid; j < D; j += blockDim.x) {
        float u = 0.f, g[kRefMaxK] = {0.f, 0.f, 0.f};
        for (int i = 0; i < D; ++i) {
            const float gij = Gp[(int64_t)i * D + j];
            u = fmaf(gij, r[i], u);
#pragma unroll
            for (int q = 0; q < kRefMaxK; ++q)
                if (q < k) g[q] = fmaf(gij, Jo[q * D + i], g[q]);
        }
        for (int c = 0; c < Pn; ++c) u = fmaf(Ht[(int64_t)c * D + j], zn[c], u);
        yv[j] = u;
        for (int q = 0; q < k; ++q) GJ[q * D + j] = g[q];
    }
    __syncthreads();
    // S = J_o^T Gp J_o, bv = J_o^T y (block sums)
    float part[kRefMaxK * kRefMaxK + kRefMaxK];
    const int ns = k * k + k;
    for (int e = 0; e < ns; ++e) part[e] = 0.f;
    for (int j = tid; j < D; j += blockDim.x)
        for (int q1 = 0; q1 < k; ++q1) {
            const float jq = Jo[q1 * D + j];
            for (int q2 = 0; q2 < k; ++q2) part[q1 * k + q2] = fmaf(jq, GJ[q2 * D + j], part[q1 * k + q2]);
            part[k * k + q1] = fmaf(jq, yv[j], part[k * k + q1]);
        }
    for (int e = 0; e < ns; ++e) {
        float v = part[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][e] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double S[kRefMaxK][kRefMaxK], bv[kRefMaxK];
        for (int q1 = 0; q1 < k; ++q1) {
            for (int q2 = 0; q2 < k; ++q2) {
                double acc = 0.0;
                for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) acc += red[wi][q1 * k + q2];
                S[q1][q2] = acc;
            }
            double acc = 0.0;
            for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) acc += red[wi][k * k + q1];
            S[q1][q1] += lam_o[q1];
            bv[q1] = acc - (double)lam_o[q1] * zb[o_param[q1]];
        }
        // Gaussian elimination with partial pivoting (k <= 3)
        for (int c = 0; c < k; ++c) {
            int pv = c;
            for (int rr = c + 1; rr < k; ++rr)
                if (fabs(S[rr][c]) > fabs(S[pv][c])) pv = rr;
            for (int cc = 0; cc < k; ++cc) {
                const double t = S[c][cc];
                S[c][cc] = S[pv][cc];
                S[pv][cc] = t;
            }
            const double tb = bv[c];
            bv[c] = bv[pv];
            bv[pv] = tb;
            const double piv = S[c][c];
            for (int rr = c + 1; rr < k; ++rr) {
                const double f = piv != 0.0 ? S[rr][c] / piv : 0.0;
                for (int cc = c; cc < k; ++cc) S[rr][cc] -= f * S[c][cc];
                bv[rr] -= f * bv[c];
            }
        }
        for (int c = k - 1; c >= 0; --c) {
            double acc = bv[c];
            for (int cc = c + 1; cc < k; ++cc) acc -= S[c][cc] * (double)dlt[cc];
            dlt[c] = S[c][c] != 0.0 ? (float)(acc / S[c][c]) : 0.f;
        }
    }
    __syncthreads();
    // targets: a warp per target
    for (int t = warp; t < n_out; t += blockDim.x >> 5) {
        float v = 0.f;
        if (t < n_t) {
            const int kind = tkind[t];
            float d = 0.f;
            if (kind >= 0) {
                d = dlt[kind];
            } else {
                const int row = -1 - kind;
                float acc = 0.f;
                for (int j = lane; j < D; j += 32) {
                    float rj = r[j];
                    for (int q = 0; q < k; ++q) rj = fmaf(-Jo[q * D + j], dlt[q], rj);
                    acc = fmaf(R1[(int64_t)row * D + j], rj, acc);
                }
                for (int c = lane; c < Pn; c += 32) acc = fmaf(-R2[(int64_t)row * Pn + c], zn[c], acc);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                d = acc;
            }
            const int p = idx[t];
            v = (float)((theta[(int64_t)b * P + p] - theta0[p]) / scale[t]) + zf[var * n_t + t] * d;
        }
        if (lane == 0) y[(int64_t)b * n_out + t] = v;
    }
}

}  // namespace

int perturb_theta(int B, int P, int k, const double *theta, const int *o_param, const float *zscale, double hz,
                  double *out, cudaStream_t s) {
    const int64_t n = (int64_t)B * 2 * k * P;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
    perturb_kernel<<<grid, 256, 0, s>>>(B, P, k, theta, o_param, zscale, hz, out);
    fitcore_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, std::string("warm-start refresh: ") + cudaGetErrorString(e));
    return FIT_OK;
}

int refresh_targets(int B, int P, int D, int k, int Pn, int n_rows, const double *theta, const double *theta0,
                    const float *z, const float *cnt, const float *mu, const float *mup, const int *st_p,
                    const int *o_param, const int *n_param, const int *tkind, const float *lam_o, const float *bufs,
                    int64_t var_floats, double hz, int n_t, const int *idx, const double *scale, const float *zf,
                    int n_var, const uint32_t *choices, const uint32_t *masks, int n_out, const int *status, float *y,
                    cudaStream_t s) {
    if (k < 1 || k > kRefMaxK) return fitcore_fail(FIT_ERR_INVALID_ARG, "warm-start refresh: 1..3 columns");
    const size_t smem = sizeof(float) * ((size_t)(2 + 2 * k) * D + Pn);
    if (smem > 48 * 1024) return fitcore_fail(FIT_ERR_INVALID_ARG, "warm-start refresh: model too large");
    refresh_targets_kernel<<<B, 256, smem, s>>>(B, P, D, k, Pn, n_rows, theta, theta0, z, cnt, mu, mup, st_p, o_param,
                                                n_param, tkind, lam_o, bufs, var_floats, (float)(0.5 / hz), n_t, idx,
                                                scale, zf, n_var, choices, masks, n_out, status, y);
    fitcore_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, std::string("warm-start refresh: ") + cudaGetErrorString(e));
    return FIT_OK;
}

}  // namespace fitcore
