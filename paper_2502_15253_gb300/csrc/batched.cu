// Batched expectation with the response fold on tensor cores: for B parameter vectors,
//   V_d[b][k] = (M(a) u)_k        energy-corrected true spectrum of dataset d (CUDA cores)
//   F_d = V_d R_d^T               fold, one GEMM per dataset (tcgen05, TF32 or split 3xTF32)
//   mu[b][d][j] = eps F + backgrounds
// The fold is the one dense contraction of the path: one response matrix times many spectra.
// Plain TF32 keeps 11 significant bits per operand (training-set generation for the warm
// start); the split form F = Vh Rh^T + Vh Rl^T + Vl Rh^T, with x = xh + xl and xh exact in TF32,
// restores FP32-level accuracy where the expectation is compared with the FP64 oracle.
#include <algorithm>
#include <cstring>
#include <string>

#include "gemm_tc.cuh"
#include "kernels.cuh"

int fitcore_fail(int code, const std::string &msg);
void fitcore_count_launch();

namespace fitcore {

namespace {

// TF32-exact round-to-nearest of x (10 explicit mantissa bits), as a float
__device__ __forceinline__ float tf32_round(float x) {
    uint32_t b = __float_as_uint(x);
    b = (b + 0x1000u) & 0xFFFFE000u;
    return __uint_as_float(b);
}

// One block per (instance b, dataset d): survival (FP32 float-pair phases and the fitted
// sin^2(pi r) polynomial, as the event kernel) x reweights on the true grid, energy
// correction gathered per target bin, written as V_hi / V_lo rows of length ldt. Blocks of
// dataset 0 also store the instance's parameter pairs for the epilogue.
__global__ void __launch_bounds__(256) signal_v_kernel(const DevModel *__restrict__ gm, int B,
                                                       const double *__restrict__ theta, float *__restrict__ vhi,
                                                       float *__restrict__ vlo, float *__restrict__ pv_out,
                                                       float *__restrict__ pd_out, int *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DevModel &m = *reinterpret_cast<DevModel *>(smem_raw);
    {
        const int n = (int)(sizeof(DevModel) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(gm);
        int *dst = reinterpret_cast<int *>(smem_raw);
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    float *pv = reinterpret_cast<float *>(smem_raw + sizeof(DevModel));
    float *pd = pv + m.P;
    float *u = pd + m.P;
    __shared__ OscCoefN<6> kco;
    const int b = blockIdx.x, d = blockIdx.y, tid = threadIdx.x, nth = blockDim.x;
    const DevDataset &ds = m.ds[d];
    const int N_t = m.N_t;
    const double *th = theta + (int64_t)b * m.P;
    for (int i = tid; i < m.P; i += nth) {
        const double t = th[i];
        pv[i] = (float)t;
        pd[i] = (float)(t - m.theta0[i]);
        if (d == 0) {
            pv_out[(int64_t)b * m.P + i] = pv[i];
            pd_out[(int64_t)b * m.P + i] = pd[i];
        }
    }
    float eta[kMaxOsc], eta_lo[kMaxOsc];
#pragma unroll
    for (int i = 0; i < kMaxOsc; ++i) {
        const int p = i < m.n_osc ? m.osc_idx[i] : -1;
        if (osc_is_dm(m.osc_mode, i)) {
            eta[i] = p >= 0 ? m.theta0_f[p] : m.osc_val[i];
            eta_lo[i] = p >= 0 ? m.theta0_lo[p] + (float)(th[p] - m.theta0[p]) : m.osc_val_lo[i];
        } else {
            eta[i] = p >= 0 ? (float)th[p] : m.osc_val[i];
            eta_lo[i] = 0.f;
        }
    }
    if (tid == 0) {
        double e[kMaxOsc];
        for (int i = 0; i < kMaxOsc; ++i)
            e[i] = i >= m.n_osc ? 0.0 : (m.osc_idx[i] >= 0 ? th[m.osc_idx[i]] : m.osc_val_d[i]);
        double c[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (m.osc_mode == FIT_OSC_EQ1) {
            const double c2 = 0.5 * (1.0 + sqrt(fmax(1.0 - e[0], 0.0)));
            c[0] = e[0];
            c[1] = c2 * c2 * e[2];
        } else {
            const double S12 = 4.0 * e[0] * (1.0 - e[0]), S13 = 4.0 * e[1] * (1.0 - e[1]);
            double C4 = 1.0;   // cos^4 th14 (3+1 formula; 1 without a sterile state)
            if (m.osc_mode == FIT_OSC_STERILE4) {
                const double c14 = 0.5 * (1.0 + sqrt(fmax(1.0 - e[4], 0.0)));
                C4 = c14 * c14;
                c[3] = e[4] * (1.0 - e[1]) * (1.0 - e[0]);
                c[4] = e[4] * (1.0 - e[1]) * e[0];
                c[5] = e[4] * e[1];
            }
            c[0] = C4 * (1.0 - e[1]) * (1.0 - e[1]) * S12;
            c[1] = C4 * S13 * (1.0 - e[0]);
            c[2] = C4 * S13 * e[0];
        }
        for (int i = 0; i < 6; ++i) {
            kco.hi[i] = (float)c[i];
            kco.lo[i] = (float)(c[i] - (double)kco.hi[i]);
        }
    }
    __syncthreads();
    const OscCoefN<6> kc6 = kco;
    // the phases of the sin^2 terms in the order of the coefficients: Eq. 1: x_ee, x_21;
    // three-flavour: x_21, x_31, x_32; 3+1: and x_41, x_42, x_43 (mass splittings as float pairs)
    float pdm[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, pdl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int nph;
    {
        // normalised pairs: sin2_phase needs the low part to stay below an ulp of the high one
        // (the parameter offset sits in eta_lo here), so that the reduced phase is within 1/2
        auto pr = [&](int i) { return f2_norm(eta[i], eta_lo[i]); };
        auto sub = [](F2 a, F2 b) { return f2_add(a, F2{-b.h, -b.l}); };
        F2 d[6];
        if (m.osc_mode == FIT_OSC_EQ1) {
            nph = 2;
            d[0] = pr(1);
            d[1] = pr(3);
        } else {
            nph = 3;
            d[0] = pr(2);
            d[1] = pr(3);
            d[2] = sub(pr(3), pr(2));
            if (m.osc_mode == FIT_OSC_STERILE4) {
                nph = 6;
                d[3] = pr(5);
                d[4] = sub(pr(5), pr(2));
                d[5] = sub(pr(5), pr(3));
            }
        }
        for (int i = 0; i < nph; ++i) {
            pdm[i] = d[i].h;
            pdl[i] = d[i].l;
        }
    }
    const PP nrm = ppair(m, pv, pd, ds.norm_idx, 1.f);
    const EMap em = make_emap(m, ds, pv, pd);
    {
        const float s0 = em.slope(m.e_edge[0]), s1 = em.slope(m.e_edge[N_t]);
        if (!(s0 > 0.25f && s0 < 4.f && s1 > 0.25f && s1 < 4.f)) {
            if (tid == 0) atomicOr(&status[b], kStEscale);
            for (int k = tid; k < m.ldt; k += nth) {
                vhi[((int64_t)d * B + b) * m.ldt + k] = 0.f;
                vlo[((int64_t)d * B + b) * m.ldt + k] = 0.f;
            }
            return;
        }
    }
    for (int k = tid; k < N_t; k += nth) {
        const float ih = m.inv_e_hi[k], il = m.inv_e_lo[k];
        float pt = 0.f;
        for (int c = 0; c < m.C; ++c) {
            const float w = ds.w[c];
            if (w == 0.f) continue;
            const float ch = ds.kl_hi[c] * ih;
            const float cl = fmaf(ds.kl_hi[c], ih, -ch) + ds.kl_hi[c] * il + ds.kl_lo[c] * ih;
            // P = 1 - sum_i C_i sin^2(x_i) with the fitted sin^2(pi r) polynomial (no
            // derivatives are needed here)
            float P = 1.f;
#pragma unroll
            for (int i = 0; i < 6; ++i)
                if (i < nph) P -= cterm(kc6, i, sin2_phase(pdm[i], pdl[i], ch, cl));
            pt += pmul(ppair(m, pv, pd, m.core_power_idx[c], 1.f), w * P);
        }
        const float ts = pmul(ppair(m, pv, pd, ds.shape_idx[k], 1.f), ds.t[k]);
        u[k] = pmul(nrm, ts * pt);
    }
    __syncthreads();
    for (int t = tid; t < m.ldt; t += nth) {
        float acc = 0.f;
        if (t < N_t && m.remap_mode == FIT_REMAP_SPLINE) {
            acc = spline_target(u, m.e_edge, em, t, N_t);
        } else if (t < N_t) {
            int k = t - (int)floorf(em.disp(m.e_edge[t]));
            k = min(max(k, 0), N_t - 1);
            k = t - (int)floorf(em.disp(m.e_edge[k]));
            k = min(max(k - 1, 0), N_t - 1);
            while (k > 0 && (float)(k - t) + em.disp(m.e_edge[k]) > 0.f) --k;
            float dlo = em.disp(m.e_edge[k]);
            for (int it = 0; it < 64 && k < N_t; ++it, ++k) {
                const float dhi = em.disp(m.e_edge[k + 1]);
                const float ylo = (float)(k - t) + dlo, yhi = (float)(k + 1 - t) + dhi;
                if (ylo >= 1.f) break;
                const float ov = fminf(yhi, 1.f) - fmaxf(ylo, 0.f);
                if (ov > 0.f) acc = fmaf(u[k], ov / (1.f + (dhi - dlo)), acc);
                dlo = dhi;
            }
        }
        const float hi = tf32_round(acc);
        vhi[((int64_t)d * B + b) * m.ldt + t] = hi;
        vlo[((int64_t)d * B + b) * m.ldt + t] = acc - hi;
    }
}

// mu[b][off_d + j] = eps_d F_d[b][j] + sum_b r B (1 + delta); status bits become FIT_STATUS_*
__global__ void mu_epilogue_kernel(const DevModel *__restrict__ gm, int B, const float *__restrict__ F,
                                   int ldf, const float *__restrict__ pv_all, const float *__restrict__ pd_all,
                                   float *__restrict__ mu, int *__restrict__ status) {
    const DevModel &m = *gm;
    const int64_t total = (int64_t)B * m.n_data;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / m.n_data), q = (int)(e % m.n_data);
        int d = 0;
        while (d + 1 < m.n_ds && m.ds[d + 1].data_off <= q) ++d;
        const int j = q - m.ds[d].data_off;
        const DevDataset &ds = m.ds[d];
        const float *pv = pv_all + (int64_t)b * m.P, *pd = pd_all + (int64_t)b * m.P;
        const float f = F[((int64_t)d * B + b) * ldf + j];
        float v = pmul(ppair(m, pv, pd, ds.eff_idx, 1.f), f);
        for (int k = ds.bkg_begin; k < ds.bkg_end; ++k) {
            const DevBkg &bk = m.bkg[k];
            const float tm = bk.tmpl[j];
            const float shaped = bk.shape_idx[j] >= 0 ? fmaf(tm, pv[bk.shape_idx[j]], tm) : tm;
            v += pmul(ppair(m, pv, pd, bk.rate_idx, 1.f), shaped);
        }
        mu[e] = status[b] ? NAN : v;
    }
}

__global__ void status_finish_kernel(int B, int *status) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
        status[b] = (status[b] & kStEscale) ? FIT_STATUS_ESCALE_NONMONOTONE : 0;
}

}  // namespace

// theta, mu, status: device buffers. precision 0 = TF32 fold, 1 = split 3xTF32 fold.
int expected_tc(const DevModel &h, const DevModel *dev, int B, const double *theta, float *mu, int *status,
                int precision, cudaStream_t s) {
    const int nds = h.n_ds, ldt = h.ldt;
    int ldf = 0;
    for (int d = 0; d < nds; ++d) ldf = std::max(ldf, h.ds[d].n_reco);
    ldf = (ldf + 3) / 4 * 4;
    float *vhi = nullptr, *vlo = nullptr, *F = nullptr, *pv = nullptr, *pd = nullptr;
    auto cleanup = [&]() {
        for (float *p : {vhi, vlo, F, pv, pd})
            if (p) cudaFreeAsync(p, s);
    };
    if (cudaMallocAsync(&vhi, sizeof(float) * (size_t)nds * B * ldt, s) ||
        cudaMallocAsync(&vlo, sizeof(float) * (size_t)nds * B * ldt, s) ||
        cudaMallocAsync(&F, sizeof(float) * (size_t)nds * B * ldf, s) ||
        cudaMallocAsync(&pv, sizeof(float) * (size_t)B * h.P, s) ||
        cudaMallocAsync(&pd, sizeof(float) * (size_t)B * h.P, s)) {
        cudaGetLastError();
        cleanup();
        return fitcore_fail(FIT_ERR_OOM, "fit_model_expected_tc: workspace");
    }
    cudaMemsetAsync(status, 0, sizeof(int) * B, s);
    const size_t smem = sizeof(DevModel) + sizeof(float) * (2 * (size_t)h.P + h.N_t);
    cudaFuncSetAttribute(signal_v_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    signal_v_kernel<<<dim3(B, nds), 256, smem, s>>>(dev, B, theta, vhi, vlo, pv, pd, status);
    fitcore_count_launch();
    int rc = FIT_OK;
    for (int d = 0; d < nds && rc == FIT_OK; ++d) {
        const DevDetector &dt = h.det[h.ds[d].det];
        GemmOut o;
        o.epi = EPI_F32;
        o.C = F + (size_t)d * B * ldf;
        o.ldc = ldf;
        const float *Vh = vhi + (size_t)d * B * ldt, *Vl = vlo + (size_t)d * B * ldt;
        rc = tc_gemm(true, B, dt.n_reco, h.N_t, Vh, ldt, dt.rdense_hi, ldt, o, s, nullptr);
        if (rc == FIT_OK && precision == 1) {
            o.epi = EPI_F32_ADD;
            rc = tc_gemm(true, B, dt.n_reco, h.N_t, Vh, ldt, dt.rdense_lo, ldt, o, s, nullptr);
            if (rc == FIT_OK) rc = tc_gemm(true, B, dt.n_reco, h.N_t, Vl, ldt, dt.rdense_hi, ldt, o, s, nullptr);
        }
    }
    if (rc == FIT_OK) {
        mu_epilogue_kernel<<<std::min<int64_t>(((int64_t)B * h.n_data + 255) / 256, 4096), 256, 0, s>>>(
            dev, B, F, ldf, pv, pd, mu, status);
        status_finish_kernel<<<(B + 255) / 256, 256, 0, s>>>(B, status);
        fitcore_count_launch();
        fitcore_count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = fitcore_fail(FIT_ERR_CUDA, std::string("fit_model_expected_tc: ") + cudaGetErrorString(e));
    }
    cleanup();
    return rc;
}

}  // namespace fitcore
