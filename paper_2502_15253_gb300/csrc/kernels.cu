// Kernels of the forward-folding fit: batched expectation, batched -2lnL + gradient, and the
// persistent batched L-BFGS fit. See dev_model.cuh for the per-block evaluation.
#include "kernels.cuh"

namespace fitcore {

// ------------------------------------------------------------------------------------
// shared-memory helpers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void copy_model(DevModel *dst, const DevModel *src) {
    const int n = (int)(sizeof(DevModel) / sizeof(int));
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(dst);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Prior in theta space (Eq. 6): sum ((theta-theta0)/sigma)^2 + sum_B d_B^T V_B^-1 d_B with
// V^-1 = W^T W (W = L^-1), evaluated as |W d|^2; gradient 2 W^T W d added to grad.
// zs: shared scratch of P floats. Returns the prior term (all threads).
__device__ double prior_theta(const DevModel &m, const float *pd, float *grad, float *zs,
                              double *red) {
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nth >> 5;
    float acc[1] = {0.f};
    for (int i = tid; i < m.P; i += nth) {
        const float pi = m.prior_inv[i];
        if (pi > 0.f) {
            const float r = pd[i] * pi;
            acc[0] = fmaf(r, r, acc[0]);
            if (grad) grad[i] += 2.f * r * pi;
        }
    }
    for (int b = 0; b < m.n_blocks; ++b) {
        const int n = m.blk_size[b];
        const int *idx = m.blk_idx + m.blk_idx_off[b];
        const float *W = m.blk_W + m.blk_mat_off[b];
        // z = W d, warp per row (rows of the lower triangle)
        for (int i = warp; i < n; i += nw) {
            float s = 0.f;
            for (int j = lane; j <= i; j += 32) s = fmaf(W[(int64_t)i * n + j], pd[idx[j]], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                zs[i] = s;
                acc[0] = fmaf(s, s, acc[0]);
            }
        }
        __syncthreads();
        if (grad) {
            // grad_d += 2 W^T z: column j of W, rows i >= j (W^T stored after W)
            const float *Wt = W + (int64_t)n * n;
            for (int j = warp; j < n; j += nw) {
                float s = 0.f;
                for (int i = j + lane; i < n; i += 32) s = fmaf(Wt[(int64_t)j * n + i], zs[i], s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) grad[idx[j]] += 2.f * s;
            }
        }
        __syncthreads();
    }
    double tot[1];
    block_sum<1>(acc, red, tot);
    return tot[0];
}

// ------------------------------------------------------------------------------------
// batched expectation / evaluation in theta space: block per parameter vector
// ------------------------------------------------------------------------------------
struct EvalSmem {
    DevModel m;
    double red[kMaxWarps * 24 + 24];
    int status;
};

__global__ void __launch_bounds__(256) eval_kernel(const DevModel *__restrict__ gm, int B,
                                                   const double *__restrict__ theta,
                                                   const float *__restrict__ data,
                                                   const uint32_t *__restrict__ masks,
                                                   double *__restrict__ nll_out,
                                                   float *__restrict__ grad_out,
                                                   float *__restrict__ mu_out,
                                                   int *__restrict__ status_out,
                                                   float *__restrict__ ws_global, int ws_in_smem) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EvalSmem &S = *reinterpret_cast<EvalSmem *>(smem_raw);
    copy_model(&S.m, gm);
    const DevModel &m = S.m;
    float *pv = reinterpret_cast<float *>(smem_raw + sizeof(EvalSmem));
    float *pd = pv + m.P;
    float *grad = pd + m.P;
    float *zs = grad + m.P;
    float *wsb = ws_in_smem ? (zs + m.P) : (ws_global + (int64_t)blockIdx.x * m.ws_eval_floats);
    const EvalWs ws = carve_eval_ws(wsb, m.N_t, m.C, m.max_reco);
    const bool want_grad = grad_out != nullptr;

    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        const double *th = theta + (int64_t)b * m.P;
        for (int i = threadIdx.x; i < m.P; i += blockDim.x) {
            const double t = th[i];
            pv[i] = (float)t;
            pd[i] = (float)(t - m.theta0[i]);
            grad[i] = 0.f;
        }
        if (threadIdx.x == 0) S.status = 0;
        __syncthreads();
        const float *dat = mu_out ? nullptr : (data ? data + (int64_t)b * m.n_data : m.asimov);
        const uint32_t mask = masks ? masks[b] : 0xffffffffu;
        double nll = 0.0;
        for (int d = 0; d < m.n_ds; ++d) {
            const bool on = mu_out ? true : ((mask >> d) & 1u);
            if (!on) continue;
            float *mo = mu_out ? mu_out + (int64_t)b * m.n_data + m.ds[d].data_off : nullptr;
            nll += eval_dataset(m, d, pv, pd, dat, ws, want_grad ? grad : nullptr, S.red,
                                &S.status, mo);
            __syncthreads();
            if (S.status) break;
        }
        const int st = S.status;
        if (mu_out == nullptr && st == 0) nll += prior_theta(m, pd, want_grad ? grad : nullptr, zs, S.red);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (nll_out) nll_out[b] = st ? INFINITY : nll;
            if (status_out)
                status_out[b] = (st & kStEscale) ? FIT_STATUS_ESCALE_NONMONOTONE
                                : (st & kStMuNonpos) ? FIT_STATUS_MU_NONPOSITIVE : 0;
        }
        if (want_grad)
            for (int i = threadIdx.x; i < m.P; i += blockDim.x)
                grad_out[(int64_t)b * m.P + i] = st ? NAN : grad[i];
        __syncthreads();
    }
}

size_t eval_smem_bytes(const DevModel &hm, bool ws_in_smem) {
    size_t b = sizeof(EvalSmem) + sizeof(float) * 4 * (size_t)hm.P;
    if (ws_in_smem) b += sizeof(float) * (size_t)hm.ws_eval_floats;
    return (b + 15) & ~size_t(15);
}

// ------------------------------------------------------------------------------------
// persistent batched L-BFGS
// ------------------------------------------------------------------------------------
struct FitSmem {
    DevModel m;
    double red[kMaxWarps * 24 + 24];
    double rho[16], alf[16];
    int status;
    int inst;
};

struct FitVecs {
    float *z, *g, *d, *zt, *gt, *zlo, *glo, *zcr, *gcr, *pv, *pd, *gth, *S, *Y;
};

__device__ __forceinline__ FitVecs carve_fit_vecs(float *base, int P, int hist) {
    FitVecs v;
    v.z = base;
    v.g = v.z + P;
    v.d = v.g + P;
    v.zt = v.d + P;
    v.gt = v.zt + P;
    v.zlo = v.gt + P;
    v.glo = v.zlo + P;
    v.zcr = v.glo + P;
    v.gcr = v.zcr + P;
    v.pv = v.gcr + P;
    v.pd = v.pv + P;
    v.gth = v.pd + P;
    v.S = v.gth + P;
    v.Y = v.S + (int64_t)hist * P;
    return v;
}

// block-wide dot product of two P-vectors (double result on every thread)
__device__ __forceinline__ double bdot(const float *a, const float *b, int n, double *red) {
    float acc[1] = {0.f};
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc[0] = fmaf(a[i], b[i], acc[0]);
    double out[1];
    block_sum<1>(acc, red, out);
    return out[0];
}

// theta from z (transformation layer): pd = J z, pv = theta0 + pd
__device__ void theta_of_z(const DevModel &m, const float *z, float *pv, float *pd) {
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nth >> 5;
    for (int i = tid; i < m.P; i += nth) {
        const float s = m.zscale[i];
        if (s > 0.f) pd[i] = s * z[i];
    }
    for (int b = 0; b < m.n_blocks; ++b) {
        const int n = m.blk_size[b];
        const int *idx = m.blk_idx + m.blk_idx_off[b];
        const float *L = m.blk_L + m.blk_mat_off[b];
        for (int i = warp; i < n; i += nw) {
            float s = 0.f;
            for (int j = lane; j <= i; j += 32) s = fmaf(L[(int64_t)i * n + j], z[idx[j]], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) pd[idx[i]] = s;
        }
    }
    __syncthreads();
    for (int i = tid; i < m.P; i += nth) pv[i] = m.theta0_f[i] + pd[i];
    __syncthreads();
}

// -2lnL(theta(z)) and its z-gradient gz. Returns +inf on an invalid point.
__device__ double eval_z(const DevModel &m, const float *z, float *gz, FitVecs &V, EvalWs ws,
                         const float *data, uint32_t mask, FitSmem &S) {
    theta_of_z(m, z, V.pv, V.pd);
    for (int i = threadIdx.x; i < m.P; i += blockDim.x) V.gth[i] = 0.f;
    if (threadIdx.x == 0) S.status = 0;
    __syncthreads();
    double nll = 0.0;
    for (int d = 0; d < m.n_ds; ++d) {
        if (!((mask >> d) & 1u)) continue;
        nll += eval_dataset(m, d, V.pv, V.pd, data, ws, V.gth, S.red, &S.status, nullptr);
        __syncthreads();
        if (S.status) return INFINITY;
    }
    // prior = |z|^2 over constrained coordinates; gz = J^T gth + 2 z
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nth >> 5;
    float acc[1] = {0.f};
    for (int i = tid; i < m.P; i += nth) {
        const float s = m.zscale[i];
        if (s > 0.f) {
            const bool con = m.prior_inv[i] > 0.f;
            gz[i] = s * V.gth[i] + (con ? 2.f * z[i] : 0.f);
            if (con) acc[0] = fmaf(z[i], z[i], acc[0]);
        }
    }
    for (int b = 0; b < m.n_blocks; ++b) {
        const int n = m.blk_size[b];
        const int *idx = m.blk_idx + m.blk_idx_off[b];
        const float *Lt = m.blk_L + m.blk_mat_off[b] + (int64_t)n * n;   // L^T, row-major
        for (int j = warp; j < n; j += nw) {
            float s = 0.f;
            for (int i = j + lane; i < n; i += 32) s = fmaf(Lt[(int64_t)j * n + i], V.gth[idx[i]], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                const float zj = z[idx[j]];
                gz[idx[j]] = s + 2.f * zj;
                acc[0] = fmaf(zj, zj, acc[0]);
            }
        }
    }
    double tot[1];
    block_sum<1>(acc, S.red, tot);
    return nll + tot[0];
}

// cubic minimiser through (a, fa, ga), (b, fb, gb), or the secant of the slopes when the
// values are not informative (difference within the noise allowance)
__device__ __forceinline__ double ls_interp(double a, double fa, double ga, double b, double fb,
                                            double gb, double eps_f) {
    double t;
    if (isfinite(fb) && fabs(fb - fa) > eps_f) {
        const double d1 = ga + gb - 3.0 * (fa - fb) / (a - b);
        const double disc = d1 * d1 - ga * gb;
        if (disc >= 0.0) {
            const double d2 = copysign(sqrt(disc), b - a);
            t = b - (b - a) * (gb + d2 - d1) / (gb - ga + 2.0 * d2);
        } else {
            t = 0.5 * (a + b);
        }
    } else if (isfinite(gb) && gb != ga) {
        t = a - ga * (b - a) / (gb - ga);
    } else {
        t = 0.5 * (a + b);
    }
    const double lo = fmin(a, b), hi = fmax(a, b), w = hi - lo;
    if (!(t >= lo + 0.1 * w && t <= hi - 0.1 * w)) t = 0.5 * (a + b);
    return t;
}

__device__ __forceinline__ void vcopy(float *dst, const float *src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

__global__ void __launch_bounds__(256, 2) fit_kernel(FitArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FitSmem &S = *reinterpret_cast<FitSmem *>(smem_raw);
    float *dyn = reinterpret_cast<float *>(smem_raw + sizeof(FitSmem));
    float *gws = A.ws_global + (int64_t)blockIdx.x * A.ws_stride;
    const uint64_t deadline = global_ns() + A.budget_ns;   // per-block clock budget
    const int tid = threadIdx.x;
    const int hist_max = A.hist;
    const double c1 = 1e-4, c2 = 0.9;

    while (true) {
        if (tid == 0) S.inst = atomicAdd(A.queue, 1);
        __syncthreads();
        const int ii = S.inst;
        __syncthreads();
        if (ii >= A.n_inst) break;
        const fit_instance in = A.inst[ii];
        copy_model(&S.m, A.models + in.model);
        const DevModel &m = S.m;
        const int P = m.P;
        // workspace: shared memory when the model fits, else this block's global slice
        const int need = fit_vec_floats(P, hist_max) + m.ws_eval_floats;
        float *base = (need <= A.smem_floats) ? dyn : gws;
        FitVecs V = carve_fit_vecs(base, P, hist_max);
        const EvalWs ws = carve_eval_ws(base + fit_vec_floats(P, hist_max), m.N_t, m.C, m.max_reco);
        const float *data = A.data + in.data_off;
        fit_result res;
        res.iters = 0;
        res.n_evals = 0;
        res.edm = INFINITY;
        res.nll_min = INFINITY;
        res.pad = 0;
        int status = FIT_STATUS_MAXITER;

        if (global_ns() > deadline) {
            status = FIT_STATUS_TIMEOUT;
            for (int i = tid; i < P; i += blockDim.x) V.z[i] = 0.f;
            __syncthreads();
        } else {
            // start point z0 = J^-1 (theta_start - theta0)
            const double *st = A.start ? A.start + in.param_off : nullptr;
            for (int i = tid; i < P; i += blockDim.x) {
                const float dd = st ? (float)(st[i] - m.theta0[i]) : 0.f;
                V.pd[i] = dd;
                const float s = m.zscale[i];
                if (s > 0.f) V.z[i] = dd / s;
            }
            __syncthreads();
            {
                const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
                for (int b = 0; b < m.n_blocks; ++b) {
                    const int n = m.blk_size[b];
                    const int *idx = m.blk_idx + m.blk_idx_off[b];
                    const float *W = m.blk_W + m.blk_mat_off[b];
                    for (int i = warp; i < n; i += nw) {
                        float s = 0.f;
                        for (int j = lane; j <= i; j += 32) s = fmaf(W[(int64_t)i * n + j], V.pd[idx[j]], s);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                        if (lane == 0) V.z[idx[i]] = s;
                    }
                }
            }
            __syncthreads();

            double f = eval_z(m, V.z, V.g, V, ws, data, in.mask, S);
            res.n_evals = 1;
            if (!isfinite(f)) status = FIT_STATUS_NONFINITE;
            int hn = 0, head = 0;   // history size and next slot
            double gamma = 1.0;
            // After the first EDM convergence the history is dropped and rebuilt (at least
            // hist_max iterations) up to A.restarts times: the fresh pairs come from the
            // directions still moving, which are the flat ones a short history had not seen,
            // and where its EDM estimate was too small.
            int restarts_left = A.restarts, since_restart = hist_max;
            while (status == FIT_STATUS_MAXITER) {
                // ---- direction d = -H g, two-loop recursion ------------------------------
                vcopy(V.d, V.g, P);
                __syncthreads();
                for (int q = 0; q < hn; ++q) {
                    const int slot = (head - 1 - q + hist_max) % hist_max;
                    const float *s = V.S + (int64_t)slot * P, *y = V.Y + (int64_t)slot * P;
                    const double a = S.rho[slot] * bdot(s, V.d, P, S.red);
                    if (tid == 0) S.alf[slot] = a;
                    const float af = (float)a;
                    for (int i = tid; i < P; i += blockDim.x) V.d[i] = fmaf(-af, y[i], V.d[i]);
                    __syncthreads();
                }
                {
                    const float gf = (float)gamma;
                    for (int i = tid; i < P; i += blockDim.x) V.d[i] *= gf;
                    __syncthreads();
                }
                for (int q = hn - 1; q >= 0; --q) {
                    const int slot = (head - 1 - q + hist_max) % hist_max;
                    const float *s = V.S + (int64_t)slot * P, *y = V.Y + (int64_t)slot * P;
                    const double bta = S.rho[slot] * bdot(y, V.d, P, S.red);
                    const float cf = (float)(S.alf[slot] - bta);
                    for (int i = tid; i < P; i += blockDim.x) V.d[i] = fmaf(cf, s[i], V.d[i]);
                    __syncthreads();
                }
                for (int i = tid; i < P; i += blockDim.x) V.d[i] = -V.d[i];
                __syncthreads();
                double gd = bdot(V.g, V.d, P, S.red);
                if (!(gd < 0.0)) {   // not a descent direction: drop the history
                    hn = 0;
                    head = 0;
                    gamma = 1.0;
                    for (int i = tid; i < P; i += blockDim.x) V.d[i] = -V.g[i];
                    __syncthreads();
                    gd = -bdot(V.g, V.g, P, S.red);
                }
                const double edm = -0.5 * gd;
                res.edm = edm;
                if (edm < A.edm_tol && since_restart >= hist_max) {
                    if (restarts_left == 0) {
                        status = FIT_STATUS_CONVERGED;
                        break;
                    }
                    --restarts_left;
                    since_restart = 0;
                    hn = 0;
                    head = 0;
                    continue;
                }
                if (res.iters >= A.max_iter) break;
                if (global_ns() > deadline) {
                    status = FIT_STATUS_TIMEOUT;
                    break;
                }

                // ---- line search on phi(alpha) = f(z + alpha d) -----------------------------
                const double dphi0 = gd;
                const double eps_f = A.f_noise_rel * (1.0 + fabs(f));
                double alpha;
                if (hn == 0) {
                    const double dn = sqrt(bdot(V.d, V.d, P, S.red));
                    alpha = fmin(1.0, 1.0 / fmax(dn, 1e-30));
                } else {
                    alpha = 1.0;
                }
                double lo = 0.0, flo = f, dlo = dphi0, hi = INFINITY, fhi = INFINITY, dhi = INFINITY;
                double a_cr = INFINITY, f_cr = 0.0;
                bool have_lo = false, accepted = false;
                double fa = 0.0;
                for (int it = 0; it < A.max_ls; ++it) {
                    const float af = (float)alpha;
                    for (int i = tid; i < P; i += blockDim.x) V.zt[i] = fmaf(af, V.d[i], V.z[i]);
                    __syncthreads();
                    fa = eval_z(m, V.zt, V.gt, V, ws, data, in.mask, S);
                    res.n_evals++;
                    const double da = isfinite(fa) ? bdot(V.gt, V.d, P, S.red) : INFINITY;
                    const bool armijo = fa <= f + c1 * alpha * dphi0;
                    const bool approx = fa <= f + eps_f;
                    const bool val_ok = isfinite(fa) && (armijo || approx);
                    if (val_ok && fabs(da) <= -c2 * dphi0) {
                        accepted = true;
                        break;
                    }
                    if (val_ok && da >= c2 * dphi0 && alpha < a_cr) {   // crossed a kink
                        a_cr = alpha;
                        f_cr = fa;
                        vcopy(V.zcr, V.zt, P);
                        vcopy(V.gcr, V.gt, P);
                    }
                    if (!val_ok || fa > flo + eps_f || da >= 0.0) {
                        hi = alpha;
                        fhi = fa;
                        dhi = da;
                    } else {
                        lo = alpha;
                        flo = fa;
                        dlo = da;
                        have_lo = true;
                        vcopy(V.zlo, V.zt, P);
                        vcopy(V.glo, V.gt, P);
                    }
                    __syncthreads();
                    if (!isfinite(hi)) {
                        alpha = 4.0 * alpha;
                    } else {
                        alpha = ls_interp(lo, flo, dlo, hi, fhi, dhi, eps_f);
                        if (hi - lo <= 1e-7 * hi) break;
                    }
                }
                if (!accepted) {
                    if (isfinite(a_cr)) {
                        vcopy(V.zt, V.zcr, P);
                        vcopy(V.gt, V.gcr, P);
                        fa = f_cr;
                        accepted = true;
                    } else if (have_lo) {
                        vcopy(V.zt, V.zlo, P);
                        vcopy(V.gt, V.glo, P);
                        fa = flo;
                        accepted = true;
                    }
                    __syncthreads();
                }
                if (!accepted) {
                    if (hn > 0) {   // retry from steepest descent
                        hn = 0;
                        head = 0;
                        gamma = 1.0;
                        continue;
                    }
                    status = FIT_STATUS_LINESEARCH_FAIL;
                    break;
                }
                // ---- curvature pair -------------------------------------------------------
                float *s_new = V.S + (int64_t)head * P, *y_new = V.Y + (int64_t)head * P;
                for (int i = tid; i < P; i += blockDim.x) {
                    s_new[i] = V.zt[i] - V.z[i];
                    y_new[i] = V.gt[i] - V.g[i];
                }
                __syncthreads();
                const double sy = bdot(s_new, y_new, P, S.red);
                const double yy = bdot(y_new, y_new, P, S.red);
                if (sy > 1e-10 * yy && yy > 0.0) {
                    if (tid == 0) S.rho[head] = 1.0 / sy;
                    head = (head + 1) % hist_max;
                    hn = min(hn + 1, hist_max);
                    gamma = sy / yy;
                }
                vcopy(V.z, V.zt, P);
                vcopy(V.g, V.gt, P);
                __syncthreads();
                f = fa;
                res.iters++;
                since_restart++;
            }
            res.nll_min = f;
        }
        // ---- result: theta = theta0 + J z in double ---------------------------------------
        double *best = A.best + in.param_off;
        for (int i = tid; i < P; i += blockDim.x) {
            const float s = m.zscale[i];
            if (s > 0.f) best[i] = m.theta0[i] + (double)s * (double)V.z[i];
        }
        for (int b = 0; b < m.n_blocks; ++b) {
            const int n = m.blk_size[b];
            const int *idx = m.blk_idx + m.blk_idx_off[b];
            const double *L = m.blk_L64 + m.blk_mat_off[b];
            for (int i = tid; i < n; i += blockDim.x) {
                double s = 0.0;
                for (int j = 0; j <= i; ++j) s += L[(int64_t)i * n + j] * (double)V.z[idx[j]];
                best[idx[i]] = m.theta0[idx[i]] + s;
            }
        }
        if (tid == 0) {
            res.status = status;
            A.results[ii] = res;
        }
        __syncthreads();
    }
}

size_t fit_smem_bytes(int floats) { return sizeof(FitSmem) + sizeof(float) * (size_t)floats; }

}  // namespace fitcore
