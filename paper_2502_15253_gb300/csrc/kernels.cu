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
    const EvalWs ws = carve_eval_ws(wsb, m.N_t, m.C, m.max_reco, m.n_osc);
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
            nll += eval_dataset<6>(m, d, pv, pd, dat, ws, want_grad ? grad : nullptr, S.red,
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
constexpr int kMaxHist = 32;
constexpr int kStallWindow = 100;   // iterations per stall check
constexpr int kMaxLsFresh = 30;     // line-search trials along steepest descent
constexpr int kNDots = 4 * kMaxHist + 1;

// Minimiser state of one fit between two evaluations: in shared memory while a block works on
// the fit, in global memory between the launches of the lockstep engine.
constexpr int kPhStart = 0, kPhTrial = 1, kPhDone = 2;

struct FitState {
    // L-BFGS history in scalars: SY[i][j] = s_i.y_j (needed for i older than j and i = j),
    // YY[i][j] = y_i.y_j (symmetric), rho_i = 1 / s_i.y_i, by history slot
    double SY[kMaxHist][kMaxHist], YY[kMaxHist][kMaxHist];
    double rho[kMaxHist];
    double gamma;
    double f, edm;
    // line search on phi(alpha) = f(z + alpha d): bracket [lo, hi], kink crossing a_cr
    double alpha, dphi0, eps_f, lo, flo, dlo, hi, fhi, dhi, a_cr, f_cr;
    int hn, head, occ;
    int phase, ls_it, have_lo, pending, restarts_left, since_restart;
    int iters, n_evals, status;
    int win_it;     // stall window: iteration and value at its start
    double f_win;
};

struct alignas(16) FitSmem {
    DevModel m;
    double red[kMaxWarps * 24 + 24];
    FitState st;
    double dots[kNDots];       // fused pass: S.y_new | Y.y_new | S.g | Y.g | g.g
    float cs[kMaxHist], cy[kMaxHist];   // d = -(cg g + sum cs_j s_j + sum cy_j y_j)
    float cg;
    double gHg;
    int status;                // evaluation status bits
    int inst;
    float pre_u[kMaxPreRank];  // preconditioner scratch
};

struct FitVecs {
    float *z, *g, *d, *zt, *gt, *zlo, *glo, *zcr, *gcr, *pv, *pd, *gth, *zw, *gzw, *S, *Y;
};

// 12 P-vectors at base; the 2 hist P-vectors of the history at hbase (pitch fit_vec_pitch(P))
__device__ __forceinline__ FitVecs carve_fit_vecs(float *base, float *hbase, int P, int hist) {
    const int Pp = fit_vec_pitch(P);
    FitVecs v;
    v.z = base;
    v.g = v.z + Pp;
    v.d = v.g + Pp;
    v.zt = v.d + Pp;
    v.gt = v.zt + Pp;
    v.zlo = v.gt + Pp;
    v.glo = v.zlo + Pp;
    v.zcr = v.glo + Pp;
    v.gcr = v.zcr + Pp;
    v.pv = v.gcr + Pp;
    v.pd = v.pv + Pp;
    v.gth = v.pd + Pp;
    v.zw = v.gth + Pp;    // preconditioned fits: z of the trial point and its z-gradient
    v.gzw = v.zw + Pp;
    v.S = hbase;
    v.Y = v.S + (int64_t)hist * Pp;
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

// One pass of block-wide dot products, a warp per product (lanes stride the P entries, a
// shuffle tree adds them). Products q < 4 kMaxHist: type q / kMaxHist (0: s_j.y_new,
// 1: y_j.y_new, 2: s_j.g, 3: y_j.g) for the history slots set in `occ`; q = 4 kMaxHist: g.g.
// The results land in S.dots; ends with a barrier.
__device__ void fused_dots(const float *Sv, const float *Yv, const float *ynew, const float *g, int P,
                           unsigned occ, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int pitch = fit_vec_pitch(P);
    // Each warp takes four products at a time, so four independent 16-byte loads per lane are
    // in flight before the first shuffle reduction.
    for (int q0 = warp * 4; q0 < kNDots; q0 += nw * 4) {
        const float *a[4], *b[4];
        bool on[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u;
            on[u] = q < kNDots;
            a[u] = g;
            b[u] = g;
            if (on[u] && q < kNDots - 1) {
                const int type = q / kMaxHist, slot = q % kMaxHist;
                on[u] = ((occ >> slot) & 1u) && !(type < 2 && ynew == nullptr);
                a[u] = ((type & 1) ? Yv : Sv) + (int64_t)slot * pitch;
                b[u] = (type < 2) ? ynew : g;
            }
        }
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = lane; k < (P >> 2); k += 32) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!on[u]) continue;
                const float4 x = reinterpret_cast<const float4 *>(a[u])[k];
                const float4 y = reinterpret_cast<const float4 *>(b[u])[k];
                acc[u] = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, acc[u]))));
            }
        }
        const int tail = (P & ~3) + lane;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (on[u] && tail < P) acc[u] = fmaf(a[u][tail], b[u][tail], acc[u]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (on[u]) out[q0 + u] = (double)acc[u];
        }
    }
    __syncthreads();
}

// Warp 0: folds the pending curvature pair (slot S.head, if `pending`) into the scalar
// history and runs the L-BFGS two-loop recursion on scalars. Every inner product the
// recursion needs is one of s_i.g, y_i.g, s_i.y_j (i older than j) or y_i.y_j, so the
// direction is d = -(cg g + sum_j cs_j s_j + sum_j cy_j y_j) with coefficients from the
// recurrence, and g^T H g follows from the same scalars. Lane k holds chronological history
// position k; both triangular recurrences run column by column (one shuffle per step).
__device__ void lbfgs_scalars(FitSmem &S, int hist_max, bool pending) {
    const int lane = threadIdx.x & 31;
    const double *dt = S.dots;
    if (pending && lane == 0) {
        const int c = S.st.head;
        const double sy = dt[c], yy = dt[kMaxHist + c];
        if (sy > 1e-10 * yy && yy > 0.0) {
            for (int j = 0; j < hist_max; ++j)
                if (((S.st.occ >> j) & 1) && j != c) {
                    S.st.SY[j][c] = dt[j];
                    S.st.YY[j][c] = S.st.YY[c][j] = dt[kMaxHist + j];
                }
            S.st.SY[c][c] = sy;
            S.st.YY[c][c] = yy;
            S.st.rho[c] = 1.0 / sy;
            S.st.occ |= 1u << c;
            S.st.head = (c + 1) % hist_max;
            S.st.hn = min(S.st.hn + 1, hist_max);
            S.st.gamma = sy / yy;
        } else if ((S.st.occ >> c) & 1) {
            // rejected pair written over the oldest one: that pair is gone as well
            S.st.occ &= ~(1u << c);
            S.st.hn -= 1;
        }
    }
    __syncwarp();
    const int hn = S.st.hn, oldest = (S.st.head - hn + hist_max) % hist_max;
    const double gam = S.st.gamma, gg = dt[kNDots - 1];
    const bool live = lane < hn;
    const int sl = live ? (oldest + lane) % hist_max : 0;    // this lane's history slot
    const double sg = live ? dt[2 * kMaxHist + sl] : 0.0, yg = live ? dt[3 * kMaxHist + sl] : 0.0;
    const double rho = live ? S.st.rho[sl] : 0.0;
    // alpha_k = rho_k (s_k.g - sum_{l > k} alpha_l s_k.y_l), newest first
    double acc = sg, alpha = 0.0;
    for (int l = hn - 1; l >= 0; --l) {
        const double al = __shfl_sync(0xffffffffu, rho * acc, l);
        if (lane == l) alpha = al;
        const int sll = (oldest + l) % hist_max;
        if (lane < l) acc -= al * S.st.SY[sl][sll];
    }
    // u_k = sum_l alpha_l y_k.y_l
    double u = 0.0;
    for (int l = 0; l < hn; ++l) {
        const double al = __shfl_sync(0xffffffffu, alpha, l);
        if (live) u += al * S.st.YY[sl][(oldest + l) % hist_max];
    }
    // beta_k = rho_k (gam (y_k.g - u_k) + sum_{l < k} (alpha_l - beta_l) s_l.y_k), oldest first
    double acc2 = gam * (yg - u), beta = 0.0;
    for (int l = 0; l < hn; ++l) {
        const double bl = __shfl_sync(0xffffffffu, rho * acc2, l);
        const double cl = __shfl_sync(0xffffffffu, alpha, l) - bl;
        if (lane == l) beta = bl;
        if (live && lane > l) acc2 += cl * S.st.SY[(oldest + l) % hist_max][sl];
    }
    const double cs = alpha - beta, cy = -gam * alpha;
    double part = live ? cs * sg + cy * yg : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    double ghg = gam * gg + part;
    if (lane < kMaxHist) {
        S.cs[lane] = 0.f;
        S.cy[lane] = 0.f;
    }
    __syncwarp();
    if (live) {
        S.cs[sl] = (float)cs;
        S.cy[sl] = (float)cy;
    }
    if (lane == 0) S.cg = (float)gam;
    __syncwarp();
    if (!(ghg > 0.0)) {   // not a descent direction: drop the history, steepest descent
        if (lane < kMaxHist) S.cs[lane] = S.cy[lane] = 0.f;
        if (lane == 0) {
            S.st.hn = 0;
            S.st.occ = 0;
            S.st.head = 0;
            S.st.gamma = 1.0;
            S.cg = 1.f;
        }
        ghg = gg;
    }
    if (lane == 0) S.gHg = ghg;
}

// Row r of the concatenated prior blocks: its block b and the row i within it.
__device__ __forceinline__ int prior_row_block(const DevModel &m, int r) {
    int b = 0;
    while (b + 1 < m.n_blocks && m.blk_idx_off[b + 1] <= r) ++b;
    return b;
}

__device__ __forceinline__ int prior_rows(const DevModel &m) {
    return m.n_blocks > 0 ? m.blk_idx_off[m.n_blocks - 1] + m.blk_size[m.n_blocks - 1] : 0;
}

// theta from z (transformation layer): pd = J z, pv = theta0 + pd. The rows of all prior
// blocks are spread over the threads together (a thread per row of L z, formed over the stored
// L^T so that each step is a coalesced load plus a broadcast of z); four partial sums keep
// four independent loads per thread in flight.
__device__ void theta_of_z(const DevModel &m, const float *z, float *pv, float *pd) {
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < m.P; i += nth) {
        const float s = m.zscale[i];
        if (s > 0.f) pd[i] = s * z[i];
    }
    const int rows = prior_rows(m);
    for (int r = tid; r < rows; r += nth) {
        const int b = prior_row_block(m, r);
        const int n = m.blk_size[b], i = r - m.blk_idx_off[b], first = m.blk_first[b];
        const int *idx = m.blk_idx + m.blk_idx_off[b];
        const float *Lt = m.blk_L + m.blk_mat_off[b] + (int64_t)n * n;   // L^T, row-major
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        int j = 0;
        if (first >= 0) {   // consecutive indices: z read directly, sixteen loads in flight
            const float *zb = z + first;
            for (; j + 15 <= i; j += 16) {
#pragma unroll
                for (int q = 0; q < 16; ++q) s[q & 3] = fmaf(Lt[(int64_t)(j + q) * n + i], zb[j + q], s[q & 3]);
            }
            for (; j <= i; ++j) s[0] = fmaf(Lt[(int64_t)j * n + i], zb[j], s[0]);
        } else {
            for (; j + 3 <= i; j += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) s[q] = fmaf(Lt[(int64_t)(j + q) * n + i], z[idx[j + q]], s[q]);
            }
            for (; j <= i; ++j) s[0] = fmaf(Lt[(int64_t)j * n + i], z[idx[j]], s[0]);
        }
        pd[idx[i]] = (s[0] + s[1]) + (s[2] + s[3]);
    }
    __syncthreads();
    for (int i = tid; i < m.P; i += nth) pv[i] = m.theta0_f[i] + pd[i];
    __syncthreads();
}

// Prior in z space and the chain rule back to z: gz = J^T gth + 2 z over the constrained
// coordinates (J = diag(scale) outside the prior blocks, the Cholesky factor L inside);
// returns the prior |z|^2 (all threads).
__device__ double eval_z_prior(const DevModel &m, const float *z, const float *gth, float *gz, double *red) {
    const int tid = threadIdx.x, nth = blockDim.x;
    float acc[1] = {0.f};
    for (int i = tid; i < m.P; i += nth) {
        const float s = m.zscale[i];
        if (s > 0.f) {
            const bool con = m.prior_inv[i] > 0.f;
            gz[i] = s * gth[i] + (con ? 2.f * z[i] : 0.f);
            if (con) acc[0] = fmaf(z[i], z[i], acc[0]);
        }
    }
    const int rows = prior_rows(m);
    for (int r = tid; r < rows; r += nth) {
        const int b = prior_row_block(m, r);
        const int n = m.blk_size[b], j = r - m.blk_idx_off[b], first = m.blk_first[b];
        const int *idx = m.blk_idx + m.blk_idx_off[b];
        const float *L = m.blk_L + m.blk_mat_off[b];   // L, row-major: (L^T g)_j = sum_i L_ij g_i
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        int i = j;
        if (first >= 0) {   // consecutive indices: gth read directly, sixteen loads in flight
            const float *gb = gth + first;
            for (; i + 15 < n; i += 16) {
#pragma unroll
                for (int q = 0; q < 16; ++q) s[q & 3] = fmaf(L[(int64_t)(i + q) * n + j], gb[i + q], s[q & 3]);
            }
            for (; i < n; ++i) s[0] = fmaf(L[(int64_t)i * n + j], gb[i], s[0]);
        } else {
            for (; i + 3 < n; i += 4) {
#pragma unroll
                for (int q = 0; q < 4; ++q) s[q] = fmaf(L[(int64_t)(i + q) * n + j], gth[idx[i + q]], s[q]);
            }
            for (; i < n; ++i) s[0] = fmaf(L[(int64_t)i * n + j], gth[idx[i]], s[0]);
        }
        const float zj = z[idx[j]];
        gz[idx[j]] = ((s[0] + s[1]) + (s[2] + s[3])) + 2.f * zj;
        acc[0] = fmaf(zj, zj, acc[0]);
    }
    double tot[1];
    block_sum<1>(acc, red, tot);
    return tot[0];
}

// Parameters held at their start values (a profile-likelihood point): a zero z-gradient keeps
// every L-BFGS direction, and so the parameter, where it is. Only parameters outside the prior
// blocks can be held (their z coordinate is the parameter itself, scaled).
__device__ __forceinline__ void hold_fixed(const uint8_t *fixed, float *gz, int P) {
    if (fixed == nullptr) return;
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        if (fixed[i]) gz[i] = 0.f;
}

// y = x + Q (coef o (Q^T x)) for the model's preconditioner (coef = pre_c: y = T x; coef =
// pre_c + r: y = T^-1 x). Q^T rows: a warp per row, 16-byte loads, the last P mod 4 entries
// scalar (the padding of x is never read); then a thread per entry over the r rows. x and y
// may be the same vector. u: r floats of shared scratch. Held parameters (fixed) are left out
// of Q: T then maps them to themselves and mixes them into nothing, so they stay held in w
// (T^-1 is then only approximate for the free part, which only moves the start). Ends with a
// barrier.
__device__ void pre_apply(const DevModel &m, const float *coef, const float *x, float *y, float *u,
                          const uint8_t *fixed) {
    const int P = m.P, Pp = fit_vec_pitch(P), r = m.pre_r;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nfull = P >> 2;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    for (int k = warp; k < r; k += nw) {
        const float *q = m.pre_Q + (int64_t)k * Pp;
        const float4 *q4 = reinterpret_cast<const float4 *>(q);
        float acc = 0.f;
        for (int c = lane; c < nfull; c += 32) {
            float4 a = __ldg(q4 + c);
            const float4 b = x4[c];
            if (fixed) {
                const uint8_t *f = fixed + 4 * c;
                if (f[0]) a.x = 0.f;
                if (f[1]) a.y = 0.f;
                if (f[2]) a.z = 0.f;
                if (f[3]) a.w = 0.f;
            }
            acc = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
        }
        if (lane < (P & 3) && !(fixed && fixed[4 * nfull + lane]))
            acc = fmaf(__ldg(q + 4 * nfull + lane), x[4 * nfull + lane], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) u[k] = __ldg(coef + k) * acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        float acc = x[i];
        if (!(fixed && fixed[i])) {
#pragma unroll 8
            for (int k = 0; k < r; ++k) acc = fmaf(__ldg(m.pre_Q + (int64_t)k * Pp + i), u[k], acc);
        }
        y[i] = acc;
    }
    __syncthreads();
}

// -2lnL(theta(z)) and its z-gradient gz. Returns +inf on an invalid point.
template <int NOSC>
__device__ double eval_z(const DevModel &m, const float *z, float *gz, FitVecs &V, EvalWs ws,
                         const float *data, uint32_t mask, FitSmem &S, const uint8_t *fixed) {
    theta_of_z(m, z, V.pv, V.pd);
    for (int i = threadIdx.x; i < m.P; i += blockDim.x) V.gth[i] = 0.f;
    if (threadIdx.x == 0) S.status = 0;
    __syncthreads();
    double nll = 0.0;
    for (int d = 0; d < m.n_ds; ++d) {
        if (!((mask >> d) & 1u)) continue;
        nll += eval_dataset<NOSC>(m, d, V.pv, V.pd, data, ws, V.gth, S.red, &S.status, nullptr);
        __syncthreads();
        if (S.status) return INFINITY;
    }
    const double prior = eval_z_prior(m, z, V.gth, gz, S.red);
    hold_fixed(fixed, gz, m.P);
    return nll + prior;
}

// The same in the preconditioned coordinates w (z = T w): -2lnL and g_w = T^T g_z.
template <int NOSC>
__device__ double eval_w(const DevModel &m, const float *w, float *gw, FitVecs &V, EvalWs ws,
                         const float *data, uint32_t mask, FitSmem &S, const uint8_t *fixed) {
    pre_apply(m, m.pre_c, w, V.zw, S.pre_u, fixed);
    const double f = eval_z<NOSC>(m, V.zw, V.gzw, V, ws, data, mask, S, fixed);
    __syncthreads();
    pre_apply(m, m.pre_c, V.gzw, gw, S.pre_u, fixed);   // T is symmetric; held entries stay 0
    return f;
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

struct FitParams {
    int hist, max_iter, max_ls, restarts;
    double edm_tol, f_noise_rel;
    uint64_t deadline;         // %globaltimer value past which a fit stops with TIMEOUT
};

__device__ __forceinline__ void reset_history(FitState &st) {
    st.hn = 0;
    st.head = 0;
    st.occ = 0;
    st.gamma = 1.0;
}

// One step of the minimiser: consumes the evaluation (fa, V.gt) of the point V.zt and leaves
// the next point to evaluate in V.zt (returns true), or ends the fit (returns false, S.st.phase
// = kPhDone, S.st.status set). Block-wide; every thread holds the same copies of the scalars.
//
// L-BFGS in whitened coordinates with the two-loop recursion on scalars (fused_dots,
// lbfgs_scalars). Line search on phi(alpha) = f(z + alpha d): accepts a strong-Wolfe point or
// the approximate-Wolfe point of Hager & Zhang (value within the noise allowance eps_f, slope
// condition), brackets with cubic / secant interpolation, and falls back to the smallest trial
// that crossed a kink (value not increased, slope risen past c2 phi'(0)) or to the best lower
// point. A failed search with a history retries from steepest descent. Stop: EDM =
// 1/2 g^T H g < edm_tol (optionally after `restarts` history rebuilds), max_iter, or the clock.
__device__ bool fit_decide(FitSmem &S, FitVecs &V, int P, double fa, const FitParams &F) {
    const double c1 = 1e-4, c2 = 0.9;
    const int tid = threadIdx.x;
    FitState &st = S.st;
    __syncthreads();
    // block-uniform copies of the scalars
    double f = st.f, edm = st.edm;
    double alpha = st.alpha, dphi0 = st.dphi0, eps_f = st.eps_f;
    double lo = st.lo, flo = st.flo, dlo = st.dlo, hi = st.hi, fhi = st.fhi, dhi = st.dhi;
    double a_cr = st.a_cr, f_cr = st.f_cr;
    int phase = st.phase, ls_it = st.ls_it, restarts_left = st.restarts_left, since_restart = st.since_restart;
    int iters = st.iters, n_evals = st.n_evals + 1, status = st.status;
    bool have_lo = st.have_lo != 0, pending = st.pending != 0;
    __syncthreads();

    enum { kDirection, kTrial, kDone } next = kDirection;
    bool stall_mark = false;   // a stall window ended in this pass
    if (phase == kPhStart) {
        // the start point's evaluation
        f = fa;
        vcopy(V.z, V.zt, P);
        vcopy(V.g, V.gt, P);
        if (tid == 0) reset_history(st);
        restarts_left = F.restarts;
        since_restart = F.hist;
        pending = false;
        if (tid == 0) {
            st.f_win = f;
            st.win_it = 0;
        }
        if (!isfinite(f)) {
            status = FIT_STATUS_NONFINITE;
            next = kDone;
        }
    } else {
        // ---- a line-search trial at alpha came back -------------------------------------
        const double da = isfinite(fa) ? bdot(V.gt, V.d, P, S.red) : INFINITY;
        const bool armijo = fa <= f + c1 * alpha * dphi0;
        const bool approx = fa <= f + eps_f;
        const bool val_ok = isfinite(fa) && (armijo || approx);
        bool accepted = false, stop = false;
        double f_acc = fa;
        if (val_ok && fabs(da) <= -c2 * dphi0) {
            accepted = true;
        } else {
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
                if (hi - lo <= 1e-7 * hi) stop = true;
            }
            // a quasi-Newton direction is well scaled (the unit step is usually right), so its
            // search stops after max_ls trials; a steepest-descent search (fresh history) has
            // to find the scale and gets kMaxLsFresh
            if (!stop && ++ls_it < (st.hn == 0 ? kMaxLsFresh : F.max_ls)) next = kTrial;
        }
        if (next != kTrial) {
            if (!accepted) {
                if (isfinite(a_cr)) {
                    vcopy(V.zt, V.zcr, P);
                    vcopy(V.gt, V.gcr, P);
                    f_acc = f_cr;
                    accepted = true;
                } else if (have_lo) {
                    vcopy(V.zt, V.zlo, P);
                    vcopy(V.gt, V.glo, P);
                    f_acc = flo;
                    accepted = true;
                }
                __syncthreads();
            }
            if (accepted) {
                // curvature pair into the next slot; folded in by the next fused pass
                const int c = st.head;
                float *s_new = V.S + (int64_t)c * fit_vec_pitch(P), *y_new = V.Y + (int64_t)c * fit_vec_pitch(P);
                for (int i = tid; i < P; i += blockDim.x) {
                    s_new[i] = V.zt[i] - V.z[i];
                    y_new[i] = V.gt[i] - V.g[i];
                    V.z[i] = V.zt[i];
                    V.g[i] = V.gt[i];
                }
                pending = true;
                f = f_acc;
                iters++;
                since_restart++;
                // stall: a whole window of iterations that lowered the value by no more than
                // the FP32 noise allowance (the line search then only trades noise, e.g. on a
                // crease of the energy correction)
                // (the window's start lives in shared memory only: read here, written by thread 0
                // after the barrier at the end of this pass)
                if (iters - st.win_it >= kStallWindow) {
                    if (st.f_win - f <= 2.0 * F.f_noise_rel * (1.0 + fabs(f))) {
                        status = FIT_STATUS_STALLED;
                        next = kDone;
                    }
                    stall_mark = true;
                }
            } else if (st.hn > 0) {   // retry from steepest descent
                __syncthreads();
                if (tid == 0) reset_history(st);
            } else {
                status = FIT_STATUS_LINESEARCH_FAIL;
                next = kDone;
            }
        }
    }

    // ---- direction d = -H g: fused dot products, scalar two-loop, one combination ------------
    while (next == kDirection) {
        __syncthreads();
        fused_dots(V.S, V.Y, pending ? V.Y + (int64_t)st.head * fit_vec_pitch(P) : nullptr, V.g, P,
                   (unsigned)st.occ | (pending ? 1u << st.head : 0u), S.dots);
        if (tid < 32) lbfgs_scalars(S, F.hist, pending);
        pending = false;
        __syncthreads();
        {
            // d = -(cg g + sum cs_j s_j + sum cy_j y_j), four consecutive entries per thread
            // (16-byte loads; the pitch padding of d receives values nothing reads)
            const float cg = S.cg;
            const unsigned occ = (unsigned)st.occ;
            const int Pp = fit_vec_pitch(P);
            for (int k = tid; k < (Pp >> 2); k += blockDim.x) {
                const float4 gv = reinterpret_cast<const float4 *>(V.g)[k];
                float4 h = make_float4(cg * gv.x, cg * gv.y, cg * gv.z, cg * gv.w);
                for (int j = 0; j < F.hist; ++j)
                    if ((occ >> j) & 1u) {
                        const float a = S.cs[j], b = S.cy[j];
                        const float4 sv = reinterpret_cast<const float4 *>(V.S + (int64_t)j * Pp)[k];
                        const float4 yv = reinterpret_cast<const float4 *>(V.Y + (int64_t)j * Pp)[k];
                        h.x = fmaf(b, yv.x, fmaf(a, sv.x, h.x));
                        h.y = fmaf(b, yv.y, fmaf(a, sv.y, h.y));
                        h.z = fmaf(b, yv.z, fmaf(a, sv.z, h.z));
                        h.w = fmaf(b, yv.w, fmaf(a, sv.w, h.w));
                    }
                reinterpret_cast<float4 *>(V.d)[k] = make_float4(-h.x, -h.y, -h.z, -h.w);
            }
        }
        __syncthreads();
        const double gd = -S.gHg;
        const int hn = st.hn;
        edm = -0.5 * gd;
        if (edm < F.edm_tol && since_restart >= F.hist) {
            if (restarts_left == 0) {
                status = FIT_STATUS_CONVERGED;
                next = kDone;
                break;
            }
            // drop the history and rebuild it (at least hist iterations): the fresh pairs come
            // from the directions still moving, the flat ones a short history may not have seen
            --restarts_left;
            since_restart = 0;
            __syncthreads();
            if (tid == 0) reset_history(st);
            continue;
        }
        if (iters >= F.max_iter) {
            status = FIT_STATUS_MAXITER;
            next = kDone;
            break;
        }
        if (global_ns() > F.deadline) {
            status = FIT_STATUS_TIMEOUT;
            next = kDone;
            break;
        }
        // first trial: the unit step, or a step of length 1 along steepest descent
        dphi0 = gd;
        eps_f = F.f_noise_rel * (1.0 + fabs(f));
        if (hn == 0) {
            const double dn = (double)S.cg * sqrt(S.dots[kNDots - 1]);
            alpha = fmin(1.0, 1.0 / fmax(dn, 1e-30));
        } else {
            alpha = 1.0;
        }
        lo = 0.0;
        flo = f;
        dlo = dphi0;
        hi = fhi = dhi = INFINITY;
        a_cr = INFINITY;
        f_cr = 0.0;
        have_lo = false;
        ls_it = 0;
        next = kTrial;
    }
    if (next == kTrial) {
        const float af = (float)alpha;
        for (int i = tid; i < P; i += blockDim.x) V.zt[i] = fmaf(af, V.d[i], V.z[i]);
    }
    __syncthreads();
    if (tid == 0) {
        st.f = f;
        st.edm = edm;
        st.alpha = alpha;
        st.dphi0 = dphi0;
        st.eps_f = eps_f;
        st.lo = lo;
        st.flo = flo;
        st.dlo = dlo;
        st.hi = hi;
        st.fhi = fhi;
        st.dhi = dhi;
        st.a_cr = a_cr;
        st.f_cr = f_cr;
        st.phase = next == kTrial ? kPhTrial : kPhDone;
        st.ls_it = ls_it;
        st.have_lo = have_lo;
        st.pending = pending;
        st.restarts_left = restarts_left;
        st.since_restart = since_restart;
        st.iters = iters;
        st.n_evals = n_evals;
        st.status = status;
        if (stall_mark) {
            st.f_win = f;
            st.win_it = iters;
        }
    }
    __syncthreads();
    return next == kTrial;
}

__device__ __forceinline__ void init_state(FitState &st) {
    st.phase = kPhStart;
    st.f = INFINITY;
    st.edm = INFINITY;
    st.iters = 0;
    st.n_evals = 0;
    st.win_it = 0;
    st.f_win = INFINITY;
    st.status = FIT_STATUS_MAXITER;
    st.pending = 0;
    st.have_lo = 0;
    st.ls_it = 0;
    reset_history(st);
}

// Start point z0 = J^-1 (theta_start - theta0) into z (theta_start = theta0 if st == nullptr);
// pd is scratch. Ends with a barrier.
__device__ void start_z(const DevModel &m, const double *st, float *z, float *pd) {
    const int tid = threadIdx.x, P = m.P;
    for (int i = tid; i < P; i += blockDim.x) {
        const float dd = st ? (float)(st[i] - m.theta0[i]) : 0.f;
        pd[i] = dd;
        const float s = m.zscale[i];
        if (s > 0.f) z[i] = dd / s;
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int b = 0; b < m.n_blocks; ++b) {
        const int n = m.blk_size[b];
        const int *idx = m.blk_idx + m.blk_idx_off[b];
        const float *W = m.blk_W + m.blk_mat_off[b];
        for (int i = warp; i < n; i += nw) {
            float s = 0.f;
            for (int j = lane; j <= i; j += 32) s = fmaf(W[(int64_t)i * n + j], pd[idx[j]], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) z[idx[i]] = s;
        }
    }
    __syncthreads();
}

// Result: theta = theta0 + J z in double, and the fit's summary.
// Held parameters (fixed) are reported at their start values exactly (their z carries the
// start's FP32 rounding, ~1e-8 relative).
__device__ void write_result(const DevModel &m, const FitState &st, const float *z, double *best,
                             fit_result *out, const double *start, const uint8_t *fixed) {
    const int tid = threadIdx.x;
    for (int i = tid; i < m.P; i += blockDim.x) {
        const float s = m.zscale[i];
        if (fixed && fixed[i]) best[i] = start ? start[i] : m.theta0[i];
        else if (s > 0.f) best[i] = m.theta0[i] + (double)s * (double)z[i];
    }
    for (int b = 0; b < m.n_blocks; ++b) {
        const int n = m.blk_size[b];
        const int *idx = m.blk_idx + m.blk_idx_off[b];
        const double *L = m.blk_L64 + m.blk_mat_off[b];
        for (int i = tid; i < n; i += blockDim.x) {
            double s = 0.0;
            for (int j = 0; j <= i; ++j) s += L[(int64_t)i * n + j] * (double)z[idx[j]];
            best[idx[i]] = m.theta0[idx[i]] + s;
        }
    }
    if (tid == 0) {
        fit_result r;
        r.nll_min = st.f;
        r.edm = st.edm;
        r.iters = st.iters;
        r.n_evals = st.n_evals;
        r.status = st.status;
        r.pad = 0;
        *out = r;
    }
}

// At most 128 threads; MINB resident blocks per SM (4: <= 128 registers, 5: <= 96). Each block
// fits one instance at a time, so MINB instances share an SM and cover each other's barrier and
// load latencies. With the working set in shared memory four blocks of the larger register
// budget measured faster; with it in global memory (L2) the fifth instance pays for itself.
// NOSC = 4: models of Eq. 1 or the three-flavour formula with the overlap-length energy
// correction; NOSC = 6: any model, the 3+1 formula and the spline correction included (a
// separate build, so that the common case carries none of their registers).
// PRE: the preconditioned build (fits in w, z = T w), used when the launch asks for it and every
// model of the batch has its preconditioner.
template <int MINB, int NOSC, bool PRE>
__global__ void __launch_bounds__(128, MINB) fit_kernel(FitArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FitSmem &S = *reinterpret_cast<FitSmem *>(smem_raw);
    float *dyn = reinterpret_cast<float *>(smem_raw + sizeof(FitSmem));
    float *gws = A.ws_global + (int64_t)blockIdx.x * A.ws_stride;
    FitParams F;
    F.hist = A.hist;
    F.max_iter = A.max_iter;
    F.max_ls = A.max_ls;
    F.restarts = A.restarts;
    F.edm_tol = A.edm_tol;
    F.f_noise_rel = A.f_noise_rel;
    F.deadline = global_ns() + A.budget_ns;   // per-block clock budget
    const int tid = threadIdx.x;

    while (true) {
        if (tid == 0) S.inst = atomicAdd(A.queue, 1);
        __syncthreads();
        const int q = S.inst;
        __syncthreads();
        if (q >= A.n_inst) break;
        const int ii = A.order ? A.order[q] : q;   // queue position -> instance
        const fit_instance in = A.inst[ii];
        copy_model(&S.m, A.models + in.model);
        if (PRE && A.pre_tab) {   // the preconditioner of the datasets this instance fits
            if (tid == 0) {
                const uint32_t mk = in.mask & ((1u << S.m.n_ds) - 1u);
                const PreEntry *e = A.pre_tab + (int64_t)in.model * A.pre_per_model;
                for (int k = 0; k < A.pre_per_model; ++k)
                    if (e[k].Q && e[k].mask == mk) {
                        S.m.pre_Q = e[k].Q;
                        S.m.pre_c = e[k].c;
                        S.m.pre_r = e[k].r;
                        break;
                    }
            }
            __syncthreads();
        }
        const DevModel &m = S.m;
        const int P = m.P;
        // workspace: the 12 working vectors and the evaluation workspace in shared memory when
        // they fit, else in this block's global slice; the history in shared memory after them
        // unless it is placed in the global slice (hist_global)
        // (global slice: history first, then the rest)
        const int hfl = fit_hist_floats(P, F.hist), loc = fit_work_floats(P) + ((m.ws_eval_floats + 3) & ~3);
        const bool loc_smem = loc + (A.hist_global ? 0 : hfl) <= A.smem_floats;
        float *base = loc_smem ? dyn : gws + (A.hist_global ? hfl : 0);
        float *hbase = A.hist_global ? gws : base + loc;
        FitVecs V = carve_fit_vecs(base, hbase, P, F.hist);
        const EvalWs ws = carve_eval_ws(base + fit_work_floats(P), m.N_t, m.C, m.max_reco, m.n_osc);
        const float *data = A.data + in.data_off;
        constexpr bool pre = PRE;
        if (tid == 0) init_state(S.st);
        __syncthreads();
        if (global_ns() > F.deadline) {
            for (int i = tid; i < P; i += blockDim.x) V.z[i] = 0.f;
            if (tid == 0) S.st.status = FIT_STATUS_TIMEOUT;
            __syncthreads();
        } else {
            start_z(m, A.start ? A.start + in.param_off : nullptr, V.zt, V.pd);
            const uint8_t *fx = A.fixed ? A.fixed + in.param_off : nullptr;
            if (pre) pre_apply(m, m.pre_c + m.pre_r, V.zt, V.zt, S.pre_u, fx);   // w0 = T^-1 z0
            while (true) {
                const double fa = pre ? eval_w<NOSC>(m, V.zt, V.gt, V, ws, data, in.mask, S, fx)
                                      : eval_z<NOSC>(m, V.zt, V.gt, V, ws, data, in.mask, S, fx);
                if (!fit_decide(S, V, P, fa, F)) break;
            }
        }
        const float *zres = V.z;
        if (pre) {   // back to z = T w
            pre_apply(m, m.pre_c, V.z, V.zw, S.pre_u, A.fixed ? A.fixed + in.param_off : nullptr);
            zres = V.zw;
        }
        write_result(m, S.st, zres, A.best + in.param_off, A.results + ii,
                     A.start ? A.start + in.param_off : nullptr, A.fixed ? A.fixed + in.param_off : nullptr);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// lockstep engine
// ------------------------------------------------------------------------------------
size_t ls_state_bytes() { return sizeof(FitState); }
size_t ls_step_smem_bytes() { return sizeof(FitSmem); }

struct LsEvalSmem {
    DevModel m;
    double red[kMaxWarps * 24 + 24];
    int status;
};

size_t ls_eval_smem_bytes(int P, int ws_floats) {
    return sizeof(LsEvalSmem) + sizeof(float) * (2 * (size_t)P + (size_t)ws_floats);
}

__device__ __forceinline__ FitVecs ls_vecs(const LsArgs &A, int g, int P) {
    float *base = A.vec + (int64_t)g * A.vec_stride;
    return carve_fit_vecs(base, base + fit_work_floats(P), P, A.hist);
}

__device__ __forceinline__ void copy_state(FitState *dst, const FitState *src) {
    const int n = (int)(sizeof(FitState) / sizeof(double));
    const double *s = reinterpret_cast<const double *>(src);
    double *d = reinterpret_cast<double *>(dst);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ FitParams ls_params(const LsArgs &A) {
    FitParams F;
    F.hist = A.hist;
    F.max_iter = A.max_iter;
    F.max_ls = A.max_ls;
    F.restarts = A.restarts;
    F.edm_tol = A.edm_tol;
    F.f_noise_rel = A.f_noise_rel;
    F.deadline = *A.deadline;
    return F;
}

// Start points, theta of the first evaluation, state, and the first active list (all of them).
__global__ void __launch_bounds__(128) ls_init_kernel(LsArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FitSmem &S = *reinterpret_cast<FitSmem *>(smem_raw);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *A.deadline = global_ns() + A.budget_ns;
        *A.n_act_next = A.n;
    }
    copy_model(&S.m, A.model);
    const DevModel &m = S.m;
    const int P = m.P, nd = m.n_ds;
    for (int g = blockIdx.x; g < A.n; g += gridDim.x) {
        const fit_instance in = A.inst[A.group[g]];
        FitVecs V = ls_vecs(A, g, P);
        start_z(m, A.start ? A.start + in.param_off : nullptr, V.zt, V.pd);
        if (A.precond) {   // w0 = T^-1 z0; the trial's z = T w0 is kept in zw
            const uint8_t *fx = A.fixed ? A.fixed + in.param_off : nullptr;
            pre_apply(m, m.pre_c + m.pre_r, V.zt, V.zt, S.pre_u, fx);
            pre_apply(m, m.pre_c, V.zt, V.zw, S.pre_u, fx);
            theta_of_z(m, V.zw, V.pv, V.pd);
        } else {
            theta_of_z(m, V.zt, V.pv, V.pd);
        }
        for (int i = threadIdx.x; i < nd * P; i += blockDim.x) A.gsl[(int64_t)g * nd * P + i] = 0.f;
        if (threadIdx.x == 0) {
            init_state(S.st);
            A.stat[g] = 0;
            A.act_next[g] = g;
        }
        __syncthreads();
        copy_state(A.state + g, &S.st);
        __syncthreads();
    }
}

// Forward pass and likelihood of one (instance, dataset) per block iteration: stages A (no
// partials), B, C, C2; stores the dataset's -2lnL, dD/dmu and the efficiency / background
// gradient contributions.
template <int NOSC, bool SPL>
__device__ __forceinline__ void ls_forward_body(LsArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LsEvalSmem &S = *reinterpret_cast<LsEvalSmem *>(smem_raw);
    copy_model(&S.m, A.model);
    const DevModel &m = S.m;
    const int P = m.P, nd = m.n_ds, na = *A.n_act;
    float *pv = reinterpret_cast<float *>(smem_raw + sizeof(LsEvalSmem));
    float *pd = pv + P;
    float *wsb = A.ws_in_smem ? pd + P : A.ws_global + (int64_t)blockIdx.x * A.ws_stride;
    EvalWs ws;
    ws.u = wsb;
    ws.v = ws.u + m.N_t;
    ws.f0 = ws.v + m.N_t;
    ws.gmu = ws.f0 + m.max_reco;
    ws.ts = ws.ptot = ws.dp = ws.pcw = nullptr;
    for (int it = blockIdx.x; it < na * nd; it += gridDim.x) {
        const int g = A.act[it / nd], d = it % nd;
        const fit_instance in = A.inst[A.group[g]];
        const int64_t gd = (int64_t)g * nd + d;
        if (!((in.mask >> d) & 1u)) {
            if (threadIdx.x == 0) A.nll_ds[gd] = 0.0;
            continue;
        }
        const FitVecs V = ls_vecs(A, g, P);
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            pv[i] = V.pv[i];
            pd[i] = V.pd[i];
        }
        if (threadIdx.x == 0) S.status = 0;
        __syncthreads();
        DsCtxT<NOSC> c;
        double nll = 0.0;
        if (ds_setup(m, d, pv, pd, c, &S.status)) {
            ds_signal<false>(m, d, pv, pd, c, ws);
            ds_remap<SPL>(m, d, c, ws);
            nll = ds_fold_lik(m, d, pv, pd, c, A.data + in.data_off, ws, A.gsl + gd * P, S.red, &S.status,
                              nullptr);
            const int nr = m.ds[d].n_reco;
            float *gm = A.gmu + gd * m.max_reco;
            for (int j = threadIdx.x; j < nr; j += blockDim.x) gm[j] = ws.gmu[j];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            A.nll_ds[gd] = nll;
            if (S.status) atomicOr(&A.stat[g], S.status);
        }
        __syncthreads();
    }
}

// basic build (Eq. 1 / three-flavour, overlap correction) and general build (any model)
__global__ void __launch_bounds__(128) ls_forward_kernel(LsArgs A) { ls_forward_body<4, false>(A); }
__global__ void __launch_bounds__(128) ls_forward_kernel6(LsArgs A) {
    if (A.model->osc_mode == FIT_OSC_STERILE4)
        ls_forward_body<6, true>(A);
    else
        ls_forward_body<4, true>(A);
}

// Adjoint of one (instance, dataset) per block iteration: stage A again with the partials,
// then stages D, E, F into the dataset's gradient slice.
template <int NOSC, bool SPL>
__device__ __forceinline__ void ls_adjoint_body(LsArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LsEvalSmem &S = *reinterpret_cast<LsEvalSmem *>(smem_raw);
    copy_model(&S.m, A.model);
    const DevModel &m = S.m;
    const int P = m.P, nd = m.n_ds, na = *A.n_act;
    float *pv = reinterpret_cast<float *>(smem_raw + sizeof(LsEvalSmem));
    float *pd = pv + P;
    float *wsb = A.ws_in_smem ? pd + P : A.ws_global + (int64_t)blockIdx.x * A.ws_stride;
    const EvalWs ws = carve_eval_ws(wsb, m.N_t, m.C, m.max_reco, m.n_osc);
    for (int it = blockIdx.x; it < na * nd; it += gridDim.x) {
        const int g = A.act[it / nd], d = it % nd;
        const fit_instance in = A.inst[A.group[g]];
        if (!((in.mask >> d) & 1u) || A.stat[g] != 0) continue;
        const int64_t gd = (int64_t)g * nd + d;
        const FitVecs V = ls_vecs(A, g, P);
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            pv[i] = V.pv[i];
            pd[i] = V.pd[i];
        }
        const int nr = m.ds[d].n_reco;
        const float *gm = A.gmu + gd * m.max_reco;
        for (int j = threadIdx.x; j < nr; j += blockDim.x) ws.gmu[j] = gm[j];
        if (threadIdx.x == 0) S.status = 0;
        __syncthreads();
        DsCtxT<NOSC> c;
        if (ds_setup(m, d, pv, pd, c, &S.status)) {
            ds_signal<true>(m, d, pv, pd, c, ws);
            ds_adjoint<SPL>(m, d, pv, pd, c, ws, A.gsl + gd * P, S.red);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(128) ls_adjoint_kernel(LsArgs A) { ls_adjoint_body<4, false>(A); }
__global__ void __launch_bounds__(128) ls_adjoint_kernel6(LsArgs A) {
    if (A.model->osc_mode == FIT_OSC_STERILE4)
        ls_adjoint_body<6, true>(A);
    else
        ls_adjoint_body<4, true>(A);
}

// ---- lockstep rounds with the folds on the tensor cores (engine 2) ---------------------------
// Between these kernels the library runs, per dataset d, F_d = V_d R^T and GV_d = G_d R as
// split-TF32 GEMMs over the active instances (row a of each matrix = active position a). Each
// (instance, dataset) pair keeps its own evaluation workspace for the whole round, so the
// survival partials of the forward pass serve the adjoint without being recomputed.

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t b = __float_as_uint(x);
    b = (b + 0x1000u) & 0xFFFFE000u;   // nearest value with 10 mantissa bits
    return __uint_as_float(b);
}

__device__ __forceinline__ EvalWs ls_pair_ws(const LsArgs &A, const DevModel &m, int it) {
    return carve_eval_ws(A.ws_global + (int64_t)it * A.ws_stride, m.N_t, m.C, m.max_reco, m.n_osc);
}

// Stage A (with the partials) and B per (instance, dataset); v as TF32 high part and rest.
template <int NOSC, bool SPL>
__device__ __forceinline__ void ls_tc_fwd_body(LsArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LsEvalSmem &S = *reinterpret_cast<LsEvalSmem *>(smem_raw);
    copy_model(&S.m, A.model);
    const DevModel &m = S.m;
    const int P = m.P, nd = m.n_ds, na = *A.n_act;
    float *pv = reinterpret_cast<float *>(smem_raw + sizeof(LsEvalSmem));
    float *pd = pv + P;
    for (int it = blockIdx.x; it < na * nd; it += gridDim.x) {
        const int a = it / nd, d = it % nd, g = A.act[a];
        const fit_instance in = A.inst[A.group[g]];
        const int64_t gd = (int64_t)g * nd + d;
        if (!((in.mask >> d) & 1u)) {
            if (threadIdx.x == 0) A.nll_ds[gd] = 0.0;
            continue;
        }
        const EvalWs ws = ls_pair_ws(A, m, it);
        const FitVecs V = ls_vecs(A, g, P);
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            pv[i] = V.pv[i];
            pd[i] = V.pd[i];
        }
        if (threadIdx.x == 0) S.status = 0;
        __syncthreads();
        DsCtxT<NOSC> c;
        if (ds_setup(m, d, pv, pd, c, &S.status)) {
            ds_signal<true>(m, d, pv, pd, c, ws);
            ds_remap<SPL>(m, d, c, ws);
            float *vh = A.vhi + ((int64_t)d * A.n + a) * m.ldt, *vl = A.vlo + ((int64_t)d * A.n + a) * m.ldt;
            for (int t = threadIdx.x; t < m.ldt; t += blockDim.x) {
                const float x = t < m.N_t ? ws.v[t] : 0.f;
                const float hi = tf32_hi(x);
                vh[t] = hi;
                vl[t] = x - hi;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && S.status) atomicOr(&A.stat[g], S.status);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(128) ls_tc_fwd_kernel(LsArgs A) { ls_tc_fwd_body<4, false>(A); }
__global__ void __launch_bounds__(128) ls_tc_fwd_kernel6(LsArgs A) {
    if (A.model->osc_mode == FIT_OSC_STERILE4)
        ls_tc_fwd_body<6, true>(A);
    else
        ls_tc_fwd_body<4, true>(A);
}

// Stage C2 per (instance, dataset) from the fold F = R v of the GEMM: -2lnL, dD/dmu (TF32
// high part and rest for the adjoint GEMM), efficiency and background gradients.
template <int NOSC>
__device__ __forceinline__ void ls_tc_lik_body(LsArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LsEvalSmem &S = *reinterpret_cast<LsEvalSmem *>(smem_raw);
    copy_model(&S.m, A.model);
    const DevModel &m = S.m;
    const int P = m.P, nd = m.n_ds, na = *A.n_act;
    float *pv = reinterpret_cast<float *>(smem_raw + sizeof(LsEvalSmem));
    float *pd = pv + P;
    for (int it = blockIdx.x; it < na * nd; it += gridDim.x) {
        const int a = it / nd, d = it % nd, g = A.act[a];
        const fit_instance in = A.inst[A.group[g]];
        const int64_t gd = (int64_t)g * nd + d;
        if (!((in.mask >> d) & 1u) || A.stat[g] != 0) continue;
        const EvalWs ws = ls_pair_ws(A, m, it);
        const FitVecs V = ls_vecs(A, g, P);
        const int nr = m.ds[d].n_reco;
        const float *fr = A.fbuf + ((int64_t)d * A.n + a) * A.ldf;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            pv[i] = V.pv[i];
            pd[i] = V.pd[i];
        }
        for (int j = threadIdx.x; j < nr; j += blockDim.x) ws.f0[j] = fr[j];
        if (threadIdx.x == 0) S.status = 0;
        __syncthreads();
        DsCtxT<NOSC> c;
        double nll = 0.0;
        if (ds_setup(m, d, pv, pd, c, &S.status)) {
            nll = ds_lik(m, d, pv, pd, c, A.data + in.data_off, ws, A.gsl + gd * P, S.red, &S.status, nullptr);
            float *gh = A.ghi + ((int64_t)d * A.n + a) * A.ldr, *gl = A.glo + ((int64_t)d * A.n + a) * A.ldr;
            for (int j = threadIdx.x; j < A.ldr; j += blockDim.x) {
                const float x = j < nr ? ws.gmu[j] : 0.f;
                const float hi = tf32_hi(x);
                gh[j] = hi;
                gl[j] = x - hi;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            A.nll_ds[gd] = nll;
            if (S.status) atomicOr(&A.stat[g], S.status);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(128) ls_tc_lik_kernel(LsArgs A) { ls_tc_lik_body<4>(A); }
__global__ void __launch_bounds__(128) ls_tc_lik_kernel6(LsArgs A) {
    if (A.model->osc_mode == FIT_OSC_STERILE4)
        ls_tc_lik_body<6>(A);
    else
        ls_tc_lik_body<4>(A);
}

// Stages E and F per (instance, dataset) from GV = R^T dD/dmu of the GEMM (gv = eff GV).
template <int NOSC, bool SPL>
__device__ __forceinline__ void ls_tc_adj_body(LsArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LsEvalSmem &S = *reinterpret_cast<LsEvalSmem *>(smem_raw);
    copy_model(&S.m, A.model);
    const DevModel &m = S.m;
    const int P = m.P, nd = m.n_ds, na = *A.n_act;
    float *pv = reinterpret_cast<float *>(smem_raw + sizeof(LsEvalSmem));
    float *pd = pv + P;
    for (int it = blockIdx.x; it < na * nd; it += gridDim.x) {
        const int a = it / nd, d = it % nd, g = A.act[a];
        const fit_instance in = A.inst[A.group[g]];
        if (!((in.mask >> d) & 1u) || A.stat[g] != 0) continue;
        const int64_t gd = (int64_t)g * nd + d;
        const EvalWs ws = ls_pair_ws(A, m, it);
        const FitVecs V = ls_vecs(A, g, P);
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            pv[i] = V.pv[i];
            pd[i] = V.pd[i];
        }
        if (threadIdx.x == 0) S.status = 0;
        __syncthreads();
        DsCtxT<NOSC> c;
        if (ds_setup(m, d, pv, pd, c, &S.status)) {
            const float *gr = A.gvbuf + ((int64_t)d * A.n + a) * m.ldt;
            for (int k = threadIdx.x; k < m.N_t; k += blockDim.x) ws.v[k] = pmul(c.eff, gr[k]);
            __syncthreads();
            ds_adjoint_rest<SPL>(m, d, pv, pd, c, ws, A.gsl + gd * P, S.red);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(128) ls_tc_adj_kernel(LsArgs A) { ls_tc_adj_body<4, false>(A); }
__global__ void __launch_bounds__(128) ls_tc_adj_kernel6(LsArgs A) {
    if (A.model->osc_mode == FIT_OSC_STERILE4)
        ls_tc_adj_body<6, true>(A);
    else
        ls_tc_adj_body<4, true>(A);
}

// Minimiser step per active instance: gathers the round's evaluation (dataset sums, prior,
// gradient in z), runs fit_decide, and either prepares theta of the next trial point and puts
// the instance on the next active list, or writes its result.
__global__ void __launch_bounds__(128) ls_step_kernel(LsArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FitSmem &S = *reinterpret_cast<FitSmem *>(smem_raw);
    copy_model(&S.m, A.model);
    const DevModel &m = S.m;
    const int P = m.P, nd = m.n_ds, na = *A.n_act;
    const FitParams F = ls_params(A);
    for (int a = blockIdx.x; a < na; a += gridDim.x) {
        const int g = A.act[a];
        const int ii = A.group[g];
        const fit_instance in = A.inst[ii];
        FitVecs V = ls_vecs(A, g, P);
        copy_state(&S.st, A.state + g);
        // theta gradient = sum of the dataset slices in a fixed order; the slices are cleared
        float *gs = A.gsl + (int64_t)g * nd * P;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            float t = 0.f;
            for (int d = 0; d < nd; ++d) {
                if ((in.mask >> d) & 1u) t += gs[(int64_t)d * P + i];
                gs[(int64_t)d * P + i] = 0.f;
            }
            V.gth[i] = t;
        }
        const int st = A.stat[g];
        double fa = 0.0;
        for (int d = 0; d < nd; ++d)
            if ((in.mask >> d) & 1u) fa += A.nll_ds[(int64_t)g * nd + d];
        __syncthreads();
        const uint8_t *fx = A.fixed ? A.fixed + in.param_off : nullptr;
        if (st != 0) {
            fa = INFINITY;
        } else if (A.precond) {   // z of the trial in zw; g_w = T g_z
            fa += eval_z_prior(m, V.zw, V.gth, V.gzw, S.red);
            hold_fixed(fx, V.gzw, P);
            __syncthreads();
            pre_apply(m, m.pre_c, V.gzw, V.gt, S.pre_u, fx);
        } else {
            fa += eval_z_prior(m, V.zt, V.gth, V.gt, S.red);
            hold_fixed(fx, V.gt, P);
        }
        const bool more = fit_decide(S, V, P, fa, F);
        if (more) {
            if (A.precond) {
                pre_apply(m, m.pre_c, V.zt, V.zw, S.pre_u, fx);
                theta_of_z(m, V.zw, V.pv, V.pd);
            } else {
                theta_of_z(m, V.zt, V.pv, V.pd);
            }
            if (threadIdx.x == 0) {
                A.stat[g] = 0;
                A.act_next[atomicAdd(A.n_act_next, 1)] = g;
            }
        } else {
            const float *zres = V.z;
            if (A.precond) {   // back to z = T w
                pre_apply(m, m.pre_c, V.z, V.zw, S.pre_u, fx);
                zres = V.zw;
            }
            write_result(m, S.st, zres, A.best + in.param_off, A.results + ii,
                         A.start ? A.start + in.param_off : nullptr, fx);
        }
        __syncthreads();
        copy_state(A.state + g, &S.st);
        __syncthreads();
    }
}

const void *fit_kernel_func(int variant, int n_osc, bool pre) {
    if (pre) {
        if (n_osc == 6)
            return variant == 5 ? reinterpret_cast<const void *>(&fit_kernel<5, 6, true>)
                                : reinterpret_cast<const void *>(&fit_kernel<4, 6, true>);
        return variant == 5 ? reinterpret_cast<const void *>(&fit_kernel<5, 4, true>)
                            : reinterpret_cast<const void *>(&fit_kernel<4, 4, true>);
    }
    if (n_osc == 6)
        return variant == 5 ? reinterpret_cast<const void *>(&fit_kernel<5, 6, false>)
                            : reinterpret_cast<const void *>(&fit_kernel<4, 6, false>);
    return variant == 5 ? reinterpret_cast<const void *>(&fit_kernel<5, 4, false>)
                        : reinterpret_cast<const void *>(&fit_kernel<4, 4, false>);
}

size_t fit_smem_bytes(int floats) { return sizeof(FitSmem) + sizeof(float) * (size_t)floats; }

}  // namespace fitcore
