// Device-side model layout and block-level building blocks of the forward-folding fit.
//
// One thread block evaluates one parameter vector of one model: the expectation of every
// dataset (survival x reweights on the fine true grid, energy correction by overlap length,
// banded response fold, backgrounds), the Poisson -2lnL and its adjoint gradient. The same
// device functions serve the batched evaluation kernels and the persistent fit kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fitcore.h"

namespace fitcore {

constexpr int kMaxWarps = 16;      // blocks of at most 512 threads
constexpr int kMaxBkgDs = 6;       // backgrounds per dataset
constexpr int kMaxOsc = 6;         // survival parameters (6 for the 3+1 formula, else 4)

struct DevDetector {
    int n_reco;
    int col_w;               // padded width of the column bands
    const int *row_lo;       // [N_r] first true bin of row j's band
    const int *row_len;      // [N_r] band length
    const int *row_off;      // [N_r] offset of the row's band in rrow
    const float *rrow;       // packed row bands
    const int *col_lo;       // [N_t] first reco row of column k's band
    const float *rcol;       // [col_w x N_t]: rcol[b * N_t + k] = R[col_lo[k] + b][k] (0 past the band)
    const float *rdense_hi;  // [N_r x ldt] dense response, TF32-exact high part (tensor-core fold)
    const float *rdense_lo;  // [N_r x ldt] R - rdense_hi
    const int *col_len;      // [N_t] band length of column k
    const float *rdt_hi;     // [N_t x ldr] R^T, TF32-exact high part (tensor-core adjoint fold)
    const float *rdt_lo;     // [N_t x ldr] R^T - rdt_hi
    int ldr;                 // row stride of R^T (N_r rounded up to 4)
};

struct DevBkg {
    const float *tmpl;       // [N_r] expected counts at nominal
    const int *shape_idx;    // [N_r] parameter of delta_j or -1
    int rate_idx;
    int pad;
};

struct DevDataset {
    int det, n_reco, data_off;
    int norm_idx, eff_idx;
    int esc_idx[3];
    float a1_off;            // theta0(a1) - 1, so that a1 - 1 = a1_off + (theta - theta0)
    int bkg_begin, bkg_end;  // backgrounds of this dataset in DevModel::bkg
    int n_sp;                // distinct shape parameters used by this dataset
    const float *t;          // [N_t] un-oscillated signal
    const int *shape_idx;    // [N_t]
    const int *sp_param;     // [n_sp] parameter index
    const int *sp_ptr;       // [n_sp + 1] CSR offsets into sp_k
    const int *sp_k;         // true bins of each shape parameter
    float w[FIT_MAX_CORES];  // core flux shares
    float kl_hi[FIT_MAX_CORES], kl_lo[FIT_MAX_CORES];  // K L_dc / pi as a float pair (half-turns)
};

struct DevModel {
    int P, N_t, C, n_ds, n_data, osc_mode, n_blocks, n_bkg;
    float e_lo, de, inv_de;
    int n_osc;               // survival parameters of osc_mode: 4, or 6 (FIT_OSC_STERILE4)
    int remap_mode;          // FIT_REMAP_OVERLAP or FIT_REMAP_SPLINE
    int osc_idx[kMaxOsc];
    float osc_val[kMaxOsc];
    float osc_val_lo[kMaxOsc];   // low parts of the constant survival parameters
    double osc_val_d[kMaxOsc];   // the constant survival parameters in double
    int core_power_idx[FIT_MAX_CORES];
    const float *e_edge;     // [N_t + 1]
    const float *inv_e_hi;   // [N_t] 1 / E_k (true-bin centre) as a float pair
    const float *inv_e_lo;
    DevDataset ds[FIT_MAX_DATASETS];
    DevDetector det[FIT_MAX_DETECTORS];
    DevBkg bkg[FIT_MAX_BACKGROUNDS];
    // parameters, priors and the transformation layer
    const double *theta0;    // [P]
    const float *theta0_f;   // [P] theta0 rounded to float
    const float *theta0_lo;  // [P] theta0 - theta0_f (the low part of a float pair)
    const float *zscale;     // [P] sigma (individual prior) or scale (free); 0 in a block
    const float *prior_inv;  // [P] 1/sigma for individually constrained parameters, else 0
    const int *blk_size;     // [n_blocks]
    const int *blk_idx_off;  // [n_blocks]
    const int *blk_idx;      // concatenated parameter indices
    const int *blk_first;    // [n_blocks] first index when a block's indices are consecutive, else -1
    const int64_t *blk_mat_off;  // [n_blocks] offset of the block's m x m matrices
    const float *blk_L;      // lower Cholesky factor of V (row-major, dense)
    const float *blk_W;      // L^-1 (row-major, dense lower triangle)
    const double *blk_L64;   // L in double (final theta of a fit)
    const float *asimov;     // [n_data] expectation at theta0
    const int *slot_ds;      // [n_data] dataset of each data bin
    int ws_eval_floats;      // per-block workspace of one evaluation
    int max_reco;
    int ldt;                 // row stride of the dense response (N_t rounded up to 4)
    // Fisher preconditioner (nullptr until built): z = T w, T = I + Q diag(c) Q^T; pre_Q holds
    // Q^T as pre_r rows on the vector pitch, pre_c the r coefficients c then the r of T^-1
    const float *pre_Q, *pre_c;
    int pre_r;
};

// ------------------------------------------------------------------------------------
// Reductions: FP32 within a warp, FP64 across warps.
// ------------------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void warp_sum(float (&v)[N]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
}

// Sums N per-thread values over the block. red: shared scratch of kMaxWarps * N doubles
// (+ N result slots). Every thread returns the N totals. Contains two __syncthreads.
template <int N>
__device__ __forceinline__ void block_sum(float (&v)[N], double *red, double (&out)[N]) {
    warp_sum<N>(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) red[warp * N + i] = (double)v[i];
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w * N + threadIdx.x];
        red[kMaxWarps * N + threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = red[kMaxWarps * N + i];
    __syncthreads();
}

// Same with double per-thread inputs (used where a thread already sums many terms).
template <int N>
__device__ __forceinline__ void block_sum_d(double (&v)[N], double *red, double (&out)[N]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) red[warp * N + i] = v[i];
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w * N + threadIdx.x];
        red[kMaxWarps * N + threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = red[kMaxWarps * N + i];
    __syncthreads();
}

// ------------------------------------------------------------------------------------
// Survival probability with phase arithmetic in float pairs.
// ------------------------------------------------------------------------------------
// Phase in half-turns: y = x / pi = (dm_hi + dm_lo) * (c_hi + c_lo), c = K L / (pi E), carried
// as a float pair. The probability depends on sin^2 x and sin 2x only, so y is reduced by
// its nearest integer, which is exact (y_hi - rint(y_hi) is representable), and sin, cos of
// pi r, |r| <= 1/2, come from sincospif. The pair keeps r accurate to ~1e-8 even at 50 km
// (y ~ 30), and no pi constant or multi-word reduction enters the arithmetic.
__device__ __forceinline__ void phase_sc(float dm, float dm_lo, float c_hi, float c_lo, float &s,
                                         float &c) {
    const float yh = dm * c_hi;
    const float yl = fmaf(dm, c_hi, -yh) + fmaf(dm, c_lo, dm_lo * c_hi);
    const float r = (yh - rintf(yh)) + yl;
    sincospif(r, &s, &c);
}

// sin^2(pi r) for |r| <= 1/2: u q(u), u = r^2, q a degree-7 polynomial fitted for the
// smallest largest absolute error (Lawson iteration; sin2pi_fit.py in this directory). Its
// FP32 evaluation is within 1.8e-7 of sin^2.
__device__ __forceinline__ float sin2pi(float r) {
    const float u = r * r;
    float q = -0.122019291f;
    q = fmaf(q, u, 0.848584056f);
    q = fmaf(q, u, -3.94964409f);
    q = fmaf(q, u, 13.2128229f);
    q = fmaf(q, u, -30.1222954f);
    q = fmaf(q, u, 42.7284088f);
    q = fmaf(q, u, -32.469696f);
    q = fmaf(q, u, 9.86960411f);
    return u * q;
}

// sin^2 of the phase pi (dm + dm_lo)(c_hi + c_lo): the half-turn count reduced by its nearest
// integer as in the binned evaluation. Both pairs normalised (|low| <= ulp(high) / 2), so the
// reduced phase stays within 1/2 (the polynomial's range) up to rounding.
__device__ __forceinline__ float sin2_phase(float dm, float dm_lo, float c_hi, float c_lo) {
    const float yh = dm * c_hi;
    const float yl = fmaf(dm, c_hi, -yh) + fmaf(dm, c_lo, dm_lo * c_hi);
    return sin2pi((yh - rintf(yh)) + yl);
}

// Coefficients of the sin^2 terms of P, formed once per evaluation in double from the exact
// parameter values and applied as float pairs (a single FP32 rounding of a coefficient would
// bias every bin coherently).
//   FIT_OSC_EQ1:     P = 1 - C0 sin^2 x_ee - C1 sin^2 x_21,  C0 = sin^2 2th13,
//                    C1 = cos^4 th13 sin^2 2th12
//   FIT_OSC_VACUUM3: P = 1 - C0 sin^2 x_21 - C1 sin^2 x_31 - C2 sin^2 x_32,
//                    C0 = cos^4 th13 sin^2 2th12, C1 = sin^2 2th13 cos^2 th12,
//                    C2 = sin^2 2th13 sin^2 th12
template <int NT>
struct OscCoefN {
    float hi[NT], lo[NT];
};
using OscCoef = OscCoefN<3>;

template <int NT>
__device__ __forceinline__ float cterm(const OscCoefN<NT> &k, int i, float q) {
    return fmaf(q, k.lo[i], k.hi[i] * q);
}

// Float-pair ("double-float") arithmetic: a value h + l with |l| <= ulp(h) / 2, carried in two
// floats (error-free transformations of Knuth's two-sum and the FMA two-product, Dekker's
// normalisation). Used where a few coefficients need more than 24 bits but FP64 would sit on
// the critical path (GB300 runs FP64 at 1/64 of the FP32 rate).
struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 f2_norm(float h, float l) {
    const float s = h + l;
    return F2{s, l - (s - h)};
}

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b.h - bb);
    return f2_norm(s, e + (a.l + b.l));
}

__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p);
    return f2_norm(p, fmaf(a.h, b.l, fmaf(a.l, b.h, e)));
}

__device__ __forceinline__ F2 f2_scale(F2 a, float c) {   // c a power of two
    return F2{a.h * c, a.l * c};
}

__device__ __forceinline__ F2 f2_one_minus(F2 a) { return f2_add(F2{1.f, 0.f}, F2{-a.h, -a.l}); }

// square root: s = sqrtf(h) refined by one Newton step on the residual a - s^2
__device__ __forceinline__ F2 f2_sqrt(F2 a) {
    if (!(a.h > 0.f)) return F2{0.f, 0.f};
    const float s = sqrtf(a.h);
    const float r = fmaf(-s, s, a.h) + a.l;
    return f2_norm(s, r / (2.f * s));
}

// P(L_dc, E_k) and dP/d(eta_i) for the four survival parameters.
//  mode FIT_OSC_EQ1:     eta = (sin^2 2th13, dm2_ee, sin^2 2th12, dm2_21), Eq. 1
//  mode FIT_OSC_VACUUM3: eta = (sin^2 th12, sin^2 th13, dm2_21, dm2_31), exact vacuum P
// eta_lo carries the low parts of the two mass splittings; dx = pi c (dx/d dm2).
__device__ __forceinline__ float survival_mode(int mode, const float (&eta)[4],
                                               const float (&eta_lo)[4], const OscCoef &k,
                                               float c_hi, float c_lo, float (&dP)[4]) {
    const float dx = 3.14159265358979f * c_hi;
    if (mode == FIT_OSC_EQ1) {
        const float S13 = eta[0], S12 = eta[2];
        const float root = sqrtf(fmaxf(1.f - S13, 1e-12f));
        const float c2 = 0.5f * (1.f + root);
        const float c4 = c2 * c2;
        float se, ce, s2, cc2;
        phase_sc(eta[1], eta_lo[1], c_hi, c_lo, se, ce);
        phase_sc(eta[3], eta_lo[3], c_hi, c_lo, s2, cc2);
        const float qe = se * se, q21 = s2 * s2;
        const float P = (1.f - cterm(k, 0, qe)) - cterm(k, 1, q21);
        const float dc4 = -c2 * 0.5f / root;
        dP[0] = -qe - dc4 * S12 * q21;
        dP[1] = -S13 * 2.f * se * ce * dx;
        dP[2] = -c4 * q21;
        dP[3] = -c4 * S12 * 2.f * s2 * cc2 * dx;
        return P;
    } else {
        const float s12 = eta[0], s13 = eta[1];
        const float c12 = 1.f - s12, c13 = 1.f - s13;
        const float S12 = 4.f * s12 * c12, S13 = 4.f * s13 * c13;
        float a21, b21, a31, b31;
        phase_sc(eta[2], eta_lo[2], c_hi, c_lo, a21, b21);
        phase_sc(eta[3], eta_lo[3], c_hi, c_lo, a31, b31);
        const float a32 = a31 * b21 - b31 * a21;   // sin(x31 - x21)
        const float b32 = b31 * b21 + a31 * a21;   // cos(x31 - x21)
        const float q21 = a21 * a21, q31 = a31 * a31, q32 = a32 * a32;
        const float d21 = 2.f * a21 * b21 * dx, d31 = 2.f * a31 * b31 * dx,
                    d32 = 2.f * a32 * b32 * dx;
        const float P = ((1.f - cterm(k, 0, q21)) - cterm(k, 1, q31)) - cterm(k, 2, q32);
        dP[0] = -c13 * c13 * 4.f * (1.f - 2.f * s12) * q21 - S13 * (q32 - q31);
        dP[1] = 2.f * c13 * S12 * q21 - 4.f * (1.f - 2.f * s13) * (c12 * q31 + s12 * q32);
        dP[2] = -c13 * c13 * S12 * d21 + S13 * s12 * d32;
        dP[3] = -S13 * (c12 * d31 + s12 * d32);
        return P;
    }
}

// The sin^2 coefficients of survival_mode from float pairs e of the exact parameter values.
__device__ __forceinline__ OscCoef osc_coef(int mode, const F2 (&e)[4]) {
    F2 cf[3];
    if (mode == FIT_OSC_EQ1) {
        // cos^4 th13 = ((1 + sqrt(1 - sin^2 2th13)) / 2)^2
        const F2 c2 = f2_scale(f2_add(F2{1.f, 0.f}, f2_sqrt(f2_one_minus(e[0]))), 0.5f);
        cf[0] = e[0];
        cf[1] = f2_mul(f2_mul(c2, c2), e[2]);
        cf[2] = F2{0.f, 0.f};
    } else {
        const F2 S12 = f2_scale(f2_mul(e[0], f2_one_minus(e[0])), 4.f);
        const F2 S13 = f2_scale(f2_mul(e[1], f2_one_minus(e[1])), 4.f);
        const F2 c13 = f2_one_minus(e[1]);
        cf[0] = f2_mul(f2_mul(c13, c13), S12);
        cf[1] = f2_mul(S13, f2_one_minus(e[0]));
        cf[2] = f2_mul(S13, e[0]);
    }
    OscCoef k;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        k.hi[i] = cf[i].h;
        k.lo[i] = cf[i].l;
    }
    return k;
}

__device__ __forceinline__ float survival(const DevModel &m, const float (&eta)[4],
                                          const float (&eta_lo)[4], const OscCoef &k,
                                          float c_hi, float c_lo, float (&dP)[4]) {
    return survival_mode(m.osc_mode, eta, eta_lo, k, c_hi, c_lo, dP);
}

// Exact 3+1 vacuum survival (FIT_OSC_STERILE4), one sterile state added to the three-flavour
// formula: eta = (sin^2 th12, sin^2 th13, dm2_21, dm2_31, sin^2 2th14, dm2_41),
//   P = 1 - cos^4 th14 [C0 sin^2 x21 + C1 sin^2 x31 + C2 sin^2 x32]
//         - sin^2 2th14 [cos^2 th13 (cos^2 th12 sin^2 x41 + sin^2 th12 sin^2 x42)
//                        + sin^2 th13 sin^2 x43]
// (the first row of the 4x4 mixing matrix is (c12 c13 c14, s12 c13 c14, s13 c14, s14)), with
// the coefficients k.hi/lo[0..5] of the six sin^2 terms; x32, x42 and x43 from the angle
// differences of x21, x31 and x41.
__device__ __forceinline__ float survival_sterile(const float (&eta)[6], const float (&eta_lo)[6],
                                                  const OscCoefN<6> &k, float c_hi, float c_lo,
                                                  float (&dP)[6]) {
    const float dx = 3.14159265358979f * c_hi;
    const float s12 = eta[0], s13 = eta[1], S14 = eta[4];
    const float c12 = 1.f - s12, c13 = 1.f - s13;
    const float S12 = 4.f * s12 * c12, S13 = 4.f * s13 * c13;
    const float root = sqrtf(fmaxf(1.f - S14, 1e-12f));
    const float c14 = 0.5f * (1.f + root), C4 = c14 * c14;
    float a21, b21, a31, b31, a41, b41;
    phase_sc(eta[2], eta_lo[2], c_hi, c_lo, a21, b21);
    phase_sc(eta[3], eta_lo[3], c_hi, c_lo, a31, b31);
    phase_sc(eta[5], eta_lo[5], c_hi, c_lo, a41, b41);
    const float a32 = a31 * b21 - b31 * a21, b32 = b31 * b21 + a31 * a21;   // x31 - x21
    const float a42 = a41 * b21 - b41 * a21, b42 = b41 * b21 + a41 * a21;   // x41 - x21
    const float a43 = a41 * b31 - b41 * a31, b43 = b41 * b31 + a41 * a31;   // x41 - x31
    const float q21 = a21 * a21, q31 = a31 * a31, q32 = a32 * a32;
    const float q41 = a41 * a41, q42 = a42 * a42, q43 = a43 * a43;
    const float P = ((((((1.f - cterm(k, 0, q21)) - cterm(k, 1, q31)) - cterm(k, 2, q32)) -
                      cterm(k, 3, q41)) - cterm(k, 4, q42)) - cterm(k, 5, q43));
    const float d21 = 2.f * a21 * b21 * dx, d31 = 2.f * a31 * b31 * dx, d32 = 2.f * a32 * b32 * dx;
    const float d41 = 2.f * a41 * b41 * dx, d42 = 2.f * a42 * b42 * dx, d43 = 2.f * a43 * b43 * dx;
    const float A = c13 * c13 * S12 * q21 + S13 * (c12 * q31 + s12 * q32);
    const float Bs = c13 * (c12 * q41 + s12 * q42) + s13 * q43;
    const float dC4 = -c14 * 0.5f / root;
    dP[0] = -C4 * (c13 * c13 * 4.f * (1.f - 2.f * s12) * q21 + S13 * (q32 - q31)) - S14 * c13 * (q42 - q41);
    dP[1] = -C4 * (-2.f * c13 * S12 * q21 + 4.f * (1.f - 2.f * s13) * (c12 * q31 + s12 * q32)) -
            S14 * (q43 - (c12 * q41 + s12 * q42));
    dP[2] = -C4 * (c13 * c13 * S12 * d21 - S13 * s12 * d32) + S14 * c13 * s12 * d42;
    dP[3] = -C4 * S13 * (c12 * d31 + s12 * d32) + S14 * s13 * d43;
    dP[4] = -dC4 * A - Bs;
    dP[5] = -S14 * (c13 * (c12 * d41 + s12 * d42) + s13 * d43);
    return P;
}

// The six coefficients of survival_sterile from float pairs e of the exact parameter values.
__device__ __forceinline__ OscCoefN<6> osc_coef_sterile(const F2 (&e)[6]) {
    const F2 one{1.f, 0.f};
    const F2 c12 = f2_one_minus(e[0]), c13 = f2_one_minus(e[1]);
    const F2 S12 = f2_scale(f2_mul(e[0], c12), 4.f), S13 = f2_scale(f2_mul(e[1], c13), 4.f);
    const F2 c14 = f2_scale(f2_add(one, f2_sqrt(f2_one_minus(e[4]))), 0.5f);   // cos^2 th14
    const F2 C4 = f2_mul(c14, c14);
    F2 cf[6];
    cf[0] = f2_mul(C4, f2_mul(f2_mul(c13, c13), S12));
    cf[1] = f2_mul(C4, f2_mul(S13, c12));
    cf[2] = f2_mul(C4, f2_mul(S13, e[0]));
    cf[3] = f2_mul(e[4], f2_mul(c13, c12));
    cf[4] = f2_mul(e[4], f2_mul(c13, e[0]));
    cf[5] = f2_mul(e[4], e[1]);
    OscCoefN<6> k;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        k.hi[i] = cf[i].h;
        k.lo[i] = cf[i].l;
    }
    return k;
}

// whether survival parameter i of a formula is a mass splitting (carried as a float pair)
__host__ __device__ __forceinline__ bool osc_is_dm(int mode, int i) {
    return mode == FIT_OSC_EQ1 ? (i == 1 || i == 3) : (i == 2 || i == 3 || i == 5);
}

// Survival of the formula with NOSC parameters: 4 (Eq. 1 or the three-flavour formula) or 6
// (the 3+1 formula).
template <int NOSC>
struct OscTraits;
template <>
struct OscTraits<4> {
    using Coef = OscCoefN<3>;
    static __device__ __forceinline__ float survival(int mode, const float (&eta)[4], const float (&eta_lo)[4],
                                                     const Coef &k, float c_hi, float c_lo, float (&dP)[4]) {
        return survival_mode(mode, eta, eta_lo, k, c_hi, c_lo, dP);
    }
    static __device__ __forceinline__ Coef coef(int mode, const F2 (&e)[4]) { return osc_coef(mode, e); }
};
template <>
struct OscTraits<6> {
    using Coef = OscCoefN<6>;
    static __device__ __forceinline__ float survival(int, const float (&eta)[6], const float (&eta_lo)[6],
                                                     const Coef &k, float c_hi, float c_lo, float (&dP)[6]) {
        return survival_sterile(eta, eta_lo, k, c_hi, c_lo, dP);
    }
    static __device__ __forceinline__ Coef coef(int, const F2 (&e)[6]) { return osc_coef_sterile(e); }
};

// Poisson deviance 2[mu - n + n ln(n/mu)] = 2 mu h(r), r = (n - mu)/mu,
// h(r) = (1+r) ln(1+r) - r, by its alternating series for |r| < 1/4.
__device__ __forceinline__ float deviance(float n, float mu) {
    if (n == 0.f) return 2.f * mu;
    const float r = (n - mu) / mu;
    float h;
    if (fabsf(r) < 0.25f) {
        // h = sum_{j>=2} (-1)^j r^j / (j (j-1))
        float acc = 0.f;
#pragma unroll
        for (int j = 14; j >= 2; --j) {
            const float cj = ((j & 1) ? -1.f : 1.f) / (float)(j * (j - 1));
            acc = fmaf(acc, r, cj);
        }
        h = acc * r * r;
    } else {
        h = (1.f + r) * log1pf(r) - r;
    }
    return 2.f * mu * h;
}

// ------------------------------------------------------------------------------------
// Per-dataset workspace (floats), all of length N_t unless noted:
//   u, v(->gv), ts = t s, ptot, dp0..dp3 (dp0 is reused for the shape gradient),
//   pcw[C] = w_c P_c per core, f0[max_reco], gmu[max_reco]
// ------------------------------------------------------------------------------------
struct EvalWs {
    float *u, *v, *ts, *ptot, *dp, *pcw, *f0, *gmu;
};

__host__ __device__ inline int eval_ws_floats(int N_t, int C, int max_reco, int n_osc) {
    return (4 + n_osc + C) * N_t + 2 * max_reco;
}

__device__ __forceinline__ EvalWs carve_eval_ws(float *base, int N_t, int C, int max_reco, int n_osc) {
    EvalWs w;
    w.u = base;
    w.v = w.u + N_t;
    w.ts = w.v + N_t;
    w.ptot = w.ts + N_t;
    w.dp = w.ptot + N_t;          // n_osc * N_t
    w.pcw = w.dp + n_osc * N_t;   // C * N_t
    w.f0 = w.pcw + C * N_t;       // max_reco
    w.gmu = w.f0 + max_reco;      // max_reco
    return w;
}

// Parameter access: pv = value, pd = value - theta0 (kept separately for precision).
__device__ __forceinline__ float pval(const float *pv, int idx, float dflt) {
    return idx >= 0 ? pv[idx] : dflt;
}

// A parameter as the float pair h + l: h = its float value, l = the exact rounding residual
// (theta0_f - h) + delta + theta0_lo. Products x * theta are then formed as fma(x, l, x h),
// so the kernels evaluate at the caller's double-precision point, not at its float rounding
// (high-statistics normalisations have enough curvature for that rounding to show).
struct PP {
    float h, l;
};

__device__ __forceinline__ PP ppair(const DevModel &m, const float *pv, const float *pd, int p,
                                    float dflt) {
    if (p < 0) return PP{dflt, 0.f};
    const float h = pv[p];
    return PP{h, ((m.theta0_f[p] - h) + pd[p]) + m.theta0_lo[p]};
}

__device__ __forceinline__ float pmul(PP a, float x) { return fmaf(x, a.l, x * a.h); }

// Status bits raised during an evaluation
constexpr int kStMuNonpos = 1;
constexpr int kStEscale = 2;

// Energy map of dataset d in grid units: displacement D(e) = (a0 + (a1-1) e + a2 e^2) / de.
struct EMap {
    float a0, a1m1, a2, inv_de, e_lo, de;
    __device__ __forceinline__ float disp(float e) const {
        return fmaf(fmaf(a2, e, a1m1), e, a0) * inv_de;
    }
    __device__ __forceinline__ float slope(float e) const { return 1.f + a1m1 + 2.f * a2 * e; }
};

// ---- area-conserving spline remap --------------------------------------------------------
// The grid's cumulative content C(e_k) is interpolated on each bin by the cubic Hermite
// polynomial with end slopes de f(e_k) = S_k = (u_{k-1} + u_k) / 2 (u_0, u_{N-1} at the ends):
//   F(e_k + t de) = C(e_k) + G_k(t),  G_k(t) = u_k h01(t) + S_k h10(t) + S_{k+1} h11(t),
// which keeps every bin's content and has a continuous density. The corrected spectrum is
// v_j = F(x_{j+1}) - F(x_j), x_j = E'^{-1}(e_j), evaluated locally as
//   v_j = sum_{k0 <= k < k1} u_k + G_{k1}(t1) - G_{k0}(t0)
// with each x on the grid as e + r (exact integer edge index + small FP32 offset r).
__device__ __forceinline__ float hermite_S(const float *u, int k, int N) {
    return k <= 0 ? u[0] : (k >= N ? u[N - 1] : 0.5f * (u[k - 1] + u[k]));
}

__device__ __forceinline__ float hermite_G(const float *u, int k, float t, int N) {
    const float t2 = t * t, t3 = t2 * t;
    const float h01 = fmaf(-2.f, t3, 3.f * t2), h10 = t3 - 2.f * t2 + t, h11 = t3 - t2;
    return fmaf(u[k], h01, fmaf(hermite_S(u, k, N), h10, hermite_S(u, k + 1, N) * h11));
}

// r with E'(e_e + r de) = e_e (two Newton steps from -D(e_e); |r| is a few bins at most)
template <class Map>
__device__ __forceinline__ float edge_inv_r(const float *e_edge, const Map &em, int e) {
    const float xe = e_edge[e];
    float r = -em.disp(xe);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float x = fmaf(r, em.de, xe);
        r -= (r + em.disp(x)) / em.slope(x);
    }
    return r;
}

// bin k and fraction t of the grid position e + r, clamped to the grid: below it (0, 0)
// (F = 0), above it (N - 1, 1) (F = total); `inside` tells whether it was on the grid
__device__ __forceinline__ void edge_bin(int e, float r, int N, int &k, float &t, bool &inside) {
    const float fl = floorf(r);
    k = e + (int)fl;
    t = r - fl;
    inside = true;
    if (k < 0) {
        k = 0;
        t = 0.f;
        inside = false;
    } else if (k >= N) {
        k = N - 1;
        t = 1.f;
        inside = false;
    }
}

// v_j for target bin j
template <class Map>
__device__ __forceinline__ float spline_target(const float *u, const float *e_edge, const Map &em, int j, int N) {
    int k0, k1;
    float t0, t1;
    bool in0, in1;
    edge_bin(j, edge_inv_r(e_edge, em, j), N, k0, t0, in0);
    edge_bin(j + 1, edge_inv_r(e_edge, em, j + 1), N, k1, t1, in1);
    float acc = 0.f;
    for (int k = k0, it = 0; k < k1 && it < 64; ++k, ++it) acc += u[k];
    return acc + (hermite_G(u, k1, t1, N) - hermite_G(u, k0, t0, N));
}

// Adjoint of the spline remap for source bin i: d(-2lnL)/du_i. With w_e = gv_{e-1} - gv_e the
// weight of F(x_e) (gv outside the grid 0), dF(x_e)/du_i is 1 for i < k_e (the cumulative)
// plus the Hermite weights of u_i in G_{k_e}; the cumulative part sums to gv_{e*-1}, e* the
// first edge with k_e > i.
template <class Map>
__device__ __forceinline__ float spline_adjoint_source(const float *gv, const float *e_edge, const Map &em,
                                                       int i, int N) {
    auto kb = [&](int e, int &k, float &t) {
        bool in;
        edge_bin(e, edge_inv_r(e_edge, em, e), N, k, t, in);
    };
    // e*: start from the inverse shift at edge i and walk to the first edge with k_e > i
    int e = min(max(i + 1 - (int)floorf(edge_inv_r(e_edge, em, i)), 0), N + 1);
    int k;
    float t;
    for (int it = 0; it < 64 && e > 0; ++it) {   // step down while the edge before is past i
        kb(e - 1, k, t);
        if (k <= i) break;
        --e;
    }
    for (int it = 0; it < 64 && e <= N; ++it) {  // step up while this edge is not past i
        kb(e, k, t);
        if (k > i) break;
        ++e;
    }
    float g = (e >= 1 && e <= N) ? gv[e - 1] : 0.f;
    // local Hermite weights: edges with k_e in [i - 1, i + 1] lie around e*
    auto local = [&](int ee) -> bool {
        int kk;
        float tt;
        kb(ee, kk, tt);
        if (kk < i - 1 || kk > i + 1) return false;
        const float we = (ee >= 1 ? gv[ee - 1] : 0.f) - (ee <= N - 1 ? gv[ee] : 0.f);
        const float t2 = tt * tt, t3 = t2 * tt;
        const float h01 = fmaf(-2.f, t3, 3.f * t2), h10 = t3 - 2.f * t2 + tt, h11 = t3 - t2;
        float c = 0.f;
        if (kk == i) c = h01 + (kk == 0 ? h10 : 0.5f * h10) + (kk == N - 1 ? h11 : 0.5f * h11);
        else if (kk == i + 1) c = 0.5f * h10;   // S_{i+1} = (u_i + u_{i+1}) / 2
        else c = 0.5f * h11;                    // kk == i - 1: S_i = (u_{i-1} + u_i) / 2
        g = fmaf(we, c, g);
        return true;
    };
    for (int ee = e - 1, it = 0; ee >= 0 && it < 64; --ee, ++it)
        if (!local(ee)) break;
    for (int ee = e, it = 0; ee <= N && it < 64; ++ee, ++it)
        if (!local(ee)) break;
    return g;
}

// Edge e's share of d(-2lnL)/d(a0, a1, a2): w_e f(x_e) dx_e/da_i, dx/da_i = -x^i / E''(x)
// (f the spline's density per MeV, 0 off the grid); added to ep[0..2].
template <class Map>
__device__ __forceinline__ void spline_adjoint_edge(const float *u, const float *gv, const float *e_edge,
                                                    const Map &em, int e, int N, float *ep) {
    const float r = edge_inv_r(e_edge, em, e);
    int k;
    float t;
    bool in;
    edge_bin(e, r, N, k, t, in);
    if (!in) return;
    const float we = (e >= 1 ? gv[e - 1] : 0.f) - (e <= N - 1 ? gv[e] : 0.f);
    const float t2 = t * t;
    const float dG = fmaf(u[k], 6.f * (t - t2), fmaf(hermite_S(u, k, N), 3.f * t2 - 4.f * t + 1.f,
                                                      hermite_S(u, k + 1, N) * (3.f * t2 - 2.f * t)));
    const float x = fmaf(r, em.de, e_edge[e]);
    const float q = -we * dG * em.inv_de / em.slope(x);
    ep[0] += q;
    ep[1] = fmaf(q, x, ep[1]);
    ep[2] = fmaf(q, x * x, ep[2]);
}

__device__ __forceinline__ EMap make_emap(const DevModel &m, const DevDataset &ds, const float *pv,
                                          const float *pd) {
    EMap em;
    em.a0 = ds.esc_idx[0] >= 0 ? pv[ds.esc_idx[0]] : 0.f;
    em.a1m1 = ds.esc_idx[1] >= 0 ? ds.a1_off + pd[ds.esc_idx[1]] : 0.f;
    em.a2 = ds.esc_idx[2] >= 0 ? pv[ds.esc_idx[2]] : 0.f;
    em.inv_de = m.inv_de;
    em.e_lo = m.e_lo;
    em.de = m.de;
    return em;
}

// ------------------------------------------------------------------------------------
// Block-level evaluation of one dataset, in stages that the fit kernels call either in one
// sequence (eval_dataset) or split over two launches (forward + likelihood, then adjoint).
// ------------------------------------------------------------------------------------
// Per-dataset constants of one evaluation: survival parameters and coefficients,
// normalisation, efficiency, energy map.
template <int NOSC>
struct DsCtxT {
    typename OscTraits<NOSC>::Coef kc;
    float eta[NOSC], eta_lo[NOSC];
    PP nrm, eff;
    EMap em;
};
using DsCtx = DsCtxT<4>;

// Fills c; false (and status |= kStEscale) when the energy map is not increasing with slope in
// (1/4, 4) on the grid. Contains a barrier.
template <int NOSC>
static __device__ bool ds_setup(const DevModel &m, int d, const float *pv, const float *pd, DsCtxT<NOSC> &c,
                                int *status) {
    const DevDataset &ds = m.ds[d];
    const int N_t = m.N_t;
    const int tid = threadIdx.x;
    // Survival parameters: mass splittings as theta0_f + (theta0_lo + delta) inside the
    // phase.
    float *eta = c.eta, *eta_lo = c.eta_lo;
#pragma unroll
    for (int i = 0; i < NOSC; ++i) {
        const int p = m.osc_idx[i];
        if (osc_is_dm(m.osc_mode, i)) {
            eta[i] = p >= 0 ? m.theta0_f[p] : m.osc_val[i];
            eta_lo[i] = p >= 0 ? m.theta0_lo[p] + pd[p] : m.osc_val_lo[i];
        } else {
            eta[i] = p >= 0 ? pv[p] : m.osc_val[i];
            eta_lo[i] = 0.f;
        }
    }
    // the sin^2 coefficients from float pairs of the exact parameter values (every thread
    // forms the same values; no barrier)
    F2 e[NOSC];
#pragma unroll
    for (int i = 0; i < NOSC; ++i) {
        const int p = m.osc_idx[i];
        if (p >= 0) {
            const float h = pv[p];
            e[i] = f2_norm(h, ((m.theta0_f[p] - h) + pd[p]) + m.theta0_lo[p]);
        } else {
            e[i] = F2{m.osc_val[i], m.osc_val_lo[i]};
        }
    }
    c.kc = OscTraits<NOSC>::coef(m.osc_mode, e);
    c.nrm = ppair(m, pv, pd, ds.norm_idx, 1.f);
    c.eff = ppair(m, pv, pd, ds.eff_idx, 1.f);
    c.em = make_emap(m, ds, pv, pd);
    const EMap &em = c.em;

    // the map must be increasing with slope in (1/4, 4) everywhere on the grid
    {
        const float s0 = em.slope(m.e_edge[0]), s1 = em.slope(m.e_edge[N_t]);
        if (!(s0 > 0.25f && s0 < 4.f && s1 > 0.25f && s1 < 4.f)) {
            if (tid == 0) atomicOr(status, kStEscale);
            return false;
        }
    }

    return true;
}

// Stage A: u_k (and with DERIV the per-bin partials the adjoint needs). Ends with a barrier.
template <bool DERIV, int NOSC>
static __device__ void ds_signal(const DevModel &m, int d, const float *pv, const float *pd,
                                 const DsCtxT<NOSC> &c, EvalWs ws) {
    const DevDataset &ds = m.ds[d];
    const int N_t = m.N_t, C = m.C;
    const int tid = threadIdx.x, nth = blockDim.x;
    // ---- stage A: signal on the true grid (Eq. 1/2 x shares x reweights) -----------------
    for (int k = tid; k < N_t; k += nth) {
        const float ih = m.inv_e_hi[k], il = m.inv_e_lo[k];
        float pt = 0.f, dpt[NOSC];
#pragma unroll
        for (int i = 0; i < NOSC; ++i) dpt[i] = 0.f;
        for (int cc = 0; cc < C; ++cc) {
            const float w = ds.w[cc];
            if (w == 0.f) {
                if (DERIV) ws.pcw[cc * N_t + k] = 0.f;
                continue;
            }
            const float ch = ds.kl_hi[cc] * ih;
            const float cl = fmaf(ds.kl_hi[cc], ih, -ch) + ds.kl_hi[cc] * il + ds.kl_lo[cc] * ih;
            float dP[NOSC];
            const float P = OscTraits<NOSC>::survival(m.osc_mode, c.eta, c.eta_lo, c.kc, ch, cl, dP);
            const PP pw = ppair(m, pv, pd, m.core_power_idx[cc], 1.f);
            const float wP = w * P;
            if (DERIV) ws.pcw[cc * N_t + k] = wP;
            pt += pmul(pw, wP);
#pragma unroll
            for (int i = 0; i < NOSC; ++i) if (DERIV) dpt[i] = fmaf(pw.h * w, dP[i], dpt[i]);
        }
        const float ts = pmul(ppair(m, pv, pd, ds.shape_idx[k], 1.f), ds.t[k]);
        if (DERIV) {
            ws.ts[k] = ts;
            ws.ptot[k] = pt;
        }
#pragma unroll
        for (int i = 0; i < NOSC; ++i)
            if (DERIV) ws.dp[i * N_t + k] = dpt[i];
        ws.u[k] = pmul(c.nrm, ts * pt);
    }
    __syncthreads();

}

// Stage B: v = M(a) u. Ends with a barrier.
// SPL: compiled with the area-conserving spline option (the general kernel builds)
template <bool SPL, class Ctx>
static __device__ void ds_remap(const DevModel &m, int d, const Ctx &c, EvalWs ws) {
    (void)d;   // the energy map is in c
    const int N_t = m.N_t;
    const int tid = threadIdx.x, nth = blockDim.x;
    const EMap &em = c.em;
    if (SPL && m.remap_mode == FIT_REMAP_SPLINE) {
        for (int t = tid; t < N_t; t += nth) ws.v[t] = spline_target(ws.u, m.e_edge, em, t, N_t);
        __syncthreads();
        return;
    }
    // ---- stage B: energy correction, gather per target bin ------------------------------
    // Source bin k covers [Y_k, Y_k+1] in grid units, Y_k = k + D(e_k). Target m gathers the
    // sources whose mapped interval overlaps [m, m+1]; overlaps are computed relative to the
    // target (k - m is an exact small integer), which keeps them accurate in FP32.
    for (int t = tid; t < N_t; t += nth) {
        // first source whose mapped upper edge lies above t: start from the fixed point
        // k ~ t - D(k) and step until the bracket is right
        int k = t - (int)floorf(em.disp(m.e_edge[t]));
        k = min(max(k, 0), N_t - 1);
        k = t - (int)floorf(em.disp(m.e_edge[k]));
        k = min(max(k - 1, 0), N_t - 1);
        while (k > 0 && (float)(k - t) + em.disp(m.e_edge[k]) > 0.f) --k;
        float acc = 0.f;
        float dlo = em.disp(m.e_edge[k]);
        for (int it = 0; it < 64 && k < N_t; ++it, ++k) {
            const float dhi = em.disp(m.e_edge[k + 1]);
            const float ylo = (float)(k - t) + dlo;      // mapped edges relative to target t
            const float yhi = (float)(k + 1 - t) + dhi;
            if (ylo >= 1.f) break;
            const float ov = fminf(yhi, 1.f) - fmaxf(ylo, 0.f);
            if (ov > 0.f) acc = fmaf(ws.u[k], ov / (1.f + (dhi - dlo)), acc);
            dlo = dhi;
        }
        ws.v[t] = acc;
    }
    __syncthreads();

}

// Stage C: fold into reco bins, ws.f0 = R v (before the efficiency). Ends with a barrier.
static __device__ void ds_fold(const DevModel &m, int d, EvalWs ws) {
    const DevDataset &ds = m.ds[d];
    const DevDetector &dt = m.det[ds.det];
    const int nr = ds.n_reco;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
    // ---- stage C: fold into reco bins (banded rows, warp per row) ------------------------
    // Each warp takes four rows at a time and two strides of each, so eight independent
    // load/FMA chains per lane are in flight.
    for (int j0 = warp; j0 < nr; j0 += 4 * nw) {
        int lo[4], len[4];
        const float *rr[4];
        int lmax = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * nw;
            const bool on = j < nr;
            lo[u] = on ? dt.row_lo[j] : 0;
            len[u] = on ? dt.row_len[j] : 0;
            rr[u] = dt.rrow + (on ? dt.row_off[j] : 0);
            lmax = max(lmax, len[u]);
        }
        float s[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        for (int b = lane; b < lmax; b += 64) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (b < len[u]) s[u][0] = fmaf(rr[u][b], ws.v[lo[u] + b], s[u][0]);
                if (b + 32 < len[u]) s[u][1] = fmaf(rr[u][b + 32], ws.v[lo[u] + b + 32], s[u][1]);
            }
        }
        float t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = s[u][0] + s[u][1];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int u = 0; u < 4; ++u) t[u] += __shfl_xor_sync(0xffffffffu, t[u], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + u * nw < nr) ws.f0[j0 + u * nw] = t[u];
        }
    }
    __syncthreads();
}

// Stage C2: backgrounds, deviance, dD/dmu (ws.gmu) and the background-shape gradient from the
// folded spectrum ws.f0; returns the dataset's -2lnL (all threads). The efficiency and rate
// gradients are added when grad != nullptr, data != nullptr and no status bit is set.
template <class Ctx>
static __device__ double ds_lik(const DevModel &m, int d, const float *pv, const float *pd, const Ctx &c,
                                const float *data, EvalWs ws, float *grad, double *red, int *status,
                                float *mu_out) {
    const DevDataset &ds = m.ds[d];
    const int nr = ds.n_reco;
    const int tid = threadIdx.x, nth = blockDim.x;
    // ---- stage C2: backgrounds, deviance, dD/dmu ----------------------------------------
    const int nb = ds.bkg_end - ds.bkg_begin;
    float part[2 + kMaxBkgDs];
    // part[0] = deviance, part[1] = d/d eff, part[2+b] = d/d rate_b
#pragma unroll
    for (int i = 0; i < 2 + kMaxBkgDs; ++i) part[i] = 0.f;
    for (int j = tid; j < nr; j += nth) {
        float mu = pmul(c.eff, ws.f0[j]);
#pragma unroll
        for (int b = 0; b < kMaxBkgDs; ++b) {
            if (b >= nb) break;
            const DevBkg &bk = m.bkg[ds.bkg_begin + b];
            const float tm = bk.tmpl[j];
            const float shaped = bk.shape_idx[j] >= 0 ? fmaf(tm, pv[bk.shape_idx[j]], tm) : tm;
            mu += pmul(ppair(m, pv, pd, bk.rate_idx, 1.f), shaped);
        }
        if (mu_out) mu_out[j] = mu;
        if (data == nullptr) continue;
        const float n = data[ds.data_off + j];
        if (!(mu > 0.f)) {
            atomicOr(status, kStMuNonpos);
            continue;
        }
        part[0] += deviance(n, mu);
        const float g = 2.f * (mu - n) / mu;
        ws.gmu[j] = g;
        if (grad) {
            part[1] = fmaf(g, ws.f0[j], part[1]);
#pragma unroll
            for (int b = 0; b < kMaxBkgDs; ++b) {
                if (b >= nb) break;
                const DevBkg &bk = m.bkg[ds.bkg_begin + b];
                const int si = bk.shape_idx[j];
                const float sh = 1.f + (si >= 0 ? pv[si] : 0.f);
                part[2 + b] = fmaf(g * bk.tmpl[j], sh, part[2 + b]);
                if (si >= 0) atomicAdd(&grad[si], g * pval(pv, bk.rate_idx, 1.f) * bk.tmpl[j]);
            }
        }
    }
    double tot[2 + kMaxBkgDs];
    block_sum<2 + kMaxBkgDs>(part, red, tot);
    const double nll_d = tot[0];
    if (data == nullptr || grad == nullptr || (*(volatile int *)status) != 0) return nll_d;
    if (tid == 0) {
        if (ds.eff_idx >= 0) grad[ds.eff_idx] += (float)tot[1];
#pragma unroll
        for (int b = 0; b < kMaxBkgDs; ++b) {
            if (b >= nb) break;
            const int ri = m.bkg[ds.bkg_begin + b].rate_idx;
            if (ri >= 0) grad[ri] += (float)tot[2 + b];
        }
    }

    return nll_d;
}

// Stages C and C2 in one sequence.
template <class Ctx>
static __device__ double ds_fold_lik(const DevModel &m, int d, const float *pv, const float *pd, const Ctx &c,
                                     const float *data, EvalWs ws, float *grad, double *red, int *status,
                                     float *mu_out) {
    ds_fold(m, d, ws);
    return ds_lik(m, d, pv, pd, c, data, ws, grad, red, status, mu_out);
}

// Stage D: adjoint of the fold, ws.v <- gv = eff R^T gmu (column bands). Ends with a barrier.
template <int NOSC>
static __device__ void ds_adjoint_fold(const DevModel &m, int d, const DsCtxT<NOSC> &c, EvalWs ws) {
    const DevDataset &ds = m.ds[d];
    const DevDetector &dt = m.det[ds.det];
    const int N_t = m.N_t, nr = ds.n_reco;
    const int tid = threadIdx.x, nth = blockDim.x;
    // ---- stage D: adjoint of the fold, gv = eff R^T gmu (column bands) --------------------
    float *gv = ws.v;   // v is dead after the fold
    // rcol is exactly 0 past each column's band, so the loop runs the widest band of the
    // warp's 32 adjacent columns (nearly their own widths: the resolution changes slowly with
    // energy) with the row index clamped (no early exit) and four partial sums
    for (int k = tid; k < N_t; k += nth) {
        const int lo = dt.col_lo[k], jmax = nr - 1;
        const int cw = __reduce_max_sync(__activemask(), dt.col_len[k]);
        const float *rc = dt.rcol + k;
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        int b = 0;
        for (; b + 7 < cw; b += 8) {   // eight loads in flight
#pragma unroll
            for (int q = 0; q < 8; ++q)
                s[q & 3] = fmaf(rc[(int64_t)(b + q) * N_t], ws.gmu[min(lo + b + q, jmax)], s[q & 3]);
        }
        for (; b < cw; ++b) s[0] = fmaf(rc[(int64_t)b * N_t], ws.gmu[min(lo + b, jmax)], s[0]);
        gv[k] = pmul(c.eff, (s[0] + s[1]) + (s[2] + s[3]));
    }
    __syncthreads();
}

// Stages E and F: adjoint of the energy map and of the signal from gv (in ws.v); adds the
// gradient contributions to grad. Needs ws.u/ts/ptot/dp/pcw (ds_signal<true>).
template <int NC, int NOSC, bool SPL>
static __device__ void ds_adjoint_ef(const DevModel &m, int d, const float *pv, const float *pd,
                                     const DsCtxT<NOSC> &c, EvalWs ws, float *grad, double *red) {
    const DevDataset &ds = m.ds[d];
    const int N_t = m.N_t, C = m.C;
    const int tid = threadIdx.x, nth = blockDim.x;
    const EMap &em = c.em;
    const float *gv = ws.v;
    (void)pv;
    (void)pd;
    // ---- stage E: adjoint of the energy map and of the signal ---------------------------
    // per source k: gu = sum_t F_kt gv_t; A0 = (gu - gv(floor Y_k)) / w, A1 = (gv(floor Y_k+1) - gu) / w
    constexpr int kN = 3 + NOSC, kP = 4 + NOSC;   // index of d/d norm, first d/d power
    float ep[kP + NC];
    // ep[0..2] d/da, ep[3..3+NOSC) d/d eta, ep[kN] d/d norm, ep[kP+c] d/d power_c (NC >= C)
#pragma unroll
    for (int i = 0; i < kP + NC; ++i) ep[i] = 0.f;
    const bool spline = SPL && m.remap_mode == FIT_REMAP_SPLINE;
    for (int k = tid; k < N_t; k += nth) {
        float gu = 0.f;
        if (spline) {
            gu = spline_adjoint_source(gv, m.e_edge, em, k, N_t);
            spline_adjoint_edge(ws.u, gv, m.e_edge, em, k, N_t, ep);
            if (k == N_t - 1) spline_adjoint_edge(ws.u, gv, m.e_edge, em, N_t, N_t, ep);
        } else {
        const float e0 = m.e_edge[k], e1 = m.e_edge[k + 1];
        const float d0 = em.disp(e0), d1 = em.disp(e1);
        const float w = 1.f + (d1 - d0), iw = 1.f / w;
        const int f0i = (int)floorf(d0), f1i = (int)floorf(d1);
        const int t0 = k + f0i, t1 = k + 1 + f1i;
        for (int t = max(t0, 0); t <= min(t1, N_t - 1); ++t) {
            const float ylo = (float)(k - t) + d0, yhi = (float)(k + 1 - t) + d1;
            const float ov = fminf(yhi, 1.f) - fmaxf(ylo, 0.f);
            if (ov > 0.f) gu = fmaf(ov * iw, gv[t], gu);
        }
        const float g0 = (t0 >= 0 && t0 < N_t) ? gv[t0] : 0.f;
        const float g1 = (t1 >= 0 && t1 < N_t) ? gv[t1] : 0.f;
        const float uk = ws.u[k] * iw;
        const float A0 = uk * (gu - g0), A1 = uk * (g1 - gu);
        ep[0] += (A0 + A1) * em.inv_de;
        ep[1] += (A0 * e0 + A1 * e1) * em.inv_de;
        ep[2] += (A0 * e0 * e0 + A1 * e1 * e1) * em.inv_de;
        }
        const float ts = ws.ts[k], pt = ws.ptot[k];
        const float gb = pmul(c.nrm, gu * ts);    // d nll / d(ptot)
#pragma unroll
        for (int i = 0; i < NOSC; ++i) ep[3 + i] = fmaf(gb, ws.dp[i * N_t + k], ep[3 + i]);
        ep[kN] = fmaf(gu * ts, pt, ep[kN]);
#pragma unroll
        for (int cc = 0; cc < NC; ++cc)
            if (cc < C) ep[kP + cc] = fmaf(gb, ws.pcw[cc * N_t + k], ep[kP + cc]);
        ws.dp[k] = pmul(c.nrm, gu * ds.t[k] * pt);    // d nll / d s for this bin (dp0 reused)
    }
    double etot[kP + NC];
    block_sum<kP + NC>(ep, red, etot);
    if (tid == 0) {
        for (int i = 0; i < 3; ++i)
            if (ds.esc_idx[i] >= 0) grad[ds.esc_idx[i]] += (float)etot[i];
        for (int i = 0; i < NOSC; ++i)
            if (m.osc_idx[i] >= 0) grad[m.osc_idx[i]] += (float)etot[3 + i];
        if (ds.norm_idx >= 0) grad[ds.norm_idx] += (float)etot[kN];
#pragma unroll
        for (int cc = 0; cc < NC; ++cc)
            if (cc < C && m.core_power_idx[cc] >= 0) grad[m.core_power_idx[cc]] += (float)etot[kP + cc];
    }
    // ---- stage F: shape reweights (one thread per distinct parameter, CSR over bins) -----
    for (int i = tid; i < ds.n_sp; i += nth) {
        float s = 0.f;
        for (int q = ds.sp_ptr[i]; q < ds.sp_ptr[i + 1]; ++q) s += ws.dp[ds.sp_k[q]];
        grad[ds.sp_param[i]] += s;
    }
    __syncthreads();
}

// Stages E-F with the per-core sums sized for the model's core count.
template <bool SPL, int NOSC>
static __device__ void ds_adjoint_rest(const DevModel &m, int d, const float *pv, const float *pd,
                                       const DsCtxT<NOSC> &c, EvalWs ws, float *grad, double *red) {
    if (m.C <= 2)
        ds_adjoint_ef<2, NOSC, SPL>(m, d, pv, pd, c, ws, grad, red);
    else
        ds_adjoint_ef<FIT_MAX_CORES, NOSC, SPL>(m, d, pv, pd, c, ws, grad, red);
}

// Stages D-F: adjoint of the fold, of the energy map and of the signal; adds the gradient
// contributions to grad. Needs ws.u/ts/ptot/dp/pcw (ds_signal<true>) and ws.gmu.
template <bool SPL, int NOSC>
static __device__ void ds_adjoint(const DevModel &m, int d, const float *pv, const float *pd,
                                  const DsCtxT<NOSC> &c, EvalWs ws, float *grad, double *red) {
    ds_adjoint_fold(m, d, c, ws);
    ds_adjoint_rest<SPL>(m, d, pv, pd, c, ws, grad, red);
}

// One dataset in one sequence: adds its Poisson -2lnL and (if grad != nullptr) its gradient
// contributions (theta space, P floats). Returns the dataset's -2lnL (all threads); *status |=
// kSt* bits on failure.

template <int NOSC, bool SPL>
static __device__ double eval_dataset_n(const DevModel &m, int d, const float *pv, const float *pd,
                                        const float *data, EvalWs ws, float *grad, double *red,
                                        int *status, float *mu_out) {
    DsCtxT<NOSC> c;
    if (!ds_setup(m, d, pv, pd, c, status)) return 0.0;
    if (grad != nullptr && data != nullptr)
        ds_signal<true>(m, d, pv, pd, c, ws);
    else
        ds_signal<false>(m, d, pv, pd, c, ws);
    ds_remap<SPL>(m, d, c, ws);
    const double nll_d = ds_fold_lik(m, d, pv, pd, c, data, ws, grad, red, status, mu_out);
    if (data == nullptr || grad == nullptr || (*(volatile int *)status) != 0) return nll_d;
    ds_adjoint<SPL>(m, d, pv, pd, c, ws, grad, red);
    return nll_d;
}

// One dataset's -2lnL (and gradient). NOSC = 4 (the basic build): models of Eq. 1 or the
// three-flavour formula with the overlap-length energy correction; NOSC = 6 (the general
// build): any model (the 3+1 formula, the spline energy correction).
template <int NOSC = 4>
static __device__ double eval_dataset(const DevModel &m, int d, const float *pv, const float *pd,
                                      const float *data, EvalWs ws, float *grad, double *red,
                                      int *status, float *mu_out) {
    if constexpr (NOSC == 6) {
        if (m.osc_mode == FIT_OSC_STERILE4)
            return eval_dataset_n<6, true>(m, d, pv, pd, data, ws, grad, red, status, mu_out);
        return eval_dataset_n<4, true>(m, d, pv, pd, data, ws, grad, red, status, mu_out);
    }
    return eval_dataset_n<4, false>(m, d, pv, pd, data, ws, grad, red, status, mu_out);
}

}  // namespace fitcore
