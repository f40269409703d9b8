/*
 * FP64 CPU oracle for the forward-folding profile-likelihood fit (PhyLiNO, arXiv 2502.15253).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference that the CUDA library is
 * checked against. Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it; the library never calls it and shares no code with it.
 *
 * Citations: [S] = section "Structure of the framework" of the paper, [L] = section
 * "Likelihood implementation for Double Chooz within the framework".
 *
 * What it computes (all in double precision, written loop by loop):
 *
 *   per dataset d, true bin k (centre E_k), core c with baseline L_dc:
 *     Ptot_dk = sum_c p_c w_dc P(L_dc, E_k; eta)                 survival, Eq. 1 / Eq. 2
 *                                                                 (or exact 3-flavour vacuum,
 *                                                                  the quantity Eq. 10 expands)
 *     u_dk    = t_dk * n_d * s_(g(k)) * Ptot_dk                   flux x xsec x reweights [S]
 *     v_d     = M(a_d) u_d   energy correction E' = a0 + a1 E + a2 E^2, each true bin's content
 *                            spread over the original binning by overlap length [S]
 *     f_dj    = eps_d sum_k R_d[j,k] v_dk                         fold into reco bins [S]
 *     mu_dj   = f_dj + sum_b r_b B_bj (1 + delta_bj)              backgrounds [L], Eq. 9
 *   -2lnL     = sum_d sum_j 2 [mu - n + n ln(n/mu)]               Poisson, Eq. 3-5, normalised
 *                                                                 to the saturated model, Eq. 8
 *             + sum_i ((theta_i - theta0_i)/sigma_i)^2            Gaussian priors, Eq. 6
 *             + sum_B (theta_B - theta0_B)^T V_B^-1 (theta_B - theta0_B)   Eq. 6 / Eq. 9
 *             + sum_maps (A theta - b0)^T V^-1 (A theta - b0)       Eq. 6, generalised
 *                                                                 parametrisation b = A theta
 *
 * plus the analytic gradient of -2lnL with respect to every parameter, and a dense BFGS
 * minimiser with a strong-Wolfe line search that stops when the estimated distance to the
 * minimum, EDM = 1/2 g^T H g, falls below a threshold ([S], the variable-metric method
 * with EDM stop). As in [S] ("transformation layer") the minimiser works in coordinates
 * z in which the prior is uncorrelated: theta_B = theta0_B + L_B z_B with V_B = L_B L_B^T,
 * theta_i = theta0_i + sigma_i z_i otherwise (sigma_i = the parameter's step scale).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_K_OSC 1.266932679815373 /* dm2[eV^2] L[m] / (4 E[MeV]) -> phase, from hbar c */

enum { ORC_OK = 0, ORC_MAXITER = 1, ORC_LINESEARCH_FAIL = 2, ORC_NONFINITE = 3, ORC_BAD_FIXED = 4 };

typedef struct {
    int n_params;
    const double *theta0, *prior_sigma, *scale;
    int n_cov;
    const int *cov_size;   /* [n_cov] */
    const int *cov_idx;    /* concatenated parameter indices */
    const double *cov;     /* concatenated row-major m x m covariances */
    int osc_mode;          /* 0: Eq. 1 ; 1: exact 3-flavour vacuum ; 2: exact 3+1 vacuum */
    int osc_idx[6];        /* entries 4, 5 used by mode 2 only */
    double osc_val[6];
    int n_cores;
    const int *core_power_idx;
    int n_true;
    double e_lo, e_hi;
    int n_det;
    const int *det_n_reco;
    const double *det_response;   /* concatenated [N_r x N_t] per detector */
    int n_ds;
    const int *ds_det;
    const double *ds_t;           /* [n_ds x N_t] */
    const double *ds_baseline;    /* [n_ds x C] */
    const double *ds_weight;      /* [n_ds x C] */
    const int *ds_norm_idx, *ds_eff_idx;
    const int *ds_escale_idx;     /* [n_ds x 3] */
    const int *ds_shape_idx;      /* [n_ds x N_t] */
    int n_bkg;
    const int *bkg_ds;
    const double *bkg_template;   /* concatenated, N_r of its dataset each */
    const int *bkg_rate_idx;
    const int *bkg_shape_idx;     /* concatenated, N_r each */
    int remap_mode;               /* 0: overlap length ; 1: area-conserving spline */
    /* Eq. 6 with a generalised parametrisation b(theta) = A theta_idx: per map, k parameters,
     * m >= 1 constrained quantities with measured values b0 and covariance V (m x m) */
    int n_map;
    const int *map_k, *map_m;     /* [n_map] */
    const int *map_idx;           /* concatenated, k per map */
    const double *map_A;          /* concatenated row-major m x k */
    const double *map_b0;         /* concatenated, m per map */
    const double *map_V;          /* concatenated row-major m x m */
} orc_model;

typedef struct {
    orc_model m;
    int n_data;            /* total reco bins over datasets */
    int *ds_off;           /* data offset per dataset */
    int *det_off;          /* response offset per detector */
    int *bkg_off;          /* template offset per background */
    int *cov_off, *cov_moff;
    double *vinv;          /* concatenated V_B^-1 */
    double *chol;          /* concatenated lower Cholesky factors of V_B */
    int *in_block;         /* per parameter: 1 if it belongs to a covariance block */
    int *map_ioff, *map_aoff, *map_boff, *map_voff;   /* offsets into the map arrays */
    double *map_vinv;      /* concatenated V^-1 of the maps */
} orc_handle;

/* ------------------------------------------------------------------------------------ */
/* Small dense linear algebra (Cholesky) used only at set-up                              */
/* ------------------------------------------------------------------------------------ */
static int cholesky(int n, const double *a, double *l)
{
    memset(l, 0, sizeof(double) * n * n);
    for (int j = 0; j < n; ++j) {
        double s = a[j * n + j];
        for (int k = 0; k < j; ++k) s -= l[j * n + k] * l[j * n + k];
        if (!(s > 0.0)) return -1;
        l[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = a[i * n + j];
            for (int k = 0; k < j; ++k) t -= l[i * n + k] * l[j * n + k];
            l[i * n + j] = t / l[j * n + j];
        }
    }
    return 0;
}

/* inverse of an SPD matrix from its Cholesky factor: solve L L^T X = I column by column */
static void chol_inverse(int n, const double *l, double *inv)
{
    double *col = (double *)malloc(sizeof(double) * n);
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= l[i * n + k] * col[k];
            col[i] = s / l[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = col[i];
            for (int k = i + 1; k < n; ++k) s -= l[k * n + i] * col[k];
            col[i] = s / l[i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[i * n + c] = col[i];
    }
    free(col);
}

void orc_destroy(orc_handle *h)
{
    if (!h) return;
    free(h->ds_off); free(h->det_off); free(h->bkg_off); free(h->cov_off); free(h->cov_moff);
    free(h->vinv); free(h->chol); free(h->in_block);
    free(h->map_ioff); free(h->map_aoff); free(h->map_boff); free(h->map_voff); free(h->map_vinv);
    free(h);
}

/* Builds the handle. The arrays referenced by *m must outlive it. Returns NULL if a
 * covariance block is not symmetric positive definite. */
orc_handle *orc_create(const orc_model *m)
{
    orc_handle *h = (orc_handle *)calloc(1, sizeof(orc_handle));
    h->m = *m;
    h->ds_off = (int *)malloc(sizeof(int) * (m->n_ds + 1));
    h->det_off = (int *)malloc(sizeof(int) * (m->n_det + 1));
    h->bkg_off = (int *)malloc(sizeof(int) * (m->n_bkg + 1));
    h->det_off[0] = 0;
    for (int d = 0; d < m->n_det; ++d) h->det_off[d + 1] = h->det_off[d] + m->det_n_reco[d] * m->n_true;
    h->ds_off[0] = 0;
    for (int d = 0; d < m->n_ds; ++d) h->ds_off[d + 1] = h->ds_off[d] + m->det_n_reco[m->ds_det[d]];
    h->n_data = h->ds_off[m->n_ds];
    h->bkg_off[0] = 0;
    for (int b = 0; b < m->n_bkg; ++b)
        h->bkg_off[b + 1] = h->bkg_off[b] + m->det_n_reco[m->ds_det[m->bkg_ds[b]]];
    h->cov_off = (int *)malloc(sizeof(int) * (m->n_cov + 1));
    h->cov_moff = (int *)malloc(sizeof(int) * (m->n_cov + 1));
    h->cov_off[0] = h->cov_moff[0] = 0;
    for (int b = 0; b < m->n_cov; ++b) {
        h->cov_off[b + 1] = h->cov_off[b] + m->cov_size[b];
        h->cov_moff[b + 1] = h->cov_moff[b] + m->cov_size[b] * m->cov_size[b];
    }
    int nm = h->cov_moff[m->n_cov];
    h->vinv = (double *)malloc(sizeof(double) * (nm > 0 ? nm : 1));
    h->chol = (double *)malloc(sizeof(double) * (nm > 0 ? nm : 1));
    h->in_block = (int *)calloc(m->n_params, sizeof(int));
    for (int b = 0; b < m->n_cov; ++b) {
        int n = m->cov_size[b];
        const double *v = m->cov + h->cov_moff[b];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (fabs(v[i * n + j] - v[j * n + i]) > 1e-12 * (fabs(v[i * n + i]) + fabs(v[j * n + j]))) {
                    orc_destroy(h);
                    return NULL;
                }
        if (cholesky(n, v, h->chol + h->cov_moff[b]) != 0) {
            orc_destroy(h);
            return NULL;
        }
        chol_inverse(n, h->chol + h->cov_moff[b], h->vinv + h->cov_moff[b]);
        for (int i = 0; i < n; ++i) h->in_block[m->cov_idx[h->cov_off[b] + i]] = 1;
    }
    /* covariances of the Eq. 6 maps: symmetric positive definite, inverted once */
    int nmap = m->n_map > 0 ? m->n_map : 0;
    h->map_ioff = (int *)malloc(sizeof(int) * (nmap + 1));
    h->map_aoff = (int *)malloc(sizeof(int) * (nmap + 1));
    h->map_boff = (int *)malloc(sizeof(int) * (nmap + 1));
    h->map_voff = (int *)malloc(sizeof(int) * (nmap + 1));
    h->map_ioff[0] = h->map_aoff[0] = h->map_boff[0] = h->map_voff[0] = 0;
    for (int q = 0; q < nmap; ++q) {
        int k = m->map_k[q], r = m->map_m[q];
        h->map_ioff[q + 1] = h->map_ioff[q] + k;
        h->map_aoff[q + 1] = h->map_aoff[q] + r * k;
        h->map_boff[q + 1] = h->map_boff[q] + r;
        h->map_voff[q + 1] = h->map_voff[q] + r * r;
    }
    h->map_vinv = (double *)malloc(sizeof(double) * (h->map_voff[nmap] > 0 ? h->map_voff[nmap] : 1));
    for (int q = 0; q < nmap; ++q) {
        int r = m->map_m[q];
        const double *v = m->map_V + h->map_voff[q];
        double *l = (double *)malloc(sizeof(double) * r * r);
        int bad = 0;
        for (int i = 0; i < r && !bad; ++i)
            for (int j = 0; j < r; ++j)
                if (fabs(v[i * r + j] - v[j * r + i]) > 1e-12 * (fabs(v[i * r + i]) + fabs(v[j * r + j]))) bad = 1;
        if (!bad) bad = cholesky(r, v, l) != 0;
        if (!bad) chol_inverse(r, l, h->map_vinv + h->map_voff[q]);
        free(l);
        if (bad) {
            orc_destroy(h);
            return NULL;
        }
    }
    return h;
}

int orc_n_data(const orc_handle *h) { return h->n_data; }

/* ------------------------------------------------------------------------------------ */
/* Survival probability and its partial derivatives                                       */
/* ------------------------------------------------------------------------------------ */
/* mode 0 - Eq. 1 with Delta m^2_ee of Eq. 2 as a parameter:
 *   p = (sin^2 2th13, dm2_ee, sin^2 2th12, dm2_21)
 *   P = 1 - sin^2 2th13 sin^2(x_ee) - cos^4 th13 sin^2 2th12 sin^2(x_21),
 *   x_ab = K dm2_ab L / E, cos^2 th13 = (1 + sqrt(1 - sin^2 2th13)) / 2.
 * mode 1 - exact vacuum three-flavour survival, normal ordering for dm2_31 > 0 and inverted for
 *   dm2_31 < 0 (the quantity the
 *   medium-baseline expansion of Eq. 10 approximates):
 *   p = (sin^2 th12, sin^2 th13, dm2_21, dm2_31), dm2_32 = dm2_31 - dm2_21,
 *   P = 1 - cos^4 th13 sin^2 2th12 sin^2 x_21
 *         - sin^2 2th13 (cos^2 th12 sin^2 x_31 + sin^2 th12 sin^2 x_32).
 * mode 2 - exact vacuum 3+1 survival (one sterile state; the 3+1 model of the sterile
 *   search, with the two new parameters sin^2 2th14 and dm2_41):
 *   p = (sin^2 th12, sin^2 th13, dm2_21, dm2_31, sin^2 2th14, dm2_41),
 *   P = 1 - 4 sum_{i<j} |U_ei|^2 |U_ej|^2 sin^2 x_ji with the first row of the mixing matrix
 *   |U_e| = (c12 c13 c14, s12 c13 c14, s13 c14, s14), i.e.
 *   P = 1 - cos^4 th14 [cos^4 th13 sin^2 2th12 sin^2 x_21
 *                       + sin^2 2th13 (cos^2 th12 sin^2 x_31 + sin^2 th12 sin^2 x_32)]
 *         - sin^2 2th14 [cos^2 th13 (cos^2 th12 sin^2 x_41 + sin^2 th12 sin^2 x_42)
 *                        + sin^2 th13 sin^2 x_43],
 *   dm2_42 = dm2_41 - dm2_21, dm2_43 = dm2_41 - dm2_31, cos^2 th14 = (1 + sqrt(1 - sin^2 2th14))/2.
 * Returns P; dP (if not NULL) receives dP/dp_i. */
double orc_survival(int mode, const double *p, double L, double E, double *dP)
{
    double kl = ORC_K_OSC * L / E;
    if (mode == 0) {
        double s2t13 = p[0], dmee = p[1], s2t12 = p[2], dm21 = p[3];
        double root = sqrt(1.0 - s2t13);
        double c2 = 0.5 * (1.0 + root);           /* cos^2 th13 */
        double c4 = c2 * c2;
        double xee = dmee * kl, x21 = dm21 * kl;
        double see = sin(xee), s21 = sin(x21);
        double P = 1.0 - s2t13 * see * see - c4 * s2t12 * s21 * s21;
        if (dP) {
            double dc4 = 2.0 * c2 * (-0.25 / root);   /* d cos^4 th13 / d sin^2 2th13 */
            dP[0] = -see * see - dc4 * s2t12 * s21 * s21;
            dP[1] = -s2t13 * 2.0 * see * cos(xee) * kl;
            dP[2] = -c4 * s21 * s21;
            dP[3] = -c4 * s2t12 * 2.0 * s21 * cos(x21) * kl;
        }
        return P;
    } else if (mode == 2) {
        double s12 = p[0], s13 = p[1], dm21 = p[2], dm31 = p[3], S14 = p[4], dm41 = p[5];
        double c12 = 1.0 - s12, c13 = 1.0 - s13;
        double S12 = 4.0 * s12 * c12, S13 = 4.0 * s13 * c13;
        double root = sqrt(1.0 - S14);
        double c14 = 0.5 * (1.0 + root);          /* cos^2 th14 */
        double C4 = c14 * c14;
        double x21 = dm21 * kl, x31 = dm31 * kl, x32 = (dm31 - dm21) * kl;
        double x41 = dm41 * kl, x42 = (dm41 - dm21) * kl, x43 = (dm41 - dm31) * kl;
        double q21 = sin(x21) * sin(x21), q31 = sin(x31) * sin(x31), q32 = sin(x32) * sin(x32);
        double q41 = sin(x41) * sin(x41), q42 = sin(x42) * sin(x42), q43 = sin(x43) * sin(x43);
        double A = c13 * c13 * S12 * q21 + S13 * (c12 * q31 + s12 * q32);   /* three-flavour bracket */
        double Bs = c13 * (c12 * q41 + s12 * q42) + s13 * q43;              /* sterile bracket */
        double P = 1.0 - C4 * A - S14 * Bs;
        if (dP) {
            /* d sin^2 x / d dm2 = 2 sin x cos x kl */
            double d21 = sin(2.0 * x21) * kl, d31 = sin(2.0 * x31) * kl, d32 = sin(2.0 * x32) * kl;
            double d41 = sin(2.0 * x41) * kl, d42 = sin(2.0 * x42) * kl, d43 = sin(2.0 * x43) * kl;
            double dC4 = -c14 / (2.0 * root);      /* d cos^4 th14 / d sin^2 2th14 */
            dP[0] = -C4 * (c13 * c13 * 4.0 * (1.0 - 2.0 * s12) * q21 + S13 * (q32 - q31))
                    - S14 * c13 * (q42 - q41);
            dP[1] = -C4 * (-2.0 * c13 * S12 * q21 + 4.0 * (1.0 - 2.0 * s13) * (c12 * q31 + s12 * q32))
                    - S14 * (q43 - (c12 * q41 + s12 * q42));
            dP[2] = -C4 * (c13 * c13 * S12 * d21 - S13 * s12 * d32) + S14 * c13 * s12 * d42;
            dP[3] = -C4 * S13 * (c12 * d31 + s12 * d32) + S14 * s13 * d43;
            dP[4] = -dC4 * A - Bs;
            dP[5] = -S14 * (c13 * (c12 * d41 + s12 * d42) + s13 * d43);
        }
        return P;
    } else {
        double s12 = p[0], s13 = p[1], dm21 = p[2], dm31 = p[3];
        double dm32 = dm31 - dm21;
        double c12 = 1.0 - s12, c13 = 1.0 - s13;
        double S12 = 4.0 * s12 * c12, S13 = 4.0 * s13 * c13;
        double x21 = dm21 * kl, x31 = dm31 * kl, x32 = dm32 * kl;
        double a21 = sin(x21), a31 = sin(x31), a32 = sin(x32);
        double q21 = a21 * a21, q31 = a31 * a31, q32 = a32 * a32;
        double P = 1.0 - c13 * c13 * S12 * q21 - S13 * (c12 * q31 + s12 * q32);
        if (dP) {
            double d21 = 2.0 * a21 * cos(x21) * kl;   /* d sin^2 x21 / d dm21 */
            double d31 = 2.0 * a31 * cos(x31) * kl;
            double d32 = 2.0 * a32 * cos(x32) * kl;
            dP[0] = -c13 * c13 * 4.0 * (1.0 - 2.0 * s12) * q21 - S13 * (-q31 + q32);
            dP[1] = 2.0 * c13 * S12 * q21 - 4.0 * (1.0 - 2.0 * s13) * (c12 * q31 + s12 * q32);
            dP[2] = -c13 * c13 * S12 * d21 - S13 * s12 * (-d32);
            dP[3] = -S13 * (c12 * d31 + s12 * d32);
        }
        return P;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Energy correction: quadratic map re-integrated over the original binning [S]           */
/* ------------------------------------------------------------------------------------ */
/* Source bin k = [E_k, E_k+1] is mapped to [y0, y1] = [E'(E_k), E'(E_k+1)] and its content is
 * shared among target bins m = [T_m, T_m+1] in proportion to the overlap length
 * ov = min(y1, T_m+1) - max(y0, T_m) divided by the mapped width y1 - y0. Content mapped
 * outside the grid is dropped. Only targets between floor of y0 and floor of y1 (one extra
 * on either side) can overlap or touch the mapped interval; the loop visits exactly those. */
static inline double qmap(const double *a, double e) { return a[0] + a[1] * e + a[2] * e * e; }

static int remap_monotone(const orc_model *m, const double *a)
{
    return (a[1] + 2.0 * a[2] * m->e_lo > 0.0) && (a[1] + 2.0 * a[2] * m->e_hi > 0.0);
}

static void target_window(const orc_model *m, double y0, double y1, int *mlo, int *mhi)
{
    double de = (m->e_hi - m->e_lo) / m->n_true;
    double f0 = floor((y0 - m->e_lo) / de), f1 = floor((y1 - m->e_lo) / de);
    if (f0 < -2.0) f0 = -2.0;
    if (f1 > m->n_true + 1.0) f1 = m->n_true + 1.0;
    int lo = (int)f0 - 1, hi = (int)f1 + 1;
    *mlo = lo < 0 ? 0 : lo;
    *mhi = hi > m->n_true - 1 ? m->n_true - 1 : hi;
}

static int remap_spline(const orc_model *m, const double *a, const double *u, double *v);

/* v = M(a) u. Returns 0, or 1 if E' is not increasing on the grid (v untouched). */
int orc_remap(const orc_model *m, const double *a, const double *u, double *v)
{
    if (!remap_monotone(m, a)) return 1;
    if (m->remap_mode == 1) return remap_spline(m, a, u, v);
    double de = (m->e_hi - m->e_lo) / m->n_true;
    for (int i = 0; i < m->n_true; ++i) v[i] = 0.0;
    for (int k = 0; k < m->n_true; ++k) {
        double y0 = qmap(a, m->e_lo + k * de), y1 = qmap(a, m->e_lo + (k + 1) * de);
        double w = y1 - y0;
        int mlo, mhi;
        target_window(m, y0, y1, &mlo, &mhi);
        for (int t = mlo; t <= mhi; ++t) {
            double t0 = m->e_lo + t * de, t1 = m->e_lo + (t + 1) * de;
            double ov = fmin(y1, t1) - fmax(y0, t0);
            if (ov > 0.0) v[t] += u[k] * (ov / w);
        }
    }
    return 0;
}

/* ---- area-conserving spline remap ----------------------------------------------------
 * The energy correction of the paper's signal chain taken literally: the bin contents u on
 * the uniform true grid define the cumulative C(e_k) = sum_{i<k} u_i at the edges; an area-
 * conserving spline F interpolates C with continuous first derivative (the density f = F'),
 * F is energy-corrected (E' = a0 + a1 E + a2 E^2) and integrated over the original binning:
 *   v_j = F(x_{j+1}) - F(x_j),  x_j = E'^{-1}(e_j)  (content mapped off the grid is dropped).
 * Spline (reading; the paper names only "area conserving spline"): on bin k the cubic Hermite
 * interpolant of C with end slopes f(e_k) = (rho_{k-1} + rho_k) / 2, rho = u / de (one-sided
 * at the grid ends): F(e_k + t de) = C(e_k) + u_k h01(t) + de f(e_k) h10(t) + de f(e_{k+1}) h11(t)
 * with the Hermite basis h01 = 3t^2 - 2t^3, h10 = t^3 - 2t^2 + t, h11 = t^3 - t^2. F matches C
 * at every edge (each bin keeps its content) and f is continuous, so v is continuously
 * differentiable in (a0, a1, a2) (the overlap rule is not). */
static double edge_slope(const orc_model *m, const double *u, int k, double de)
{
    int n = m->n_true;
    if (k <= 0) return u[0] / de;
    if (k >= n) return u[n - 1] / de;
    return 0.5 * (u[k - 1] + u[k]) / de;
}

/* F(x) and f(x) = F'(x); cum[k] = sum_{i<k} u_i */
static double spline_F(const orc_model *m, const double *u, const double *cum, double x, double *f)
{
    double de = (m->e_hi - m->e_lo) / m->n_true;
    double y = (x - m->e_lo) / de;
    if (y <= 0.0) { if (f) *f = 0.0; return 0.0; }
    if (y >= m->n_true) { if (f) *f = 0.0; return cum[m->n_true]; }
    int k = (int)floor(y);
    if (k > m->n_true - 1) k = m->n_true - 1;
    double t = y - k, t2 = t * t, t3 = t2 * t;
    double s0 = edge_slope(m, u, k, de) * de, s1 = edge_slope(m, u, k + 1, de) * de;
    double F = cum[k] + u[k] * (3.0 * t2 - 2.0 * t3) + s0 * (t3 - 2.0 * t2 + t) + s1 * (t3 - t2);
    if (f) *f = (u[k] * (6.0 * t - 6.0 * t2) + s0 * (3.0 * t2 - 4.0 * t + 1.0) + s1 * (3.0 * t2 - 2.0 * t)) / de;
    return F;
}

/* x with a0 + a1 x + a2 x^2 = e on the increasing branch */
static double qmap_inv(const double *a, double e)
{
    double r = e - a[0];
    return 2.0 * r / (a[1] + sqrt(a[1] * a[1] + 4.0 * a[2] * r));
}

static int remap_spline(const orc_model *m, const double *a, const double *u, double *v)
{
    int n = m->n_true;
    double de = (m->e_hi - m->e_lo) / n;
    double *cum = (double *)malloc(sizeof(double) * (n + 1));
    cum[0] = 0.0;
    for (int k = 0; k < n; ++k) cum[k + 1] = cum[k] + u[k];
    double Fprev = spline_F(m, u, cum, qmap_inv(a, m->e_lo), NULL);
    for (int j = 0; j < n; ++j) {
        double F1 = spline_F(m, u, cum, qmap_inv(a, m->e_lo + (j + 1) * de), NULL);
        v[j] = F1 - Fprev;
        Fprev = F1;
    }
    free(cum);
    return 0;
}

/* Adjoint of the spline remap: gu = M^T gv and ga += dv/da^T gv.
 * dF(x)/du_i: 1 for i < k (the cumulative), the Hermite weights of u_k and of the two edge
 * slopes for i = k - 1, k, k + 1; 1 for every i when x is past the grid, 0 below it.
 * dx/da_i = -x^i / (a1 + 2 a2 x). */
static void remap_spline_adjoint(const orc_model *m, const double *a, const double *u, const double *gv,
                                 double *gu, double *ga)
{
    int n = m->n_true;
    double de = (m->e_hi - m->e_lo) / n;
    double *cum = (double *)malloc(sizeof(double) * (n + 1));
    double *w = (double *)malloc(sizeof(double) * (n + 1));   /* d(-2lnL)/dF at each edge */
    double *below = (double *)calloc(n + 1, sizeof(double));  /* below[k]: added to gu[i], i < k */
    cum[0] = 0.0;
    for (int k = 0; k < n; ++k) cum[k + 1] = cum[k] + u[k];
    for (int k = 0; k < n; ++k) gu[k] = 0.0;
    for (int e = 0; e <= n; ++e) w[e] = (e > 0 ? gv[e - 1] : 0.0) - (e < n ? gv[e] : 0.0);
    for (int e = 0; e <= n; ++e) {
        double x = qmap_inv(a, m->e_lo + e * de), f;
        spline_F(m, u, cum, x, &f);
        double dxd = -1.0 / (a[1] + 2.0 * a[2] * x);
        ga[0] += w[e] * f * dxd;
        ga[1] += w[e] * f * dxd * x;
        ga[2] += w[e] * f * dxd * x * x;
        double y = (x - m->e_lo) / de;
        if (y <= 0.0) continue;
        if (y >= n) {
            below[n] += w[e];
            continue;
        }
        int k = (int)floor(y);
        if (k > n - 1) k = n - 1;
        double t = y - k, t2 = t * t, t3 = t2 * t;
        double h01 = 3.0 * t2 - 2.0 * t3, h10 = t3 - 2.0 * t2 + t, h11 = t3 - t2;
        below[k] += w[e];
        gu[k] += w[e] * h01;
        /* de * f(e_k) = (u_{k-1} + u_k) / 2, or u_0 at the lower end */
        if (k == 0) gu[0] += w[e] * h10;
        else { gu[k - 1] += w[e] * 0.5 * h10; gu[k] += w[e] * 0.5 * h10; }
        /* de * f(e_{k+1}) = (u_k + u_{k+1}) / 2, or u_{n-1} at the upper end */
        if (k + 1 >= n) gu[n - 1] += w[e] * h11;
        else { gu[k] += w[e] * 0.5 * h11; gu[k + 1] += w[e] * 0.5 * h11; }
    }
    double acc = 0.0;
    for (int i = n - 1; i >= 0; --i) {
        acc += below[i + 1];
        gu[i] += acc;
    }
    free(cum);
    free(w);
    free(below);
}

/* Adjoint of the remap: given gv = d(-2lnL)/dv, accumulate gu = M^T gv and
 * ga[i] += d(-2lnL)/da_i (right-sided derivative where a mapped edge sits on a grid edge). */
static void remap_adjoint(const orc_model *m, const double *a, const double *u, const double *gv,
                          double *gu, double *ga)
{
    double de = (m->e_hi - m->e_lo) / m->n_true;
    for (int k = 0; k < m->n_true; ++k) {
        double e0 = m->e_lo + k * de, e1 = e0 + de;
        double y0 = qmap(a, e0), y1 = qmap(a, e1);
        double w = y1 - y0;
        int mlo, mhi;
        target_window(m, y0, y1, &mlo, &mhi);
        double acc = 0.0, dy0 = 0.0, dy1 = 0.0;
        for (int t = mlo; t <= mhi; ++t) {
            double t0 = m->e_lo + t * de, t1 = m->e_lo + (t + 1) * de;
            double ov = fmin(y1, t1) - fmax(y0, t0);
            double F = ov > 0.0 ? ov / w : 0.0;
            /* right derivatives of the overlap length */
            double dov1 = (t0 <= y1 && y1 < t1) ? 1.0 : 0.0;
            double dov0 = (t0 <= y0 && y0 < t1) ? -1.0 : 0.0;
            double dF0 = (dov0 + F) / w;   /* dw/dy0 = -1 */
            double dF1 = (dov1 - F) / w;   /* dw/dy1 = +1 */
            acc += F * gv[t];
            dy0 += dF0 * gv[t];
            dy1 += dF1 * gv[t];
        }
        gu[k] = acc;
        ga[0] += u[k] * (dy0 + dy1);
        ga[1] += u[k] * (dy0 * e0 + dy1 * e1);
        ga[2] += u[k] * (dy0 * e0 * e0 + dy1 * e1 * e1);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Forward model and -2lnL                                                               */
/* ------------------------------------------------------------------------------------ */
static inline double pval(const double *theta, int idx, double dflt)
{
    return idx >= 0 ? theta[idx] : dflt;
}

static void escale_of(const orc_model *m, const double *theta, int d, double *a)
{
    const int *ai = m->ds_escale_idx + 3 * d;
    a[0] = pval(theta, ai[0], 0.0);
    a[1] = pval(theta, ai[1], 1.0);
    a[2] = pval(theta, ai[2], 0.0);
}

/* number of survival parameters of a formula */
static int n_osc(int mode) { return mode == 2 ? 6 : 4; }

static void osc_params(const orc_model *m, const double *theta, double *p)
{
    for (int i = 0; i < 6; ++i) p[i] = 0.0;
    for (int i = 0; i < n_osc(m->osc_mode); ++i)
        p[i] = m->osc_idx[i] >= 0 ? theta[m->osc_idx[i]] : m->osc_val[i];
}

/* u_d (signal per true bin before energy correction) for dataset d */
static void signal_true(const orc_handle *h, const double *theta, int d, double *u)
{
    const orc_model *m = &h->m;
    double de = (m->e_hi - m->e_lo) / m->n_true, p[6];
    osc_params(m, theta, p);
    double n = pval(theta, m->ds_norm_idx[d], 1.0);
    for (int k = 0; k < m->n_true; ++k) {
        double E = m->e_lo + (k + 0.5) * de, ptot = 0.0;
        for (int c = 0; c < m->n_cores; ++c) {
            double w = m->ds_weight[d * m->n_cores + c];
            if (w == 0.0) continue;
            ptot += pval(theta, m->core_power_idx[c], 1.0) * w *
                    orc_survival(m->osc_mode, p, m->ds_baseline[d * m->n_cores + c], E, NULL);
        }
        double s = pval(theta, m->ds_shape_idx[d * m->n_true + k], 1.0);
        u[k] = m->ds_t[d * m->n_true + k] * n * s * ptot;
    }
}

/* expectation mu for dataset d into mu (N_r of its detector); returns 0 or 1 (non-monotone) */
static int expected_ds(const orc_handle *h, const double *theta, int d, double *u, double *v, double *mu)
{
    const orc_model *m = &h->m;
    int det = m->ds_det[d], nr = m->det_n_reco[det];
    const double *R = m->det_response + h->det_off[det];
    double a[3];
    escale_of(m, theta, d, a);
    signal_true(h, theta, d, u);
    if (orc_remap(m, a, u, v)) return 1;
    double eff = pval(theta, m->ds_eff_idx[d], 1.0);
    for (int j = 0; j < nr; ++j) {
        double f = 0.0;
        for (int k = 0; k < m->n_true; ++k) f += R[j * m->n_true + k] * v[k];
        mu[j] = eff * f;
    }
    for (int b = 0; b < m->n_bkg; ++b) {
        if (m->bkg_ds[b] != d) continue;
        double r = pval(theta, m->bkg_rate_idx[b], 1.0);
        const double *B = m->bkg_template + h->bkg_off[b];
        const int *si = m->bkg_shape_idx + h->bkg_off[b];
        for (int j = 0; j < nr; ++j) mu[j] += r * B[j] * (1.0 + pval(theta, si[j], 0.0));
    }
    return 0;
}

/* All datasets' expectations, concatenated. Returns 0, or 1 if an energy map is non-monotone. */
int orc_expected(const orc_handle *h, const double *theta, double *mu)
{
    const orc_model *m = &h->m;
    double *u = (double *)malloc(sizeof(double) * m->n_true);
    double *v = (double *)malloc(sizeof(double) * m->n_true);
    int st = 0;
    for (int d = 0; d < m->n_ds && !st; ++d) st = expected_ds(h, theta, d, u, v, mu + h->ds_off[d]);
    free(u); free(v);
    return st;
}

/* Poisson deviance term 2[mu - n + n ln(n/mu)], the saturated-model normalisation of Eq. 8 */
double orc_deviance(double n, double mu)
{
    if (!(mu > 0.0)) return INFINITY;
    if (n == 0.0) return 2.0 * mu;
    return 2.0 * (mu - n + n * log(n / mu));
}

/* Prior part of -2lnL (Eq. 6 / Eq. 9) and its gradient */
static double prior_term(const orc_handle *h, const double *theta, double *grad)
{
    const orc_model *m = &h->m;
    double q = 0.0;
    for (int i = 0; i < m->n_params; ++i) {
        double s = m->prior_sigma[i];
        if (s > 0.0) {
            double r = (theta[i] - m->theta0[i]) / s;
            q += r * r;
            if (grad) grad[i] += 2.0 * r / s;
        }
    }
    for (int b = 0; b < m->n_cov; ++b) {
        int n = m->cov_size[b];
        const int *idx = m->cov_idx + h->cov_off[b];
        const double *vi = h->vinv + h->cov_moff[b];
        for (int i = 0; i < n; ++i) {
            double row = 0.0;
            for (int j = 0; j < n; ++j) row += vi[i * n + j] * (theta[idx[j]] - m->theta0[idx[j]]);
            q += (theta[idx[i]] - m->theta0[idx[i]]) * row;
            if (grad) grad[idx[i]] += 2.0 * row;
        }
    }
    /* Eq. 6 with b(theta) = A theta_idx: q += (b - b0)^T V^-1 (b - b0); its gradient is
     * A^T 2 V^-1 (b - b0) */
    for (int p = 0; p < m->n_map; ++p) {
        int k = m->map_k[p], r = m->map_m[p];
        const int *idx = m->map_idx + h->map_ioff[p];
        const double *A = m->map_A + h->map_aoff[p];
        const double *b0 = m->map_b0 + h->map_boff[p];
        const double *vi = h->map_vinv + h->map_voff[p];
        double *res = (double *)malloc(sizeof(double) * r);
        for (int i = 0; i < r; ++i) {
            double b = 0.0;
            for (int j = 0; j < k; ++j) b += A[i * k + j] * theta[idx[j]];
            res[i] = b - b0[i];
        }
        for (int i = 0; i < r; ++i) {
            double row = 0.0;
            for (int j = 0; j < r; ++j) row += vi[i * r + j] * res[j];
            q += res[i] * row;
            if (grad)
                for (int j = 0; j < k; ++j) grad[idx[j]] += 2.0 * A[i * k + j] * row;
        }
        free(res);
    }
    return q;
}

/* -2lnL at theta for data (concatenated reco bins), datasets selected by mask. If grad is not
 * NULL it receives d(-2lnL)/dtheta. Returns +inf if some mu <= 0 on a used bin or an energy
 * map is not increasing. */
double orc_nll(const orc_handle *h, const double *theta, const double *data, uint32_t mask, double *grad)
{
    const orc_model *m = &h->m;
    int nt = m->n_true, C = m->n_cores;
    double de = (m->e_hi - m->e_lo) / nt;
    double *u = (double *)malloc(sizeof(double) * nt);
    double *v = (double *)malloc(sizeof(double) * nt);
    double *gv = (double *)malloc(sizeof(double) * nt);
    double *gu = (double *)malloc(sizeof(double) * nt);
    double *mu = (double *)malloc(sizeof(double) * (h->n_data > 0 ? h->n_data : 1));
    double *gmu = (double *)malloc(sizeof(double) * (h->n_data > 0 ? h->n_data : 1));
    double nll = 0.0, p[6];
    osc_params(m, theta, p);
    if (grad) memset(grad, 0, sizeof(double) * m->n_params);

    for (int d = 0; d < m->n_ds; ++d) {
        if (!((mask >> d) & 1u)) continue;
        int det = m->ds_det[d], nr = m->det_n_reco[det];
        double *mud = mu + h->ds_off[d], *gmud = gmu + h->ds_off[d];
        const double *nd = data + h->ds_off[d];
        if (expected_ds(h, theta, d, u, v, mud)) { nll = INFINITY; break; }
        for (int j = 0; j < nr; ++j) {
            nll += orc_deviance(nd[j], mud[j]);
            gmud[j] = 2.0 * (1.0 - nd[j] / mud[j]);
        }
        if (!isfinite(nll)) break;
        if (!grad) continue;

        /* backgrounds: mu_j += r B_j (1 + delta_j) */
        for (int b = 0; b < m->n_bkg; ++b) {
            if (m->bkg_ds[b] != d) continue;
            double r = pval(theta, m->bkg_rate_idx[b], 1.0);
            const double *B = m->bkg_template + h->bkg_off[b];
            const int *si = m->bkg_shape_idx + h->bkg_off[b];
            for (int j = 0; j < nr; ++j) {
                double sh = 1.0 + pval(theta, si[j], 0.0);
                if (m->bkg_rate_idx[b] >= 0) grad[m->bkg_rate_idx[b]] += gmud[j] * B[j] * sh;
                if (si[j] >= 0) grad[si[j]] += gmud[j] * r * B[j];
            }
        }
        /* fold: f_j = eps sum_k R[j,k] v_k */
        const double *R = m->det_response + h->det_off[det];
        double eff = pval(theta, m->ds_eff_idx[d], 1.0);
        for (int k = 0; k < nt; ++k) {
            double s = 0.0;
            for (int j = 0; j < nr; ++j) s += R[j * nt + k] * gmud[j];
            gv[k] = eff * s;
        }
        if (m->ds_eff_idx[d] >= 0) {
            double s = 0.0;
            for (int j = 0; j < nr; ++j) {
                double f = 0.0;
                for (int k = 0; k < nt; ++k) f += R[j * nt + k] * v[k];
                s += gmud[j] * f;
            }
            grad[m->ds_eff_idx[d]] += s;
        }
        /* energy correction */
        double a[3], ga[3] = {0.0, 0.0, 0.0};
        escale_of(m, theta, d, a);
        if (m->remap_mode == 1)
            remap_spline_adjoint(m, a, u, gv, gu, ga);
        else
            remap_adjoint(m, a, u, gv, gu, ga);
        for (int i = 0; i < 3; ++i)
            if (m->ds_escale_idx[3 * d + i] >= 0) grad[m->ds_escale_idx[3 * d + i]] += ga[i];
        /* signal: u_k = t_k n s_k sum_c p_c w_c P(L_c, E_k) */
        double n = pval(theta, m->ds_norm_idx[d], 1.0);
        for (int k = 0; k < nt; ++k) {
            double E = m->e_lo + (k + 0.5) * de;
            double t = m->ds_t[d * nt + k];
            int si = m->ds_shape_idx[d * nt + k];
            double s = pval(theta, si, 1.0);
            double ptot = 0.0, dptot[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int c = 0; c < C; ++c) {
                double w = m->ds_weight[d * C + c];
                if (w == 0.0) continue;
                double dP[6];
                double P = orc_survival(m->osc_mode, p, m->ds_baseline[d * C + c], E, dP);
                double pw = pval(theta, m->core_power_idx[c], 1.0);
                ptot += pw * w * P;
                for (int i = 0; i < n_osc(m->osc_mode); ++i) dptot[i] += pw * w * dP[i];
                if (m->core_power_idx[c] >= 0) grad[m->core_power_idx[c]] += gu[k] * t * n * s * w * P;
            }
            for (int i = 0; i < n_osc(m->osc_mode); ++i)
                if (m->osc_idx[i] >= 0) grad[m->osc_idx[i]] += gu[k] * t * n * s * dptot[i];
            if (m->ds_norm_idx[d] >= 0) grad[m->ds_norm_idx[d]] += gu[k] * t * s * ptot;
            if (si >= 0) grad[si] += gu[k] * t * n * ptot;
        }
    }
    if (isfinite(nll)) nll += prior_term(h, theta, grad);
    free(u); free(v); free(gv); free(gu); free(mu); free(gmu);
    return nll;
}

/* ------------------------------------------------------------------------------------ */
/* Transformation layer: theta(z) and the chain rule [S]                                  */
/* ------------------------------------------------------------------------------------ */
static void theta_of_z(const orc_handle *h, const double *z, double *theta)
{
    const orc_model *m = &h->m;
    for (int i = 0; i < m->n_params; ++i)
        if (!h->in_block[i]) {
            double s = m->prior_sigma[i] > 0.0 ? m->prior_sigma[i] : m->scale[i];
            theta[i] = m->theta0[i] + s * z[i];
        }
    for (int b = 0; b < m->n_cov; ++b) {
        int n = m->cov_size[b];
        const int *idx = m->cov_idx + h->cov_off[b];
        const double *L = h->chol + h->cov_moff[b];
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j <= i; ++j) s += L[i * n + j] * z[idx[j]];
            theta[idx[i]] = m->theta0[idx[i]] + s;
        }
    }
}

static void z_of_theta(const orc_handle *h, const double *theta, double *z)
{
    const orc_model *m = &h->m;
    for (int i = 0; i < m->n_params; ++i)
        if (!h->in_block[i]) {
            double s = m->prior_sigma[i] > 0.0 ? m->prior_sigma[i] : m->scale[i];
            z[i] = (theta[i] - m->theta0[i]) / s;
        }
    for (int b = 0; b < m->n_cov; ++b) {
        int n = m->cov_size[b];
        const int *idx = m->cov_idx + h->cov_off[b];
        const double *L = h->chol + h->cov_moff[b];
        for (int i = 0; i < n; ++i) {
            double s = theta[idx[i]] - m->theta0[idx[i]];
            for (int j = 0; j < i; ++j) s -= L[i * n + j] * z[idx[j]];
            z[idx[i]] = s / L[i * n + i];
        }
    }
}

static void grad_z_of_theta(const orc_handle *h, const double *gt, double *gz)
{
    const orc_model *m = &h->m;
    for (int i = 0; i < m->n_params; ++i)
        if (!h->in_block[i]) {
            double s = m->prior_sigma[i] > 0.0 ? m->prior_sigma[i] : m->scale[i];
            gz[i] = s * gt[i];
        }
    for (int b = 0; b < m->n_cov; ++b) {
        int n = m->cov_size[b];
        const int *idx = m->cov_idx + h->cov_off[b];
        const double *L = h->chol + h->cov_moff[b];
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int i = j; i < n; ++i) s += L[i * n + j] * gt[idx[i]];
            gz[idx[j]] = s;
        }
    }
}

void orc_theta_of_z(const orc_handle *h, const double *z, double *theta) { theta_of_z(h, z, theta); }
void orc_z_of_theta(const orc_handle *h, const double *theta, double *z) { z_of_theta(h, theta, z); }

typedef struct {
    const orc_handle *h;
    const double *data;
    uint32_t mask;
    double *theta, *gt;
    int n_evals;
    const unsigned char *fixed;   /* parameters held at their start value, or NULL */
} objective;

/* A fixed parameter (one outside the prior blocks, so that its z coordinate is the parameter
 * itself up to a scale) gets a zero z-gradient: the BFGS directions then never move it, which
 * is the constrained minimisation of the profile likelihood (Eq. 7, likelihood ratio). */
static double obj_eval(objective *o, const double *z, double *gz)
{
    theta_of_z(o->h, z, o->theta);
    double f = orc_nll(o->h, o->theta, o->data, o->mask, o->gt);
    grad_z_of_theta(o->h, o->gt, gz);
    if (o->fixed)
        for (int i = 0; i < o->h->m.n_params; ++i)
            if (o->fixed[i]) gz[i] = 0.0;
    o->n_evals++;
    return f;
}

/* ------------------------------------------------------------------------------------ */
/* Dense BFGS with a strong-Wolfe line search (Nocedal & Wright, Alg. 6.1, 3.5, 3.6)       */
/* ------------------------------------------------------------------------------------ */
static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* minimiser of the cubic through (a, fa, ga), (b, fb, gb); falls back to bisection */
static double cubic_min(double a, double fa, double ga, double b, double fb, double gb)
{
    double d1 = ga + gb - 3.0 * (fa - fb) / (a - b);
    double disc = d1 * d1 - ga * gb;
    if (disc < 0.0 || !isfinite(disc)) return 0.5 * (a + b);
    double d2 = copysign(sqrt(disc), b - a);
    double t = b - (b - a) * (gb + d2 - d1) / (gb - ga + 2.0 * d2);
    if (!isfinite(t)) return 0.5 * (a + b);
    return t;
}

typedef struct {
    double alpha, f;
} ls_point;

/* phi(alpha) = f(z + alpha p). On success returns 0 and leaves z_new, g_new, f_new at the
 * accepted step; returns 1 if no acceptable step was found. */
static int line_search(objective *o, int n, const double *z, double f0, const double *g0, const double *p,
                       double alpha_init, double *z_new, double *g_new, double *f_new, double *alpha_out)
{
    const double c1 = 1e-4, c2 = 0.9;
    double dphi0 = dot(n, g0, p);
    double a_prev = 0.0, f_prev = f0, d_prev = dphi0;
    double alpha = alpha_init;
    double lo = 0, flo = 0, dlo = 0, hi = 0, fhi = 0, dhi = 0;
    /* crease fallback: the smallest trial step whose value is within rounding of phi(0) and
     * whose slope has risen above c2 phi'(0) (the line crossed a kink of the energy map) */
    const double eps_f = 1e-12 * (1.0 + fabs(f0));
    double a_crease = INFINITY;
    int zoom = 0;
    for (int it = 0; it < 40; ++it) {
        for (int i = 0; i < n; ++i) z_new[i] = z[i] + alpha * p[i];
        double f = obj_eval(o, z_new, g_new);
        double dphi = isfinite(f) ? dot(n, g_new, p) : INFINITY;
        if (isfinite(f) && f <= f0 + eps_f && dphi >= c2 * dphi0 && alpha < a_crease) a_crease = alpha;
        if (!zoom) {
            if (!isfinite(f) || f > f0 + c1 * alpha * dphi0 || (it > 0 && f >= f_prev)) {
                lo = a_prev; flo = f_prev; dlo = d_prev; hi = alpha; fhi = f; dhi = dphi; zoom = 1;
            } else if (fabs(dphi) <= -c2 * dphi0) {
                *f_new = f; *alpha_out = alpha; return 0;
            } else if (dphi >= 0.0) {
                lo = alpha; flo = f; dlo = dphi; hi = a_prev; fhi = f_prev; dhi = d_prev; zoom = 1;
            } else {
                a_prev = alpha; f_prev = f; d_prev = dphi;
                alpha *= 4.0;
                continue;
            }
        } else {
            if (!isfinite(f) || f > f0 + c1 * alpha * dphi0 || f >= flo) {
                hi = alpha; fhi = f; dhi = dphi;
            } else {
                if (fabs(dphi) <= -c2 * dphi0) { *f_new = f; *alpha_out = alpha; return 0; }
                if (dphi * (hi - lo) >= 0.0) { hi = lo; fhi = flo; dhi = dlo; }
                lo = alpha; flo = f; dlo = dphi;
            }
        }
        /* next trial inside the bracket [lo, hi], safeguarded away from its ends */
        double a = lo < hi ? lo : hi, b = lo < hi ? hi : lo;
        double t = isfinite(fhi) && isfinite(dhi) ? cubic_min(lo, flo, dlo, hi, fhi, dhi) : 0.5 * (lo + hi);
        double lo_b = a + 0.1 * (b - a), hi_b = b - 0.1 * (b - a);
        if (!(t >= lo_b && t <= hi_b)) t = 0.5 * (a + b);
        alpha = t;
        if (fabs(b - a) < 1e-16 * (1.0 + fabs(b))) break;
    }
    /* No strong-Wolfe point. Prefer a step across the kink (it carries the kink's curvature
     * into the BFGS update, as in BFGS for nonsmooth functions, Lewis & Overton 2013), else
     * the best sufficient-decrease point of the bracket. */
    double a_acc = isfinite(a_crease) ? a_crease : ((zoom && lo > 0.0 && flo < f0) ? lo : 0.0);
    if (a_acc > 0.0) {
        for (int i = 0; i < n; ++i) z_new[i] = z[i] + a_acc * p[i];
        *f_new = obj_eval(o, z_new, g_new);
        *alpha_out = a_acc;
        return 0;
    }
    return 1;
}

/* Minimises -2lnL(theta(z)) from theta_start. Writes the best fit to theta_out and returns a
 * status: 0 converged (EDM < edm_tol), 1 iteration limit, 2 line search failed, 3 non-finite
 * start. */
int orc_fit_ex(const orc_handle *h, const double *data, uint32_t mask, const double *theta_start,
               const unsigned char *fixed, double edm_tol, int max_iter, double *theta_out, double *nll_out,
               int *iters_out, int *nevals_out, double *edm_out)
{
    const orc_model *m = &h->m;
    int n = m->n_params;
    if (fixed)
        for (int i = 0; i < n; ++i)
            if (fixed[i] && h->in_block[i]) return ORC_BAD_FIXED;
    objective o = {h, data, mask, (double *)malloc(sizeof(double) * n), (double *)malloc(sizeof(double) * n), 0,
                   fixed};
    double *z = (double *)malloc(sizeof(double) * n), *g = (double *)malloc(sizeof(double) * n);
    double *zn = (double *)malloc(sizeof(double) * n), *gn = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n), *H = (double *)malloc(sizeof(double) * n * n);
    double *s = (double *)malloc(sizeof(double) * n), *y = (double *)malloc(sizeof(double) * n);
    double *Hy = (double *)malloc(sizeof(double) * n);
    z_of_theta(h, theta_start, z);
    double f = obj_eval(&o, z, g), edm = INFINITY;
    int status = isfinite(f) ? ORC_MAXITER : ORC_NONFINITE, iter = 0, fresh = 1;
    memset(H, 0, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) H[i * n + i] = 1.0;
    while (status == ORC_MAXITER && iter < max_iter) {
        for (int i = 0; i < n; ++i) p[i] = -dot(n, H + i * n, g);
        edm = -0.5 * dot(n, g, p);
        if (edm < edm_tol) { status = ORC_OK; break; }
        double pn = sqrt(dot(n, p, p));
        double alpha0 = fresh ? fmin(1.0, 1.0 / pn) : 1.0, alpha, fn;
        if (line_search(&o, n, z, f, g, p, alpha0, zn, gn, &fn, &alpha)) {
            if (fresh) { status = ORC_LINESEARCH_FAIL; break; }
            memset(H, 0, sizeof(double) * n * n);          /* restart from steepest descent */
            for (int i = 0; i < n; ++i) H[i * n + i] = 1.0;
            fresh = 1;
            continue;
        }
        for (int i = 0; i < n; ++i) { s[i] = zn[i] - z[i]; y[i] = gn[i] - g[i]; }
        double sy = dot(n, s, y);
        if (sy > 1e-12 * sqrt(dot(n, s, s) * dot(n, y, y))) {
            if (fresh) {   /* scale the initial inverse Hessian (N&W eq. 6.20) */
                double gam = sy / dot(n, y, y);
                for (int i = 0; i < n * n; ++i) H[i] *= gam;
            }
            /* H <- (I - r s y^T) H (I - r y s^T) + r s s^T, r = 1/(y^T s) */
            double r = 1.0 / sy;
            for (int i = 0; i < n; ++i) Hy[i] = dot(n, H + i * n, y);
            double yHy = dot(n, y, Hy);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j)
                    H[i * n + j] += -r * (s[i] * Hy[j] + Hy[i] * s[j]) + (r * r * yHy + r) * s[i] * s[j];
            fresh = 0;
        }
        memcpy(z, zn, sizeof(double) * n);
        memcpy(g, gn, sizeof(double) * n);
        f = fn;
        ++iter;
    }
    theta_of_z(h, z, theta_out);
    *nll_out = f;
    *iters_out = iter;
    *nevals_out = o.n_evals;
    *edm_out = edm;
    free(o.theta); free(o.gt); free(z); free(g); free(zn); free(gn); free(p); free(H);
    free(s); free(y); free(Hy);
    return status;
}

int orc_fit(const orc_handle *h, const double *data, uint32_t mask, const double *theta_start,
            double edm_tol, int max_iter, double *theta_out, double *nll_out, int *iters_out,
            int *nevals_out, double *edm_out)
{
    return orc_fit_ex(h, data, mask, theta_start, NULL, edm_tol, max_iter, theta_out, nll_out, iters_out,
                      nevals_out, edm_out);
}

/* Fits n_inst instances on n_threads host threads (OpenMP when compiled with it).
 * Instance i uses handle hs[model_of[i]], data[i], mask[i], starts[i] and writes
 * theta_out[i] (n_params of its model), nll[i], iters[i], nevals[i], status[i]. */
void orc_fit_many(orc_handle *const *hs, int n_inst, const int *model_of, const double *const *data,
                  const uint32_t *mask, const double *const *starts, double edm_tol, int max_iter,
                  double *const *theta_out, double *nll, int *iters, int *nevals, int *status, int n_threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int i = 0; i < n_inst; ++i) {
        double edm;
        status[i] = orc_fit(hs[model_of[i]], data[i], mask[i], starts[i], edm_tol, max_iter, theta_out[i],
                            &nll[i], &iters[i], &nevals[i], &edm);
    }
    (void)n_threads;
}

/* Event-level reweighting ([S], "GPU accelerated computation"): the oscillated spectrum of
 * simulated events, out[b] = sum over the events in reco bin b of weight_e P(L_core(e), E_e)
 * with the survival formula `mode` at the parameters p (4, or 6 for mode 2). Events in any order; bins outside
 * [0, n_bins) are skipped. */
void orc_event_spectrum(int mode, const double *p, const double *core_L, long long n_events, const float *energy,
                        const unsigned char *core, const float *weight, const int *bin, int n_bins, double *out)
{
    for (int b = 0; b < n_bins; ++b) out[b] = 0.0;
    for (long long e = 0; e < n_events; ++e) {
        int b = bin[e];
        if (b < 0 || b >= n_bins) continue;
        out[b] += (double)weight[e] * orc_survival(mode, p, core_L[core[e]], (double)energy[e], NULL);
    }
}

int orc_openmp_enabled(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
