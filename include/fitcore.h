/*
 * fitcore.h - C ABI of the GB300 forward-folding likelihood-fit library.
 *
 * The library evaluates the binned expectation of a reactor-neutrino oscillation model, the
 * Poisson -2lnL with Gaussian and covariance priors, its gradient, and runs many quasi-Newton
 * fits at once, all on one GPU (sm_103a). It follows PhyLiNO (arXiv 2502.15253):
 *
 *   expectation per dataset d, true bin k, reco bin j (Eq. 9; [L], [S]):
 *     u_dk  = t_dk n_d s_g(k) sum_c p_c w_dc P(L_dc, E_k; eta)        survival: Eq. 1 with
 *             Delta m^2_ee of Eq. 2, or the exact 3-flavour vacuum probability (Eq. 10)
 *     v_d   = M(a_d) u_d  energy correction E' = a0 + a1 E + a2 E^2, each true bin's content
 *             spread over the original binning by overlap length ([S], third signal step)
 *     mu_dj = eps_d sum_k R_d[j,k] v_dk + sum_b r_b B_bj (1 + delta_bj)
 *   -2lnL = sum_d sum_j 2[mu - n + n ln(n/mu)]            Eq. 3-5 normalised as in Eq. 8
 *         + sum_i ((theta_i - theta0_i)/sigma_i)^2          Eq. 6
 *         + sum_B (theta_B - theta0_B)^T V_B^-1 (theta_B - theta0_B)   Eq. 6, Eq. 9
 *
 * [S] = the paper's section "Structure of the framework"; [L] = its section "Likelihood
 * implementation for Double Chooz within the framework".
 *
 * Conventions
 *  - Every function returns FIT_OK (0) or a negative FIT_ERR_* code; fit_last_error() then
 *    gives a message (thread-local). No function traps the GPU; device-side failures become
 *    per-instance statuses.
 *  - Pointers marked "host or device" may point to either; the library asks the CUDA runtime
 *    which (cudaPointerGetAttributes) and stages host buffers through device memory itself.
 *    Pointers marked "host" must be host memory. The caller owns all buffers it passes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls that
 *    read or write only device buffers are asynchronous on that stream; calls with a host
 *    output synchronise the stream before returning.
 *  - Parameter vectors are double at the boundary. The kernels compute in FP32; the -2lnL
 *    bin sum, the prior quadratic form and the minimiser's curvature scalars are accumulated
 *    in double precision.
 *  - A model is immutable after creation and may be used from several streams at once.
 *    fit_batch() uses a library-owned device workspace guarded by a lock.
 */
#ifndef FITCORE_H
#define FITCORE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------------------- */
#define FIT_OK 0
#define FIT_ERR_INVALID_ARG (-1)    /* null pointer, size out of range, bad index          */
#define FIT_ERR_INVALID_CONFIG (-2) /* inconsistent model description                      */
#define FIT_ERR_NON_SPD_COV (-3)    /* a prior covariance block is not symmetric pos. def. */
#define FIT_ERR_CUDA (-4)           /* a CUDA runtime call failed (message has the name)   */
#define FIT_ERR_TIMEOUT (-5)        /* a device wait exceeded its bound                    */
#define FIT_ERR_OOM (-6)            /* device allocation failed                            */

/* ---- per-evaluation / per-instance statuses ------------------------------------------ */
#define FIT_STATUS_CONVERGED 0          /* EDM below tolerance                                */
#define FIT_STATUS_MAXITER 1            /* iteration limit reached                            */
#define FIT_STATUS_LINESEARCH_FAIL 2    /* no acceptable step along a descent direction       */
#define FIT_STATUS_NONFINITE 3          /* -2lnL or its gradient not finite at the start      */
#define FIT_STATUS_MU_NONPOSITIVE 4     /* an expected count <= 0 on a used bin (nll = +inf)  */
#define FIT_STATUS_ESCALE_NONMONOTONE 5 /* dE'/dE outside (0.25, 4) on the grid (nll = +inf)  */
#define FIT_STATUS_TIMEOUT 6            /* the fit exceeded its clock budget                  */
#define FIT_STATUS_STALLED 7            /* 100 iterations lowered -2lnL by less than twice the
                                         * FP32 noise allowance (f_noise_rel (1 + |f|)): the
                                         * point is that close in value to a minimum, but EDM
                                         * stayed above edm_tol (e.g. on a crease of the
                                         * overlap-length energy correction)                  */

/* Survival-probability forms */
#define FIT_OSC_EQ1 0     /* eta = (sin^2 2th13, dm2_ee, sin^2 2th12, dm2_21)       Eq. 1, 2 */
#define FIT_OSC_VACUUM3 1 /* eta = (sin^2 th12, sin^2 th13, dm2_21, dm2_31); dm2_31 > 0 normal, < 0 inverted ordering (Eq. 10 with +phi / -phi) */
/* exact 3+1 vacuum survival of the sterile-neutrino search ("Sterile neutrino searches": the
 * two new parameters sin^2 2th14 and dm2_41, 0 <= sin^2 2th14 < 1):
 * eta = (sin^2 th12, sin^2 th13, dm2_21, dm2_31, sin^2 2th14, dm2_41) */
#define FIT_OSC_STERILE4 2

/* Energy correction (the third step of the signal chain in "Structure of the framework": the
 * spectrum smoothed with a second-degree polynomial energy map and integrated again over the
 * original binning; "Neutrino signal" for the area-conserving spline): how the corrected
 * spectrum is integrated over the original binning */
#define FIT_REMAP_OVERLAP 0 /* each true bin's content spread uniformly over its mapped interval */
#define FIT_REMAP_SPLINE 1  /* area-conserving spline: C1 cubic Hermite interpolant of the
                             * cumulative content, slopes (rho_{k-1} + rho_k) / 2 at the edges */

/* Size limits of one model */
#define FIT_MAX_DATASETS 8
#define FIT_MAX_DETECTORS 4
#define FIT_MAX_BACKGROUNDS 24
#define FIT_MAX_CORES 16
#define FIT_MAX_PARAMS 1024
#define FIT_MAX_TRUE_BINS 4096
#define FIT_MAX_RECO_BINS 1024

/*
 * Model description (all pointers host memory, read during fit_model_create only).
 * A parameter index of -1 means "fixed at its nominal value": 1 for multiplicative factors
 * (norm, efficiency, shape reweight, rate, core power), (0, 1, 0) for (a0, a1, a2), 0 for a
 * background shape delta. Arrays marked "concatenated" list the items back to back.
 * Every number must be finite; ds_t, det_response and bkg_template entries must be >= 0.
 */
typedef struct fit_model_desc {
    int n_params;
    const double *theta0;      /* [P] nominal values = prior means                             */
    const double *prior_sigma; /* [P] Gaussian prior width; 0 = no individual prior            */
    const double *scale;       /* [P] minimiser step scale (> 0) for parameters without prior  */
    int n_cov;                 /* covariance-prior blocks (Eq. 6); their parameters need sigma 0 */
    const int *cov_size;       /* [n_cov] block sizes m_b                                      */
    const int *cov_idx;        /* concatenated parameter indices, sum m_b                      */
    const double *cov;         /* concatenated row-major m_b x m_b covariance matrices         */
    int osc_mode;              /* FIT_OSC_EQ1, FIT_OSC_VACUUM3 or FIT_OSC_STERILE4              */
    int osc_idx[6];            /* parameter index of each survival parameter, or -1 (entries    */
    double osc_val[6];         /* 4, 5 only for FIT_OSC_STERILE4); value where osc_idx is -1    */
    int n_cores;               /* reactor cores, <= FIT_MAX_CORES                              */
    const int *core_power_idx; /* [C] parameter index of each core's power factor              */
    int n_true;                /* true-energy grid: n_true uniform bins over [e_lo, e_hi] MeV  */
    double e_lo, e_hi;
    int n_det;
    const int *det_n_reco;       /* [n_det] reco bins per detector                            */
    const double *det_response;  /* concatenated row-major [N_r x n_true] per detector        */
    int n_ds;
    const int *ds_det;           /* [n_ds] detector of each dataset                           */
    const double *ds_t;          /* [n_ds x n_true] un-oscillated expected signal counts      */
    const double *ds_baseline;   /* [n_ds x C] baseline of each core, metres                  */
    const double *ds_weight;     /* [n_ds x C] flux share per core (0 = core not seen)        */
    const int *ds_norm_idx;      /* [n_ds] signal normalisation parameter                     */
    const int *ds_eff_idx;       /* [n_ds] efficiency parameter                               */
    const int *ds_escale_idx;    /* [n_ds x 3] (a0, a1, a2) parameters                        */
    const int *ds_shape_idx;     /* [n_ds x n_true] shape-reweight parameter per true bin     */
    int n_bkg;
    const int *bkg_ds;           /* [n_bkg] dataset of each background                        */
    const double *bkg_template;  /* concatenated [N_r of its dataset] expected counts         */
    const int *bkg_rate_idx;     /* [n_bkg] rate parameter                                    */
    const int *bkg_shape_idx;    /* concatenated [N_r] shape-delta parameter per reco bin     */
    int remap_mode;              /* FIT_REMAP_OVERLAP or FIT_REMAP_SPLINE                      */
} fit_model_desc;

typedef struct fit_model fit_model; /* opaque, device-resident constants */

typedef struct fit_model_info_t {
    int n_params;
    int n_data;       /* total reco bins over all datasets = length of one data vector */
    int n_datasets;
    int n_true;
    size_t device_bytes; /* device memory held by the model */
} fit_model_info_t;

/* Builds a model from its description: validates it, computes the banded response layout,
 * the Cholesky factors of the prior blocks (the transformation layer of [S]) and uploads
 * everything to the current device. *out receives the model (free with fit_model_destroy).
 * Errors: INVALID_ARG / INVALID_CONFIG (message names the field), NON_SPD_COV, OOM, CUDA. */
int fit_model_create(const fit_model_desc *desc, fit_model **out);
void fit_model_destroy(fit_model *model);
/* Sizes of a model: parameter count (the likelihood's parameter vector, signal and nuisance
 * parameters of the general concept, "General concept and statistical methods"), the data
 * vector's length (reco bins of all datasets, Eq. 9's product over datasets and bins), the
 * dataset and true-bin counts, and the device memory the model holds. model: from
 * fit_model_create*; info: host, written. Errors: INVALID_ARG on NULL. Synchronous, no
 * device call. */
int fit_model_info(const fit_model *model, fit_model_info_t *info);

/* Builds a model from a JSON configuration ([S]: the framework's first component reads a
 * configuration file naming the parameters, their priors and the datasets). `json` is a
 * NUL-terminated UTF-8 string (host memory, read during the call only). Schema (fields in
 * brackets are optional; a parameter reference is a name string, an index, or null = held
 * at its nominal value as in fit_model_desc):
 *   parameters:  [{name, value, [sigma], [scale]}, ...]        -> theta0, prior_sigma, scale
 *                an entry {namespace: ns, parameters: [...]} groups parameters whose names
 *                then read "ns.name" (nested groups "a.b.name"; [S]: parameter namespaces)
 *   [covariances]: [{params: [ref, ...], cov: [[...], ...]}]   -> Eq. 6 blocks
 *                or, for a prior on b = A theta (Eq. 6's generalised parametrisation, linear):
 *                {params: [k refs], map: [[k numbers] x m], mean: [m], cov: [[m x m]]}, m >= k,
 *                taken as the equivalent block C = (A^T V^-1 A)^-1 on the parameters with
 *                nominal values C A^T V^-1 b0 (these replace the parameters' "value"); the
 *                constant left over does not depend on theta and is dropped
 *   oscillation: {formula: "eq1" | "vacuum3" | "sterile4",
 *                 params: [4 or 6 entries: a parameter name, or a number = held constant]}
 *   true_grid:   {bins, e_lo, e_hi}          [energy_correction]: "overlap" (default) | "spline"
 *   core_powers: [ref per reactor core]
 *   detectors:   [{[name], response: [[n_true numbers] per reco bin]}]
 *   datasets:    [{detector: name | index, t: [n_true], baseline: [C], weight: [C],
 *                  [norm], [efficiency], [escale: [a0, a1, a2]], [shape: [n_true refs]],
 *                  [backgrounds: [{template: [N_r], [rate], [shape: [N_r refs]]}]]}]
 * Backgrounds take the order datasets, then their lists. Unknown keys are ignored. The model
 * keeps the parameter names (fit_model_param_name).
 * Errors: INVALID_ARG (null), INVALID_CONFIG (malformed JSON with its byte offset, a missing
 * or mistyped field, an unknown name, a size mismatch; the message names the field),
 * NON_SPD_COV (a map's V or A^T V^-1 A not positive definite), then those of
 * fit_model_create. All configuration errors are found before any device call. */
int fit_model_create_json(const char *json, fit_model **out);

/* Nominal values and prior widths ([S] parameter handling; Eq. 5, 6), host buffers [n_params]
 * (either may be NULL). prior_sigma is the individual Gaussian width, sqrt(V_ii) for a member
 * of a covariance block, 0 for a parameter without prior. */
int fit_model_params(const fit_model *model, double *theta0, double *prior_sigma);

/* Name of parameter i of a model created by fit_model_create_json; NULL for a model created
 * from a fit_model_desc or for i out of range. The string lives as long as the model. */
const char *fit_model_param_name(const fit_model *model, int i);

/* Expected counts mu ([L], [S]) for B parameter vectors.
 * theta: host or device, [B x P] double. mu_out: host or device, [B x n_data] float.
 * status_out: host or device [B] int (FIT_STATUS_*) or NULL. */
int fit_model_expected(fit_model *model, int B, const double *theta, float *mu_out,
                       int *status_out, void *stream);

/* -2lnL and its gradient for B parameter vectors at once (Eq. 3-9).
 * theta: host or device [B x P] double; data: host or device [B x n_data] float counts
 * (NULL = every row uses the model's Asimov data at theta0); masks: host or device [B]
 * uint32, bit d set = dataset d enters the Poisson term (NULL = all datasets).
 * nll_out: host or device [B] double (+inf where mu <= 0 or the energy map is invalid).
 * grad_out: host or device [B x P] float d(-2lnL)/dtheta, or NULL to skip.
 * status_out: host or device [B] int or NULL. */
int fit_model_eval(fit_model *model, int B, const double *theta, const float *data,
                   const uint32_t *masks, double *nll_out, float *grad_out, int *status_out,
                   void *stream);

/* One fit instance of fit_batch. */
typedef struct fit_instance {
    int model;         /* index into the models array                                  */
    uint32_t mask;     /* datasets entering the Poisson term                            */
    int64_t data_off;  /* offset (floats) of its data vector in `data`                  */
    int64_t param_off; /* offset (doubles) of its start / result vector in start / best */
} fit_instance;

typedef struct fit_batch_opts {
    double edm_tol;       /* stop when EDM = 1/2 g^T H g < edm_tol (default 1e-8)             */
    int max_iter;         /* iteration limit (default 2000)                                  */
    int history;          /* L-BFGS pairs kept, 1..32 (default 32; the two-loop recursion runs
                             on one warp, a lane per pair)                                   */
    double f_noise_rel;   /* relative noise allowance of -2lnL in the line search (1e-6)     */
    int threads;          /* threads per block, multiple of 32 in [64, 128]; 0 = default 128 */
    int blocks_per_sm;    /* resident blocks per SM (an upper bound): 5 or more selects the
                             96-register build of the kernel, 1-4 the 128-register one;
                             0 = automatic                                                  */
    int use_graph;        /* 1 = launch through a cached CUDA graph (work-queue memset and
                             kernel nodes, parameters updated in place for each call)        */
    double time_budget_s; /* per-launch clock budget (0 = 60 s); exceeded -> FIT_STATUS_TIMEOUT */
    int restarts;         /* history restarts after the first EDM convergence, 0..8 (default 0):
                             each rebuilds the L-BFGS pairs for at least `history` iterations,
                             which firms up the EDM estimate in flat directions             */
    int placement;        /* per-fit workspace: 0 = automatic (most resident fits per SM),
                             1 = all in shared memory, 2 = L-BFGS history in global memory
                             (L2-resident) and the rest in shared memory, 3 = all global      */
    int engine;           /* 0 = persistent kernel (one block per fit at a time); 1 = lockstep:
                             the fits of a model advance one evaluation per round, each round
                             three launches over all of them (threads, blocks_per_sm and
                             placement then do not apply); 2 = lockstep with the response
                             fold and its adjoint as tensor-core GEMMs over all active fits
                             of a model (F = V R^T, G R; split TF32, the fold of [S] "one
                             response matrix times many spectra"), one workspace per
                             (fit, dataset) kept through the round                          */
    int precondition;     /* 1 (default) = persistent engine fits in Fisher-preconditioned
                             coordinates: the expected Hessian of -2lnL at the model's nominal
                             point, built once per model on first use, makes the quasi-Newton
                             problem nearly isotropic (fewer iterations); 0 = plain whitened
                             coordinates. Held parameters are left out of the transform.    */
} fit_batch_opts;

/* Result of one instance. */
typedef struct fit_result {
    double nll_min; /* -2lnL at the returned point           */
    double edm;     /* EDM at the returned point             */
    int iters;      /* quasi-Newton iterations                */
    int n_evals;    /* expectation + gradient evaluations     */
    int status;     /* FIT_STATUS_*                           */
    int pad;
} fit_result;

/* Sets *opts to the defaults. */
void fit_batch_default_opts(fit_batch_opts *opts);

/* The best fit of one instance as a JSON object ([S]: the output component writes the
 * converged fit as JSON, the interface to the rest of an analysis chain):
 *   {"nll_min": x, "edm": x, "iters": n, "n_evals": n, "status": "converged" | ...,
 *    "params": {"<name>": value, ...}}
 * with the model's parameter names (p0, p1, ... for a model built from a description);
 * numbers print with 17 significant digits (exact FP64 round trip), non-finite ones as null.
 * best: host [n_params] doubles; res: host. buf: host, or NULL to query the size only.
 * *needed receives the size in bytes including the terminating NUL.
 * Errors: INVALID_ARG (null argument, buf_len < *needed: nothing is written). */
int fit_result_json(const fit_model *model, const double *best, const fit_result *res, char *buf,
                    size_t buf_len, size_t *needed);

/* Fits n_inst pseudo-experiments of possibly different models in one persistent launch:
 * one block per instance at a time, per-instance L-BFGS state on the device, the whole
 * expectation / -2lnL / adjoint evaluated inside the block ([S]: minimiser loop around the
 * likelihood; many fits in parallel as in the paper's ensemble studies).
 * models: host [n_models]; inst: host [n_inst];
 * data: host or device floats, instance i reads data + inst[i].data_off (n_data of its model);
 * start: host or device doubles, instance i starts at start + inst[i].param_off (NULL = the
 *        model's theta0);
 * best: host or device doubles, receives the best fit at best + inst[i].param_off;
 * results: host or device [n_inst];
 * opts: host, NULL = defaults. Synchronises `stream` if any output is host memory. */
int fit_batch(fit_model *const *models, int n_models, const fit_instance *inst, int n_inst,
              const float *data, const double *start, double *best, fit_result *results,
              const fit_batch_opts *opts, void *stream);

/* Batched -2lnL and gradient, as fit_model_eval, for callers that cannot allocate device
 * memory: a host application that owns a fixed device-memory budget and hands out every
 * buffer itself, a plugin running under another framework's allocator that forbids direct
 * cudaMalloc / cudaFree, or a latency-critical loop that must not call into the allocator.
 * The paper has no counterpart; this is a deployment variant of the same evaluation.
 *  - Allocates nothing: it calls no cudaMalloc / cudaFree / allocating library routine. Its
 *    per-block workspace is a 16 MiB array in this library's device memory, which every GPU
 *    that loads the library holds until the process exits.
 *  - theta, data, masks, nll_out, grad_out, status_out must all be device memory of the
 *    current device, or managed memory (host buffers are rejected with FIT_ERR_INVALID_ARG,
 *    since staging them would allocate; so is another GPU's memory). The model must have
 *    been created on the current device (else FIT_ERR_INVALID_ARG).
 *    data and masks may be NULL with the meaning they have in fit_model_eval, whose outputs
 *    and semantics this call shares.
 *  - A model whose per-block workspace exceeds the 16 MiB is rejected (FIT_ERR_INVALID_ARG);
 *    larger batches are processed by fewer resident blocks, never by a larger workspace.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *    with that device current); make that first call before any stream capture.
 *  - Every call shares the one array and leaves its last contents in it: calls whose
 *    executions overlap on the GPU (on different streams, or from different threads) race
 *    on it and must be serialised by the caller. Asynchronous on `stream`. */
int fit_model_eval_noalloc(fit_model *model, int B, const double *theta, const float *data,
                           const uint32_t *masks, double *nll_out, float *grad_out,
                           int *status_out, void *stream);

/* Tensor-core GEMM of the library (tcgen05 on sm_103a), used by the warm-start MLP and the
 * batched response fold, exposed for callers and tests. D = A B^T with A [M x K] and
 * B [N x K] row-major; tf32 = 0: bf16 operands (kind::f16), tf32 = 1: float operands read as
 * TF32 (kind::tf32); FP32 accumulation. All pointers device memory; rows 16-byte aligned
 * (lda, ldb multiples of 8 for bf16, of 4 for float). Epilogue `epi`:
 *   0: C = D;  1: C = D + bias[n];  2: C = D + bias[n] and Y = gelu(C) (bf16, exact erf GELU);
 *   3: Y = D * gelu'(aux[m][n]) (bf16);  4: C += D.
 * Asynchronous on `stream`. fit_tc_gemm_status() synchronises and returns (and clears) a
 * nonzero flag if a pipeline wait inside the kernel gave up (bounded waits, no hang). */
int fit_tc_gemm(int tf32, int M, int N, int K, const void *A, int lda, const void *B, int ldb, int epi,
                float *C, int ldc, void *Y, int ldy, const float *bias, const float *aux, int ldaux,
                void *stream);
int fit_tc_gemm_status(void);

/* Expected counts for B parameter vectors with the response fold on tensor cores (Eq. 9
 * expectation as fit_model_expected): the energy-corrected true spectra of all instances form
 * V_d [B x N_t] per dataset and F_d = V_d R_d^T is one tcgen05 GEMM (the dense contraction of
 * the path: one response matrix times many spectra). precision 0: TF32 operands (about 3e-4
 * relative per product; used to generate training spectra); precision 1: split 3xTF32,
 * x = x_hi + x_lo with x_hi exact in TF32, F = Vh Rh^T + Vh Rl^T + Vl Rh^T (FP32-level).
 * theta: host or device [B x P] double; mu_out: host or device [B x n_data] float (NaN rows
 * where the energy map is invalid); status_out: host or device [B] int or NULL. */
int fit_model_expected_tc(fit_model *model, int B, const double *theta, float *mu_out,
                          int *status_out, int precision, void *stream);

/* Poisson pseudo-data: out[i] ~ Poisson(mu[i]) as floats, i < n. Philox4x32-10 counters
 * (i + offset, draw, 0, 0) under key = seed, so results do not depend on the launch shape;
 * Knuth's multiplication method below mu = 10, Hormann's PTRS above. Domain 0 <= mu < 2^22;
 * mu = 0 gives 0, negative, non-finite or larger mu give NaN. mu, out: host or device. */
int fit_poisson_sample(int64_t n, const float *mu, uint64_t seed, uint64_t offset, float *out,
                       void *stream);

/* Warm-start network (not in the paper): an MLP n_in -> n_hidden (GELU) x n_hidden_layers ->
 * n_out with bf16 weights / activations, FP32 master weights and accumulation, every product
 * on the tensor-core GEMM, trained with AdamW on an MSE loss. */
typedef struct fit_mlp fit_mlp;
int fit_mlp_create(int n_in, int n_hidden, int n_hidden_layers, int n_out, uint64_t seed,
                   fit_mlp **out);
void fit_mlp_destroy(fit_mlp *mlp);
/* y = mlp(x): x device [B x n_in] float, y host or device [B x n_out] float. */
int fit_mlp_forward(fit_mlp *mlp, int B, const float *x, float *y, void *stream);
/* One AdamW step on the mean squared error against target (device [B x n_out]); x device
 * [B x n_in]; loss_out (host or device double, or NULL) receives the batch loss before the step. */
int fit_mlp_train_step(fit_mlp *mlp, int B, const float *x, const float *target, float lr,
                       float weight_decay, double *loss_out, void *stream);
/* Layer `layer` (0-based) master weights [out x in], bias [out] and the last step's gradients
 * (host or device buffers, any may be NULL); set_layer replaces weights and bias. Synchronous. */
int fit_mlp_get_layer(const fit_mlp *mlp, int layer, float *w, float *b, float *gw, float *gb);
int fit_mlp_set_layer(fit_mlp *mlp, int layer, const float *w, const float *b);

/* Network inputs of pseudo-experiments: x[b][slot0 + q] = log(1 + n_q) / log(1 + nbar_q) - 1
 * with nbar the model's expectation at theta0; bins of datasets whose bit is clear in masks[b]
 * (device [B], or NULL = all datasets) are 0; other slots 0 and x[b][onehot_slot] = 1 (if
 * >= 0). data device [B x n_data], x device [B x n_in]. */
int fit_warmstart_features(const fit_model *model, int B, const float *data, const uint32_t *masks,
                           int n_in, int slot0, int onehot_slot, float *x, void *stream);
/* Start points for fit_batch: the linearised best fit of every parameter (fit_linear_start),
 * then the network's corrections on its targets, theta[target_idx[t]] += y_t * target_scale[t]
 * for the first n_targets outputs (the network is trained on where a fit ends minus that
 * linearised start, see fit_warmstart_train). data device [B x n_data]; masks device [B] or
 * NULL; target arrays host; theta_out device [B x P]. Synchronous. */
int fit_warmstart_predict(fit_mlp *mlp, const fit_model *model, int B, const float *data,
                          const uint32_t *masks, int slot0, int onehot_slot, int n_targets,
                          const int *target_idx, const double *target_scale, double *theta_out,
                          void *stream);
/* Linearised best fit as start points (the warm start's deterministic part; the paper fits
 * from the nominal point). Near theta0 the expectation of Eq. 9 is mu0 + J z in the whitened
 * coordinates z of the transformation layer, and -2lnL (Poisson deviance plus the Gaussian and
 * covariance priors of Eq. 6, |z|^2 over the constrained coordinates) is minimised to second
 * order, with the expected Hessian, by one Gauss-Newton (Fisher scoring) step from z = 0:
 *   dz = (J^T W J + Lambda)^-1 J^T W (n - mu0),  W = diag(1/mu0) over the fitted datasets,
 *   Lambda = 1 on the constrained coordinates, 0 on the free ones;  theta = theta(dz).
 * Linear parameters (normalisations, rates, shapes, efficiencies) land close to their best
 * fit; oscillation parameters move by their linearised step (fit_warmstart_predict adds the
 * network's corrections to its targets). The rows (J from central differences of the
 * expectation, step 0.01 in z) are built on the host on first use for each dataset subset and
 * kept with the model; the product with the residuals n - mu0 runs on the tensor cores as a
 * split-TF32 product per subset (three GEMMs, FP32 accuracy; deterministic).
 * data device [B x n_data]; masks host or device [B] or NULL (all datasets; a mask with no
 * fitted dataset is FIT_ERR_INVALID_ARG; at most 16 distinct subsets per call); theta_out
 * device [B x P]. The model's device must be current. Synchronous. Errors: INVALID_ARG,
 * INVALID_CONFIG (an expectation near theta0 failed), OOM, CUDA, TIMEOUT (GEMM wait). */
int fit_linear_start(fit_model *model, int B, const float *data, const uint32_t *masks,
                     double *theta_out, void *stream);

#define FIT_WS_MAX_TARGETS 16
#define FIT_WS_MAX_MASKS 8

/* How one model (geometry) enters the warm-start network: where its bins sit among the inputs,
 * which parameters the outputs predict (standardised: y = (theta - theta0) / scale), which
 * parameters training draws uniformly in theta0 +- half instead of from their priors, and the
 * dataset masks a training sample draws from (uniformly; none = all datasets). */
typedef struct fit_warmstart_geom {
    int slot0;
    int onehot_slot;                          /* -1 = none                                  */
    int n_targets;
    int target_idx[FIT_WS_MAX_TARGETS];
    double target_scale[FIT_WS_MAX_TARGETS];
    int n_uniform;
    int uniform_idx[FIT_WS_MAX_TARGETS];
    double uniform_half[FIT_WS_MAX_TARGETS];
    int n_masks;
    uint32_t masks[FIT_WS_MAX_MASKS];
} fit_warmstart_geom;

/* Training parameter vectors: parameters in a covariance block theta0 + L z (V = L L^T), other
 * parameters theta0 + sigma z (sigma = prior width, or the free parameter's scale), z standard
 * normal; the geometry's uniform parameters theta0 + half (2u - 1). Sample b uses Philox4x32-10
 * counters (b + offset, i, 0x0D8A0001, 0) under key seed. theta_out device [B x P]; masks_out
 * device [B] or NULL. */
int fit_warmstart_draw(fit_model *model, const fit_warmstart_geom *geom, int B, uint64_t seed,
                       uint64_t offset, double *theta_out, uint32_t *masks_out, void *stream);

/* Trains the network for n_steps AdamW steps of `batch` fresh samples each, the geometries in
 * turn: draw theta and masks, expected spectra with the TF32 tensor-core fold, Poisson counts,
 * inputs and standardised targets, one step. The target of a sample is where a fit of its
 * counts would end, to first order: the drawn point moved by one Gauss-Newton step of -2lnL
 * with the expected Hessian, standardised by target_scale. The Jacobian of the expectation is
 * taken at the nominal point (built once per geometry and dataset mask from 2P + 1
 * expectations), except the columns of the free mass splittings among the uniform parameters,
 * which turn with the oscillation phase: those are re-evaluated at each drawn point (two
 * expectations per column and sample) and the step is solved by the Schur complement against
 * the block of all other parameters. The network learns that target minus the linearised
 * start of the same counts (fit_linear_start's step from theta0, standardised the same way),
 * so that fit_warmstart_predict adds its outputs to that start. Learning rate lr (0.05 + 0.95
 * (1 + cos(pi s / n_steps)) / 2) at step s. losses_out (host or device [n_steps] double, or
 * NULL) receives each step's batch loss. Synchronous. */
int fit_warmstart_train(fit_mlp *mlp, fit_model *const *models, const fit_warmstart_geom *geoms,
                        int n_geoms, int n_steps, int batch, float lr, float weight_decay,
                        uint64_t seed, double *losses_out, void *stream);

/* fit_batch with held parameters: fixed (host or device, indexed like start / best, or NULL)
 * marks parameters kept at their start values, e.g. the scanned parameters of a profile
 * likelihood (Eq. 7). Only parameters outside the covariance blocks can be held (their whitened
 * coordinate is the parameter itself); others give FIT_ERR_INVALID_ARG. */
int fit_batch_ex(fit_model *const *models, int n_models, const fit_instance *inst, int n_inst,
                 const float *data, const double *start, const uint8_t *fixed, double *best,
                 fit_result *results, const fit_batch_opts *opts, void *stream);

/* Profile likelihood on a raster (Eq. 7: -2 ln lambda = -2lnL(held point, best nuisances) -
 * -2lnL(best)): one launch fits the data vector (host or device, n_data floats, dataset mask
 * `mask`) without constraint and at each of the n_points rows of `points` (host, [n_points x
 * n_scan], values of the parameters scan_idx[0..n_scan), held fixed), all from `start` (host or
 * device, P doubles, or NULL = theta0). Outputs (host): *nll_min (the lowest -2lnL met, normally
 * the unconstrained fit), theta_best [P] or NULL, dchi2 [n_points] (-2 ln lambda), theta_points
 * [n_points x P] or NULL, status [n_points] or NULL. Synchronous. */
int fit_profile_scan(fit_model *model, const float *data, uint32_t mask, int n_scan,
                     const int *scan_idx, int n_points, const double *points, const double *start,
                     const fit_batch_opts *opts, double *nll_min, double *theta_best, double *dchi2,
                     double *theta_points, int *status, void *stream);

/* Wilks interval from a 1-D profile: the points x (increasing) where dchi2 crosses `level`
 * (1 for 68.27 %, 3.84 for 95 % with one parameter, Wilks' theorem), linearly between raster
 * points, on each side of the raster minimum. Returns 0, or bit 1 / bit 2 when the lower /
 * upper side stays below `level` up to the raster edge (then that edge is returned). */
int fit_wilks_interval(int n, const double *x, const double *dchi2, double level, double *lo,
                       double *hi);

/* Goodness of fit: P(chi^2_dof >= chi2), the p-value of a deviance (Eq. 8) with dof degrees of
 * freedom. NaN for dof < 1 or chi2 < 0. */
double fit_chi2_sf(double chi2, int dof);

/* Event-level reweighting ([S], "GPU accelerated computation": the oscillation weights of the
 * simulated events are the step the paper moves to the GPU). A set of simulated signal events
 * of one detector stays on the device: true energy (MeV, > 0), emitting core (< n_cores, with
 * baseline core_L[c] in m), weight (expected events it represents), reco bin (0..n_bins-1,
 * non-decreasing: the events sorted by bin). Arrays host or device, copied. */
typedef struct fit_mc fit_mc;
int fit_mc_create(int osc_mode, int n_cores, const double *core_L, int64_t n_events,
                  const float *energy, const uint8_t *core, const float *weight, const int *bin,
                  int n_bins, fit_mc **out);
void fit_mc_destroy(fit_mc *mc);
/* out[b][j] = sum over the events e of bin j of weight_e P(L_core(e), E_e; params[b]) for
 * b < B <= 64 parameter sets (params [B x 4], [B x 6] for FIT_OSC_STERILE4, in the
 * osc_mode's order, host or device; out
 * [B x n_bins] double, host or device). One pass over the events serves all B sets. With
 * device buffers the call is asynchronous on stream; with host buffers it returns when out is
 * written. */
int fit_mc_spectrum(fit_mc *mc, int B, const double *params, double *out, void *stream);
/* Synchronises the device and returns FIT_ERR_CUDA if any fit_mc_spectrum call on mc gave up
 * waiting for its staged event copies (bounded waits of 2 s; its spectra are then incomplete). */
int fit_mc_status(fit_mc *mc);

/* Chooses threads per block and resident blocks per SM for fit_batch on the current device by
 * timing the candidate configurations (64 threads with 8 or 10 blocks per SM, 96 or 128
 * threads with 4 or 5) on the first
 * n_sample instances (0 = ten per SM, at most n_inst), and writes the fastest into
 * opts->threads and opts->blocks_per_sm (other fields are used as given). Arguments as for
 * fit_batch; results of the timing runs are discarded. Synchronous. */
int fit_batch_autotune(fit_model *const *models, int n_models, const fit_instance *inst, int n_inst,
                       const float *data, const double *start, int n_sample, fit_batch_opts *opts,
                       void *stream);

/* Message of the last error on this thread ("" if none). */
const char *fit_last_error(void);

/* Number of kernels the library launched on this thread since the last call (and resets). */
int64_t fit_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* FITCORE_H */
