// Kernel entry points and launch arguments shared by kernels.cu and capi.cu.
#pragma once
#include "dev_model.cuh"

namespace fitcore {

// Fisher preconditioner of one dataset subset of a model (see the model's pre_Q / pre_c)
struct PreEntry {
    uint32_t mask;               // the datasets it covers
    int r;
    const float *Q, *c;          // Q^T rows on the vector pitch; c then the coefficients of T^-1
};

struct FitArgs {
    const DevModel *models;      // device array, one per model
    const fit_instance *inst;    // device [n_inst]
    int n_inst;
    int hist;                    // L-BFGS pairs
    int max_iter;
    int max_ls;                  // trial steps per line search
    int restarts;                // history restarts after the first EDM convergence
    double edm_tol;
    double f_noise_rel;
    const float *data;           // device
    const double *start;         // device or nullptr
    double *best;                // device
    fit_result *results;         // device [n_inst]
    int *queue;                  // device counter, zero at launch
    float *ws_global;            // per-block global workspace slices (or nullptr)
    int64_t ws_stride;           // floats per block slice
    int smem_floats;             // dynamic shared floats available for the workspace
    int hist_global;             // 1: the L-BFGS history lives in the global slice
    const uint8_t *fixed;        // device, indexed like start/best, or nullptr: held parameters
    uint64_t budget_ns;
    int precond;                 // 1: fit in the models' preconditioned coordinates (if built)
    const int *order;            // device [n_inst] or nullptr: the instance taken at each queue
                                 // position (costliest first, so no long fit starts last)
    const PreEntry *pre_tab;     // device [n_models x pre_per_model] or nullptr: preconditioners
    int pre_per_model;           // of the dataset subsets the instances fit
};

__global__ void eval_kernel(const DevModel *gm, int B, const double *theta, const float *data,
                            const uint32_t *masks, double *nll_out, float *grad_out,
                            float *mu_out, int *status_out, float *ws_global, int ws_in_smem);
// Lockstep engine: the instances of one model advance together, one evaluation per round;
// a round is three launches (forward + likelihood per (instance, dataset), adjoint per
// (instance, dataset), minimiser step per instance). Group-local index g addresses the state
// arrays; `group[g]` is the instance's index in the call.
struct FitState;
struct LsArgs {
    const DevModel *model;       // device
    const fit_instance *inst;    // device [n_inst of the call]
    const int *group;            // device [n]
    int n;
    const float *data;
    const double *start;         // device or nullptr
    const uint8_t *fixed;        // device, indexed like start, or nullptr
    double *best;
    fit_result *results;
    FitState *state;             // [n]
    float *vec;                  // [n x vec_stride]: 12 working P-vectors, then the history
    int64_t vec_stride;
    float *gsl;                  // [n x n_ds x P] gradient contributions per dataset
    double *nll_ds;              // [n x n_ds]
    float *gmu;                  // [n x n_ds x max_reco] dD/dmu of the last forward pass
    int *stat;                   // [n] evaluation status bits
    const int *act;              // active group indices this round
    const int *n_act;
    int *act_next;               // filled by the step kernel
    int *n_act_next;
    float *ws_global;            // evaluation workspace per resident block (when not in smem)
    int64_t ws_stride;
    int ws_in_smem;
    int hist, max_iter, max_ls, restarts;
    double edm_tol, f_noise_rel;
    uint64_t budget_ns;
    uint64_t *deadline;          // device: set by the init kernel
    int precond;                 // 1: fit in the model's preconditioned coordinates
    // engine 2 (folds on the tensor cores): ws_global holds one workspace per (active position,
    // dataset) pair; matrices per dataset d of n rows (row = active position)
    float *vhi, *vlo;            // [n_ds][n x ldt] corrected spectra, TF32 high part and rest
    float *fbuf;                 // [n_ds][n x ldf] fold R v (before the efficiency)
    float *ghi, *glo;            // [n_ds][n x ldr] dD/dmu, TF32 high part and rest
    float *gvbuf;                // [n_ds][n x ldt] R^T dD/dmu
    int ldf, ldr;
};

__global__ void ls_init_kernel(LsArgs A);
__global__ void ls_tc_fwd_kernel(LsArgs A);
__global__ void ls_tc_fwd_kernel6(LsArgs A);
__global__ void ls_tc_lik_kernel(LsArgs A);
__global__ void ls_tc_lik_kernel6(LsArgs A);
__global__ void ls_tc_adj_kernel(LsArgs A);
__global__ void ls_tc_adj_kernel6(LsArgs A);
__global__ void ls_forward_kernel(LsArgs A);
__global__ void ls_adjoint_kernel(LsArgs A);
__global__ void ls_forward_kernel6(LsArgs A);   // models with the 3+1 formula
__global__ void ls_adjoint_kernel6(LsArgs A);
__global__ void ls_step_kernel(LsArgs A);
size_t ls_state_bytes();
size_t ls_step_smem_bytes();
size_t ls_eval_smem_bytes(int P, int ws_floats);

// the persistent fit kernel compiled for 4 or 5 resident blocks per SM (host entry address)
const void *fit_kernel_func(int variant, int n_osc, bool pre);

size_t eval_smem_bytes(const DevModel &hm, bool ws_in_smem);

// batched.cu / poisson.cu / mlp.cu
// linstart.cu: theta_out = theta0 + K_{sel[b]} (data_b - mu0) (fit_linear_start)
int linear_start_apply(int B, int P, int D, const double *theta0_dev, const float *mu0_dev, const float *data,
                       const float *const *K, int n_var, const int *sel_dev, double *theta_out, cudaStream_t s);
int expected_tc(const DevModel &h, const DevModel *dev, int B, const double *theta, float *mu, int *status,
                int precision, cudaStream_t s);
int poisson_sample(int64_t n, const float *mu, uint64_t seed, uint64_t offset, float *out, cudaStream_t s);
int features(int B, int n_data, const float *data, const float *nbar, const uint32_t *masks, const int *slot_ds,
             const int *status, int n_in, int slot0, int onehot, float *x, cudaStream_t s);
int draw_theta(const DevModel &h, const DevModel *dev, int B, uint64_t seed, uint64_t offset, int n_uni,
               const int *uidx, const double *uhalf, int n_masks, const uint32_t *choices, double *theta,
               uint32_t *masks, cudaStream_t s, float *z_out = nullptr);
int targets(int B, int P, const double *theta, const double *theta0, int n_t, const int *idx, const double *scale,
            int n_out, const int *status, float *y, cudaStream_t s);
int perturb_theta(int B, int P, int k, const double *theta, const int *o_param, const float *zscale, double hz,
                  double *out, cudaStream_t s);
int refresh_targets(int B, int P, int D, int k, int Pn, int n_rows, const double *theta, const double *theta0,
                    const float *z, const float *cnt, const float *mu, const float *mup, const int *st_p,
                    const int *o_param, const int *n_param, const int *tkind, const float *lam_o, const float *bufs,
                    int64_t var_floats, double hz, int n_t, const int *idx, const double *scale, const float *zf,
                    int n_var, const uint32_t *choices, const uint32_t *masks, int n_out, const int *status, float *y,
                    cudaStream_t s);
int mle_targets(int B, int P, int D, const double *theta, const double *theta0, const float *z, const float *cnt,
                const float *mu, int n_t, const int *idx, const double *scale, const float *K1, const float *K2,
                const float *zf, int n_var, const uint32_t *choices, const uint32_t *masks, int n_out,
                const int *status, float *y, cudaStream_t s);
// y[b][t] -= Kt[var(b)][t] . (cnt[b] - mu0) (targets relative to the linearised start)
int lin_residual_targets(int B, int D, int n_t, const float *Kt, const float *mu0, const float *cnt, int n_var,
                         const uint32_t *choices, const uint32_t *masks, int n_out, const int *status, float *y,
                         cudaStream_t s);
int starts(int B, int P, const double *theta0, int n_t, const int *idx, const double *scale, const float *out,
           int n_out, const double *base, double *theta, cudaStream_t s);
size_t fit_smem_bytes(int floats);
// Fit vectors are spaced by P rounded up to 4 floats, so that every vector starts on a
// 16-byte boundary and the history can be read as float4.
__host__ __device__ inline int fit_vec_pitch(int P) { return (P + 3) & ~3; }
constexpr int kMaxPreRank = 32;   // eigen-directions of the Fisher preconditioner
__host__ __device__ inline int fit_vec_floats(int P, int hist) { return (14 + 2 * hist) * fit_vec_pitch(P); }
__host__ __device__ inline int fit_hist_floats(int P, int hist) { return 2 * hist * fit_vec_pitch(P); }
__host__ __device__ inline int fit_work_floats(int P) { return 14 * fit_vec_pitch(P); }

}  // namespace fitcore
