// Host side of the C ABI (include/fitcore.h): model construction, argument staging, launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <vector>

#include "gemm_tc.cuh"
#include "kernels.cuh"

namespace fitcore {
float *mlp_input_buffer(fit_mlp *m, int B);
int mlp_dims(const fit_mlp *m, int *n_in, int *n_out);
}

using fitcore::DevModel;

namespace {

thread_local std::string g_err;
thread_local int64_t g_launches = 0;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define FIT_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? FIT_ERR_OOM : FIT_ERR_CUDA,      \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
        }                                                                                  \
    } while (0)

constexpr double kOscK = 1.266932679815373;  // dm2[eV^2] L[m] / (4 E[MeV]) in radians, from hbar c

bool on_device(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Host staging of arrays into one device allocation.
struct Arena {
    std::vector<unsigned char> buf;
    std::vector<std::pair<const void **, size_t>> fix;
    size_t put(const void *p, size_t n) {
        size_t off = (buf.size() + 255) & ~size_t(255);
        buf.resize(off + std::max<size_t>(n, 16));
        if (n) std::memcpy(buf.data() + off, p, n);
        return off;
    }
    template <class T>
    void put(const T **field, const std::vector<T> &v) {
        fix.emplace_back(reinterpret_cast<const void **>(field), put(v.data(), v.size() * sizeof(T)));
    }
    void bind(void *base) {
        for (auto &f : fix) *f.first = static_cast<unsigned char *>(base) + f.second;
    }
};

// Cholesky V = L L^T (lower, row-major); returns false if V is not positive definite.
bool cholesky_lower(int n, const double *v, std::vector<double> &L) {
    L.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = v[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double ljj = std::sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = v[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = s / ljj;
        }
    }
    return true;
}

// W = L^-1 for lower-triangular L (forward substitution on the identity's columns)
void lower_inverse(int n, const std::vector<double> &L, std::vector<double> &W) {
    W.assign((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c) {
        for (int i = c; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s -= L[(size_t)i * n + k] * W[(size_t)k * n + c];
            W[(size_t)i * n + c] = s / L[(size_t)i * n + i];
        }
    }
}

struct LaunchCfg {
    int sms = 0;
    size_t smem_optin = 0;
};

int device_cfg(LaunchCfg &c) {
    int dev;
    FIT_CUDA(cudaGetDevice(&dev));
    FIT_CUDA(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev));
    int v;
    FIT_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    c.smem_optin = (size_t)v;
    return FIT_OK;
}

// A device buffer that is either the caller's device pointer or a stream-ordered staging copy.
struct Staged {
    void *dev = nullptr;
    bool owned = false;
};

int stage_in(const void *src, size_t bytes, cudaStream_t s, Staged &out) {
    if (!src || bytes == 0) {
        out.dev = const_cast<void *>(src);
        return FIT_OK;
    }
    if (on_device(src)) {
        out.dev = const_cast<void *>(src);
        return FIT_OK;
    }
    FIT_CUDA(cudaMallocAsync(&out.dev, bytes, s));
    out.owned = true;
    FIT_CUDA(cudaMemcpyAsync(out.dev, src, bytes, cudaMemcpyHostToDevice, s));
    return FIT_OK;
}

int stage_out(void *dst, size_t bytes, cudaStream_t s, Staged &out, bool &host) {
    host = false;
    if (!dst || bytes == 0) {
        out.dev = dst;
        return FIT_OK;
    }
    if (on_device(dst)) {
        out.dev = dst;
        return FIT_OK;
    }
    host = true;
    FIT_CUDA(cudaMallocAsync(&out.dev, bytes, s));
    out.owned = true;
    return FIT_OK;
}

void release(Staged &b, cudaStream_t s) {
    if (b.owned && b.dev) cudaFreeAsync(b.dev, s);
    b.dev = nullptr;
    b.owned = false;
}

std::mutex g_ws_mutex;
std::mutex g_pre_mutex;   // guards building a model's preconditioner

}  // namespace

struct fit_model {
    DevModel host;         // field values with device pointers
    DevModel *dev = nullptr;
    void *arena = nullptr;
    size_t bytes = 0;
    int n_params = 0, n_data = 0, n_ds = 0, n_true = 0;
    std::vector<uint8_t> in_block;   // parameter belongs to a covariance block (host copy)
    // host copy of the transformation layer theta = theta0 + J z (for the preconditioner)
    std::vector<double> theta0, zscale, blk_L;   // blk_L: the blocks' lower factors, packed
    std::vector<int> bsz, bidx;
    // Fisher preconditioner (built on first use): device matrices T, T^T, T^-1, state
    float *pre = nullptr;
    int pre_state = 0;     // 0 not built, 1 built, -1 failed (fits run unpreconditioned)
    std::vector<double> pre_U;                   // J^T diag(mu0)^(-1/2), P x D (host)
    std::vector<fitcore::PreEntry> pre_masks;    // preconditioners of dataset subsets
    // linearised best fit (fit_linear_start, built on first use): theta-space rows per dataset
    // subset, device [P x D'] (D' = D rounded up to 4), and the nominal expectation
    struct LinEntry {
        uint32_t mask;
        float *K;                 // device: [P x D'] TF32 parts, then [P x D'] rests
        std::vector<float> Kh;    // host copy (the warm start's training reads target rows)
    };
    std::deque<LinEntry> lin;          // (a deque: entries stay where they are as it grows)
    float *lin_mu0 = nullptr;          // device [D]
    std::vector<double> lin_mu0_host;
    std::vector<std::string> names;   // parameter names (models created from a configuration)
    std::vector<double> sigma;        // prior width per parameter (block members: sqrt(V_ii))
    int device = -1;                  // the CUDA device holding the model's memory
};

// error / launch-count hooks for the other translation units of the library
int fitcore_fail(int code, const std::string &msg) { return fail(code, msg); }

// hooks for noalloc.cu (same library)
int fitcore_noalloc_fail(int code, const std::string &msg) { return fail(code, msg); }
int fitcore_model_device(fit_model *model, const DevModel **dev, const DevModel **host, int *device) {
    *dev = model->dev;
    *host = &model->host;
    *device = model->device;
    return FIT_OK;
}

// The largest dynamic shared memory eval_kernel has been allowed on each device. The attribute
// is shared by every thread of the process, so the evaluation paths only ever raise it (under
// this lock): a smaller request never lowers a limit another thread's launch relies on.
namespace {
std::mutex g_eval_smem_mutex;
std::vector<size_t> g_eval_smem_limit;
}  // namespace

int fitcore_raise_eval_smem(size_t bytes) {
    int dev = 0;
    FIT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_eval_smem_mutex);
    if ((int)g_eval_smem_limit.size() <= dev) g_eval_smem_limit.resize(dev + 1, 0);
    if (bytes <= g_eval_smem_limit[dev]) return FIT_OK;
    FIT_CUDA(cudaFuncSetAttribute(fitcore::eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    g_eval_smem_limit[dev] = bytes;
    return FIT_OK;
}
void fitcore_count_launch() { g_launches++; }
void fitcore_model_set_names(fit_model *model, const std::vector<std::string> &names) { model->names = names; }

extern "C" {

const char *fit_last_error(void) { return g_err.c_str(); }

int64_t fit_kernel_launches(void) {
    int64_t n = g_launches;
    g_launches = 0;
    return n;
}

void fit_model_destroy(fit_model *model) {
    if (!model) return;
    if (model->dev) cudaFree(model->dev);
    if (model->arena) cudaFree(model->arena);
    if (model->pre) cudaFree(model->pre);
    for (auto &pm : model->pre_masks)
        if (pm.Q) cudaFree(const_cast<float *>(pm.Q));
    for (auto &le : model->lin)
        if (le.K) cudaFree(le.K);
    if (model->lin_mu0) cudaFree(model->lin_mu0);
    delete model;
}

int fit_model_info(const fit_model *model, fit_model_info_t *info) {
    if (!model || !info) return fail(FIT_ERR_INVALID_ARG, "fit_model_info: null argument");
    info->n_params = model->n_params;
    info->n_data = model->n_data;
    info->n_datasets = model->n_ds;
    info->n_true = model->n_true;
    info->device_bytes = model->bytes;
    return FIT_OK;
}

int fit_model_params(const fit_model *model, double *theta0, double *prior_sigma) {
    if (!model) return fail(FIT_ERR_INVALID_ARG, "fit_model_params: null model");
    if (theta0) std::copy(model->theta0.begin(), model->theta0.end(), theta0);
    if (prior_sigma) std::copy(model->sigma.begin(), model->sigma.end(), prior_sigma);
    return FIT_OK;
}

const char *fit_model_param_name(const fit_model *model, int i) {
    if (!model || i < 0 || i >= (int)model->names.size()) return nullptr;
    return model->names[i].c_str();
}

static int launch_eval(fit_model *model, int B, const double *theta_d, const float *data_d,
                       const uint32_t *masks_d, double *nll_d, float *grad_d, float *mu_d,
                       int *st_d, cudaStream_t s);

int fit_model_create(const fit_model_desc *d, fit_model **out) {
    using std::vector;
    if (!d || !out) return fail(FIT_ERR_INVALID_ARG, "fit_model_create: null argument");
    *out = nullptr;
    const int P = d->n_params, Nt = d->n_true, C = d->n_cores;
    auto bad = [](const std::string &m) { return fail(FIT_ERR_INVALID_CONFIG, "fit_model_create: " + m); };
    if (P < 1 || P > FIT_MAX_PARAMS) return bad("n_params out of range");
    if (Nt < 2 || Nt > FIT_MAX_TRUE_BINS) return bad("n_true out of range");
    if (C < 1 || C > FIT_MAX_CORES) return bad("n_cores out of range");
    if (d->n_det < 1 || d->n_det > FIT_MAX_DETECTORS) return bad("n_det out of range");
    if (d->n_ds < 1 || d->n_ds > FIT_MAX_DATASETS) return bad("n_ds out of range");
    if (d->n_bkg < 0 || d->n_bkg > FIT_MAX_BACKGROUNDS) return bad("n_bkg out of range");
    if (d->osc_mode != FIT_OSC_EQ1 && d->osc_mode != FIT_OSC_VACUUM3 && d->osc_mode != FIT_OSC_STERILE4)
        return bad("osc_mode");
    const int n_osc = d->osc_mode == FIT_OSC_STERILE4 ? 6 : 4;
    if (d->remap_mode != FIT_REMAP_OVERLAP && d->remap_mode != FIT_REMAP_SPLINE) return bad("remap_mode");
    if (!(d->e_lo > 0.0 && d->e_hi > d->e_lo) || !std::isfinite(d->e_hi)) return bad("energy grid");
    if (!d->theta0 || !d->prior_sigma || !d->scale || !d->core_power_idx || !d->det_n_reco ||
        !d->det_response || !d->ds_det || !d->ds_t || !d->ds_baseline || !d->ds_weight ||
        !d->ds_norm_idx || !d->ds_eff_idx || !d->ds_escale_idx || !d->ds_shape_idx)
        return bad("missing array");
    if (d->n_cov > 0 && (!d->cov_size || !d->cov_idx || !d->cov)) return bad("missing covariance arrays");
    if (d->n_bkg > 0 && (!d->bkg_ds || !d->bkg_template || !d->bkg_rate_idx || !d->bkg_shape_idx))
        return bad("missing background arrays");
    auto pidx_ok = [P](int i) { return i >= -1 && i < P; };
    for (int i = 0; i < P; ++i)
        if (!std::isfinite(d->theta0[i])) return bad("theta0 entries must be finite");
    for (int i = 0; i < n_osc; ++i) {
        if (!pidx_ok(d->osc_idx[i])) return bad("osc_idx");
        if (d->osc_idx[i] < 0 && !std::isfinite(d->osc_val[i])) return bad("osc_val entries must be finite");
    }
    if (n_osc == 6 && d->osc_idx[4] < 0 && !(d->osc_val[4] >= 0.0 && d->osc_val[4] < 1.0))
        return bad("sin^2 2th14 outside [0, 1)");
    for (int c = 0; c < C; ++c)
        if (!pidx_ok(d->core_power_idx[c])) return bad("core_power_idx");
    for (int i = 0; i < d->n_det; ++i)
        if (d->det_n_reco[i] < 1 || d->det_n_reco[i] > FIT_MAX_RECO_BINS) return bad("det_n_reco");

    fit_model *M = new fit_model();
    DevModel &h = M->host;
    std::memset(&h, 0, sizeof(DevModel));
    Arena A;
    h.P = P;
    h.N_t = Nt;
    h.C = C;
    h.n_ds = d->n_ds;
    h.osc_mode = d->osc_mode;
    const double de = (d->e_hi - d->e_lo) / Nt;
    h.e_lo = (float)d->e_lo;
    h.de = (float)de;
    h.inv_de = (float)(1.0 / de);
    h.n_osc = n_osc;
    h.remap_mode = d->remap_mode;
    for (int i = 0; i < fitcore::kMaxOsc; ++i) {
        const double v = i < n_osc ? d->osc_val[i] : 0.0;
        h.osc_idx[i] = i < n_osc ? d->osc_idx[i] : -1;
        h.osc_val[i] = (float)v;
        h.osc_val_lo[i] = (float)(v - (double)h.osc_val[i]);
        h.osc_val_d[i] = v;
    }
    for (int c = 0; c < C; ++c) h.core_power_idx[c] = d->core_power_idx[c];
    {
        vector<float> edge(Nt + 1), ih(Nt), il(Nt);
        for (int k = 0; k <= Nt; ++k) edge[k] = (float)(d->e_lo + k * de);
        for (int k = 0; k < Nt; ++k) {
            const double inv = 1.0 / (d->e_lo + (k + 0.5) * de);
            ih[k] = (float)inv;
            il[k] = (float)(inv - (double)ih[k]);
        }
        A.put(&h.e_edge, edge);
        A.put(&h.inv_e_hi, ih);
        A.put(&h.inv_e_lo, il);
    }
    // ---- detectors: banded response -------------------------------------------------------
    vector<int> det_off(d->n_det + 1, 0);
    for (int i = 0; i < d->n_det; ++i) det_off[i + 1] = det_off[i] + d->det_n_reco[i] * Nt;
    int max_reco = 0;
    for (int i = 0; i < d->n_det; ++i) {
        const int nr = d->det_n_reco[i];
        max_reco = std::max(max_reco, nr);
        const double *R = d->det_response + det_off[i];
        vector<int> rlo(nr), rlen(nr), roff(nr);
        vector<float> rrow;
        for (int j = 0; j < nr; ++j) {
            int a = Nt, b = -1;
            for (int k = 0; k < Nt; ++k) {
                const double x = R[(size_t)j * Nt + k];
                if (!std::isfinite(x) || x < 0.0) {
                    delete M;
                    return bad("response entries must be finite and >= 0");
                }
                if (x != 0.0) {
                    a = std::min(a, k);
                    b = std::max(b, k);
                }
            }
            if (b < a) a = b = 0;   // empty row: one zero entry
            rlo[j] = a;
            rlen[j] = b - a + 1;
            roff[j] = (int)rrow.size();
            for (int k = a; k <= b; ++k) rrow.push_back((float)R[(size_t)j * Nt + k]);
            while (rrow.size() % 4) rrow.push_back(0.f);
        }
        vector<int> clo(Nt), clen(Nt);
        int cw = 1;
        for (int k = 0; k < Nt; ++k) {
            int a = nr, b = -1;
            for (int j = 0; j < nr; ++j)
                if (R[(size_t)j * Nt + k] != 0.0) {
                    a = std::min(a, j);
                    b = std::max(b, j);
                }
            if (b < a) a = b = 0;
            clo[k] = a;
            clen[k] = b - a + 1;
            cw = std::max(cw, b - a + 1);
        }
        vector<float> rcol((size_t)cw * Nt, 0.f);
        for (int k = 0; k < Nt; ++k)
            for (int b = 0; b < cw && clo[k] + b < nr; ++b)
                rcol[(size_t)b * Nt + k] = (float)R[(size_t)(clo[k] + b) * Nt + k];
        fitcore::DevDetector &dt = h.det[i];
        dt.n_reco = nr;
        dt.col_w = cw;
        A.put(&dt.row_lo, rlo);
        A.put(&dt.row_len, rlen);
        A.put(&dt.row_off, roff);
        A.put(&dt.rrow, rrow);
        A.put(&dt.col_lo, clo);
        A.put(&dt.col_len, clen);
        A.put(&dt.rcol, rcol);
        // dense copy for the tensor-core fold, split into a TF32-exact high part and the rest
        const int ldt = (Nt + 3) / 4 * 4;
        vector<float> rhi((size_t)nr * ldt, 0.f), rlow((size_t)nr * ldt, 0.f);
        for (int j = 0; j < nr; ++j)
            for (int k = 0; k < Nt; ++k) {
                const float x = (float)R[(size_t)j * Nt + k];
                uint32_t bits;
                std::memcpy(&bits, &x, 4);
                bits = (bits + 0x1000u) & 0xFFFFE000u;   // nearest value with 10 mantissa bits
                float hi;
                std::memcpy(&hi, &bits, 4);
                rhi[(size_t)j * ldt + k] = hi;
                rlow[(size_t)j * ldt + k] = x - hi;
            }
        A.put(&dt.rdense_hi, rhi);
        A.put(&dt.rdense_lo, rlow);
        // and its transpose [N_t x ldr] for the adjoint fold G R on the tensor cores
        const int ldr = (nr + 3) / 4 * 4;
        vector<float> thi((size_t)Nt * ldr, 0.f), tlo((size_t)Nt * ldr, 0.f);
        for (int j = 0; j < nr; ++j)
            for (int k = 0; k < Nt; ++k) {
                thi[(size_t)k * ldr + j] = rhi[(size_t)j * ldt + k];
                tlo[(size_t)k * ldr + j] = rlow[(size_t)j * ldt + k];
            }
        dt.ldr = ldr;
        A.put(&dt.rdt_hi, thi);
        A.put(&dt.rdt_lo, tlo);
    }
    h.max_reco = max_reco;
    // ---- datasets -------------------------------------------------------------------------
    int data_off = 0;
    vector<int> bkg_order;
    for (int ds = 0; ds < d->n_ds; ++ds) {
        fitcore::DevDataset &D = h.ds[ds];
        const int det = d->ds_det[ds];
        if (det < 0 || det >= d->n_det) {
            delete M;
            return bad("ds_det");
        }
        D.det = det;
        D.n_reco = d->det_n_reco[det];
        D.data_off = data_off;
        data_off += D.n_reco;
        D.norm_idx = d->ds_norm_idx[ds];
        D.eff_idx = d->ds_eff_idx[ds];
        if (!pidx_ok(D.norm_idx) || !pidx_ok(D.eff_idx)) {
            delete M;
            return bad("ds_norm_idx / ds_eff_idx");
        }
        for (int i = 0; i < 3; ++i) {
            D.esc_idx[i] = d->ds_escale_idx[3 * ds + i];
            if (!pidx_ok(D.esc_idx[i])) {
                delete M;
                return bad("ds_escale_idx");
            }
        }
        D.a1_off = D.esc_idx[1] >= 0 ? (float)(d->theta0[D.esc_idx[1]] - 1.0) : 0.f;
        for (int c = 0; c < C; ++c) {
            const double w = d->ds_weight[ds * C + c], L = d->ds_baseline[ds * C + c];
            if (!(w >= 0.0) || !std::isfinite(w) || (w > 0.0 && !(L > 0.0 && std::isfinite(L)))) {
                delete M;
                return bad("ds_weight / ds_baseline");
            }
            D.w[c] = (float)w;
            const double kl = kOscK * L / M_PI;   // phase per (dm2 / E) in half-turns
            D.kl_hi[c] = (float)kl;
            D.kl_lo[c] = (float)(kl - (double)D.kl_hi[c]);
        }
        vector<float> t(Nt);
        vector<int> sidx(Nt);
        for (int k = 0; k < Nt; ++k) {
            t[k] = (float)d->ds_t[(size_t)ds * Nt + k];
            sidx[k] = d->ds_shape_idx[(size_t)ds * Nt + k];
            if (!pidx_ok(sidx[k]) || !(t[k] >= 0.f) || !std::isfinite(t[k])) {
                delete M;
                return bad("ds_t / ds_shape_idx");
            }
        }
        // CSR of true bins per distinct shape parameter
        vector<int> params;
        for (int k = 0; k < Nt; ++k)
            if (sidx[k] >= 0) params.push_back(sidx[k]);
        std::sort(params.begin(), params.end());
        params.erase(std::unique(params.begin(), params.end()), params.end());
        vector<int> ptr(params.size() + 1, 0), ks;
        for (size_t q = 0; q < params.size(); ++q) {
            for (int k = 0; k < Nt; ++k)
                if (sidx[k] == params[q]) ks.push_back(k);
            ptr[q + 1] = (int)ks.size();
        }
        D.n_sp = (int)params.size();
        A.put(&D.t, t);
        A.put(&D.shape_idx, sidx);
        A.put(&D.sp_param, params);
        A.put(&D.sp_ptr, ptr);
        A.put(&D.sp_k, ks);
        // backgrounds of this dataset, in description order
        D.bkg_begin = (int)bkg_order.size();
        for (int b = 0; b < d->n_bkg; ++b)
            if (d->bkg_ds[b] == ds) bkg_order.push_back(b);
        D.bkg_end = (int)bkg_order.size();
        if (D.bkg_end - D.bkg_begin > fitcore::kMaxBkgDs) {
            delete M;
            return bad("more than 6 backgrounds in one dataset");
        }
    }
    h.n_data = data_off;
    {
        vector<int> boff(d->n_bkg + 1, 0);
        for (int b = 0; b < d->n_bkg; ++b) {
            if (d->bkg_ds[b] < 0 || d->bkg_ds[b] >= d->n_ds) {
                delete M;
                return bad("bkg_ds");
            }
            boff[b + 1] = boff[b] + d->det_n_reco[d->ds_det[d->bkg_ds[b]]];
        }
        h.n_bkg = d->n_bkg;
        for (size_t q = 0; q < bkg_order.size(); ++q) {
            const int b = bkg_order[q];
            const int nr = boff[b + 1] - boff[b];
            vector<float> tm(nr);
            vector<int> si(nr);
            for (int j = 0; j < nr; ++j) {
                tm[j] = (float)d->bkg_template[boff[b] + j];
                si[j] = d->bkg_shape_idx[boff[b] + j];
                if (!pidx_ok(si[j])) {
                    delete M;
                    return bad("bkg_shape_idx");
                }
                if (!(tm[j] >= 0.f) || !std::isfinite(tm[j])) {
                    delete M;
                    return bad("bkg_template entries must be finite and >= 0");
                }
            }
            if (!pidx_ok(d->bkg_rate_idx[b])) {
                delete M;
                return bad("bkg_rate_idx");
            }
            h.bkg[q].rate_idx = d->bkg_rate_idx[b];
            A.put(&h.bkg[q].tmpl, tm);
            A.put(&h.bkg[q].shape_idx, si);
        }
    }
    // ---- parameters, priors, transformation layer ----------------------------------------
    {
        vector<double> th0(d->theta0, d->theta0 + P);
        vector<float> th0f(P), th0lo(P), zscale(P, 0.f), pinv(P, 0.f);
        vector<int> in_block(P, 0);
        vector<int> bsz, boff, bidx;
        vector<int64_t> moff;
        vector<float> Lf, Wf;
        vector<double> L64;
        int64_t mo = 0;
        for (int b = 0, ioff = 0; b < d->n_cov; ++b) {
            const int n = d->cov_size[b];
            if (n < 1 || ioff + n > P * 4) {
                delete M;
                return bad("cov_size");
            }
            const int *idx = d->cov_idx + ioff;
            for (int i = 0; i < n; ++i) {
                if (idx[i] < 0 || idx[i] >= P || in_block[idx[i]] || d->prior_sigma[idx[i]] != 0.0) {
                    delete M;
                    return bad("cov_idx: a parameter is out of range, in two blocks, or also has prior_sigma");
                }
                in_block[idx[i]] = 1;
            }
            const double *V = d->cov + mo / 2;   // blocks are packed m*m back to back
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < i; ++j)
                    if (std::fabs(V[(size_t)i * n + j] - V[(size_t)j * n + i]) >
                        1e-12 * (std::fabs(V[(size_t)i * n + i]) + std::fabs(V[(size_t)j * n + j]))) {
                        delete M;
                        return fail(FIT_ERR_NON_SPD_COV, "fit_model_create: covariance block not symmetric");
                    }
            vector<double> L, W;
            if (!cholesky_lower(n, V, L)) {
                delete M;
                return fail(FIT_ERR_NON_SPD_COV, "fit_model_create: covariance block not positive definite");
            }
            lower_inverse(n, L, W);
            bsz.push_back(n);
            boff.push_back(ioff);
            for (int i = 0; i < n; ++i) bidx.push_back(idx[i]);
            moff.push_back(mo);
            // [L | L^T] and [W | W^T], dense row-major
            const size_t base = Lf.size();
            Lf.resize(base + 2 * (size_t)n * n);
            Wf.resize(base + 2 * (size_t)n * n);
            L64.resize(base + 2 * (size_t)n * n);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    Lf[base + (size_t)i * n + j] = (float)L[(size_t)i * n + j];
                    Lf[base + (size_t)n * n + (size_t)j * n + i] = (float)L[(size_t)i * n + j];
                    Wf[base + (size_t)i * n + j] = (float)W[(size_t)i * n + j];
                    Wf[base + (size_t)n * n + (size_t)j * n + i] = (float)W[(size_t)i * n + j];
                    L64[base + (size_t)i * n + j] = L[(size_t)i * n + j];
                }
            mo += 2 * (int64_t)n * n;
            ioff += n;
        }
        for (int i = 0; i < P; ++i) {
            th0f[i] = (float)th0[i];
            th0lo[i] = (float)(th0[i] - (double)th0f[i]);
            if (in_block[i]) continue;
            const double ps = d->prior_sigma[i], sc = d->scale[i];
            if (ps < 0.0 || !std::isfinite(ps)) {
                delete M;
                return bad("prior_sigma");
            }
            if (ps > 0.0) {
                zscale[i] = (float)ps;
                pinv[i] = (float)(1.0 / ps);
            } else {
                if (!(sc > 0.0) || !std::isfinite(sc)) {
                    delete M;
                    return bad("scale must be > 0 for a parameter without prior");
                }
                zscale[i] = (float)sc;
            }
        }
        h.n_blocks = d->n_cov;
        A.put(&h.theta0, th0);
        A.put(&h.theta0_f, th0f);
        A.put(&h.theta0_lo, th0lo);
        A.put(&h.zscale, zscale);
        A.put(&h.prior_inv, pinv);
        if (bsz.empty()) {
            bsz.push_back(0);
            boff.push_back(0);
            bidx.push_back(0);
            moff.push_back(0);
            Lf.push_back(0.f);
            Wf.push_back(0.f);
            L64.push_back(0.0);
        }
        A.put(&h.blk_size, bsz);
        A.put(&h.blk_idx_off, boff);
        A.put(&h.blk_idx, bidx);
        vector<int> bfirst(bsz.size(), -1);
        for (size_t b = 0; b < bsz.size(); ++b) {
            bool contig = bsz[b] > 0;
            for (int i = 1; i < bsz[b] && contig; ++i) contig = bidx[boff[b] + i] == bidx[boff[b]] + i;
            if (contig) bfirst[b] = bidx[boff[b]];
        }
        A.put(&h.blk_first, bfirst);
        M->in_block.assign(in_block.begin(), in_block.end());
        M->theta0 = th0;
        M->sigma.assign(d->prior_sigma, d->prior_sigma + P);
        for (int b = 0, q = 0, mo = 0; b < d->n_cov; mo += d->cov_size[b] * d->cov_size[b], q += d->cov_size[b], ++b)
            for (int i = 0; i < d->cov_size[b]; ++i)
                M->sigma[d->cov_idx[q + i]] = std::sqrt(d->cov[mo + i * d->cov_size[b] + i]);
        M->zscale.assign(P, 0.0);
        for (int i = 0; i < P; ++i)
            if (!in_block[i]) M->zscale[i] = d->prior_sigma[i] > 0.0 ? d->prior_sigma[i] : d->scale[i];
        for (int b = 0; b < d->n_cov; ++b) {
            const int n = bsz[b];
            M->bsz.push_back(n);
            for (int i = 0; i < n; ++i) M->bidx.push_back(bidx[boff[b] + i]);
            for (int64_t q = 0; q < (int64_t)n * n; ++q) M->blk_L.push_back(L64[moff[b] + q]);
        }
        A.put(&h.blk_mat_off, moff);
        A.put(&h.blk_L, Lf);
        A.put(&h.blk_W, Wf);
        A.put(&h.blk_L64, L64);
    }
    {
        vector<float> asimov(h.n_data, 0.f);
        A.put(&h.asimov, asimov);
        vector<int> slot_ds(h.n_data, 0);
        for (int ds = 0; ds < h.n_ds; ++ds)
            for (int j = 0; j < h.ds[ds].n_reco; ++j) slot_ds[h.ds[ds].data_off + j] = ds;
        A.put(&h.slot_ds, slot_ds);
    }
    h.ws_eval_floats = fitcore::eval_ws_floats(Nt, C, max_reco, n_osc);
    h.ldt = (Nt + 3) / 4 * 4;

    // ---- upload ---------------------------------------------------------------------------
    cudaError_t e = cudaMalloc(&M->arena, A.buf.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete M;
        return fail(FIT_ERR_OOM, std::string("fit_model_create: cudaMalloc: ") + cudaGetErrorString(e));
    }
    A.bind(M->arena);
    e = cudaMemcpy(M->arena, A.buf.data(), A.buf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&M->dev, sizeof(DevModel));
    if (e == cudaSuccess) e = cudaMemcpy(M->dev, &h, sizeof(DevModel), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fit_model_destroy(M);
        return fail(FIT_ERR_CUDA, std::string("fit_model_create: upload: ") + cudaGetErrorString(e));
    }
    M->bytes = A.buf.size() + sizeof(DevModel);
    if (cudaGetDevice(&M->device) != cudaSuccess) {
        cudaGetLastError();
        fit_model_destroy(M);
        return fail(FIT_ERR_CUDA, "fit_model_create: cudaGetDevice");
    }
    M->n_params = P;
    M->n_data = h.n_data;
    M->n_ds = h.n_ds;
    M->n_true = Nt;
    // Asimov data = expectation at theta0
    {
        double *th = nullptr;
        int rc = FIT_OK;
        if (cudaMalloc(&th, sizeof(double) * P) != cudaSuccess ||
            cudaMemcpy(th, d->theta0, sizeof(double) * P, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = fail(FIT_ERR_CUDA, "fit_model_create: asimov staging");
        if (rc == FIT_OK)
            rc = launch_eval(M, 1, th, nullptr, nullptr, nullptr, nullptr,
                             const_cast<float *>(h.asimov), nullptr, 0);
        if (rc == FIT_OK && cudaDeviceSynchronize() != cudaSuccess)
            rc = fail(FIT_ERR_CUDA, "fit_model_create: asimov evaluation");
        if (th) cudaFree(th);
        if (rc != FIT_OK) {
            cudaGetLastError();
            fit_model_destroy(M);
            return rc;
        }
    }
    *out = M;
    return FIT_OK;
}

// one block per parameter vector (grid-strided), workspace in shared memory when small
static int launch_eval(fit_model *model, int B, const double *theta_d, const float *data_d,
                       const uint32_t *masks_d, double *nll_d, float *grad_d, float *mu_d,
                       int *st_d, cudaStream_t s) {
    LaunchCfg cfg;
    int rc = device_cfg(cfg);
    if (rc) return rc;
    const DevModel &h = model->host;
    const int threads = 256;
    bool in_smem = fitcore::eval_smem_bytes(h, true) <= 96 * 1024;
    size_t smem = fitcore::eval_smem_bytes(h, in_smem);
    rc = fitcore_raise_eval_smem(std::min(smem, cfg.smem_optin));
    if (rc) return rc;
    int per_sm = 0;
    FIT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fitcore::eval_kernel, threads, smem));
    if (per_sm < 1) return fail(FIT_ERR_INVALID_CONFIG, "fit_model_eval: model too large for one block");
    const int grid = std::max(1, std::min(B, per_sm * cfg.sms));
    float *ws = nullptr;
    if (!in_smem) FIT_CUDA(cudaMallocAsync(&ws, sizeof(float) * (size_t)grid * h.ws_eval_floats, s));
    fitcore::eval_kernel<<<grid, threads, smem, s>>>(model->dev, B, theta_d, data_d, masks_d, nll_d,
                                                     grad_d, mu_d, st_d, ws, in_smem ? 1 : 0);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (ws) cudaFreeAsync(ws, s);
    if (e != cudaSuccess) return fail(FIT_ERR_CUDA, std::string("eval_kernel launch: ") + cudaGetErrorString(e));
    return FIT_OK;
}

int fit_model_expected(fit_model *model, int B, const double *theta, float *mu_out, int *status_out,
                       void *stream) {
    if (!model || !theta || !mu_out || B < 0) return fail(FIT_ERR_INVALID_ARG, "fit_model_expected: bad argument");
    if (B == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t P = model->n_params, D = model->n_data;
    Staged th, mu, st;
    bool hmu = false, hst = false;
    int rc = stage_in(theta, sizeof(double) * P * B, s, th);
    if (!rc) rc = stage_out(mu_out, sizeof(float) * D * B, s, mu, hmu);
    if (!rc) rc = stage_out(status_out, sizeof(int) * B, s, st, hst);
    if (!rc) rc = launch_eval(model, B, (const double *)th.dev, nullptr, nullptr, nullptr, nullptr,
                              (float *)mu.dev, (int *)st.dev, s);
    if (!rc && hmu) rc = cudaMemcpyAsync(mu_out, mu.dev, sizeof(float) * D * B, cudaMemcpyDeviceToHost, s)
                             ? fail(FIT_ERR_CUDA, "fit_model_expected: copy back") : FIT_OK;
    if (!rc && hst) rc = cudaMemcpyAsync(status_out, st.dev, sizeof(int) * B, cudaMemcpyDeviceToHost, s)
                             ? fail(FIT_ERR_CUDA, "fit_model_expected: copy back") : FIT_OK;
    release(th, s);
    release(mu, s);
    release(st, s);
    if (!rc && (hmu || hst) && cudaStreamSynchronize(s) != cudaSuccess)
        rc = fail(FIT_ERR_CUDA, "fit_model_expected: synchronise");
    return rc;
}

int fit_model_eval(fit_model *model, int B, const double *theta, const float *data, const uint32_t *masks,
                   double *nll_out, float *grad_out, int *status_out, void *stream) {
    if (!model || !theta || !nll_out || B < 0) return fail(FIT_ERR_INVALID_ARG, "fit_model_eval: bad argument");
    if (B == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t P = model->n_params, D = model->n_data;
    Staged th, da, mk, nl, gr, st;
    bool hnl = false, hgr = false, hst = false;
    int rc = stage_in(theta, sizeof(double) * P * B, s, th);
    if (!rc) rc = stage_in(data, sizeof(float) * D * B, s, da);
    if (!rc) rc = stage_in(masks, sizeof(uint32_t) * B, s, mk);
    if (!rc) rc = stage_out(nll_out, sizeof(double) * B, s, nl, hnl);
    if (!rc) rc = stage_out(grad_out, sizeof(float) * P * B, s, gr, hgr);
    if (!rc) rc = stage_out(status_out, sizeof(int) * B, s, st, hst);
    if (!rc) rc = launch_eval(model, B, (const double *)th.dev, (const float *)da.dev, (const uint32_t *)mk.dev,
                              (double *)nl.dev, (float *)gr.dev, nullptr, (int *)st.dev, s);
    if (!rc && hnl && cudaMemcpyAsync(nll_out, nl.dev, sizeof(double) * B, cudaMemcpyDeviceToHost, s))
        rc = fail(FIT_ERR_CUDA, "fit_model_eval: copy back");
    if (!rc && hgr && cudaMemcpyAsync(grad_out, gr.dev, sizeof(float) * P * B, cudaMemcpyDeviceToHost, s))
        rc = fail(FIT_ERR_CUDA, "fit_model_eval: copy back");
    if (!rc && hst && cudaMemcpyAsync(status_out, st.dev, sizeof(int) * B, cudaMemcpyDeviceToHost, s))
        rc = fail(FIT_ERR_CUDA, "fit_model_eval: copy back");
    release(th, s);
    release(da, s);
    release(mk, s);
    release(nl, s);
    release(gr, s);
    release(st, s);
    if (!rc && (hnl || hgr || hst) && cudaStreamSynchronize(s) != cudaSuccess)
        rc = fail(FIT_ERR_CUDA, "fit_model_eval: synchronise");
    return rc;
}

int fit_tc_gemm(int tf32, int M, int N, int K, const void *A, int lda, const void *B, int ldb, int epi, float *C,
                int ldc, void *Y, int ldy, const float *bias, const float *aux, int ldaux, void *stream) {
    fitcore::GemmOut o;
    o.epi = epi;
    o.C = C;
    o.ldc = ldc;
    o.Y = static_cast<__nv_bfloat16 *>(Y);
    o.ldy = ldy;
    o.bias = bias;
    o.aux = aux;
    o.ldaux = ldaux;
    if (epi < fitcore::EPI_F32 || epi > fitcore::EPI_F32_ADD) return fail(FIT_ERR_INVALID_ARG, "fit_tc_gemm: epilogue");
    const bool needC = epi != fitcore::EPI_DGELU, needY = epi == fitcore::EPI_BIAS_GELU || epi == fitcore::EPI_DGELU;
    if ((needC && !C) || (needY && !Y) || ((epi == fitcore::EPI_BIAS_F32 || epi == fitcore::EPI_BIAS_GELU) && !bias) ||
        (epi == fitcore::EPI_DGELU && !aux))
        return fail(FIT_ERR_INVALID_ARG, "fit_tc_gemm: missing output for the epilogue");
    return fitcore::tc_gemm(tf32 != 0, M, N, K, A, lda, B, ldb, o, (cudaStream_t)stream, nullptr);
}

int fit_tc_gemm_status(void) { return fitcore::tc_gemm_take_error(); }

int fit_model_expected_tc(fit_model *model, int B, const double *theta, float *mu_out, int *status_out, int precision,
                          void *stream) {
    if (!model || !theta || !mu_out || B < 0 || (precision != 0 && precision != 1))
        return fail(FIT_ERR_INVALID_ARG, "fit_model_expected_tc: bad argument");
    if (B == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t P = model->n_params, D = model->n_data;
    Staged th, mu, st;
    bool hmu = false, hst = false;
    int rc = stage_in(theta, sizeof(double) * P * B, s, th);
    if (!rc) rc = stage_out(mu_out, sizeof(float) * D * B, s, mu, hmu);
    if (!rc) {
        if (status_out) {
            rc = stage_out(status_out, sizeof(int) * B, s, st, hst);
        } else {
            if (cudaMallocAsync(&st.dev, sizeof(int) * B, s)) rc = fail(FIT_ERR_OOM, "fit_model_expected_tc: status");
            st.owned = true;
        }
    }
    if (!rc) rc = fitcore::expected_tc(model->host, model->dev, B, (const double *)th.dev, (float *)mu.dev,
                                       (int *)st.dev, precision, s);
    if (!rc && hmu && cudaMemcpyAsync(mu_out, mu.dev, sizeof(float) * D * B, cudaMemcpyDeviceToHost, s))
        rc = fail(FIT_ERR_CUDA, "fit_model_expected_tc: copy back");
    if (!rc && hst && cudaMemcpyAsync(status_out, st.dev, sizeof(int) * B, cudaMemcpyDeviceToHost, s))
        rc = fail(FIT_ERR_CUDA, "fit_model_expected_tc: copy back");
    release(th, s);
    release(mu, s);
    release(st, s);
    if (!rc && (hmu || hst) && cudaStreamSynchronize(s) != cudaSuccess) rc = fail(FIT_ERR_CUDA, "fit_model_expected_tc: sync");
    return rc;
}

int fit_poisson_sample(int64_t n, const float *mu, uint64_t seed, uint64_t offset, float *out, void *stream) {
    if (n < 0 || (n > 0 && (!mu || !out))) return fail(FIT_ERR_INVALID_ARG, "fit_poisson_sample: bad argument");
    if (n == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Staged a, b;
    bool hb = false;
    int rc = stage_in(mu, sizeof(float) * n, s, a);
    if (!rc) rc = stage_out(out, sizeof(float) * n, s, b, hb);
    if (!rc) rc = fitcore::poisson_sample(n, (const float *)a.dev, seed, offset, (float *)b.dev, s);
    if (!rc && hb && cudaMemcpyAsync(out, b.dev, sizeof(float) * n, cudaMemcpyDeviceToHost, s))
        rc = fail(FIT_ERR_CUDA, "fit_poisson_sample: copy back");
    release(a, s);
    release(b, s);
    if (!rc && hb && cudaStreamSynchronize(s) != cudaSuccess) rc = fail(FIT_ERR_CUDA, "fit_poisson_sample: sync");
    return rc;
}

int fit_warmstart_features(const fit_model *model, int B, const float *data, const uint32_t *masks, int n_in,
                           int slot0, int onehot_slot, float *x, void *stream) {
    if (!model || !data || !x || B < 0 || n_in < 1 || slot0 < 0 || slot0 + model->n_data > n_in ||
        onehot_slot >= n_in || (onehot_slot >= slot0 && onehot_slot < slot0 + model->n_data))
        return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_features: bad argument");
    if (B == 0) return FIT_OK;
    if (!on_device(data) || !on_device(x) || (masks && !on_device(masks)))
        return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_features: device buffers");
    return fitcore::features(B, model->n_data, data, model->host.asimov, masks, model->host.slot_ds, nullptr, n_in,
                             slot0, onehot_slot, x, (cudaStream_t)stream);
}

int fit_warmstart_predict(fit_mlp *mlp, const fit_model *model, int B, const float *data, const uint32_t *masks,
                          int slot0, int onehot_slot, int n_targets, const int *target_idx,
                          const double *target_scale, double *theta_out, void *stream) {
    int n_in = 0, n_out = 0;
    if (!mlp || !model || !data || !theta_out || !target_idx || !target_scale || B < 0)
        return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_predict: bad argument");
    fitcore::mlp_dims(mlp, &n_in, &n_out);
    if (n_targets < 1 || n_targets > n_out) return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_predict: n_targets");
    for (int t = 0; t < n_targets; ++t)
        if (target_idx[t] < 0 || target_idx[t] >= model->n_params || !(target_scale[t] > 0.0))
            return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_predict: target index or scale");
    if (B == 0) return FIT_OK;
    if (!on_device(data) || !on_device(theta_out) || (masks && !on_device(masks)))
        return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_predict: device buffers");
    cudaStream_t s = (cudaStream_t)stream;
    float *x = fitcore::mlp_input_buffer(mlp, B);
    if (!x) return fail(FIT_ERR_OOM, "fit_warmstart_predict: input buffer");
    // the linearised best fit of every parameter (the model's cached rows are logically part of
    // the constant model), then the network's corrections on its targets
    int rc = fit_linear_start(const_cast<fit_model *>(model), B, data, masks, theta_out, stream);
    if (!rc) rc = fit_warmstart_features(model, B, data, masks, n_in, slot0, onehot_slot, x, stream);
    float *out = nullptr;
    int *idx = nullptr;
    double *scl = nullptr;
    if (!rc && (cudaMallocAsync(&out, sizeof(float) * (size_t)B * n_out, s) ||
                cudaMallocAsync(&idx, sizeof(int) * n_targets, s) || cudaMallocAsync(&scl, sizeof(double) * n_targets, s)))
        rc = fail(FIT_ERR_OOM, "fit_warmstart_predict: workspace");
    if (!rc && (cudaMemcpyAsync(idx, target_idx, sizeof(int) * n_targets, cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(scl, target_scale, sizeof(double) * n_targets, cudaMemcpyHostToDevice, s)))
        rc = fail(FIT_ERR_CUDA, "fit_warmstart_predict: upload");
    if (!rc) rc = fit_mlp_forward(mlp, B, x, out, stream);
    if (!rc)
        rc = fitcore::starts(B, model->n_params, model->host.theta0, n_targets, idx, scl, out, n_out, theta_out,
                             theta_out, s);
    for (void *p : {(void *)out, (void *)idx, (void *)scl})
        if (p) cudaFreeAsync(p, s);
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = fail(FIT_ERR_CUDA, "fit_warmstart_predict: sync");
    return rc;
}

namespace {

int check_geom(const fit_model *m, const fit_warmstart_geom *g, int n_in, int n_out) {
    if (!g || g->n_targets < 1 || g->n_targets > FIT_WS_MAX_TARGETS || g->n_targets > n_out || g->n_uniform < 0 ||
        g->n_uniform > FIT_WS_MAX_TARGETS || g->n_masks < 0 || g->n_masks > FIT_WS_MAX_MASKS || g->slot0 < 0 ||
        g->slot0 + m->n_data > n_in || g->onehot_slot >= n_in ||
        (g->onehot_slot >= g->slot0 && g->onehot_slot < g->slot0 + m->n_data))
        return fail(FIT_ERR_INVALID_ARG, "warm start: bad geometry description");
    for (int t = 0; t < g->n_targets; ++t)
        if (g->target_idx[t] < 0 || g->target_idx[t] >= m->n_params || !(g->target_scale[t] > 0.0))
            return fail(FIT_ERR_INVALID_ARG, "warm start: target index or scale");
    for (int t = 0; t < g->n_uniform; ++t)
        if (g->uniform_idx[t] < 0 || g->uniform_idx[t] >= m->n_params || !(g->uniform_half[t] >= 0.0))
            return fail(FIT_ERR_INVALID_ARG, "warm start: uniform index or half-width");
    return FIT_OK;
}

// device copy of one geometry's index and scale tables
struct GeomDev {
    int *tidx = nullptr, *uidx = nullptr;
    double *tscale = nullptr, *uhalf = nullptr;
    uint32_t *choices = nullptr;
};

int upload_geom(const fit_warmstart_geom &g, GeomDev &d, cudaStream_t s) {
    if (cudaMallocAsync(&d.tidx, sizeof(int) * FIT_WS_MAX_TARGETS, s) ||
        cudaMallocAsync(&d.uidx, sizeof(int) * FIT_WS_MAX_TARGETS, s) ||
        cudaMallocAsync(&d.tscale, sizeof(double) * FIT_WS_MAX_TARGETS, s) ||
        cudaMallocAsync(&d.uhalf, sizeof(double) * FIT_WS_MAX_TARGETS, s) ||
        cudaMallocAsync(&d.choices, sizeof(uint32_t) * FIT_WS_MAX_MASKS, s))
        return fail(FIT_ERR_OOM, "warm start: geometry tables");
    if (cudaMemcpyAsync(d.tidx, g.target_idx, sizeof(int) * FIT_WS_MAX_TARGETS, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d.uidx, g.uniform_idx, sizeof(int) * FIT_WS_MAX_TARGETS, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d.tscale, g.target_scale, sizeof(double) * FIT_WS_MAX_TARGETS, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d.uhalf, g.uniform_half, sizeof(double) * FIT_WS_MAX_TARGETS, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d.choices, g.masks, sizeof(uint32_t) * FIT_WS_MAX_MASKS, cudaMemcpyHostToDevice, s))
        return fail(FIT_ERR_CUDA, "warm start: geometry upload");
    return FIT_OK;
}

void free_geom(GeomDev &d, cudaStream_t s) {
    for (void *p : {(void *)d.tidx, (void *)d.uidx, (void *)d.tscale, (void *)d.uhalf, (void *)d.choices})
        if (p) cudaFreeAsync(p, s);
    d = GeomDev();
}

}  // namespace

int fit_warmstart_draw(fit_model *model, const fit_warmstart_geom *geom, int B, uint64_t seed, uint64_t offset,
                       double *theta_out, uint32_t *masks_out, void *stream) {
    if (!model || !geom || B < 0 || !theta_out) return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_draw: bad argument");
    int rc = check_geom(model, geom, 1 << 30, FIT_WS_MAX_TARGETS);
    if (rc) return rc;
    if (B == 0) return FIT_OK;
    if (!on_device(theta_out) || (masks_out && !on_device(masks_out)))
        return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_draw: device buffers");
    cudaStream_t s = (cudaStream_t)stream;
    GeomDev gd;
    rc = upload_geom(*geom, gd, s);
    if (!rc) rc = fitcore::draw_theta(model->host, model->dev, B, seed, offset, geom->n_uniform, gd.uidx, gd.uhalf,
                                      geom->n_masks, gd.choices, theta_out, masks_out, s);
    free_geom(gd, s);
    return rc;
}

}  // extern "C"

namespace {

void theta_of_z_host(const fit_model *M, const double *z, double *th);
const fit_model::LinEntry *lin_entry(fit_model *M, uint32_t mask, cudaStream_t s, int &rc);

// Rows of the linearised maximum-likelihood step for the targets of a warm-start geometry, per
// dataset-mask variant v: with J = d mu / d z at the nominal point (central differences of the
// device expectation), W = diag(1 / mu0) over the variant's bins and Lambda = 1 on the
// constrained coordinates, the step from a drawn point z_t is (J^T W J + Lambda)^-1 (J^T W
// (n - mu_t) - Lambda z_t). Row p of that inverse (p = target t's parameter) gives K1[v][t] =
// (A^-1 J^T W)_p [D], K2[v][t] = (A^-1 Lambda)_p [P] and zf[v][t] = zscale_p / scale_t.
// Refresh of the mass-splitting columns (free survival parameters whose Jacobian turns with the
// oscillation phase): with J_o taken at each drawn point instead of the nominal one, the step
// splits by the Schur complement of the fixed block n = (all other parameters) of
// A = J^T W J + Lambda: with N = A_nn,
//   S = J_o^T Gp J_o + Lambda_o,  Gp = W - W J_n N^-1 J_n^T W   (symmetric, D x D)
//   delta_o = S^-1 (J_o^T (Gp r + H z_n) - Lambda_o z_o),  H = W J_n N^-1 Lambda_n (D x P_n)
//   delta_n = N^-1 J_n^T W (r - J_o delta_o) - N^-1 Lambda_n z_n   (rows of the targets only)
// Per variant: Gp [D x D], H^T [P_n x D], R1 = (N^-1 J_n^T W)_T [T_n x D], R2 = (N^-1 Lambda_n)_T
// [T_n x P_n]; per target t: tkind[t] = q >= 0 (the q-th refreshed column) or -1 - row.
struct WsRefresh {
    int k = 0;                         // refreshed columns (0: none)
    std::vector<int> o_param, n_param; // parameter indices of the two blocks
    std::vector<int> tkind;            // per target
    std::vector<float> lam_o;          // Lambda of the refreshed coordinates
    std::vector<float> buf;            // per variant: Gp | H^T | R1 | R2
    size_t var_floats = 0;
    int n_rows = 0;                    // T_n
};

int linear_mle_rows(fit_model *M, const fit_warmstart_geom &G, cudaStream_t s, std::vector<float> &K1,
                    std::vector<float> &K2, std::vector<float> &zf, int &n_var, WsRefresh *ref = nullptr) {
    const int P = M->n_params, D = M->n_data, nt = G.n_targets;
    const double hz = 1e-2;
    const int R = 2 * P + 1;
    std::vector<double> th((size_t)R * P), z(P, 0.0);
    for (int q = 0; q < R; ++q) {
        std::fill(z.begin(), z.end(), 0.0);
        if (q > 0) z[(q - 1) / 2] = (q % 2) ? hz : -hz;
        theta_of_z_host(M, z.data(), th.data() + (size_t)q * P);
    }
    std::vector<float> mu((size_t)R * D);
    std::vector<int> st(R, 0);
    int rc = fit_model_expected(M, R, th.data(), mu.data(), st.data(), s);
    if (rc) return rc;
    for (int q = 0; q < R; ++q)
        if (st[q] != 0) return fail(FIT_ERR_INVALID_CONFIG, "warm start: expectation near the nominal point failed");
    std::vector<double> J((size_t)D * P);
    for (int j = 0; j < D; ++j)
        for (int i = 0; i < P; ++i)
            J[(size_t)j * P + i] =
                ((double)mu[(size_t)(2 * i + 1) * D + j] - (double)mu[(size_t)(2 * i + 2) * D + j]) / (2.0 * hz);
    std::vector<double> con(P);
    for (int i = 0; i < P; ++i) con[i] = (M->sigma[i] > 0.0 || M->in_block[i]) ? 1.0 : 0.0;
    n_var = std::max(1, G.n_masks);
    K1.assign((size_t)n_var * nt * D, 0.f);
    K2.assign((size_t)n_var * nt * P, 0.f);
    zf.assign((size_t)n_var * nt, 0.f);
    std::vector<double> w(D), A((size_t)P * P), L, x(P), y(P);
    if (ref) {
        *ref = WsRefresh();
        std::vector<char> is_o(P, 0);
        for (int i = 0; i < M->host.n_osc; ++i) {
            const int p = M->host.osc_idx[i];
            if (p >= 0 && fitcore::osc_is_dm(M->host.osc_mode, i) && !M->in_block[p] && !is_o[p]) {
                is_o[p] = 1;
                ref->o_param.push_back(p);
            }
        }
        for (int i = 0; i < P; ++i)
            if (!is_o[i]) ref->n_param.push_back(i);
        ref->k = (int)ref->o_param.size();
        for (int t = 0; t < nt; ++t) {
            const int p = G.target_idx[t];
            int q = -1;
            for (int a = 0; a < ref->k; ++a)
                if (ref->o_param[a] == p) q = a;
            ref->tkind.push_back(q >= 0 ? q : -1 - ref->n_rows);
            if (q < 0) ref->n_rows++;
        }
        for (int a = 0; a < ref->k; ++a) ref->lam_o.push_back((float)con[ref->o_param[a]]);
        const size_t Pn = ref->n_param.size();
        ref->var_floats = (size_t)D * D + Pn * D + (size_t)ref->n_rows * D + (size_t)ref->n_rows * Pn;
        if (ref->k > 0) ref->buf.assign(ref->var_floats * n_var, 0.f);
    }
    for (int v = 0; v < n_var; ++v) {
        const uint32_t mask = G.n_masks > 0 ? G.masks[v] : 0xFFFFFFFFu;
        std::fill(w.begin(), w.end(), 0.0);
        for (int d = 0; d < M->host.n_ds; ++d) {
            if (!((mask >> d) & 1u)) continue;
            const int o = M->host.ds[d].data_off;
            for (int j = 0; j < M->host.ds[d].n_reco; ++j) w[o + j] = mu[o + j] > 0.f ? 1.0 / mu[o + j] : 0.0;
        }
        std::fill(A.begin(), A.end(), 0.0);
        for (int j = 0; j < D; ++j) {
            if (w[j] == 0.0) continue;
            const double *Jj = J.data() + (size_t)j * P;
            for (int a = 0; a < P; ++a) {
                const double ja = Jj[a] * w[j];
                if (ja == 0.0) continue;
                double *Aa = A.data() + (size_t)a * P;
                for (int b = 0; b <= a; ++b) Aa[b] += ja * Jj[b];
            }
        }
        double dmax = 0.0;
        for (int a = 0; a < P; ++a) {
            A[(size_t)a * P + a] += con[a];
            dmax = std::max(dmax, A[(size_t)a * P + a]);
        }
        for (int a = 0; a < P; ++a) {   // a coordinate with neither data nor prior stays put
            double &daa = A[(size_t)a * P + a];
            daa += daa > 1e-9 * dmax ? 1e-12 * dmax : 1.0;
            for (int b = 0; b < a; ++b) A[(size_t)b * P + a] = A[(size_t)a * P + b];
        }
        if (!cholesky_lower(P, A.data(), L))
            return fail(FIT_ERR_INVALID_CONFIG, "warm start: expected Hessian not positive definite");
        for (int t = 0; t < nt; ++t) {
            const int p = G.target_idx[t];
            // A x = e_p: forward then backward substitution with L L^T
            for (int i = 0; i < P; ++i) {
                double acc = (i == p) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) acc -= L[(size_t)i * P + k] * y[k];
                y[i] = acc / L[(size_t)i * P + i];
            }
            for (int i = P - 1; i >= 0; --i) {
                double acc = y[i];
                for (int k = i + 1; k < P; ++k) acc -= L[(size_t)k * P + i] * x[k];
                x[i] = acc / L[(size_t)i * P + i];
            }
            float *k1 = K1.data() + ((size_t)v * nt + t) * D, *k2 = K2.data() + ((size_t)v * nt + t) * P;
            for (int j = 0; j < D; ++j) {
                if (w[j] == 0.0) continue;
                double acc = 0.0;
                const double *Jj = J.data() + (size_t)j * P;
                for (int i = 0; i < P; ++i) acc += x[i] * Jj[i];
                k1[j] = (float)(acc * w[j]);
            }
            for (int i = 0; i < P; ++i) k2[i] = (float)(x[i] * con[i]);
            zf[(size_t)v * nt + t] = (float)(M->zscale[p] / G.target_scale[t]);
        }
        if (ref && ref->k > 0) {
            // N = A_nn (A holds both triangles), its Cholesky factor and inverse
            const std::vector<int> &nx = ref->n_param;
            const int Pn = (int)nx.size();
            std::vector<double> Nm((size_t)Pn * Pn), Ln, Ni((size_t)Pn * Pn, 0.0), col(Pn), tmp(Pn);
            for (int a = 0; a < Pn; ++a)
                for (int b = 0; b < Pn; ++b) Nm[(size_t)a * Pn + b] = A[(size_t)nx[a] * P + nx[b]];
            if (!cholesky_lower(Pn, Nm.data(), Ln))
                return fail(FIT_ERR_INVALID_CONFIG, "warm start: nuisance block not positive definite");
            for (int c = 0; c < Pn; ++c) {   // column c of N^-1
                for (int i = 0; i < Pn; ++i) {
                    double acc = (i == c) ? 1.0 : 0.0;
                    for (int k2i = 0; k2i < i; ++k2i) acc -= Ln[(size_t)i * Pn + k2i] * tmp[k2i];
                    tmp[i] = acc / Ln[(size_t)i * Pn + i];
                }
                for (int i = Pn - 1; i >= 0; --i) {
                    double acc = tmp[i];
                    for (int k2i = i + 1; k2i < Pn; ++k2i) acc -= Ln[(size_t)k2i * Pn + i] * col[k2i];
                    col[i] = acc / Ln[(size_t)i * Pn + i];
                }
                for (int i = 0; i < Pn; ++i) Ni[(size_t)i * Pn + c] = col[i];
            }
            // X = N^-1 J_n^T W [Pn x D]
            std::vector<double> X((size_t)Pn * D, 0.0);
            for (int a = 0; a < Pn; ++a)
                for (int j = 0; j < D; ++j) {
                    if (w[j] == 0.0) continue;
                    double acc = 0.0;
                    for (int b = 0; b < Pn; ++b) acc += Ni[(size_t)a * Pn + b] * J[(size_t)j * P + nx[b]];
                    X[(size_t)a * D + j] = acc * w[j];
                }
            float *base = ref->buf.data() + (size_t)v * ref->var_floats;
            float *Gp = base, *Ht = Gp + (size_t)D * D, *R1 = Ht + (size_t)Pn * D, *R2 = R1 + (size_t)ref->n_rows * D;
            // Gp = W - W J_n X (symmetric)
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) {
                    double acc = 0.0;
                    if (w[i] != 0.0)
                        for (int a = 0; a < Pn; ++a) acc += J[(size_t)i * P + nx[a]] * X[(size_t)a * D + j];
                    Gp[(size_t)i * D + j] = (float)((i == j ? w[i] : 0.0) - w[i] * acc);
                }
            // H^T [Pn x D]: H = W J_n N^-1 Lambda_n
            for (int c = 0; c < Pn; ++c) {
                const double lc = con[nx[c]];
                for (int j = 0; j < D; ++j) {
                    double acc = 0.0;
                    if (lc != 0.0 && w[j] != 0.0)
                        for (int a = 0; a < Pn; ++a) acc += J[(size_t)j * P + nx[a]] * Ni[(size_t)a * Pn + c];
                    Ht[(size_t)c * D + j] = (float)(w[j] * acc * lc);
                }
            }
            // target rows of the n block
            int row = 0;
            for (int t = 0; t < nt; ++t) {
                if (ref->tkind[t] >= 0) continue;
                int a = -1;
                for (int q = 0; q < Pn; ++q)
                    if (nx[q] == G.target_idx[t]) a = q;
                for (int j = 0; j < D; ++j) R1[(size_t)row * D + j] = (float)X[(size_t)a * D + j];
                for (int c = 0; c < Pn; ++c) R2[(size_t)row * Pn + c] = (float)(Ni[(size_t)a * Pn + c] * con[nx[c]]);
                ++row;
            }
        }
    }
    return FIT_OK;
}

}  // namespace

extern "C" {

int fit_warmstart_train(fit_mlp *mlp, fit_model *const *models, const fit_warmstart_geom *geoms, int n_geoms,
                        int n_steps, int batch, float lr, float weight_decay, uint64_t seed, double *losses_out,
                        void *stream) {
    int n_in = 0, n_out = 0;
    if (!mlp || !models || !geoms || n_geoms < 1 || n_geoms > 16 || n_steps < 0 || batch < 1 || !(lr > 0.f))
        return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_train: bad argument");
    fitcore::mlp_dims(mlp, &n_in, &n_out);
    int max_p = 0, max_d = 0;
    for (int g = 0; g < n_geoms; ++g) {
        if (!models[g]) return fail(FIT_ERR_INVALID_ARG, "fit_warmstart_train: null model");
        int rc = check_geom(models[g], &geoms[g], n_in, n_out);
        if (rc) return rc;
        max_p = std::max(max_p, models[g]->n_params);
        max_d = std::max(max_d, models[g]->n_data);
    }
    if (n_steps == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    double *theta = nullptr, *loss = nullptr;
    float *mu = nullptr, *cnt = nullptr, *y = nullptr;
    uint32_t *masks = nullptr;
    int *status = nullptr;
    GeomDev gd[16];
    int rc = FIT_OK;
    if (cudaMallocAsync(&theta, sizeof(double) * (size_t)batch * max_p, s) ||
        cudaMallocAsync(&mu, sizeof(float) * (size_t)batch * max_d, s) ||
        cudaMallocAsync(&cnt, sizeof(float) * (size_t)batch * max_d, s) ||
        cudaMallocAsync(&y, sizeof(float) * (size_t)batch * n_out, s) ||
        cudaMallocAsync(&masks, sizeof(uint32_t) * (size_t)batch, s) ||
        cudaMallocAsync(&status, sizeof(int) * (size_t)batch, s) ||
        cudaMallocAsync(&loss, sizeof(double) * (size_t)n_steps, s))
        rc = fail(FIT_ERR_OOM, "fit_warmstart_train: workspace");
    for (int g = 0; g < n_geoms && !rc; ++g) rc = upload_geom(geoms[g], gd[g], s);
    // linearised maximum-likelihood rows per geometry (targets = where a fit of the sample ends,
    // to first order, rather than the drawn point)
    float *zbuf = nullptr, *krows[16] = {nullptr}, *ktl[16] = {nullptr};
    int n_var[16] = {0};
    // the refreshed mass-splitting columns: device tables per geometry
    WsRefresh refs[16];
    float *rbuf[16] = {nullptr}, *rlam[16] = {nullptr};
    int *rint[16] = {nullptr};   // o_param | n_param | tkind
    double *thp = nullptr;
    float *mup = nullptr;
    int *stp = nullptr;
    int max_k = 0;
    if (!rc && cudaMallocAsync(&zbuf, sizeof(float) * (size_t)batch * max_p, s) != cudaSuccess)
        rc = fail(FIT_ERR_OOM, "fit_warmstart_train: workspace");
    for (int g = 0; g < n_geoms && !rc; ++g) {
        std::vector<float> K1, K2, zf;
        rc = linear_mle_rows(models[g], geoms[g], s, K1, K2, zf, n_var[g], &refs[g]);
        if (rc) break;
        WsRefresh &R = refs[g];
        if (R.k > 3) R.k = 0;   // more than three mass splittings: the nominal-point rows only
        if (R.k > 0) {
            max_k = std::max(max_k, R.k);
            std::vector<int> ints;
            ints.insert(ints.end(), R.o_param.begin(), R.o_param.end());
            ints.insert(ints.end(), R.n_param.begin(), R.n_param.end());
            ints.insert(ints.end(), R.tkind.begin(), R.tkind.end());
            if (cudaMallocAsync(&rbuf[g], sizeof(float) * R.buf.size(), s) != cudaSuccess ||
                cudaMallocAsync(&rlam[g], sizeof(float) * R.lam_o.size(), s) != cudaSuccess ||
                cudaMallocAsync(&rint[g], sizeof(int) * ints.size(), s) != cudaSuccess) {
                rc = fail(FIT_ERR_OOM, "fit_warmstart_train: workspace");
                break;
            }
            if (cudaMemcpyAsync(rbuf[g], R.buf.data(), sizeof(float) * R.buf.size(), cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(rlam[g], R.lam_o.data(), sizeof(float) * R.lam_o.size(), cudaMemcpyHostToDevice, s) ||
                cudaMemcpyAsync(rint[g], ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, s) ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                rc = fail(FIT_ERR_CUDA, "fit_warmstart_train: upload");
                break;
            }
        }
        const size_t n = K1.size() + K2.size() + zf.size();
        if (cudaMallocAsync(&krows[g], sizeof(float) * n, s) != cudaSuccess) {
            rc = fail(FIT_ERR_OOM, "fit_warmstart_train: workspace");
            break;
        }
        std::vector<float> all;
        all.reserve(n);
        all.insert(all.end(), K1.begin(), K1.end());
        all.insert(all.end(), K2.begin(), K2.end());
        all.insert(all.end(), zf.begin(), zf.end());
        if (cudaMemcpyAsync(krows[g], all.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = fail(FIT_ERR_CUDA, "fit_warmstart_train: upload");
        // standardised target rows of the linearised start per dataset subset: the network
        // learns the correction to it
        if (!rc) {
            fit_model *M = models[g];
            const int P = M->n_params, D = M->n_data, Dp = (D + 3) & ~3, nt = geoms[g].n_targets;
            const uint32_t all = (M->n_ds >= 32) ? 0xFFFFFFFFu : ((1u << M->n_ds) - 1u);
            std::vector<float> kt((size_t)n_var[g] * nt * D, 0.f);
            for (int v = 0; v < n_var[g] && !rc; ++v) {
                const uint32_t mk = geoms[g].n_masks > 0 ? (geoms[g].masks[v] & all) : all;
                const fit_model::LinEntry *le = lin_entry(M, mk, s, rc);
                if (!le) break;
                for (int t = 0; t < nt; ++t) {
                    const int p = geoms[g].target_idx[t];
                    const double sc = geoms[g].target_scale[t];
                    for (int j = 0; j < D; ++j)
                        kt[((size_t)v * nt + t) * D + j] = (float)(le->Kh[(size_t)p * Dp + j] / sc);
                }
                (void)P;
            }
            if (!rc && (cudaMallocAsync(&ktl[g], sizeof(float) * kt.size(), s) != cudaSuccess ||
                        cudaMemcpyAsync(ktl[g], kt.data(), sizeof(float) * kt.size(), cudaMemcpyHostToDevice, s) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
                rc = fail(FIT_ERR_OOM, "fit_warmstart_train: linearised rows");
        }
    }
    if (!rc && max_k > 0 &&
        (cudaMallocAsync(&thp, sizeof(double) * (size_t)batch * 2 * max_k * max_p, s) != cudaSuccess ||
         cudaMallocAsync(&mup, sizeof(float) * (size_t)batch * 2 * max_k * max_d, s) != cudaSuccess ||
         cudaMallocAsync(&stp, sizeof(int) * (size_t)batch * 2 * max_k, s) != cudaSuccess))
        rc = fail(FIT_ERR_OOM, "fit_warmstart_train: workspace");
    float *x = rc ? nullptr : fitcore::mlp_input_buffer(mlp, batch);
    if (!rc && !x) rc = fail(FIT_ERR_OOM, "fit_warmstart_train: input buffer");
    for (int step = 0; step < n_steps && !rc; ++step) {
        const int g = step % n_geoms;
        const fit_model *m = models[g];
        const fit_warmstart_geom &G = geoms[g];
        // per-step streams of the generator: theta/masks under seed, counts under a derived key
        const uint64_t off = (uint64_t)step * (uint64_t)batch;
        const uint64_t pseed = seed ^ 0xA5A5A5A55A5A5A5Aull;
        const float lr_s = lr * (float)(0.05 + 0.95 * 0.5 * (1.0 + std::cos(M_PI * step / n_steps)));
        rc = fitcore::draw_theta(m->host, m->dev, batch, seed, off, G.n_uniform, gd[g].uidx, gd[g].uhalf, G.n_masks,
                                 gd[g].choices, theta, masks, s, zbuf);
        if (!rc) rc = fitcore::expected_tc(m->host, m->dev, batch, theta, mu, status, 0, s);
        if (!rc) rc = fitcore::poisson_sample((int64_t)batch * m->n_data, mu, pseed, off * (uint64_t)m->n_data, cnt, s);
        if (!rc) rc = fitcore::features(batch, m->n_data, cnt, m->host.asimov, G.n_masks > 0 ? masks : nullptr,
                                        m->host.slot_ds, status, n_in, G.slot0, G.onehot_slot, x, s);
        if (!rc) {
            const int P = m->n_params, D = m->n_data, nt = G.n_targets, nv = n_var[g];
            const float *K1 = krows[g], *K2 = K1 + (size_t)nv * nt * D, *zf = K2 + (size_t)nv * nt * P;
            const WsRefresh &R = refs[g];
            if (R.k > 0) {
                // the mass-splitting columns of J at each drawn point (split-TF32 expectations)
                const double hz = 1e-2;
                const int Pn = (int)R.n_param.size();
                rc = fitcore::perturb_theta(batch, P, R.k, theta, rint[g], m->host.zscale, hz, thp, s);
                if (!rc) rc = fitcore::expected_tc(m->host, m->dev, batch * 2 * R.k, thp, mup, stp, 1, s);
                if (!rc)
                    rc = fitcore::refresh_targets(batch, P, D, R.k, Pn, R.n_rows, theta, m->host.theta0, zbuf, cnt, mu,
                                                  mup, stp, rint[g], rint[g] + R.k, rint[g] + R.k + Pn, rlam[g],
                                                  rbuf[g], (int64_t)R.var_floats, hz, nt, gd[g].tidx, gd[g].tscale, zf,
                                                  nv, gd[g].choices, masks, n_out, status, y, s);
            } else {
                rc = fitcore::mle_targets(batch, P, D, theta, m->host.theta0, zbuf, cnt, mu, nt, gd[g].tidx,
                                          gd[g].tscale, K1, K2, zf, nv, gd[g].choices, masks, n_out, status, y, s);
            }
        }
        if (!rc)
            rc = fitcore::lin_residual_targets(batch, m->n_data, G.n_targets, ktl[g], m->lin_mu0, cnt, n_var[g],
                                               gd[g].choices, masks, n_out, status, y, s);
        if (!rc) rc = fit_mlp_train_step(mlp, batch, x, y, lr_s, weight_decay, loss + step, stream);
    }
    if (!rc && losses_out &&
        cudaMemcpyAsync(losses_out, loss, sizeof(double) * (size_t)n_steps, cudaMemcpyDefault, s) != cudaSuccess)
        rc = fail(FIT_ERR_CUDA, "fit_warmstart_train: losses");
    for (int g = 0; g < n_geoms; ++g) {
        free_geom(gd[g], s);
        for (void *p : {(void *)krows[g], (void *)ktl[g], (void *)rbuf[g], (void *)rlam[g], (void *)rint[g]})
            if (p) cudaFreeAsync(p, s);
    }
    for (void *p : {(void *)thp, (void *)mup, (void *)stp})
        if (p) cudaFreeAsync(p, s);
    for (void *p : {(void *)theta, (void *)mu, (void *)cnt, (void *)y, (void *)masks, (void *)status, (void *)loss,
                    (void *)zbuf})
        if (p) cudaFreeAsync(p, s);
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = fail(FIT_ERR_CUDA, "fit_warmstart_train: sync");
    return rc;
}

}  // extern "C"

namespace {

// One instantiated graph per launch shape: a memset node (work queue = 0) followed by the fit
// kernel node. A call with the same shape updates both nodes' parameters in the executable
// graph and relaunches it, which skips the per-launch driver work of a plain launch.
struct FitGraph {
    const void *func = nullptr;
    int grid = 0, threads = 0;
    size_t smem = 0;
    int device = -1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t memset_node = nullptr, kernel_node = nullptr;
};
std::vector<FitGraph> g_graphs;   // guarded by g_ws_mutex (held by fit_batch)

int graph_launch(const void *kern, int grid, int threads, size_t smem, fitcore::FitArgs &a,
                 int *queue, cudaStream_t s) {
    int dev = 0;
    FIT_CUDA(cudaGetDevice(&dev));
    cudaMemsetParams mp = {};
    mp.dst = queue;
    mp.value = 0;
    mp.elementSize = sizeof(int);
    mp.width = 1;
    mp.height = 1;
    mp.pitch = 0;
    void *args[] = {&a};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void *>(kern);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(threads);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    FitGraph *G = nullptr;
    for (auto &g : g_graphs)
        if (g.func == kern && g.grid == grid && g.threads == threads && g.smem == smem && g.device == dev)
            G = &g;
    if (G) {
        if (cudaGraphExecMemsetNodeSetParams(G->exec, G->memset_node, &mp) != cudaSuccess ||
            cudaGraphExecKernelNodeSetParams(G->exec, G->kernel_node, &kp) != cudaSuccess) {
            cudaGetLastError();
            return fail(FIT_ERR_CUDA, "fit_batch: graph update");
        }
    } else {
        FitGraph g;
        g.func = kern;
        g.grid = grid;
        g.threads = threads;
        g.smem = smem;
        g.device = dev;
        if (cudaGraphCreate(&g.graph, 0) != cudaSuccess ||
            cudaGraphAddMemsetNode(&g.memset_node, g.graph, nullptr, 0, &mp) != cudaSuccess ||
            cudaGraphAddKernelNode(&g.kernel_node, g.graph, &g.memset_node, 1, &kp) != cudaSuccess ||
            cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess) {
            cudaGetLastError();
            if (g.graph) cudaGraphDestroy(g.graph);
            return fail(FIT_ERR_CUDA, "fit_batch: graph construction");
        }
        g_graphs.push_back(g);
        G = &g_graphs.back();
    }
    if (cudaGraphLaunch(G->exec, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(FIT_ERR_CUDA, "fit_batch: graph launch");
    }
    return FIT_OK;
}

// Lockstep engine driver: per model, the instances of that model advance together; each round
// is the forward, adjoint and step launches over the active ones. The host reads the number
// still active after every round (a 4-byte copy) to size the next launches and to stop.
int fit_batch_lockstep(fit_model *const *models, int n_models, const fit_instance *inst, int n_inst,
                       const float *data, const double *start, const uint8_t *fixed, double *best,
                       fit_result *results, const fit_batch_opts &o, cudaStream_t s, int64_t data_len,
                       int64_t par_len, bool precond, bool tc) {
    LaunchCfg cfg;
    int rc = device_cfg(cfg);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    Staged di, dd, dst, dfx, dbe, dre;
    bool hbe = false, hre = false;
    rc = stage_in(inst, sizeof(fit_instance) * n_inst, s, di);
    if (!rc) rc = stage_in(data, sizeof(float) * data_len, s, dd);
    if (!rc && start) rc = stage_in(start, sizeof(double) * par_len, s, dst);
    if (!rc && fixed) rc = stage_in(fixed, (size_t)par_len, s, dfx);
    if (!rc) rc = stage_out(best, sizeof(double) * par_len, s, dbe, hbe);
    if (!rc) rc = stage_out(results, sizeof(fit_result) * n_inst, s, dre, hre);
    int *cnt_host = nullptr;
    if (!rc && cudaMallocHost(&cnt_host, sizeof(int)) != cudaSuccess) rc = fail(FIT_ERR_OOM, "fit_batch: pinned counter");
    for (int mi = 0; mi < n_models && !rc; ++mi) {
        std::vector<int> grp;
        for (int i = 0; i < n_inst; ++i)
            if (inst[i].model == mi) grp.push_back(i);
        if (grp.empty()) continue;
        const DevModel &h = models[mi]->host;
        const int n = (int)grp.size(), P = h.P, nd = h.n_ds;
        fitcore::LsArgs A{};
        A.model = models[mi]->dev;
        A.inst = (const fit_instance *)di.dev;
        A.n = n;
        A.data = (const float *)dd.dev;
        A.start = start ? (const double *)dst.dev : nullptr;
        A.fixed = fixed ? (const uint8_t *)dfx.dev : nullptr;
        A.best = (double *)dbe.dev;
        A.results = (fit_result *)dre.dev;
        A.vec_stride = ((int64_t)fitcore::fit_vec_floats(P, o.history) + 3) / 4 * 4;
        A.hist = o.history;
        A.max_iter = o.max_iter;
        A.max_ls = 8;
        A.restarts = o.restarts;
        A.edm_tol = o.edm_tol;
        A.f_noise_rel = o.f_noise_rel;
        A.budget_ns = (uint64_t)(o.time_budget_s * 1e9);
        A.precond = precond && models[mi]->pre_state == 1 ? 1 : 0;
        // evaluation workspace: the adjoint needs the full per-dataset arrays (engine 2: one
        // per (active instance, dataset) pair in global memory, kept for the round)
        const int ws_floats = h.ws_eval_floats;
        const size_t eval_smem = fitcore::ls_eval_smem_bytes(P, ws_floats);
        A.ws_in_smem = !tc && eval_smem <= 48 * 1024 ? 1 : 0;
        const size_t esm = A.ws_in_smem ? eval_smem : fitcore::ls_eval_smem_bytes(P, 0);
        const size_t ssm = fitcore::ls_step_smem_bytes();
        // the general builds of the evaluation kernels (3+1 formula, spline correction)
        const bool six = h.n_osc == 6 || h.remap_mode == FIT_REMAP_SPLINE;
        const void *kf = six ? (const void *)fitcore::ls_forward_kernel6 : (const void *)fitcore::ls_forward_kernel;
        const void *ka = six ? (const void *)fitcore::ls_adjoint_kernel6 : (const void *)fitcore::ls_adjoint_kernel;
        const void *kl = nullptr;
        if (tc) {
            kf = six ? (const void *)fitcore::ls_tc_fwd_kernel6 : (const void *)fitcore::ls_tc_fwd_kernel;
            kl = six ? (const void *)fitcore::ls_tc_lik_kernel6 : (const void *)fitcore::ls_tc_lik_kernel;
            ka = six ? (const void *)fitcore::ls_tc_adj_kernel6 : (const void *)fitcore::ls_tc_adj_kernel;
        }
        int per_sm_f = 0, per_sm_a = 0, per_sm_s = 0, per_sm_l = 0;
        for (const void *k : {kf, ka, kl})
            if (k && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm) != cudaSuccess)
                rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep shared memory");
        if (!rc && kl && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_l, kl, 128, esm) || per_sm_l < 1))
            rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep occupancy");
        for (const void *k : {(const void *)fitcore::ls_step_kernel, (const void *)fitcore::ls_init_kernel})
            if (!rc && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm) != cudaSuccess)
                rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep shared memory");
        if (!rc && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, kf, 128, esm) ||
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, ka, 128, esm) ||
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, fitcore::ls_step_kernel, 128, ssm)))
            rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep occupancy");
        if (!rc && (per_sm_f < 1 || per_sm_a < 1 || per_sm_s < 1))
            rc = fail(FIT_ERR_INVALID_CONFIG, "fit_batch: lockstep kernels do not fit an SM");
        if (rc) break;
        const int cap_f = per_sm_f * cfg.sms, cap_a = per_sm_a * cfg.sms, cap_s = per_sm_s * cfg.sms,
                  cap_l = per_sm_l * cfg.sms;
        A.ws_stride = A.ws_in_smem ? 0 : ws_floats;
        std::vector<void *> bufs;
        auto al = [&](void **p, size_t bytes) {
            if (rc) return;
            if (cudaMallocAsync(p, std::max<size_t>(bytes, 16), s) != cudaSuccess) {
                cudaGetLastError();
                rc = fail(FIT_ERR_OOM, "fit_batch: lockstep buffers");
                return;
            }
            bufs.push_back(*p);
        };
        int *grp_d = nullptr, *act0 = nullptr, *act1 = nullptr, *cnt = nullptr, *stat = nullptr;
        uint64_t *deadline = nullptr;
        al((void **)&grp_d, sizeof(int) * n);
        al((void **)&A.state, fitcore::ls_state_bytes() * n);
        al((void **)&A.vec, sizeof(float) * (size_t)n * A.vec_stride);
        al((void **)&A.gsl, sizeof(float) * (size_t)n * nd * P);
        al((void **)&A.nll_ds, sizeof(double) * (size_t)n * nd);
        al((void **)&A.gmu, sizeof(float) * (size_t)n * nd * h.max_reco);
        al((void **)&stat, sizeof(int) * n);
        al((void **)&act0, sizeof(int) * n);
        al((void **)&act1, sizeof(int) * n);
        al((void **)&cnt, sizeof(int) * 2);
        al((void **)&deadline, sizeof(uint64_t));
        if (tc) {
            // per (active instance, dataset) workspace and the GEMM operands per dataset
            A.ldf = (h.max_reco + 3) / 4 * 4;
            A.ldr = A.ldf;
            const size_t rows = (size_t)nd * n;
            al((void **)&A.ws_global, sizeof(float) * rows * ws_floats);
            al((void **)&A.vhi, sizeof(float) * rows * h.ldt);
            al((void **)&A.vlo, sizeof(float) * rows * h.ldt);
            al((void **)&A.fbuf, sizeof(float) * rows * A.ldf);
            al((void **)&A.ghi, sizeof(float) * rows * A.ldr);
            al((void **)&A.glo, sizeof(float) * rows * A.ldr);
            al((void **)&A.gvbuf, sizeof(float) * rows * h.ldt);
            // rows of datasets an instance does not fit are still multiplied: keep them finite
            for (float *p : {A.vhi, A.vlo})
                if (!rc && cudaMemsetAsync(p, 0, sizeof(float) * rows * h.ldt, s) != cudaSuccess)
                    rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep clear");
            for (float *p : {A.ghi, A.glo})
                if (!rc && cudaMemsetAsync(p, 0, sizeof(float) * rows * A.ldr, s) != cudaSuccess)
                    rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep clear");
        } else if (!A.ws_in_smem) {
            al((void **)&A.ws_global, sizeof(float) * (size_t)std::max(cap_f, cap_a) * ws_floats);
        }
        if (!rc && cudaMemcpyAsync(grp_d, grp.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
            rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep upload");
        A.group = grp_d;
        A.stat = stat;
        A.deadline = deadline;
        int *acts[2] = {act0, act1};
        if (!rc) {
            A.act = act1;
            A.n_act = cnt + 1;
            A.act_next = act0;
            A.n_act_next = cnt;
            fitcore::ls_init_kernel<<<std::min(n, cap_s), 128, ssm, s>>>(A);
            g_launches++;
            if (cudaGetLastError() != cudaSuccess) rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep init launch");
        }
        int active = n;
        const int max_rounds = o.max_iter * 34 + 64;
        for (int r = 0; !rc && active > 0 && r < max_rounds; ++r) {
            const int cur = r & 1, nxt = cur ^ 1;
            A.act = acts[cur];
            A.n_act = cnt + cur;
            A.act_next = acts[nxt];
            A.n_act_next = cnt + nxt;
            if (cudaMemsetAsync(cnt + nxt, 0, sizeof(int), s) != cudaSuccess) {
                rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep counter");
                break;
            }
            void *largs[] = {&A};
            cudaLaunchKernel(kf, dim3(std::max(1, std::min(active * nd, cap_f))), dim3(128), largs, esm, s);
            if (tc) {
                // F_d = V_d R^T and, after the likelihood, GV_d = G_d R, each as the split
                // product hi hi + hi lo + lo hi (TF32 operands, FP32 accumulation)
                for (int d = 0; d < nd && !rc; ++d) {
                    const fitcore::DevDetector &dt = h.det[h.ds[d].det];
                    const size_t vo = (size_t)d * n * h.ldt;
                    fitcore::GemmOut go;
                    go.C = A.fbuf + (size_t)d * n * A.ldf;
                    go.ldc = A.ldf;
                    go.epi = fitcore::EPI_F32;
                    rc = fitcore::tc_gemm(true, active, dt.n_reco, h.N_t, A.vhi + vo, h.ldt, dt.rdense_hi, h.ldt, go, s,
                                          nullptr);
                    go.epi = fitcore::EPI_F32_ADD;
                    if (!rc)
                        rc = fitcore::tc_gemm(true, active, dt.n_reco, h.N_t, A.vhi + vo, h.ldt, dt.rdense_lo, h.ldt,
                                              go, s, nullptr);
                    if (!rc)
                        rc = fitcore::tc_gemm(true, active, dt.n_reco, h.N_t, A.vlo + vo, h.ldt, dt.rdense_hi, h.ldt,
                                              go, s, nullptr);
                }
                if (rc) break;
                cudaLaunchKernel(kl, dim3(std::max(1, std::min(active * nd, cap_l))), dim3(128), largs, esm, s);
                g_launches++;
                for (int d = 0; d < nd && !rc; ++d) {
                    const fitcore::DevDetector &dt = h.det[h.ds[d].det];
                    const size_t go_ = (size_t)d * n * A.ldr;
                    fitcore::GemmOut go;
                    go.C = A.gvbuf + (size_t)d * n * h.ldt;
                    go.ldc = h.ldt;
                    go.epi = fitcore::EPI_F32;
                    rc = fitcore::tc_gemm(true, active, h.N_t, dt.n_reco, A.ghi + go_, A.ldr, dt.rdt_hi, dt.ldr, go, s,
                                          nullptr);
                    go.epi = fitcore::EPI_F32_ADD;
                    if (!rc)
                        rc = fitcore::tc_gemm(true, active, h.N_t, dt.n_reco, A.ghi + go_, A.ldr, dt.rdt_lo, dt.ldr, go,
                                              s, nullptr);
                    if (!rc)
                        rc = fitcore::tc_gemm(true, active, h.N_t, dt.n_reco, A.glo + go_, A.ldr, dt.rdt_hi, dt.ldr, go,
                                              s, nullptr);
                }
                if (rc) break;
            }
            cudaLaunchKernel(ka, dim3(std::max(1, std::min(active * nd, cap_a))), dim3(128), largs, esm, s);
            fitcore::ls_step_kernel<<<std::max(1, std::min(active, cap_s)), 128, ssm, s>>>(A);
            g_launches += 3;
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(cnt_host, cnt + nxt, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep round");
                break;
            }
            active = *cnt_host;
        }
        if (!rc && active > 0) rc = fail(FIT_ERR_CUDA, "fit_batch: lockstep did not finish");
        for (void *p : bufs) cudaFreeAsync(p, s);
    }
    if (!rc && hbe) {
        std::vector<std::pair<int64_t, int64_t>> iv;
        for (int i = 0; i < n_inst; ++i)
            iv.emplace_back(inst[i].param_off, inst[i].param_off + models[inst[i].model]->n_params);
        std::sort(iv.begin(), iv.end());
        int64_t a = iv[0].first, b = iv[0].second;
        for (size_t q = 1; q <= iv.size() && !rc; ++q) {
            if (q < iv.size() && iv[q].first <= b) {
                b = std::max(b, iv[q].second);
                continue;
            }
            if (cudaMemcpyAsync(best + a, (double *)dbe.dev + a, sizeof(double) * (b - a), cudaMemcpyDeviceToHost, s))
                rc = fail(FIT_ERR_CUDA, "fit_batch: copy back");
            if (q < iv.size()) {
                a = iv[q].first;
                b = iv[q].second;
            }
        }
    }
    if (!rc && hre && cudaMemcpyAsync(results, dre.dev, sizeof(fit_result) * n_inst, cudaMemcpyDeviceToHost, s))
        rc = fail(FIT_ERR_CUDA, "fit_batch: copy back");
    for (Staged *b : {&di, &dd, &dst, &dfx, &dbe, &dre}) release(*b, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = fail(FIT_ERR_CUDA, "fit_batch: synchronise");
    if (cnt_host) cudaFreeHost(cnt_host);
    return rc;
}

// theta = theta0 + J z on the host (single parameters: z times their scale; blocks: L z)
void theta_of_z_host(const fit_model *M, const double *z, double *th) {
    const int P = M->n_params;
    for (int i = 0; i < P; ++i) th[i] = M->theta0[i] + M->zscale[i] * z[i];
    size_t io = 0, lo = 0;
    for (size_t b = 0; b < M->bsz.size(); ++b) {
        const int n = M->bsz[b];
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j <= i; ++j) acc += M->blk_L[lo + (size_t)i * n + j] * z[M->bidx[io + j]];
            th[M->bidx[io + i]] = M->theta0[M->bidx[io + i]] + acc;
        }
        io += n;
        lo += (size_t)n * n;
    }
}

// Eigen-decomposition of a small symmetric matrix A (n x n, row-major, destroyed) by cyclic
// Jacobi rotations; eigenvalues into lam, eigenvectors into the columns of V.
void jacobi_eigen(int n, std::vector<double> &A, std::vector<double> &lam, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double th = 0.5 * (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / apq;
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {   // V <- V J
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

// Fisher preconditioner of the whitened coordinates z (not in the paper). The expected Hessian
// of -2lnL at theta0 over the fitted datasets is H0 = 2 (I + U U^T), U = J^T diag(mu0)^(-1/2) with
// J = d mu / d z (central differences, step 0.01 in z, of the device expectation). Its few
// large eigen-directions (the data constrain ~10-40 combinations; the whitened prior gives 2 I
// elsewhere) are found by subspace iteration on U U^T with a Rayleigh-Ritz step: U U^T ~
// Q diag(lam) Q^T, Q orthonormal P x r, r = min(32, n_data, P). The fit then runs in w,
//   z = T w,  T = I + Q diag(c) Q^T,  c_k = (1 + lam_k)^(-1/2) - 1,
// where the expected Hessian is 2 I along Q and unchanged elsewhere; T is symmetric (the
// gradient maps with the same product) and T^-1 = I + Q diag(c') Q^T, c'_k = (1 + lam_k)^(1/2) - 1.
// Device storage: Q^T as r rows of P floats on the vector pitch, then c and c'. A model whose
// expectation fails keeps pre_state = -1 and fits unpreconditioned. The model's own
// preconditioner covers all its datasets; an instance fitting a subset of them (a dataset
// mask) gets the one of that subset, built from the same J on first use: the expected
// Hessian of data it does not fit would stretch its coordinates in the wrong directions.
// U = J^T diag(mu0)^(-1/2) [P x D] of the model (cached on the host); false if an expectation
// near the nominal point failed.
bool fisher_U(fit_model *M, cudaStream_t s) {
    if (!M->pre_U.empty()) return true;
    const int P = M->n_params, D = M->n_data;
    const double hz = 1e-2;
    const int R = 2 * P + 1;
    std::vector<double> th((size_t)R * P), z(P, 0.0);
    for (int q = 0; q < R; ++q) {
        std::fill(z.begin(), z.end(), 0.0);
        if (q > 0) z[(q - 1) / 2] = (q % 2) ? hz : -hz;
        theta_of_z_host(M, z.data(), th.data() + (size_t)q * P);
    }
    std::vector<float> mu((size_t)R * D);
    std::vector<int> st(R, 0);
    if (fit_model_expected(M, R, th.data(), mu.data(), st.data(), s) != FIT_OK) return false;
    for (int q = 0; q < R; ++q)
        if (st[q] != 0) return false;
    std::vector<double> U((size_t)P * D, 0.0);
    for (int j = 0; j < D; ++j) {
        const double m0 = mu[j];
        if (!(m0 > 0.0)) continue;
        const double w = 1.0 / (2.0 * hz * std::sqrt(m0));
        for (int i = 0; i < P; ++i)
            U[(size_t)i * D + j] = ((double)mu[(size_t)(2 * i + 1) * D + j] - (double)mu[(size_t)(2 * i + 2) * D + j]) * w;
    }
    M->pre_U.swap(U);
    return true;
}

// Rows of the linearised best fit for the datasets selected by `mask` (not in the paper; the
// warm start's deterministic part). Near the nominal point the expectation is mu0 + J z and
// -2lnL (Eq. 9 with the whitened priors of Eq. 6, |z|^2 over the constrained coordinates) is
// to second order, with the expected Hessian, minimised by the Gauss-Newton (Fisher scoring)
// step from z = 0:
//   dz = (J^T W J + Lambda)^-1 J^T W (n - mu0),  W = diag(1/mu0) on the fitted bins,
// Lambda = 1 on the constrained coordinates (individual priors and covariance blocks), 0 on
// the free ones. With U = J^T diag(mu0)^(-1/2) (fisher_U), J^T W J = U_m U_m^T and the column of
// bin j is (U_m U_m^T + Lambda)^-1 U[:, j] / sqrt(mu0_j). theta = theta0 + T dz (T the linear
// transformation layer), so the theta-space rows are T applied to those columns. Device
// buffer [P x D'] (row-major, D' = D rounded up to 4, zero columns for bins not fitted).
bool build_lin_rows(fit_model *M, uint32_t mask, std::vector<float> &K) {
    const int P = M->n_params, D = M->n_data, Dp = (D + 3) & ~3;
    const std::vector<double> &U = M->pre_U;
    std::vector<char> keep(D, 0);
    for (int d = 0; d < M->host.n_ds; ++d)
        if ((mask >> d) & 1u)
            for (int j = 0; j < M->host.ds[d].n_reco; ++j) keep[M->host.ds[d].data_off + j] = 1;
    // H = U_m U_m^T + Lambda (+ a ridge for directions neither data nor priors constrain)
    std::vector<double> H((size_t)P * P, 0.0);
    for (int a = 0; a < P; ++a)
        for (int b = 0; b <= a; ++b) {
            double acc = 0.0;
            for (int j = 0; j < D; ++j)
                if (keep[j]) acc += U[(size_t)a * D + j] * U[(size_t)b * D + j];
            H[(size_t)a * P + b] = H[(size_t)b * P + a] = acc;
        }
    double dmax = 0.0;
    for (int i = 0; i < P; ++i) {
        if (M->sigma[i] > 0.0 || M->in_block[i]) H[(size_t)i * P + i] += 1.0;
        dmax = std::max(dmax, H[(size_t)i * P + i]);
    }
    for (int i = 0; i < P; ++i) H[(size_t)i * P + i] += 1e-9 * dmax;
    // Cholesky H = C C^T (lower, in place)
    for (int j = 0; j < P; ++j) {
        double dj = H[(size_t)j * P + j];
        for (int k = 0; k < j; ++k) dj -= H[(size_t)j * P + k] * H[(size_t)j * P + k];
        if (!(dj > 0.0)) return false;
        const double cj = std::sqrt(dj);
        H[(size_t)j * P + j] = cj;
        for (int i = j + 1; i < P; ++i) {
            double v = H[(size_t)i * P + j];
            for (int k = 0; k < j; ++k) v -= H[(size_t)i * P + k] * H[(size_t)j * P + k];
            H[(size_t)i * P + j] = v / cj;
        }
    }
    K.assign((size_t)P * Dp, 0.f);
    std::vector<double> x(P), th(P);
    for (int j = 0; j < D; ++j) {
        if (!keep[j] || !(M->lin_mu0_host[j] > 0.0)) continue;
        const double is = 1.0 / std::sqrt(M->lin_mu0_host[j]);
        for (int i = 0; i < P; ++i) {   // forward substitution C y = U[:, j] / sqrt(mu0_j)
            double v = U[(size_t)i * D + j] * is;
            for (int k = 0; k < i; ++k) v -= H[(size_t)i * P + k] * x[k];
            x[i] = v / H[(size_t)i * P + i];
        }
        for (int i = P - 1; i >= 0; --i) {   // back substitution C^T x = y
            double v = x[i];
            for (int k = i + 1; k < P; ++k) v -= H[(size_t)k * P + i] * x[k];
            x[i] = v / H[(size_t)i * P + i];
        }
        theta_of_z_host(M, x.data(), th.data());
        for (int i = 0; i < P; ++i) K[(size_t)i * Dp + j] = (float)(th[i] - M->theta0[i]);
    }
    return true;
}

// The nominal expectation (host and device) and the Jacobian factor of the linearised fit.
int lin_base(fit_model *M, cudaStream_t s) {
    if (M->lin_mu0) return FIT_OK;
    const int D = M->n_data;
    std::vector<float> mu(D);
    std::vector<int> st(1, 0);
    int rc = fit_model_expected(M, 1, M->theta0.data(), mu.data(), st.data(), s);
    if (rc) return rc;
    if (st[0] != 0) return fail(FIT_ERR_INVALID_CONFIG, "linearised fit: expectation at theta0 failed");
    if (!fisher_U(M, s)) return fail(FIT_ERR_INVALID_CONFIG, "linearised fit: expectation near theta0 failed");
    float *d = nullptr;
    if (cudaMalloc(&d, sizeof(float) * D) != cudaSuccess ||
        cudaMemcpy(d, mu.data(), sizeof(float) * D, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        if (d) cudaFree(d);
        return fail(FIT_ERR_OOM, "linearised fit: nominal expectation");
    }
    M->lin_mu0_host.assign(mu.begin(), mu.end());
    M->lin_mu0 = d;
    return FIT_OK;
}

// The linearised fit's rows of one dataset subset (built on first use, kept with the model).
// Guarded by the lock of the preconditioner builds, which share the Jacobian factor (fisher_U),
// so that calls from several host threads on one model are safe.
const fit_model::LinEntry *lin_entry(fit_model *M, uint32_t mask, cudaStream_t s, int &rc) {
    std::lock_guard<std::mutex> lock(g_pre_mutex);
    rc = lin_base(M, s);
    if (rc) return nullptr;
    for (auto &le : M->lin)
        if (le.mask == mask) return &le;
    fit_model::LinEntry e;
    e.mask = mask;
    e.K = nullptr;
    if (!build_lin_rows(M, mask, e.Kh)) {
        rc = fail(FIT_ERR_INVALID_CONFIG, "linearised fit: the expected Hessian is not positive definite");
        return nullptr;
    }
    // device copy split for the tensor cores: the nearest TF32 values, then the rest
    std::vector<float> split(2 * e.Kh.size());
    for (size_t i = 0; i < e.Kh.size(); ++i) {
        uint32_t b;
        std::memcpy(&b, &e.Kh[i], 4);
        b = (b + 0x1000u) & 0xFFFFE000u;
        float h;
        std::memcpy(&h, &b, 4);
        split[i] = h;
        split[e.Kh.size() + i] = e.Kh[i] - h;
    }
    if (cudaMalloc(&e.K, sizeof(float) * split.size()) != cudaSuccess ||
        cudaMemcpy(e.K, split.data(), sizeof(float) * split.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        if (e.K) cudaFree(e.K);
        rc = fail(FIT_ERR_OOM, "linearised fit: rows");
        return nullptr;
    }
    M->lin.push_back(std::move(e));
    return &M->lin.back();
}

// Preconditioner of the datasets selected by `mask` (the expected Hessian of the data an
// instance actually fits): U restricted to those datasets' bins, its leading eigen-directions,
// device buffer [Q^T rows | c | c']. Returns nullptr on failure.
float *build_pre_buffer(fit_model *M, uint32_t mask, int &r_out) {
    const int P = M->n_params, D = M->n_data, Pp = fitcore::fit_vec_pitch(P);
    const int r = std::min(fitcore::kMaxPreRank, std::min(D, P));
    std::vector<char> keep(D, 0);
    for (int d = 0; d < M->host.n_ds; ++d)
        if ((mask >> d) & 1u)
            for (int j = 0; j < M->host.ds[d].n_reco; ++j) keep[M->host.ds[d].data_off + j] = 1;
    const std::vector<double> &U = M->pre_U;
    // subspace iteration X <- orth(U U^T X), X [P x r] (column k at X[k * P ...])
    std::vector<double> X((size_t)r * P), Y((size_t)r * P), t((size_t)D);
    uint64_t seed = 0x9e3779b97f4a7c15ull;
    for (auto &x : X) {
        seed ^= seed << 13; seed ^= seed >> 7; seed ^= seed << 17;
        x = (double)(seed >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    auto apply = [&](const double *x, double *y) {   // y = U_mask (U_mask^T x)
        for (int j = 0; j < D; ++j) t[j] = 0.0;
        for (int i = 0; i < P; ++i) {
            const double xi = x[i];
            if (xi == 0.0) continue;
            const double *Ui = U.data() + (size_t)i * D;
            for (int j = 0; j < D; ++j) t[j] += Ui[j] * xi;
        }
        for (int j = 0; j < D; ++j)
            if (!keep[j]) t[j] = 0.0;
        for (int i = 0; i < P; ++i) {
            const double *Ui = U.data() + (size_t)i * D;
            double acc = 0.0;
            for (int j = 0; j < D; ++j) acc += Ui[j] * t[j];
            y[i] = acc;
        }
    };
    auto orth = [&](std::vector<double> &B) {   // modified Gram-Schmidt on the r columns
        for (int k = 0; k < r; ++k) {
            double *bk = B.data() + (size_t)k * P;
            for (int l = 0; l < k; ++l) {
                const double *bl = B.data() + (size_t)l * P;
                double d = 0.0;
                for (int i = 0; i < P; ++i) d += bk[i] * bl[i];
                for (int i = 0; i < P; ++i) bk[i] -= d * bl[i];
            }
            double nn = 0.0;
            for (int i = 0; i < P; ++i) nn += bk[i] * bk[i];
            nn = std::sqrt(nn);
            for (int i = 0; i < P; ++i) bk[i] = nn > 0.0 ? bk[i] / nn : 0.0;
        }
    };
    orth(X);
    for (int it = 0; it < 40; ++it) {
        for (int k = 0; k < r; ++k) apply(X.data() + (size_t)k * P, Y.data() + (size_t)k * P);
        X.swap(Y);
        orth(X);
    }
    // Rayleigh-Ritz: B = X^T U U^T X, B = E diag(lam) E^T, Q = X E
    for (int k = 0; k < r; ++k) apply(X.data() + (size_t)k * P, Y.data() + (size_t)k * P);
    std::vector<double> B((size_t)r * r), lam, E;
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            double d = 0.0;
            for (int i = 0; i < P; ++i) d += X[(size_t)a * P + i] * Y[(size_t)b * P + i];
            B[(size_t)a * r + b] = d;
        }
    for (int a = 0; a < r; ++a)   // symmetrise the rounding
        for (int b = 0; b < a; ++b) B[(size_t)a * r + b] = B[(size_t)b * r + a] = 0.5 * (B[(size_t)a * r + b] + B[(size_t)b * r + a]);
    jacobi_eigen(r, B, lam, E);
    std::vector<float> buf((size_t)r * Pp + 2 * (size_t)r, 0.f);
    for (int k = 0; k < r; ++k) {
        for (int i = 0; i < P; ++i) {
            double q = 0.0;
            for (int a = 0; a < r; ++a) q += X[(size_t)a * P + i] * E[(size_t)a * r + k];
            buf[(size_t)k * Pp + i] = (float)q;
        }
        const double l = std::max(lam[k], 0.0);
        buf[(size_t)r * Pp + k] = (float)(1.0 / std::sqrt(1.0 + l) - 1.0);
        buf[(size_t)r * Pp + r + k] = (float)(std::sqrt(1.0 + l) - 1.0);
    }
    float *dev = nullptr;
    if (cudaMalloc(&dev, sizeof(float) * buf.size()) != cudaSuccess ||
        cudaMemcpy(dev, buf.data(), sizeof(float) * buf.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        if (dev) cudaFree(dev);
        return nullptr;
    }
    r_out = r;
    return dev;
}

int build_preconditioner(fit_model *M, cudaStream_t s) {
    if (M->pre_state != 0) return FIT_OK;
    M->pre_state = -1;
    if (!fisher_U(M, s)) return FIT_OK;
    const int P = M->n_params, Pp = fitcore::fit_vec_pitch(P);
    int r = 0;
    float *dev = build_pre_buffer(M, 0xFFFFFFFFu, r);
    if (!dev) return FIT_OK;
    M->pre = dev;
    M->host.pre_Q = dev;
    M->host.pre_c = dev + (size_t)r * Pp;
    M->host.pre_r = r;
    // the device copy of the model too (the lockstep kernels read it)
    if (cudaMemcpy(M->dev, &M->host, sizeof(DevModel), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        M->host.pre_Q = M->host.pre_c = nullptr;
        M->host.pre_r = 0;
        return FIT_OK;
    }
    M->pre_state = 1;
    return FIT_OK;
}

// The preconditioner of a dataset subset (built on first use and kept with the model); the
// all-datasets one is the model's own. Returns false if it could not be built.
bool pre_for_mask(fit_model *M, uint32_t mask, fitcore::PreEntry &e) {
    const uint32_t all = (1u << M->host.n_ds) - 1u;
    mask &= all;
    const int Pp = fitcore::fit_vec_pitch(M->n_params);
    e.mask = mask;
    if (mask == all) {
        e.Q = M->host.pre_Q;
        e.c = M->host.pre_c;
        e.r = M->host.pre_r;
        return M->pre_state == 1;
    }
    for (auto &pm : M->pre_masks)
        if (pm.mask == mask) {
            e = pm;
            return e.Q != nullptr;
        }
    fitcore::PreEntry n{};
    n.mask = mask;
    int r = 0;
    float *dev = M->pre_U.empty() ? nullptr : build_pre_buffer(M, mask, r);
    if (dev) {
        n.Q = dev;
        n.c = dev + (size_t)r * Pp;
        n.r = r;
    }
    M->pre_masks.push_back(n);
    e = n;
    return dev != nullptr;
}

}  // namespace

extern "C" {

int fit_linear_start(fit_model *model, int B, const float *data, const uint32_t *masks, double *theta_out,
                     void *stream) {
    if (!model || !data || !theta_out || B < 0) return fail(FIT_ERR_INVALID_ARG, "fit_linear_start: bad argument");
    if (B == 0) return FIT_OK;
    if (!on_device(data) || !on_device(theta_out))
        return fail(FIT_ERR_INVALID_ARG, "fit_linear_start: data and theta_out must be device memory");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != model->device)
        return fail(FIT_ERR_INVALID_ARG, "fit_linear_start: the model's device must be current");
    cudaStream_t s = (cudaStream_t)stream;
    fit_model *M = model;
    const int P = M->n_params, D = M->n_data;
    const uint32_t all = (M->n_ds >= 32) ? 0xFFFFFFFFu : ((1u << M->n_ds) - 1u);
    // the instances' dataset subsets (host copy; masks may be host or device memory)
    std::vector<uint32_t> hm((size_t)B, all);
    if (masks) {
        if (cudaMemcpyAsync(hm.data(), masks, sizeof(uint32_t) * (size_t)B, cudaMemcpyDefault, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(FIT_ERR_CUDA, "fit_linear_start: masks");
        for (auto &m : hm) {
            m &= all;
            if (m == 0) return fail(FIT_ERR_INVALID_ARG, "fit_linear_start: an instance fits no dataset");
        }
    }
    std::vector<uint32_t> subsets;
    std::vector<int> sel((size_t)B);
    for (int b = 0; b < B; ++b) {
        int v = (int)(std::find(subsets.begin(), subsets.end(), hm[b]) - subsets.begin());
        if (v == (int)subsets.size()) {
            if (subsets.size() >= 16) return fail(FIT_ERR_INVALID_ARG, "fit_linear_start: more than 16 dataset subsets");
            subsets.push_back(hm[b]);
        }
        sel[b] = v;
    }
    // the rows of each subset (built on first use and kept with the model)
    std::vector<const float *> K(subsets.size(), nullptr);
    for (size_t v = 0; v < subsets.size(); ++v) {
        int rc = FIT_OK;
        const fit_model::LinEntry *le = lin_entry(M, subsets[v], s, rc);
        if (!le) return rc;
        K[v] = le->K;
    }
    int *sel_d = nullptr;
    if (cudaMallocAsync(&sel_d, sizeof(int) * (size_t)B, s) != cudaSuccess ||
        cudaMemcpyAsync(sel_d, sel.data(), sizeof(int) * (size_t)B, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        if (sel_d) cudaFreeAsync(sel_d, s);
        return fail(FIT_ERR_OOM, "fit_linear_start: subset table");
    }
    int rc = fitcore::linear_start_apply(B, P, D, M->host.theta0, M->lin_mu0, data, K.data(), (int)K.size(), sel_d,
                                         theta_out, s);
    cudaFreeAsync(sel_d, s);
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = fail(FIT_ERR_CUDA, "fit_linear_start: synchronise");
    if (!rc && fitcore::tc_gemm_take_error() != 0) rc = fail(FIT_ERR_TIMEOUT, "fit_linear_start: GEMM pipeline wait");
    return rc;
}

void fit_batch_default_opts(fit_batch_opts *o) {
    if (!o) return;
    o->edm_tol = 1e-8;
    o->max_iter = 2000;
    o->history = 32;
    o->f_noise_rel = 1e-6;
    o->threads = 0;
    o->blocks_per_sm = 0;
    o->use_graph = 0;
    o->time_budget_s = 60.0;
    o->restarts = 0;
    o->placement = 0;
    o->engine = 0;
    o->precondition = 1;
}

int fit_batch(fit_model *const *models, int n_models, const fit_instance *inst, int n_inst, const float *data,
              const double *start, double *best, fit_result *results, const fit_batch_opts *opts_in,
              void *stream) {
    return fit_batch_ex(models, n_models, inst, n_inst, data, start, nullptr, best, results, opts_in, stream);
}

int fit_batch_ex(fit_model *const *models, int n_models, const fit_instance *inst, int n_inst, const float *data,
                 const double *start, const uint8_t *fixed, double *best, fit_result *results,
                 const fit_batch_opts *opts_in, void *stream) {
    if (!models || n_models < 1 || !inst || n_inst < 0 || !data || !best || !results)
        return fail(FIT_ERR_INVALID_ARG, "fit_batch: bad argument");
    if (n_inst == 0) return FIT_OK;
    fit_batch_opts o;
    fit_batch_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.history < 1 || o.history > 32) return fail(FIT_ERR_INVALID_ARG, "fit_batch: history must be 1..32");
    if (o.restarts < 0 || o.restarts > 8) return fail(FIT_ERR_INVALID_ARG, "fit_batch: restarts must be 0..8");
    if (o.threads == 0) o.threads = 128;
    if (o.threads < 64 || o.threads > 128 || o.threads % 32)
        return fail(FIT_ERR_INVALID_ARG, "fit_batch: threads must be a multiple of 32 in [64, 128]");
    if (!(o.edm_tol > 0.0) || o.max_iter < 0) return fail(FIT_ERR_INVALID_ARG, "fit_batch: edm_tol / max_iter");
    if (o.time_budget_s <= 0.0) o.time_budget_s = 60.0;
    cudaStream_t s = (cudaStream_t)stream;
    // extents of the flat data / parameter arrays
    int64_t data_len = 0, par_len = 0;
    int max_need = 0;
    for (int i = 0; i < n_inst; ++i) {
        const fit_instance &q = inst[i];
        if (q.model < 0 || q.model >= n_models || !models[q.model] || q.data_off < 0 || q.param_off < 0)
            return fail(FIT_ERR_INVALID_ARG, "fit_batch: instance " + std::to_string(i) + " out of range");
        data_len = std::max<int64_t>(data_len, q.data_off + models[q.model]->n_data);
        par_len = std::max<int64_t>(par_len, q.param_off + models[q.model]->n_params);
    }
    // held parameters: only outside the prior blocks (checked on a host copy)
    std::vector<uint8_t> fixed_h;
    if (fixed) {
        fixed_h.resize(par_len);
        if (cudaMemcpy(fixed_h.data(), fixed, par_len, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            return fail(FIT_ERR_INVALID_ARG, "fit_batch: fixed flags not readable");
        }
        for (int i = 0; i < n_inst; ++i) {
            const fit_model *mm = models[inst[i].model];
            for (int p = 0; p < mm->n_params; ++p)
                if (fixed_h[inst[i].param_off + p] && mm->in_block[p])
                    return fail(FIT_ERR_INVALID_ARG, "fit_batch: parameter " + std::to_string(p) +
                                                         " of a prior block cannot be held fixed");
        }
    }
    if (o.engine == 1 || o.engine == 2) {
        bool pre = o.precondition != 0;
        if (pre) {
            std::lock_guard<std::mutex> plock(g_pre_mutex);
            for (int i = 0; i < n_models; ++i) build_preconditioner(models[i], s);
        }
        return fit_batch_lockstep(models, n_models, inst, n_inst, data, start, fixed, best, results, o, s,
                                  data_len, par_len, pre, o.engine == 2);
    }
    if (o.engine != 0) return fail(FIT_ERR_INVALID_ARG, "fit_batch: engine must be 0, 1 or 2");
    int max_loc = 0;   // working vectors + evaluation workspace, without the history
    int n_osc = 4;     // the general build when any model uses the 3+1 formula or the spline
    for (int mi = 0; mi < n_models; ++mi) {
        const DevModel &h = models[mi]->host;
        n_osc = std::max(n_osc, h.remap_mode == FIT_REMAP_SPLINE ? 6 : h.n_osc);
        // (multiples of 4 floats: the fit vectors start on 16-byte boundaries)
        const int ws4 = (h.ws_eval_floats + 3) & ~3;
        max_need = std::max(max_need, fitcore::fit_vec_floats(h.P, o.history) + ws4);
        max_loc = std::max(max_loc, fitcore::fit_work_floats(h.P) + ws4);
    }
    if (o.placement < 0 || o.placement > 3) return fail(FIT_ERR_INVALID_ARG, "fit_batch: placement must be 0..3");
    LaunchCfg cfg;
    int rc = device_cfg(cfg);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    // Workspace placement and kernel variant (resident blocks per SM the registers allow).
    // Shared memory holds what fits in ~1/2 of an SM's share; the automatic choice takes the
    // combination with the most resident fits per SM (ties: more in shared memory).
    const size_t kSmemCap = 112 * 1024;
    auto smem_for = [&](int pl) -> size_t {
        if (pl == 1) return fitcore::fit_smem_bytes(max_need);
        if (pl == 2) return fitcore::fit_smem_bytes(max_loc);
        return fitcore::fit_smem_bytes(0);
    };
    // the preconditioned build when asked for and every model has its preconditioner
    bool precond = o.precondition != 0;
    std::vector<fitcore::PreEntry> pre_tab;   // [n_models x pre_k]: dataset-subset preconditioners
    int pre_k = 0;
    if (precond) {
        std::lock_guard<std::mutex> plock(g_pre_mutex);
        for (int i = 0; i < n_models; ++i) {
            build_preconditioner(models[i], s);
            precond = precond && models[i]->pre_state == 1;
        }
        if (precond) {
            // the distinct dataset subsets each model's instances fit (up to 8 per model; an
            // instance whose subset has no entry uses the all-datasets preconditioner)
            constexpr int kMaxSubsets = 8;
            std::vector<std::vector<uint32_t>> subsets(n_models);
            for (int i = 0; i < n_inst; ++i) {
                const fit_model *mm = models[inst[i].model];
                const uint32_t all = (1u << mm->host.n_ds) - 1u, mk = inst[i].mask & all;
                auto &v = subsets[inst[i].model];
                if (mk != all && (int)v.size() < kMaxSubsets && std::find(v.begin(), v.end(), mk) == v.end())
                    v.push_back(mk);
            }
            for (auto &v : subsets) pre_k = std::max(pre_k, (int)v.size());
            if (pre_k > 0) {
                pre_tab.assign((size_t)n_models * pre_k, fitcore::PreEntry{});
                for (int mi = 0; mi < n_models; ++mi)
                    for (size_t q = 0; q < subsets[mi].size(); ++q) {
                        fitcore::PreEntry e{};
                        if (pre_for_mask(models[mi], subsets[mi][q], e)) pre_tab[(size_t)mi * pre_k + q] = e;
                    }
            }
        }
    }
    auto kernel_for = [n_osc, precond](int variant) { return fitcore::fit_kernel_func(variant, n_osc, precond); };
    auto blocks_for = [&](int pl, int variant) -> int {
        const size_t sm = smem_for(pl);
        if (sm > std::min(kSmemCap, cfg.smem_optin)) return 0;
        auto k = kernel_for(variant);
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, o.threads, sm) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return n;
    };
    int placement = o.placement, variant = o.blocks_per_sm >= 5 ? 5 : 4;
    if (placement == 0) {
        int best_n = -1;
        for (int pl : {1, 2, 3}) {
            const int v = o.blocks_per_sm > 0 ? variant : (pl == 3 ? 5 : 4);
            const int n = blocks_for(pl, v);
            if (n > best_n) {
                best_n = n;
                placement = pl;
                variant = v;
            }
        }
    } else if (o.blocks_per_sm == 0) {
        variant = placement == 3 ? 5 : 4;
    }
    if (blocks_for(placement, variant) < 1)
        return fail(FIT_ERR_INVALID_CONFIG, "fit_batch: the requested workspace placement does not fit an SM");
    const bool in_smem = placement == 1;
    const size_t smem = smem_for(placement);
    auto kern = kernel_for(variant);
    FIT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::min(smem, cfg.smem_optin)));
    int per_sm = 0;
    FIT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, o.threads, smem));
    if (per_sm < 1) return fail(FIT_ERR_INVALID_CONFIG, "fit_batch: launch configuration does not fit an SM");
    if (o.blocks_per_sm > 0) per_sm = std::min(per_sm, o.blocks_per_sm);
    const int grid = std::max(1, std::min(n_inst, per_sm * cfg.sms));

    Staged dm, di, dd, dst, dfx, dbe, dre, dws, dq, dord;
    bool hbe = false, hre = false;
    std::vector<DevModel> hm(n_models);
    for (int i = 0; i < n_models; ++i) hm[i] = models[i]->host;
    // Queue order: the costliest fits first, so that no long fit is picked up last and holds
    // the launch while the other blocks are idle (instances of uneven size). Cost of one
    // evaluation ~ the survival and energy-correction work, true bins x (cores + 4) per fitted
    // dataset, plus the parameter vector.
    std::vector<int> order(n_inst);
    bool reordered = false;
    {
        std::vector<double> cost(n_inst);
        for (int i = 0; i < n_inst; ++i) {
            const DevModel &h = hm[inst[i].model];
            int nd = 0;
            for (int d = 0; d < h.n_ds; ++d) nd += (inst[i].mask >> d) & 1u;
            cost[i] = (double)nd * h.N_t * (h.C + 4) + h.P;
            order[i] = i;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        for (int i = 0; i < n_inst && !reordered; ++i) reordered = order[i] != i;
    }
    Staged dpre;
    rc = stage_in(hm.data(), sizeof(DevModel) * n_models, s, dm);
    if (!rc && reordered) rc = stage_in(order.data(), sizeof(int) * n_inst, s, dord);
    if (!rc && precond && pre_k > 0)
        rc = stage_in(pre_tab.data(), sizeof(fitcore::PreEntry) * pre_tab.size(), s, dpre);
    if (!rc) rc = stage_in(inst, sizeof(fit_instance) * n_inst, s, di);
    if (!rc) rc = stage_in(data, sizeof(float) * data_len, s, dd);
    if (!rc && start) rc = stage_in(start, sizeof(double) * par_len, s, dst);
    if (!rc && fixed) rc = stage_in(fixed, (size_t)par_len, s, dfx);
    if (!rc) rc = stage_out(best, sizeof(double) * par_len, s, dbe, hbe);
    if (!rc) rc = stage_out(results, sizeof(fit_result) * n_inst, s, dre, hre);
    if (!rc && !in_smem) {
        if (cudaMallocAsync(&dws.dev, sizeof(float) * (size_t)grid * max_need, s))
            rc = fail(FIT_ERR_OOM, "fit_batch: workspace");
        dws.owned = true;
    }
    if (!rc) {
        if (cudaMallocAsync(&dq.dev, sizeof(int), s) || (!o.use_graph && cudaMemsetAsync(dq.dev, 0, sizeof(int), s)))
            rc = fail(FIT_ERR_CUDA, "fit_batch: queue");
        dq.owned = true;
    }
    if (!rc) {
        fitcore::FitArgs a;
        a.models = (const DevModel *)dm.dev;
        a.inst = (const fit_instance *)di.dev;
        a.n_inst = n_inst;
        a.hist = o.history;
        a.max_iter = o.max_iter;
        a.max_ls = 8;
        a.restarts = o.restarts;
        a.edm_tol = o.edm_tol;
        a.f_noise_rel = o.f_noise_rel;
        a.data = (const float *)dd.dev;
        a.start = start ? (const double *)dst.dev : nullptr;
        a.fixed = fixed ? (const uint8_t *)dfx.dev : nullptr;
        a.best = (double *)dbe.dev;
        a.results = (fit_result *)dre.dev;
        a.queue = (int *)dq.dev;
        a.ws_global = (float *)dws.dev;
        a.ws_stride = max_need;
        a.smem_floats = placement == 1 ? max_need : placement == 2 ? max_loc : 0;
        a.hist_global = placement == 1 ? 0 : 1;
        a.budget_ns = (uint64_t)(o.time_budget_s * 1e9);
        a.precond = precond ? 1 : 0;
        a.order = reordered ? (const int *)dord.dev : nullptr;
        a.pre_tab = (precond && pre_k > 0) ? (const fitcore::PreEntry *)dpre.dev : nullptr;
        a.pre_per_model = pre_k;
        if (o.use_graph) {
            rc = graph_launch(kern, grid, o.threads, smem, a, (int *)dq.dev, s);
        } else {
            void *args[] = {&a};
            cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(o.threads), args, smem, s);
            if (e != cudaSuccess) rc = fail(FIT_ERR_CUDA, std::string("fit_kernel launch: ") + cudaGetErrorString(e));
        }
        g_launches++;
    }
    if (!rc && hbe) {
        // copy back only the parameter ranges the instances own (merged intervals), so that
        // other entries of a host `best` array keep their values
        std::vector<std::pair<int64_t, int64_t>> iv;
        iv.reserve(n_inst);
        for (int i = 0; i < n_inst; ++i)
            iv.emplace_back(inst[i].param_off, inst[i].param_off + models[inst[i].model]->n_params);
        std::sort(iv.begin(), iv.end());
        int64_t a = iv[0].first, b = iv[0].second;
        for (size_t q = 1; q <= iv.size() && !rc; ++q) {
            if (q < iv.size() && iv[q].first <= b) {
                b = std::max(b, iv[q].second);
                continue;
            }
            if (cudaMemcpyAsync(best + a, (double *)dbe.dev + a, sizeof(double) * (b - a),
                                cudaMemcpyDeviceToHost, s))
                rc = fail(FIT_ERR_CUDA, "fit_batch: copy back");
            if (q < iv.size()) {
                a = iv[q].first;
                b = iv[q].second;
            }
        }
    }
    if (!rc && hre && cudaMemcpyAsync(results, dre.dev, sizeof(fit_result) * n_inst, cudaMemcpyDeviceToHost, s))
        rc = fail(FIT_ERR_CUDA, "fit_batch: copy back");
    for (Staged *b : {&dm, &di, &dd, &dst, &dfx, &dbe, &dre, &dws, &dq, &dord, &dpre}) release(*b, s);
    // the staged model table and instance table are host vectors: finish before they go away
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = fail(FIT_ERR_CUDA, "fit_batch: synchronise");
    return rc;
}


int fit_batch_autotune(fit_model *const *models, int n_models, const fit_instance *inst, int n_inst,
                       const float *data, const double *start, int n_sample, fit_batch_opts *opts, void *stream) {
    if (!models || n_models < 1 || !inst || n_inst < 1 || !data || !opts || n_sample < 0)
        return fail(FIT_ERR_INVALID_ARG, "fit_batch_autotune: bad argument");
    LaunchCfg cfg;
    int rc = device_cfg(cfg);
    if (rc) return rc;
    const int n = n_sample > 0 ? std::min(n_sample, n_inst) : std::min(n_inst, 10 * cfg.sms);
    int64_t par_len = 0;
    for (int i = 0; i < n; ++i) {
        if (inst[i].model < 0 || inst[i].model >= n_models || !models[inst[i].model])
            return fail(FIT_ERR_INVALID_ARG, "fit_batch_autotune: instance out of range");
        par_len = std::max<int64_t>(par_len, inst[i].param_off + models[inst[i].model]->n_params);
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *best = nullptr;
    fit_result *res = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&best, sizeof(double) * (size_t)par_len) || cudaMalloc(&res, sizeof(fit_result) * (size_t)n) ||
        cudaEventCreate(&e0) || cudaEventCreate(&e1))
        rc = fail(FIT_ERR_OOM, "fit_batch_autotune: scratch");
    fit_batch_opts o = *opts, best_o = *opts;
    float best_ms = 0.f;
    bool found = false;
    // (threads, blocks per SM): 64-thread blocks put twice the fits on an SM at the same
    // warp count; a cap of 5 or more selects the 96-register build
    const int cand[][2] = {{64, 8}, {64, 10}, {96, 4}, {96, 5}, {128, 4}, {128, 5}};
    for (const auto &cb : cand) {
        const int threads = cb[0], bps = cb[1];
        {
            if (rc) break;
            o.threads = threads;
            o.blocks_per_sm = bps;
            if (fit_batch(models, n_models, inst, n, data, start, best, res, &o, stream) != FIT_OK) {
                rc = FIT_OK;   // a configuration that does not fit is skipped
                continue;
            }
            cudaEventRecord(e0, s);
            int r2 = fit_batch(models, n_models, inst, n, data, start, best, res, &o, stream);
            cudaEventRecord(e1, s);
            if (r2 != FIT_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (!found || ms < best_ms) {
                found = true;
                best_ms = ms;
                best_o = o;
            }
        }
    }
    if (best) cudaFree(best);
    if (res) cudaFree(res);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    if (!found) return fail(FIT_ERR_INVALID_CONFIG, "fit_batch_autotune: no configuration ran");
    opts->threads = best_o.threads;
    opts->blocks_per_sm = best_o.blocks_per_sm;
    return FIT_OK;
}


int fit_profile_scan(fit_model *model, const float *data, uint32_t mask, int n_scan, const int *scan_idx,
                     int n_points, const double *points, const double *start, const fit_batch_opts *opts,
                     double *nll_min, double *theta_best, double *dchi2, double *theta_points, int *status,
                     void *stream) {
    if (!model || !data || n_scan < 1 || n_scan > 8 || !scan_idx || n_points < 1 || !points || !nll_min ||
        !dchi2)
        return fail(FIT_ERR_INVALID_ARG, "fit_profile_scan: bad argument");
    const int P = model->n_params;
    for (int q = 0; q < n_scan; ++q)
        if (scan_idx[q] < 0 || scan_idx[q] >= P || model->in_block[scan_idx[q]])
            return fail(FIT_ERR_INVALID_ARG, "fit_profile_scan: scan parameters must lie outside the prior blocks");
    const int n = n_points + 1;   // instance 0: the unconstrained fit
    std::vector<double> st((size_t)n * P), best((size_t)n * P);
    std::vector<uint8_t> fx((size_t)n * P, 0);
    std::vector<double> st0(P);
    if (start) {
        if (cudaMemcpy(st0.data(), start, sizeof(double) * P, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            return fail(FIT_ERR_INVALID_ARG, "fit_profile_scan: start not readable");
        }
    } else {
        if (cudaMemcpy(st0.data(), model->host.theta0, sizeof(double) * P, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(FIT_ERR_CUDA, "fit_profile_scan: theta0");
    }
    std::vector<fit_instance> inst(n);
    for (int k = 0; k < n; ++k) {
        inst[k].model = 0;
        inst[k].mask = mask;
        inst[k].data_off = 0;   // every point fits the same data vector
        inst[k].param_off = (int64_t)k * P;
        std::copy(st0.begin(), st0.end(), st.begin() + (size_t)k * P);
        if (k > 0)
            for (int q = 0; q < n_scan; ++q) {
                st[(size_t)k * P + scan_idx[q]] = points[(size_t)(k - 1) * n_scan + q];
                fx[(size_t)k * P + scan_idx[q]] = 1;
            }
    }
    std::vector<fit_result> res(n);
    fit_model *ms[1] = {model};
    int rc = fit_batch_ex(ms, 1, inst.data(), n, data, st.data(), fx.data(), best.data(), res.data(), opts,
                          stream);
    if (rc) return rc;
    // the profile's minimum: the unconstrained fit, unless a raster point went lower
    int kmin = 0;
    for (int k = 1; k < n; ++k)
        if (res[k].nll_min < res[kmin].nll_min) kmin = k;
    *nll_min = res[kmin].nll_min;
    if (theta_best) std::copy(best.begin() + (size_t)kmin * P, best.begin() + (size_t)(kmin + 1) * P, theta_best);
    for (int k = 1; k < n; ++k) {
        dchi2[k - 1] = res[k].nll_min - res[kmin].nll_min;
        if (status) status[k - 1] = res[k].status;
        if (theta_points)
            std::copy(best.begin() + (size_t)k * P, best.begin() + (size_t)(k + 1) * P,
                      theta_points + (size_t)(k - 1) * P);
    }
    return FIT_OK;
}

int fit_wilks_interval(int n, const double *x, const double *dchi2, double level, double *lo, double *hi) {
    if (n < 2 || !x || !dchi2 || !lo || !hi || !(level > 0.0))
        return fail(FIT_ERR_INVALID_ARG, "fit_wilks_interval: bad argument");
    for (int i = 1; i < n; ++i)
        if (!(x[i] > x[i - 1])) return fail(FIT_ERR_INVALID_ARG, "fit_wilks_interval: x must increase");
    int im = 0;
    for (int i = 1; i < n; ++i)
        if (dchi2[i] < dchi2[im]) im = i;
    int open = 0;
    // crossing of `level` on each side of the minimum, linear between the raster points
    int i = im;
    while (i > 0 && dchi2[i - 1] < level) --i;
    if (i == 0) {
        *lo = x[0];
        open |= 1;
    } else {
        const double t = (level - dchi2[i]) / (dchi2[i - 1] - dchi2[i]);
        *lo = x[i] + t * (x[i - 1] - x[i]);
    }
    i = im;
    while (i < n - 1 && dchi2[i + 1] < level) ++i;
    if (i == n - 1) {
        *hi = x[n - 1];
        open |= 2;
    } else {
        const double t = (level - dchi2[i]) / (dchi2[i + 1] - dchi2[i]);
        *hi = x[i] + t * (x[i + 1] - x[i]);
    }
    return open;
}

double fit_chi2_sf(double chi2, int dof) {
    // Q(a, x) = Gamma(a, x) / Gamma(a) with a = dof / 2, x = chi2 / 2: the series of the lower
    // function P(a, x) = x^a e^-x / Gamma(a) sum_n x^n / (a (a+1) ... (a+n)) below x = a + 1, the
    // continued fraction of the upper one (evaluated by the modified Lentz method) above.
    if (dof < 1 || !(chi2 >= 0.0)) return NAN;
    const double a = 0.5 * dof, x = 0.5 * chi2;
    if (x == 0.0) return 1.0;
    const double lpre = a * std::log(x) - x - std::lgamma(a);
    if (x < a + 1.0) {
        double term = 1.0 / a, sum = term;
        for (int k = 1; k < 100000; ++k) {
            term *= x / (a + k);
            sum += term;
            if (std::fabs(term) < 1e-17 * std::fabs(sum)) break;
        }
        return 1.0 - std::exp(lpre) * sum;
    }
    const double tiny = 1e-300;
    double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, f = d;
    for (int k = 1; k < 100000; ++k) {
        const double an = -k * (k - a);
        b += 2.0;
        d = an * d + b;
        if (std::fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (std::fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = d * c;
        f *= del;
        if (std::fabs(del - 1.0) < 1e-16) break;
    }
    return std::exp(lpre) * f;
}

}  // extern "C"
