// Warm-start network: a multilayer perceptron n_in -> [n_hidden, GELU] x n_hid_layers -> n_out
// that maps a pseudo-experiment's log-normalised reco spectra to a start point of the fit.
// Weights and activations are bf16 with FP32 master weights; every product runs on the
// tensor-core GEMM (tcgen05, FP32 accumulation) with the bias/GELU (forward) and
// GELU-derivative (backward) epilogues fused; AdamW updates the master weights and rewrites
// the bf16 copies (W and W^T, the operand layouts of the forward and backward products).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fitcore.h"
#include "gemm_tc.cuh"
#include "kernels.cuh"

int fitcore_fail(int code, const std::string &msg);
void fitcore_count_launch();

namespace {

constexpr int kMaxLayers = 8;

inline int pad8(int x) { return (x + 7) / 8 * 8; }

__global__ void prep_input_kernel(int B, int n_in, int ld, const float *__restrict__ x, __nv_bfloat16 *__restrict__ a0) {
    const int64_t total = (int64_t)B * ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / ld), i = (int)(e % ld);
        a0[e] = __float2bfloat16(i < n_in ? x[(int64_t)b * n_in + i] : 0.f);
    }
}

// d loss / d out for the mean squared error over B x n_out (n_out <= 256): a thread per sample
// writes its row of dout (ld per row, zero padding) and its column of the transpose doutT (ldt
// per feature row, coalesced over the samples); the output layer's bias gradient db (cleared
// by the caller) gets the column sums of the bf16 values, and the loss (double) is
// accumulated; one atomic per block and column / per block.
__global__ void __launch_bounds__(256) mse_kernel(int B, int n_out, int ld, const float *__restrict__ out,
                                                  const float *__restrict__ tgt, __nv_bfloat16 *__restrict__ dout,
                                                  int ldt, __nv_bfloat16 *__restrict__ doutT, float *__restrict__ db,
                                                  double *__restrict__ loss) {
    __shared__ double part[8];
    __shared__ float col[256];
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) col[o] = 0.f;
    __syncthreads();
    const float scale = 2.f / (float)((int64_t)B * n_out);
    double acc = 0.0;
    // the loop bound is uniform over the block, so every lane takes part in the shuffles
    for (int b0 = blockIdx.x * blockDim.x; b0 < B; b0 += gridDim.x * blockDim.x) {
        const int b = b0 + threadIdx.x;
        const bool valid = b < B;
        for (int o = 0; o < ld; ++o) {
            float q = 0.f;   // the bf16-rounded gradient (0 past B and in the padding)
            if (valid) {
                float g = 0.f;
                if (o < n_out) {
                    const float r = out[(int64_t)b * n_out + o] - tgt[(int64_t)b * n_out + o];
                    acc += (double)r * r;
                    g = scale * r;
                    doutT[(int64_t)o * ldt + b] = __float2bfloat16(g);
                }
                const __nv_bfloat16 h = __float2bfloat16(g);
                dout[(int64_t)b * ld + o] = h;
                q = __bfloat162float(h);
            }
            if (o < n_out) {   // column sum: a shuffle tree, one shared atomic per warp
                for (int k = 16; k > 0; k >>= 1) q += __shfl_xor_sync(0xffffffffu, q, k);
                if ((threadIdx.x & 31) == 0) atomicAdd(&col[o], q);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) atomicAdd(db + o, col[o]);
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(loss, t / (double)((int64_t)B * n_out));
    }
}

// Input of a training step: a0[b][i] = bf16(x[b][i]) (0 in the padding columns i >= n_in) and
// the transpose a0t[i][b] for i < n_in; 32 x 32 tiles through shared memory so that both the
// row-major and the transposed writes are coalesced. Block (32, 8).
__global__ void prep_input_t_kernel(int B, int n_in, int ld, const float *__restrict__ x,
                                    __nv_bfloat16 *__restrict__ a0, int ldt, __nv_bfloat16 *__restrict__ a0t) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int i0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int b = b0 + r, i = i0 + threadIdx.x;
        const __nv_bfloat16 q = __float2bfloat16((b < B && i < n_in) ? x[(int64_t)b * n_in + i] : 0.f);
        tile[r][threadIdx.x] = q;
        if (b < B && i < ld) a0[(int64_t)b * ld + i] = q;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, b = b0 + threadIdx.x;
        if (i < n_in && b < B) a0t[(int64_t)i * ldt + b] = tile[threadIdx.x][r];
    }
}

// db[o] += sum_b d[b][o] (db cleared by the caller): block (32, 8) covers 64 columns (a column
// pair per thread, read as bf16x2 along the row, so a warp reads 128 contiguous bytes) and
// kColRows rows; partial sums meet in shared memory and go out with one atomic per column.
constexpr int kColRows = 256;
__global__ void colsum_kernel(int B, int n, int ld, const __nv_bfloat16 *__restrict__ d, float *__restrict__ db) {
    __shared__ float2 part[8][33];
    const int cp = blockIdx.x * 32 + threadIdx.x;   // column pair
    const int c = 2 * cp;
    const int b0 = blockIdx.y * kColRows;
    float2 acc = make_float2(0.f, 0.f);
    if (c < n) {
        for (int b = b0 + threadIdx.y; b < min(B, b0 + kColRows); b += 8) {
            const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(d + (int64_t)b * ld + c);
            acc.x += __low2float(v);
            acc.y += __high2float(v);
        }
    }
    part[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && c < n) {
        float2 t = part[0][threadIdx.x];
        for (int y = 1; y < 8; ++y) {
            t.x += part[y][threadIdx.x].x;
            t.y += part[y][threadIdx.x].y;
        }
        atomicAdd(&db[c], t.x);
        if (c + 1 < n) atomicAdd(&db[c + 1], t.y);
    }
}

struct AdamW {
    float lr, b1, b2, eps, wd, c1, c2;   // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
};

// One AdamW update of parameter p with gradient gr and moments m, v (decay: weights only).
__device__ __forceinline__ void adamw_one(const AdamW &h, float *p, float gr, float *m, float *v, bool decay) {
    *m = h.b1 * *m + (1.f - h.b1) * gr;
    *v = h.b2 * *v + (1.f - h.b2) * gr * gr;
    const float upd = (*m * h.c1) / (sqrtf(*v * h.c2) + h.eps) + (decay ? h.wd * *p : 0.f);
    *p -= h.lr * upd;
}

// Per-layer arguments of the fused AdamW launch: the [out x in] weights (W bf16 copy with rows
// of ldw, W^T with rows of ldwt) and the bias.
struct AdamLayer {
    int out, in, ldw, ldwt, tiles_i, wtiles;   // wtiles = ceil(out/32) ceil(in/32) weight tiles
    float *w, *g, *mw, *vw, *b, *gb, *mb, *vb;
    __nv_bfloat16 *wbf, *wt;
};
struct AdamAll {
    int n;
    int first[kMaxLayers + 1];   // first block of each layer: its weight tiles, then its bias blocks
    AdamLayer L[kMaxLayers];
};

// AdamW on every layer in one launch. A block (32 x 8 threads) updates a 32 x 32 weight tile
// (rows of W along the lanes) and rewrites both bf16 copies, the transposed one through a
// shared-memory tile so that its writes are coalesced too; the bias blocks update 256 biases.
__global__ void __launch_bounds__(256) adamw_all_kernel(AdamW h, AdamAll A) {
    __shared__ __nv_bfloat16 tile[32][34];
    int t = blockIdx.x, l = 0;
    while (l + 1 < A.n && t >= A.first[l + 1]) ++l;
    const AdamLayer &L = A.L[l];
    t -= A.first[l];
    if (t < L.wtiles) {
        const int o0 = (t / L.tiles_i) * 32, i0 = (t % L.tiles_i) * 32;
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int o = o0 + r, i = i0 + threadIdx.x;
            __nv_bfloat16 q = __float2bfloat16(0.f);
            if (o < L.out && i < L.in) {
                const int64_t e = (int64_t)o * L.in + i;
                adamw_one(h, L.w + e, L.g[e], L.mw + e, L.vw + e, true);
                q = __float2bfloat16(L.w[e]);
                L.wbf[(int64_t)o * L.ldw + i] = q;
            }
            tile[r][threadIdx.x] = q;
        }
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int i = i0 + r, o = o0 + threadIdx.x;
            if (i < L.in && o < L.out) L.wt[(int64_t)i * L.ldwt + o] = tile[threadIdx.x][r];
        }
    } else {
        const int k = (t - L.wtiles) * 256 + threadIdx.y * 32 + threadIdx.x;
        if (k < L.out) adamw_one(h, L.b + k, L.gb[k], L.mb + k, L.vb + k, false);
    }
}

__global__ void cast_weights_kernel(int out, int in, const float *__restrict__ w, __nv_bfloat16 *__restrict__ wbf,
                                    int ldw, __nv_bfloat16 *__restrict__ wt, int ldwt) {
    const int64_t total = (int64_t)out * in;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(e / in), i = (int)(e % in);
        const __nv_bfloat16 q = __float2bfloat16(w[e]);
        wbf[(int64_t)o * ldw + i] = q;
        wt[(int64_t)i * ldwt + o] = q;
    }
}

// Log-normalised spectra: x[b][slot0 + q] = log(1 + n_q) / log(1 + nbar_q) - 1, other slots 0,
// the geometry's one-hot slot 1.
// Bins of datasets left out by the sample's mask, and all slots of a sample whose expectation
// failed (status != 0), are 0.
__global__ void features_kernel(int B, int n_data, const float *__restrict__ data, const float *__restrict__ nbar,
                                const uint32_t *__restrict__ masks, const int *__restrict__ slot_ds,
                                const int *__restrict__ status, int n_in, int slot0, int onehot,
                                float *__restrict__ x) {
    const int64_t total = (int64_t)B * n_in;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / n_in), s = (int)(e % n_in);
        const int q = s - slot0;
        float v = 0.f;
        if (status && status[b]) {
            v = 0.f;
        } else if (q >= 0 && q < n_data) {
            if (masks && !((masks[b] >> slot_ds[q]) & 1u)) {
                x[e] = 0.f;
                continue;
            }
            const float nb = nbar[q];
            v = nb > 0.f ? log1pf(data[(int64_t)b * n_data + q]) / log1pf(nb) - 1.f : 0.f;
        } else if (s == onehot) {
            v = 1.f;
        }
        x[e] = v;
    }
}

// theta[b] = theta0, then theta[b][idx_t] = theta0 + out[b][t] * scale_t
// theta[b][i] = base[b][i] + y_bt scale_t for the network's targets (i = idx[t]), base[b][i]
// for the other parameters; base may be theta itself, and null stands for theta0
__global__ void starts_kernel(int B, int P, const double *__restrict__ theta0, int n_t, const int *__restrict__ idx,
                              const double *__restrict__ scale, const float *__restrict__ out, int n_out,
                              const double *base, double *theta) {
    const int64_t total = (int64_t)B * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / P), i = (int)(e % P);
        double v = base ? base[e] : theta0[i];
        for (int t = 0; t < n_t; ++t)
            if (idx[t] == i) v += (double)out[(int64_t)b * n_out + t] * scale[t];
        theta[e] = v;
    }
}

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

struct fit_mlp {
    int n_layers = 0;               // linear layers
    int dims[kMaxLayers + 1] = {0};
    int ld[kMaxLayers + 1] = {0};   // padded row lengths (multiples of 8)
    uint64_t seed = 0;
    int step = 0;
    // parameters (device)
    float *w[kMaxLayers] = {nullptr}, *b[kMaxLayers] = {nullptr};
    float *mw[kMaxLayers] = {nullptr}, *vw[kMaxLayers] = {nullptr}, *mb[kMaxLayers] = {nullptr}, *vb[kMaxLayers] = {nullptr};
    float *gw[kMaxLayers] = {nullptr}, *gb[kMaxLayers] = {nullptr};
    __nv_bfloat16 *wbf[kMaxLayers] = {nullptr}, *wt[kMaxLayers] = {nullptr};
    // batch buffers
    int cap = 0;
    __nv_bfloat16 *act[kMaxLayers] = {nullptr};      // act[0] = input, act[l] = GELU(pre[l-1])
    float *pre[kMaxLayers] = {nullptr};              // pre-activation of layer l (hidden layers)
    __nv_bfloat16 *dpre[kMaxLayers] = {nullptr};     // d loss / d pre of layer l (bf16)
    float *out = nullptr, *x32 = nullptr;
    // transposed copies [features x pad8(B)] for the weight gradients, written by the kernels
    // that produce act / dpre (input preparation, forward and backward epilogues, MSE)
    __nv_bfloat16 *actT[kMaxLayers] = {nullptr};
    __nv_bfloat16 *dpreT[kMaxLayers] = {nullptr};
    double *loss = nullptr;
    std::vector<void *> owned;
};

namespace {

int dev_alloc(fit_mlp *m, void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fitcore_fail(FIT_ERR_OOM, "fit_mlp: device allocation");
    }
    cudaMemset(*p, 0, bytes);
    m->owned.push_back(*p);
    return FIT_OK;
}

bool is_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ensure_batch(fit_mlp *m, int B) {
    if (B <= m->cap) return FIT_OK;
    for (int l = 0; l < m->n_layers; ++l) {
        if (m->act[l]) cudaFree(m->act[l]);
        if (m->pre[l]) cudaFree(m->pre[l]);
        if (m->dpre[l]) cudaFree(m->dpre[l]);
        if (m->actT[l]) cudaFree(m->actT[l]);
        if (m->dpreT[l]) cudaFree(m->dpreT[l]);
        m->act[l] = nullptr;
        m->pre[l] = nullptr;
        m->dpre[l] = nullptr;
        m->actT[l] = nullptr;
        m->dpreT[l] = nullptr;
    }
    for (void *p : {(void *)m->out, (void *)m->x32})
        if (p) cudaFree(p);
    int rc = FIT_OK;
    const int L = m->n_layers, Bp = pad8(B);
    auto al = [&](void **p, size_t bytes) {
        if (rc) return;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            rc = fitcore_fail(FIT_ERR_OOM, "fit_mlp: batch buffers");
            return;
        }
        cudaMemset(*p, 0, bytes);
    };
    for (int l = 0; l < L; ++l) al((void **)&m->act[l], sizeof(__nv_bfloat16) * (size_t)B * m->ld[l]);
    for (int l = 0; l < L; ++l) al((void **)&m->pre[l], sizeof(float) * (size_t)B * m->dims[l + 1]);
    for (int l = 0; l < L; ++l) al((void **)&m->dpre[l], sizeof(__nv_bfloat16) * (size_t)B * m->ld[l + 1]);
    al((void **)&m->out, sizeof(float) * (size_t)B * m->dims[L]);
    al((void **)&m->x32, sizeof(float) * (size_t)B * m->dims[0]);
    for (int l = 0; l < L; ++l) al((void **)&m->actT[l], sizeof(__nv_bfloat16) * (size_t)m->dims[l] * Bp);
    for (int l = 0; l < L; ++l) al((void **)&m->dpreT[l], sizeof(__nv_bfloat16) * (size_t)m->dims[l + 1] * Bp);
    if (rc == FIT_OK) m->cap = B;
    return rc;
}

// forward through all layers from m->act[0]; result (fp32) in m->out; with `train` the hidden
// activations are also written transposed (actT) for the weight gradients
int forward(fit_mlp *m, int B, cudaStream_t s, bool train) {
    const int L = m->n_layers;
    for (int l = 0; l < L; ++l) {
        fitcore::GemmOut o;
        if (l + 1 < L) {
            o.epi = fitcore::EPI_BIAS_GELU;
            o.C = m->pre[l];
            o.ldc = m->dims[l + 1];
            o.Y = m->act[l + 1];
            o.ldy = m->ld[l + 1];
            if (train) {
                o.Yt = m->actT[l + 1];
                o.ldyt = pad8(B);
            }
        } else {
            o.epi = fitcore::EPI_BIAS_F32;
            o.C = m->out;
            o.ldc = m->dims[L];
        }
        o.bias = m->b[l];
        int rc = fitcore::tc_gemm(false, B, m->dims[l + 1], m->dims[l], m->act[l], m->ld[l], m->wbf[l], m->ld[l], o, s,
                                  nullptr);
        if (rc) return rc;
    }
    return FIT_OK;
}

}  // namespace

extern "C" {

int fit_mlp_create(int n_in, int n_hidden, int n_hidden_layers, int n_out, uint64_t seed, fit_mlp **out) {
    if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || n_hidden_layers < 0 || n_hidden_layers + 1 > kMaxLayers ||
        n_in > 65536 || n_hidden > 65536 || n_out > 256)
        return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mlp_create: bad dimensions");
    fit_mlp *m = new fit_mlp();
    m->n_layers = n_hidden_layers + 1;
    m->dims[0] = n_in;
    for (int l = 1; l <= n_hidden_layers; ++l) m->dims[l] = n_hidden;
    m->dims[m->n_layers] = n_out;
    for (int l = 0; l <= m->n_layers; ++l) m->ld[l] = pad8(m->dims[l]);
    m->seed = seed;
    // He-normal initial weights from a SplitMix64 stream (Box-Muller), biases 0
    uint64_t st = seed;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    int rc = FIT_OK;
    for (int l = 0; l < m->n_layers && rc == FIT_OK; ++l) {
        const int o = m->dims[l + 1], in = m->dims[l];
        std::vector<float> w((size_t)o * in);
        const double sd = std::sqrt(2.0 / in);
        for (size_t e = 0; e < w.size(); ++e) {
            const double u1 = next(), u2 = next();
            w[e] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
        const size_t nw = (size_t)o * in;
        rc = dev_alloc(m, (void **)&m->w[l], sizeof(float) * nw);
        if (!rc) rc = dev_alloc(m, (void **)&m->b[l], sizeof(float) * o);
        if (!rc) rc = dev_alloc(m, (void **)&m->mw[l], sizeof(float) * nw);
        if (!rc) rc = dev_alloc(m, (void **)&m->vw[l], sizeof(float) * nw);
        if (!rc) rc = dev_alloc(m, (void **)&m->mb[l], sizeof(float) * o);
        if (!rc) rc = dev_alloc(m, (void **)&m->vb[l], sizeof(float) * o);
        if (!rc) rc = dev_alloc(m, (void **)&m->gw[l], sizeof(float) * nw);
        if (!rc) rc = dev_alloc(m, (void **)&m->gb[l], sizeof(float) * o);
        if (!rc) rc = dev_alloc(m, (void **)&m->wbf[l], sizeof(__nv_bfloat16) * (size_t)o * m->ld[l]);
        if (!rc) rc = dev_alloc(m, (void **)&m->wt[l], sizeof(__nv_bfloat16) * (size_t)in * m->ld[l + 1]);
        if (!rc && cudaMemcpy(m->w[l], w.data(), sizeof(float) * nw, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = fitcore_fail(FIT_ERR_CUDA, "fit_mlp_create: upload");
        if (!rc) {
            cast_weights_kernel<<<grid_for((int64_t)nw), 256>>>(o, in, m->w[l], m->wbf[l], m->ld[l], m->wt[l], m->ld[l + 1]);
            fitcore_count_launch();
        }
    }
    if (!rc) rc = dev_alloc(m, (void **)&m->loss, sizeof(double));
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = fitcore_fail(FIT_ERR_CUDA, "fit_mlp_create: init");
    if (rc) {
        fit_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return FIT_OK;
}

void fit_mlp_destroy(fit_mlp *m) {
    if (!m) return;
    for (void *p : m->owned) cudaFree(p);
    for (int l = 0; l < m->n_layers; ++l) {
        if (m->act[l]) cudaFree(m->act[l]);
        if (m->pre[l]) cudaFree(m->pre[l]);
        if (m->dpre[l]) cudaFree(m->dpre[l]);
        if (m->actT[l]) cudaFree(m->actT[l]);
        if (m->dpreT[l]) cudaFree(m->dpreT[l]);
    }
    for (void *p : {(void *)m->out, (void *)m->x32})
        if (p) cudaFree(p);
    delete m;
}

int fit_mlp_forward(fit_mlp *m, int B, const float *x, float *y, void *stream) {
    if (!m || !x || !y || B < 1) return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mlp_forward: bad argument");
    if (!is_device(x)) return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mlp_forward: x must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_batch(m, B);
    if (rc) return rc;
    prep_input_kernel<<<grid_for((int64_t)B * m->ld[0]), 256, 0, s>>>(B, m->dims[0], m->ld[0], x, m->act[0]);
    fitcore_count_launch();
    rc = forward(m, B, s, false);
    if (rc) return rc;
    if (cudaMemcpyAsync(y, m->out, sizeof(float) * (size_t)B * m->dims[m->n_layers], cudaMemcpyDefault, s) != cudaSuccess)
        return fitcore_fail(FIT_ERR_CUDA, "fit_mlp_forward: copy out");
    return FIT_OK;
}

int fit_mlp_train_step(fit_mlp *m, int B, const float *x, const float *target, float lr, float weight_decay,
                       double *loss_out, void *stream) {
    if (!m || !x || !target || B < 1 || !(lr >= 0.f))
        return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mlp_train_step: bad argument");
    if (!is_device(x) || !is_device(target))
        return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mlp_train_step: x and target must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_batch(m, B);
    if (rc) return rc;
    const int L = m->n_layers, Bp = pad8(B);
    prep_input_t_kernel<<<dim3((m->ld[0] + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, s>>>(
        B, m->dims[0], m->ld[0], x, m->act[0], Bp, m->actT[0]);
    cudaMemsetAsync(m->loss, 0, sizeof(double), s);
    fitcore_count_launch();
    if ((rc = forward(m, B, s, true))) return rc;
    // bias gradients (column sums of the bf16 backward signals): the output layer's from the
    // MSE kernel, the hidden layers' from colsum_kernel
    for (int l = 0; l < L; ++l) cudaMemsetAsync(m->gb[l], 0, sizeof(float) * m->dims[l + 1], s);
    mse_kernel<<<(B + 255) / 256, 256, 0, s>>>(
        B, m->dims[L], m->ld[L], m->out, target, m->dpre[L - 1], Bp, m->dpreT[L - 1], m->gb[L - 1], m->loss);
    fitcore_count_launch();
    for (int l = L - 1; l >= 0; --l) {
        const int o = m->dims[l + 1], in = m->dims[l];
        if (l < L - 1) {   // bias gradient of a hidden layer (the output layer's: mse_kernel)
            colsum_kernel<<<dim3((o + 63) / 64, (B + kColRows - 1) / kColRows), dim3(32, 8), 0, s>>>(
                B, o, m->ld[l + 1], m->dpre[l], m->gb[l]);
            fitcore_count_launch();
        }
        // dW = dpre^T act: both operands K-major over the batch, as the producing kernels
        // wrote them (dpreT, actT)
        fitcore::GemmOut gw;
        gw.epi = fitcore::EPI_F32;
        gw.C = m->gw[l];
        gw.ldc = in;
        if ((rc = fitcore::tc_gemm(false, o, in, B, m->dpreT[l], Bp, m->actT[l], Bp, gw, s, nullptr))) return rc;
        if (l > 0) {
            // d pre_{l-1} = (d pre_l W_l) * gelu'(pre_{l-1})
            fitcore::GemmOut gx;
            gx.epi = fitcore::EPI_DGELU;
            gx.Y = m->dpre[l - 1];
            gx.ldy = m->ld[l];
            gx.aux = m->pre[l - 1];
            gx.ldaux = in;
            gx.Yt = m->dpreT[l - 1];
            gx.ldyt = Bp;
            if ((rc = fitcore::tc_gemm(false, B, in, o, m->dpre[l], m->ld[l + 1], m->wt[l], m->ld[l + 1], gx, s, nullptr)))
                return rc;
        }
    }
    m->step++;
    AdamW h;
    h.lr = lr;
    h.b1 = 0.9f;
    h.b2 = 0.999f;
    h.eps = 1e-8f;
    h.wd = weight_decay;
    h.c1 = (float)(1.0 / (1.0 - std::pow(0.9, m->step)));
    h.c2 = (float)(1.0 / (1.0 - std::pow(0.999, m->step)));
    AdamAll A;
    A.n = L;
    int nblk = 0;
    for (int l = 0; l < L; ++l) {
        AdamLayer &q = A.L[l];
        q.out = m->dims[l + 1];
        q.in = m->dims[l];
        q.ldw = m->ld[l];
        q.ldwt = m->ld[l + 1];
        q.tiles_i = (q.in + 31) / 32;
        q.wtiles = ((q.out + 31) / 32) * q.tiles_i;
        q.w = m->w[l];
        q.g = m->gw[l];
        q.mw = m->mw[l];
        q.vw = m->vw[l];
        q.b = m->b[l];
        q.gb = m->gb[l];
        q.mb = m->mb[l];
        q.vb = m->vb[l];
        q.wbf = m->wbf[l];
        q.wt = m->wt[l];
        A.first[l] = nblk;
        nblk += q.wtiles + (q.out + 255) / 256;
    }
    A.first[L] = nblk;
    adamw_all_kernel<<<nblk, dim3(32, 8), 0, s>>>(h, A);
    fitcore_count_launch();
    if (loss_out && cudaMemcpyAsync(loss_out, m->loss, sizeof(double), cudaMemcpyDefault, s) != cudaSuccess)
        return fitcore_fail(FIT_ERR_CUDA, "fit_mlp_train_step: loss");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, std::string("fit_mlp_train_step: ") + cudaGetErrorString(e));
    return FIT_OK;
}

int fit_mlp_get_layer(const fit_mlp *m, int layer, float *w, float *b, float *gw, float *gb) {
    if (!m || layer < 0 || layer >= m->n_layers) return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mlp_get_layer: layer");
    const size_t nw = (size_t)m->dims[layer + 1] * m->dims[layer], nb = m->dims[layer + 1];
    cudaDeviceSynchronize();
    if ((w && cudaMemcpy(w, m->w[layer], sizeof(float) * nw, cudaMemcpyDefault)) ||
        (b && cudaMemcpy(b, m->b[layer], sizeof(float) * nb, cudaMemcpyDefault)) ||
        (gw && cudaMemcpy(gw, m->gw[layer], sizeof(float) * nw, cudaMemcpyDefault)) ||
        (gb && cudaMemcpy(gb, m->gb[layer], sizeof(float) * nb, cudaMemcpyDefault)))
        return fitcore_fail(FIT_ERR_CUDA, "fit_mlp_get_layer: copy");
    return FIT_OK;
}

int fit_mlp_set_layer(fit_mlp *m, int layer, const float *w, const float *b) {
    if (!m || layer < 0 || layer >= m->n_layers || !w || !b)
        return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mlp_set_layer: bad argument");
    const int o = m->dims[layer + 1], in = m->dims[layer];
    const size_t nw = (size_t)o * in;
    if (cudaMemcpy(m->w[layer], w, sizeof(float) * nw, cudaMemcpyDefault) ||
        cudaMemcpy(m->b[layer], b, sizeof(float) * o, cudaMemcpyDefault))
        return fitcore_fail(FIT_ERR_CUDA, "fit_mlp_set_layer: copy");
    cast_weights_kernel<<<grid_for((int64_t)nw), 256>>>(o, in, m->w[layer], m->wbf[layer], m->ld[layer], m->wt[layer],
                                                        m->ld[layer + 1]);
    fitcore_count_launch();
    if (cudaDeviceSynchronize() != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, "fit_mlp_set_layer: cast");
    return FIT_OK;
}

}  // extern "C"

namespace fitcore {

int features(int B, int n_data, const float *data, const float *nbar, const uint32_t *masks, const int *slot_ds,
             const int *status, int n_in, int slot0, int onehot, float *x, cudaStream_t s) {
    features_kernel<<<grid_for((int64_t)B * n_in), 256, 0, s>>>(B, n_data, data, nbar, masks, slot_ds, status, n_in,
                                                                slot0, onehot, x);
    fitcore_count_launch();
    return cudaGetLastError() == cudaSuccess ? FIT_OK : fitcore_fail(FIT_ERR_CUDA, "warm start: features");
}

int starts(int B, int P, const double *theta0, int n_t, const int *idx, const double *scale, const float *out,
           int n_out, const double *base, double *theta, cudaStream_t s) {
    starts_kernel<<<grid_for((int64_t)B * P), 256, 0, s>>>(B, P, theta0, n_t, idx, scale, out, n_out, base, theta);
    fitcore_count_launch();
    return cudaGetLastError() == cudaSuccess ? FIT_OK : fitcore_fail(FIT_ERR_CUDA, "warm start: starts");
}

float *mlp_input_buffer(fit_mlp *m, int B) { return ensure_batch(m, B) == FIT_OK ? m->x32 : nullptr; }
int mlp_dims(const fit_mlp *m, int *n_in, int *n_out) {
    *n_in = m->dims[0];
    *n_out = m->dims[m->n_layers];
    return FIT_OK;
}

}  // namespace fitcore
