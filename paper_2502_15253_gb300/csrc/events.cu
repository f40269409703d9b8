// Event-level reweighting of simulated signal events: for B sets of survival parameters,
//   S_b[j] = sum over the events e in reco bin j of w_e P(L_core(e), E_e; eta_b),
// the step the paper moves to the GPU ([S], "GPU accelerated computation"). Events are stored
// sorted by reco bin as separate arrays (energy, weight float; core uint8; bin int32: 13 bytes
// per event) and stay resident; a call streams them once for all B parameter sets.
//
// Staging: a CTA streams a contiguous range of blocks of 2048 events (26 KB each) through a
// two-stage ring in shared memory, filled by 1-D bulk copies (cp.async.bulk) that complete on
// an mbarrier, so that the next block is in flight while the current one is evaluated. The
// arrays are padded to a whole number of blocks (bin -1, weight 0): no ragged tail.
// A warp takes 32 x kV consecutive events of a block, each lane kV of them in a row; a lane
// sums its run (flushing at the rare bin change inside the run), then the warp adds equal-bin
// lanes with a segmented shuffle reduction. The chunk's last bin segment stays open as a
// per-warp carry that the next chunk (the same warp's share of the next block) continues, so
// a warp adds to the output (in double) only when its bin changes: with sorted events a few
// atomics per warp and set instead of one per chunk, which matters when few bins take all the
// events.
// Per event and parameter set the work is FP32 only: float-pair phases reduced to |r| <= 1/2
// half-turns and a fitted polynomial for sin^2(pi r) (no derivatives are needed here).
#include <algorithm>
#include <string>
#include <vector>

#include "dev_model.cuh"
#include "kernels.cuh"
#include "umma.cuh"

int fitcore_fail(int code, const std::string &msg);
void fitcore_count_launch();

struct fit_mc {
    int mode = 0, n_cores = 0, n_bins = 0;
    int64_t n_events = 0, n_pad = 0;   // n_pad: events rounded up to whole staging blocks
    float *energy = nullptr, *weight = nullptr;
    uint8_t *core = nullptr;
    int *bin = nullptr;
    int *err = nullptr;                // device flag: a staging wait ran out of time
    float kl_hi[FIT_MAX_CORES] = {0.f}, kl_lo[FIT_MAX_CORES] = {0.f};   // K L / pi as float pairs
};

namespace fitcore {
namespace {

constexpr int kV = 8;                      // events per lane and chunk
constexpr int kMaxSets = 64;               // parameter sets per launch
constexpr int kThreads = 256;
constexpr int kBlockEv = kThreads * kV;    // events per staging block (2048)
constexpr uint32_t kStageBytes = kBlockEv * 13;
constexpr uint64_t kWaitNs = 2000000000ull;

// one staging block: the four arrays of 2048 consecutive events
struct Stage {
    float energy[kBlockEv];
    float weight[kBlockEv];
    int bin[kBlockEv];
    uint8_t core[kBlockEv];
};
static_assert(sizeof(Stage) == kStageBytes, "stage layout");

struct McArgs {
    const float *energy, *weight;
    const uint8_t *core;
    const int *bin;
    int64_t n_pad;
    int n_bins, mode, n_cores, B;
    int *err;
    float kl_hi[FIT_MAX_CORES], kl_lo[FIT_MAX_CORES];
    const double *params;   // [B x 4]
    double *out;            // [B x n_bins], cleared by the caller
};

// One parameter set: the phases' mass splittings as float pairs (Eq. 1: x_ee, x_21; exact
// 3-flavour: x_21, x_31, x_32; 3+1: those and x_41, x_42, x_43) and the sin^2 coefficients C
// rounded once to FP32 (a relative 6e-8, below the error of the sin^2 polynomial).
struct __align__(16) McSet {
    float dm[6], dm_lo[6], C[6];
};

__device__ McSet make_set(int mode, const double *p) {
    McSet s;
    const int n = mode == FIT_OSC_STERILE4 ? 6 : 4;
    F2 e[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float h = i < n ? (float)p[i] : 0.f;
        e[i] = f2_norm(h, i < n ? (float)(p[i] - (double)h) : 0.f);
    }
    auto sub = [](F2 a, F2 b) { return f2_add(a, F2{-b.h, -b.l}); };
    F2 d[6] = {};
    float C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (mode == FIT_OSC_EQ1) {
        d[0] = e[1];
        d[1] = e[3];
    } else {
        d[0] = e[2];
        d[1] = e[3];
        d[2] = sub(e[3], e[2]);   // dm2_32 = dm2_31 - dm2_21
    }
    if (mode == FIT_OSC_STERILE4) {
        d[3] = e[5];
        d[4] = sub(e[5], e[2]);   // dm2_42
        d[5] = sub(e[5], e[3]);   // dm2_43
        const OscCoefN<6> k = osc_coef_sterile(e);
#pragma unroll
        for (int i = 0; i < 6; ++i) C[i] = k.hi[i] + k.lo[i];
    } else {
        const F2 (&e4)[4] = reinterpret_cast<const F2 (&)[4]>(e);
        const OscCoef k = osc_coef(mode, e4);
#pragma unroll
        for (int i = 0; i < 3; ++i) C[i] = k.hi[i] + k.lo[i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        s.dm[i] = d[i].h;
        s.dm_lo[i] = d[i].l;
        s.C[i] = C[i];
    }
    return s;
}

// P(L, E) of one event for one set: 1 - sum_i C_i sin^2(x_i)
template <int NPH>
__device__ __forceinline__ float survival_ev(const McSet &S, float c_hi, float c_lo) {
    float P = 1.f;
#pragma unroll
    for (int i = 0; i < NPH; ++i) P = fmaf(-S.C[i], sin2_phase(S.dm[i], S.dm_lo[i], c_hi, c_lo), P);
    return P;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int NPH>
__global__ void __launch_bounds__(kThreads, 3) mc_spectrum_kernel(McArgs a) {
    extern __shared__ __align__(128) unsigned char dyn[];
    Stage *stage = reinterpret_cast<Stage *>(dyn);   // [2]
    __shared__ McSet sets[kMaxSets];
    __shared__ float klh[FIT_MAX_CORES], kll[FIT_MAX_CORES];
    __shared__ __align__(8) uint64_t full[2];
    // per warp and set: the open bin segment carried from one chunk to the next, its sum as a
    // float pair (hi, lo)
    __shared__ float carry_h[kThreads / 32][kMaxSets], carry_l[kThreads / 32][kMaxSets];
    __shared__ int carry_k[kThreads / 32][kMaxSets];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // a contiguous range of staging blocks per CTA, so that consecutive chunks of a warp
    // mostly fall in the same bin
    const int64_t n_blk = a.n_pad / kBlockEv;
    const int64_t blk0 = (int64_t)blockIdx.x * n_blk / gridDim.x;
    const int64_t blk1 = (int64_t)(blockIdx.x + 1) * n_blk / gridDim.x;
    auto issue = [&](int64_t blk, int s) {   // one thread: the four copies of a block
        const int64_t e = blk * kBlockEv;
        umma::mbar_arrive_expect_tx(&full[s], kStageBytes);
        umma::bulk_load(stage[s].energy, a.energy + e, sizeof(float) * kBlockEv, &full[s]);
        umma::bulk_load(stage[s].weight, a.weight + e, sizeof(float) * kBlockEv, &full[s]);
        umma::bulk_load(stage[s].bin, a.bin + e, sizeof(int) * kBlockEv, &full[s]);
        umma::bulk_load(stage[s].core, a.core + e, kBlockEv, &full[s]);
    };
    if (tid == 0) {
        umma::mbar_init(&full[0], 1);
        umma::mbar_init(&full[1], 1);
        umma::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        if (blk0 < blk1) issue(blk0, 0);
        if (blk0 + 1 < blk1) issue(blk0 + 1, 1);
    }
    for (int i = tid; i < (kThreads / 32) * kMaxSets; i += kThreads) {
        (&carry_h[0][0])[i] = 0.f;
        (&carry_l[0][0])[i] = 0.f;
        (&carry_k[0][0])[i] = -1;
    }
    const int np = a.mode == FIT_OSC_STERILE4 ? 6 : 4;
    for (int b = tid; b < a.B; b += kThreads) sets[b] = make_set(a.mode, a.params + np * b);
    if (tid < FIT_MAX_CORES) {
        klh[tid] = a.kl_hi[tid];
        kll[tid] = a.kl_lo[tid];
    }
    __syncthreads();
    int it = 0;
    for (int64_t blk = blk0; blk < blk1; ++blk, ++it) {
        const int s = it & 1;
        const bool ok = umma::mbar_wait(&full[s], (it >> 1) & 1, kWaitNs);
        // this lane's run of kV events: c = K L / (pi E) as a float pair, weight, bin
        float E[kV], w[kV];
        int cr[kV], bn[kV];
        const int o = warp * 32 * kV + lane * kV;
        if (ok) {
            const Stage &S = stage[s];
            const float4 E0 = *reinterpret_cast<const float4 *>(S.energy + o);
            const float4 E1 = *reinterpret_cast<const float4 *>(S.energy + o + 4);
            const float4 W0 = *reinterpret_cast<const float4 *>(S.weight + o);
            const float4 W1 = *reinterpret_cast<const float4 *>(S.weight + o + 4);
            const int4 B0 = *reinterpret_cast<const int4 *>(S.bin + o);
            const int4 B1 = *reinterpret_cast<const int4 *>(S.bin + o + 4);
            const uint2 C8 = *reinterpret_cast<const uint2 *>(S.core + o);
            E[0] = E0.x; E[1] = E0.y; E[2] = E0.z; E[3] = E0.w;
            E[4] = E1.x; E[5] = E1.y; E[6] = E1.z; E[7] = E1.w;
            w[0] = W0.x; w[1] = W0.y; w[2] = W0.z; w[3] = W0.w;
            w[4] = W1.x; w[5] = W1.y; w[6] = W1.z; w[7] = W1.w;
            bn[0] = B0.x; bn[1] = B0.y; bn[2] = B0.z; bn[3] = B0.w;
            bn[4] = B1.x; bn[5] = B1.y; bn[6] = B1.z; bn[7] = B1.w;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                cr[v] = (C8.x >> (8 * v)) & 0xff;
                cr[v + 4] = (C8.y >> (8 * v)) & 0xff;
            }
        }
        // every thread has read the stage (or some wait gave up): refill it with the block
        // two steps ahead
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(a.err, 1);
                // copies may still be in flight into both stages: let them land (bounded)
                umma::mbar_wait(&full[s], (it >> 1) & 1, kWaitNs);
                if (blk + 1 < blk1) umma::mbar_wait(&full[s ^ 1], ((it + 1) >> 1) & 1, kWaitNs);
            }
            __syncthreads();
            return;
        }
        if (tid == 0 && blk + 2 < blk1) issue(blk + 2, s);
        float ch_[kV], cl_[kV];
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            // 1/E as a pair: any close first guess ih, then the residual 1 - ih E (exact by
            // FMA) times ih; the pair's error is second order in that residual
            const float ih = rcp_approx(E[v]);
            const float il = fmaf(-ih, E[v], 1.f) * ih;
            const float kh = klh[cr[v]], kl = kll[cr[v]];
            ch_[v] = kh * ih;
            cl_[v] = fmaf(kh, ih, -ch_[v]) + fmaf(kh, il, kl * ih);
        }
        // the whole chunk in one bin (the common case with sorted events): plain warp sums
        const int k0 = __shfl_sync(0xffffffffu, bn[0], 0);
        if (__all_sync(0xffffffffu, bn[0] == k0 && bn[kV - 1] == k0)) {
            for (int b = 0; b < a.B; ++b) {
                const McSet S = sets[b];
                float run = 0.f;
#pragma unroll
                for (int v = 0; v < kV; ++v) run = fmaf(w[v], survival_ev<NPH>(S, ch_[v], cl_[v]), run);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) run += __shfl_xor_sync(0xffffffffu, run, off);
                if (lane == 0) {
                    const int ck = carry_k[warp][b];
                    const float c_h = carry_h[warp][b], c_l = carry_l[warp][b];
                    float nh = run, nl = 0.f;
                    if (ck == k0) {   // two-sum of the carry's high part and the chunk
                        nh = c_h + run;
                        const float bb = nh - c_h;
                        nl = c_l + ((c_h - (nh - bb)) + (run - bb));
                    } else if (ck >= 0) {
                        atomicAdd(&a.out[(int64_t)b * a.n_bins + ck], (double)c_h + (double)c_l);
                    }
                    carry_h[warp][b] = nh;
                    carry_l[warp][b] = nl;
                    carry_k[warp][b] = k0;
                }
            }
            __syncwarp();
            continue;
        }
        for (int b = 0; b < a.B; ++b) {
            const McSet S = sets[b];
            double *out = a.out + (int64_t)b * a.n_bins;
            float run = 0.f;
            int key = bn[0];
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                if (bn[v] != key) {   // bin boundary inside the run
                    if (key >= 0) atomicAdd(&out[key], (double)run);
                    run = 0.f;
                    key = bn[v];
                }
                run = fmaf(w[v], survival_ev<NPH>(S, ch_[v], cl_[v]), run);
            }
            // segmented sum over lanes with equal keys: valid keys do not decrease along the
            // lanes and the padding key -1 only follows them, so equal keys are contiguous
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float o2 = __shfl_down_sync(0xffffffffu, run, off);
                const int k2 = __shfl_down_sync(0xffffffffu, key, off);
                if (lane + off < 32 && k2 == key) run += o2;
            }
            // head lanes now hold their segment's sum; the last segment stays open as the
            // carry, the others are complete (the first one joined with the old carry when it
            // continues its bin)
            const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
            const bool head = lane == 0 || kprev != key;
            const int h_last = 31 - __clz(__ballot_sync(0xffffffffu, head));
            const int key0 = __shfl_sync(0xffffffffu, key, 0);
            const int ck = carry_k[warp][b];
            const float c_h = carry_h[warp][b], c_l = carry_l[warp][b];
            const bool merge = ck == key0;
            if (lane == 0 && !merge && ck >= 0) atomicAdd(&out[ck], (double)c_h + (double)c_l);
            if (head && lane != h_last && key >= 0)
                atomicAdd(&out[key], (double)run + ((lane == 0 && merge) ? (double)c_h + (double)c_l : 0.0));
            __syncwarp();
            if (lane == h_last) {
                float nh = run, nl = 0.f;
                if (lane == 0 && merge) {   // two-sum of the carry's high part and the run
                    nh = c_h + run;
                    const float bb = nh - c_h;
                    nl = c_l + ((c_h - (nh - bb)) + (run - bb));
                }
                carry_h[warp][b] = nh;
                carry_l[warp][b] = nl;
                carry_k[warp][b] = key;
            }
            __syncwarp();
        }
    }
    // close the open segments
    for (int b = lane; b < a.B; b += 32) {
        const int ck = carry_k[warp][b];
        if (ck >= 0) atomicAdd(&a.out[(int64_t)b * a.n_bins + ck], (double)carry_h[warp][b] + (double)carry_l[warp][b]);
    }
}

}  // namespace
}  // namespace fitcore

extern "C" {

int fit_mc_create(int osc_mode, int n_cores, const double *core_L, int64_t n_events, const float *energy,
                  const uint8_t *core, const float *weight, const int *bin, int n_bins, fit_mc **out) {
    if (!out || (osc_mode != FIT_OSC_EQ1 && osc_mode != FIT_OSC_VACUUM3 && osc_mode != FIT_OSC_STERILE4) ||
        n_cores < 1 ||
        n_cores > FIT_MAX_CORES || !core_L || n_events < 0 || n_bins < 1 ||
        (n_events > 0 && (!energy || !core || !weight || !bin)))
        return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mc_create: bad argument");
    // events must be sorted by bin, with cores in range and positive energies
    for (int64_t e = 0; e < n_events; ++e) {
        if (core[e] >= n_cores || !(energy[e] > 0.f) || bin[e] < 0 || bin[e] >= n_bins ||
            (e > 0 && bin[e] < bin[e - 1]))
            return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mc_create: event " + std::to_string(e) +
                                                         " out of range or not sorted by bin");
    }
    fit_mc *m = new fit_mc();
    m->mode = osc_mode;
    m->n_cores = n_cores;
    m->n_bins = n_bins;
    m->n_events = n_events;
    const double K_OVER_PI = 1.266932679815373 / 3.14159265358979323846;   // dm2 L / (4E) per pi
    for (int c = 0; c < n_cores; ++c) {
        const double kl = K_OVER_PI * core_L[c];
        m->kl_hi[c] = (float)kl;
        m->kl_lo[c] = (float)(kl - (double)m->kl_hi[c]);
    }
    // padded to whole staging blocks: energy 1, weight 0, core 0, bin -1
    const int64_t kb = fitcore::kBlockEv;
    const int64_t np = std::max<int64_t>(1, (n_events + kb - 1) / kb) * kb;
    m->n_pad = np;
    if (cudaMalloc(&m->energy, sizeof(float) * np) || cudaMalloc(&m->weight, sizeof(float) * np) ||
        cudaMalloc(&m->core, np) || cudaMalloc(&m->bin, sizeof(int) * np) ||
        cudaMalloc(&m->err, sizeof(int))) {
        cudaGetLastError();
        fit_mc_destroy(m);
        return fitcore_fail(FIT_ERR_OOM, "fit_mc_create: device allocation");
    }
    const int64_t tail = np - n_events;
    const std::vector<float> ones((size_t)tail, 1.f);
    if ((n_events > 0 &&
         (cudaMemcpy(m->energy, energy, sizeof(float) * n_events, cudaMemcpyDefault) ||
          cudaMemcpy(m->weight, weight, sizeof(float) * n_events, cudaMemcpyDefault) ||
          cudaMemcpy(m->core, core, n_events, cudaMemcpyDefault) ||
          cudaMemcpy(m->bin, bin, sizeof(int) * n_events, cudaMemcpyDefault))) ||
        cudaMemcpy(m->energy + n_events, ones.data(), sizeof(float) * tail, cudaMemcpyHostToDevice) ||
        cudaMemset(m->weight + n_events, 0, sizeof(float) * tail) ||
        cudaMemset(m->core + n_events, 0, tail) ||
        cudaMemset(m->bin + n_events, 0xff, sizeof(int) * tail) || cudaMemset(m->err, 0, sizeof(int))) {
        cudaGetLastError();
        fit_mc_destroy(m);
        return fitcore_fail(FIT_ERR_CUDA, "fit_mc_create: upload");
    }
    *out = m;
    return FIT_OK;
}

void fit_mc_destroy(fit_mc *m) {
    if (!m) return;
    for (void *p : {(void *)m->energy, (void *)m->weight, (void *)m->core, (void *)m->bin, (void *)m->err})
        if (p) cudaFree(p);
    delete m;
}

int fit_mc_status(fit_mc *m) {
    if (!m) return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mc_status: null");
    int e = 0;
    if (cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fitcore_fail(FIT_ERR_CUDA, "fit_mc_status: read");
    return e ? fitcore_fail(FIT_ERR_CUDA, "fit_mc_spectrum: a staging wait ran out of time") : FIT_OK;
}

int fit_mc_spectrum(fit_mc *m, int B, const double *params, double *out, void *stream) {
    if (!m || B < 0 || B > fitcore::kMaxSets || (B > 0 && (!params || !out)))
        return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_mc_spectrum: bad argument (B <= 64)");
    if (B == 0) return FIT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaPointerAttributes pa, po;
    const bool p_dev = cudaPointerGetAttributes(&pa, params) == cudaSuccess &&
                       (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    const bool o_dev = cudaPointerGetAttributes(&po, out) == cudaSuccess &&
                       (po.type == cudaMemoryTypeDevice || po.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    double *pd = nullptr, *od = nullptr;
    int rc = FIT_OK;
    const size_t np = m->mode == FIT_OSC_STERILE4 ? 6 : 4;   // survival parameters per set
    if (!p_dev && (cudaMallocAsync(&pd, sizeof(double) * np * B, s) ||
                   cudaMemcpyAsync(pd, params, sizeof(double) * np * B, cudaMemcpyHostToDevice, s)))
        rc = fitcore_fail(FIT_ERR_CUDA, "fit_mc_spectrum: parameters");
    if (!rc && !o_dev && cudaMallocAsync(&od, sizeof(double) * (size_t)B * m->n_bins, s))
        rc = fitcore_fail(FIT_ERR_OOM, "fit_mc_spectrum: output");
    double *outd = o_dev ? out : od;
    if (!rc && cudaMemsetAsync(outd, 0, sizeof(double) * (size_t)B * m->n_bins, s))
        rc = fitcore_fail(FIT_ERR_CUDA, "fit_mc_spectrum: clear");
    if (!rc && m->n_events > 0) {
        fitcore::McArgs a;
        a.energy = m->energy;
        a.weight = m->weight;
        a.core = m->core;
        a.bin = m->bin;
        a.n_pad = m->n_pad;
        a.err = m->err;
        a.n_bins = m->n_bins;
        a.mode = m->mode;
        a.n_cores = m->n_cores;
        a.B = B;
        for (int c = 0; c < FIT_MAX_CORES; ++c) {
            a.kl_hi[c] = m->kl_hi[c];
            a.kl_lo[c] = m->kl_lo[c];
        }
        a.params = p_dev ? params : pd;
        a.out = outd;
        // one wave of resident blocks, each with a contiguous range of staging blocks
        const void *fn = m->mode == FIT_OSC_EQ1       ? (const void *)fitcore::mc_spectrum_kernel<2>
                         : m->mode == FIT_OSC_VACUUM3 ? (const void *)fitcore::mc_spectrum_kernel<3>
                                                      : (const void *)fitcore::mc_spectrum_kernel<6>;
        const int dyn = 2 * (int)sizeof(fitcore::Stage);
        int dev = 0, n_sm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, fitcore::kThreads, dyn);
        const int64_t n_blk = m->n_pad / fitcore::kBlockEv;
        const int64_t wave = (int64_t)std::max(1, n_sm) * std::max(1, per_sm);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_blk, wave));
        void *args[] = {&a};
        cudaLaunchKernel(fn, dim3(grid), dim3(fitcore::kThreads), args, dyn, s);
        fitcore_count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = fitcore_fail(FIT_ERR_CUDA, std::string("fit_mc_spectrum: ") + cudaGetErrorString(e));
    }
    if (!rc && !o_dev &&
        cudaMemcpyAsync(out, od, sizeof(double) * (size_t)B * m->n_bins, cudaMemcpyDeviceToHost, s))
        rc = fitcore_fail(FIT_ERR_CUDA, "fit_mc_spectrum: copy back");
    if (pd) cudaFreeAsync(pd, s);
    if (od) cudaFreeAsync(od, s);
    if (!rc && !o_dev && cudaStreamSynchronize(s) != cudaSuccess)
        rc = fitcore_fail(FIT_ERR_CUDA, "fit_mc_spectrum: sync");
    return rc;
}

}  // extern "C"
