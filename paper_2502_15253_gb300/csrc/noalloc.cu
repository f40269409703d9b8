// fit_model_eval_noalloc: the batched -2lnL + gradient evaluation for callers that cannot
// allocate device memory: a host application that owns a fixed device-memory budget and
// hands out all buffers itself, a plugin running under another framework's allocator that
// forbids direct cudaMalloc / cudaFree, or a latency-critical loop that must not call into
// the allocator. Its per-block workspace lives in a fixed, file-scope device array instead
// of being allocated per call.
#include <algorithm>
#include <mutex>
#include <string>

#include "kernels.cuh"

namespace {

// 16 MiB of workspace, held by every GPU that loads the library until the process exits.
// Nothing in it has to start at zero: each evaluation writes every workspace entry it reads.
constexpr size_t kScratchFloats = size_t(4) << 20;
__device__ __align__(256) float g_eval_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
float *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

}  // namespace

int fitcore_noalloc_fail(int code, const std::string &msg);  // capi.cu (thread-local message)

extern "C" int fit_model_eval_noalloc(fit_model *model, int B, const double *theta, const float *data,
                                      const uint32_t *masks, double *nll_out, float *grad_out,
                                      int *status_out, void *stream);

// The model's device layout lives in capi.cu; it hands the pieces needed here through this hook.
int fitcore_model_device(fit_model *model, const fitcore::DevModel **dev, const fitcore::DevModel **host,
                         int *device);
int fitcore_raise_eval_smem(size_t bytes);
void fitcore_count_launch();

// Host-side decision on where the call's memory lives (no CUDA call): the model must be on the
// current device, and every buffer either managed memory or device memory of that device
// (another GPU's memory is not readable there without peer access). types[i] / devices[i]:
// the cudaMemoryType and device of buffer i. Returns FIT_OK or FIT_ERR_INVALID_ARG.
extern "C" int fitcore_noalloc_check_devices(int model_device, int current_device, int n, const int *types,
                                             const int *devices) {
    if (model_device != current_device) return FIT_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (types[i] == cudaMemoryTypeManaged) continue;
        if (types[i] != cudaMemoryTypeDevice || devices[i] != current_device) return FIT_ERR_INVALID_ARG;
    }
    return FIT_OK;
}

extern "C" int fit_model_eval_noalloc(fit_model *model, int B, const double *theta, const float *data,
                                      const uint32_t *masks, double *nll_out, float *grad_out,
                                      int *status_out, void *stream) {
    if (!model || !theta || !nll_out || B < 0)
        return fitcore_noalloc_fail(FIT_ERR_INVALID_ARG, "fit_model_eval_noalloc: bad argument");
    if (B == 0) return FIT_OK;
    const fitcore::DevModel *dev = nullptr, *h = nullptr;
    int model_device = -1;
    fitcore_model_device(model, &dev, &h, &model_device);
    const size_t per_block = (size_t)h->ws_eval_floats;
    if (per_block > kScratchFloats)
        return fitcore_noalloc_fail(FIT_ERR_INVALID_ARG,
                                    "fit_model_eval_noalloc: the model needs " + std::to_string(per_block * 4) +
                                        " bytes of workspace per block, more than the 16 MiB scratch");
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
        cudaGetLastError();
        return fitcore_noalloc_fail(FIT_ERR_CUDA, "fit_model_eval_noalloc: cudaGetDevice");
    }
    float *scratch = nullptr;
    {
        // first call on this device: resolve the array's device address (device is current)
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[device]) {
            cudaError_t e = cudaGetSymbolAddress((void **)&g_scratch_addr[device], g_eval_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                g_scratch_addr[device] = nullptr;
                return fitcore_noalloc_fail(FIT_ERR_CUDA, std::string("fit_model_eval_noalloc: cudaGetSymbolAddress: ") +
                                                              cudaGetErrorString(e));
            }
        }
        scratch = g_scratch_addr[device];
    }
    // every buffer must already be memory of the current device (or managed): staging a host
    // buffer would allocate, and another GPU's memory is not readable here
    const void *ptrs[] = {theta, data, masks, nll_out, grad_out, status_out};
    int types[6], devices[6], n = 0;
    for (const void *p : ptrs) {
        if (!p) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return fitcore_noalloc_fail(FIT_ERR_INVALID_ARG, "fit_model_eval_noalloc: every buffer must be device memory");
        }
        types[n] = (int)a.type;
        devices[n] = a.device;
        ++n;
    }
    if (model_device != device)
        return fitcore_noalloc_fail(FIT_ERR_INVALID_ARG,
                                    "fit_model_eval_noalloc: the model was created on device " +
                                        std::to_string(model_device) + ", the current device is " +
                                        std::to_string(device));
    if (fitcore_noalloc_check_devices(model_device, device, n, types, devices) != FIT_OK)
        return fitcore_noalloc_fail(FIT_ERR_INVALID_ARG,
                                    "fit_model_eval_noalloc: every buffer must be device memory of the current "
                                    "device (or managed memory)");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return fitcore_noalloc_fail(FIT_ERR_CUDA, "fit_model_eval_noalloc: device attribute");
    }
    const int threads = 256;
    const size_t smem = fitcore::eval_smem_bytes(*h, false);
    // (raised only: the attribute is shared with fit_model_eval's launches in other threads)
    if (fitcore_raise_eval_smem(smem) != FIT_OK) {
        cudaGetLastError();
        return fitcore_noalloc_fail(FIT_ERR_CUDA, "fit_model_eval_noalloc: cudaFuncSetAttribute");
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fitcore::eval_kernel, threads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return fitcore_noalloc_fail(FIT_ERR_CUDA, "fit_model_eval_noalloc: occupancy");
    }
    // one workspace slice per block: the grid never exceeds what the scratch holds
    const int slices = (int)(kScratchFloats / per_block);
    const int grid = std::max(1, std::min(std::min(B, per_sm * sms), slices));
    fitcore::eval_kernel<<<grid, threads, smem, (cudaStream_t)stream>>>(
        dev, B, theta, data, masks, nll_out, grad_out, nullptr, status_out, scratch, 0);
    fitcore_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fitcore_noalloc_fail(FIT_ERR_CUDA, std::string("fit_model_eval_noalloc: launch: ") + cudaGetErrorString(e));
    return FIT_OK;
}
