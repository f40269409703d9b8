// Tensor-core GEMM (see gemm_tc.cuh). One CTA of 4 warps computes a 128 x n_tile output tile:
// warp 0 (one thread) streams 128-byte-wide K slices of A and B into a 4-stage shared-memory
// ring with TMA (128-byte swizzle), warp 1 (one thread) issues tcgen05.mma into a tensor-memory
// accumulator and frees each stage with tcgen05.commit, and all four warps then read the
// accumulator rows (warp w owns lanes 32w..32w+31) with tcgen05.ld for the fused epilogue.
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "../../include/fitcore.h"
#include "gemm_tc.cuh"
#include "umma.cuh"

int fitcore_fail(int code, const std::string &msg);   // capi.cu: sets the error string
void fitcore_count_launch();

namespace fitcore {

namespace {

constexpr int kStages = 3;
constexpr int kRowBytes = 128;           // one K slice: 128 bytes per row
constexpr int kTileM = 128;
constexpr int kNumSMs = 152;
constexpr int kThreads = 256;   // 8 warps: warp w reads accumulator lanes 32 (w % 4).. in the epilogue
constexpr uint64_t kMaxTries = 2000000000ull;  // bound of every barrier wait: 2 s

__device__ int g_gemm_err;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

template <bool TF32>
__global__ void __launch_bounds__(kThreads, 2)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                   int K, int n_tile, int kt_per, GemmOut out, int *err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int a_bytes = kTileM * kRowBytes;
    const int b_bytes = n_tile * kRowBytes;
    const int stage_bytes = a_bytes + b_bytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * stage_bytes);
    uint64_t *empty = full + kStages;
    uint64_t *done = empty + kStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kTileM, n0 = blockIdx.y * n_tile;
    const int kel = TF32 ? 32 : 64;
    // split K: this CTA reduces K tiles [kt0, kt0 + ktiles) and adds its partial product
    const int kt0 = blockIdx.z * kt_per;
    const int ktiles = min(kt_per, (K + kel - 1) / kel - kt0);
    const bool split = gridDim.z > 1;
    uint32_t ncols = 32;
    while ((int)ncols < n_tile) ncols <<= 1;

    if (warp == 0) umma::tmem_alloc(tmem_slot, ncols);
    if (threadIdx.x == 32) {
        for (int s = 0; s < kStages; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(done, 1);
        umma::fence_mbar_init();
    }
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- producer: TMA slices of A (128 rows) and B (n_tile rows) ---------------------
        umma::prefetch_tmap(&tmA);
        umma::prefetch_tmap(&tmB);
        for (int t = 0; t < ktiles; ++t) {
            const int s = t % kStages;
            if (t >= kStages && !umma::mbar_wait(&empty[s], ((t / kStages) - 1) & 1, kMaxTries)) {
                atomicOr(err, 1);
                break;
            }
            uint8_t *sa = smem + s * stage_bytes;
            umma::mbar_arrive_expect_tx(&full[s], stage_bytes);
            umma::tma_load_2d(sa, &tmA, &full[s], (kt0 + t) * kel, m0);
            umma::tma_load_2d(sa + a_bytes, &tmB, &full[s], (kt0 + t) * kel, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: 4 MMAs of 32 bytes of K per slice --------------------------------
        const uint32_t idesc = umma::idesc_f32(TF32 ? 2u : 1u, kTileM, n_tile);
        for (int t = 0; t < ktiles; ++t) {
            const int s = t % kStages;
            if (!umma::mbar_wait(&full[s], (t / kStages) & 1, kMaxTries)) {
                atomicOr(err, 2);
                break;
            }
            umma::tc_fence_after();
            const uint32_t sa = umma::smem_u32(smem + s * stage_bytes);
            const uint64_t da = umma::desc_kmajor_sw128(sa), db = umma::desc_kmajor_sw128(sa + a_bytes);
#pragma unroll
            for (int kk = 0; kk < kRowBytes / 32; ++kk)
                umma::mma<TF32>(tmem, da + 2 * kk, db + 2 * kk, idesc, (t > 0 || kk > 0) ? 1u : 0u);
            umma::mma_commit(&empty[s]);
        }
        umma::mma_commit(done);
    }
    __syncwarp();

    // ---- epilogue ------------------------------------------------------------------------
    // Phase 1: warp w reads its 32 accumulator lanes (rows) with tcgen05.ld, 16 columns per
    // load, and parks them in a shared-memory tile laid over the (now idle) operand ring (row
    // pitch n_tile + 1 floats: the 32 rows of a store land in 32 different banks). Phase 2:
    // the warps walk the tile row by row with the lanes along the columns, so every global
    // load, store or atomic of the fused epilogue is coalesced.
    bool ready = umma::mbar_wait(done, 0, kMaxTries);
    ready = __syncthreads_and(ready) != 0;
    if (!ready && threadIdx.x == 0) atomicOr(err, 4);
    umma::tc_fence_after();
    if (ready) {
        float *tile = reinterpret_cast<float *>(smem);
        const int ldt = n_tile + 1;
        const int quad = warp & 3, half = warp >> 2, nwarps = kThreads / 32;
        const int r = quad * 32 + lane;
        // warps w and w + 4 share a lane quadrant and split its columns
        for (int c = half * 16; c < n_tile; c += 32) {
            float v[16];
            umma::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) tile[r * ldt + c + i] = v[i];
        }
        __syncthreads();
        const int n_valid = min(n_tile, N - n0);
        for (int rr = warp; rr < kTileM; rr += nwarps) {
            const int row = m0 + rr;
            if (row >= M) break;
            const float *trow = tile + rr * ldt;
            // the aux operand of the GELU' epilogue is loaded four strides ahead of its use
            float ax[4] = {0.f, 0.f, 0.f, 0.f};
            if (out.epi == EPI_DGELU) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = lane + 32 * q;
                    if (c < n_valid) ax[q] = out.aux[(int64_t)row * out.ldaux + n0 + c];
                }
            }
            for (int c0 = 0; c0 < n_valid; c0 += 128) {
                float axn[4] = {0.f, 0.f, 0.f, 0.f};
                if (out.epi == EPI_DGELU) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = c0 + 128 + lane + 32 * q;
                        if (c < n_valid) axn[q] = out.aux[(int64_t)row * out.ldaux + n0 + c];
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = c0 + lane + 32 * q;
                    if (c >= n_valid) continue;
                    const int n = n0 + c;
                    const float d = trow[c];
                    const int64_t oc = (int64_t)row * out.ldc + n;
                    switch (out.epi) {
                        case EPI_F32:
                            if (split)
                                atomicAdd(&out.C[oc], d);
                            else
                                out.C[oc] = d;
                            break;
                        case EPI_BIAS_F32:
                            out.C[oc] = d + out.bias[n];
                            break;
                        case EPI_BIAS_GELU: {
                            const float pre = d + out.bias[n];
                            out.C[oc] = pre;
                            out.Y[(int64_t)row * out.ldy + n] = __float2bfloat16(gelu(pre));
                            break;
                        }
                        case EPI_DGELU:
                            out.Y[(int64_t)row * out.ldy + n] = __float2bfloat16(d * gelu_grad(ax[q]));
                            break;
                        case EPI_F32_ADD:
                            if (split)
                                atomicAdd(&out.C[oc], d);
                            else
                                out.C[oc] += d;
                            break;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) ax[q] = axn[q];
            }
        }
    }
    umma::tc_fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mutex;

int get_encoder() {
    std::lock_guard<std::mutex> lock(g_encode_mutex);
    if (g_encode) return FIT_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return fitcore_fail(FIT_ERR_CUDA, "tensor-core GEMM: cuTensorMapEncodeTiled not available");
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return FIT_OK;
}

// Tensor map of a row-major [rows x K] matrix read in boxes of (128 bytes of K) x box_rows.
int make_map(CUtensorMap *map, bool tf32, const void *base, int rows, int K, int ld, int box_rows) {
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const int esz = tf32 ? 4 : 2;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
    const cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fitcore_fail(FIT_ERR_INVALID_ARG, "tensor-core GEMM: cuTensorMapEncodeTiled failed (" +
                                                             std::to_string((int)r) + ")");
    return FIT_OK;
}

}  // namespace

int tc_gemm(bool tf32, int M, int N, int K, const void *A, int lda, const void *B, int ldb, const GemmOut &out,
            cudaStream_t stream, int *err_dev) {
    if (M <= 0 || N <= 0 || K <= 0 || !A || !B)
        return fitcore_fail(FIT_ERR_INVALID_ARG, "tensor-core GEMM: empty or null operand");
    const int esz = tf32 ? 4 : 2;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((size_t)lda * esz) % 16 || ((size_t)ldb * esz) % 16 ||
        lda < K || ldb < K)
        return fitcore_fail(FIT_ERR_INVALID_ARG, "tensor-core GEMM: operands must be 16-byte aligned rows");
    int rc = get_encoder();
    if (rc) return rc;
    // Tiles of 128 x (<= 128): a 3-stage ring of 96 KB, so two CTAs share an SM and one's
    // epilogue overlaps the other's main loop.
    const int ntn = (N + 127) / 128;
    const int n_tile = (((N + ntn - 1) / ntn) + 15) / 16 * 16;
    // Output tiles that cannot fill the SMs (a weight gradient: small M x N, K = the batch)
    // split K over grid z; the partial products are added with atomics (plain FP32 outputs).
    const int mt = (M + kTileM - 1) / kTileM;
    const int ktiles = (K + (tf32 ? 32 : 64) - 1) / (tf32 ? 32 : 64);
    int splits = 1;
    if (out.epi == EPI_F32 || out.epi == EPI_F32_ADD)
        while (mt * ntn * splits * 2 <= 2 * kNumSMs && ktiles / (splits * 2) >= 4) splits *= 2;
    const int kt_per = (ktiles + splits - 1) / splits;
    splits = (ktiles + kt_per - 1) / kt_per;   // no empty split
    CUtensorMap ta, tb;
    if ((rc = make_map(&ta, tf32, A, M, K, lda, kTileM))) return rc;
    if ((rc = make_map(&tb, tf32, B, N, K, ldb, n_tile))) return rc;
    if (!err_dev) {
        if (cudaGetSymbolAddress((void **)&err_dev, g_gemm_err) != cudaSuccess) {
            cudaGetLastError();
            return fitcore_fail(FIT_ERR_CUDA, "tensor-core GEMM: error flag");
        }
    }
    const size_t smem = 1024 + (size_t)kStages * (kTileM + n_tile) * kRowBytes + (2 * kStages + 1) * 8 + 16;
    auto kern = tf32 ? tc_gemm_kernel<true> : tc_gemm_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return fitcore_fail(FIT_ERR_CUDA, "tensor-core GEMM: shared memory attribute");
    }
    if (splits > 1 && out.epi == EPI_F32) {
        // C = 0 first: rows of ldc floats (the row tails beyond N are left as they were)
        cudaError_t e = (out.ldc == N) ? cudaMemsetAsync(out.C, 0, sizeof(float) * (size_t)M * N, stream)
                                       : cudaMemset2DAsync(out.C, sizeof(float) * (size_t)out.ldc, 0,
                                                           sizeof(float) * (size_t)N, M, stream);
        if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, "tensor-core GEMM: clearing C");
    }
    dim3 grid(mt, ntn, splits);
    kern<<<grid, kThreads, smem, stream>>>(ta, tb, M, N, K, n_tile, kt_per, out, err_dev);
    fitcore_count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fitcore_fail(FIT_ERR_CUDA, std::string("tensor-core GEMM launch: ") + cudaGetErrorString(e));
    return FIT_OK;
}

// Reads and clears the GEMM pipeline-timeout flag (synchronises the device).
int tc_gemm_take_error() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_gemm_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    const int z = 0;
    cudaMemcpyToSymbol(g_gemm_err, &z, sizeof(int));
    return v;
}

}  // namespace fitcore
