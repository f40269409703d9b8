// Tensor-core GEMM (see gemm_tc.cuh). Persistent and warp-specialised: each CTA (one per SM,
// 20 warps) walks a static list of work units (128-row x n_tile output tiles, optionally a
// share of K). Warp 0 (one thread) streams 128-byte-wide K slices of A and B into a shared-
// memory ring with TMA (128-byte swizzle); warp 1 (one thread) issues tcgen05.mma into one of
// two tensor-memory accumulators and frees each ring stage with tcgen05.commit; warps 4-19
// drain the other accumulator (warp w reads lanes 32 (w % 4).., four warps per lane quadrant
// taking every fourth 16-column chunk) through the fused epilogue and hand it back. So one
// tile's epilogue runs while the next tile's products accumulate.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/fitcore.h"
#include "gemm_tc.cuh"
#include "umma.cuh"

int fitcore_fail(int code, const std::string &msg);   // capi.cu: sets the error string
void fitcore_count_launch();

namespace fitcore {

namespace {

constexpr int kRowBytes = 128;           // one K slice: 128 bytes per row
constexpr int kTileM = 128;
constexpr int kNumSMs = 152;
constexpr int kThreads = 640;            // 20 warps: producer, MMA, allocator, spare, 16 epilogue
constexpr int kEpiWarp0 = 4;
constexpr int kEpiWarps = 16;
constexpr int kRingBytes = 144 * 1024;   // operand ring budget (+ 64 KB of epilogue staging)
constexpr int kMaxStages = 8;
constexpr uint64_t kWaitNs = 2000000000ull;  // bound of every barrier wait: 2 s

__device__ int g_gemm_err;

// Standard normal CDF Phi(x) = (1 + erf(x / sqrt 2)) / 2 and density phi(x), with erfc from the
// rational approximation of Abramowitz & Stegun, Handbook of Mathematical Functions, 7.1.26
// (Hastings): erfc(z) = (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-z^2), t = 1 / (1 + p z),
// z >= 0, absolute error <= 1.5e-7 (the level of FP32 rounding of erf itself). For x < 0 Phi
// is formed directly as erfc(|x| / sqrt 2) / 2, so the left tail has no cancellation. The GELU
// of the network is x Phi(x) ("exact erf" form), its derivative Phi(x) + x phi(x); both share
// the one exponential.
__device__ __forceinline__ void phi_pair(float x, float &cdf, float &e) {
    const float z = fabsf(x) * 0.70710678118654752f;
    const float t = __fdividef(1.f, fmaf(0.3275911f, z, 1.f));
    const float q = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                             0.254829592f);
    e = __expf(-0.5f * x * x);
    const float h = 0.5f * q * e;   // erfc(z) / 2
    cdf = x < 0.f ? h : 1.f - h;
}

__device__ __forceinline__ float gelu(float x) {
    float c, e;
    phi_pair(x, c, e);
    return x * c;
}

__device__ __forceinline__ float gelu_grad(float x) {
    float c, e;
    phi_pair(x, c, e);
    return fmaf(x * 0.39894228040143268f, e, c);
}

// Bounded wait that also gives up as soon as another role of the CTA has given up.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (umma::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = umma::now_ns();
    while (true) {
        if (umma::mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (umma::now_ns() - t0 > kWaitNs) {
            *abort_flag = 1;
            return false;
        }
    }
}

struct Plan {
    int n_tile, ntn, mt, splits, kt_per, units, stages, acc_cols;
};

// Packs two floats as bf16 (round to nearest) into one 32-bit word, the first in the low half.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// Per-warp staging of one 32-row x 16-column chunk (4 KB): the FP32 tile (C, or the aux operand
// on its way in), the bf16 tile (Y) and the transposed bf16 tile (Yt). Threads own rows (the
// tensor-memory layout); the warp then writes the tiles out in row segments (64 / 32 bytes,
// eight or sixteen rows per instruction) or, for Yt, in 64-byte column segments. The FP32 and
// bf16 tiles are XOR-swizzled by 16-byte unit so that both the row-per-thread accesses and the
// warp-wide segment accesses take the minimum number of shared-memory wavefronts.
struct EpiStage {
    float4 c[32 * 4];      // row r, unit j (4 floats) at r * 4 + (j ^ ((r >> 1) & 3))
    uint4 y[32 * 2];       // row r, unit j (8 bf16) at r * 2 + (j ^ ((r >> 2) & 1))
    uint16_t t[16 * 32];   // column i, row r at i * 32 + r
};
__device__ __forceinline__ int cidx(int r, int j) { return r * 4 + (j ^ ((r >> 1) & 3)); }
__device__ __forceinline__ int yidx(int r, int j) { return r * 2 + (j ^ ((r >> 2) & 1)); }

// Writes the staged FP32 tile (rows [0, nrow), columns [0, nv)) to C at (row0, n): a warp
// instruction covers eight rows of 16 floats. split: atomic accumulation; add: C += tile.
__device__ __forceinline__ void flush_c(const EpiStage &st, float *C, int64_t ldc, int row0, int n, int nrow, int nv,
                                        bool vec, bool split, bool add) {
    const int lane = threadIdx.x & 31, j = lane & 3;
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        const int rr = it * 8 + (lane >> 2);
        if (rr >= nrow || 4 * j >= nv) continue;
        const float4 q = st.c[cidx(rr, j)];
        float *g = C + (int64_t)(row0 + rr) * ldc + n + 4 * j;
        if (vec && 4 * j + 4 <= nv) {
            float4 *g4 = reinterpret_cast<float4 *>(g);
            if (split) {
                atomicAdd(g4, q);
            } else if (add) {
                const float4 o = *g4;
                *g4 = make_float4(o.x + q.x, o.y + q.y, o.z + q.z, o.w + q.w);
            } else {
                *g4 = q;
            }
        } else {
            const float e[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (4 * j + k >= nv) break;
                if (split)
                    atomicAdd(g + k, e[k]);
                else if (add)
                    g[k] += e[k];
                else
                    g[k] = e[k];
            }
        }
    }
}

// Writes the staged bf16 tile to Y at (row0, n): a warp instruction covers sixteen rows.
__device__ __forceinline__ void flush_y(const EpiStage &st, __nv_bfloat16 *Y, int64_t ldy, int row0, int n, int nrow,
                                        int nv, bool vec) {
    const int lane = threadIdx.x & 31, j = lane & 1;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int rr = it * 16 + (lane >> 1);
        if (rr >= nrow || 8 * j >= nv) continue;
        const uint4 q = st.y[yidx(rr, j)];
        __nv_bfloat16 *g = Y + (int64_t)(row0 + rr) * ldy + n + 8 * j;
        if (vec && 8 * j + 8 <= nv) {
            *reinterpret_cast<uint4 *>(g) = q;
        } else {
            const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (8 * j + k >= nv) break;
                g[k] = __ushort_as_bfloat16((unsigned short)(wd[k >> 1] >> (16 * (k & 1))));
            }
        }
    }
}

// Writes the staged transposed tile to Yt at (n, row0): Yt[(n + i) * ldyt + row0 + r]; a warp
// instruction covers eight columns of 32 rows.
__device__ __forceinline__ void flush_yt(const EpiStage &st, __nv_bfloat16 *Yt, int64_t ldyt, int row0, int n,
                                         int nrow, int nv, bool vec) {
    const int lane = threadIdx.x & 31, j = lane & 3;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int cc = it * 8 + (lane >> 2);
        if (cc >= nv || 8 * j >= nrow) continue;
        __nv_bfloat16 *g = Yt + (int64_t)(n + cc) * ldyt + row0 + 8 * j;
        const uint16_t *src = st.t + cc * 32 + 8 * j;
        if (vec && 8 * j + 8 <= nrow) {
            *reinterpret_cast<uint4 *>(g) = *reinterpret_cast<const uint4 *>(src);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (8 * j + k >= nrow) break;
                g[k] = __ushort_as_bfloat16(src[k]);
            }
        }
    }
}

// Stores this thread's 16 bf16 values (packed pairs) into its row of the bf16 tile and its
// column of the transposed tile.
__device__ __forceinline__ void stage_bf16(EpiStage &st, const uint32_t (&w)[8], bool with_t) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 2; ++j) st.y[yidx(lane, j)] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
    if (with_t) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            st.t[(2 * k) * 32 + lane] = (uint16_t)(w[k] & 0xFFFFu);
            st.t[(2 * k + 1) * 32 + lane] = (uint16_t)(w[k] >> 16);
        }
    }
}

// v[i] += bias[n + i] for the valid columns (four 16-byte loads when aligned and complete)
__device__ __forceinline__ void add_bias(const GemmOut &out, int n, int nv, float (&v)[16]) {
    if (nv == 16 && (out.vec & 16)) {
        const float4 *b4 = reinterpret_cast<const float4 *>(out.bias + n);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 b = __ldg(b4 + j);
            v[4 * j] += b.x;
            v[4 * j + 1] += b.y;
            v[4 * j + 2] += b.z;
            v[4 * j + 3] += b.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] += (i < nv) ? __ldg(out.bias + n + i) : 0.f;
    }
}

// The aux operand of the GELU' epilogue for one chunk, read coalesced (eight rows of 16 floats
// per warp instruction, four independent loads per thread) into registers; the caller issues
// it a chunk ahead so that its latency hides behind the previous chunk's arithmetic.
__device__ __forceinline__ void load_aux(const GemmOut &out, int row0, int n, int nrow, int nv, float4 (&q)[4]) {
    const int lane = threadIdx.x & 31, j = lane & 3;
    const float *base = out.aux + (int64_t)row0 * out.ldaux + n + 4 * j;
    if ((out.vec & 4) && nrow == 32 && nv == 16) {
#pragma unroll
        for (int it = 0; it < 4; ++it)
            q[it] = __ldg(reinterpret_cast<const float4 *>(base + (int64_t)(it * 8 + (lane >> 2)) * out.ldaux));
        return;
    }
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        const int rr = it * 8 + (lane >> 2);
        float e[4] = {0.f, 0.f, 0.f, 0.f};
        if (rr < nrow) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (4 * j + k < nv) e[k] = __ldg(base + (int64_t)rr * out.ldaux + k);
        }
        q[it] = make_float4(e[0], e[1], e[2], e[3]);
    }
}

__device__ __forceinline__ void stage_aux(EpiStage &st, const float4 (&q)[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int it = 0; it < 4; ++it) st.c[cidx(it * 8 + (lane >> 2), lane & 3)] = q[it];
    __syncwarp();
}

// Epilogue of one 32-row x 16-column chunk: rows row0 + [0, nrow), columns n + [0, nv); v holds
// this thread's row (row0 + lane) of the accumulator.
__device__ __forceinline__ void epi_chunk(const GemmOut &out, EpiStage &st, bool split, int row0, int n, int nrow,
                                          int nv, float (&v)[16]) {
    const int lane = threadIdx.x & 31;
    const bool vc = out.vec & 1, vy = out.vec & 2, vt = out.vec & 8;
    switch (out.epi) {
        case EPI_F32:
        case EPI_F32_ADD:
        case EPI_BIAS_F32: {
            if (out.epi == EPI_BIAS_F32) add_bias(out, n, nv, v);
#pragma unroll
            for (int j = 0; j < 4; ++j) st.c[cidx(lane, j)] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            __syncwarp();
            flush_c(st, out.C, out.ldc, row0, n, nrow, nv, vc, split, out.epi == EPI_F32_ADD);
            break;
        }
        case EPI_BIAS_GELU: {
            add_bias(out, n, nv, v);
            uint32_t w[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) w[k] = pack_bf16(gelu(v[2 * k]), gelu(v[2 * k + 1]));
#pragma unroll
            for (int j = 0; j < 4; ++j) st.c[cidx(lane, j)] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            stage_bf16(st, w, out.Yt != nullptr);
            __syncwarp();
            flush_c(st, out.C, out.ldc, row0, n, nrow, nv, vc, false, false);
            flush_y(st, out.Y, out.ldy, row0, n, nrow, nv, vy);
            if (out.Yt) flush_yt(st, out.Yt, out.ldyt, row0, n, nrow, nv, vt);
            break;
        }
        case EPI_DGELU: {
            // the aux tile is already in the FP32 stage (load_aux / stage_aux by the caller)
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 a = st.c[cidx(lane, j)];
                w[2 * j] = pack_bf16(v[4 * j] * gelu_grad(a.x), v[4 * j + 1] * gelu_grad(a.y));
                w[2 * j + 1] = pack_bf16(v[4 * j + 2] * gelu_grad(a.z), v[4 * j + 3] * gelu_grad(a.w));
            }
            stage_bf16(st, w, out.Yt != nullptr);
            __syncwarp();
            flush_y(st, out.Y, out.ldy, row0, n, nrow, nv, vy);
            if (out.Yt) flush_yt(st, out.Yt, out.ldyt, row0, n, nrow, nv, vt);
            break;
        }
    }
    __syncwarp();   // the stage is reused by the next chunk
}

template <bool TF32>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                   int K, Plan pl, GemmOut out, int *err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int n_tile = pl.n_tile, S = pl.stages;
    const int a_bytes = kTileM * kRowBytes;
    const int stage_bytes = a_bytes + n_tile * kRowBytes;
    EpiStage *epi_stage = reinterpret_cast<EpiStage *>(smem + S * stage_bytes);   // [kEpiWarps]
    uint64_t *full = reinterpret_cast<uint64_t *>(epi_stage + kEpiWarps);
    uint64_t *empty = full + S;
    uint64_t *acc_full = empty + S;    // [2]
    uint64_t *acc_empty = acc_full + 2;  // [2]
    uint64_t *drain = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kel = TF32 ? 32 : 64;
    const int ktiles = (K + kel - 1) / kel;
    const bool split = pl.splits > 1;
    const uint32_t tcols = 2u * (uint32_t)pl.acc_cols;

    if (warp == 2) umma::tmem_alloc(tmem_slot, tcols);
    if (threadIdx.x == 32) {
        for (int s = 0; s < S; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            umma::mbar_init(&acc_full[a], 1);
            umma::mbar_init(&acc_empty[a], kEpiWarps);
        }
        umma::mbar_init(drain, 1);
        *abort_flag = 0;
        umma::fence_mbar_init();
    }
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // unit u -> (n tile, m tile, K share), n fastest: the units that share a 128-row slice of A
    // run on neighbouring CTAs at the same time, so the slice comes from DRAM once
    auto unit = [&](int u, int &m0, int &n0, int &kt0, int &kn) {
        const int ni = u % pl.ntn, r = u / pl.ntn, mi = r % pl.mt, zi = r / pl.mt;
        m0 = mi * kTileM;
        n0 = ni * n_tile;
        kt0 = zi * pl.kt_per;
        kn = min(pl.kt_per, ktiles - kt0);
    };

    if (warp == 0 && lane == 0) {
        // ---- producer: TMA slices of A (128 rows) and B (n_tile rows) ---------------------
        umma::prefetch_tmap(&tmA);
        umma::prefetch_tmap(&tmB);
        int it = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < pl.units && ok; u += gridDim.x) {
            int m0, n0, kt0, kn;
            unit(u, m0, n0, kt0, kn);
            for (int t = 0; t < kn; ++t, ++it) {
                const int s = it % S;
                if (it >= S && !wait_bar(&empty[s], ((it / S) - 1) & 1, abort_flag)) {
                    atomicOr(err, 1);
                    ok = false;
                    break;
                }
                uint8_t *sa = smem + s * stage_bytes;
                umma::mbar_arrive_expect_tx(&full[s], stage_bytes);
                umma::tma_load_2d(sa, &tmA, &full[s], (kt0 + t) * kel, m0);
                umma::tma_load_2d(sa + a_bytes, &tmB, &full[s], (kt0 + t) * kel, n0);
            }
        }
        // no copy may still be landing when the CTA leaves: wait for the last load of every
        // stage (already complete on the normal path)
        for (int s = 0; s < S && s < it; ++s)
            if (!umma::mbar_wait(&full[s], ((it - 1 - s) / S) & 1, kWaitNs)) atomicOr(err, 8);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: 128-byte K slices as 4 MMAs of 32 bytes of K ----------------------
        const uint32_t idesc = umma::idesc_f32(TF32 ? 2u : 1u, kTileM, n_tile);
        int it = 0, lt = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < pl.units && ok; u += gridDim.x, ++lt) {
            int m0, n0, kt0, kn;
            unit(u, m0, n0, kt0, kn);
            const int a = lt & 1;
            if (lt >= 2 && !wait_bar(&acc_empty[a], ((lt >> 1) - 1) & 1, abort_flag)) {
                atomicOr(err, 2);
                break;
            }
            umma::tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(a * pl.acc_cols);
            for (int t = 0; t < kn; ++t, ++it) {
                const int s = it % S;
                if (!wait_bar(&full[s], (it / S) & 1, abort_flag)) {
                    atomicOr(err, 2);
                    ok = false;
                    break;
                }
                umma::tc_fence_after();
                const uint32_t sa = umma::smem_u32(smem + s * stage_bytes);
                const uint64_t da = umma::desc_kmajor_sw128(sa), db = umma::desc_kmajor_sw128(sa + a_bytes);
#pragma unroll
                for (int kk = 0; kk < kRowBytes / 32; ++kk)
                    umma::mma<TF32>(d, da + 2 * kk, db + 2 * kk, idesc, (t > 0 || kk > 0) ? 1u : 0u);
                umma::mma_commit(&empty[s]);
            }
            if (ok) umma::mma_commit(&acc_full[a]);
        }
        // every product issued has landed before the accumulators are released
        umma::mma_commit(drain);
        if (!umma::mbar_wait(drain, 0, kWaitNs)) atomicOr(err, 8);
    } else if (warp >= kEpiWarp0) {
        // ---- epilogue: 16 warps, lane quadrant warp % 4, every fourth 16-column chunk -------
        const int quad = warp & 3, sub = (warp - kEpiWarp0) >> 2;
        EpiStage &st = epi_stage[warp - kEpiWarp0];
        const bool dgelu = out.epi == EPI_DGELU;
        float4 qa[4];
        int lt = 0;
        for (int u = blockIdx.x; u < pl.units; u += gridDim.x, ++lt) {
            int m0, n0, kt0, kn;
            unit(u, m0, n0, kt0, kn);
            const int a = lt & 1;
            const int row0 = m0 + quad * 32, nrow = min(32, M - row0);
            auto chunk_nv = [&](int c) { return c < n_tile ? min(min(16, n_tile - c), N - (n0 + c)) : 0; };
            if (dgelu && nrow > 0 && chunk_nv(sub * 16) > 0)   // travels while the products accumulate
                load_aux(out, row0, n0 + sub * 16, nrow, chunk_nv(sub * 16), qa);
            if (!wait_bar(&acc_full[a], (lt >> 1) & 1, abort_flag)) {
                if (lane == 0) atomicOr(err, 4);
                break;
            }
            umma::tc_fence_after();
            const uint32_t tbase = tmem + (uint32_t)(a * pl.acc_cols) + ((uint32_t)(quad * 32) << 16);
            for (int c = sub * 16; c < n_tile; c += 64) {
                const int nv = chunk_nv(c);
                if (nv <= 0) break;   // uniform over the warp
                float v[16];
                umma::tmem_ld16(tbase + (uint32_t)c, v);
                if (nrow > 0) {
                    if (dgelu) {
                        stage_aux(st, qa);
                        const int nv2 = chunk_nv(c + 64);
                        if (nv2 > 0) load_aux(out, row0, n0 + c + 64, nrow, nv2, qa);
                    }
                    epi_chunk(out, st, split, row0, n0 + c, nrow, nv, v);
                }
            }
            umma::tc_fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&acc_empty[a]);
        }
    }
    __syncwarp();
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    if (warp == 2) umma::tmem_dealloc(tmem, tcols);
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

// Tile width, K split and ring depth: the candidate widths (up to 256, 128 or 64 columns, in
// multiples of 16) are scored by waves of work units over the SMs times a unit's time: its
// operand streaming (rows of A and B per K slice; the main loop waits on these loads) plus a
// share of its epilogue (output columns x an issue cost per element, high for the GELU forms).
Plan make_plan(bool tf32, int M, int N, int K, int epi, bool deterministic) {
    const int kel = tf32 ? 32 : 64;
    const int ktiles = (K + kel - 1) / kel;
    const int mt = (M + kTileM - 1) / kTileM;
    const bool can_split = (epi == EPI_F32 || epi == EPI_F32_ADD) && !deterministic;
    const double epi_cost = (epi == EPI_BIAS_GELU || epi == EPI_DGELU) ? 30.0 : 4.0;
    Plan best{};
    double best_cost = 1e300;
    for (int nmax : {256, 128, 64}) {
        const int ntn = (N + nmax - 1) / nmax;
        const int nt = ((N + ntn - 1) / ntn + 15) / 16 * 16;
        const int tiles = mt * ntn;
        int splits = 1;
        if (can_split && tiles < kNumSMs) splits = std::max(1, std::min(kNumSMs / tiles, ktiles / 4));
        const int kt_per = (ktiles + splits - 1) / splits;
        splits = (ktiles + kt_per - 1) / kt_per;
        const int units = tiles * splits;
        const int waves = (units + kNumSMs - 1) / kNumSMs;
        // the main loop streams (128 + nt) rows per K slice; the epilogue overlaps the next
        // unit's main loop except at the end of a CTA's list
        const double unit_cost = kt_per * 1.3 * (kTileM + nt) + epi_cost * nt / 8.0;
        const double cost = waves * unit_cost;
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best.n_tile = nt;
            best.ntn = ntn;
            best.mt = mt;
            best.splits = splits;
            best.kt_per = kt_per;
            best.units = units;
        }
    }
    const int stage_bytes = (kTileM + best.n_tile) * kRowBytes;
    best.stages = std::min(kMaxStages, kRingBytes / stage_bytes);
    int ac = 32;
    while (ac < best.n_tile) ac <<= 1;
    best.acc_cols = ac;
    return best;
}

}  // namespace

int tc_gemm(bool tf32, int M, int N, int K, const void *A, int lda, const void *B, int ldb, const GemmOut &out_in,
            cudaStream_t stream, int *err_dev) {
    if (M <= 0 || N <= 0 || K <= 0 || !A || !B)
        return fitcore_fail(FIT_ERR_INVALID_ARG, "tensor-core GEMM: empty or null operand");
    const int esz = tf32 ? 4 : 2;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((size_t)lda * esz) % 16 || ((size_t)ldb * esz) % 16 ||
        lda < K || ldb < K)
        return fitcore_fail(FIT_ERR_INVALID_ARG, "tensor-core GEMM: operands must be 16-byte aligned rows");
    int rc = get_encoder();
    if (rc) return rc;
    GemmOut out = out_in;
    out.vec = ((out.C && !((uintptr_t)out.C & 15) && out.ldc % 4 == 0) ? 1 : 0) |
              ((out.Y && !((uintptr_t)out.Y & 15) && out.ldy % 8 == 0) ? 2 : 0) |
              ((out.aux && !((uintptr_t)out.aux & 15) && out.ldaux % 4 == 0) ? 4 : 0) |
              ((out.Yt && !((uintptr_t)out.Yt & 15) && out.ldyt % 8 == 0) ? 8 : 0) |
              ((out.bias && !((uintptr_t)out.bias & 15)) ? 16 : 0);
    const Plan pl = make_plan(tf32, M, N, K, out.epi, out.deterministic);
    CUtensorMap ta, tb;
    if ((rc = make_map(&ta, tf32, A, M, K, lda, kTileM))) return rc;
    if ((rc = make_map(&tb, tf32, B, N, K, ldb, pl.n_tile))) return rc;
    if (!err_dev) {   // the library's flag: its device address, looked up once per device
        static std::mutex flag_mutex;
        static int *flag_addr[64] = {nullptr};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
            cudaGetLastError();
            return fitcore_fail(FIT_ERR_CUDA, "tensor-core GEMM: current device");
        }
        std::lock_guard<std::mutex> lock(flag_mutex);
        if (!flag_addr[dev] && cudaGetSymbolAddress((void **)&flag_addr[dev], g_gemm_err) != cudaSuccess) {
            cudaGetLastError();
            flag_addr[dev] = nullptr;
            return fitcore_fail(FIT_ERR_CUDA, "tensor-core GEMM: error flag");
        }
        err_dev = flag_addr[dev];
    }
    const size_t smem = 1024 + (size_t)pl.stages * (kTileM + pl.n_tile) * kRowBytes + kEpiWarps * sizeof(EpiStage) +
                        (2 * pl.stages + 5) * 8 + 16;
    auto kern = tf32 ? tc_gemm_kernel<true> : tc_gemm_kernel<false>;
    {
        static std::mutex attr_mutex;
        static int attr_set[2] = {0, 0};
        std::lock_guard<std::mutex> lock(attr_mutex);
        int &cur = attr_set[tf32 ? 1 : 0];
        if ((int)smem > cur) {   // only ever raised
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                cudaGetLastError();
                return fitcore_fail(FIT_ERR_CUDA, "tensor-core GEMM: shared memory attribute");
            }
            cur = (int)smem;
        }
    }
    if (pl.splits > 1 && out.epi == EPI_F32) {
        // C = 0 first: rows of ldc floats (the row tails beyond N are left as they were)
        cudaError_t e = (out.ldc == N) ? cudaMemsetAsync(out.C, 0, sizeof(float) * (size_t)M * N, stream)
                                       : cudaMemset2DAsync(out.C, sizeof(float) * (size_t)out.ldc, 0,
                                                           sizeof(float) * (size_t)N, M, stream);
        if (e != cudaSuccess) return fitcore_fail(FIT_ERR_CUDA, "tensor-core GEMM: clearing C");
    }
    const int grid = std::min(pl.units, kNumSMs);
    kern<<<grid, kThreads, smem, stream>>>(ta, tb, M, N, K, pl, out, err_dev);
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
