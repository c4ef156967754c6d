// goat_gemm.cu -- K1: the two n x n x n products of the GOAT gradient on the
// 5th-generation tensor cores (tcgen05 + TMEM), fed by TMA.
//
// Alg. 3 step 1 needs grad f(Q) = A Q B^T + A^T Q B, which for symmetric A, B is
// 2 A Q B.  Both products are computed as "D = X Y^T" with X and Y row-major
// (K contiguous), so every operand is K-major and is staged by TMA with the
// 128-byte swizzle the MMA descriptors expect:
//
//   product 1:  C1 = B Q^T      (X = B, Y = Q)    C1[j][i] = (Q B)[i][j]  -> C1 = (Q B)^T
//   product 2:  G_Q = -2 A C1^T (X = A, Y = C1)   G_Q[i][j] = -2 (A Q B)[i][j]
//
// A K-period on X lets one launch accumulate several split terms of Y
// (Y = [Y_hi | Y_lo] along K, X re-read for each term): that is how the
// FP32-accurate form adds A Q_hi B + A Q_lo B in one TMEM accumulator.
//
// A launch may also cover one K range of a longer product (k_offset) and add an
// FP32 addend in its epilogue: the FP32-accurate form splits long K into chunks
// so that the tensor core's FP32 accumulation, which truncates (every sampled
// entry of a K = 65536 product came out smaller in magnitude, by 1.6e-5 relative),
// runs over fewer steps, and the chunks are added in the epilogue with
// round-to-nearest FP32.
//
// The same kernel runs the 8-bit form (KIND = KIND_E4M3): E4M3 operands,
// kind::f8f6f4.  A stage then holds 128 elements of K instead of 64 -- the same 128
// bytes per swizzled row, so the shared-memory layout, the descriptors and their
// 32-byte K steps are unchanged; only the element type, the K extent per stage and
// the instruction kind differ.  KIND_MIXED runs both in one accumulator: the first
// num_kb_hi K blocks from the BF16 maps (kind::f16), the rest from a second pair of
// E4M3 maps (kind::f8f6f4) -- the second product of the split form whose low term
// is 8-bit.
//
// Kernel structure (one persistent CTA per SM, 192 threads):
//   warp 0      TMA producer: X tile 128x64 and Y tile 256x64 per stage (BF16), 4 stages
//   warp 1      TMEM owner and MMA issuer: 4 x tcgen05.mma M=128 N=256 K=16 (K=32 for E4M3) per stage
//   warps 2-5   epilogue: tcgen05.ld 32 lanes x 32 columns, scale, convert, store
// Two TMEM accumulators (2 x 256 columns) let the epilogue of tile t overlap
// the MMAs of tile t+1.  Every wait is bounded (see mbar_wait_bounded).
#include <cstdio>
#include <cstring>
#include <mutex>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int KIND_BF16 = 0, KIND_E4M3 = 1, KIND_MIXED = 2;
constexpr uint32_t TILE_X_BYTES = BM * BK * 2;
constexpr uint32_t TILE_Y_BYTES = BN * BK * 2;
constexpr uint32_t STAGE_BYTES = TILE_X_BYTES + TILE_Y_BYTES;
constexpr uint32_t TMEM_COLS = 2 * BN;
constexpr int GEMM_THREADS = 192;
constexpr int GROUP_M = 16;
constexpr size_t GEMM_SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + 256;

struct GemmParams {
    int M, N;            // output rows (from X) and columns (from Y)
    int kx_period;       // X is read at k mod kx_period (multiple of BK)
    int num_kb;          // K blocks (stages) of the launch
    int num_kb_hi;       // KIND_MIXED: the first num_kb_hi blocks are BF16 (64 elements), the rest E4M3 (128)
    int kx8_period;      // KIND_MIXED: period of the E4M3 X operand's K (multiple of 128)
    int k_offset_kb;     // first K block of this launch (K positions k_offset_kb * BK + ...)
    const float *addend; // FP32 matrix added in the epilogue (nullable), ld_addend, columns < addend_cols
    long long ld_addend;
    int addend_cols;
    int tiles_m, tiles_n;
    float scale;
    const float *scale_dev;  // device factor on top of scale (nullable)
    int mode;            // GEMM_OUT_F32 or GEMM_OUT_BF16_TERMS
    float *out_f32;
    long long ld_out;    // FP32 output leading dimension
    __nv_bfloat16 *out_b16;
    int out_terms;       // 1 or 2 (hi, lo) BF16 terms
    long long term_stride;  // elements between the hi and lo term of a row
    long long row_stride;   // elements between rows of the BF16 output
    int out_rows, out_cols; // rows / columns actually written
    int *err;
    // grouped mode (many independent problems in one launch): work items
    // {problem, tile_m, tile_n, 0} and one descriptor per problem
    const int4 *items;
    int num_items;
    const GemmGroupDesc *descs;
};

// Where one output tile comes from and goes to.
struct TileJob {
    int x_row, y_row;       // TMA row coordinates of the X and Y tiles
    int num_kb;             // K blocks of this tile
    int row0, col0;         // output coordinates of the tile's first element
    int out_rows, out_cols; // write bounds
    int valid_cols;         // columns in [valid_cols, out_cols) are written as zero
    float *out_f32;
    long long ld_out;
    __nv_bfloat16 *out_b16;
    long long row_stride;
};

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int &tm, int &tn) {
    const int group = GROUP_M * tiles_n;
    const int g = t / group;
    const int first = g * GROUP_M;
    const int gm = min(tiles_m - first, GROUP_M);
    const int r = t - g * group;
    tm = first + r % gm;
    tn = r / gm;
}

template <bool GROUPED>
__device__ __forceinline__ TileJob make_job(const GemmParams &p, int t) {
    TileJob j;
    if constexpr (GROUPED) {
        const int4 it = p.items[t];
        const GemmGroupDesc d = p.descs[it.x];
        j.x_row = (int)(d.x_row0 + (long long)it.y * 128);
        j.y_row = (int)(d.y_row0 + (long long)it.z * 256);
        j.num_kb = d.num_kb;
        j.row0 = it.y * 128;
        j.col0 = it.z * 256;
        j.out_rows = d.M;
        j.out_cols = d.out_cols;
        j.valid_cols = d.N;
        j.out_f32 = d.out_f32;
        j.ld_out = d.ld_out;
        j.out_b16 = d.out_b16;
        j.row_stride = d.row_stride;
    } else {
        int tm, tn;
        tile_coords(t, p.tiles_m, p.tiles_n, tm, tn);
        j.x_row = tm * 128;
        j.y_row = tn * 256;
        j.num_kb = p.num_kb;
        j.row0 = tm * 128;
        j.col0 = tn * 256;
        j.out_rows = p.out_rows;
        j.out_cols = p.out_cols;
        j.valid_cols = 0x7fffffff;
        j.out_f32 = p.out_f32;
        j.ld_out = p.ld_out;
        j.out_b16 = p.out_b16;
        j.row_stride = p.row_stride;
    }
    return j;
}

__device__ __forceinline__ bool wait_timeout_ns(uint32_t bar, uint32_t parity, uint64_t ns) {
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_timer_ns() - t0 > ns) return false;
    return true;
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t *>(&h); }

// Writes one accumulator row segment (32 consecutive columns) held by this thread.
// All indexing is static so the segment stays in registers.  Columns at or beyond
// j.valid_cols are written as zero (padding of a grouped problem's operand).
__device__ __forceinline__ void store_tile_row(const GemmParams &p, const TileJob &j, int row, int col0,
                                               const float (&v)[32]) {
    if (row >= j.out_rows || col0 >= j.out_cols) return;
    const float s = p.scale_dev ? p.scale * *p.scale_dev : p.scale;
    float x[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) x[c] = (col0 + c < j.valid_cols) ? v[c] * s : 0.0f;
    if (p.addend) {
        const float *ad = p.addend + (long long)row * p.ld_addend + col0;
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (col0 + c < p.addend_cols) x[c] += ad[c];
    }
    if (p.mode == GEMM_OUT_F32) {
        float *dst = j.out_f32 + (long long)row * j.ld_out + col0;
        const bool full = (col0 + 32 <= j.out_cols) && ((j.ld_out & 3) == 0) &&
                          ((reinterpret_cast<uintptr_t>(dst) & 15) == 0);
        if (full) {
#pragma unroll
            for (int c = 0; c < 32; c += 4)
                *reinterpret_cast<float4 *>(dst + c) = make_float4(x[c], x[c + 1], x[c + 2], x[c + 3]);
        } else {
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (col0 + c < j.out_cols) dst[c] = x[c];
        }
        return;
    }
    __nv_bfloat16 *hi = j.out_b16 + (long long)row * j.row_stride + col0;
    __nv_bfloat16 *lo = hi + p.term_stride;
    const bool two = p.out_terms > 1;
    const bool full = (col0 + 32 <= j.out_cols) && ((j.row_stride & 7) == 0) && ((p.term_stride & 7) == 0);
    uint32_t hw[16], lw[16];
#pragma unroll
    for (int c = 0; c < 32; c += 2) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[c], x[c + 1]);
        const float2 hf = __bfloat1622float2(h2);
        hw[c / 2] = bf16x2_bits(h2);
        lw[c / 2] = bf16x2_bits(__floats2bfloat162_rn(x[c] - hf.x, x[c + 1] - hf.y));
    }
    if (full) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4 *>(hi + 8 * q) = make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
        if (two) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                *reinterpret_cast<uint4 *>(lo + 8 * q) =
                    make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            if (col0 + c < j.out_cols) {
                const uint32_t hb = hw[c / 2], lb = lw[c / 2];
                const unsigned short h16 = (c & 1) ? (unsigned short)(hb >> 16) : (unsigned short)(hb & 0xFFFFu);
                const unsigned short l16 = (c & 1) ? (unsigned short)(lb >> 16) : (unsigned short)(lb & 0xFFFFu);
                hi[c] = __ushort_as_bfloat16(h16);
                if (two) lo[c] = __ushort_as_bfloat16(l16);
            }
        }
    }
}

template <bool GROUPED, int KIND>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm_xyT(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
               const __grid_constant__ CUtensorMap tmX8, const __grid_constant__ CUtensorMap tmY8, const GemmParams p) {
    constexpr bool FP8 = KIND == KIND_E4M3;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)STAGES * STAGE_BYTES);
    // bars: [0,S) full, [S,2S) empty, 2S..2S+1 tmem full, 2S+2..2S+3 tmem empty, 2S+4 drain
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
    auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
    const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), 128);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        prefetch_tmap(&tmX);
        prefetch_tmap(&tmY);
        if constexpr (KIND == KIND_MIXED) {
            prefetch_tmap(&tmX8);
            prefetch_tmap(&tmY8);
        }
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int num_tiles = GROUPED ? p.num_items : p.tiles_m * p.tiles_n;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_mask = 0, issued_parity = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
                const TileJob job = make_job<GROUPED>(p, t);
                for (int kb = 0; kb < job.num_kb; ++kb) {
                    if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sx = sbase + stage * STAGE_BYTES;
                    mbar_arrive_expect_tx(full_bar(stage), STAGE_BYTES);
                    if (KIND == KIND_MIXED && kb >= p.num_kb_hi) {
                        const int kk = (kb - p.num_kb_hi) * 2 * BK;  // E4M3 block: 128 elements = 128 bytes
                        tma_load_2d(sx, &tmX8, full_bar(stage), kk % p.kx8_period, job.x_row);
                        tma_load_2d(sx + TILE_X_BYTES, &tmY8, full_bar(stage), kk, job.y_row);
                    } else {
                        const int kk = (p.k_offset_kb + kb) * (FP8 ? 2 * BK : BK);  // K elements per stage: 128 bytes
                        tma_load_2d(sx, &tmX, full_bar(stage), kk % p.kx_period, job.x_row);
                        tma_load_2d(sx + TILE_X_BYTES, &tmY, full_bar(stage), kk, job.y_row);
                    }
                    issued_mask |= 1u << stage;
                    issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // let every copy in flight land before the CTA releases its shared memory
                for (int s = 0; s < STAGES; ++s)
                    if (issued_mask & (1u << s)) wait_timeout_ns(full_bar(s), (issued_parity >> s) & 1u, 200000000ull);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        const uint32_t idesc = FP8 ? idesc_e4m3_f32(BM, BN) : idesc_bf16_f32(BM, BN);
        const uint32_t idesc8 = idesc_e4m3_f32(BM, BN);
        int stage = 0;
        uint32_t phase = 0;
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
            int w = (lane == 0) ? (int)mbar_wait_bounded(tempty_bar(acc), acc_phase ^ 1u, abort_flag) : 1;
            if (!__shfl_sync(0xffffffffu, w, 0)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
            const int num_kb = GROUPED ? make_job<GROUPED>(p, t).num_kb : p.num_kb;
            for (int kb = 0; kb < num_kb; ++kb) {
                w = (lane == 0) ? (int)mbar_wait_bounded(full_bar(stage), phase, abort_flag) : 1;
                if (!__shfl_sync(0xffffffffu, w, 0)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t sx = sbase + stage * STAGE_BYTES;
                    const uint32_t sy = sx + TILE_X_BYTES;
                    const bool e4m3 = FP8 || (KIND == KIND_MIXED && kb >= p.num_kb_hi);
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) {  // 32 bytes of K per instruction
                        if (e4m3)
                            umma_f8(d_tmem, smem_desc_sw128(sx + 32u * k), smem_desc_sw128(sy + 32u * k),
                                    FP8 ? idesc : idesc8, (kb | k) != 0 ? 1u : 0u);
                        else
                            umma_bf16(d_tmem, smem_desc_sw128(sx + 32u * k), smem_desc_sw128(sy + 32u * k), idesc,
                                      (kb | k) != 0 ? 1u : 0u);
                    }
                    umma_commit(empty_bar(stage));
                }
                __syncwarp();
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok) break;
            if (lane == 0) umma_commit(tfull_bar(acc));
            __syncwarp();
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
        // every MMA issued by this warp has finished before TMEM is released
        if (lane == 0) {
            umma_commit(drain_bar);
            if (!wait_timeout_ns(drain_bar, 0, 200000000ull)) *abort_flag = 1;
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue (warps 2..5)
        const int q = warp & 3;  // TMEM lane quarter this warp may address
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < num_tiles; t += gridDim.x) {
            const TileJob job = make_job<GROUPED>(p, t);
            int w = (lane == 0) ? (int)mbar_wait_bounded(tfull_bar(acc), acc_phase, abort_flag) : 1;
            if (!__shfl_sync(0xffffffffu, w, 0)) break;
            tc_fence_after();
            const int row = job.row0 + q * 32 + lane;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                tmem_ld_32x32b_x32(taddr + 32u * c, v);
                tmem_wait_ld();
                if (c == BN / 32 - 1) {
                    tc_fence_before();
                    mbar_arrive(tempty_bar(acc));
                }
                store_tile_row(p, job, row, job.col0 + c * 32, v);
            }
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
    if (threadIdx.x == 0 && *abort_flag) atomicCAS(p.err, 0, (int)GOAT_ERR_TIMEOUT);
}

// ---------------------------------------------------------------- host side

typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                      const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                      CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);

static PFN_encodeTiled_t get_encode_fn() {
    static PFN_encodeTiled_t fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled_t>(p);
    });
    return fn;
}

// 2-D tensor map of BF16 (or, fp8, E4M3 bytes): inner extent `inner` (elements), `rows`
// rows `stride` elements apart, box of 128 bytes x box_rows with the 128-byte swizzle;
// out-of-range elements read as zero.
static int make_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint64_t stride,
                    uint32_t box_rows, bool fp8 = false) {
    PFN_encodeTiled_t enc = get_encode_fn();
    if (!enc) return GOAT_ERR_CUDA;
    const uint64_t es = fp8 ? 1 : 2;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || ((stride * es) & 15)) return GOAT_ERR_INVALID_ARG;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {stride * es};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                     const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GOAT_OK : GOAT_ERR_CUDA;
}

static int g_sm_count = 0;

// One-time per process: SM count and the kernels' dynamic shared memory limit.
static int prepare_launch() {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        attr_err = cudaFuncSetAttribute(k_gemm_xyT<false, KIND_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)GEMM_SMEM_BYTES);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(k_gemm_xyT<true, KIND_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)GEMM_SMEM_BYTES);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(k_gemm_xyT<false, KIND_E4M3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)GEMM_SMEM_BYTES);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(k_gemm_xyT<false, KIND_MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)GEMM_SMEM_BYTES);
    });
    return (attr_err != cudaSuccess || g_sm_count <= 0) ? GOAT_ERR_CUDA : GOAT_OK;
}

int gemm_xyT(const GemmCall &c, cudaStream_t stream) {
    const int bk = c.fp8 ? 2 * BK : BK;  // K elements per stage
    if (c.M < 1 || c.N < 1 || c.k_total < 1 || (c.k_total % bk) || (c.kx_period % bk) || c.kx_period < 1 ||
        c.k_begin < 0 || (c.k_begin % bk))
        return GOAT_ERR_INVALID_ARG;
    {
        const int ps = prepare_launch();
        if (ps) return ps;
    }
    const int sm_count = g_sm_count;

    CUtensorMap mx, my;
    int st = make_map(&mx, c.X, (uint64_t)c.kx_period, (uint64_t)c.x_rows, (uint64_t)c.x_stride, BM, c.fp8 != 0);
    if (st) return st;
    st = make_map(&my, c.Y, (uint64_t)(c.k_begin + c.k_total), (uint64_t)c.y_rows, (uint64_t)c.y_stride, BN,
                  c.fp8 != 0);
    if (st) return st;

    GemmParams p;
    std::memset(&p, 0, sizeof(p));
    p.k_offset_kb = c.k_begin / bk;
    p.addend = c.addend;
    p.ld_addend = c.ld_addend;
    p.addend_cols = c.addend_cols;
    p.M = c.M;
    p.N = c.N;
    p.kx_period = c.kx_period;
    p.num_kb = c.k_total / bk;
    p.scale_dev = c.scale_dev;
    p.tiles_m = (int)ceil_div(c.M, BM);
    p.tiles_n = (int)ceil_div(c.N, BN);
    p.scale = c.scale;
    p.mode = c.mode;
    p.out_f32 = c.out_f32;
    p.ld_out = c.ld_out;
    p.out_b16 = c.out_b16;
    p.out_terms = c.out_terms;
    p.term_stride = c.term_stride;
    p.row_stride = c.row_stride;
    p.out_rows = c.out_rows;
    p.out_cols = c.out_cols;
    p.err = c.err;
    const int tiles = p.tiles_m * p.tiles_n;
    const int grid = tiles < sm_count ? tiles : sm_count;
    if (c.X8) {
        // mixed: the BF16 maps above cover K [0, k_total), the E4M3 maps K8 [0, k8_total)
        if (c.fp8 || c.k_begin || c.addend || c.k8_total < 1 || (c.k8_total % (2 * BK)) || c.kx8_period < 1 ||
            (c.kx8_period % (2 * BK)))
            return GOAT_ERR_INVALID_ARG;
        CUtensorMap mx8, my8;
        st = make_map(&mx8, c.X8, (uint64_t)c.kx8_period, (uint64_t)c.x_rows, (uint64_t)c.x8_stride, BM, true);
        if (st) return st;
        st = make_map(&my8, c.Y8, (uint64_t)c.k8_total, (uint64_t)c.y_rows, (uint64_t)c.y8_stride, BN, true);
        if (st) return st;
        p.num_kb_hi = p.num_kb;
        p.num_kb += c.k8_total / (2 * BK);
        p.kx8_period = c.kx8_period;
        k_gemm_xyT<false, KIND_MIXED><<<grid, GEMM_THREADS, GEMM_SMEM_BYTES, stream>>>(mx, my, mx8, my8, p);
    } else if (c.fp8) {
        k_gemm_xyT<false, KIND_E4M3><<<grid, GEMM_THREADS, GEMM_SMEM_BYTES, stream>>>(mx, my, mx, my, p);
    } else {
        k_gemm_xyT<false, KIND_BF16><<<grid, GEMM_THREADS, GEMM_SMEM_BYTES, stream>>>(mx, my, mx, my, p);
    }
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

int gemm_grouped(const GemmGroupCall &c, cudaStream_t stream) {
    if (c.num_items < 1 || c.k_extent < BK || (c.k_extent % BK)) return GOAT_ERR_INVALID_ARG;
    int st = prepare_launch();
    if (st) return st;
    CUtensorMap mx, my;
    st = make_map(&mx, c.X, (uint64_t)c.k_extent, (uint64_t)c.x_rows, (uint64_t)c.x_stride, BM);
    if (st) return st;
    st = make_map(&my, c.Y, (uint64_t)c.k_extent, (uint64_t)c.y_rows, (uint64_t)c.y_stride, BN);
    if (st) return st;
    GemmParams p;
    std::memset(&p, 0, sizeof(p));
    p.kx_period = c.k_extent;
    p.scale = c.scale;
    p.mode = c.mode;
    p.out_terms = 1;
    p.term_stride = 0;
    p.err = c.err;
    p.items = c.items;
    p.num_items = c.num_items;
    p.descs = c.descs;
    const int grid = c.num_items < g_sm_count ? c.num_items : g_sm_count;
    k_gemm_xyT<true, KIND_BF16><<<grid, GEMM_THREADS, GEMM_SMEM_BYTES, stream>>>(mx, my, mx, my, p);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

}  // namespace goat
