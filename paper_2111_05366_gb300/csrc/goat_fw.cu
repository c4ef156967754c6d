// goat_fw.cu -- the memory-bound kernels of the Frank-Wolfe loop (Alg. 3):
// operand preparation, the closed-form first gradient, the line-search
// reductions (K3), the update (K4) and the objective at a permutation.
#include <algorithm>

#include <cuda_fp8.h>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

// ---------------------------------------------------------------- operands

// A rows x cols window of an adjacency matrix (uint8 or float32, leading dimension
// lda) -> BF16 GEMM operand rows of `width` elements (zero beyond cols), `stride`
// elements apart, plus the window's row sums in FP32 (deg, nullable).  One warp per row.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_to_bf16(const T *__restrict__ A, long long lda, int rows, int cols,
                                                     __nv_bfloat16 *__restrict__ A16, int width, long long stride,
                                                     float *__restrict__ deg) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < rows; i += gridDim.x * wpb) {
        const T *src = A + (long long)i * lda;
        __nv_bfloat16 *dst = A16 + (long long)i * stride;
        float s = 0.0f;
        for (int j = lane; j < width; j += 32) {
            const float v = (j < cols) ? (float)src[j] : 0.0f;
            dst[j] = __float2bfloat16_rn(v);
            s += v;
        }
        s = warp_sum(s);
        if (lane == 0 && deg) deg[i] = s;
    }
}

// ---------------------------------------------------------------- 8-bit operands

// Two floats -> two E4M3 bytes (round to nearest, saturating at +-448).
__device__ __forceinline__ unsigned short e4m3x2(float a, float b) {
    return (unsigned short)__nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
}

// The same window -> E4M3 GEMM operand rows (`width` bytes, even, zero beyond
// cols, `stride` bytes apart).  0/1 entries are exact (1.0 = 0x38); other weights
// round to E4M3.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_to_e4m3(const T *__restrict__ A, long long lda, int rows, int cols,
                                                     uint8_t *__restrict__ A8, int width, long long stride) {
    const int pairs = width / 2;
    const long long total = (long long)rows * pairs;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / pairs), j = (int)(t - (long long)i * pairs) * 2;
        const T *src = A + (long long)i * lda;
        const float a = j < cols ? (float)src[j] : 0.0f, b = j + 1 < cols ? (float)src[j + 1] : 0.0f;
        *reinterpret_cast<unsigned short *>(A8 + (long long)i * stride + j) = e4m3x2(a, b);
    }
}

// The transpose of a rows x cols window -> operand rows (dst row c = source column
// c): dst[c][r] = A[r][c] for r < rows, zero for rows <= r < width; dst rows
// 0..cols-1, `stride` elements apart.  32 x 32 tiles through shared memory; grid
// (ceil(width / 32), ceil(cols / 32)), block 32 x 8.  O is __nv_bfloat16 or uint8_t (E4M3).
template <typename T, typename O>
__global__ void k_adj_transpose(const T *__restrict__ A, long long lda, int rows, int cols, O *__restrict__ dst,
                                int width, long long stride) {
    __shared__ float tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int k = ty; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + tx;
        tile[k][tx] = (r < rows && c < cols) ? (float)A[(long long)r * lda + c] : 0.0f;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + tx;
        if (c < cols && r < width) {
            const float v = tile[tx][k];
            if constexpr (sizeof(O) == 1)
                dst[(long long)c * stride + r] = (O)(e4m3x2(v, 0.0f) & 0xFFu);
            else
                dst[(long long)c * stride + r] = __float2bfloat16_rn(v);
        }
    }
}

// Column sums of a rows x cols window in FP32 (the in-degrees of a directed graph);
// one thread per column, the rows in order.
template <typename T>
__global__ void __launch_bounds__(256) k_col_sums(const T *__restrict__ A, long long lda, int rows, int cols,
                                                  float *__restrict__ out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int r = 0; r < rows; ++r) s += (float)A[(long long)r * lda + c];
        out[c] = s;
    }
}

// max |x| of a BF16 matrix (non-negative float bits, atomicMax); total is a
// multiple of 8 and X 16-byte aligned (operand buffers), read 16 bytes at a time.
__global__ void __launch_bounds__(256) k_absmax_bf16(const __nv_bfloat16 *__restrict__ X, long long total,
                                                     unsigned *out) {
    float m = 0.0f;
    const uint4 *X8 = reinterpret_cast<const uint4 *>(X);
    const long long total8 = total >> 3;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total8;
         t += (long long)gridDim.x * blockDim.x) {
        const uint4 v = __ldg(X8 + t);
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // |x| of a BF16 is its bits without the sign; as the upper half of a float it orders the same
            m = fmaxf(m, __uint_as_float((w[k] & 0x7FFFu) << 16));
            m = fmaxf(m, __uint_as_float(w[k] & 0x7FFF0000u));
        }
    }
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(out, __float_as_uint(m));
}

// BF16 matrix (rows x ld_src) -> E4M3 (rows x ld8, zero padding) scaled by s, the
// largest power of two with s max|x| <= 448; inv_scale <- 1 / s (exact).  One
// thread per 16 output bytes; ld_src is a multiple of 64 and ld8 of 128, so a
// 16-column chunk lies wholly inside the source row or wholly in the padding.
__global__ void __launch_bounds__(256) k_bf16_to_e4m3(const __nv_bfloat16 *__restrict__ X, int rows, int ld_src,
                                                      uint8_t *__restrict__ X8, int ld8, const unsigned *amax_bits,
                                                      float *inv_scale) {
    const float amax = __uint_as_float(*amax_bits);
    // power of two at or below 448 / amax: keep the exponent bits of the quotient
    const float q = amax > 0.0f ? 448.0f / amax : 1.0f;
    const float sc = __uint_as_float(__float_as_uint(q) & 0x7F800000u);
    if (blockIdx.x == 0 && threadIdx.x == 0) *inv_scale = 1.0f / sc;
    const int cpr = ld8 / 16;  // 16-column chunks per row
    const long long total = (long long)rows * cpr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / cpr), j = (int)(t - (long long)i * cpr) * 16;
        uint4 out = make_uint4(0u, 0u, 0u, 0u);
        if (j < ld_src) {
            const uint4 *src = reinterpret_cast<const uint4 *>(X + (long long)i * ld_src + j);
            const uint4 v0 = __ldg(src), v1 = __ldg(src + 1);
            const unsigned w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            unsigned b[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                b[k] = e4m3x2(__uint_as_float(w[k] << 16) * sc, __uint_as_float(w[k] & 0xFFFF0000u) * sc);
            out = make_uint4(b[0] | (b[1] << 16), b[2] | (b[3] << 16), b[4] | (b[5] << 16), b[6] | (b[7] << 16));
        }
        *reinterpret_cast<uint4 *>(X8 + (long long)i * ld8 + j) = out;
    }
}

// The split intermediate C1 = hi + lo (BF16 terms, rows of `parts` hi blocks then
// `parts` lo blocks of ld elements, row stride cs) prepared for a second product
// whose lo term is 8-bit: with amax = max|C1| (so max|hi| <= amax, and |lo| is at
// most half a BF16 unit of hi, <= 2^-8 |hi|), s is the largest power of two with
// s amax 2^-8 <= 448; lo -> E4M3(s lo) in C8 (rows of `parts` blocks of w8 bytes,
// zero beyond ld), hi -> s hi in place (exact: a power of two), inv_scale <- 1/s.
// One thread per 16 output bytes; ld is a multiple of 64, so a chunk never
// straddles a block edge.
__global__ void __launch_bounds__(256) k_split_lo_to_e4m3(__nv_bfloat16 *__restrict__ C1, int rows, int ld,
                                                          int parts, long long cs, uint8_t *__restrict__ C8, int w8,
                                                          const unsigned *amax_bits, float *inv_scale) {
    const float amax = __uint_as_float(*amax_bits);
    const float q = amax > 0.0f ? (448.0f * 256.0f) / amax : 1.0f;
    const float sc = __uint_as_float(__float_as_uint(q) & 0x7F800000u);
    if (blockIdx.x == 0 && threadIdx.x == 0) *inv_scale = 1.0f / sc;
    const int cpr = parts * w8 / 16;  // 16-byte output chunks per row
    const long long total = (long long)rows * cpr;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / cpr), jc = (int)(t - (long long)i * cpr) * 16;
        const int part = jc / w8, j = jc - part * w8;
        uint4 out = make_uint4(0u, 0u, 0u, 0u);
        if (j < ld) {
            __nv_bfloat16 *hi = C1 + (long long)i * cs + (long long)part * ld + j;
            const __nv_bfloat16 *lo = C1 + (long long)i * cs + (long long)(parts + part) * ld + j;
            const uint4 l0 = __ldg(reinterpret_cast<const uint4 *>(lo)), l1 = __ldg(reinterpret_cast<const uint4 *>(lo) + 1);
            const unsigned w[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
            unsigned b[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                b[k] = e4m3x2(__uint_as_float(w[k] << 16) * sc, __uint_as_float(w[k] & 0xFFFF0000u) * sc);
            out = make_uint4(b[0] | (b[1] << 16), b[2] | (b[3] << 16), b[4] | (b[5] << 16), b[6] | (b[7] << 16));
            uint4 *h4 = reinterpret_cast<uint4 *>(hi);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                uint4 h = h4[u];
                unsigned hw[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const __nv_bfloat162 v =
                        __floats2bfloat162_rn(__uint_as_float(hw[k] << 16) * sc, __uint_as_float(hw[k] & 0xFFFF0000u) * sc);
                    hw[k] = *reinterpret_cast<const unsigned *>(&v);
                }
                h4[u] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            }
        }
        *reinterpret_cast<uint4 *>(C8 + (long long)i * parts * w8 + jc) = out;
    }
}

// Counts entries with A[i][j] != A[j][i] (32 x 32 tiles through shared memory).
template <typename T>
__global__ void k_count_asym(const T *__restrict__ A, int n, int *__restrict__ count) {
    __shared__ float tile[32][33];
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    if (bj < bi) return;  // each unordered tile pair once
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int i = bj + r, j = bi + tx;
        tile[r][tx] = (i < n && j < n) ? (float)A[(long long)i * n + j] : 0.0f;
    }
    __syncthreads();
    int bad = 0;
    for (int r = ty; r < 32; r += 8) {
        const int i = bi + r, j = bj + tx;
        if (i < n && j < n) {
            const float a = (float)A[(long long)i * n + j];
            if (a != tile[tx][r]) ++bad;
        }
    }
    if (bad) atomicAdd(count, bad);
}

// FP32 matrix (ld n) -> BF16 split terms (hi [, lo]) with row stride terms*ld16.
__global__ void __launch_bounds__(256) k_f32_to_terms(const float *__restrict__ X, int n, long long ldx,
                                                      __nv_bfloat16 *__restrict__ Xb, int ld16, int terms) {
    const int chunks = ld16 / 8;
    const long long total = (long long)n * chunks;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / chunks);
        const int j0 = (int)(t - (long long)i * chunks) * 8;
        float q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = (j0 + k < n) ? X[(long long)i * ldx + j0 + k] : 0.0f;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(q[k], q[k + 1]);
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(q[k] - hf.x, q[k + 1] - hf.y);
            hw[k / 2] = *reinterpret_cast<const uint32_t *>(&h2);
            lw[k / 2] = *reinterpret_cast<const uint32_t *>(&l2);
        }
        __nv_bfloat16 *row = Xb + (long long)i * ((long long)terms * ld16);
        *reinterpret_cast<uint4 *>(row + j0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        if (terms > 1) *reinterpret_cast<uint4 *>(row + ld16 + j0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// ---------------------------------------------------------------- first gradient

// At the barycenter J = 11^T/n:  grad f(J) = (A 1)(B 1)^T / n + (A^T 1)(B^T 1)^T / n,
// the out-degrees d_A, d_B and in-degrees e_A, e_B, so
//   G = scale (d_A d_B^T + e_A e_B^T) [+ C]
// with scale = -sigma / n (sigma = +1 to maximise f, -1 to minimise it); for
// symmetric graphs e = d and the kernel is called with scale = -2 sigma / n and no
// in-degrees.  C (nullable) is a constant term of the gradient (the seeds' share),
// P (nullable) is set to J.  max|G| goes to st->gmax_bits.
__global__ void __launch_bounds__(256) k_barycenter(const float *__restrict__ dA, const float *__restrict__ dB,
                                                    const float *__restrict__ eA, const float *__restrict__ eB, int n,
                                                    float scale, const float *__restrict__ C, float *__restrict__ G,
                                                    float *__restrict__ P, DevState *st) {
    const float inv_n = 1.0f / (float)n;
    float gm = 0.0f;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const float ai = scale * dA[i];
        const float bi = eA ? scale * eA[i] : 0.0f;
        float *Gi = G + (long long)i * n;
        float *Pi = P ? P + (long long)i * n : nullptr;
        const float *Ci = C ? C + (long long)i * n : nullptr;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            float v = ai * dB[j];
            if (eA) v = fmaf(bi, eB[j], v);
            if (Ci) v += Ci[j];
            Gi[j] = v;
            if (Pi) Pi[j] = inv_n;
            gm = fmaxf(gm, fabsf(v));
        }
    }
    gm = warp_max(gm);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&st->gmax_bits, gm);
}

// X += C elementwise (the seeds' constant share of every gradient): float4 at a time
// over the first total - total % 4 elements (both 16-byte aligned), then the tail.
__global__ void __launch_bounds__(256) k_add_f32(float *__restrict__ X, const float *__restrict__ C, long long total) {
    const long long total4 = total >> 2;
    float4 *x4 = reinterpret_cast<float4 *>(X);
    const float4 *c4 = reinterpret_cast<const float4 *>(C);
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    for (long long t = tid; t < total4; t += stride) {
        float4 a = x4[t];
        const float4 b = __ldg(c4 + t);
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
        x4[t] = a;
    }
    for (long long t = (total4 << 2) + tid; t < total; t += stride) X[t] += C[t];
}

// Seeded matching: the block solution perm[m..n) (indices into the unseeded block)
// becomes the full permutation, and the seeds map to themselves.
__global__ void k_seed_perm(int32_t *perm, int n, int m) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        perm[i] = i < m ? i : perm[i] + m;
}

// out (n_full x n_full) = I_m (+) P22, P22 the n x n block iterate (n = n_full - m).
__global__ void __launch_bounds__(256) k_embed_block(const float *__restrict__ P22, int n, int m,
                                                     float *__restrict__ out) {
    const int nf = n + m;
    for (int i = blockIdx.x; i < nf; i += gridDim.x) {
        float *row = out + (long long)i * nf;
        for (int j = threadIdx.x; j < nf; j += blockDim.x) {
            float v;
            if (i < m || j < m)
                v = (i == j) ? 1.0f : 0.0f;
            else
                v = P22[(long long)(i - m) * n + (j - m)];
            row[j] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_absmax(const float *__restrict__ X, long long total, unsigned *out) {
    float gm = 0.0f;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x)
        gm = fmaxf(gm, fabsf(X[t]));
    gm = warp_max(gm);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, gm);
}

// ---------------------------------------------------------------- line search (K3)

// Q value at (row i, column j) from the BF16 split terms the GEMMs consumed.
__device__ __forceinline__ float q_terms(const __nv_bfloat16 *row, int ldq, int terms, int j) {
    float q = __bfloat162float(row[j]);
    if (terms > 1) q += __bfloat162float(row[ldq + j]);
    return q;
}

// Four columns of one row for the line-search sums: G, G_Q, P and Q (BF16 terms).
struct LsQuad {
    float4 g, h, p;
    float q[4];
};

__device__ __forceinline__ LsQuad ls_load(const float *__restrict__ G, const float *__restrict__ GQ,
                                          const float *__restrict__ P, const __nv_bfloat16 *__restrict__ qrow, int ldq,
                                          int terms, long long base, int j) {
    LsQuad u;
    u.g = *reinterpret_cast<const float4 *>(G + base + j);
    u.h = *reinterpret_cast<const float4 *>(GQ + base + j);
    u.p = *reinterpret_cast<const float4 *>(P + base + j);
    const uint2 qh = *reinterpret_cast<const uint2 *>(qrow + j);
    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&qh.x));
    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&qh.y));
    u.q[0] = lo.x; u.q[1] = lo.y; u.q[2] = hi.x; u.q[3] = hi.y;
    if (terms > 1) {
        const uint2 ql = *reinterpret_cast<const uint2 *>(qrow + ldq + j);
        const float2 l2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&ql.x));
        const float2 h2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&ql.y));
        u.q[0] += l2.x; u.q[1] += l2.y; u.q[2] += h2.x; u.q[3] += h2.y;
    }
    return u;
}

// The same four columns with Q recomputed in FP32 from the LOT duals,
// Q_ij = 2^(c (f_i + g_j - G_ij)) -- the expression (and so the value) the Q writer
// rounds for the products -- instead of read back from the products' BF16 operand.
__device__ __forceinline__ LsQuad ls_load_dual(const float *__restrict__ G, const float *__restrict__ GQ,
                                               const float *__restrict__ P, float fi, const float *__restrict__ g,
                                               float c, long long base, int j) {
    LsQuad u;
    u.g = *reinterpret_cast<const float4 *>(G + base + j);
    u.h = *reinterpret_cast<const float4 *>(GQ + base + j);
    u.p = *reinterpret_cast<const float4 *>(P + base + j);
    const float4 gj = __ldg(reinterpret_cast<const float4 *>(g + j));
    u.q[0] = fast_exp2((fi + gj.x - u.g.x) * c);
    u.q[1] = fast_exp2((fi + gj.y - u.g.y) * c);
    u.q[2] = fast_exp2((fi + gj.z - u.g.z) * c);
    u.q[3] = fast_exp2((fi + gj.w - u.g.w) * c);
    return u;
}

__device__ __forceinline__ void ls_accumulate(const LsQuad &u, float &a1, float &a2, float &a3) {
    const float d0 = u.q[0] - u.p.x, d1 = u.q[1] - u.p.y, d2 = u.q[2] - u.p.z, d3 = u.q[3] - u.p.w;
    a1 += u.g.x * d0 + u.g.y * d1 + u.g.z * d2 + u.g.w * d3;
    a2 += u.h.x * d0 + u.h.y * d1 + u.h.z * d2 + u.h.w * d3;
    a3 += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
}

// Per-block partial sums of <G, D>, <G_Q, D>, <D, D> with D = Q - P, where Q is
// recomputed in FP32 from the LOT duals (f, g non-null: the value the Sinkhorn step
// defines, unrounded), or given as BF16 split terms (FAQ's permutation, exact) or as
// FP32.  One block per row at a time; FP32 within a row segment, FP64 across.
__global__ void __launch_bounds__(256) k_ls_partial(const float *__restrict__ G, const float *__restrict__ GQ,
                                                    const float *__restrict__ P, const __nv_bfloat16 *__restrict__ Qb,
                                                    int ldq, int terms, const float *__restrict__ Qf,
                                                    const float *__restrict__ fd, const float *__restrict__ gd,
                                                    const DevState *__restrict__ st, int n, double *__restrict__ out) {
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const bool dual = fd != nullptr;
    const float c = dual ? st->c : 0.0f;
    const bool vec = ((n & 3) == 0) && (Qf == nullptr) &&
                     (((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(GQ) |
                        reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(gd)) & 15) == 0);
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const long long base = (long long)i * n;
        const __nv_bfloat16 *qrow = Qb ? Qb + (long long)i * ((long long)terms * ldq) : nullptr;
        const float fi = dual ? __ldg(fd + i) : 0.0f;
        float a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (vec) {
            // two steps' loads in flight before either is accumulated; the terms
            // are still added in the order of j
            const int step = blockDim.x * 4;
            int j = threadIdx.x * 4;
            if (dual) {
                for (; j + step < n; j += 2 * step) {
                    const LsQuad u = ls_load_dual(G, GQ, P, fi, gd, c, base, j);
                    const LsQuad v = ls_load_dual(G, GQ, P, fi, gd, c, base, j + step);
                    ls_accumulate(u, a1, a2, a3);
                    ls_accumulate(v, a1, a2, a3);
                }
                if (j < n) ls_accumulate(ls_load_dual(G, GQ, P, fi, gd, c, base, j), a1, a2, a3);
            } else {
                for (; j + step < n; j += 2 * step) {
                    const LsQuad u = ls_load(G, GQ, P, qrow, ldq, terms, base, j);
                    const LsQuad v = ls_load(G, GQ, P, qrow, ldq, terms, base, j + step);
                    ls_accumulate(u, a1, a2, a3);
                    ls_accumulate(v, a1, a2, a3);
                }
                if (j < n) ls_accumulate(ls_load(G, GQ, P, qrow, ldq, terms, base, j), a1, a2, a3);
            }
        } else {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const float q = dual ? fast_exp2((fi + __ldg(gd + j) - G[base + j]) * c)
                                     : (Qf ? Qf[base + j] : q_terms(qrow, ldq, terms, j));
                const float d = q - P[base + j];
                a1 = fmaf(G[base + j], d, a1);
                a2 = fmaf(GQ[base + j], d, a2);
                a3 = fmaf(d, d, a3);
            }
        }
        s1 += a1;
        s2 += a2;
        s3 += a3;
    }
    s1 = warp_sum_d(s1);
    s2 = warp_sum_d(s2);
    s3 = warp_sum_d(s3);
    __shared__ double red[3][8];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = s1;
        red[1][w] = s2;
        red[2][w] = s3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r1 = 0, r2 = 0, r3 = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            r1 += red[0][k];
            r2 += red[1][k];
            r3 += red[2][k];
        }
        out[3 * blockIdx.x + 0] = r1;
        out[3 * blockIdx.x + 1] = r2;
        out[3 * blockIdx.x + 2] = r3;
    }
}

// Sums the partials in a fixed order and solves the 1-D quadratic.
// b = -<G, D>, a = (1/2)(<G, D> - <G_Q, D>); alpha = argmax (maximize) over [0,1]
// of b t + a t^2.  Also applies the Frank-Wolfe stop test ||alpha D||_F / sqrt(n) < tol
// and records the trace.
__global__ void k_ls_final(const double *__restrict__ part, int nblocks, int n, DevState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s1 = 0, s2 = 0, s3 = 0;
    for (int k = 0; k < nblocks; ++k) {
        s1 += part[3 * k];
        s2 += part[3 * k + 1];
        s3 += part[3 * k + 2];
    }
    const double b = -s1, a = 0.5 * (s1 - s2);
    double alpha;
    if (st->maximize) {
        if (a < 0.0) {
            alpha = -b / (2.0 * a);
            alpha = alpha < 0.0 ? 0.0 : (alpha > 1.0 ? 1.0 : alpha);
        } else {
            alpha = (a + b > 0.0) ? 1.0 : 0.0;
        }
    } else {
        if (a > 0.0) {
            alpha = -b / (2.0 * a);
            alpha = alpha < 0.0 ? 0.0 : (alpha > 1.0 ? 1.0 : alpha);
        } else {
            alpha = (a + b < 0.0) ? 1.0 : 0.0;
        }
    }
    if (!(alpha == alpha)) {
        alpha = 0.0;
        if (!st->error) st->error = GOAT_ERR_NAN;
    }
    st->ls_a = a;
    st->ls_b = b;
    st->ls_dd = s3;
    st->alpha = alpha;
    const double change = alpha * sqrt(s3 > 0.0 ? s3 : 0.0) / sqrt((double)(st->stop_n > 0 ? st->stop_n : n));
    const int it = st->fw_iter;
    if (it < GOAT_TRACE_MAX) {
        st->tr_alpha[it] = alpha;
        st->tr_sk_iters[it] = st->sk_iters;
        st->tr_sk_resid[it] = st->sk_resid;
    }
    st->fw_iter = it + 1;
    if (change < (double)st->fw_tol) st->fw_done = 1;
}

// ---------------------------------------------------------------- update (K4)

// P <- P + alpha (Q - P), G <- G + alpha (G_Q - G); accumulates max|G_new|.
__global__ void __launch_bounds__(256) k_fw_update(float *__restrict__ P, float *__restrict__ G,
                                                   const float *__restrict__ GQ, const __nv_bfloat16 *__restrict__ Qb,
                                                   int ldq, int terms, const float *__restrict__ Qf,
                                                   const float *__restrict__ fd, const float *__restrict__ gd, int n,
                                                   const DevState *__restrict__ st, float alpha_value,
                                                   unsigned *gmax_out) {
    const float alpha = st ? (float)st->alpha : alpha_value;
    const bool dual = fd != nullptr;  // Q from the LOT duals and the G before the update
    const float c = dual ? st->c : 0.0f;
    float gm = 0.0f;
    const bool vec = ((n & 3) == 0) && (Qf == nullptr) &&
                     (((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(GQ) |
                        reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(gd)) & 15) == 0);
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const long long base = (long long)i * n;
        const __nv_bfloat16 *qrow = Qb ? Qb + (long long)i * ((long long)terms * ldq) : nullptr;
        const float fi = dual ? __ldg(fd + i) : 0.0f;
        if (vec) {
            for (int j = threadIdx.x * 4; j < n; j += blockDim.x * 4) {
                float4 p4 = *reinterpret_cast<const float4 *>(P + base + j);
                float4 g4 = *reinterpret_cast<const float4 *>(G + base + j);
                const float4 h4 = *reinterpret_cast<const float4 *>(GQ + base + j);
                float q[4];
                if (dual) {
                    const float4 gj = __ldg(reinterpret_cast<const float4 *>(gd + j));
                    q[0] = fast_exp2((fi + gj.x - g4.x) * c);
                    q[1] = fast_exp2((fi + gj.y - g4.y) * c);
                    q[2] = fast_exp2((fi + gj.z - g4.z) * c);
                    q[3] = fast_exp2((fi + gj.w - g4.w) * c);
                } else {
                    const uint2 qh = *reinterpret_cast<const uint2 *>(qrow + j);
                    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&qh.x));
                    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&qh.y));
                    q[0] = lo.x; q[1] = lo.y; q[2] = hi.x; q[3] = hi.y;
                }
                if (!dual && terms > 1) {
                    const uint2 ql = *reinterpret_cast<const uint2 *>(qrow + ldq + j);
                    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&ql.x));
                    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&ql.y));
                    q[0] += lo.x; q[1] += lo.y; q[2] += hi.x; q[3] += hi.y;
                }
                p4.x = fmaf(alpha, q[0] - p4.x, p4.x);
                p4.y = fmaf(alpha, q[1] - p4.y, p4.y);
                p4.z = fmaf(alpha, q[2] - p4.z, p4.z);
                p4.w = fmaf(alpha, q[3] - p4.w, p4.w);
                g4.x = fmaf(alpha, h4.x - g4.x, g4.x);
                g4.y = fmaf(alpha, h4.y - g4.y, g4.y);
                g4.z = fmaf(alpha, h4.z - g4.z, g4.z);
                g4.w = fmaf(alpha, h4.w - g4.w, g4.w);
                *reinterpret_cast<float4 *>(P + base + j) = p4;
                *reinterpret_cast<float4 *>(G + base + j) = g4;
                gm = fmaxf(gm, fmaxf(fmaxf(fabsf(g4.x), fabsf(g4.y)), fmaxf(fabsf(g4.z), fabsf(g4.w))));
            }
        } else {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const float p = P[base + j], g = G[base + j];
                const float q = dual ? fast_exp2((fi + __ldg(gd + j) - g) * c)
                                     : (Qf ? Qf[base + j] : q_terms(qrow, ldq, terms, j));
                P[base + j] = fmaf(alpha, q - p, p);
                const float gn = fmaf(alpha, GQ[base + j] - g, g);
                G[base + j] = gn;
                gm = fmaxf(gm, fabsf(gn));
            }
        }
    }
    gm = warp_max(gm);
    if (gmax_out && (threadIdx.x & 31) == 0) atomic_max_nonneg(gmax_out, gm);
}

// Moves the max|G| accumulated by the update into the current slot.
__global__ void k_fw_roll(DevState *st) {
    st->gmax_bits = st->gmax_next;
    st->gmax_next = 0u;
}

// ---------------------------------------------------------------- FAQ's first direction

// FAQ (Alg. 1) started at the barycenter: the direction step solves the linear
// assignment max_perm sum_i grad f(J)[i][perm i] with grad f(J) = (2/n) d_A d_B^T
// (symmetric A, B).  The matrix is rank one, so by the rearrangement inequality
// the optimum pairs the k-th largest degree of A with the k-th largest of B.
// Solving the assignment on the FP32 matrix instead is not exact: two pairings
// that swap vertices of nearly equal degree differ by about (relative degree
// gap)^2 of an entry, below FP32's resolution of G.  The degrees here are FP64
// sums (exact for 0/1 and for weights with few significant bits); equal degrees
// are ordered by vertex index, and every such order is an optimum.

// deg[i] = sum_j A[i][j] in FP64; one warp per row, a fixed lane order and tree.
template <typename T>
__global__ void __launch_bounds__(256) k_degrees_f64(const T *__restrict__ A, int n, double *__restrict__ deg) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) {
        const T *row = A + (long long)i * n;
        double acc = 0.0;
        for (int j = lane; j < n; j += 32) acc += (double)row[j];
        acc = warp_sum_d(acc);
        if (lane == 0) deg[i] = acc;
    }
}

// rank[i] = #{k : d_k > d_i, or d_k = d_i and k < i} (0 = largest), for two degree
// vectors at once (blockIdx.y selects A or B); the degrees pass through shared
// memory in tiles of 256.  With ascending_b the second vector is ranked from its
// smallest entry (QAP minimisation pairs large with small: the rearrangement
// inequality's other extreme).
__global__ void __launch_bounds__(256) k_degree_rank(const double *__restrict__ deg, int n, int ascending_b,
                                                     int *__restrict__ rank) {
    __shared__ double tile[256];
    const double *d = deg + (long long)blockIdx.y * n;
    const double sg = (blockIdx.y == 1 && ascending_b) ? -1.0 : 1.0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double di = i < n ? sg * d[i] : 0.0;
    int r = 0;
    for (int k0 = 0; k0 < n; k0 += 256) {
        __syncthreads();
        if (k0 + (int)threadIdx.x < n) tile[threadIdx.x] = sg * d[k0 + threadIdx.x];
        __syncthreads();
        const int lim = min(256, n - k0);
        for (int t = 0; t < lim; ++t) {
            const double dk = tile[t];
            r += (dk > di) || (dk == di && k0 + t < i);
        }
    }
    if (i < n) rank[(long long)blockIdx.y * n + i] = r;
}

// inv[rank_B[j]] = j; then perm[i] = inv[rank_A[i]].
__global__ void k_rank_invert(const int *__restrict__ rankB, int n, int *__restrict__ inv) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) inv[rankB[j]] = j;
}
__global__ void k_rank_pair(const int *__restrict__ rankA, const int *__restrict__ inv, int n, int32_t *perm) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) perm[i] = inv[rankA[i]];
}

// ---------------------------------------------------------------- objective

// Block-wide FP64 sum in a fixed order (a warp tree, then the warps in order);
// the result is valid in thread 0.  Every thread of the block calls it.
__device__ __forceinline__ double block_sum_fixed(double v) {
    __shared__ double s_part[32];
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
    __syncthreads();
    return t;
}

// sum_ij A_ij B[perm i][perm j]: exact 64-bit integer sums for byte inputs; for
// float inputs FP64 sums, one partial per block (fixed grid kObjBlocks) added in
// block order by k_sum_in_order, so the value is the same on every run.  Block b
// takes the rows b, b + gridDim.x, ...
template <typename T>
__global__ void __launch_bounds__(256) k_objective(const T *__restrict__ A, const T *__restrict__ B,
                                                   const int32_t *__restrict__ perm, int n,
                                                   unsigned long long *isum, double *fpart, int *bad_perm) {
    long long acc_i = 0;
    double acc_f = 0.0;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int pi = perm[i];
        if (pi < 0 || pi >= n) {
            if (threadIdx.x == 0) atomicAdd(bad_perm, 1);
            continue;
        }
        const T *ai = A + (long long)i * n;
        const T *bp = B + (long long)pi * n;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const T a = ai[j];
            if (a != (T)0) {
                const int pj = perm[j];
                if (pj < 0 || pj >= n) continue;
                const T b = bp[pj];
                if (sizeof(T) == 1)
                    acc_i += (long long)a * (long long)b;
                else
                    acc_f += (double)a * (double)b;
            }
        }
    }
    if (sizeof(T) == 1) {
        for (int o = 16; o > 0; o >>= 1) acc_i += __shfl_xor_sync(0xffffffffu, acc_i, o);
        if ((threadIdx.x & 31) == 0 && acc_i) atomicAdd(isum, (unsigned long long)acc_i);  // exact in any order
    } else {
        const double t = block_sum_fixed(acc_f);
        if (threadIdx.x == 0) fpart[blockIdx.x] = t;
    }
}

// Sum of squared entries (||A||_F^2) for the disagreement count; same scheme.
template <typename T>
__global__ void __launch_bounds__(256) k_sqnorm(const T *__restrict__ A, long long total, unsigned long long *isum,
                                                double *fpart) {
    long long ai = 0;
    double af = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const T a = A[t];
        if (sizeof(T) == 1)
            ai += (long long)a * a;
        else
            af += (double)a * (double)a;
    }
    if (sizeof(T) == 1) {
        for (int o = 16; o > 0; o >>= 1) ai += __shfl_xor_sync(0xffffffffu, ai, o);
        if ((threadIdx.x & 31) == 0 && ai) atomicAdd(isum, (unsigned long long)ai);
    } else {
        const double t = block_sum_fixed(af);
        if (threadIdx.x == 0) fpart[blockIdx.x] = t;
    }
}

// out[k] = sum_b part[k * count + b] over b in increasing order, k < sets; one thread per set.
__global__ void k_sum_in_order(const double *__restrict__ part, int count, int sets, double *out) {
    const int k = threadIdx.x;
    if (k >= sets) return;
    double t = 0.0;
    for (int b = 0; b < count; ++b) t += part[(long long)k * count + b];
    out[k] = t;
}

// ---------------------------------------------------------------- host wrappers

static int grid_for(long long work, int per_block = 256, int cap_per_sm = 16) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long g = ceil_div(work, per_block);
    return (int)std::max<long long>(1, std::min<long long>(g, (long long)sms * cap_per_sm));
}

static int rows_grid(int n, int cap_per_sm = 8) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, std::min(n, sms * cap_per_sm));
}

static const void *window(const AdjView &v, int r0, int c0) {
    const size_t es = v.dtype == GOAT_DTYPE_U8 ? 1 : 4;
    return (const uint8_t *)v.p + ((size_t)r0 * (size_t)v.ld + (size_t)c0) * es;
}

int adj_to_bf16(const AdjView &v, int r0, int c0, int rows, int cols, __nv_bfloat16 *dst, int width, long long stride,
                float *deg, cudaStream_t s) {
    note_launches(1);
    const int grid = grid_for((long long)rows * 32, 256, 16);
    const void *src = window(v, r0, c0);
    if (v.dtype == GOAT_DTYPE_U8)
        k_adj_to_bf16<uint8_t><<<grid, 256, 0, s>>>((const uint8_t *)src, v.ld, rows, cols, dst, width, stride, deg);
    else
        k_adj_to_bf16<float><<<grid, 256, 0, s>>>((const float *)src, v.ld, rows, cols, dst, width, stride, deg);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

int adj_to_e4m3(const AdjView &v, int r0, int c0, int rows, int cols, uint8_t *dst, int width, long long stride,
                cudaStream_t s) {
    note_launches(1);
    const int grid = grid_for((long long)rows * (width / 2));
    const void *src = window(v, r0, c0);
    if (v.dtype == GOAT_DTYPE_U8)
        k_adj_to_e4m3<uint8_t><<<grid, 256, 0, s>>>((const uint8_t *)src, v.ld, rows, cols, dst, width, stride);
    else
        k_adj_to_e4m3<float><<<grid, 256, 0, s>>>((const float *)src, v.ld, rows, cols, dst, width, stride);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

template <typename O>
static int adj_transpose(const AdjView &v, int r0, int c0, int rows, int cols, O *dst, int width, long long stride,
                         cudaStream_t s) {
    note_launches(1);
    const dim3 grid((unsigned)ceil_div(width, 32), (unsigned)ceil_div(cols, 32)), block(32, 8);
    const void *src = window(v, r0, c0);
    if (v.dtype == GOAT_DTYPE_U8)
        k_adj_transpose<uint8_t, O><<<grid, block, 0, s>>>((const uint8_t *)src, v.ld, rows, cols, dst, width, stride);
    else
        k_adj_transpose<float, O><<<grid, block, 0, s>>>((const float *)src, v.ld, rows, cols, dst, width, stride);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

int adj_to_bf16_t(const AdjView &v, int r0, int c0, int rows, int cols, __nv_bfloat16 *dst, int width,
                  long long stride, cudaStream_t s) {
    return adj_transpose<__nv_bfloat16>(v, r0, c0, rows, cols, dst, width, stride, s);
}

int adj_to_e4m3_t(const AdjView &v, int r0, int c0, int rows, int cols, uint8_t *dst, int width, long long stride,
                  cudaStream_t s) {
    return adj_transpose<uint8_t>(v, r0, c0, rows, cols, dst, width, stride, s);
}

int adj_col_sums(const AdjView &v, int r0, int c0, int rows, int cols, float *out, cudaStream_t s) {
    note_launches(1);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(cols, 256), 4096));
    const void *src = window(v, r0, c0);
    if (v.dtype == GOAT_DTYPE_U8)
        k_col_sums<uint8_t><<<grid, 256, 0, s>>>((const uint8_t *)src, v.ld, rows, cols, out);
    else
        k_col_sums<float><<<grid, 256, 0, s>>>((const float *)src, v.ld, rows, cols, out);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

int bf16_to_e4m3(const __nv_bfloat16 *X, int rows, int ld_src, uint8_t *X8, int ld8, unsigned *amax_bits,
                 float *inv_scale, cudaStream_t s) {
    note_launches(2);
    cudaMemsetAsync(amax_bits, 0, sizeof(unsigned), s);
    k_absmax_bf16<<<grid_for((long long)rows * ld_src / 8), 256, 0, s>>>(X, (long long)rows * ld_src, amax_bits);
    k_bf16_to_e4m3<<<grid_for((long long)rows * (ld8 / 16)), 256, 0, s>>>(X, rows, ld_src, X8, ld8, amax_bits,
                                                                          inv_scale);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

int split_lo_to_e4m3(__nv_bfloat16 *C1, int rows, int ld, int parts, uint8_t *C8, int w8, unsigned *amax_bits,
                     float *inv_scale, cudaStream_t s) {
    if ((ld % 64) || (w8 % 128) || w8 < ld) return GOAT_ERR_INVALID_ARG;
    note_launches(2);
    const long long cs = 2LL * parts * ld;
    cudaMemsetAsync(amax_bits, 0, sizeof(unsigned), s);
    k_absmax_bf16<<<grid_for((long long)rows * cs / 8), 256, 0, s>>>(C1, (long long)rows * cs, amax_bits);
    k_split_lo_to_e4m3<<<grid_for((long long)rows * parts * (w8 / 16)), 256, 0, s>>>(C1, rows, ld, parts, cs, C8, w8,
                                                                                     amax_bits, inv_scale);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

int count_asym(const void *A, int dtype, int n, int *count_dev, cudaStream_t s) {
    note_launches(1);
    dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(n, 32)), block(32, 8);
    if (dtype == GOAT_DTYPE_U8)
        k_count_asym<uint8_t><<<grid, block, 0, s>>>((const uint8_t *)A, n, count_dev);
    else
        k_count_asym<float><<<grid, block, 0, s>>>((const float *)A, n, count_dev);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

void f32_to_terms(const float *X, int n, long long ldx, __nv_bfloat16 *Xb, int ld16, int terms, cudaStream_t s) {
    note_launches(1);
    k_f32_to_terms<<<grid_for((long long)n * (ld16 / 8)), 256, 0, s>>>(X, n, ldx, Xb, ld16, terms);
}

void barycenter(const float *dA, const float *dB, const float *eA, const float *eB, int n, float scale,
                const float *C, float *G, float *P, DevState *st, cudaStream_t s) {
    note_launches(1);
    k_barycenter<<<rows_grid(n), 256, 0, s>>>(dA, dB, eA, eB, n, scale, C, G, P, st);
}

void add_f32(float *X, const float *C, long long total, cudaStream_t s) {
    note_launches(1);
    k_add_f32<<<grid_for(total / 4 + 1), 256, 0, s>>>(X, C, total);
}

void seed_perm(int32_t *perm, int n, int m, cudaStream_t s) {
    note_launches(1);
    k_seed_perm<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 1024)), 256, 0, s>>>(perm, n, m);
}

void embed_block(const float *P22, int n, int m, float *out, cudaStream_t s) {
    note_launches(1);
    k_embed_block<<<rows_grid(n + m), 256, 0, s>>>(P22, n, m, out);
}

void absmax(const float *X, long long total, unsigned *out, cudaStream_t s) {
    note_launches(1);
    k_absmax<<<grid_for(total), 256, 0, s>>>(X, total, out);
}

size_t rearrangement_scratch_bytes(int n) { return (size_t)n * (2 * sizeof(double) + 3 * sizeof(int)); }

int rearrangement_perm(const void *A, const void *B, int dtype, int n, int maximize, void *scratch, int32_t *perm,
                       cudaStream_t s) {
    double *deg = reinterpret_cast<double *>(scratch);
    int *rank = reinterpret_cast<int *>(deg + 2 * (size_t)n);
    int *inv = rank + 2 * (size_t)n;
    const int gw = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 8), 152LL * 16));
    if (dtype == GOAT_DTYPE_U8) {
        k_degrees_f64<uint8_t><<<gw, 256, 0, s>>>((const uint8_t *)A, n, deg);
        k_degrees_f64<uint8_t><<<gw, 256, 0, s>>>((const uint8_t *)B, n, deg + n);
    } else {
        k_degrees_f64<float><<<gw, 256, 0, s>>>((const float *)A, n, deg);
        k_degrees_f64<float><<<gw, 256, 0, s>>>((const float *)B, n, deg + n);
    }
    k_degree_rank<<<dim3((unsigned)ceil_div(n, 256), 2), 256, 0, s>>>(deg, n, maximize ? 0 : 1, rank);
    const int g = (int)std::min<int64_t>(ceil_div(n, 256), 1024);
    k_rank_invert<<<g, 256, 0, s>>>(rank + n, n, inv);
    k_rank_pair<<<g, 256, 0, s>>>(rank, inv, n, perm);
    note_launches(5);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

// FAQ's direction (Alg. 1): Q = the permutation matrix of perm (Q[i][perm i] = 1),
// as BF16 terms in the GEMM operand buffer, which the caller zeroed.
__global__ void __launch_bounds__(256) k_write_perm_q(const int32_t *__restrict__ perm, int n,
                                                      __nv_bfloat16 *__restrict__ Qb, int ldq, int terms) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = perm[i];
        if (j >= 0 && j < n) Qb[(long long)i * ((long long)terms * ldq) + j] = __float2bfloat16(1.0f);
    }
}

int write_perm_q(const int32_t *perm, int n, __nv_bfloat16 *Qb, int ldq, int terms, cudaStream_t s) {
    if (cudaMemsetAsync(Qb, 0, (size_t)n * terms * ldq * sizeof(__nv_bfloat16), s) != cudaSuccess)
        return GOAT_ERR_CUDA;
    note_launches(1);
    k_write_perm_q<<<(int)std::min<int64_t>(ceil_div(n, 256), 1024), 256, 0, s>>>(perm, n, Qb, ldq, terms);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

int ls_blocks(int n) { return rows_grid(n, 4); }

void line_search(const float *G, const float *GQ, const float *P, const __nv_bfloat16 *Qb, int ldq, int terms,
                 const float *Qf, const float *f, const float *g, int n, double *partial, DevState *st,
                 cudaStream_t s) {
    note_launches(2);
    const int nb = ls_blocks(n);
    k_ls_partial<<<nb, 256, 0, s>>>(G, GQ, P, Qb, ldq, terms, Qf, f, g, st, n, partial);
    k_ls_final<<<1, 32, 0, s>>>(partial, nb, n, st);
}

void fw_update(float *P, float *G, const float *GQ, const __nv_bfloat16 *Qb, int ldq, int terms, const float *Qf,
               const float *f, const float *g, int n, const DevState *st, float alpha_value, unsigned *gmax_out,
               cudaStream_t s) {
    note_launches(1);
    k_fw_update<<<rows_grid(n), 256, 0, s>>>(P, G, GQ, Qb, ldq, terms, Qf, f, g, n, st, alpha_value, gmax_out);
}

void fw_roll(DevState *st, cudaStream_t s) { k_fw_roll<<<1, 1, 0, s>>>(st); }

int objective(const void *A, const void *B, int dtype, int n, const int32_t *perm, unsigned long long *isum,
              double *fsum, unsigned long long *nA, unsigned long long *nB, double *fA, double *fB, int *bad,
              double *fpart, cudaStream_t s) {
    const long long total = (long long)n * n;
    if (dtype == GOAT_DTYPE_U8) {
        note_launches(3);
        const int grid = (int)std::min<long long>(n, 152LL * 8);
        k_objective<uint8_t><<<grid, 256, 0, s>>>((const uint8_t *)A, (const uint8_t *)B, perm, n, isum, nullptr, bad);
        k_sqnorm<uint8_t><<<grid_for(total), 256, 0, s>>>((const uint8_t *)A, total, nA, nullptr);
        k_sqnorm<uint8_t><<<grid_for(total), 256, 0, s>>>((const uint8_t *)B, total, nB, nullptr);
    } else {
        // fixed grids: the FP64 partial sums and their order do not depend on the device
        note_launches(4);
        k_objective<float><<<kObjBlocks, 256, 0, s>>>((const float *)A, (const float *)B, perm, n, isum, fpart, bad);
        k_sqnorm<float><<<kObjBlocks, 256, 0, s>>>((const float *)A, total, nA, fpart + kObjBlocks);
        k_sqnorm<float><<<kObjBlocks, 256, 0, s>>>((const float *)B, total, nB, fpart + 2 * kObjBlocks);
        // fsum, fA, fB are consecutive doubles (the callers' layout)
        if (fA != fsum + 1 || fB != fsum + 2) return GOAT_ERR_INVALID_ARG;
        k_sum_in_order<<<1, 32, 0, s>>>(fpart, kObjBlocks, 3, fsum);
    }
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

}  // namespace goat
