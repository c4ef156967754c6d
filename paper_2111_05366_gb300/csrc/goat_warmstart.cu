// goat_warmstart.cu -- the learned Sinkhorn warm start: a small MLP that predicts
// the dual potentials of LOT (Alg. 2) from per-node features, with hand-written
// feature (K6), inference (K7) and training (K8: backward + Adam) kernels.
//
// Nodes.  The A-side nodes are the rows of G (their dual is f_i), the B-side
// nodes its columns (dual g_j).  Features of a node, all scale-free:
//   0 degree / mean degree          (row sums of A, or of B)
//   1 2-hop degree / its mean       ((A d_A)_i, or (B d_B)_j)
//   2 mean of its line of G, / eps  (row i of G, or column j)
//   3 max of the line / eps
//   4 std of the line / eps
//   5 min of the line / eps
//   6 side (0: A / row, 1: B / column)
//   7 ln(n) / 10
// Network: y = w2 . tanh(W1 x + b1) + b2, hidden width 64, weights stored in BF16
// (the forward pass, training and inference all use the BF16 values; the
// optimiser keeps FP32 master copies).  y predicts the node's dual in units of
// eps with each side's mean removed (duals are defined up to f + c, g - c).
// Packed parameters: W1 [64][8] at 0, b1 at 512, w2 at 576, b2 at 640 (641 values).
#include <algorithm>
#include <cmath>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

constexpr int MLP_IN = 8, MLP_H = 64, MLP_NP = GOAT_MLP_PARAMS;
constexpr int OFF_B1 = 512, OFF_W2 = 576, OFF_B2 = 640;

// ---------------------------------------------------------------- K6: features

// Row statistics of G and row sums of A and B (one warp per row).  stats layout:
// [2n][4] = mean, max, std, min of each node's line in units of eps.
template <typename T>
__global__ void __launch_bounds__(256) k_feat_rows(const float *__restrict__ G, const T *__restrict__ A,
                                                   const T *__restrict__ B, int n, float inv_eps,
                                                   float *__restrict__ stats, float *__restrict__ deg,
                                                   double *__restrict__ sums) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    double dA_sum = 0.0, dB_sum = 0.0;
    for (int i = gw; i < n; i += nw) {
        const float *Gi = G + (long long)i * n;
        float s = 0.f, s2 = 0.f, mx = -INFINITY, mn = INFINITY, da = 0.f, db = 0.f;
        for (int j = lane; j < n; j += 32) {
            const float x = Gi[j] * inv_eps;
            s += x;
            s2 += x * x;
            mx = fmaxf(mx, x);
            mn = fminf(mn, x);
            da += (float)A[(long long)i * n + j];
            db += (float)B[(long long)i * n + j];
        }
        s = warp_sum(s);
        s2 = warp_sum(s2);
        da = warp_sum(da);
        db = warp_sum(db);
        mx = warp_max(mx);
        for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        if (lane == 0) {
            const float mean = s / n;
            stats[(long long)i * 4 + 0] = mean;
            stats[(long long)i * 4 + 1] = mx;
            stats[(long long)i * 4 + 2] = sqrtf(fmaxf(s2 / n - mean * mean, 0.f));
            stats[(long long)i * 4 + 3] = mn;
            deg[i] = da;
            deg[n + i] = db;
            dA_sum += da;
            dB_sum += db;
        }
    }
    if (lane == 0) {
        atomicAdd(sums + 0, dA_sum);
        atomicAdd(sums + 1, dB_sum);
    }
}

// Column statistics of G in two steps.  k_feat_colpart: a CTA takes 1024 columns
// (4 adjacent ones per thread: float4 loads when G is 16-byte aligned and n a
// multiple of 4, else scalar) and one chunk of rows, four rows' loads in flight;
// it writes the chunk's sum, sum of squares, max and min of every column (in units
// of eps).  k_feat_colmerge adds the chunks in chunk order, so the result does not
// depend on the launch's timing.
constexpr int kFeatColsPerCta = 1024;
constexpr int kFeatMaxChunks = 64;

__global__ void __launch_bounds__(256) k_feat_colpart(const float *__restrict__ G, int n, float inv_eps,
                                                      int rows_per_chunk, float4 *__restrict__ part) {
    const int j0 = blockIdx.x * kFeatColsPerCta + 4 * threadIdx.x;
    if (j0 >= n) return;
    const int r0 = blockIdx.y * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    const bool vec = (j0 + 3 < n) && (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(G) & 15) == 0);
    const int kmax = min(4, n - j0);
    float s[4], s2[4], mx[4], mn[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        s[k] = 0.f;
        s2[k] = 0.f;
        mx[k] = -INFINITY;
        mn[k] = INFINITY;
    }
    auto add = [&](int k, float x) {
        const float v = x * inv_eps;
        s[k] += v;
        s2[k] = fmaf(v, v, s2[k]);
        mx[k] = fmaxf(mx[k], v);
        mn[k] = fminf(mn[k], v);
    };
    int i = r0;
    if (vec) {
        for (; i + 3 < r1; i += 4) {
            float4 a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = __ldg(reinterpret_cast<const float4 *>(G + (long long)(i + u) * n + j0));
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                add(0, a[u].x);
                add(1, a[u].y);
                add(2, a[u].z);
                add(3, a[u].w);
            }
        }
    }
    for (; i < r1; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < kmax) add(k, __ldg(G + (long long)i * n + j0 + k));
    }
    for (int k = 0; k < kmax; ++k) part[(size_t)blockIdx.y * n + j0 + k] = make_float4(s[k], s2[k], mx[k], mn[k]);
}

__global__ void k_feat_colmerge(const float4 *__restrict__ part, int chunks, int n, float *__restrict__ stats) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float s = 0.f, s2 = 0.f, mx = -INFINITY, mn = INFINITY;
    for (int c = 0; c < chunks; ++c) {
        const float4 p = part[(size_t)c * n + j];
        s += p.x;
        s2 += p.y;
        mx = fmaxf(mx, p.z);
        mn = fminf(mn, p.w);
    }
    const float mean = s / n;
    float *o = stats + (long long)(n + j) * 4;
    o[0] = mean;
    o[1] = mx;
    o[2] = sqrtf(fmaxf(s2 / n - mean * mean, 0.f));
    o[3] = mn;
}

// 2-hop degrees (A d_A)_i and (B d_B)_j (one warp per row).
template <typename T>
__global__ void __launch_bounds__(256) k_feat_hop2(const T *__restrict__ A, const T *__restrict__ B, int n,
                                                   const float *__restrict__ deg, float *__restrict__ hop2,
                                                   double *__restrict__ sums) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    double ha = 0.0, hb = 0.0;
    for (int i = gw; i < n; i += nw) {
        float sa = 0.f, sb = 0.f;
        for (int k = lane; k < n; k += 32) {
            sa += (float)A[(long long)i * n + k] * deg[k];
            sb += (float)B[(long long)i * n + k] * deg[n + k];
        }
        sa = warp_sum(sa);
        sb = warp_sum(sb);
        if (lane == 0) {
            hop2[i] = sa;
            hop2[n + i] = sb;
            ha += sa;
            hb += sb;
        }
    }
    if (lane == 0) {
        atomicAdd(sums + 2, ha);
        atomicAdd(sums + 3, hb);
    }
}

__global__ void k_feat_assemble(int n, const float *__restrict__ stats, const float *__restrict__ deg,
                                const float *__restrict__ hop2, const double *__restrict__ sums,
                                float *__restrict__ feats) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= 2 * n) return;
    const int side = v >= n;
    const double mdeg = sums[side ? 1 : 0] / n, mhop = sums[side ? 3 : 2] / n;
    float *o = feats + (long long)v * MLP_IN;
    o[0] = mdeg > 0 ? (float)(deg[v] / mdeg) : 0.f;
    o[1] = mhop > 0 ? (float)(hop2[v] / mhop) : 0.f;
    o[2] = stats[(long long)v * 4 + 0];
    o[3] = stats[(long long)v * 4 + 1];
    o[4] = stats[(long long)v * 4 + 2];
    o[5] = stats[(long long)v * 4 + 3];
    o[6] = (float)side;
    o[7] = logf((float)n) * 0.1f;
}

// ---------------------------------------------------------------- K7: inference

__device__ __forceinline__ void load_weights(const __nv_bfloat16 *__restrict__ w, float *sw) {
    for (int k = threadIdx.x; k < MLP_NP; k += blockDim.x) sw[k] = __bfloat162float(w[k]);
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_mlp_forward(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ x,
                                                     int N, float *__restrict__ y) {
    __shared__ float sw[MLP_NP];
    load_weights(w, sw);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        float xi[MLP_IN];
#pragma unroll
        for (int d = 0; d < MLP_IN; ++d) xi[d] = x[(long long)s * MLP_IN + d];
        float out = sw[OFF_B2];
#pragma unroll 8
        for (int k = 0; k < MLP_H; ++k) {
            float z = sw[OFF_B1 + k];
#pragma unroll
            for (int d = 0; d < MLP_IN; ++d) z = fmaf(sw[k * MLP_IN + d], xi[d], z);
            out = fmaf(sw[OFF_W2 + k], tanhf(z), out);
        }
        y[s] = out;
    }
}

// ---------------------------------------------------------------- K8: training

constexpr int TS = 128;  // samples per block in the backward pass

// Forward + backward of the mean squared error over N samples; gradients are
// accumulated (per block in shared memory, then atomically) into grad[641];
// loss[0] += mean squared error.
__global__ void __launch_bounds__(TS) k_mlp_backward(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ x,
                                                     const float *__restrict__ t, int N, float *__restrict__ grad,
                                                     float *__restrict__ loss) {
    __shared__ float sw[MLP_NP];
    __shared__ float sx[TS][MLP_IN];
    __shared__ float sdy[TS];
    __shared__ float sH[TS][MLP_H + 1];
    __shared__ float sdZ[TS][MLP_H + 1];
    load_weights(w, sw);
    const int s0 = blockIdx.x * TS;
    const int s = s0 + threadIdx.x;
    const bool valid = s < N;
    float xi[MLP_IN];
#pragma unroll
    for (int d = 0; d < MLP_IN; ++d) {
        xi[d] = valid ? x[(long long)s * MLP_IN + d] : 0.f;
        sx[threadIdx.x][d] = xi[d];
    }
    float out = sw[OFF_B2];
    for (int k = 0; k < MLP_H; ++k) {
        float z = sw[OFF_B1 + k];
#pragma unroll
        for (int d = 0; d < MLP_IN; ++d) z = fmaf(sw[k * MLP_IN + d], xi[d], z);
        const float h = tanhf(z);
        sH[threadIdx.x][k] = h;
        out = fmaf(sw[OFF_W2 + k], h, out);
    }
    const float err = valid ? out - t[s] : 0.f;
    const float dy = 2.0f * err / (float)N;
    sdy[threadIdx.x] = dy;
    for (int k = 0; k < MLP_H; ++k) {
        const float h = sH[threadIdx.x][k];
        sdZ[threadIdx.x][k] = dy * sw[OFF_W2 + k] * (1.0f - h * h);
    }
    float l = warp_sum(err * err / (float)N);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
    __syncthreads();
    // reduce over the block's samples: thread r handles parameters r, r + TS, ...
    for (int prm = threadIdx.x; prm < MLP_NP; prm += TS) {
        float acc = 0.f;
        if (prm < OFF_B1) {  // W1[k][d]
            const int k = prm / MLP_IN, d = prm % MLP_IN;
            for (int q = 0; q < TS; ++q) acc = fmaf(sdZ[q][k], sx[q][d], acc);
        } else if (prm < OFF_W2) {  // b1[k]
            const int k = prm - OFF_B1;
            for (int q = 0; q < TS; ++q) acc += sdZ[q][k];
        } else if (prm < OFF_B2) {  // w2[k]
            const int k = prm - OFF_W2;
            for (int q = 0; q < TS; ++q) acc = fmaf(sdy[q], sH[q][k], acc);
        } else {  // b2
            for (int q = 0; q < TS; ++q) acc += sdy[q];
        }
        atomicAdd(grad + prm, acc);
    }
}

// Adam (Kingma and Ba): FP32 master weights and moments, BF16 copy for the kernels.
__global__ void k_mlp_adam(float *__restrict__ master, float *__restrict__ m, float *__restrict__ v,
                           __nv_bfloat16 *__restrict__ w, const float *__restrict__ grad, float lr, int step) {
    const float b1 = 0.9f, b2 = 0.999f, e = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    for (int k = threadIdx.x; k < MLP_NP; k += blockDim.x) {
        const float g = grad[k];
        const float mk = b1 * m[k] + (1.0f - b1) * g;
        const float vk = b2 * v[k] + (1.0f - b2) * g * g;
        m[k] = mk;
        v[k] = vk;
        const float p = master[k] - lr * (mk / c1) / (sqrtf(vk / c2) + e);
        master[k] = p;
        w[k] = __float2bfloat16_rn(p);
    }
}

// ---------------------------------------------------------------- host wrappers

// Row chunks of the column statistics: as many as fill one wave of 8 CTAs per SM,
// at least 32 rows each, at most kFeatMaxChunks.
static int feat_col_chunks(int n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = ceil_div(n, kFeatColsPerCta);
    long long c = std::max<long long>(1, (long long)sms * 8 / tiles);
    c = std::min<long long>(c, std::max<long long>(1, n / 32));
    return (int)std::min<long long>(c, kFeatMaxChunks);
}

int dual_features(const float *G, const void *A, const void *B, int n, int dtype, float eps, float *feats,
                  float *scratch, cudaStream_t s) {
    // scratch: stats 8n floats, deg 2n, hop2 2n, sums 4 doubles, then (16-byte aligned)
    // the column chunks' partial statistics, kFeatMaxChunks x n float4
    float *stats = scratch, *deg = scratch + 8LL * n, *hop2 = deg + 2LL * n;
    double *sums = reinterpret_cast<double *>(hop2 + round_up(2LL * n, 4));
    float4 *colpart = reinterpret_cast<float4 *>(round_up(reinterpret_cast<uintptr_t>(sums + 4), 16));
    cudaMemsetAsync(sums, 0, 4 * sizeof(double), s);
    const int gw = (int)std::max<long long>(1, std::min<long long>(ceil_div(n, 8), 152LL * 16));
    const float inv_eps = 1.0f / eps;
    if (dtype == GOAT_DTYPE_U8) {
        k_feat_rows<uint8_t><<<gw, 256, 0, s>>>(G, (const uint8_t *)A, (const uint8_t *)B, n, inv_eps, stats, deg,
                                                sums);
        k_feat_hop2<uint8_t><<<gw, 256, 0, s>>>((const uint8_t *)A, (const uint8_t *)B, n, deg, hop2, sums);
    } else {
        k_feat_rows<float><<<gw, 256, 0, s>>>(G, (const float *)A, (const float *)B, n, inv_eps, stats, deg, sums);
        k_feat_hop2<float><<<gw, 256, 0, s>>>((const float *)A, (const float *)B, n, deg, hop2, sums);
    }
    const int chunks = feat_col_chunks(n);
    k_feat_colpart<<<dim3((unsigned)ceil_div(n, kFeatColsPerCta), chunks), 256, 0, s>>>(
        G, n, inv_eps, (int)ceil_div(n, chunks), colpart);
    k_feat_colmerge<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(colpart, chunks, n, stats);
    k_feat_assemble<<<(unsigned)ceil_div(2LL * n, 256), 256, 0, s>>>(n, stats, deg, hop2, sums, feats);
    note_launches(5);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

size_t dual_features_scratch_bytes(int n) {
    return (size_t)(12LL * n + 8) * sizeof(float) + 4 * sizeof(double) + 16 + (size_t)kFeatMaxChunks * n * sizeof(float4);
}

int mlp_forward(const __nv_bfloat16 *w, const float *x, int N, float *y, cudaStream_t s) {
    const int grid = (int)std::max<long long>(1, std::min<long long>(ceil_div(N, 256), 152LL * 8));
    k_mlp_forward<<<grid, 256, 0, s>>>(w, x, N, y);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

// Training targets of the network: t = [f / eps - mean(f / eps), g / eps - mean(g / eps)]
// (the duals are defined up to f + c, g - c).  One CTA; the means are FP64 sums in a
// fixed order (strided per thread, then a tree), so t does not depend on timing.
__global__ void __launch_bounds__(1024) k_dual_targets(const float *__restrict__ f, const float *__restrict__ g, int n,
                                                       float eps, float *__restrict__ t) {
    __shared__ double sf[1024], sg[1024];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += (double)f[i] / eps;
        b += (double)g[i] / eps;
    }
    sf[threadIdx.x] = a;
    sg[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sf[threadIdx.x] += sf[threadIdx.x + o];
            sg[threadIdx.x] += sg[threadIdx.x + o];
        }
        __syncthreads();
    }
    const double mf = sf[0] / n, mg = sg[0] / n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        t[i] = (float)((double)f[i] / eps - mf);
        t[n + i] = (float)((double)g[i] / eps - mg);
    }
}

// Sets g_j = eps * (MLP prediction of the B-side node j) as the Sinkhorn warm start.
__global__ void k_scale_duals(const float *__restrict__ y, int n, float eps, float *__restrict__ g) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) g[j] = eps * y[n + j];
}

int mlp_warm_start_g(const float *G, const void *A, const void *B, int n, int dtype, float eps,
                     const __nv_bfloat16 *w, float *g, float *scratch, cudaStream_t s) {
    float *feats = scratch;
    float *y = feats + 16LL * n;
    float *fs = y + 2LL * n;
    int st = dual_features(G, A, B, n, dtype, eps, feats, fs, s);
    if (st) return st;
    st = mlp_forward(w, feats, 2 * n, y, s);
    if (st) return st;
    k_scale_duals<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(y, n, eps, g);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

size_t mlp_warm_start_scratch_bytes(int n) {
    return (size_t)18LL * n * sizeof(float) + dual_features_scratch_bytes(n) + 256;
}

}  // namespace goat

using namespace goat;

extern "C" {

int goat_dual_features(const float *G, const void *A, const void *B, int n, int dtype_AB, float eps, float *feats,
                       void *workspace, size_t workspace_bytes, goat_stream_t stream) {
    if (!G || !A || !B || !feats || n < 1 || !(eps > 0.f) || (dtype_AB != GOAT_DTYPE_U8 && dtype_AB != GOAT_DTYPE_F32))
        return GOAT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t need = dual_features_scratch_bytes(n);
    float *scratch = (float *)workspace;
    bool own = false;
    if (scratch) {
        if (workspace_bytes < need) return GOAT_ERR_OUT_OF_MEMORY;
    } else {
        if (cudaMallocAsync((void **)&scratch, need, s) != cudaSuccess) {
            cudaGetLastError();
            return GOAT_ERR_OUT_OF_MEMORY;
        }
        own = true;
    }
    const int st = dual_features(G, A, B, n, dtype_AB, eps, feats, scratch, s);
    if (own) cudaFreeAsync(scratch, s);
    return st;
}

int goat_mlp_warm_start(const float *G, const void *A, const void *B, int n, int dtype_AB, float eps,
                        const void *weights_bf16, float *g_out, void *workspace, size_t workspace_bytes,
                        goat_stream_t stream) {
    if (!G || !A || !B || !weights_bf16 || !g_out || n < 1 || !(eps > 0.f) ||
        (dtype_AB != GOAT_DTYPE_U8 && dtype_AB != GOAT_DTYPE_F32))
        return GOAT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t need = mlp_warm_start_scratch_bytes(n);
    float *scratch = (float *)workspace;
    bool own = false;
    if (scratch) {
        if (workspace_bytes < need) return GOAT_ERR_OUT_OF_MEMORY;
    } else {
        if (cudaMallocAsync((void **)&scratch, need, s) != cudaSuccess) {
            cudaGetLastError();
            return GOAT_ERR_OUT_OF_MEMORY;
        }
        own = true;
    }
    const int st = mlp_warm_start_g(G, A, B, n, dtype_AB, eps, (const __nv_bfloat16 *)weights_bf16, g_out, scratch, s);
    if (own) cudaFreeAsync(scratch, s);
    return st;
}

int goat_dual_targets(const float *f, const float *g, int n, float eps, float *t_out, goat_stream_t stream) {
    if (!f || !g || !t_out || n < 1 || !(eps > 0.0f)) return GOAT_ERR_INVALID_ARG;
    k_dual_targets<<<1, 1024, 0, (cudaStream_t)stream>>>(f, g, n, eps, t_out);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

int goat_mlp_forward(const void *weights_bf16, const float *x, int N, float *y, goat_stream_t stream) {
    if (!weights_bf16 || !x || !y || N < 1) return GOAT_ERR_INVALID_ARG;
    return mlp_forward((const __nv_bfloat16 *)weights_bf16, x, N, y, (cudaStream_t)stream);
}

int goat_mlp_train_step(float *master, float *adam_state, void *weights_bf16, const float *x, const float *t, int N,
                        float lr, int step, float *loss_out, float *grad_out, goat_stream_t stream) {
    if (!master || !adam_state || !weights_bf16 || !x || !t || N < 1 || step < 1 || !loss_out || !grad_out)
        return GOAT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(grad_out, 0, MLP_NP * sizeof(float), s);
    cudaMemsetAsync(loss_out, 0, sizeof(float), s);
    k_mlp_backward<<<(unsigned)ceil_div(N, TS), TS, 0, s>>>((const __nv_bfloat16 *)weights_bf16, x, t, N, grad_out,
                                                            loss_out);
    if (lr > 0.f)
        k_mlp_adam<<<1, 1024, 0, s>>>(master, adam_state, adam_state + MLP_NP, (__nv_bfloat16 *)weights_bf16,
                                      grad_out, lr, step);
    note_launches(lr > 0.f ? 2 : 1);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

}  // extern "C"
