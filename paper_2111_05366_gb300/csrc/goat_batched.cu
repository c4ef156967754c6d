// goat_batched.cu -- many independent GOAT solves (Alg. 3) advanced together:
// graph pairs of uneven n, each from several starting points (the paper's
// random restarts, Sec. 3.4), every Frank-Wolfe iteration of every problem
// being one replay of a captured CUDA graph.
//
// Problems q = pair * restarts + restart.  Per FW iteration the graph holds:
//   k_b_sinkhorn   one CTA per problem runs the whole LOT solve (Alg. 2) with its
//                  duals in shared memory; small problems also stage G there
//   k_b_write_q    Q -> BF16 rows of the stacked GEMM operand
//   gemm_grouped   C1 = B Q^T and G_Q = -2 A C1^T for all problems (tcgen05, one launch each)
//   k_b_step       line search (Alg. 3 step 3) and update (step 4), one CTA per problem
// Converged problems skip their CTA work.  Block sizes and shared-memory staging
// of the Sinkhorn kernel are chosen per n-bucket by a small autotuner that times
// the candidates on the batch itself the first time a bucket shape is seen.
// Then: the integer auction projection (as goat_lap.cu, one CTA per problem),
// the exact objective, and the best restart per pair.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

constexpr int BATCH_MAX_N = 2048;
constexpr float kLog2eB = 1.4426950408889634f;

struct ProbState {
    float eps, c, gmax, eps_rel;
    double alpha;
    int done, fw_iters, sk_iters, pad;
    float sk_resid, fw_tol;
    long long objective;
    int lap_flag, pad2;
};

struct BatchView {
    int num_pairs, restarts, ld;  // ld: row stride of the BF16 operand stacks
    const int *n;                 // per problem
    const long long *row_off;     // per problem: first row in the Q / C1 stacks
    const long long *mat_off;     // per problem: offset of its n x n FP32 matrices
    const long long *vec_off;     // per problem: offset of its n-vectors
    const long long *prow_off;    // per pair: first row in the A / B stacks
    const long long *adj_off;     // per pair: byte offset of its packed uint8 A / B
    const uint8_t *A, *B;         // packed input adjacency
    __nv_bfloat16 *A16, *B16, *Xq, *C1;
    float *G, *GQ, *P, *f, *g, *degA, *degB;
    ProbState *ps;
    int32_t *perm;                // per problem, packed like the vectors
};

// ---------------------------------------------------------------- counter-based noise

// SplitMix64 (Steele, Lea, Flood 2014) used counter-style: the k-th output of the
// generator seeded with `seed`, i.e. the mix of seed + (k + 1) * golden gamma.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uniform in (0, 1] with 24 random bits for entry (i, j) of problem q.
__device__ __forceinline__ float noise_u(uint64_t seed, int q, int i, int j, int n) {
    const uint64_t k = ((uint64_t)q << 32) | (uint64_t)((uint32_t)i * (uint32_t)n + (uint32_t)j);
    return (float)((splitmix64_at(seed, k) >> 40) + 1ull) * (1.0f / 16777216.0f);
}

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ float block_max(float v, float *red) {
    v = warp_max(v);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    float r = threadIdx.x < nw ? red[threadIdx.x] : 0.0f;
    if (w == 0) r = warp_max(r);
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    return red[0];
}

__device__ __forceinline__ double block_sum_d(double v, double *red) {
    v = warp_sum_d(v);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double r = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
    if (w == 0) r = warp_sum_d(r);
    if (threadIdx.x == 0) red[0] = r;
    __syncthreads();
    return red[0];
}

// ---------------------------------------------------------------- operands and init

// One block per pair: BF16 operand rows (zero padding to ld) and degrees.
__global__ void k_b_operands(BatchView V) {
    const int p = blockIdx.x;
    const int q0 = p * V.restarts;
    const int n = V.n[q0];
    const uint8_t *A = V.A + V.adj_off[p], *B = V.B + V.adj_off[p];
    __nv_bfloat16 *A16 = V.A16 + V.prow_off[p] * V.ld, *B16 = V.B16 + V.prow_off[p] * V.ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < n; i += nw) {
        float sa = 0.f, sb = 0.f;
        for (int j = lane; j < V.ld; j += 32) {
            const float a = j < n ? (float)A[(long long)i * n + j] : 0.f;
            const float b = j < n ? (float)B[(long long)i * n + j] : 0.f;
            A16[(long long)i * V.ld + j] = __float2bfloat16_rn(a);
            B16[(long long)i * V.ld + j] = __float2bfloat16_rn(b);
            sa += a;
            sb += b;
        }
        sa = warp_sum(sa);
        sb = warp_sum(sb);
        if (lane == 0) {
            V.degA[V.prow_off[p] + i] = sa;
            V.degB[V.prow_off[p] + i] = sb;
        }
    }
}

// Restart 0: P = J.  Restart r >= 1: the cost M = -ln U of the noise, whose
// Sinkhorn scaling with eps = 1 is K = Sinkhorn-Knopp(U); P is formed from it later.
__global__ void k_b_init(BatchView V, uint64_t seed, float eps_rel, float fw_tol) {
    const int q = blockIdx.x;
    const int n = V.n[q];
    const int r = q % V.restarts;
    float *P = V.P + V.mat_off[q], *G = V.G + V.mat_off[q];
    const float inv_n = 1.0f / (float)n;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        const int i = (int)(t / n), j = (int)(t - (long long)i * n);
        if (r == 0) {
            P[t] = inv_n;
        } else {
            G[t] = -logf(noise_u(seed, q, i, j, n));
        }
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) V.g[V.vec_off[q] + j] = 0.0f;
    if (threadIdx.x == 0) {
        ProbState s;
        memset(&s, 0, sizeof(s));
        s.eps_rel = eps_rel;
        s.fw_tol = fw_tol;
        s.eps = 1.0f;  // the noise scaling runs at eps = 1
        s.c = kLog2eB;
        s.gmax = 0.f;
        s.done = (r == 0) ? 1 : 0;  // only the random restarts run the noise scaling
        V.ps[q] = s;
    }
}

// P = (J + K)/2 with K = exp((f + g - M)) the scaled noise (restarts >= 1); all problems then
// become active.
__global__ void k_b_init_mix(BatchView V) {
    const int q = blockIdx.x;
    const int n = V.n[q];
    const int r = q % V.restarts;
    if (r != 0) {
        float *P = V.P + V.mat_off[q];
        const float *M = V.G + V.mat_off[q];
        const float *f = V.f + V.vec_off[q], *g = V.g + V.vec_off[q];
        const float inv_n = 1.0f / (float)n;
        for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
            const int i = (int)(t / n), j = (int)(t - (long long)i * n);
            P[t] = 0.5f * inv_n + 0.5f * exp2f((f[i] + g[j] - M[t]) * kLog2eB);
        }
    }
    __syncthreads();  // every thread has read g before any thread clears it
    for (int j = threadIdx.x; j < n; j += blockDim.x) V.g[V.vec_off[q] + j] = 0.0f;
    __syncthreads();
    if (threadIdx.x == 0) {
        V.ps[q].done = 0;
        V.ps[q].sk_iters = 0;
    }
}

// P (FP32) -> BF16 rows of the operand stack, for the initial gradient.
__global__ void k_b_p_to_operand(BatchView V) {
    const int q = blockIdx.x;
    const int n = V.n[q];
    const int w = (int)round_up(n, 64);
    const float *P = V.P + V.mat_off[q];
    __nv_bfloat16 *X = V.Xq + V.row_off[q] * V.ld;
    for (long long t = threadIdx.x; t < (long long)n * w; t += blockDim.x) {
        const int i = (int)(t / w), j = (int)(t - (long long)i * w);
        X[(long long)i * V.ld + j] = __float2bfloat16_rn(j < n ? P[(long long)i * n + j] : 0.0f);
    }
}

// Restart 0 keeps the exact closed-form gradient at the barycenter,
// G = -(2/n) d_A d_B^T; every problem records max|G|.
__global__ void k_b_init_gmax(BatchView V) {
    const int q = blockIdx.x;
    const int n = V.n[q];
    const int p = q / V.restarts, r = q % V.restarts;
    float *G = V.G + V.mat_off[q];
    const float *dA = V.degA + V.prow_off[p], *dB = V.degB + V.prow_off[p];
    __shared__ float red[32];
    float gm = 0.f;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        if (r == 0) {
            const int i = (int)(t / n), j = (int)(t - (long long)i * n);
            G[t] = -2.0f / (float)n * dA[i] * dB[j];
        }
        gm = fmaxf(gm, fabsf(G[t]));
    }
    gm = block_max(gm, red);
    if (threadIdx.x == 0) V.ps[q].gmax = gm;
}

// ---------------------------------------------------------------- Sinkhorn, one CTA per problem

// The whole LOT solve of each active problem (see goat_sinkhorn.cu for the
// iteration): row log-sum-exp by warps, column sums by threads, duals in shared
// memory, G from global memory or (STAGED) from shared memory.
template <bool STAGED>
__global__ void k_b_sinkhorn(BatchView V, const int *qlist, int nq, int sk_max_iter, float sk_tol, int warm,
                             int use_gmax) {
    extern __shared__ float sm[];
    __shared__ float red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int w = blockIdx.x; w < nq; w += gridDim.x) {
        const int q = qlist[w];
        if (V.ps[q].done) continue;
        const int n = V.n[q];
        const float *Gg = V.G + V.mat_off[q];
        float *fo = V.f + V.vec_off[q], *go = V.g + V.vec_off[q];
        float *f = sm, *g = sm + BATCH_MAX_N;
        float *Gs = sm + 2 * BATCH_MAX_N;
        const float *G = STAGED ? Gs : Gg;
        float eps = V.ps[q].eps;
        if (use_gmax) {
            eps = V.ps[q].eps_rel * V.ps[q].gmax;
            if (!(eps > 0.f)) eps = 1.0f;
        }
        const float c = kLog2eB / eps;
        for (int j = threadIdx.x; j < n; j += blockDim.x) g[j] = warm ? go[j] : 0.0f;
        if (STAGED)
            for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) Gs[t] = Gg[t];
        __syncthreads();
        int it = 0;
        float resid = INFINITY;
        while (it < sk_max_iter) {
            for (int i = warp; i < n; i += nw) {
                const float *Gi = G + (long long)i * n;
                float m = -INFINITY, s = 0.f;
                for (int j = lane; j < n; j += 32) {
                    const float x = (g[j] - Gi[j]) * c;
                    if (x > m) {
                        s = s * fast_exp2(m - x) + 1.0f;
                        m = x;
                    } else {
                        s += fast_exp2(x - m);
                    }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const float m2 = __shfl_xor_sync(0xffffffffu, m, o);
                    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
                    const float M = fmaxf(m, m2);
                    s = (M == -INFINITY) ? 0.f : s * fast_exp2(m - M) + s2 * fast_exp2(m2 - M);
                    m = M;
                }
                if (lane == 0) f[i] = -(m + __log2f(s)) / c;
            }
            __syncthreads();
            float r = 0.f;
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                double S = 0.0;
                const float gj = g[j];
                for (int i0 = 0; i0 < n; i0 += 16) {
                    float s16 = 0.f;
                    const int ie = min(n, i0 + 16);
                    for (int i = i0; i < ie; ++i) s16 += fast_exp2((f[i] + gj - G[(long long)i * n + j]) * c);
                    S += s16;
                }
                if (S > 1e-30 && S < 1e30) {
                    g[j] = gj - (float)log2(S) / c;
                    r = fmaxf(r, (float)fabs(S - 1.0));
                } else {
                    r = INFINITY;
                }
            }
            resid = block_max(r, red);
            ++it;
            if (!(resid < INFINITY) || resid < sk_tol) break;
        }
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            fo[j] = f[j];
            go[j] = g[j];
        }
        if (threadIdx.x == 0) {
            V.ps[q].sk_iters += it;
            V.ps[q].sk_resid = resid;
            V.ps[q].eps = eps;
            V.ps[q].c = c;
        }
        __syncthreads();
    }
}

// Q = 2^(c (f + g - G)) -> BF16 operand rows, zero up to the next multiple of 64.
__global__ void k_b_write_q(BatchView V) {
    const int q = blockIdx.x;
    if (V.ps[q].done) return;
    const int n = V.n[q];
    const int w = (int)round_up(n, 64);
    const float c = V.ps[q].c;
    const float *G = V.G + V.mat_off[q], *f = V.f + V.vec_off[q], *g = V.g + V.vec_off[q];
    __nv_bfloat16 *X = V.Xq + V.row_off[q] * V.ld;
    for (long long t = threadIdx.x; t < (long long)n * w; t += blockDim.x) {
        const int i = (int)(t / w), j = (int)(t - (long long)i * w);
        const float v = j < n ? fast_exp2((f[i] + g[j] - G[(long long)i * n + j]) * c) : 0.0f;
        X[(long long)i * V.ld + j] = __float2bfloat16_rn(v);
    }
}

// Line search (Alg. 3 step 3) and update (step 4) of one problem per CTA.  A
// problem that converges empties its GEMM descriptors so later products skip it.
__global__ void k_b_step(BatchView V, int max_iter, GemmGroupDesc *desc1, GemmGroupDesc *desc2) {
    const int q = blockIdx.x;
    if (V.ps[q].done) return;
    __shared__ double redd[32];
    __shared__ float red[32];
    const int n = V.n[q];
    float *G = V.G + V.mat_off[q], *P = V.P + V.mat_off[q];
    const float *GQ = V.GQ + V.mat_off[q];
    const __nv_bfloat16 *X = V.Xq + V.row_off[q] * V.ld;
    double s1 = 0, s2 = 0, s3 = 0;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        const int i = (int)(t / n), j = (int)(t - (long long)i * n);
        const float d = __bfloat162float(X[(long long)i * V.ld + j]) - P[t];
        s1 += (double)(G[t] * d);
        s2 += (double)(GQ[t] * d);
        s3 += (double)(d * d);
    }
    s1 = block_sum_d(s1, redd);
    s2 = block_sum_d(s2, redd);
    s3 = block_sum_d(s3, redd);
    const double b = -s1, a = 0.5 * (s1 - s2);
    double alpha;
    if (a < 0.0) {
        alpha = -b / (2.0 * a);
        alpha = alpha < 0.0 ? 0.0 : (alpha > 1.0 ? 1.0 : alpha);
    } else {
        alpha = (a + b > 0.0) ? 1.0 : 0.0;
    }
    if (!(alpha == alpha)) alpha = 0.0;
    const float al = (float)alpha;
    float gm = 0.f;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        const int i = (int)(t / n), j = (int)(t - (long long)i * n);
        const float qv = __bfloat162float(X[(long long)i * V.ld + j]);
        P[t] = fmaf(al, qv - P[t], P[t]);
        const float gn = fmaf(al, GQ[t] - G[t], G[t]);
        G[t] = gn;
        gm = fmaxf(gm, fabsf(gn));
    }
    gm = block_max(gm, red);
    if (threadIdx.x == 0) {
        ProbState &s = V.ps[q];
        s.gmax = gm;
        s.alpha = alpha;
        s.fw_iters += 1;
        const double change = alpha * sqrt(s3 > 0 ? s3 : 0.0) / sqrt((double)n);
        if (change < (double)s.fw_tol || s.fw_iters >= max_iter) {
            s.done = 1;
            desc1[q].num_kb = 0;
            desc1[q].M = 0;
            desc2[q].num_kb = 0;
            desc2[q].M = 0;
        }
    }
}

__global__ void k_b_reset_duals(BatchView V) {
    const int q = blockIdx.x;
    const int n = V.n[q];
    for (int j = threadIdx.x; j < n; j += blockDim.x) V.g[V.vec_off[q] + j] = 0.0f;
    if (threadIdx.x == 0) {
        V.ps[q].sk_iters = 0;
        V.ps[q].done = 0;
        V.ps[q].fw_iters = 0;
    }
}

__global__ void k_b_count_active(BatchView V, int nq, int *out) {
    int c = 0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) c += !V.ps[q].done;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Best restart of each pair: largest objective, lowest restart on ties (Sec. 3.4).
__global__ void k_b_best(BatchView V, int *best_q) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= V.num_pairs) return;
    int bq = p * V.restarts;
    for (int r = 1; r < V.restarts; ++r) {
        const int q = p * V.restarts + r;
        if (V.ps[q].objective > V.ps[bq].objective) bq = q;
    }
    best_q[p] = bq;
}

// ---------------------------------------------------------------- projection: integer auction per CTA

typedef long long i64b;

__device__ __forceinline__ i64b qbenefit(float m, float mul, i64b qm) { return __float2ll_rn(m * mul) * qm; }

// Exact eps-scaling auction on one problem per CTA (quantised as in goat_lap.cu):
// Gauss-Seidel bids, prices / owners / queue in shared memory.
__global__ void __launch_bounds__(512) k_b_lap(BatchView V, long long budget_per_phase) {
    const int q = blockIdx.x;
    const int n = V.n[q];
    const float *M = V.P + V.mat_off[q];
    int32_t *perm = V.perm + V.vec_off[q];
    extern __shared__ unsigned char smraw[];
    i64b *price = reinterpret_cast<i64b *>(smraw);
    int *owner = reinterpret_cast<int *>(price + BATCH_MAX_N);
    int *assign = owner + BATCH_MAX_N;
    int *queue = assign + BATCH_MAX_N;
    __shared__ i64b s_b1[16], s_b2[16];
    __shared__ int s_j1[16];
    __shared__ float red[32];
    __shared__ int s_head, s_tail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

    float cm = 0.f;
    for (long long t = tid; t < (long long)n * n; t += blockDim.x) cm = fmaxf(cm, fabsf(M[t]));
    cm = block_max(cm, red);
    int e = 0;
    if (cm > 0.f) frexpf(cm, &e);
    int qbits = 1;
    while ((1 << qbits) <= n) ++qbits;
    const float mul = ldexpf(1.0f, 40 - e);
    const i64b qm = 1LL << qbits;
    const i64b c_int = (1LL << 40) * qm;
    for (int j = tid; j < n; j += blockDim.x) price[j] = 0;
    i64b eps = c_int / 4;
    bool exhausted = false;
    for (;;) {
        const bool last = eps <= 1;
        for (int j = tid; j < n; j += blockDim.x) {
            owner[j] = -1;
            assign[j] = -1;
            queue[j] = j;
        }
        if (tid == 0) {
            s_head = 0;
            s_tail = n;
        }
        __syncthreads();
        long long bids = 0;
        const long long budget = last ? 16 * budget_per_phase : budget_per_phase;
        while (s_head != s_tail && bids < budget) {
            const int i = queue[s_head % n];
            const float *Mi = M + (long long)i * n;
            i64b b1 = LLONG_MIN / 4, b2 = LLONG_MIN / 4;
            int j1 = INT_MAX;
            for (int j = tid; j < n; j += blockDim.x) {
                const i64b v = qbenefit(Mi[j], mul, qm) - price[j];
                if (v > b1) {
                    b2 = b1;
                    b1 = v;
                    j1 = j;
                } else if (v > b2) {
                    b2 = v;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const i64b o1 = __shfl_xor_sync(0xffffffffu, b1, o);
                const i64b o2 = __shfl_xor_sync(0xffffffffu, b2, o);
                const int oj = __shfl_xor_sync(0xffffffffu, j1, o);
                if (o1 > b1 || (o1 == b1 && oj < j1)) {
                    b2 = max(b1, o2);
                    b1 = o1;
                    j1 = oj;
                } else {
                    b2 = max(b2, o1);
                }
            }
            if (lane == 0) {
                s_b1[warp] = b1;
                s_b2[warp] = b2;
                s_j1[warp] = j1;
            }
            __syncthreads();
            if (tid == 0) {
                for (int w2 = 1; w2 < nw; ++w2) {
                    const i64b o1 = s_b1[w2], o2 = s_b2[w2];
                    const int oj = s_j1[w2];
                    if (o1 > b1 || (o1 == b1 && oj < j1)) {
                        b2 = max(b1, o2);
                        b1 = o1;
                        j1 = oj;
                    } else {
                        b2 = max(b2, o1);
                    }
                }
                const i64b inc = (b2 == LLONG_MIN / 4) ? eps : (b1 - b2) + eps;
                price[j1] += inc;
                const int old = owner[j1];
                owner[j1] = i;
                assign[i] = j1;
                ++s_head;
                if (old >= 0) {
                    assign[old] = -1;
                    queue[s_tail % n] = old;
                    ++s_tail;
                }
            }
            ++bids;
            __syncthreads();
        }
        if (last) {
            exhausted = (s_head != s_tail);
            break;
        }
        eps = max(1LL, eps / 8);
    }
    // any row left unassigned (budget exhausted) takes the first free object
    if (tid == 0 && exhausted) {
        int jf = 0;
        for (int i = 0; i < n; ++i)
            if (assign[i] < 0) {
                while (jf < n && owner[jf] >= 0) ++jf;
                if (jf < n) {
                    owner[jf] = i;
                    assign[i] = jf;
                }
            }
        V.ps[q].lap_flag = 1;
    }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) perm[i] = assign[i];
}

// f(perm) = sum_ij A_ij B[perm i][perm j] for each problem (exact, 0/1 inputs).
__global__ void k_b_objective(BatchView V) {
    const int q = blockIdx.x;
    const int p = q / V.restarts;
    const int n = V.n[q];
    const uint8_t *A = V.A + V.adj_off[p], *B = V.B + V.adj_off[p];
    const int32_t *perm = V.perm + V.vec_off[q];
    long long acc = 0;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        const int i = (int)(t / n), j = (int)(t - (long long)i * n);
        if (A[t]) {
            const int pi = perm[i], pj = perm[j];
            if (pi >= 0 && pi < n && pj >= 0 && pj < n) acc += (long long)A[t] * B[(long long)pi * n + pj];
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ long long r[32];
    if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += r[w];
        V.ps[q].objective = s;
    }
}

// ---------------------------------------------------------------- autotuner

// Candidate launch shapes of the batched Sinkhorn kernel.
struct SkShape {
    int threads;
    bool staged;
};

static const SkShape kSkShapes[] = {{128, false}, {256, false}, {512, false}, {256, true}, {512, true}};

static size_t sk_smem(const SkShape &s, int nmax) {
    size_t b = 2 * BATCH_MAX_N * sizeof(float);
    if (s.staged) b += (size_t)nmax * nmax * sizeof(float);
    return b;
}

static bool sk_shape_fits(const SkShape &s, int nmax) { return sk_smem(s, nmax) <= 200 * 1024; }

static void launch_sk(const SkShape &s, const BatchView &V, const int *qlist, int nq, int nmax, int iters, float tol,
                      int warm, int use_gmax, int grid, cudaStream_t st) {
    const size_t sm = sk_smem(s, nmax);
    if (s.staged)
        k_b_sinkhorn<true><<<grid, s.threads, sm, st>>>(V, qlist, nq, iters, tol, warm, use_gmax);
    else
        k_b_sinkhorn<false><<<grid, s.threads, sm, st>>>(V, qlist, nq, iters, tol, warm, use_gmax);
    note_launches(1);
}

static int bucket_of(int n) {
    int b = 0;
    while ((64 << b) < n) ++b;
    return b;  // <= 64, <= 128, ..., <= 2048
}

// Best shape per n-bucket, keyed by (bucket, problems in bucket); timed on the batch.
static std::map<std::pair<int, int>, int> g_tuned;
static std::mutex g_tuned_mu;

}  // namespace goat

using namespace goat;

extern "C" {

size_t goat_workspace_bytes_batched(const int *n, int num_pairs, int restarts) {
    if (!n || num_pairs < 1 || restarts < 1) return 0;
    size_t rows_p = 0, rows_q = 0, mats = 0, nmax = 0, tiles = 0;
    for (int p = 0; p < num_pairs; ++p) {
        if (n[p] < 1 || n[p] > BATCH_MAX_N) return 0;
        rows_p += n[p];
        rows_q += (size_t)n[p] * restarts;
        mats += (size_t)n[p] * n[p] * restarts;
        nmax = std::max<size_t>(nmax, n[p]);
        tiles += (size_t)ceil_div(n[p], 128) * ceil_div(n[p], 256) * restarts;
    }
    const size_t ld = round_up((int64_t)nmax, 64);
    const size_t nq = (size_t)num_pairs * restarts;
    size_t b = 0;
    auto add = [&](size_t x) { b += round_up((int64_t)x, 256); };
    add(2 * rows_p * ld * 2);      // A16, B16
    add(2 * rows_q * ld * 2);      // Xq, C1
    add(3 * mats * 4);             // G, GQ, P
    add(3 * rows_q * 4);           // f, g, perm
    add(2 * rows_p * 4);           // degrees
    add(nq * sizeof(ProbState));
    add(nq * 4 * sizeof(long long) + num_pairs * 2 * sizeof(long long));  // offsets
    add(nq * sizeof(int) * 2);     // n per problem, problem list
    add(2 * nq * sizeof(GemmGroupDesc));
    add(tiles * sizeof(int4));
    add(64);
    return b + 64 * 256;
}

int goat_match_batched(const void *A, const void *B, const long long *adj_off, const int *n, int num_pairs,
                       int restarts, unsigned long long seed, float eps_rel, int max_iter, float tol,
                       const goat_params *params, int32_t *perm_out, double *objective_out, int *best_restart,
                       int *fw_iters_out, float *relaxed_out, void *workspace, size_t workspace_bytes,
                       goat_stream_t stream) {
    if (!A || !B || !adj_off || !n || num_pairs < 1 || restarts < 1 || !perm_out || max_iter < 0 ||
        !(eps_rel > 0.f) || !(tol >= 0.f))
        return GOAT_ERR_INVALID_ARG;
    for (int p = 0; p < num_pairs; ++p)
        if (n[p] < 1 || n[p] > BATCH_MAX_N) return GOAT_ERR_INVALID_ARG;
    goat_params prm;
    goat_default_params(&prm);
    if (params) prm = *params;
    if (prm.direction != GOAT_DIR_LOT) return GOAT_ERR_INVALID_ARG;  // the batched path runs GOAT only
    if (prm.sk_max_iter <= 0) prm.sk_max_iter = 500;
    if (!(prm.sk_tol > 0.f)) prm.sk_tol = 1e-3f;
    int dev = 0, major = 0, minor = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (major != 10 || minor != 3) return GOAT_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;

    // ---------------- host-side layout
    const int nq = num_pairs * restarts;
    std::vector<int> nv(nq);
    std::vector<long long> row_off(nq), mat_off(nq), vec_off(nq), prow_off(num_pairs);
    long long rp = 0, rq = 0, mo = 0;
    int nmax = 1;
    for (int p = 0; p < num_pairs; ++p) {
        prow_off[p] = rp;
        rp += n[p];
        nmax = std::max(nmax, n[p]);
        for (int r = 0; r < restarts; ++r) {
            const int q = p * restarts + r;
            nv[q] = n[p];
            row_off[q] = rq;
            vec_off[q] = rq;
            rq += n[p];
            mat_off[q] = mo;
            mo += (long long)n[p] * n[p];
        }
    }
    const int ld = (int)round_up(nmax, 64);
    std::vector<int4> items;
    for (int q = 0; q < nq; ++q)
        for (int tm = 0; tm < (int)ceil_div(nv[q], 128); ++tm)
            for (int tn = 0; tn < (int)ceil_div(nv[q], 256); ++tn) items.push_back(make_int4(q, tm, tn, 0));

    const size_t need = goat_workspace_bytes_batched(n, num_pairs, restarts);
    uint8_t *base = (uint8_t *)workspace;
    bool owned = false;
    if (base) {
        if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(base) & 255)) return GOAT_ERR_OUT_OF_MEMORY;
    } else {
        if (cudaMallocAsync((void **)&base, need, s) != cudaSuccess) {
            cudaGetLastError();
            return GOAT_ERR_OUT_OF_MEMORY;
        }
        owned = true;
    }
    struct Free {
        uint8_t *p;
        bool own;
        cudaStream_t s;
        ~Free() {
            if (own) cudaFreeAsync(p, s);
        }
    } fr{base, owned, s};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        uint8_t *r = base + off;
        off += round_up((int64_t)std::max<size_t>(bytes, 1), 256);
        return (void *)r;
    };
    BatchView V;
    std::memset(&V, 0, sizeof(V));
    V.num_pairs = num_pairs;
    V.restarts = restarts;
    V.ld = ld;
    V.A16 = (__nv_bfloat16 *)take((size_t)rp * ld * 2);
    V.B16 = (__nv_bfloat16 *)take((size_t)rp * ld * 2);
    V.Xq = (__nv_bfloat16 *)take((size_t)rq * ld * 2);
    V.C1 = (__nv_bfloat16 *)take((size_t)rq * ld * 2);
    V.G = (float *)take((size_t)mo * 4);
    V.GQ = (float *)take((size_t)mo * 4);
    V.P = (float *)take((size_t)mo * 4);
    V.f = (float *)take((size_t)rq * 4);
    V.g = (float *)take((size_t)rq * 4);
    V.perm = (int32_t *)take((size_t)rq * 4);
    V.degA = (float *)take((size_t)rp * 4);
    V.degB = (float *)take((size_t)rp * 4);
    V.ps = (ProbState *)take((size_t)nq * sizeof(ProbState));
    long long *d_row = (long long *)take((size_t)nq * 8), *d_mat = (long long *)take((size_t)nq * 8);
    long long *d_vec = (long long *)take((size_t)nq * 8), *d_prow = (long long *)take((size_t)num_pairs * 8);
    long long *d_adj = (long long *)take((size_t)num_pairs * 8);
    int *d_n = (int *)take((size_t)nq * 4);
    int *d_qlist = (int *)take((size_t)nq * 4);
    GemmGroupDesc *d_desc1 = (GemmGroupDesc *)take((size_t)nq * sizeof(GemmGroupDesc));
    GemmGroupDesc *d_desc2 = (GemmGroupDesc *)take((size_t)nq * sizeof(GemmGroupDesc));
    int4 *d_items = (int4 *)take(items.size() * sizeof(int4));
    int *d_err = (int *)take(64);
    V.n = d_n;
    V.row_off = d_row;
    V.mat_off = d_mat;
    V.vec_off = d_vec;
    V.prow_off = d_prow;
    V.adj_off = d_adj;
    V.A = (const uint8_t *)A;
    V.B = (const uint8_t *)B;

    std::vector<GemmGroupDesc> desc1(nq), desc2(nq);
    for (int q = 0; q < nq; ++q) {
        const int p = q / restarts;
        GemmGroupDesc d;
        std::memset(&d, 0, sizeof(d));
        d.x_row0 = prow_off[p];
        d.y_row0 = row_off[q];
        d.num_kb = (int)ceil_div(nv[q], 64);
        d.M = nv[q];
        d.N = nv[q];
        d.out_cols = (int)round_up(nv[q], 64);
        d.out_b16 = V.C1 + row_off[q] * ld;
        d.row_stride = ld;
        desc1[q] = d;
        d.out_cols = nv[q];
        d.out_b16 = nullptr;
        d.out_f32 = V.GQ + mat_off[q];
        d.ld_out = nv[q];
        desc2[q] = d;
    }
    std::vector<int> qlist(nq);
    for (int q = 0; q < nq; ++q) qlist[q] = q;
    // problems sorted by size, larger first (better tail balance of the per-problem kernels)
    std::stable_sort(qlist.begin(), qlist.end(), [&](int a, int b) { return nv[a] > nv[b]; });
    cudaMemcpyAsync(d_row, row_off.data(), nq * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_mat, mat_off.data(), nq * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_vec, vec_off.data(), nq * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_prow, prow_off.data(), num_pairs * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_adj, adj_off, num_pairs * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_n, nv.data(), nq * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_qlist, qlist.data(), nq * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_desc1, desc1.data(), nq * sizeof(GemmGroupDesc), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_desc2, desc2.data(), nq * sizeof(GemmGroupDesc), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(d_err, 0, 64, s);
    cudaMemsetAsync(V.Xq, 0, (size_t)rq * ld * 2, s);
    cudaMemsetAsync(V.C1, 0, (size_t)rq * ld * 2, s);

    GemmGroupCall g1;
    std::memset(&g1, 0, sizeof(g1));
    g1.X = V.B16;
    g1.x_rows = rp;
    g1.x_stride = ld;
    g1.Y = V.Xq;
    g1.y_rows = rq;
    g1.y_stride = ld;
    g1.k_extent = ld;
    g1.items = d_items;
    g1.num_items = (int)items.size();
    g1.descs = d_desc1;
    g1.scale = 1.0f;
    g1.mode = GEMM_OUT_BF16_TERMS;
    g1.err = d_err;
    GemmGroupCall g2 = g1;
    g2.X = V.A16;
    g2.Y = V.C1;
    g2.descs = d_desc2;
    g2.scale = -2.0f;
    g2.mode = GEMM_OUT_F32;

    const int grid_prob = std::min(nq, sms * 8);
    // ---------------- operands and starting points
    k_b_operands<<<num_pairs, 256, 0, s>>>(V);
    k_b_init<<<nq, 256, 0, s>>>(V, seed, eps_rel, tol);
    note_launches(2);
    SkShape init_shape{512, false};
    if (restarts > 1) {
        // K = Sinkhorn-Knopp(U) of the random restarts (eps = 1 on M = -ln U)
        launch_sk(init_shape, V, d_qlist, nq, nmax, 2000, 1e-6f, 0, 0, grid_prob, s);
    }
    k_b_init_mix<<<nq, 256, 0, s>>>(V);
    k_b_p_to_operand<<<nq, 256, 0, s>>>(V);
    note_launches(2);
    int st = gemm_grouped(g1, s);
    if (st) return st;
    st = gemm_grouped(g2, s);
    if (st) return st;
    // the initial gradient lands in GQ: move it to G (restart 0 then gets the closed form)
    cudaMemcpyAsync(V.G, V.GQ, (size_t)mo * 4, cudaMemcpyDeviceToDevice, s);
    k_b_init_gmax<<<nq, 256, 0, s>>>(V);
    note_launches(1);

    // ---------------- autotune the Sinkhorn launch shape for this batch's largest bucket
    const int bkt = bucket_of(nmax);
    SkShape best = {256, false};
    {
        std::lock_guard<std::mutex> lock(g_tuned_mu);
        auto key = std::make_pair(bkt, nq);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            best = kSkShapes[it->second];
        } else {
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            float best_ms = 1e30f;
            int best_k = 1;
            // time 5 Sinkhorn iterations per candidate on the real costs (g restarts from 0; results discarded)
            for (int k = 0; k < (int)(sizeof(kSkShapes) / sizeof(kSkShapes[0])); ++k) {
                if (!sk_shape_fits(kSkShapes[k], nmax)) continue;
                if (kSkShapes[k].staged && cudaFuncSetAttribute(k_b_sinkhorn<true>,
                                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                (int)sk_smem(kSkShapes[k], nmax)) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                cudaEventRecord(e0, s);
                launch_sk(kSkShapes[k], V, d_qlist, nq, nmax, 5, 0.0f, 0, 1, grid_prob, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) {
                    best_ms = ms;
                    best_k = k;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            g_tuned[key] = best_k;
            best = kSkShapes[best_k];
        }
    }
    if (best.staged)
        cudaFuncSetAttribute(k_b_sinkhorn<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sk_smem(best, nmax));
    // the tuning runs touched g, eps and the Sinkhorn counters: reset before the real loop
    k_b_reset_duals<<<nq, 256, 0, s>>>(V);
    note_launches(1);

    // ---------------- one FW iteration of every problem, captured once as a CUDA graph
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return GOAT_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    struct GraphGuard {
        cudaStream_t c;
        cudaGraph_t *g;
        cudaGraphExec_t *e;
        ~GraphGuard() {
            if (*e) cudaGraphExecDestroy(*e);
            if (*g) cudaGraphDestroy(*g);
            if (c) cudaStreamDestroy(c);
        }
    } gg{cap, &graph, &exec};
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GOAT_ERR_CUDA;
    launch_sk(best, V, d_qlist, nq, nmax, prm.sk_max_iter, prm.sk_tol, prm.sk_warm_start, 1, grid_prob, cap);
    k_b_write_q<<<nq, 256, 0, cap>>>(V);
    note_launches(1);
    int cst = gemm_grouped(g1, cap);
    if (!cst) cst = gemm_grouped(g2, cap);
    k_b_step<<<nq, 256, 0, cap>>>(V, max_iter, d_desc1, d_desc2);
    note_launches(1);
    if (cudaStreamEndCapture(cap, &graph) != cudaSuccess || cst) {
        cudaGetLastError();
        return cst ? cst : GOAT_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) return GOAT_ERR_CUDA;

    int *d_active = d_err + 4;
    int h_active = 1;
    for (int it = 0; it < max_iter; ++it) {
        if (cudaGraphLaunch(exec, s) != cudaSuccess) return GOAT_ERR_CUDA;
        if (it % 5 == 4 || it == max_iter - 1) {
            cudaMemsetAsync(d_active, 0, sizeof(int), s);
            k_b_count_active<<<std::max(1, std::min(nq / 256 + 1, sms)), 256, 0, s>>>(V, nq, d_active);
            note_launches(1);
            cudaMemcpyAsync(&h_active, d_active, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) return GOAT_ERR_CUDA;
            if (h_active == 0) break;
        }
    }

    if (relaxed_out)
        cudaMemcpyAsync(relaxed_out, V.P, (size_t)mo * sizeof(float), cudaMemcpyDeviceToDevice, s);

    // ---------------- projection, objective, best restart
    const size_t lap_smem = (size_t)BATCH_MAX_N * (8 + 4 + 4 + 4);
    cudaFuncSetAttribute(k_b_lap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lap_smem);
    k_b_lap<<<nq, 512, lap_smem, s>>>(V, 64LL * nmax + 65536);
    k_b_objective<<<nq, 256, 0, s>>>(V);
    int *d_best = d_qlist;  // the problem list is no longer needed
    k_b_best<<<(unsigned)ceil_div(num_pairs, 128), 128, 0, s>>>(V, d_best);
    note_launches(3);
    std::vector<int> h_best(num_pairs);
    std::vector<ProbState> h_ps(nq);
    std::vector<int32_t> h_perm(rq);
    cudaMemcpyAsync(h_best.data(), d_best, num_pairs * 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h_ps.data(), V.ps, nq * sizeof(ProbState), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(h_perm.data(), V.perm, rq * 4, cudaMemcpyDeviceToHost, s);
    int h_err[2] = {0, 0};
    cudaMemcpyAsync(h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return GOAT_ERR_CUDA;
    if (h_err[0]) return h_err[0];
    long long out_off = 0;
    for (int p = 0; p < num_pairs; ++p) {
        const int q = h_best[p];
        std::memcpy(perm_out + out_off, h_perm.data() + vec_off[q], (size_t)n[p] * 4);
        out_off += n[p];
        if (objective_out) objective_out[p] = (double)h_ps[q].objective;
        if (best_restart) best_restart[p] = q - p * restarts;
        if (fw_iters_out) fw_iters_out[p] = h_ps[q].fw_iters;
    }
    return GOAT_OK;
}

}  // extern "C"
