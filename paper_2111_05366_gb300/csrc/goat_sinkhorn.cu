// goat_sinkhorn.cu -- K2: LOT (Alg. 2) as log-domain Sinkhorn on exp(-G/eps),
// with K = exp(-G/eps) never stored.
//
// Cuturi's Sinkhorn-Knopp scaling to the marginals 1_n (Sec. 3.3), written on
// the duals: Q_ij = exp((f_i + g_j - G_ij)/eps).  One iteration:
//   row scaling      f_i = -eps LSE_j((g_j - G_ij)/eps)                    (k_sk_row)
//   column sums      S_j = sum_i exp((f_i + g_j - G_ij)/eps)               (k_sk_colpart + k_sk_colfinal)
//   residual         max_j |S_j - 1|   (the column marginal error of the row-scaled Q)
//   column scaling   g_j <- g_j - eps log S_j
// The kernels work in base 2: with c = log2(e)/eps, exp((x)/eps) = 2^(c x).
// After the row scaling every Q_ij <= 1, so the column sums need no max shift;
// a column whose sum underflows (possible only far from convergence) is redone
// with a max-stabilised log-sum-exp.  All kernels return at once when the
// device-side stop flag is set, so the host can queue iterations ahead.
#include <algorithm>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

constexpr float kLog2e = 1.4426950408889634f;

// ---------------------------------------------------------------- row scaling

__device__ __forceinline__ void lse_push(float &m, float &s, float x) {
    if (x > m) {
        s = s * fast_exp2(m - x) + 1.0f;
        m = x;
    } else {
        s += fast_exp2(x - m);
    }
}

__device__ __forceinline__ void lse_merge(float &m, float &s, float m2, float s2) {
    const float M = fmaxf(m, m2);
    if (M == -INFINITY) {
        m = M;
        s = 0.0f;
        return;
    }
    s = s * fast_exp2(m - M) + s2 * fast_exp2(m2 - M);
    m = M;
}

// One warp per row.  Vector path (float4) when rows are 16-byte aligned.
__global__ void __launch_bounds__(256) k_sk_row(const float *__restrict__ G, int n, long long ld,
                                                const float *__restrict__ g, float *__restrict__ f,
                                                const DevState *__restrict__ st) {
    if (st->sk_done) return;
    const float c = st->c;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(G) & 15) == 0);
    const int n4 = vec ? (n & ~3) : 0;
    for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < n; row += gridDim.x * wpb) {
        const float *Gi = G + (long long)row * ld;
        float m = -INFINITY, s = 0.0f;
        int j = lane * 4;
        if (j + 128 < n4) {
            // the next step's G loads are issued before this step's arithmetic
            float4 a0 = __ldg(reinterpret_cast<const float4 *>(Gi + j));
            float4 a1 = __ldg(reinterpret_cast<const float4 *>(Gi + j + 128));
            for (;;) {
                const int jn = j + 256;
                const bool more = jn + 128 < n4;
                float4 na0, na1;
                const float4 b0 = __ldg(reinterpret_cast<const float4 *>(g + j));
                const float4 b1 = __ldg(reinterpret_cast<const float4 *>(g + j + 128));
                if (more) {
                    na0 = __ldg(reinterpret_cast<const float4 *>(Gi + jn));
                    na1 = __ldg(reinterpret_cast<const float4 *>(Gi + jn + 128));
                }
                const float x0 = (b0.x - a0.x) * c, x1 = (b0.y - a0.y) * c, x2 = (b0.z - a0.z) * c,
                            x3 = (b0.w - a0.w) * c;
                const float x4 = (b1.x - a1.x) * c, x5 = (b1.y - a1.y) * c, x6 = (b1.z - a1.z) * c,
                            x7 = (b1.w - a1.w) * c;
                const float mx = fmaxf(fmaxf(fmaxf(x0, x1), fmaxf(x2, x3)), fmaxf(fmaxf(x4, x5), fmaxf(x6, x7)));
                if (mx > m) {
                    s *= fast_exp2(m - mx);
                    m = mx;
                }
                s += fast_exp2(x0 - m) + fast_exp2(x1 - m) + fast_exp2(x2 - m) + fast_exp2(x3 - m) +
                     fast_exp2(x4 - m) + fast_exp2(x5 - m) + fast_exp2(x6 - m) + fast_exp2(x7 - m);
                j = jn;
                if (!more) break;
                a0 = na0;
                a1 = na1;
            }
        }
        for (; j < n4; j += 128) {
            const float4 a0 = __ldg(reinterpret_cast<const float4 *>(Gi + j));
            const float4 b0 = __ldg(reinterpret_cast<const float4 *>(g + j));
            lse_push(m, s, (b0.x - a0.x) * c);
            lse_push(m, s, (b0.y - a0.y) * c);
            lse_push(m, s, (b0.z - a0.z) * c);
            lse_push(m, s, (b0.w - a0.w) * c);
        }
        for (int jj = n4 + lane; jj < n; jj += 32) lse_push(m, s, (__ldg(g + jj) - __ldg(Gi + jj)) * c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float m2 = __shfl_xor_sync(0xffffffffu, m, o);
            const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
            lse_merge(m, s, m2, s2);
        }
        if (lane == 0) f[row] = -(m + __log2f(s)) / c;
    }
}

// ---------------------------------------------------------------- column sums

// Partial column sums over a chunk of rows.  A CTA owns 2048 adjacent columns:
// each lane owns two groups of 4 columns 128 columns apart, so a warp reads two
// contiguous 512-byte runs (1 KB) of every row and keeps 2 rows x 2 float4 loads
// in flight.  Every column is summed the same way whatever the launch shape:
// FP32 over groups of 16 rows (from the chunk's first row), the groups in FP64.
// EDGE = false is launched only on CTAs whose 2048 columns all lie inside the
// matrix with G 16-byte aligned, and carries no other path (the fallback code
// alone, even at the same register count, cost 10 % of the pass).  EDGE = true
// covers the rest: a group of 4 columns cut by the matrix edge, or any group
// of a G that is not 16-byte aligned, takes the scalar path (FP64 per term).
constexpr int kSkColsPerCta = 2048;

__device__ __forceinline__ void colpart_group(const float *__restrict__ G, int n, long long ld,
                                              const float *__restrict__ f, const float *__restrict__ g, float c,
                                              int j0, int r0, int r1, bool aligned, double *__restrict__ dst) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    float gj[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) gj[k] = (j0 + k < n) ? __ldg(g + j0 + k) : 0.0f;
    if (aligned && j0 + 3 < n) {
        int i = r0;
        while (i < r1) {
            const int ie = min(r1, i + 16);
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            for (; i < ie; ++i) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(G + (long long)i * ld + j0));
                const float fi = __ldg(f + i);
                s0 += fast_exp2((fi + gj[0] - a.x) * c);
                s1 += fast_exp2((fi + gj[1] - a.y) * c);
                s2 += fast_exp2((fi + gj[2] - a.z) * c);
                s3 += fast_exp2((fi + gj[3] - a.w) * c);
            }
            acc[0] += s0;
            acc[1] += s1;
            acc[2] += s2;
            acc[3] += s3;
        }
    } else {
        for (int i = r0; i < r1; ++i) {
            const float fi = __ldg(f + i);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (j0 + k < n) acc[k] += fast_exp2((fi + gj[k] - __ldg(G + (long long)i * ld + j0 + k)) * c);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (j0 + k < n) dst[j0 + k] = acc[k];
}

template <bool EDGE>
__global__ void __launch_bounds__(256) k_sk_colpart(const float *__restrict__ G, int n, long long ld,
                                                    const float *__restrict__ f, const float *__restrict__ g,
                                                    double *__restrict__ partial, int rows_per_chunk, int col0,
                                                    const DevState *__restrict__ st) {
    if (st->sk_done) return;
    const float c = st->c;
    const int ja = col0 + blockIdx.x * kSkColsPerCta + (threadIdx.x >> 5) * 256 + (threadIdx.x & 31) * 4;
    const int jb = ja + 128;
    const int r0 = blockIdx.y * rows_per_chunk;
    const int r1 = min(n, r0 + rows_per_chunk);
    double *dst = partial + (long long)blockIdx.y * n;
    if (EDGE) {
        if (ja >= n) return;
        const bool aligned = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(G) & 15) == 0);
        if (!(aligned && jb + 3 < n)) {
            colpart_group(G, n, ld, f, g, c, ja, r0, r1, aligned, dst);
            if (jb < n) colpart_group(G, n, ld, f, g, c, jb, r0, r1, aligned, dst);
            return;
        }
    }
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    float gj[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        gj[k] = __ldg(g + ja + k);
        gj[4 + k] = __ldg(g + jb + k);
    }
    int i = r0;
    while (i < r1) {
        const int ie = min(r1, i + 16);
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
        for (; i < ie; ++i) {
            const float *Gi = G + (long long)i * ld;
            const float4 a = __ldg(reinterpret_cast<const float4 *>(Gi + ja));
            const float4 b = __ldg(reinterpret_cast<const float4 *>(Gi + jb));
            const float fi = __ldg(f + i);
            s[0] += fast_exp2((fi + gj[0] - a.x) * c);
            s[1] += fast_exp2((fi + gj[1] - a.y) * c);
            s[2] += fast_exp2((fi + gj[2] - a.z) * c);
            s[3] += fast_exp2((fi + gj[3] - a.w) * c);
            s[4] += fast_exp2((fi + gj[4] - b.x) * c);
            s[5] += fast_exp2((fi + gj[5] - b.y) * c);
            s[6] += fast_exp2((fi + gj[6] - b.z) * c);
            s[7] += fast_exp2((fi + gj[7] - b.w) * c);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += s[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        dst[ja + k] = acc[k];
        dst[jb + k] = acc[4 + k];
    }
}

// Combines the chunk partials, takes the residual and applies the column scaling.
__global__ void __launch_bounds__(256) k_sk_colfinal(const double *__restrict__ partial, int nchunks, int n,
                                                     const float *__restrict__ G, long long ld,
                                                     const float *__restrict__ f, float *__restrict__ g,
                                                     DevState *__restrict__ st) {
    if (st->sk_done) return;
    const float c = st->c;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    float r = 0.0f;
    if (j < n) {
        double S = 0.0;
        for (int k = 0; k < nchunks; ++k) S += partial[(long long)k * n + j];
        const float gj = g[j];
        if (S > 1e-30 && S < 1e30) {
            g[j] = gj - (float)(log2(S)) / c;
            r = (float)fabs(S - 1.0);
        } else {
            // stabilised: g_j = -eps LSE_i((f_i - G_ij)/eps), S_j = 2^(c g_j_old) * sum
            float m = -INFINITY, s = 0.0f;
            for (int i = 0; i < n; ++i) lse_push(m, s, (f[i] - G[(long long)i * ld + j]) * c);
            const double lS = (double)gj * c + m + log2((double)s);
            g[j] = -(m + __log2f(s)) / c;
            r = (float)fabs(exp2(lS) - 1.0);
            if (!(r == r)) r = INFINITY;
            atomicAdd(&st->sk_underflow, 1);
        }
    }
    r = warp_max(r);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        v = warp_max(v);
        if (threadIdx.x == 0) atomic_max_nonneg(&st->resid_bits, v);
    }
}

// Closes one iteration: records the residual, counts it, raises the stop flag.
__global__ void k_sk_check(DevState *st, int max_iter) {
    if (st->sk_done) return;
    const float r = __uint_as_float(st->resid_bits);
    st->resid_bits = 0u;
    st->sk_resid = r;
    st->sk_iters += 1;
    if (!(r == r) || r == INFINITY) {
        if (!st->error) st->error = GOAT_ERR_NAN;
        st->sk_done = 1;
    } else if (r < st->sk_tol || st->sk_iters >= max_iter) {
        st->sk_done = 1;
    }
}

// Resets the iteration state and the entropic weight for a new solve.
// eps <= 0 means eps = eps_rel * max|G| (the Frank-Wolfe rule).
__global__ void k_sk_begin(DevState *st, float eps, float tol, float *g_zero, int n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float e = eps;
        if (!(e > 0.0f)) {
            const float gm = __uint_as_float(st->gmax_bits);
            e = st->eps_rel * gm;
            if (!(e > 0.0f)) e = 1.0f;  // G == 0: every doubly stochastic Q is optimal
        }
        st->eps = e;
        st->c = kLog2e / e;
        st->sk_tol = tol;
        st->sk_done = 0;
        st->sk_iters = 0;
        st->sk_resid = INFINITY;
        st->resid_bits = 0u;
    }
    if (g_zero)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) g_zero[j] = 0.0f;
}

// ---------------------------------------------------------------- fused iteration

// One Sinkhorn iteration in a single read of G (kSkFusedMinN <= n <= 32768, n a
// multiple of 16, G dense and 16-byte aligned), for every iteration of a solve after
// its first.  A cluster of four CTAs takes whole rows; CTA h holds the columns
// [h W, h W + W), W = n / 4, of each row, streamed from HBM into a ring of five
// shared-memory buffers by 1-D bulk copies (issued by a control warp).
//
// The previous iteration's row duals f' stabilise the exponents: its column scaling
// made every column of exp((f'_i + g_j - G_ij)/eps) sum to exactly 1, so each term
// is at most 1 and each row sums to at least 1/n -- no maximum is needed.  For row t
// each compute thread forms e_j = 2^(c (f'_t + g_j - G_tj)) for its 16 columns (one
// exp2 per element), keeps them in registers and sums them; the control warp adds the
// warps' sums in warp order, frees the row's buffer for the next copy and stores the
// CTA's sum, asynchronously through distributed shared memory, into the other three
// CTAs.  A row later (so the exchange's latency hides behind a row of work) the
// control warp adds the four sums in rank order into the row sum S (the same bits
// in every CTA), writes f_t = f'_t - log2(S) / c and publishes 1 / S; a row after
// that the compute warps add the row-scaled entries Q_tj = e_j / S into the
// thread's column sums (FP32 over groups of 16 rows, whose sums are added in
// FP32 in shared memory, written as FP64 per cluster for k_sk_colfinal).  Shared memory sees each
// entry twice (the copy in, one read).  Every wait is bounded; on expiry the CTA
// drains its copies, meets the other CTAs and reports GOAT_ERR_TIMEOUT.
constexpr int kSkFusedThreads = 512;  // 16 compute warps; a 17th warp is the control warp
constexpr int kSkCluster = 4;
constexpr int kSkBuffers = 5;
// Rows in the exchange ring: a CTA stores its pair of row t + 8 only after it has
// received every CTA's pair of row t + 7, so the stores of row t have seven rows of
// work to land before their slot comes round again.
constexpr int kSkSlots = 8;
// A row's entries go into the column sums kSkDefer rows after its exponents (the
// exchange's latency hides behind that much work); the exponents wait in registers.
constexpr int kSkDefer = 2;
// Rows one cluster may take: their f' are staged in shared memory at the start.
constexpr int kSkMaxRows = 1024;

__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// A float into another CTA's shared memory, completing 4 transaction bytes on that
// CTA's barrier (asynchronous: the sender does not wait for it).
__device__ __forceinline__ void st_async_f32(uint32_t remote_addr, float a, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(remote_addr),
                 "f"(a), "r"(remote_bar)
                 : "memory");
}

__device__ __forceinline__ void bulk_load_1d(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Bounded wait on a barrier phase that ignores the abort flag (draining copies).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity) && global_timer_ns() - t0 < 200000000ull) {
    }
}

// Row t of a compute thread: e_q = 2^(c (f'_t + g_j - G_tj)) <= 1 for its columns
// j = 4 (tid + 512 v) + k, q = 4 v + k (float4 reads of the row in shared memory),
// kept in registers, and their sum.
template <int CPT>
__device__ __forceinline__ void fused_row_exp(const float *__restrict__ rowbuf, int W, int tid, float c, float cf,
                                              const float (&gc)[CPT], float (&e)[CPT], float &sum) {
    sum = 0.0f;
    const float4 *row4 = reinterpret_cast<const float4 *>(rowbuf);
#pragma unroll
    for (int v = 0; v < CPT / 4; ++v) {
        const int j4 = tid + v * kSkFusedThreads;
        if (4 * j4 < W) {
            const float4 x = row4[j4];
            e[4 * v + 0] = fast_exp2(fmaf(x.x, -c, gc[4 * v + 0] + cf));
            e[4 * v + 1] = fast_exp2(fmaf(x.y, -c, gc[4 * v + 1] + cf));
            e[4 * v + 2] = fast_exp2(fmaf(x.z, -c, gc[4 * v + 2] + cf));
            e[4 * v + 3] = fast_exp2(fmaf(x.w, -c, gc[4 * v + 3] + cf));
            sum += (e[4 * v + 0] + e[4 * v + 1]) + (e[4 * v + 2] + e[4 * v + 3]);
        } else {
            e[4 * v + 0] = e[4 * v + 1] = e[4 * v + 2] = e[4 * v + 3] = 0.0f;
        }
    }
}

template <int CPT>
__global__ void __cluster_dims__(kSkCluster, 1, 1) __launch_bounds__(kSkFusedThreads + 32, 1)
    k_sk_fused(const float *__restrict__ G, int n, const float *__restrict__ g, float *__restrict__ f,
               double *__restrict__ partial, DevState *st) {
    static_assert(CPT % 4 == 0 && kSkDefer == 2, "float4 columns; two register sets of deferred rows");
    if (st->sk_done) return;  // uniform over the cluster: every CTA reads the same flag
    extern __shared__ __align__(128) unsigned char sk_smem[];
    constexpr int NW = kSkFusedThreads / 32;  // compute warps; warp NW is the control warp
    const int W = n / kSkCluster;
    float *bufs = reinterpret_cast<float *>(sk_smem);  // kSkBuffers rows of W floats
    // the sums of whole groups of 16 rows, column q of thread tid at [q][tid]
    float *grp = bufs + (size_t)kSkBuffers * W;
    __shared__ __align__(8) uint64_t full_bar[kSkBuffers], sums_bar[kSkSlots], xch_bar[kSkSlots], scl_bar[kSkSlots];
    __shared__ __align__(8) float xch[kSkSlots][kSkCluster];  // the cluster's row sums, slot = row mod 8
    __shared__ float red[kSkSlots][NW];                        // the compute warps' sums, slot = row mod 8
    __shared__ float scl[kSkSlots];                            // 1 / (the row's sum), slot = row mod 8
    __shared__ float f_stage[kSkMaxRows];                      // f' of this cluster's rows
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t rank = cluster_rank();
    const int cid = blockIdx.x / kSkCluster, ncl = gridDim.x / kSkCluster;
    const int col0 = (int)rank * W;
    const int K = cid < n ? (n - 1 - cid) / ncl + 1 : 0;  // rows of this cluster: cid + t ncl
    const uint32_t bytes = (uint32_t)W * 4u;

    if (tid == 0) {
        for (int b = 0; b < kSkBuffers; ++b) mbar_init(smem_u32(&full_bar[b]), 1);
        for (int b = 0; b < kSkSlots; ++b) {
            mbar_init(smem_u32(&sums_bar[b]), NW);
            // a row's exchange completes with this CTA's own sum (one arrival, which also
            // expects the other CTAs' bytes) and the 3 x 4 bytes they store asynchronously
            mbar_init(smem_u32(&xch_bar[b]), 1);
            mbar_init(smem_u32(&scl_bar[b]), 1);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    const float c = st->c;
    for (int t = tid; t < K; t += blockDim.x) f_stage[t] = f[cid + t * ncl];
    __syncthreads();
    cluster_sync_all();  // every CTA's barriers exist before any remote store
    volatile int *abort = &abort_flag;
    const uint32_t xch_base = smem_u32(&xch[0][0]), xbar_base = smem_u32(&xch_bar[0]);
    auto issue = [&](int t) {  // the copy of row t into its ring slot
        const int b = t % kSkBuffers;
        const uint32_t bar = smem_u32(&full_bar[b]);
        mbar_arrive_expect_tx(bar, bytes);
        bulk_load_1d(smem_u32(bufs + (size_t)b * W), G + (size_t)(cid + t * ncl) * n + col0, bytes, bar);
    };
    // bounded wait for a phase; false (and the abort flag raised) on expiry or abort
    auto wait = [&](uint32_t bar, uint32_t parity) -> bool { return mbar_wait_bounded(bar, parity, abort); };

    int issued = K < kSkBuffers ? K : kSkBuffers;
    if (warp == NW) {
        // ---------------- control warp: the CTA's row sums, the exchange, the copies,
        // and the row scalings
        if (lane == 0) {
            // row tp's cluster sum S (the four CTAs' sums in rank order: the same bits in
            // every CTA), 1 / S for the compute warps, and f_tp = f'_tp - log2(S) / c
            auto scale_row = [&](int tp) -> bool {
                const int slot = tp % kSkSlots;
                if (!wait(xbar_base + 8u * (uint32_t)slot, (uint32_t)(tp / kSkSlots) & 1u)) return false;
                float S = xch[slot][0];
                for (int r = 1; r < kSkCluster; ++r) S += xch[slot][r];
                if (rank == 0) f[cid + tp * ncl] = f_stage[tp] - __log2f(S) / c;
                scl[slot] = 1.0f / S;
                mbar_arrive(smem_u32(&scl_bar[slot]));
                return true;
            };
            for (int t = 0; t < issued; ++t) issue(t);
            for (int t = 0; t < K; ++t) {
                const int slot = t % kSkSlots;
                // the previous row's exchange has had a row of work to land
                if (t >= 1 && !scale_row(t - 1)) break;
                if (!wait(smem_u32(&sums_bar[slot]), (uint32_t)(t / kSkSlots) & 1u)) break;
                float cs = 0.0f;
                for (int w = 0; w < NW; ++w) cs += red[slot][w];  // warp order: fixed
                const uint32_t off = 4u * (uint32_t)(slot * kSkCluster + (int)rank);
                xch[slot][rank] = cs;
                mbar_arrive_expect_tx(xbar_base + 8u * (uint32_t)slot, 4u * (kSkCluster - 1));
                for (int r = 0; r < kSkCluster; ++r) {
                    if (r == (int)rank) continue;
                    st_async_f32(mapa_shared(xch_base, r) + off, cs, mapa_shared(xbar_base, r) + 8u * (uint32_t)slot);
                }
                // every compute warp has read row t (its exponents are in registers):
                // its buffer takes row t + kSkBuffers
                if (issued < K) issue(issued++);
                if (t == K - 1) scale_row(t);
            }
        }
    } else {
        // ---------------- compute warps
        float gc[CPT];  // c g_j
#pragma unroll
        for (int v = 0; v < CPT / 4; ++v) {
            const int j = 4 * (tid + v * kSkFusedThreads);
#pragma unroll
            for (int k = 0; k < 4; ++k) gc[4 * v + k] = j < W ? g[col0 + j + k] * c : 0.0f;
        }
        float acc[CPT], e0[CPT], e1[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            acc[q] = 0.0f;
            grp[q * kSkFusedThreads + tid] = 0.0f;
        }
        // row t's exponents and their sum (false on abort)
        auto row_exp = [&](int t, float (&e)[CPT]) -> bool {
            const int b = t % kSkBuffers;
            const float cf = c * f_stage[t];
            if (!wait(smem_u32(&full_bar[b]), (uint32_t)(t / kSkBuffers) & 1u)) return false;
            float sum;
            fused_row_exp<CPT>(bufs + (size_t)b * W, W, tid, c, cf, gc, e, sum);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) {
                red[t % kSkSlots][warp] = sum;
                mbar_arrive(smem_u32(&sums_bar[t % kSkSlots]));  // also: this warp is done with the buffer
            }
            return true;
        };
        // row tp's entries e / S into the column sums
        auto row_acc = [&](int tp, const float (&e)[CPT]) -> bool {
            const int slot = tp % kSkSlots;
            if (!wait(smem_u32(&scl_bar[slot]), (uint32_t)(tp / kSkSlots) & 1u)) return false;
            const float scale = scl[slot];
#pragma unroll
            for (int q = 0; q < CPT; ++q) acc[q] = fmaf(e[q], scale, acc[q]);
            if ((tp & 15) == 15) {
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    grp[q * kSkFusedThreads + tid] += acc[q];
                    acc[q] = 0.0f;
                }
            }
            return true;
        };
        // row t's exponents go into set t mod 2; that set is first freed by adding row
        // t - 2 (kSkDefer) into the column sums
        bool ok = true;
        for (int t = 0; ok && t < K + kSkDefer; t += 2) {
            if (t >= 2) ok = row_acc(t - 2, e0);
            if (ok && t < K) ok = row_exp(t, e0);
            if (ok && t >= 1 && t - 1 < K) ok = row_acc(t - 1, e1);
            if (ok && t + 1 < K) ok = row_exp(t + 1, e1);
        }
        if (ok && !*abort) {
            double *dst = partial + (size_t)cid * n + col0;
#pragma unroll
            for (int v = 0; v < CPT / 4; ++v) {
                const int j = 4 * (tid + v * kSkFusedThreads);
                if (j < W) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        dst[j + k] = (double)grp[(4 * v + k) * kSkFusedThreads + tid] + (double)acc[4 * v + k];
                }
            }
        }
    }
    __syncthreads();
    const bool aborted = *abort != 0;
    if (aborted && warp == NW && lane == 0) {
        // let the copies in flight land before the shared memory is released (the last
        // kSkBuffers issued rows, one per buffer)
        for (int tt = issued > kSkBuffers ? issued - kSkBuffers : 0; tt < issued; ++tt)
            mbar_drain(smem_u32(&full_bar[tt % kSkBuffers]), (uint32_t)(tt / kSkBuffers) & 1u);
    }
    __syncthreads();
    cluster_sync_all();  // no CTA leaves while another may still write into it
    if (aborted && tid == 0 && !st->error) st->error = GOAT_ERR_TIMEOUT;
}

// ---------------------------------------------------------------- Q materialisation

// Q_ij = 2^(c (f_i + g_j - G_ij)), written as BF16 split terms (hi, and lo when
// terms == 2) into the GEMM operand buffer, zero in the padding columns, and
// optionally as FP32.  A thread writes 8 columns of a row: two float4 loads of G
// and of g where the 8 columns lie inside the row and G is 16-byte aligned,
// scalar loads at the edge; 32-bit index arithmetic when the chunk count fits.
template <typename Idx>
__device__ __forceinline__ void write_q_body(const float *__restrict__ G, int n, long long ld,
                                             const float *__restrict__ f, const float *__restrict__ g, float c,
                                             __nv_bfloat16 *__restrict__ Qb, int ldq, int terms, float *__restrict__ Qf,
                                             long long ldf, bool vec) {
    const Idx chunks = (Idx)(ldq / 8);  // 8 columns per thread
    const Idx total = (Idx)n * chunks;
    for (Idx t = (Idx)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (Idx)gridDim.x * blockDim.x) {
        const int i = (int)(t / chunks);
        const int j0 = (int)(t - (Idx)i * chunks) * 8;
        const float fi = __ldg(f + i);
        const float *Gi = G + (long long)i * ld;
        float q[8];
        if (vec && j0 + 7 < n) {
            const float4 a0 = __ldg(reinterpret_cast<const float4 *>(Gi + j0));
            const float4 a1 = __ldg(reinterpret_cast<const float4 *>(Gi + j0 + 4));
            const float4 b0 = __ldg(reinterpret_cast<const float4 *>(g + j0));
            const float4 b1 = __ldg(reinterpret_cast<const float4 *>(g + j0 + 4));
            q[0] = fast_exp2((fi + b0.x - a0.x) * c);
            q[1] = fast_exp2((fi + b0.y - a0.y) * c);
            q[2] = fast_exp2((fi + b0.z - a0.z) * c);
            q[3] = fast_exp2((fi + b0.w - a0.w) * c);
            q[4] = fast_exp2((fi + b1.x - a1.x) * c);
            q[5] = fast_exp2((fi + b1.y - a1.y) * c);
            q[6] = fast_exp2((fi + b1.z - a1.z) * c);
            q[7] = fast_exp2((fi + b1.w - a1.w) * c);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int j = j0 + k;
                q[k] = (j < n) ? fast_exp2((fi + __ldg(g + j) - __ldg(Gi + j)) * c) : 0.0f;
            }
        }
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(q[k], q[k + 1]);
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(q[k] - hf.x, q[k + 1] - hf.y);
            hw[k / 2] = *reinterpret_cast<const uint32_t *>(&h2);
            lw[k / 2] = *reinterpret_cast<const uint32_t *>(&l2);
        }
        if (Qb) {
            __nv_bfloat16 *row = Qb + (long long)i * ((long long)terms * ldq);
            *reinterpret_cast<uint4 *>(row + j0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            if (terms > 1) *reinterpret_cast<uint4 *>(row + ldq + j0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        if (Qf) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (j0 + k < n) Qf[(long long)i * ldf + j0 + k] = q[k];
        }
    }
}

__global__ void __launch_bounds__(256) k_write_q(const float *__restrict__ G, int n, long long ld,
                                                 const float *__restrict__ f, const float *__restrict__ g,
                                                 const DevState *__restrict__ st, __nv_bfloat16 *__restrict__ Qb,
                                                 int ldq, int terms, float *__restrict__ Qf, long long ldf) {
    const float c = st->c;
    const bool vec = ((ld & 3) == 0) && (((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(g)) & 15) == 0);
    const long long total = (long long)n * (ldq / 8);
    if (total + (long long)gridDim.x * blockDim.x < 0xffffffffLL)
        write_q_body<unsigned>(G, n, ld, f, g, c, Qb, ldq, terms, Qf, ldf, vec);
    else
        write_q_body<long long>(G, n, ld, f, g, c, Qb, ldq, terms, Qf, ldf, vec);
}

// ---------------------------------------------------------------- host driver

struct SinkhornLaunch {
    int row_grid, colpart_x, colpart_y, rows_per_chunk, final_grid;
};

static SinkhornLaunch sinkhorn_launch(int n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    SinkhornLaunch L;
    L.row_grid = (int)std::min<int64_t>(ceil_div(n, 8), (int64_t)sms * 16);
    // column pass: as many row chunks as fill one wave of resident CTAs (a second,
    // partial wave would leave most SMs idle at its end), at least 64 rows each
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sk_colpart<false>, 256, 0) != cudaSuccess || occ < 1)
        occ = 4;
    L.colpart_x = (int)ceil_div(n, kSkColsPerCta);
    const int64_t slots = (int64_t)sms * occ;
    int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(slots / L.colpart_x, ceil_div(n, 64)));
    L.rows_per_chunk = (int)ceil_div(n, chunks);
    L.colpart_y = (int)ceil_div(n, L.rows_per_chunk);
    L.final_grid = (int)ceil_div(n, 256);
    return L;
}

// Clusters of the fused iteration: at most one CTA per SM (the bound the partial-sum
// buffer is sized for); the launch uses as many as are co-resident.
static int fused_clusters() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, sms / kSkCluster);
}

// Clusters of k_sk_fused<CPT> that fit on the device at once with `smem` bytes each:
// the rows are spread over exactly one wave of them (a cluster must sit within one
// GPC, so fewer pairs than SMs / 2 may be co-resident, and a second, partial wave
// would double the pass).  Cached per instantiation and size.
template <typename Kern>
static int fused_wave_clusters(Kern kern, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kSkCluster * fused_clusters());
    cfg.blockDim = dim3(kSkFusedThreads + 32);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = kSkCluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, (const void *)kern, &cfg) != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        ncl = fused_clusters();
    }
    return std::min(ncl, fused_clusters());
}

static bool use_fused(const float *G, int n, long long ld) {
    return n >= kSkFusedMinN && n <= kSkCluster * kSkFusedThreads * 16 && (n % 16) == 0 && ld == n &&
           (reinterpret_cast<uintptr_t>(G) & 15) == 0;
}

long long sinkhorn_partial_elems(int n) {
    SinkhornLaunch L = sinkhorn_launch(n);
    const long long chunks = n >= kSkFusedMinN ? std::max<long long>(L.colpart_y, fused_clusters()) : L.colpart_y;
    return chunks * n;
}

// Queues the fused iteration (k_sk_fused + k_sk_colfinal over the clusters' partial
// column sums); returns false if its launch could not be configured.
static bool sinkhorn_fused(const float *G, int n, float *f, float *g, double *partial, DevState *st,
                           cudaStream_t s) {
    const int W = n / kSkCluster;
    const size_t smem = ((size_t)kSkBuffers * W + (size_t)16 * kSkFusedThreads) * sizeof(float);
    // n >= kSkFusedMinN: W >= 5120 columns, at most 16 a thread.  The kernel is
    // configured once for the largest quarter-row it takes (W = 512 * 16); the
    // clusters that fit in one wave are found once per n.
    auto kern = k_sk_fused<16>;
    static bool configured = false;
    static int wave_n = 0, wave_ncl = 0;
    if (!configured) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (kSkBuffers + 1) * kSkFusedThreads * 16 * (int)sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        configured = true;
    }
    if (wave_n != n) {
        wave_ncl = fused_wave_clusters(kern, smem);
        wave_n = n;
    }
    const int ncl = wave_ncl;
    if (ceil_div(n, ncl) > kSkMaxRows) return false;  // more rows a cluster than f' slots
    kern<<<kSkCluster * ncl, kSkFusedThreads + 32, smem, s>>>(G, n, g, f, partial, st);
    k_sk_colfinal<<<(int)ceil_div(n, 256), 256, 0, s>>>(partial, ncl, n, G, n, f, g, st);
    return true;
}

// Queues the column pass: full, aligned 2048-column CTAs take the fallback-free
// instantiation, the rest (a ragged right edge, or all of an unaligned G) the
// general one.  Returns the number of launches.
static int sinkhorn_colpart(const float *G, int n, long long ld, const float *f, const float *g, double *partial,
                            const DevState *st, const SinkhornLaunch &L, cudaStream_t s) {
    const bool aligned = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(G) & 15) == 0);
    const int full = aligned ? n / kSkColsPerCta : 0;
    const int edge = L.colpart_x - full;
    if (full > 0)
        k_sk_colpart<false><<<dim3(full, L.colpart_y), 256, 0, s>>>(G, n, ld, f, g, partial, L.rows_per_chunk, 0, st);
    if (edge > 0)
        k_sk_colpart<true><<<dim3(edge, L.colpart_y), 256, 0, s>>>(G, n, ld, f, g, partial, L.rows_per_chunk,
                                                                    full * kSkColsPerCta, st);
    return (full > 0) + (edge > 0);
}

// Queues one Sinkhorn iteration: the fused single-read form where it applies (G
// read once, 4 n^2 bytes), else the row pass and the column pass (G read twice).
static void sinkhorn_iteration(const float *G, int n, long long ld, float *f, float *g, double *partial,
                               DevState *st, int max_iter, const SinkhornLaunch &L, bool first, cudaStream_t s) {
    // the fused form takes the previous iteration's f as its stabiliser: not on the first
    if (!first && use_fused(G, n, ld) && sinkhorn_fused(G, n, f, g, partial, st, s)) {
        note_launches(3);
    } else {
        k_sk_row<<<L.row_grid, 256, 0, s>>>(G, n, ld, g, f, st);
        note_launches(3 + sinkhorn_colpart(G, n, ld, f, g, partial, st, L, s));
        k_sk_colfinal<<<L.final_grid, 256, 0, s>>>(partial, L.colpart_y, n, G, ld, f, g, st);
    }
    k_sk_check<<<1, 1, 0, s>>>(st, max_iter);
}

// Runs Sinkhorn until the device stop flag rises (tolerance or max_iter),
// polling the flag every `check_every` iterations.  `host_flag` is pinned
// host memory of at least 2 ints.  Returns a goat_status.
int sinkhorn_solve(const float *G, int n, long long ld, float *f, float *g, double *partial, DevState *st,
                   int max_iter, int check_every, int *host_flag, cudaStream_t s) {
    const SinkhornLaunch L = sinkhorn_launch(n);
    if (check_every < 1) check_every = 1;
    int done_iters = 0;
    while (done_iters < max_iter) {
        const int k = std::min(check_every, max_iter - done_iters);
        for (int t = 0; t < k; ++t) sinkhorn_iteration(G, n, ld, f, g, partial, st, max_iter, L, done_iters + t == 0, s);
        done_iters += k;
        if (cudaMemcpyAsync(host_flag, &st->sk_done, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return GOAT_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return GOAT_ERR_CUDA;
        if (host_flag[0]) break;
    }
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

// Queues exactly max_iter iteration slots without any host synchronisation; the
// kernels stop doing work once the device stop flag rises.
void sinkhorn_queue_fixed(const float *G, int n, long long ld, float *f, float *g, double *partial, DevState *st,
                          int max_iter, cudaStream_t s) {
    const SinkhornLaunch L = sinkhorn_launch(n);
    for (int t = 0; t < max_iter; ++t) sinkhorn_iteration(G, n, ld, f, g, partial, st, max_iter, L, t == 0, s);
}

void sinkhorn_begin(DevState *st, float eps, float tol, float *g_zero, int n, cudaStream_t s) {
    note_launches(1);
    k_sk_begin<<<g_zero ? (int)std::min<int64_t>(ceil_div(n, 256), 1024) : 1, 256, 0, s>>>(st, eps, tol, g_zero, n);
}

void write_q(const float *G, int n, long long ld, const float *f, const float *g, const DevState *st,
             __nv_bfloat16 *Qb, int ldq, int terms, float *Qf, long long ldf, cudaStream_t s) {
    note_launches(1);
    const long long total = (long long)n * (ldq / 8);
    const int grid = (int)std::min<long long>(ceil_div(total, 256), 152LL * 32);
    k_write_q<<<grid, 256, 0, s>>>(G, n, ld, f, g, st, Qb, ldq, terms, Qf, ldf);
}

}  // namespace goat
