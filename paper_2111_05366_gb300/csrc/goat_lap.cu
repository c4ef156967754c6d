// goat_lap.cu -- K5: the final projection onto the permutations (Alg. 1 / Alg. 3
// return line), argmax_perm sum_i a[i][perm i], on the GPU.
//
// Stage 1, auction with eps-scaling (Bertsekas): every unassigned row i finds
// its best object j1 = argmax_j (a_ij - p_j) and the runner-up value, and bids
// p_j1 + (best - second) + eps; each object goes to its highest bidder (lowest
// row on exact ties) and takes that bid as its price.  Rounds repeat until all
// rows are assigned; eps shrinks by 8x per phase down to max|a| * 2^-40.
// Prices are FP64.  The result is eps-optimal: within n * eps of the optimum.
//
// Stage 2, exact certification by LP duality: with u_i = a[i][perm i] - p[perm i]
// the assignment is optimal iff a_ij <= u_i + p_j for all (i, j).  A
// Bellman-Ford style relaxation raises p_j to max_i (a_ij - u_i) until no
// constraint is violated beyond rounding (4 ulp of the price scale).  If the
// relaxation keeps raising prices, the assignment is not optimal and the
// raised prices' predecessor links contain an improving cycle; such cycles are
// found in parallel (bounded walks) and the assignment is rotated along them.
// Every loop is bounded; running out returns GOAT_ERR_NOT_CONVERGED.
#include <algorithm>
#include <climits>
#include <cmath>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

struct LapBuffers {
    double *price, *my_bid, *u, *colmax;
    int *owner, *assign, *my_obj, *bwin, *pred, *colarg, *cyc_start;
    unsigned long long *bbest;
    int nchunks;
};

size_t lap_bytes(int n, int nchunks) {
    size_t b = 0;
    b += 3 * (size_t)n * sizeof(double);                 // price, my_bid, u
    b += (size_t)nchunks * n * sizeof(double);           // colmax partials
    b += 6 * (size_t)n * sizeof(int);                    // owner, assign, my_obj, bwin, pred, cyc_start
    b += (size_t)nchunks * n * sizeof(int);              // colarg partials
    b += (size_t)n * sizeof(unsigned long long);         // bbest
    return b + 16 * 256;
}

static LapBuffers carve(void *base, int n, int nchunks) {
    uint8_t *p = (uint8_t *)base;
    auto take = [&](size_t bytes) {
        uint8_t *r = p;
        p += round_up((int64_t)bytes, 256);
        return (void *)r;
    };
    LapBuffers L;
    L.price = (double *)take(sizeof(double) * n);
    L.my_bid = (double *)take(sizeof(double) * n);
    L.u = (double *)take(sizeof(double) * n);
    L.colmax = (double *)take(sizeof(double) * (size_t)nchunks * n);
    L.owner = (int *)take(sizeof(int) * n);
    L.assign = (int *)take(sizeof(int) * n);
    L.my_obj = (int *)take(sizeof(int) * n);
    L.bwin = (int *)take(sizeof(int) * n);
    L.pred = (int *)take(sizeof(int) * n);
    L.cyc_start = (int *)take(sizeof(int) * n);
    L.colarg = (int *)take(sizeof(int) * (size_t)nchunks * n);
    L.bbest = (unsigned long long *)take(sizeof(unsigned long long) * n);
    L.nchunks = nchunks;
    return L;
}

int lap_chunks(int n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int strips = (int)ceil_div(n, 256);
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(sms * 8, strips), ceil_div(n, 32)));
}

// ---------------------------------------------------------------- auction

__global__ void k_lap_reset(int n, const LapBuffers L, DevState *st, int reset_prices) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        L.owner[j] = -1;
        L.assign[j] = -1;
        L.bbest[j] = 0ull;
        L.bwin[j] = INT_MAX;
        L.my_obj[j] = -1;
        if (reset_prices) L.price[j] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->lap_unassigned = n;
}

__global__ void __launch_bounds__(256) k_lap_bid(const float *__restrict__ M, int n, float sgn, const LapBuffers L,
                                                 double eps, const DevState *st) {
    if (st->lap_unassigned == 0) return;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < n; i += nw) {
        if (L.assign[i] >= 0) {
            if (lane == 0) L.my_obj[i] = -1;
            continue;
        }
        const float *Mi = M + (long long)i * n;
        double b1 = -INFINITY, b2 = -INFINITY;
        int j1 = INT_MAX;
        for (int j = lane; j < n; j += 32) {
            const double v = (double)(sgn * __ldg(Mi + j)) - L.price[j];
            if (v > b1) {
                b2 = b1;
                b1 = v;
                j1 = j;
            } else if (v > b2) {
                b2 = v;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double o1 = __shfl_xor_sync(0xffffffffu, b1, o);
            const double o2 = __shfl_xor_sync(0xffffffffu, b2, o);
            const int oj = __shfl_xor_sync(0xffffffffu, j1, o);
            if (o1 > b1 || (o1 == b1 && oj < j1)) {
                b2 = fmax(b1, o2);
                b1 = o1;
                j1 = oj;
            } else {
                b2 = fmax(b2, o1);
            }
        }
        if (lane == 0) {
            const double inc = (b2 == -INFINITY) ? eps : (b1 - b2) + eps;
            const double bid = L.price[j1] + inc;
            L.my_obj[i] = j1;
            L.my_bid[i] = bid;
            atomicMax(&L.bbest[j1], (unsigned long long)__double_as_longlong(bid));
        }
    }
}

__global__ void k_lap_win(int n, const LapBuffers L, const DevState *st) {
    if (st->lap_unassigned == 0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = L.my_obj[i];
        if (j >= 0 && L.bbest[j] == (unsigned long long)__double_as_longlong(L.my_bid[i])) atomicMin(&L.bwin[j], i);
    }
}

__global__ void k_lap_assign(int n, const LapBuffers L, DevState *st) {
    if (st->lap_unassigned == 0) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int w = L.bwin[j];
        if (w == INT_MAX) continue;
        const int old = L.owner[j];
        if (old >= 0)
            L.assign[old] = -1;
        else
            atomicSub(&st->lap_unassigned, 1);
        L.owner[j] = w;
        L.assign[w] = j;
        L.price[j] = __longlong_as_double((long long)L.bbest[j]);
        L.bbest[j] = 0ull;
        L.bwin[j] = INT_MAX;
    }
}

// ---------------------------------------------------------------- certification

__global__ void k_cert_profit(const float *__restrict__ M, int n, float sgn, const LapBuffers L) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = L.assign[i];
        L.u[i] = (double)(sgn * M[(long long)i * n + j]) - L.price[j];
    }
}

// Column maxima of a_ij - u_i over a chunk of rows (with the arg row).
__global__ void __launch_bounds__(256) k_cert_colpart(const float *__restrict__ M, int n, float sgn,
                                                      const LapBuffers L, int rows_per_chunk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int r0 = blockIdx.y * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    double best = -INFINITY;
    int arg = -1;
    for (int i = r0; i < r1; ++i) {
        const double v = (double)(sgn * __ldg(M + (long long)i * n + j)) - L.u[i];
        if (v > best) {
            best = v;
            arg = i;
        }
    }
    L.colmax[(long long)blockIdx.y * n + j] = best;
    L.colarg[(long long)blockIdx.y * n + j] = arg;
}

// Raises violated prices; counts raises in st->lap_changed and the total
// violation (sum over columns of max(0, req - p)) in st->lap_gap.
__global__ void k_cert_colfinal(int n, const LapBuffers L, double tol, DevState *st) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    double viol = 0.0;
    if (j < n) {
        double best = -INFINITY;
        int arg = -1;
        for (int k = 0; k < L.nchunks; ++k) {
            const double v = L.colmax[(long long)k * n + j];
            if (v > best) {
                best = v;
                arg = L.colarg[(long long)k * n + j];
            }
        }
        const double p = L.price[j];
        if (best > p + tol) {
            viol = best - p;
            L.price[j] = best;
            L.pred[j] = arg;
            atomicAdd(&st->lap_changed, 1);
        }
    }
    for (int o = 16; o > 0; o >>= 1) viol += __shfl_xor_sync(0xffffffffu, viol, o);
    if ((threadIdx.x & 31) == 0 && viol > 0.0) atomicAdd(&st->lap_gap, viol);
}

__global__ void k_cert_reset(DevState *st) {
    st->lap_changed = 0;
    st->lap_gap = 0.0;
}

// Each object j whose price was raised starts a bounded walk along predecessor
// links: object j was raised by row i = pred[j], which holds object assign[i].
// Returning to j closes a cycle of rows that would each move one object forward.
__global__ void k_find_cycles(int n, const LapBuffers L, int max_len, int *best_start) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        if (L.pred[j] < 0) continue;
        int cur = j;
        for (int s = 0; s < max_len; ++s) {
            const int i = L.pred[cur];
            if (i < 0) break;
            cur = L.assign[i];
            if (cur == j) {
                atomicMin(best_start, j);
                break;
            }
        }
    }
}

// Rotates the assignment along the cycle through *best_start if it improves the
// objective by more than tol; clears the predecessor links.
__global__ void k_cancel_cycle(const float *__restrict__ M, int n, float sgn, const LapBuffers L, int max_len,
                               const int *best_start, double tol, DevState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j0 = *best_start;
    if (j0 == INT_MAX) return;
    // gain of moving every row of the cycle to the object it points at
    double gain = 0.0;
    int cur = j0, len = 0;
    do {
        const int i = L.pred[cur];
        gain += (double)(sgn * M[(long long)i * n + cur]) - (double)(sgn * M[(long long)i * n + L.assign[i]]);
        cur = L.assign[i];
        ++len;
    } while (cur != j0 && len <= max_len);
    if (cur == j0 && gain > tol) {
        cur = j0;
        int rows_moved = 0;
        // walk once more, collecting (row, new object) pairs before rewriting
        int i = L.pred[cur];
        int next_obj = cur;
        do {
            const int old_obj = L.assign[i];
            L.assign[i] = next_obj;
            L.owner[next_obj] = i;
            next_obj = old_obj;
            i = L.pred[old_obj];
            ++rows_moved;
        } while (next_obj != j0 && rows_moved <= max_len);
        atomicAdd(&st->lap_phase_done, 1);  // number of cycles cancelled
    }
}

__global__ void k_clear_pred(int n, const LapBuffers L, int *best_start) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) L.pred[j] = -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) *best_start = INT_MAX;
}

// sum_i M[i][perm i] in FP64 in row order (the order the oracle uses); one block.
__global__ void k_assignment_cost(const float *__restrict__ M, int n, const int *__restrict__ perm, double *out) {
    __shared__ double buf[1024];
    double acc = 0.0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        if (threadIdx.x < 1024) buf[threadIdx.x] = (i < n) ? (double)M[(long long)i * n + perm[i]] : 0.0;
        __syncthreads();
        if (threadIdx.x == 0) {
            const int lim = min(1024, n - base);
            for (int k = 0; k < lim; ++k) acc += buf[k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = acc;
}

__global__ void k_copy_perm(int n, const LapBuffers L, int32_t *perm) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) perm[i] = L.assign[i];
}

// ---------------------------------------------------------------- host driver

struct HostPoll {
    int *pinned;  // >= 4 ints
};

static int poll_int(const int *dev, int *pinned, cudaStream_t s) {
    cudaMemcpyAsync(pinned, dev, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return *pinned;
}

// Runs the projection.  lap_ws must hold lap_bytes(n, lap_chunks(n)) bytes.
int lap_solve(const float *M, int n, int maximize, int32_t *perm_out, void *lap_ws, DevState *st, int max_rounds,
              double *cost_dev, int *host_pinned, double *gap_host, int *rounds_host, cudaStream_t s) {
    const int nchunks = lap_chunks(n);
    LapBuffers L = carve(lap_ws, n, nchunks);
    const float sgn = maximize ? 1.0f : -1.0f;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g1 = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), sms * 8));
    const int gbid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 8), sms * 16));

    // scale of the benefits: C = max |M|
    unsigned *cbits = reinterpret_cast<unsigned *>(&st->gmax_next);
    cudaMemsetAsync(cbits, 0, sizeof(unsigned), s);
    absmax(M, (long long)n * n, cbits, s);
    cudaMemcpyAsync(host_pinned, cbits, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return GOAT_ERR_CUDA;
    float Cf;
    memcpy(&Cf, host_pinned, sizeof(float));
    cudaMemsetAsync(cbits, 0, sizeof(unsigned), s);
    if (!(Cf == Cf) || std::isinf(Cf)) return GOAT_ERR_NAN;
    const double C = Cf > 0.0f ? (double)Cf : 1.0;

    k_lap_reset<<<g1, 256, 0, s>>>(n, L, st, 1);
    double eps = C / 4.0;
    const double eps_final = C * std::ldexp(1.0, -40);
    int rounds = 0;
    const int batch = 8;
    for (;;) {
        // phase: all rows unassigned, prices kept
        k_lap_reset<<<g1, 256, 0, s>>>(n, L, st, 0);
        for (;;) {
            for (int b = 0; b < batch; ++b) {
                k_lap_bid<<<gbid, 256, 0, s>>>(M, n, sgn, L, eps, st);
                k_lap_win<<<g1, 256, 0, s>>>(n, L, st);
                k_lap_assign<<<g1, 256, 0, s>>>(n, L, st);
            }
            rounds += batch;
            const int left = poll_int(&st->lap_unassigned, host_pinned, s);
            if (left == 0) break;
            if (rounds >= max_rounds) return GOAT_ERR_NOT_CONVERGED;
        }
        if (eps <= eps_final) break;
        eps = std::max(eps / 8.0, eps_final);
    }

    // certification / repair
    const double tol = 4.0 * std::ldexp(1.0, -52) * std::max(C, 1.0) * 4.0;
    const int rows_per_chunk = (int)ceil_div(n, nchunks);
    const int ychunks = (int)ceil_div(n, rows_per_chunk);  // <= nchunks: the partial buffers fit
    L.nchunks = ychunks;
    int *best_start = &st->pad0;
    k_clear_pred<<<g1, 256, 0, s>>>(n, L, best_start);
    double gap = 0.0;
    bool certified = false;
    int cycles_left = 64;
    for (int round = 0; round < 512; ++round) {
        k_cert_reset<<<1, 1, 0, s>>>(st);
        k_cert_profit<<<g1, 256, 0, s>>>(M, n, sgn, L);
        k_cert_colpart<<<dim3((unsigned)ceil_div(n, 256), (unsigned)ychunks), 256, 0, s>>>(M, n, sgn, L,
                                                                                           rows_per_chunk);
        k_cert_colfinal<<<g1 > 0 ? (int)ceil_div(n, 256) : 1, 256, 0, s>>>(n, L, tol, st);
        cudaMemcpyAsync(host_pinned, &st->lap_changed, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&gap, &st->lap_gap, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return GOAT_ERR_CUDA;
        if (host_pinned[0] == 0) {
            certified = true;
            break;
        }
        if (round % 8 == 7 && cycles_left > 0) {
            k_find_cycles<<<g1, 256, 0, s>>>(n, L, std::min(n, 4096), best_start);
            k_cancel_cycle<<<1, 1, 0, s>>>(M, n, sgn, L, std::min(n, 4096), best_start, tol, st);
            k_clear_pred<<<g1, 256, 0, s>>>(n, L, best_start);
            --cycles_left;
        }
    }
    k_copy_perm<<<g1, 256, 0, s>>>(n, L, perm_out);
    k_assignment_cost<<<1, 1024, 0, s>>>(M, n, perm_out, cost_dev);
    if (gap_host) *gap_host = certified ? 0.0 : gap;
    if (rounds_host) *rounds_host = rounds;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GOAT_ERR_CUDA;
    return certified ? GOAT_OK : GOAT_ERR_NOT_CONVERGED;
}

}  // namespace goat
