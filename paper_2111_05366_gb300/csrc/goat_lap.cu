// goat_lap.cu -- K5: the final projection onto the permutations (Alg. 1 / Alg. 3
// return line), argmax_perm sum_i a[i][perm i], on the GPU, as an exact
// integer auction.
//
// Benefits.  a_ij = sgn * M_ij is quantised to 64-bit integers
//     a_int = round(a * 2^(40 - e)) * Qm,   C' = 2^e > max|M|,  Qm = 2^ceil(log2(n + 1)) > n,
// i.e. 40 bits below the largest entry (fewer above n = 2^18, so that prices stay
// far below 2^63), then scaled by a power of two above n.
// Every entry >= C' 2^-17 converts exactly (its 24-bit mantissa fits); smaller
// ones move by at most C' 2^-41.
//
// Auction with eps-scaling (Bertsekas): every unassigned row i finds its best
// object j1 = argmax_j (a_ij - p_j) and the runner-up value, and bids
// p_j1 + (best - second) + eps; each object goes to its highest bidder (lowest row
// on ties) at that price.  eps falls 8x per phase to 1.  All arithmetic is exact
// int64 (GB300's FP64 rate is far too low for these scans).  At eps = 1 the final
// assignment is within n * eps = n < Qm of the optimum, and every assignment value
// of the quantised matrix is a multiple of Qm, so it is optimal for that matrix:
// an exact LAP, no tolerance involved.
//
// Scheduling.  Each phase starts with parallel Jacobi rounds (one cooperative
// launch per phase) while many rows bid, until at most 4 rows bid or the number of
// bidders has not fallen for 16 rounds; when they end with at most 4 rows left,
// that tail (a few rows evicting each other) runs in Gauss-Seidel order in one
// CTA, or for n >= 4096 in a cluster of 8 CTAs that split the columns.  Rows that chase
// the last free objects through a large set of near-tied objects (each bid lifts
// one price by about eps, so closing a gap of D costs about |set| D / eps bids)
// are left to the next phase, which starts from the prices alone; in the last
// phase they are placed by shortest augmenting paths instead (Jonker-Volgenant's
// Dijkstra step, exact integer duals).  The search runs on the matrix a~ that
// adds to each assigned pair its eps-complementary-slackness slack
// delta_i = max_j (a_ij - p_j) - (a_i,j_i - p_j_i) in [0, eps], so that the
// auction's prices and assignment are an exactly feasible, tight starting point.
// Every assignment value of a~ is within n eps of that of a; in the last phase
// (eps = 1 < Qm / n) an optimum of a~ is therefore an optimum of a, so the last
// phase ends complete and optimal.  (The searches can also complete every phase:
// goat_lap_options.sap_every_phase.)
// Budgets bound the time on degenerate inputs: if the last phase still runs out,
// the free rows are filled greedily and the returned duality gap says how far
// from optimal that is (0 when the proof above applies).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstddef>
#include <cmath>
#include <cstring>

#include <cooperative_groups.h>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

typedef long long i64;

// Grid-wide reduction slot of the augmenting-path searches (one per barrier epoch).
struct SapSlot {
    long long minv;  // least label of the open non-free columns
    long long tmin;  // least label of the free columns
    int count;       // rows appended to the epoch's frontier list
    int pad;
    int hist[64];    // open non-free columns by bit length of (label - base)
};

struct LapBuffers {
    i64 *price, *my_bid;
    int *owner, *assign, *my_obj, *bwin, *queue;
    int *blist[2];    // rows bidding in alternate Jacobi rounds
    unsigned long long *bbest;
    int *sap_pred;    // predecessor row of every column after a search
    int *tflag, *tlist, *mark_row, *mark_col;  // augmenting-path targets and the vertices used
    i64 *ufree;       // potentials of the free rows
    i64 *mben;        // benefit a~ of every assigned row's pair
    int *frow[2];     // frontier lists (rows to scan) of alternate epochs
    i64 *fh[2];       // their label offsets
    int *fj0[2];      // their boosted columns (-1: none)
    i64 *fdl[2];      // and boosts
    SapSlot *ring;    // 4 reduction slots
};

size_t lap_bytes(int n, int /*nchunks*/) {
    return 2 * (size_t)n * sizeof(i64) + 5 * (size_t)n * sizeof(int) + (size_t)n * 8 + 16 * 256 +
           (size_t)n * sizeof(int) + 2 * (size_t)n * (sizeof(int) + sizeof(i64)) + 4 * sizeof(SapSlot) + 6 * 256 +
           4 * (size_t)n * sizeof(int) + 2 * (size_t)n * sizeof(i64) + 6 * 256 +
           2 * (size_t)n * (sizeof(int) + sizeof(i64)) + 4 * 256 + 2 * (size_t)n * sizeof(int) + 2 * 256;
}

static LapBuffers carve(void *base, int n) {
    uint8_t *p = (uint8_t *)base;
    auto take = [&](size_t bytes) {
        uint8_t *r = p;
        p += round_up((int64_t)bytes, 256);
        return (void *)r;
    };
    LapBuffers L;
    L.price = (i64 *)take(sizeof(i64) * n);
    L.my_bid = (i64 *)take(sizeof(i64) * n);
    L.owner = (int *)take(sizeof(int) * n);
    L.assign = (int *)take(sizeof(int) * n);
    L.my_obj = (int *)take(sizeof(int) * n);
    L.bwin = (int *)take(sizeof(int) * n);
    L.queue = (int *)take(sizeof(int) * n);
    L.bbest = (unsigned long long *)take(sizeof(unsigned long long) * n);
    L.sap_pred = (int *)take(sizeof(int) * n);
    L.frow[0] = (int *)take(sizeof(int) * n);
    L.frow[1] = (int *)take(sizeof(int) * n);
    L.fh[0] = (i64 *)take(sizeof(i64) * n);
    L.fh[1] = (i64 *)take(sizeof(i64) * n);
    L.fj0[0] = (int *)take(sizeof(int) * n);
    L.fj0[1] = (int *)take(sizeof(int) * n);
    L.fdl[0] = (i64 *)take(sizeof(i64) * n);
    L.fdl[1] = (i64 *)take(sizeof(i64) * n);
    L.blist[0] = (int *)take(sizeof(int) * n);
    L.blist[1] = (int *)take(sizeof(int) * n);
    L.ring = (SapSlot *)take(4 * sizeof(SapSlot));
    L.tflag = (int *)take(sizeof(int) * n);
    L.tlist = (int *)take(sizeof(int) * n);
    L.mark_row = (int *)take(sizeof(int) * n);
    L.mark_col = (int *)take(sizeof(int) * n);
    L.ufree = (i64 *)take(sizeof(i64) * n);
    L.mben = (i64 *)take(sizeof(i64) * n);
    return L;
}

int lap_chunks(int) { return 1; }

// Quantised benefit of one entry (see the header comment).
struct Quant {
    float mul;  // sgn * 2^(40 - e): an exact power-of-two scaling
    i64 qm;     // Qm
    int qsh;    // log2 Qm
};

__device__ __forceinline__ i64 benefit(float m, const Quant q) {
    return (i64)((unsigned long long)__float2ll_rn(m * q.mul) << q.qsh);  // round(m 2^(40-e)) * Qm
}

constexpr i64 kNegInf = LLONG_MIN / 4;

// ---------------------------------------------------------------- scans

// Ties between objects are broken by the key (j - i) mod n of bidder i: the first
// tied object at or after column i.  Rows with identical benefits then spread over
// a tied block of objects instead of all bidding for its lowest column (any tie
// rule leaves the auction exact).  j1 holds that key until tie_key_to_col.
__device__ __forceinline__ int col_to_tie_key(int j, int i, int n) { return j >= i ? j - i : j - i + n; }
__device__ __forceinline__ int tie_key_to_col(int k, int i, int n) { return k + i < n ? k + i : k + i - n; }

// Top-2 of v_j = a_ij - p_j over j = first, first + stride, ... < n, U loads in
// flight; j1 is the tie key of the best object of bidder `row`.
template <int U = 8>
__device__ __forceinline__ void top2_scan(const float *__restrict__ Mi, const i64 *__restrict__ price, int n,
                                          const Quant q, int first, int stride, int row, i64 &b1, i64 &b2,
                                          int &j1) {
    for (int base = first; base < n; base += U * stride) {
        float m[U];
        i64 pr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = base + u * stride;
            m[u] = j < n ? __ldg(Mi + j) : 0.0f;
            pr[u] = j < n ? price[j] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = base + u * stride;
            if (j < n) {
                const i64 v = benefit(m[u], q) - pr[u];
                const int k = col_to_tie_key(j, row, n);
                if (v > b1 || (v == b1 && k < j1)) {
                    b2 = b1;
                    b1 = v;
                    j1 = k;
                } else if (v > b2) {
                    b2 = v;
                }
            }
        }
    }
}

__device__ __forceinline__ void top2_merge(i64 &b1, i64 &b2, int &j1, i64 o1, i64 o2, int oj) {
    if (o1 > b1 || (o1 == b1 && oj < j1)) {
        b2 = max(b1, o2);
        b1 = o1;
        j1 = oj;
    } else {
        b2 = max(b2, o1);
    }
}

__device__ __forceinline__ void top2_warp(i64 &b1, i64 &b2, int &j1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const i64 o1 = __shfl_xor_sync(0xffffffffu, b1, o);
        const i64 o2 = __shfl_xor_sync(0xffffffffu, b2, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j1, o);
        top2_merge(b1, b2, j1, o1, o2, oj);
    }
}

// ---------------------------------------------------------------- auction

__global__ void k_lap_reset(int n, const LapBuffers L, DevState *st, int reset_prices) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        L.owner[j] = -1;
        L.assign[j] = -1;
        L.bbest[j] = 0ull;
        L.bwin[j] = INT_MAX;
        L.my_obj[j] = -1;
        if (reset_prices) L.price[j] = 0;
        L.blist[0][j] = j;  // every row bids in the first round of a phase
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->lap_unassigned = n;
        st->lap_nb[0] = n;
    }
}

// Appends the rows of the `want` lanes to a bidder list (one atomic per warp).
// The order of a list is run-dependent and does not matter: a Jacobi round's
// outcome depends only on the set of bidders (each object goes to its highest
// bid, the lowest row among equal bids), and the augmenting-path searches relax
// over their lists with ties broken by row index.
__device__ __forceinline__ void list_append(bool want, int row, int *dst, int *count) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    const int lane = threadIdx.x & 31, first = __ffs(m) - 1;
    int base = 0;
    if (lane == first) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, first);
    if (want) dst[base + __popc(m & ((1u << lane) - 1u))] = row;
}

// Jacobi bidding over the rows listed for this round (blist[cur], cnt entries):
// one CTA per bidding row (a row of 4n bytes is too long for one warp to stream at
// speed), CTAs blk, blk + nblk, ...
template <int THREADS>
__device__ __forceinline__ void bid_rows(const float *__restrict__ M, int n, const Quant q, const LapBuffers &L,
                                         i64 eps, int cur, int cnt, int blk, int nblk) {
    constexpr int NW = THREADS / 32;
    __shared__ i64 s_b1[NW], s_b2[NW];
    __shared__ int s_j1[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int idx = blk; idx < cnt; idx += nblk) {
        const int i = L.blist[cur][idx];
        i64 b1 = kNegInf, b2 = kNegInf;
        int j1 = INT_MAX;
        top2_scan(M + (long long)i * n, L.price, n, q, tid, THREADS, i, b1, b2, j1);
        top2_warp(b1, b2, j1);
        if (lane == 0) {
            s_b1[warp] = b1;
            s_b2[warp] = b2;
            s_j1[warp] = j1;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < NW; ++w) top2_merge(b1, b2, j1, s_b1[w], s_b2[w], s_j1[w]);
            j1 = tie_key_to_col(j1, i, n);
            const i64 inc = (b2 == kNegInf) ? eps : (b1 - b2) + eps;
            const i64 bid = L.price[j1] + inc;
            L.my_obj[i] = j1;
            L.my_bid[i] = bid;
            atomicMax(&L.bbest[j1], (unsigned long long)bid);  // bids are non-negative
        }
        __syncthreads();
    }
}

// The same bids with one warp per row (warps w, w + nwarps, ... of the grid): used
// while at least as many rows bid as the grid has warps, where the CTA-wide
// reductions and the bidding thread's serial step would stall a whole CTA per row.
__device__ __forceinline__ void bid_rows_warp(const float *__restrict__ M, int n, const Quant q, const LapBuffers &L,
                                              i64 eps, int cur, int cnt, int w, int nwarps) {
    const int lane = threadIdx.x & 31;
    for (int idx = w; idx < cnt; idx += nwarps) {
        const int i = L.blist[cur][idx];
        i64 b1 = kNegInf, b2 = kNegInf;
        int j1 = INT_MAX;
        top2_scan(M + (long long)i * n, L.price, n, q, lane, 32, i, b1, b2, j1);
        top2_warp(b1, b2, j1);
        if (lane == 0) {
            j1 = tie_key_to_col(j1, i, n);
            const i64 inc = (b2 == kNegInf) ? eps : (b1 - b2) + eps;
            const i64 bid = L.price[j1] + inc;
            L.my_obj[i] = j1;
            L.my_bid[i] = bid;
            atomicMax(&L.bbest[j1], (unsigned long long)bid);
        }
    }
}

// Each object's winner: the highest bid, the lowest row among equal ones
// (threads t, t + nthr, ... of the bidders).
__device__ __forceinline__ void win_rows(const LapBuffers &L, int cur, int cnt, int t, int nthr) {
    for (int k = t; k < cnt; k += nthr) {
        const int i = L.blist[cur][k];
        const int j = L.my_obj[i];
        if (L.bbest[j] == (unsigned long long)L.my_bid[i]) atomicMin(&L.bwin[j], i);
    }
}

// Winners take their objects at their bids and evict the previous holders; the
// evicted rows and the outbid bidders make up the next round's list.  (An outbid
// row reads bwin[j] while the winner may be resetting it: either value differs
// from the outbid row, so the outcome is the same.)  `t` and `nthr` cover whole
// warps (the list appends take warp ballots).
__device__ __forceinline__ void assign_rows(const LapBuffers &L, DevState *st, int cur, int cnt, int t, int nthr) {
    int *next = L.blist[cur ^ 1];
    int *ncount = &st->lap_nb[cur ^ 1];
    const int rounds = (cnt + nthr - 1) / nthr;  // uniform trip count for the warp ballots
    for (int r = 0; r < rounds; ++r) {
        const int k = r * nthr + t;
        int push = -1;
        if (k < cnt) {
            const int i = L.blist[cur][k];
            const int j = L.my_obj[i];
            if (L.bwin[j] == i) {
                const int old = L.owner[j];
                if (old >= 0) {
                    L.assign[old] = -1;
                    push = old;
                }
                L.owner[j] = i;
                L.assign[i] = j;
                L.price[j] = (i64)L.bbest[j];
                L.bbest[j] = 0ull;
                L.bwin[j] = INT_MAX;
            } else {
                push = i;
            }
        }
        list_append(push >= 0, push, next, ncount);
    }
}

// One Jacobi round as three launches (the form used without cooperative launch).
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_lap_bid(const float *__restrict__ M, int n, const Quant q,
                                                     const LapBuffers L, i64 eps, DevState *st, int cur) {
    const int cnt = st->lap_nb[cur];
    if (blockIdx.x == 0 && threadIdx.x == 0) st->lap_nb[cur ^ 1] = 0;  // the next round's list starts empty
    bid_rows<THREADS>(M, n, q, L, eps, cur, cnt, blockIdx.x, gridDim.x);
}

__global__ void k_lap_win(const LapBuffers L, const DevState *st, int cur) {
    win_rows(L, cur, st->lap_nb[cur], blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void k_lap_assign(const LapBuffers L, DevState *st, int cur) {
    assign_rows(L, st, cur, st->lap_nb[cur], blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// The Jacobi rounds of one eps phase in one cooperative launch: a round's bids,
// winners and assignments are separated by grid barriers, and the rounds go on
// while more than `threshold` rows bid, at most max_rounds of them, and until
// `stall` rounds in a row have not brought the number of bidders below its least
// value so far (rows chasing each other through near-tied objects, which the
// later steps place far sooner).  The list lengths are read after a barrier, so
// every block takes the same path.  Writes the rounds run and the index of the
// list left to bid into st->lap_head.
constexpr int LAP_HEAD_THREADS = 1024;
static_assert(offsetof(DevState, lap_head) == offsetof(DevState, lap_nb) + 2 * sizeof(int),
              "the head's report is read with the list lengths in one copy");
__global__ void __launch_bounds__(LAP_HEAD_THREADS, 1)
    k_lap_head(const float *__restrict__ M, int n, const Quant q, const LapBuffers L, i64 eps, DevState *st,
               int cur, int max_rounds, int threshold, int stall) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    volatile int *nb = st->lap_nb;
    int r = 0, least = INT_MAX, since = 0;
    for (; r < max_rounds; ++r) {
        const int cnt = nb[cur];
        if (cnt <= threshold) break;
        if (cnt < least) {
            least = cnt;
            since = 0;
        } else if (++since >= stall) {
            break;
        }
        if (t == 0) nb[cur ^ 1] = 0;  // read by the assignments, two barriers on
        if (cnt >= nthr / 32)
            bid_rows_warp(M, n, q, L, eps, cur, cnt, t >> 5, nthr >> 5);
        else
            bid_rows<LAP_HEAD_THREADS>(M, n, q, L, eps, cur, cnt, blockIdx.x, gridDim.x);
        grid.sync();
        win_rows(L, cur, cnt, t, nthr);
        grid.sync();
        assign_rows(L, st, cur, cnt, t, nthr);
        grid.sync();
        cur ^= 1;
    }
    if (t == 0) {
        st->lap_head[0] = r;
        st->lap_head[1] = cur;
    }
}

// Appends the unassigned rows to queue[*s_tail ...] in increasing row order (a
// block-wide ordered compaction: warp ballots, then the warps' counts in order),
// so that the sequential bidding below visits the rows in the same order on every
// run.  The order decides which of several tied optima the auction settles on.
// Every thread of the block calls it; s_cnt holds 32 ints of shared memory.
__device__ __forceinline__ void queue_free_rows_in_order(const int *__restrict__ assign, int n,
                                                         int *__restrict__ queue, int *s_tail, int *s_cnt) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + tid;
        const bool fr = i < n && assign[i] < 0;
        const unsigned m = __ballot_sync(0xffffffffu, fr);
        if (lane == 0) s_cnt[warp] = __popc(m);
        __syncthreads();
        int off = *s_tail;
        for (int w = 0; w < warp; ++w) off += s_cnt[w];
        if (fr) queue[off + __popc(m & ((1u << lane) - 1u))] = i;
        __syncthreads();
        if (tid == 0) {
            int add = 0;
            for (int w = 0; w < nwarps; ++w) add += s_cnt[w];
            *s_tail += add;
        }
        __syncthreads();
    }
}

// Gauss-Seidel tail of a phase: one CTA serves the unassigned rows one at a
// time; a bid takes its object at once and the evicted holder joins the queue
// (a ring of n slots: a row is queued only while unassigned).  All threads scan
// the bidder's row.  At most max_bids bids; stops early once `stall` bids in a
// row have not shortened the queue below its shortest length so far.
__global__ void __launch_bounds__(1024) k_lap_tail(const float *__restrict__ M, int n, const Quant q,
                                                   const LapBuffers L, i64 eps, long long max_bids, long long stall,
                                                   DevState *st) {
    __shared__ i64 s_b1[32], s_b2[32];
    __shared__ int s_j1[32];
    __shared__ int s_head, s_tail, s_stop;
    __shared__ int s_cnt[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    if (tid == 0) {
        s_head = 0;
        s_tail = 0;
        s_stop = 0;
    }
    __syncthreads();
    queue_free_rows_in_order(L.assign, n, L.queue, &s_tail, s_cnt);
    long long bids = 0, since = 0;
    int qmin = s_tail - s_head;
    while (true) {
        if (s_head == s_tail || s_stop) break;
        const int i = L.queue[s_head % n];
        i64 b1 = kNegInf, b2 = kNegInf;
        int j1 = INT_MAX;
        top2_scan(M + (long long)i * n, L.price, n, q, tid, blockDim.x, i, b1, b2, j1);
        top2_warp(b1, b2, j1);
        if (lane == 0) {
            s_b1[warp] = b1;
            s_b2[warp] = b2;
            s_j1[warp] = j1;
        }
        __syncthreads();
        if (warp == 0) {
            b1 = lane < nwarps ? s_b1[lane] : kNegInf;
            b2 = lane < nwarps ? s_b2[lane] : kNegInf;
            j1 = lane < nwarps ? s_j1[lane] : INT_MAX;
            top2_warp(b1, b2, j1);
            if (lane == 0) {
                j1 = tie_key_to_col(j1, i, n);
                const i64 inc = (b2 == kNegInf) ? eps : (b1 - b2) + eps;
                L.price[j1] += inc;
                const int old = L.owner[j1];
                L.owner[j1] = i;
                L.assign[i] = j1;
                ++s_head;
                if (old >= 0) {
                    L.assign[old] = -1;
                    L.queue[s_tail % n] = old;
                    ++s_tail;
                }
                const int len = s_tail - s_head;
                if (len < qmin) {
                    qmin = len;
                    since = 0;
                } else {
                    ++since;
                }
                if (++bids >= max_bids || since >= stall) s_stop = 1;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        st->lap_unassigned = s_tail - s_head;
        st->lap_bids += bids;
    }
}

// The same Gauss-Seidel tail spread over a cluster of 8 CTAs: CTA r owns the
// columns [r W, (r + 1) W) and keeps their prices and owners in its shared
// memory; for each bid every CTA scans its part of the bidder's row, the leader
// (rank 0) merges the 8 partial top-2s it receives through distributed shared
// memory, updates the winning column's price and owner in the owner CTA, the
// queue and assign[], and broadcasts the next bidder.  Two cluster barriers per
// bid; each CTA prefetches its part of the next queued row into L2 while it
// scans the current one.
constexpr int LAP_CLUSTER = 8;

__global__ void __cluster_dims__(LAP_CLUSTER, 1, 1) __launch_bounds__(256)
    k_lap_tail_cluster(const float *__restrict__ M, int n, const Quant q, const LapBuffers L, i64 eps,
                       long long max_bids, long long stall, DevState *st) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int W = (n + LAP_CLUSTER - 1) / LAP_CLUSTER;
    const int c0 = min(n, rank * W), c1 = min(n, c0 + W);
    extern __shared__ unsigned char lap_sm[];
    i64 *price_s = reinterpret_cast<i64 *>(lap_sm);
    int *owner_s = reinterpret_cast<int *>(price_s + W);
    __shared__ i64 s_wb1[8], s_wb2[8];
    __shared__ int s_wj1[8];
    __shared__ i64 s_b1[LAP_CLUSTER], s_b2[LAP_CLUSTER];  // leader: partial results of the cluster
    __shared__ int s_j1[LAP_CLUSTER];
    __shared__ int s_next;                                // next bidder (-1: stop), set by the leader
    __shared__ int s_pref;                                // the bidder after it, if already queued (-1: none)
    __shared__ int s_head, s_tail;
    __shared__ long long s_bids, s_since;
    __shared__ int s_qmin;

    for (int j = c0 + tid; j < c1; j += blockDim.x) {
        price_s[j - c0] = L.price[j];
        owner_s[j - c0] = L.owner[j];
    }
    cluster.sync();  // every CTA of the cluster is running before any shared memory of another is touched
    if (rank == 0) {
        if (tid == 0) {
            s_head = 0;
            s_tail = 0;
            s_bids = 0;
        }
        __syncthreads();
        __shared__ int s_cnt[32];
        queue_free_rows_in_order(L.assign, n, L.queue, &s_tail, s_cnt);
        if (tid == 0) {
            s_qmin = s_tail - s_head;
            s_since = 0;
            const bool more = s_head != s_tail && max_bids > 0 && stall > 0;
            const int nx = more ? L.queue[s_head % n] : -1;
            const int np = (more && s_tail - s_head > 1) ? L.queue[(s_head + 1) % n] : -1;
            for (int r = 0; r < LAP_CLUSTER; ++r) {
                *cluster.map_shared_rank(&s_next, r) = nx;
                *cluster.map_shared_rank(&s_pref, r) = np;
            }
        }
    }
    cluster.sync();
    while (true) {
        const int i = s_next;
        if (i < 0) break;  // uniform over the cluster: the leader wrote the same value everywhere
        const int pf = s_pref;
        if (pf >= 0) {  // the likely next bidder: pull this CTA's part of its row into L2
            const float *row = M + (long long)pf * n;
            for (int j = c0 + tid * 32; j < c1; j += blockDim.x * 32)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(row + j));
        }
        i64 b1 = kNegInf, b2 = kNegInf;
        int j1 = INT_MAX;
        const float *Mi = M + (long long)i * n;
        int j = c0 + tid;
        for (; j + 3 * (int)blockDim.x < c1; j += 4 * blockDim.x) {  // four loads in flight per thread
            float v4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v4[u] = __ldg(Mi + j + u * blockDim.x);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int jj = j + u * blockDim.x;
                const i64 v = benefit(v4[u], q) - price_s[jj - c0];
                const int k = col_to_tie_key(jj, i, n);
                if (v > b1 || (v == b1 && k < j1)) {
                    b2 = b1;
                    b1 = v;
                    j1 = k;
                } else if (v > b2) {
                    b2 = v;
                }
            }
        }
        for (; j < c1; j += blockDim.x) {
            const i64 v = benefit(__ldg(Mi + j), q) - price_s[j - c0];
            const int k = col_to_tie_key(j, i, n);
            if (v > b1 || (v == b1 && k < j1)) {
                b2 = b1;
                b1 = v;
                j1 = k;
            } else if (v > b2) {
                b2 = v;
            }
        }
        top2_warp(b1, b2, j1);
        if (lane == 0) {
            s_wb1[warp] = b1;
            s_wb2[warp] = b2;
            s_wj1[warp] = j1;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nwarps; ++w) top2_merge(b1, b2, j1, s_wb1[w], s_wb2[w], s_wj1[w]);
            *cluster.map_shared_rank(&s_b1[rank], 0) = b1;
            *cluster.map_shared_rank(&s_b2[rank], 0) = b2;
            *cluster.map_shared_rank(&s_j1[rank], 0) = j1;
        }
        cluster.sync();
        if (rank == 0 && tid == 0) {
            b1 = s_b1[0];
            b2 = s_b2[0];
            j1 = s_j1[0];
            for (int r = 1; r < LAP_CLUSTER; ++r) top2_merge(b1, b2, j1, s_b1[r], s_b2[r], s_j1[r]);
            j1 = tie_key_to_col(j1, i, n);
            const i64 inc = (b2 == kNegInf) ? eps : (b1 - b2) + eps;
            const int ro = j1 / W, jl = j1 - ro * W;
            i64 *pp = cluster.map_shared_rank(price_s, ro);
            int *po = cluster.map_shared_rank(owner_s, ro);
            pp[jl] += inc;
            const int old = po[jl];
            po[jl] = i;
            L.assign[i] = j1;
            ++s_head;
            if (old >= 0) {
                L.assign[old] = -1;
                L.queue[s_tail % n] = old;
                ++s_tail;
            }
            ++s_bids;
            const int len = s_tail - s_head;
            if (len < s_qmin) {
                s_qmin = len;
                s_since = 0;
            } else {
                ++s_since;
            }
            const bool more = s_head != s_tail && s_bids < max_bids && s_since < stall;
            const int nx = more ? L.queue[s_head % n] : -1;
            const int np = (more && s_tail - s_head > 1) ? L.queue[(s_head + 1) % n] : -1;
            for (int r = 0; r < LAP_CLUSTER; ++r) {
                *cluster.map_shared_rank(&s_next, r) = nx;
                *cluster.map_shared_rank(&s_pref, r) = np;
            }
        }
        cluster.sync();
    }
    for (int j = c0 + tid; j < c1; j += blockDim.x) {
        L.price[j] = price_s[j - c0];
        L.owner[j] = owner_s[j - c0];
    }
    if (rank == 0 && tid == 0) {
        st->lap_unassigned = s_tail - s_head;
        st->lap_bids += s_bids;
    }
}

// ---------------------------------------------------------------- shortest augmenting paths

// Slack of every assigned row, delta_i = max_j (a_ij - p_j) - (a_i,j_i - p_j_i) >= 0,
// into my_bid[i], and its object into my_obj[i] (the pairs whose benefit a~ adds
// delta_i); every unassigned row gets the potential u_i = -max_j (a_ij - p_j) in
// ufree[i] and is listed in queue[0, lap_free) (in a run-dependent order, which the
// searches do not depend on: see list_append).  One CTA per row.
__global__ void __launch_bounds__(256) k_lap_sap_prep(const float *__restrict__ M, int n, const Quant q,
                                                      const LapBuffers L, DevState *st) {
    __shared__ i64 s_b1[8], s_b2[8];
    __shared__ int s_j1[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int ji = L.assign[i];
        const float *Mi = M + (long long)i * n;
        i64 b1 = kNegInf, b2 = kNegInf;
        int j1 = INT_MAX;
        top2_scan(Mi, L.price, n, q, tid, blockDim.x, i, b1, b2, j1);
        top2_warp(b1, b2, j1);
        if (lane == 0) {
            s_b1[warp] = b1;
            s_b2[warp] = b2;
            s_j1[warp] = j1;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nwarps; ++w) top2_merge(b1, b2, j1, s_b1[w], s_b2[w], s_j1[w]);
            if (ji < 0) {
                L.my_obj[i] = -1;
                L.my_bid[i] = 0;
                L.ufree[i] = -b1;
                L.queue[atomicAdd(&st->lap_free, 1)] = i;
            } else {
                const i64 a = benefit(Mi[ji], q);
                const i64 d = b1 - (a - L.price[ji]);
                L.my_obj[i] = ji;
                L.my_bid[i] = d > 0 ? d : 0;
                L.mben[i] = a + (d > 0 ? d : 0);
            }
        }
        __syncthreads();
    }
}

constexpr int SAP_SLOTS = 256;                  // column slots per CTA (each CPT columns)
constexpr int SAP_GROUPS = 2;                   // row groups sharing the slots in a relaxation
constexpr int SAP_THREADS = SAP_SLOTS * SAP_GROUPS;
constexpr int SAP_STAGE = 512;                  // frontier entries staged in shared memory at a time
constexpr int SAP_STEP = 128;                   // default: open columns settled per parallel step (more on ties)
constexpr i64 kPosInf = LLONG_MAX / 4;

// Reduced cost of (i, j) in the minimisation form: c~_ij = -a~_ij, the benefit of
// the pair (i, j0_i) raised by the row's slack delta_i.
__device__ __forceinline__ i64 sap_cost(float m, const Quant q, int j, int j0, i64 delta) {
    return -(benefit(m, q) + (j == j0 ? delta : 0));
}

// Block-wide minima of two values at once; valid in thread 0.
__device__ __forceinline__ void block_min2(i64 &x, i64 &y, i64 *sx, i64 *sy) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x = min(x, (i64)__shfl_xor_sync(0xffffffffu, x, o));
        y = min(y, (i64)__shfl_xor_sync(0xffffffffu, y, o));
    }
    if (lane == 0) {
        sx[warp] = x;
        sy[warp] = y;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            x = min(x, sx[w]);
            y = min(y, sy[w]);
        }
    __syncthreads();
}

// Shortest augmenting paths for the rows listed in queue[0, lap_free), on the whole
// GPU (a cooperative launch; every thread owns CPT columns, j = global thread +
// c * total threads, and keeps their dual v_j = -p_j, label d_j, predecessor row,
// owner and state -- open, in the current bucket, or closed -- in registers).
// Hungarian method in Jonker-Volgenant's form: each search starts from all free
// rows at once (row potentials u_i = min_j (c~_ij - v_j) from the prep kernel;
// they stay feasible since the duals v only fall) and runs a label-correcting
// Dijkstra that settles up to step_cols columns per parallel step: the open columns
// (free columns aside) with the least labels, chosen by a histogram of the labels
// gathered in the previous step.  Their rows are scanned in parallel (each thread
// relaxes its columns over the listed rows); a settled column whose label still
// falls reopens.  Labels only fall from settled labels by non-negative reduced
// costs, so once the least free-column label d_t is at most every open label, all
// labels below d_t are final: the settled columns' duals move by d_j - d_t, which
// makes every shortest augmenting path tight, and the leader CTA flips the paths to
// all free columns of label d_t (lowest column first) that share no row or column
// with a path already flipped -- several rows per search where the matrix has
// ties.  Control flow depends only on values read after a grid barrier, so every
// block takes the same path.  At most max_scans row scans per launch; rows left
// over stay unassigned (lap_unassigned reports them).
template <int CPT>
__global__ void __launch_bounds__(SAP_THREADS) k_lap_sap_grid(const float *__restrict__ M, int n, const Quant q,
                                                              const LapBuffers L, int step_cols, long long max_scans,
                                                              DevState *st) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    const int tid = threadIdx.x, lane = tid & 31;
    const int slot = tid % SAP_SLOTS, grp = tid / SAP_SLOTS;
    const bool leader = blockIdx.x == 0 && tid == 0;
    __shared__ i64 s_x[SAP_THREADS / 32], s_x2[SAP_THREADS / 32];
    __shared__ int s_scan[SAP_THREADS];
    __shared__ int s_hist[64];
    __shared__ long long s_tau, s_nbase;
    __shared__ i64 s_v[SAP_SLOTS * CPT];                      // duals of the CTA's columns
    __shared__ i64 s_cd[SAP_GROUPS - 1][SAP_SLOTS];           // candidates of groups 1.. for one slot set
    __shared__ int s_cr[SAP_GROUPS - 1][SAP_SLOTS];
    __shared__ int s_row[SAP_STAGE], s_j0[SAP_STAGE];         // staged frontier entries
    __shared__ i64 s_h[SAP_STAGE], s_dl[SAP_STAGE];

    // Group 0 owns the CTA's columns (state in registers); groups 1.. only help to
    // scan the frontier rows of a relaxation.  rcol: the column of each slot.
    int col[CPT], rcol[CPT], pred[CPT], own[CPT];
    i64 v[CPT], d[CPT];
    unsigned char stt[CPT];  // 0 open, 2 settled
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        rcol[c] = blockIdx.x * (SAP_SLOTS * CPT) + c * SAP_SLOTS + slot;
        col[c] = grp == 0 ? rcol[c] : n;  // n: no column
        const bool ok = col[c] < n;
        v[c] = ok ? -L.price[col[c]] : 0;
        own[c] = ok ? L.owner[col[c]] : -1;
        d[c] = kPosInf;
        pred[c] = -1;
        stt[c] = 2;
        if (grp == 0) s_v[c * SAP_SLOTS + slot] = v[c];
    }
    // Reduction slots: the one of epoch e (e = barriers passed) is written during e,
    // read during e + 1 and reset by the leader during e + 2 (ring of 4).
    int e = 0;
    if (leader)
        for (int k = 0; k < 4; ++k) {
            L.ring[k].minv = kPosInf;
            L.ring[k].tmin = kPosInf;
            L.ring[k].count = 0;
        }
    if (blockIdx.x == 0 && tid < 64)
        for (int k = 0; k < 4; ++k) L.ring[k].hist[tid] = 0;
    auto barrier = [&]() {
        grid.sync();
        ++e;
        SapSlot &z = L.ring[(e + 2) & 3];
        if (leader) {
            z.minv = kPosInf;
            z.tmin = kPosInf;
            z.count = 0;
        }
        if (blockIdx.x == 0 && tid < 64) z.hist[tid] = 0;
    };
    auto cur = [&]() -> SapSlot & { return L.ring[e & 3]; };
    auto prev = [&]() -> const SapSlot & { return L.ring[(e + 3) & 3]; };
    // appends (row, h) to this epoch's frontier list, one atomic per warp
    auto append = [&](bool want, int row, i64 h) {
        const unsigned m = __ballot_sync(0xffffffffu, want);
        if (!m) return;
        int base = 0;
        const int first = __ffs(m) - 1;
        if (lane == first) base = atomicAdd(&cur().count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, first);
        if (want) {
            const int k = base + __popc(m & ((1u << lane) - 1u));
            const int j0 = L.my_obj[row];
            L.frow[e & 1][k] = row;
            L.fh[e & 1][k] = h;
            L.fj0[e & 1][k] = j0;
            L.fdl[e & 1][k] = j0 >= 0 ? L.my_bid[row] : 0;
        }
    };
    // label offset h_i = d_j - (c~_ij - v_j) of the row owning column j (c~_ij = -mben[i])
    auto row_offset = [&](int c) -> i64 { return d[c] + L.mben[own[c]] + v[c]; };
    // statistics of the open columns for the next step, into this epoch's slot: the
    // least free-column label, the least open non-free label and the histogram of
    // the open non-free labels by bit length of (label - base)
    auto step_stats = [&](i64 base) {
        if (tid < 64) s_hist[tid] = 0;
        i64 lt = kPosInf, lm = kPosInf;
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            if (col[c] >= n || stt[c] != 0) continue;
            if (own[c] < 0) {
                if (d[c] < lt) lt = d[c];
            } else {
                if (d[c] < lm) lm = d[c];
                const long long x = d[c] - base;  // >= 0 (base is a lower bound)
                atomicAdd(&s_hist[x <= 0 ? 0 : min(63, 64 - __clzll(x))], 1);
            }
        }
        block_min2(lt, lm, s_x, s_x2);
        if (tid == 0) {
            atomicMin(&cur().tmin, lt);
            atomicMin(&cur().minv, lm);
        }
        if (tid < 64 && s_hist[tid]) atomicAdd(&cur().hist[tid], s_hist[tid]);
    };
    // the widest bound tau = base + 2^b - 1 taking in at most step_cols open non-free
    // columns (never none), capped below the least free label; nbase = the lower edge
    // of the lowest non-empty histogram bin, a lower bound of every label from now on
    auto choose_tau = [&](i64 base, i64 tmin, i64 *tau, i64 *nbase) {
        if (tid < 64) s_hist[tid] = prev().hist[tid];  // one load per thread, not 64 in a row
        __syncthreads();
        if (tid == 0) {
            const int *h = s_hist;
            int cum = 0, best = -1, first = -1;
            for (int b = 0; b < 64; ++b) {
                cum += h[b];
                if (h[b] && first < 0) first = b;
                if (cum <= step_cols) best = b;
            }
            if (first < 0) first = 0;
            if (best < first) best = first;
            const i64 w = best >= 62 ? kPosInf : (1LL << best) - 1;
            i64 t = w >= kPosInf - 1 - base ? kPosInf - 1 : base + w;
            if (t > tmin - 1) t = tmin - 1;
            s_tau = t;
            s_nbase = base + (first > 0 ? (1LL << (first - 1)) : 0);
        }
        __syncthreads();
        *tau = s_tau;
        *nbase = s_nbase;
    };
    // relaxes the CTA's columns over rows[0, cnt) (the free rows when hs is null:
    // offset -ufree[row], no boost; else the list's offsets, boosted columns and
    // boosts).  The entries are staged in shared memory; row group g scans entries
    // g, g + SAP_GROUPS, ... for every slot, and group 0 merges the groups' best
    // candidates into the labels; ch[c] says whether d[c] fell.
    auto relax = [&](const int *rows_in, const i64 *hs, const int *j0s, const i64 *dls, int cnt, bool *ch) {
        constexpr int RU = CPT >= 8 ? 2 : 16 / CPT;  // rows in flight: 16 loads per thread
        i64 bd[CPT];
        int br[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            bd[c] = kPosInf;
            br[c] = INT_MAX;
        }
        i64 vv[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) vv[c] = s_v[c * SAP_SLOTS + slot];
        for (int s0 = 0; s0 < cnt; s0 += SAP_STAGE) {
            const int len = min(SAP_STAGE, cnt - s0);
            __syncthreads();  // the previous stage is consumed
            for (int k = tid; k < len; k += SAP_THREADS) {
                const int row = rows_in[s0 + k];
                s_row[k] = row;
                s_h[k] = hs ? hs[s0 + k] : -L.ufree[row];
                s_j0[k] = hs ? j0s[s0 + k] : -1;
                s_dl[k] = hs ? dls[s0 + k] : 0;
            }
            __syncthreads();
            for (int r0 = grp; r0 < len; r0 += RU * SAP_GROUPS) {
                float m[RU][CPT];
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int r = r0 + u * SAP_GROUPS;
#pragma unroll
                    for (int c = 0; c < CPT; ++c)
                        m[u][c] = (r < len && rcol[c] < n) ? __ldg(M + (long long)s_row[r] * n + rcol[c]) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < RU; ++u) {
                    const int r = r0 + u * SAP_GROUPS;
                    if (r >= len) break;
                    const i64 h = s_h[r];
                    const int j0 = s_j0[r], row = s_row[r];
                    const i64 dl = s_dl[r];
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        const i64 nd = h + sap_cost(m[u][c], q, rcol[c], j0, dl) - vv[c];
                        if (nd < bd[c] || (nd == bd[c] && row < br[c])) {
                            bd[c] = nd;
                            br[c] = row;
                        }
                    }
                }
            }
        }
        // merge the groups' candidates, one column set at a time
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            if (grp > 0) {
                s_cd[grp - 1][slot] = bd[c];
                s_cr[grp - 1][slot] = br[c];
            }
            __syncthreads();
            if (grp == 0 && col[c] < n) {
                i64 b = bd[c];
                int r = br[c];
#pragma unroll
                for (int g = 0; g < SAP_GROUPS - 1; ++g) {
                    const i64 od = s_cd[g][slot];
                    const int orow = s_cr[g][slot];
                    if (od < b || (od == b && orow < r)) {
                        b = od;
                        r = orow;
                    }
                }
                if (b < d[c]) {
                    d[c] = b;
                    pred[c] = r;
                    ch[c] = true;
                }
            }
            __syncthreads();
        }
    };
    barrier();

    const int nfree0 = *(volatile int *)&st->lap_free;
    int nfree = nfree0;  // rows still free, listed in queue[0, nfree) (kept up to date by the leader)
    long long scans = 0;
    int searches = 0;
    bool aborted = false;
    while (nfree > 0 && !aborted) {
        ++searches;
        // labels from all free rows at once, then the statistics for the first step
        i64 base = 0;  // a lower bound of every open label (all labels are reduced costs, >= 0)
        {
            bool ch[CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                ch[c] = false;
                d[c] = kPosInf;
                pred[c] = -1;
                stt[c] = col[c] < n ? 0 : 2;
            }
            relax(L.queue, nullptr, nullptr, nullptr, nfree, ch);
            scans += nfree;
            step_stats(base);
        }
        barrier();
        i64 dt = 0;
        bool found = false;
        while (true) {
            // (1) the free columns' least label ends the search once no open non-free
            // column lies below it; else the least open non-free labels are settled
            const i64 tmin = prev().tmin, minv = prev().minv;
            if (tmin <= minv) {
                if (tmin >= kPosInf) {
                    aborted = true;  // no column reachable: cannot happen while a row is free
                } else {
                    dt = tmin;
                    found = true;
                }
                break;
            }
            i64 tau, nbase;
            choose_tau(base, tmin, &tau, &nbase);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const bool in = col[c] < n && stt[c] == 0 && own[c] >= 0 && d[c] <= tau;
                if (in) stt[c] = 2;
                append(in, in ? own[c] : 0, in ? row_offset(c) : 0);
            }
            base = nbase;
            barrier();
            // (2) scan the settled columns' rows; settled columns whose label falls reopen
            const int cnt = prev().count;
            scans += cnt;
            if (scans > max_scans) {  // uniform: every block adds the same counts
                aborted = true;
                break;
            }
            bool ch[CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) ch[c] = false;
            const int pb = (e + 1) & 1;
            relax(L.frow[pb], L.fh[pb], L.fj0[pb], L.fdl[pb], cnt, ch);
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (ch[c] && stt[c] == 2) stt[c] = 0;
            step_stats(base);
            barrier();
        }
        if (aborted || !found) {
            aborted = true;
            break;
        }
        // duals of the settled columns; predecessors and the targets (free columns of
        // label d_t) for the leader CTA
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (col[c] < n) {
                if (stt[c] == 2 && d[c] < dt) {
                    v[c] += d[c] - dt;
                    s_v[c * SAP_SLOTS + slot] = v[c];
                }
                L.sap_pred[col[c]] = pred[c];
                if (own[c] < 0 && d[c] == dt) L.tflag[col[c]] = searches;
            }
        barrier();
        if (blockIdx.x == 0) {
            // targets in column order: block-wide compaction of the flagged columns
            const int chunk = (n + SAP_THREADS - 1) / SAP_THREADS;
            const int j0 = tid * chunk, j1 = min(n, j0 + chunk);
            int cntf = 0;
#pragma unroll 8
            for (int j = j0; j < j1; ++j) cntf += __ldcg(L.tflag + j) == searches;
            s_scan[tid] = cntf;
            __syncthreads();
            for (int o = 1; o < SAP_THREADS; o <<= 1) {  // inclusive scan
                const int add = tid >= o ? s_scan[tid - o] : 0;
                __syncthreads();
                s_scan[tid] += add;
                __syncthreads();
            }
            int at = s_scan[tid] - cntf;
            for (int j = j0; j < j1; ++j)
                if (L.tflag[j] == searches) L.tlist[at++] = j;
            const int ntarg = s_scan[SAP_THREADS - 1];
            __syncthreads();
            if (tid == 0) {
                const int stamp = searches;
                int placed = 0;
                for (int k = 0; k < ntarg; ++k) {
                    // check the path: no row or column already used by this search
                    bool ok = true;
                    int j = L.tlist[k];
                    for (int hop = 0; hop <= n; ++hop) {
                        const int i = L.sap_pred[j];
                        if (i < 0 || i >= n || L.mark_col[j] == stamp || L.mark_row[i] == stamp) {
                            ok = false;
                            break;
                        }
                        const int jn = L.assign[i];
                        if (jn < 0) break;
                        j = jn;
                    }
                    if (!ok) continue;
                    j = L.tlist[k];
                    for (int hop = 0; hop <= n; ++hop) {
                        const int i = L.sap_pred[j];
                        const int jn = L.assign[i];
                        L.mark_col[j] = stamp;
                        L.mark_row[i] = stamp;
                        L.owner[j] = i;
                        L.assign[i] = j;
                        L.mben[i] = -sap_cost(M[(long long)i * n + j], q, j, L.my_obj[i], L.my_bid[i]);
                        if (jn < 0) break;
                        j = jn;
                    }
                    ++placed;
                }
                // the free rows that are left
                int m = 0;
                for (int k = 0; k < nfree; ++k) {
                    const int i = L.queue[k];
                    if (L.assign[i] < 0) L.queue[m++] = i;
                }
                if (placed == 0) m = -1;  // no path could be flipped: inconsistent state, stop
                st->lap_free = m;
            }
        }
        barrier();
        const int left = *(volatile int *)&st->lap_free;
        if (left < 0) {
            aborted = true;
            break;
        }
        nfree = left;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (col[c] < n) own[c] = L.owner[col[c]];
    }
#pragma unroll
    for (int c = 0; c < CPT; ++c)
        if (col[c] < n) {
            L.price[col[c]] = -v[c];
            L.owner[col[c]] = own[c];
        }
    if (leader) {
        st->lap_unassigned = aborted ? (nfree > 0 ? nfree : nfree0) : nfree;
        st->lap_pops += scans;
        st->lap_epochs += e;
    }
}

// Completes a partial assignment: each unassigned row (in row order) takes the
// free object of largest a_ij - p_j.  One CTA; used only when the last phase ran
// out of its bid budget.
__global__ void __launch_bounds__(1024) k_lap_fill(const float *__restrict__ M, int n, const Quant q,
                                                   const LapBuffers L, DevState *st) {
    __shared__ i64 s_b[32];
    __shared__ int s_j[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int i = 0; i < n; ++i) {
        if (L.assign[i] >= 0) continue;  // uniform: every thread reads the same word
        const float *Mi = M + (long long)i * n;
        i64 b = kNegInf;
        int jb = INT_MAX;
        for (int j = tid; j < n; j += blockDim.x) {
            if (L.owner[j] >= 0) continue;
            const i64 v = benefit(Mi[j], q) - L.price[j];
            if (v > b) {
                b = v;
                jb = j;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const i64 ob = __shfl_xor_sync(0xffffffffu, b, o);
            const int oj = __shfl_xor_sync(0xffffffffu, jb, o);
            if (ob > b || (ob == b && oj < jb)) {
                b = ob;
                jb = oj;
            }
        }
        if (lane == 0) {
            s_b[warp] = b;
            s_j[warp] = jb;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nwarps; ++w)
                if (s_b[w] > s_b[0] || (s_b[w] == s_b[0] && s_j[w] < s_j[0])) {
                    s_b[0] = s_b[w];
                    s_j[0] = s_j[w];
                }
            const int j = s_j[0];
            if (j >= 0 && j < n) {
                L.owner[j] = i;
                L.assign[i] = j;
            } else if (!st->error) {
                st->error = GOAT_ERR_NOT_CONVERGED;  // no free object left: inconsistent state, skip
            }
        }
        __syncthreads();
    }
    if (tid == 0) st->lap_unassigned = 0;
}

// Duality gap of the quantised problem, sum_i (max_j (a_ij - p_j) - (a_i,perm i - p_perm i)):
// each row's term (>= 0) into term[i], one warp per row; k_lap_gap_sum adds them.
__global__ void __launch_bounds__(256) k_lap_gap(const float *__restrict__ M, int n, const Quant q,
                                                 const LapBuffers L, i64 *__restrict__ term) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = gw; i < n; i += nw) {
        i64 b1 = kNegInf, b2 = kNegInf;
        int j1 = INT_MAX;
        const float *Mi = M + (long long)i * n;
        top2_scan(Mi, L.price, n, q, lane, 32, i, b1, b2, j1);
        top2_warp(b1, b2, j1);
        if (lane == 0) {
            const int j = L.assign[i];
            term[i] = (j >= 0 && j < n) ? b1 - (benefit(Mi[j], q) - L.price[j]) : 0;
        }
    }
}

// *out = sum_i term[i] as a double, in a fixed order (thread t adds rows t, t + 1024,
// ... in turn, then the threads' sums are combined by a fixed tree): the same value
// on every run.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_lap_gap_sum(const i64 *__restrict__ term, int n, double *out) {
    __shared__ double s[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += (double)term[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        *out = t;
    }
}

// sum_i M[i][perm i] in FP64 in row order (the order the oracle uses); one block.
__global__ void k_assignment_cost(const float *__restrict__ M, int n, const int *__restrict__ perm, double *out) {
    __shared__ double buf[1024];
    double acc = 0.0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const int pi = (i < n) ? perm[i] : -1;
        buf[threadIdx.x] = (pi >= 0 && pi < n) ? (double)M[(long long)i * n + pi] : 0.0;
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

static int poll_int(const int *dev, int *pinned, cudaStream_t s) {
    cudaMemcpyAsync(pinned, dev, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return *pinned;
}

void lap_default_control(LapControl *c) {
    c->max_rounds = 1 << 20;
    c->head_rounds = 256;
    c->tail_bids = -1;
    c->tail_stall = -1;
    c->sap_pops = -1;
    c->sap_step = -1;
    c->head_stall = 16;
    c->sap_every_phase = 0;
}

// Runs the projection.  lap_ws must hold lap_bytes(n, ...) bytes; cost_dev
// points at >= 2 doubles (the assignment cost, then the gap accumulator).
int lap_solve(const float *M, int n, int maximize, int32_t *perm_out, void *lap_ws, DevState *st,
              const LapControl &ctl, double *cost_dev, int *host_pinned, double *gap_host, LapReport *rep,
              cudaStream_t s) {
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
    LapReport R{};
    LapBuffers L = carve(lap_ws, n);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g1 = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), sms * 8));
    const int gbid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 8), sms * 16));
    const int growb = (int)std::max<int64_t>(1, std::min<int64_t>(n, sms * 8));  // one CTA per bidding row

    // scale: max |M| < C' = 2^e
    unsigned *cbits = reinterpret_cast<unsigned *>(&st->gmax_next);
    cudaMemsetAsync(cbits, 0, sizeof(unsigned), s);
    absmax(M, (long long)n * n, cbits, s);
    cudaMemcpyAsync(host_pinned, cbits, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return GOAT_ERR_CUDA;
    float Cf;
    std::memcpy(&Cf, host_pinned, sizeof(float));
    cudaMemsetAsync(cbits, 0, sizeof(unsigned), s);
    if (!(Cf == Cf) || std::isinf(Cf)) return GOAT_ERR_NAN;
    int e = 0;
    if (Cf > 0.0f) std::frexp((double)Cf, &e);  // Cf < 2^e
    Quant q;
    int qbits = 1;
    while ((1LL << qbits) <= (long long)n) ++qbits;
    const int bq = std::min(40, 58 - qbits);  // keeps |a_int| and every price far below 2^63
    q.mul = (float)std::ldexp(maximize ? 1.0 : -1.0, bq - e);
    q.qm = 1LL << qbits;
    q.qsh = qbits;
    const i64 c_int = (1LL << bq) * q.qm;  // bound on |a_int|

    k_lap_reset<<<g1, 256, 0, s>>>(n, L, st, 1);
    note_launches(1);
    cudaMemsetAsync(&st->lap_bids, 0, 3 * sizeof(long long), s);
    // The first phase starts at eps = c_int / 2^10: above that the phases are greedy
    // (every bid outprices all value differences) and only cost scans.  On the relaxed
    // Frank-Wolfe iterates of a 3-block SBM pair at n = 32768 (three product forms),
    // starting at c_int / 4 took 420-580 ms, at c_int / 2^10 220-380 ms with the same
    // optimum, while from c_int / 2^14 on the last phase's searches ran out of budget.
    i64 eps = std::max<i64>(1, c_int >> 10);
    int rounds = 0;
    bool exhausted = false;
    const int head_threshold = 4;
    const int head_stall = ctl.head_stall > 0 ? ctl.head_stall : INT_MAX;
    // the cluster kernels hold per-column state of n / 8 columns in each CTA's shared memory
    const int cw = (n + LAP_CLUSTER - 1) / LAP_CLUSTER;
    const size_t tail_smem = (size_t)cw * (sizeof(i64) + sizeof(int));
    bool use_cluster_tail = n >= 4096 && tail_smem <= 160 * 1024;
    if (use_cluster_tail &&
        cudaFuncSetAttribute(k_lap_tail_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tail_smem) !=
            cudaSuccess) {
        cudaGetLastError();
        use_cluster_tail = false;
    }
    // the augmenting-path searches: a cooperative grid with CPT columns per thread
    int sap_cpt = 0, sap_grid = 0;
    if (ctl.sap_pops != 0) {
        for (int c : {1, 2, 4, 8}) {
            if ((long long)sms * SAP_SLOTS * c >= n) {
                sap_cpt = c;
                break;
            }
        }
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (!coop) sap_cpt = 0;
        if (sap_cpt) sap_grid = (int)std::max<int64_t>(1, ceil_div(n, (int64_t)SAP_SLOTS * sap_cpt));
    }
    const bool use_sap = sap_cpt > 0;
    // the Jacobi rounds: one cooperative launch per phase (one CTA per SM), else
    // three launches per round
    int head_grid = 0;
    {
        int coop = 0, occ = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lap_head, LAP_HEAD_THREADS, 0) == cudaSuccess &&
            occ >= 1)
            head_grid = sms * std::min(occ, 1);
        cudaGetLastError();
    }
    const long long stall = ctl.tail_stall >= 0 ? ctl.tail_stall : std::max(128LL, (long long)n / 256);
    for (;;) {
        const bool last = eps <= 1;
        ++R.phases;
        k_lap_reset<<<g1, 256, 0, s>>>(n, L, st, 0);
        note_launches(1);
        int left = n;
        auto t0 = clk::now();
        int cur = 0;  // the list the next round bids from
        if (head_grid > 0 && ctl.head_rounds > 0 && rounds < ctl.max_rounds) {
            // all of the phase's rounds in one launch, one poll
            const float *Mp = M;
            int nn = n, c0 = 0, maxr = std::min(ctl.head_rounds, ctl.max_rounds - rounds), thr = head_threshold,
                hstall = head_stall;
            Quant qq = q;
            LapBuffers LL = L;
            i64 ee = eps;
            DevState *stp = st;
            void *args[] = {(void *)&Mp, (void *)&nn, (void *)&qq, (void *)&LL, (void *)&ee, (void *)&stp,
                            (void *)&c0, (void *)&maxr, (void *)&thr, (void *)&hstall};
            if (cudaLaunchCooperativeKernel((const void *)k_lap_head, dim3(head_grid), dim3(LAP_HEAD_THREADS), args, 0,
                                            s) != cudaSuccess)
                return GOAT_ERR_CUDA;
            note_launches(1);
            // lap_nb[0..1] and lap_head[0..1] are adjacent (host_pinned holds 64 ints)
            cudaMemcpyAsync(host_pinned, st->lap_nb, 4 * sizeof(int), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) return GOAT_ERR_CUDA;
            rounds += host_pinned[2];
            cur = host_pinned[3] & 1;
            left = host_pinned[cur];
        }
        for (int hr = 0; head_grid == 0 && hr < ctl.head_rounds && rounds < ctl.max_rounds; hr += 4) {
            // many bidders: many CTAs of 256 threads; few: one 1024-thread CTA per row
            const bool light = left <= sms;
            const int gb = light ? std::max(1, left) : growb;
            for (int b = 0; b < 4; ++b) {
                if (light)
                    k_lap_bid<1024><<<gb, 1024, 0, s>>>(M, n, q, L, eps, st, cur);
                else
                    k_lap_bid<256><<<gb, 256, 0, s>>>(M, n, q, L, eps, st, cur);
                k_lap_win<<<g1, 256, 0, s>>>(L, st, cur);
                k_lap_assign<<<g1, 256, 0, s>>>(L, st, cur);
                note_launches(3);
                cur ^= 1;
            }
            rounds += 4;
            left = poll_int(&st->lap_nb[cur], host_pinned, s);
            if (left <= head_threshold) break;
        }
        // the tail and the searches find the free rows from assign[]
        cudaMemcpyAsync(&st->lap_unassigned, &st->lap_nb[cur], sizeof(int), cudaMemcpyDeviceToDevice, s);
        R.ms_head += ms_since(t0);
        const long long budget = ctl.tail_bids >= 0 ? ctl.tail_bids
                                 : last             ? std::max(4LL * n, 262144LL)
                                                    : std::max((long long)n, 65536LL);
        // the sequential tail serves the last few rows of a phase; rows the Jacobi rounds
        // stalled on (near-tied objects, no progress in head_stall rounds) stall it too
        // and are left to the next phase, or to the searches in the last
        const bool head_stalled = head_grid > 0 && left > head_threshold;
        if (left > 0 && budget > 0 && !head_stalled) {
            t0 = clk::now();
            if (use_cluster_tail) {
                k_lap_tail_cluster<<<LAP_CLUSTER, 256, tail_smem, s>>>(M, n, q, L, eps, budget, stall, st);
            } else {
                k_lap_tail<<<1, 1024, 0, s>>>(M, n, q, L, eps, budget, stall, st);
            }
            note_launches(1);
            left = poll_int(&st->lap_unassigned, host_pinned, s);
            R.ms_tail += ms_since(t0);
        }
        // the searches complete the last phase; earlier phases only refine the prices,
        // and rows they leave unassigned start the next phase like every other row
        if (left > 0 && use_sap && (last || ctl.sap_every_phase)) {
            t0 = clk::now();
            const long long pops =
                ctl.sap_pops > 0 ? ctl.sap_pops : (last ? 64LL * n + (1LL << 20) : 8LL * n + (1LL << 16));
            cudaMemsetAsync(&st->lap_free, 0, sizeof(int), s);
            cudaMemsetAsync(L.tflag, 0, sizeof(int) * n, s);
            cudaMemsetAsync(L.mark_row, 0, sizeof(int) * n, s);
            cudaMemsetAsync(L.mark_col, 0, sizeof(int) * n, s);
            k_lap_sap_prep<<<growb, 256, 0, s>>>(M, n, q, L, st);
            int step_cols = ctl.sap_step > 0 ? ctl.sap_step : SAP_STEP;
            long long max_scans = pops;
            DevState *stp = st;
            const float *Mp = M;
            int nn = n;
            void *args[] = {(void *)&Mp, (void *)&nn, (void *)&q, (void *)&L, (void *)&step_cols, (void *)&max_scans,
                            (void *)&stp};
            const void *fn = sap_cpt == 1   ? (const void *)k_lap_sap_grid<1>
                             : sap_cpt == 2 ? (const void *)k_lap_sap_grid<2>
                             : sap_cpt == 4 ? (const void *)k_lap_sap_grid<4>
                                            : (const void *)k_lap_sap_grid<8>;
            if (cudaLaunchCooperativeKernel(fn, dim3(sap_grid), dim3(SAP_THREADS), args, 0, s) != cudaSuccess)
                return GOAT_ERR_CUDA;
            note_launches(2);
            R.sap_rows += left;
            left = poll_int(&st->lap_unassigned, host_pinned, s);
            R.sap_rows -= left;
            R.ms_sap += ms_since(t0);
        }
        if (last) {
            if (left > 0) {
                exhausted = true;
                R.filled = left;
                k_lap_fill<<<1, 1024, 0, s>>>(M, n, q, L, st);
                note_launches(1);
            }
            break;
        }
        eps = std::max<i64>(1, eps / 8);
    }

    k_copy_perm<<<g1, 256, 0, s>>>(n, L, perm_out);
    note_launches(1);
    k_assignment_cost<<<1, 1024, 0, s>>>(M, n, perm_out, cost_dev);
    note_launches(1);
    // duality gap in quantised units; below Qm it proves the assignment optimal
    double *gap_dev = cost_dev + 1;
    k_lap_gap<<<gbid, 256, 0, s>>>(M, n, q, L, L.ufree);  // the free rows' potentials are no longer needed
    k_lap_gap_sum<<<1, 1024, 0, s>>>(L.ufree, n, gap_dev);
    note_launches(2);
    double gq = 0.0;
    long long counts[3] = {0, 0, 0};
    cudaMemcpyAsync(&gq, gap_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(counts, &st->lap_bids, sizeof(counts), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return GOAT_ERR_CUDA;
    const bool optimal = !exhausted && gq < (double)q.qm;
    const double unit = std::ldexp(1.0, e - bq) / (double)q.qm;  // one quantised unit in units of M
    if (gap_host) *gap_host = optimal ? 0.0 : gq * unit;
    R.rounds = rounds;
    R.tail_bids = counts[0];
    R.sap_pops = counts[1];
    R.sap_epochs = counts[2];
    if (rep) *rep = R;
    return optimal ? GOAT_OK : GOAT_ERR_NOT_CONVERGED;
}

}  // namespace goat
