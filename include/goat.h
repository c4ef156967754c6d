/*
 * goat.h -- C ABI of libgoat, a GB300 (sm_103a) implementation of the
 * Frank-Wolfe hot path of GOAT (Saad-Eldin, Pedigo, Priebe, Vogelstein,
 * "Graph Matching via Optimal Transport"): FAQ's relaxation of graph matching
 * with the linear-assignment direction step replaced by entropic optimal
 * transport (Sinkhorn).
 *
 * Problem (Sec. 2.1-2.2): for adjacency matrices A, B (n x n) find the
 * permutation maximising f(P) = tr(A^T P B P^T), which minimises the number of
 * edge disagreements ||A - P B P^T||_F^2 = ||A||^2 + ||B||^2 - 2 f(P).
 *
 * Conventions shared by every entry point
 *   - Matrices are dense, row-major, leading dimension n, in DEVICE memory
 *     unless the name ends in _host.  Vectors likewise.
 *   - A and B are symmetric (undirected graphs) unless a call says otherwise.
 *     With that, grad f(P) = A P B^T + A^T P B = 2 A P B.
 *   - G denotes MINUS the gradient, G = -grad f(P) (so G <= 0 for
 *     non-negative graphs); the direction step solves min_Q <Q, G> - eps H(Q).
 *   - Sinkhorn duals (f, g) give Q_ij = exp((f_i + g_j - G_ij) / eps); Q has
 *     all row and column sums equal to 1 (the Birkhoff polytope, Sec. 3.3).
 *   - perm[i] is the vertex of B matched to vertex i of A (P[i][perm[i]] = 1).
 *   - The step size alpha returned here is the weight of the new direction:
 *     P_new = P + alpha (Q - P); the paper's alpha (the weight of P) is
 *     1 - alpha.
 *   - Every call is asynchronous on `stream` except where a host output is
 *     written, in which case the call synchronises `stream` before returning.
 *   - Errors: every entry point returns GOAT_OK (0) or a negative goat_status;
 *     outputs are unspecified after an error.  No C++ exception crosses the
 *     ABI.  Device-side waits and iterative loops are bounded; exhausting a
 *     bound returns GOAT_ERR_NOT_CONVERGED or GOAT_ERR_TIMEOUT, never a hang.
 *   - Scratch memory: calls that need it take (workspace, workspace_bytes).
 *     Pass a device buffer of at least goat_workspace_bytes(...) bytes, or
 *     NULL, in which case the call allocates with cudaMallocAsync on `stream`
 *     and frees before returning.  The caller owns all buffers it passes.
 *   - The library computes only on the GPU.  It returns GOAT_ERR_UNSUPPORTED on
 *     a device that is not compute capability 10.3; there is no CPU fallback.
 */
#ifndef GOAT_H_
#define GOAT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GOAT_API __attribute__((visibility("default")))
#else
#define GOAT_API
#endif

/* CUDA stream handle (cudaStream_t); 0 is the legacy default stream. */
typedef void *goat_stream_t;

typedef enum goat_status {
    GOAT_OK = 0,
    GOAT_ERR_INVALID_ARG = -1,   /* bad size, null pointer, unsupported flag, asymmetric input */
    GOAT_ERR_NOT_CONVERGED = -2, /* an iteration cap was reached where convergence is required */
    GOAT_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    GOAT_ERR_OUT_OF_MEMORY = -4, /* workspace too small or allocation failed */
    GOAT_ERR_NAN = -5,           /* a non-finite value appeared in the iteration */
    GOAT_ERR_TIMEOUT = -6,       /* a bounded device-side wait ran out */
    GOAT_ERR_UNSUPPORTED = -7    /* device is not sm_103 */
} goat_status;

/* element type of the adjacency inputs */
enum {
    GOAT_DTYPE_U8 = 0,  /* uint8 0/1 entries */
    GOAT_DTYPE_F32 = 1  /* float32 weights */
};

/* arithmetic of the two n x n x n gradient products */
enum {
    /* BF16 operands (exact for 0/1 adjacency), FP32 accumulation in TMEM; the
     * intermediate Q B is rounded once to BF16.  Gradient error ~1e-3 relative. */
    GOAT_PREC_BF16 = 0,
    /* FP32-accurate: every non-adjacency operand is split into two BF16 terms
     * (x = hi + lo), so each product runs twice the BF16 MMA work; error ~1e-6. */
    GOAT_PREC_FP32 = 1,
    /* 8-bit: A, B as E4M3 (exact for 0/1), Q and the intermediate Q B each rounded to
     * E4M3 under one power-of-two scale per matrix (largest entry near 448), FP32
     * accumulation; twice the BF16 MMA rate.  (E4M3 x BF16 is not one tensor-core
     * operation, so Q is 8-bit too.)  Gradient error ~1e-2 relative. */
    GOAT_PREC_FP8 = 2,
    /* Q as one BF16 term, the intermediate Q B as two (hi + lo): three BF16 MMA
     * passes per gradient instead of two (BF16) or four (FP32-accurate); the rounding
     * of Q B, which the second product sums over only the degree, is removed. */
    GOAT_PREC_BF16_SPLIT = 3,
    /* the first product (C1 = B Q^T) in E4M3 (B exact, Q rounded under one
     * power-of-two scale, twice the BF16 rate), C1 written as two BF16 terms for a
     * BF16 second product: 2.5 BF16 MMA passes per gradient. */
    GOAT_PREC_FP8_SPLIT = 4,
    /* the split form with the low term of Q B in E4M3: C1 = B Q^T as hi + lo (BF16),
     * both multiplied by one power of two s (exact) so that s lo fits E4M3 (|lo| is at
     * most 2^-9 |hi|); the second product runs the hi term in BF16 and the lo term in
     * E4M3 against A in E4M3 (twice the BF16 rate) into one FP32 accumulator, then
     * divides by s.  The lo term keeps about 4 of its bits: Q B is carried to about
     * 2^-13 relative instead of 2^-9 (BF16) or 2^-17 (split).  2.5 BF16 MMA passes. */
    GOAT_PREC_BF16_SPLIT8 = 5
};

/* direction step of each Frank-Wolfe iteration (goat_params.direction) */
enum {
    /* GOAT (Alg. 3): the entropic optimal-transport (LOT, Alg. 2) solution Q on
     * -grad f(P), a doubly stochastic matrix */
    GOAT_DIR_LOT = 0,
    /* FAQ (Alg. 1): an exact linear assignment, the permutation maximising
     * <Pi, grad f(P)>, by the same solver as the final projection */
    GOAT_DIR_LAP = 1
};

#define GOAT_TRACE_MAX 256

/* Parameters of the warm-start network (W1 [64][8], b1 [64], w2 [64], b2). */
#define GOAT_MLP_PARAMS 641

typedef struct goat_params {
    int precision;        /* GOAT_PREC_*, default GOAT_PREC_BF16                          */
    int sk_max_iter;      /* Sinkhorn iterations per Frank-Wolfe step, default 500        */
    float sk_tol;         /* Sinkhorn stop: max_j |column sum - 1| < sk_tol, default 1e-3 */
    int sk_warm_start;    /* 1: start each Sinkhorn from the previous step's duals (default 1) */
    int sk_check_every;   /* Sinkhorn iterations between host convergence checks, default 8 */
    int project_on_grad;  /* 0: final LAP on P (default); 1: on grad f(P) (the paper's Alg. 3 line) */
    int lap_max_rounds;   /* cap on auction bidding rounds over all phases, default 1<<20 */
    int profile;          /* 1: time the phases with CUDA events on `stream` (stats ms_*), default 0 */
    /* Learned warm start (device, GOAT_MLP_PARAMS BF16 values, or NULL): the first
     * Sinkhorn solve of goat_match starts from the duals the network predicts; if
     * that solve fails to reach sk_tol it is redone from a cold start. */
    const void *mlp_weights;
    /* GOAT_DIR_LOT (default: GOAT) or GOAT_DIR_LAP (FAQ).  With GOAT_DIR_LAP the
     * sk_* fields and mlp_weights are unused, stats.sk_iters are 0 and
     * stats.ms_sinkhorn times the per-iteration assignments; an assignment that the
     * auction cannot certify within its budget is still a permutation and is used.
     * goat_match_batched takes GOAT_DIR_LOT only. */
    int direction;
    /* 1 (default): graph matching, maximise f (Sec. 2.2); 0: QAP, minimise f (eq. QAP).
     * Minimising runs the same iteration on G = +grad f. */
    int maximize;
    /* Seeded matching (Sec. 4's seeded experiment): vertex i of A is known to match
     * vertex i of B for i < seeds (0 <= seeds <= n).  The iterate keeps the form
     * I_seeds (+) P22; gradient, direction, step and projection run on the unseeded
     * block, the seeds entering as a constant term of its gradient; eps, the stop
     * test (with the full n) and the returned permutation follow the unseeded method.
     * init, if given, must have the I_seeds (+) P22 form (only its block is read). */
    int seeds;
    /* 0 (default): A and B must be symmetric (checked; GOAT_ERR_INVALID_ARG
     * otherwise), grad f = 2 A P B (two products).  1: general (directed or
     * asymmetric weighted) graphs, grad f = A P B^T + A^T P B (four products). */
    int directed;
    /* DEVICE n x n float (nullable): receives the final relaxed iterate P, the
     * doubly stochastic soft matching (I_seeds (+) P22 with seeds). */
    float *relaxed_out;
} goat_params;

typedef struct goat_stats {
    int fw_iters;                      /* Frank-Wolfe iterations run                         */
    int converged;                     /* 1 if ||P_new - P||_F / sqrt(n) < tol ended the loop */
    int sk_iters_total;                /* Sinkhorn iterations over all steps                */
    int sk_iters[GOAT_TRACE_MAX];      /* per Frank-Wolfe step                              */
    float sk_resid[GOAT_TRACE_MAX];    /* last marginal residual per step                  */
    double alpha[GOAT_TRACE_MAX];      /* step size per step (weight of Q)                  */
    double objective;                  /* f(perm), exact for 0/1 inputs                     */
    double disagreements;              /* ||A||^2 + ||B||^2 - 2 f(perm)                     */
    double lap_gap;                    /* dual - primal of the final LAP (0: certified)     */
    int lap_rounds;                    /* auction rounds used                               */
    float ms_total, ms_fw, ms_project; /* device time of the whole call, FW loop, projection */
    /* with params.profile = 1 (else 0): device time per phase, summed over the FW loop */
    float ms_gemm;                     /* the tensor-core products (gemm_launches launches)  */
    int gemm_launches;
    float ms_sinkhorn;                 /* Sinkhorn solves, host polls included              */
    float ms_step;                     /* Q materialisation, line search and update          */
    long long launches;                /* kernels launched by the call                       */
    long long lap_tail_bids;           /* projection: sequential auction bids                */
    int lap_sap_rows;                  /* projection: rows placed by augmenting-path searches */
    long long lap_sap_pops;            /* projection: row scans of those searches            */
    float lap_ms_head, lap_ms_tail, lap_ms_sap; /* projection: host wall time of its bidding rounds,
                                          sequential bids and augmenting-path searches         */
} goat_stats;

/* Fills *p with the defaults listed above. */
GOAT_API void goat_default_params(goat_params *p);

/* Human-readable text for a goat_status.  Never NULL. */
GOAT_API const char *goat_strerror(int status);

/* Bytes of scratch the calls below need for size n (the maximum over calls).
 * Returns 0 for n < 1. */
GOAT_API size_t goat_workspace_bytes(int n, int dtype_AB, int precision);

/* Bytes of scratch goat_match_host needs (goat_workspace_bytes plus the device
 * copies of A, B and init).  Returns 0 for n < 1. */
GOAT_API size_t goat_workspace_bytes_host(int n, int dtype_AB, int precision);

/* Bytes of scratch goat_match (host = 0) or goat_match_host (host = 1) needs with
 * goat_params.directed = directed and goat_params.seeds = seeds (the two calls
 * above are directed = 0, seeds = 0).  Returns 0 for invalid arguments. */
GOAT_API size_t goat_workspace_bytes_ex(int n, int dtype_AB, int precision, int directed, int seeds, int host);

/*
 * goat_match -- the whole GOAT solve (Alg. 3), or FAQ (Alg. 1) with
 * p->direction = GOAT_DIR_LAP; QAP minimisation, seeded matching and directed
 * graphs through p->maximize, p->seeds and p->directed.
 *   A, B       device, n x n, dtype_AB; symmetric unless p->directed = 1 (checked:
 *              GOAT_ERR_INVALID_ARG otherwise).
 *   init       device n x n float doubly stochastic start, or NULL for the
 *              barycenter J = 11^T / n (Alg. 3 "Initialize").
 *   eps_rel    entropic weight per step: eps = eps_rel * max|grad f(P)|
 *              (the paper's lambda = 1/eps, Sec. 3.3).
 *   max_iter   Frank-Wolfe steps (>= 0), tol  stop when ||P_new-P||_F/sqrt(n) < tol.
 *   p          parameters (NULL: defaults).
 *   perm_out   HOST int32[n]; objective_out HOST double (nullable); stats HOST (nullable).
 * Reaching max_iter is not an error.  Synchronises `stream`.
 */
GOAT_API int goat_match(const void *A, const void *B, int n, int dtype_AB, const float *init, float eps_rel, int max_iter,
               float tol, const goat_params *p, int32_t *perm_out, double *objective_out, goat_stats *stats,
               void *workspace, size_t workspace_bytes, goat_stream_t stream);

/* goat_match with A, B, init in HOST memory (pageable or pinned); the copies to
 * the device are part of the call.  Its workspace must hold
 * goat_workspace_bytes_host(n, dtype_AB, precision) bytes (it stages the copies). */
GOAT_API int goat_match_host(const void *A_host, const void *B_host, int n, int dtype_AB, const float *init_host,
                    float eps_rel, int max_iter, float tol, const goat_params *p, int32_t *perm_out,
                    double *objective_out, goat_stats *stats, void *workspace, size_t workspace_bytes,
                    goat_stream_t stream);

/*
 * goat_gradient -- Alg. 3 step 1: G_out = -grad f(P) = -(A P B^T + A^T P B) = -2 A P B.
 *   A, B   device n x n (dtype_AB), symmetric.   P  device n x n float.
 *   G_out  device n x n float.  precision  GOAT_PREC_*.
 */
GOAT_API int goat_gradient(const void *A, const void *B, int n, int dtype_AB, const float *P, float *G_out, int precision,
                  void *workspace, size_t workspace_bytes, goat_stream_t stream);

/*
 * goat_gradient_ex -- goat_gradient for general graphs (Alg. 1 / Alg. 3 step 1 with
 * no symmetry): with directed = 1, G_out = -(A P B^T + A^T P B) by four products
 * (C1 = B P^T, C1' = B^T P^T, then [A | A^T] [C1 | C1']^T in one accumulation);
 * directed = 0 is goat_gradient.  Workspace: goat_workspace_bytes_ex(n, dtype_AB,
 * precision, directed, 0, 0) bytes, or NULL.
 */
GOAT_API int goat_gradient_ex(const void *A, const void *B, int n, int dtype_AB, const float *P, float *G_out,
                              int precision, int directed, void *workspace, size_t workspace_bytes,
                              goat_stream_t stream);

/*
 * goat_sinkhorn -- LOT (Alg. 2): entropic rLAP min_Q <Q, G> - eps H(Q) over doubly
 * stochastic Q, as log-domain Sinkhorn.  One iteration: row scaling
 * f_i = -eps LSE_j((g_j - G_ij)/eps), then the column sums S_j of that Q,
 * residual max_j |S_j - 1|, and the column scaling g_j -= eps log S_j.
 *   G        device n x n float cost.          eps > 0.
 *   f_out    device float[n].                  g_io  device float[n]: warm start in, duals out.
 *   Q_out    device n x n float, or NULL.      stops when residual < tol or after max_iter.
 *   iters_out, resid_out  HOST (nullable).  Reaching max_iter is not an error.
 */
GOAT_API int goat_sinkhorn(const float *G, int n, float eps, float tol, int max_iter, float *f_out, float *g_io,
                  float *Q_out, int *iters_out, float *resid_out, void *workspace, size_t workspace_bytes,
                  goat_stream_t stream);

/*
 * goat_line_search -- Alg. 3 step 3 (the exact quadratic step of FAQ / SGM).
 * With D = Q - P, f(P + a D) = f(P) + b t + a t^2 where
 *   b = <grad f(P), D> = -<G, D>,   a = tr(A^T D B D^T) = (1/2) <G - G_Q, D>,
 * G = -grad f(P), G_Q = -grad f(Q) (grad f is linear, so grad f(D) = grad f(Q) - grad f(P)).
 * alpha = argmax_{[0,1]} (maximize = 1) or argmin (maximize = 0) of b t + a t^2; when
 * a >= 0 (resp. a <= 0) the end point 1 is taken only if strictly better than 0.
 *   all matrices device n x n float;  alpha_out, a_out, b_out HOST (nullable except alpha_out).
 */
GOAT_API int goat_line_search(const float *G, const float *G_Q, const float *P, const float *Q, int n, int maximize,
                     double *alpha_out, double *a_out, double *b_out, void *workspace, size_t workspace_bytes,
                     goat_stream_t stream);

/*
 * goat_fw_update -- Alg. 3 step 4 and the gradient by linearity:
 *   P <- P + alpha (Q - P),   G <- G + alpha (G_Q - G).
 * All device n x n float; P and G are updated in place.
 */
GOAT_API int goat_fw_update(float *P, float *G, const float *Q, const float *G_Q, int n, double alpha, goat_stream_t stream);

/*
 * goat_entropic_eps -- the entropic weight of Alg. 2 as goat_match chooses it
 * (the paper's lambda read as eps = 1 / lambda, relative to the cost's scale):
 *   eps = eps_rel * max|G|, or 1 when G == 0 (every doubly stochastic Q is then optimal).
 *   G device n x n float; eps_out HOST float.  Allocates 4 bytes with cudaMallocAsync
 *   on `stream` and waits for the stream.  GOAT_ERR_NAN for a non-finite entry.
 */
GOAT_API int goat_entropic_eps(const float *G, int n, float eps_rel, float *eps_out, goat_stream_t stream);

/*
 * goat_project -- the final linear assignment (Alg. 3 return line):
 * perm = argmax (maximize = 1) or argmin (0) of sum_i M[i][perm i] over permutations.
 * Exact: the entries are quantised to 64-bit integers (40 bits below the largest
 * |M|, scaled by a power of two Qm > n), solved by an eps-scaling auction whose
 * stragglers are placed by shortest augmenting paths, and certified optimal for
 * the quantised matrix by LP duality (gap < 1 quantum).
 *   M         device n x n float.     perm_out  device int32[n].
 *   cost_out  HOST double: sum_i M[i][perm i] in FP64, row order (nullable).
 *   gap_out   HOST double: dual minus primal, in units of M (0 when certified) (nullable).
 * Returns GOAT_ERR_NOT_CONVERGED (perm still a valid permutation) when the budgets
 * ran out before the certificate; GOAT_ERR_NAN for a non-finite entry.
 */
GOAT_API int goat_project(const float *M, int n, int maximize, int32_t *perm_out, double *cost_out, double *gap_out,
                 void *workspace, size_t workspace_bytes, goat_stream_t stream);

/* Schedule of the projection's auction (negative fields: built-in default). */
typedef struct goat_lap_options {
    int max_rounds;       /* parallel (Jacobi) bidding rounds over all phases, default 1<<20   */
    int head_rounds;      /* Jacobi rounds per eps phase before the sequential steps (the rounds
                             stop early once at most 4 rows bid), default 256                 */
    long long tail_bids;  /* sequential (Gauss-Seidel) bids per phase, default max(n, 65536),
                             max(4n, 262144) in the last phase; 0 skips that step            */
    long long tail_stall; /* bids in a row that do not shorten the queue of unassigned rows
                             and end the sequential bidding, default max(128, n / 256)        */
    long long sap_pops;   /* row scans the shortest-augmenting-path searches may do per phase,
                             default 8n + 2^16 (64n + 2^20 in the last phase); 0 disables them */
    int head_stall;       /* Jacobi rounds in a row without fewer bidders than before that end
                             a phase's rounds, default 16                                    */
    int sap_every_phase;  /* 1: the searches complete every eps phase; 0 (default): only the
                             last, earlier phases leave their stalled rows unassigned (their
                             prices still start the next phase)                             */
} goat_lap_options;

/* What one projection did. */
typedef struct goat_lap_info {
    int phases;           /* eps phases                                          */
    int rounds;           /* Jacobi rounds                                       */
    long long tail_bids;  /* Gauss-Seidel bids                                   */
    int sap_rows;         /* rows placed by augmenting-path searches             */
    long long sap_pops;   /* rows those searches scanned (a row again after its label fell) */
    long long sap_steps;  /* grid-wide parallel steps of those searches          */
    int filled;           /* rows filled greedily after every budget ran out     */
    double ms_head, ms_tail, ms_sap; /* host wall time of each kind of step, polls included */
} goat_lap_info;

/* Fills *o with the defaults (all fields -1 except max_rounds and head_rounds). */
GOAT_API void goat_lap_default_options(goat_lap_options *o);

/*
 * goat_project_ex -- goat_project with an explicit schedule (opts, nullable:
 * defaults) and a report of the work done (info, HOST, nullable).  The result is
 * the same optimum whatever the schedule; only the time and the budgets change.
 */
GOAT_API int goat_project_ex(const float *M, int n, int maximize, const goat_lap_options *opts, int32_t *perm_out,
                    double *cost_out, double *gap_out, goat_lap_info *info, void *workspace, size_t workspace_bytes,
                    goat_stream_t stream);

/*
 * goat_objective -- f(perm) = sum_ij A_ij B[perm i][perm j] (eq. QAP at a permutation)
 * and disagreements ||A||^2 + ||B||^2 - 2 f.  Exact (64-bit integer sums) for
 * GOAT_DTYPE_U8.  A, B, perm device; outputs HOST (nullable).
 */
GOAT_API int goat_objective(const void *A, const void *B, int n, int dtype_AB, const int32_t *perm, double *objective_out,
                   double *disagreements_out, void *workspace, size_t workspace_bytes, goat_stream_t stream);

/*
 * goat_match_batched -- many GOAT solves (Alg. 3) advanced together: num_pairs
 * graph pairs of sizes n[p] (1 <= n[p] <= 2048), each solved from `restarts`
 * starting points (Sec. 3.4): restart 0 is the barycenter J, restart r >= 1 the
 * random start (J + K)/2 where K is the Sinkhorn-Knopp scaling of noise
 * U_ij in (0, 1]: U_ij = (SplitMix64 output number ((q << 32) | (i n + j)) of the
 * generator seeded with `seed`, shifted right by 40, plus 1) / 2^24, q the problem
 * index pair * restarts + restart.  The best restart (largest objective, lowest
 * index on ties) is returned per pair.  Each Frank-Wolfe iteration of all
 * problems is one replay of a CUDA graph; the Sinkhorn launch shape is chosen per
 * batch by timing candidates on the batch (cached per process).
 *   A, B       device uint8, the pairs' symmetric 0/1 matrices packed back to back;
 *              pair p is n[p] x n[p] row-major at byte offset adj_off[p] (HOST array).
 *   n          HOST int[num_pairs].
 *   perm_out   HOST int32[sum n[p]]: the pairs' best permutations, concatenated.
 *   objective_out, best_restart, fw_iters_out  HOST [num_pairs] (nullable).
 *   relaxed_out  DEVICE float (nullable): the final relaxed P of every problem (the
 *              doubly stochastic "soft matching"), problems in order q, each n x n row-major.
 *   params     precision must be GOAT_PREC_BF16 and direction GOAT_DIR_LOT (GOAT_ERR_INVALID_ARG
 *              otherwise); the Sinkhorn and FW limits apply per problem.
 * Workspace: goat_workspace_bytes_batched(n, num_pairs, restarts) bytes, or NULL.
 */
GOAT_API size_t goat_workspace_bytes_batched(const int *n, int num_pairs, int restarts);
GOAT_API int goat_match_batched(const void *A, const void *B, const long long *adj_off, const int *n, int num_pairs,
                                int restarts, unsigned long long seed, float eps_rel, int max_iter, float tol,
                                const goat_params *params, int32_t *perm_out, double *objective_out,
                                int *best_restart, int *fw_iters_out, float *relaxed_out, void *workspace,
                                size_t workspace_bytes, goat_stream_t stream);

/*
 * goat_sinkhorn_noalloc -- goat_sinkhorn for callers that cannot allocate.
 * The paper has no counterpart: this exists for callers that must not allocate
 * device memory during the call (they run under an allocator they do not own,
 * inside a fixed memory budget, or on a thread that must not synchronise with the
 * device the way cudaMalloc/cudaFree can).  It allocates nothing and never
 * synchronises with the device: its scratch is one static device array of about
 * 2 MiB, held by every GPU that loads the library until the process exits.
 *   G, n, eps, tol, f_out, g_io  as in goat_sinkhorn; n <= 4096, larger n returns
 *                                 GOAT_ERR_INVALID_ARG (the array is sized for 4096).
 *   max_iter   iteration slots queued, 1 <= max_iter <= 1000 (GOAT_ERR_INVALID_ARG
 *              otherwise); once the residual falls below tol the remaining slots do
 *              no work, so the result equals goat_sinkhorn's.  Every slot is about
 *              five kernel launches, so a long queue can make the host block inside
 *              the launch calls until the GPU drains it (launch-queue back-pressure).
 *   iters_out, resid_out, status_out  DEVICE int / float / int (nullable), written
 *              when the stream reaches the end of the call.  *status_out is GOAT_OK
 *              or GOAT_ERR_NAN (a non-finite residual, e.g. from a non-finite G):
 *              the return value only reports errors found before the launches.
 * The first call on each device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The lookup is
 * repeated only when the device's context has changed (after cudaDeviceReset).
 * All calls share the one array and each starts by clearing its state block, so
 * calls that overlap on the GPU (other streams, other host threads) race: serialise them.
 */
GOAT_API int goat_sinkhorn_noalloc(const float *G, int n, float eps, float tol, int max_iter, float *f_out,
                                   float *g_io, int *iters_out, float *resid_out, int *status_out,
                                   goat_stream_t stream);

/*
 * Learned Sinkhorn warm start.  The paper has no counterpart; it serves Alg. 2:
 * a small network predicts the LOT duals from per-node features so each solve
 * starts close to its fixed point.  Nodes 0..n-1 are the rows of G (dual f),
 * n..2n-1 its columns (dual g).
 *
 * goat_dual_features -- feats (device, 2n x 8 float): degree / mean degree,
 *   2-hop degree / its mean, mean, max, std, min of the node's line of G over eps,
 *   side (0 rows, 1 columns), ln(n) / 10.  A, B as in goat_match.
 * goat_mlp_forward -- y = w2 . tanh(W1 x + b1) + b2 for N feature rows (device),
 *   weights in BF16 (device, GOAT_MLP_PARAMS).  y is the dual over eps, each side's
 *   mean removed.
 * goat_mlp_train_step -- one mean-squared-error step on (x, t): grad_out (device,
 *   GOAT_MLP_PARAMS floats) receives the gradient at the BF16 weights, loss_out
 *   (device float) the loss; with lr > 0 an Adam step (Kingma & Ba, beta 0.9 /
 *   0.999) updates the FP32 master weights, adam_state (2 x GOAT_MLP_PARAMS
 *   floats: first, second moments) and the BF16 copy.  step counts from 1.
 * goat_mlp_warm_start -- g_out (device, n floats) = eps * predicted g, the warm
 *   start goat_sinkhorn takes in g_io.
 */
GOAT_API int goat_dual_features(const float *G, const void *A, const void *B, int n, int dtype_AB, float eps,
                                float *feats, void *workspace, size_t workspace_bytes, goat_stream_t stream);
GOAT_API int goat_mlp_forward(const void *weights_bf16, const float *x, int N, float *y, goat_stream_t stream);
/* goat_dual_targets -- the training targets of a solve's duals f, g (device, n floats
 * each) at weight eps: t_out (device, 2n floats) = [f/eps - mean(f/eps),
 * g/eps - mean(g/eps)] (the duals are defined up to f + c, g - c), means in FP64. */
GOAT_API int goat_dual_targets(const float *f, const float *g, int n, float eps, float *t_out, goat_stream_t stream);
GOAT_API int goat_mlp_train_step(float *master, float *adam_state, void *weights_bf16, const float *x,
                                 const float *t, int N, float lr, int step, float *loss_out, float *grad_out,
                                 goat_stream_t stream);
GOAT_API int goat_mlp_warm_start(const float *G, const void *A, const void *B, int n, int dtype_AB, float eps,
                                 const void *weights_bf16, float *g_out, void *workspace, size_t workspace_bytes,
                                 goat_stream_t stream);

/*
 * goat_gemm_bf16_xyT -- kernel-level entry to the tensor-core product behind
 * goat_gradient (Alg. 3 step 1 evaluates grad f with two such products):
 *   out[r][c] = scale * sum_k X[r][k mod kx_period] * Y[c][k],  0 <= k < k_total.
 *   X  device BF16, x_rows rows of x_stride elements (16-byte aligned rows);
 *   Y  device BF16, y_rows rows of y_stride elements; k_total, kx_period multiples of 64;
 *      rows or K positions beyond the given extents read as zero.
 *   out  device float, out_rows x out_cols, leading dimension ld_out.
 * Synchronises `stream`; GOAT_ERR_TIMEOUT if the kernel's bounded pipeline waits ran out.
 */
GOAT_API int goat_gemm_bf16_xyT(const void *X, int x_rows, int x_stride, int kx_period, const void *Y, int y_rows,
                       int y_stride, int k_total, float scale, float *out, int ld_out, int out_rows, int out_cols,
                       goat_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GOAT_H_ */
