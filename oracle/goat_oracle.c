/*
 * goat_oracle.c -- plain, slow FP64 CPU oracle for GOAT and FAQ
 * (Saad-Eldin, Pedigo, Priebe, Vogelstein: "Graph Matching via Optimal Transport").
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load it.  The GPU library never
 * links, calls or includes anything from here, and nothing here comes from the
 * GPU library: the two share no code, headers, tables or helpers.
 *
 * Every routine works in FP64 on dense row-major n x n matrices (leading
 * dimension n) and follows the paper's definitions in the paper's order:
 *
 *   objective      f(P) = tr(A^T P B P^T)                          eq. (QAP)
 *   gradient       grad f(P) = A P B^T + A^T P B                   Alg. 1 / Alg. 3, step 1
 *   LOT            K = exp(-lambda M), Q = Sinkhorn(K)              Alg. 2, with eps = 1/lambda
 *   step size      alpha in argmax_{[0,1]} f(alpha P + (1-alpha) Q) Alg. 3, step 3 (exact quadratic)
 *   update         P <- alpha P + (1-alpha) Q                      Alg. 3, step 4
 *   projection     argmax_{Pi in perms} tr(Pi^T X)                  Alg. 3, return line (Hungarian)
 *   FAQ            step 2 replaced by a Hungarian LAP               Alg. 1
 *
 * Readings of the paper that this file takes (each is listed with its reason
 * in the design notes of the repository):
 *   - graph matching maximises f (the GM reduction, Sec. 2.2); QAP minimises it;
 *   - the doubly-stochastic marginals are the all-ones vectors (Sec. 3.3);
 *   - eps = eps_rel * max|grad f| is recomputed each Frank-Wolfe iteration;
 *   - one Sinkhorn iteration = row scaling then column scaling; its residual
 *     is max_j |column sum_j - 1| measured after the row scaling;
 *   - the Frank-Wolfe loop stops when ||P_new - P||_F / sqrt(n) < tol or at
 *     max_iter (the paper leaves the criterion to its code);
 *   - in the convex (a >= 0) tie case of the line search the iterate stays at P.
 *
 * Products are naive triple loops (i-k-j order); a term whose left factor is
 * exactly zero is skipped, which leaves every sum unchanged.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, n) ((size_t)(i) * (size_t)(n) + (size_t)(j))

/* ------------------------------------------------------------------ */
/* dense helpers                                                        */
/* ------------------------------------------------------------------ */

static double *alloc_mat(int n) { return (double *)calloc((size_t)n * (size_t)n, sizeof(double)); }

/* Z = X * Y by the textbook triple loop. */
static void matmul(const double *X, const double *Y, int n, double *Z)
{
    memset(Z, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int i = 0; i < n; ++i) {
        double *zi = Z + IDX(i, 0, n);
        for (int k = 0; k < n; ++k) {
            double x = X[IDX(i, k, n)];
            if (x == 0.0) continue;
            const double *yk = Y + IDX(k, 0, n);
            for (int j = 0; j < n; ++j) zi[j] += x * yk[j];
        }
    }
}

static void transpose(const double *X, int n, double *Xt)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Xt[IDX(j, i, n)] = X[IDX(i, j, n)];
}

static double frob_inner(const double *X, const double *Y, int n)
{
    double s = 0.0;
    for (size_t t = 0; t < (size_t)n * (size_t)n; ++t) s += X[t] * Y[t];
    return s;
}

/* ------------------------------------------------------------------ */
/* objective, eq. (QAP)                                                 */
/* ------------------------------------------------------------------ */

/* f(P) = tr(A^T P B P^T) = <A P, P B>_F for any square P. */
double oracle_objective(const double *A, const double *B, const double *P, int n)
{
    double *AP = alloc_mat(n), *Bt = alloc_mat(n), *Pt = alloc_mat(n), *BtPt = alloc_mat(n), *PB = alloc_mat(n);
    matmul(A, P, n, AP);
    transpose(B, n, Bt);
    transpose(P, n, Pt);
    matmul(Bt, Pt, n, BtPt); /* (P B)^T = B^T P^T */
    transpose(BtPt, n, PB);
    double f = frob_inner(AP, PB, n);
    free(AP); free(Bt); free(Pt); free(BtPt); free(PB);
    return f;
}

/* f at the permutation matrix with P[i][perm[i]] = 1:
 * (P B P^T)_{ij} = B[perm i][perm j], so f = sum_ij A_ij B[perm i][perm j]. */
double oracle_objective_perm(const double *A, const double *B, int n, const int *perm)
{
    double f = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) f += A[IDX(i, j, n)] * B[IDX(perm[i], perm[j], n)];
    return f;
}

/* Same on 0/1 (or small integer) byte matrices, exact in 64-bit integers. */
int64_t oracle_objective_perm_u8(const uint8_t *A, const uint8_t *B, int n, const int *perm)
{
    int64_t f = 0;
    for (int i = 0; i < n; ++i) {
        const uint8_t *ai = A + IDX(i, 0, n);
        const uint8_t *bi = B + IDX(perm[i], 0, n);
        for (int j = 0; j < n; ++j)
            if (ai[j]) f += (int64_t)ai[j] * (int64_t)bi[perm[j]];
    }
    return f;
}

/* ------------------------------------------------------------------ */
/* gradient, Alg. 1 / Alg. 3 step 1                                     */
/* ------------------------------------------------------------------ */

/* grad = A P B^T + A^T P B, recomputed from scratch (no symmetry assumed).
 * A P B^T is formed as (A P) B^T = (B (A P)^T)^T and A^T P B as
 * (A^T P) B = (B^T (A^T P)^T)^T, so that the adjacency matrix is always the
 * left factor of the triple loop. */
void oracle_gradient(const double *A, const double *B, const double *P, int n, double *grad)
{
    double *At = alloc_mat(n), *Bt = alloc_mat(n), *X = alloc_mat(n), *Xt = alloc_mat(n), *Y = alloc_mat(n);
    transpose(A, n, At);
    transpose(B, n, Bt);

    matmul(A, P, n, X);      /* X = A P           */
    transpose(X, n, Xt);
    matmul(B, Xt, n, Y);     /* Y = B (A P)^T      */
    transpose(Y, n, grad);   /* grad = A P B^T     */

    matmul(At, P, n, X);     /* X = A^T P         */
    transpose(X, n, Xt);
    matmul(Bt, Xt, n, Y);    /* Y = B^T (A^T P)^T  */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) grad[IDX(i, j, n)] += Y[IDX(j, i, n)]; /* += A^T P B */

    free(At); free(Bt); free(X); free(Xt); free(Y);
}

/* Selected rows of grad f(P) = A P B^T + A^T P B for large n, from byte
 * adjacency matrices and a single-precision P (all converted exactly to FP64).
 * Row i of A P B^T is w B^T with w = sum_k A_ik P_k,: ; row i of A^T P B is
 * w2 B with w2 = sum_k A_ki P_k,: .  out is nrows x n. */
void oracle_gradient_rows_u8(const uint8_t *A, const uint8_t *B, const float *P, int n,
                             const int *rows, int nrows, double *out)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *w2 = (double *)malloc(sizeof(double) * (size_t)n);
    for (int r = 0; r < nrows; ++r) {
        int i = rows[r];
        double *o = out + IDX(r, 0, n);
        for (int l = 0; l < n; ++l) { w[l] = 0.0; w2[l] = 0.0; }
        for (int k = 0; k < n; ++k) {
            double aik = (double)A[IDX(i, k, n)];
            double aki = (double)A[IDX(k, i, n)];
            const float *pk = P + IDX(k, 0, n);
            if (aik != 0.0) for (int l = 0; l < n; ++l) w[l] += aik * (double)pk[l];
            if (aki != 0.0) for (int l = 0; l < n; ++l) w2[l] += aki * (double)pk[l];
        }
        for (int j = 0; j < n; ++j) o[j] = 0.0;
        for (int j = 0; j < n; ++j) { /* (w B^T)_j = sum_l w_l B_jl */
            const uint8_t *bj = B + IDX(j, 0, n);
            double s = 0.0;
            for (int l = 0; l < n; ++l) if (bj[l]) s += w[l] * (double)bj[l];
            o[j] += s;
        }
        for (int l = 0; l < n; ++l) { /* (w2 B)_j = sum_l w2_l B_lj */
            const uint8_t *bl = B + IDX(l, 0, n);
            double wl = w2[l];
            if (wl == 0.0) continue;
            for (int j = 0; j < n; ++j) if (bl[j]) o[j] += wl * (double)bl[j];
        }
    }
    free(w); free(w2);
}

/* Same with single-precision (weighted) adjacency matrices. */
void oracle_gradient_rows_f32(const float *A, const float *B, const float *P, int n,
                              const int *rows, int nrows, double *out)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *w2 = (double *)malloc(sizeof(double) * (size_t)n);
    for (int r = 0; r < nrows; ++r) {
        int i = rows[r];
        double *o = out + IDX(r, 0, n);
        for (int l = 0; l < n; ++l) { w[l] = 0.0; w2[l] = 0.0; }
        for (int k = 0; k < n; ++k) {
            double aik = (double)A[IDX(i, k, n)];
            double aki = (double)A[IDX(k, i, n)];
            const float *pk = P + IDX(k, 0, n);
            if (aik != 0.0) for (int l = 0; l < n; ++l) w[l] += aik * (double)pk[l];
            if (aki != 0.0) for (int l = 0; l < n; ++l) w2[l] += aki * (double)pk[l];
        }
        for (int j = 0; j < n; ++j) {
            const float *bj = B + IDX(j, 0, n);
            double s = 0.0;
            for (int l = 0; l < n; ++l) if (bj[l] != 0.0f) s += w[l] * (double)bj[l];
            o[j] = s;
        }
        for (int l = 0; l < n; ++l) {
            const float *bl = B + IDX(l, 0, n);
            double wl = w2[l];
            if (wl == 0.0) continue;
            for (int j = 0; j < n; ++j) if (bl[j] != 0.0f) o[j] += wl * (double)bl[j];
        }
    }
    free(w); free(w2);
}

/* ------------------------------------------------------------------ */
/* Sinkhorn / LOT, Alg. 2 (Cuturi's Sinkhorn-Knopp on K = exp(-M/eps))  */
/* ------------------------------------------------------------------ */

/* Sinkhorn-Knopp on a positive kernel K towards marginals 1_n (Sec. 3.3):
 *   u = 1 / (K v);  S_j = v_j (K^T u)_j;  resid = max_j |S_j - 1|;  v = 1 / (K^T u)
 * repeated until resid < tol or max_iter iterations.  v may carry a warm
 * start (NULL: v = 1).  Writes Q = diag(u) K diag(v), u and v.
 * Returns the number of iterations; *resid_out gets the last residual. */
int oracle_sinkhorn_knopp(const double *K, int n, double tol, int max_iter,
                          const double *v_init, double *Q, double *u_out, double *v_out, double *resid_out)
{
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    for (int j = 0; j < n; ++j) v[j] = v_init ? v_init[j] : 1.0;
    int it = 0;
    double resid = INFINITY;
    while (it < max_iter) {
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += K[IDX(i, j, n)] * v[j];
            u[i] = 1.0 / s;
        }
        for (int j = 0; j < n; ++j) w[j] = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) w[j] += K[IDX(i, j, n)] * u[i];
        resid = 0.0;
        for (int j = 0; j < n; ++j) {
            double S = v[j] * w[j];
            double d = fabs(S - 1.0);
            if (d > resid || d != d) resid = d;
            v[j] = 1.0 / w[j];
        }
        ++it;
        if (resid < tol) break;
    }
    if (Q)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) Q[IDX(i, j, n)] = u[i] * K[IDX(i, j, n)] * v[j];
    if (u_out) memcpy(u_out, u, sizeof(double) * (size_t)n);
    if (v_out) memcpy(v_out, v, sizeof(double) * (size_t)n);
    if (resid_out) *resid_out = resid;
    free(u); free(v); free(w);
    return it;
}

/* LOT (Alg. 2) for the minimisation rLAP  min <Q, M>  over doubly stochastic Q
 * with entropic weight eps = 1/lambda:  K = exp(-M/eps), Q = Sinkhorn(K).
 * Returns duals in log form, f = eps log u and g = eps log v, so that
 * Q_ij = exp((f_i + g_j - M_ij) / eps).  g_init (nullable) warm-starts v. */
int oracle_lot(const double *M, int n, double eps, double tol, int max_iter, const double *g_init,
               double *Q, double *f, double *g, double *resid_out)
{
    double *K = alloc_mat(n);
    double *u = (double *)malloc(sizeof(double) * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *v0 = NULL;
    for (size_t t = 0; t < (size_t)n * (size_t)n; ++t) K[t] = exp(-M[t] / eps);
    if (g_init) {
        v0 = (double *)malloc(sizeof(double) * (size_t)n);
        for (int j = 0; j < n; ++j) v0[j] = exp(g_init[j] / eps);
    }
    int it = oracle_sinkhorn_knopp(K, n, tol, max_iter, v0, Q, u, v, resid_out);
    if (f) for (int i = 0; i < n; ++i) f[i] = eps * log(u[i]);
    if (g) for (int j = 0; j < n; ++j) g[j] = eps * log(v[j]);
    free(K); free(u); free(v); free(v0);
    return it;
}

/* The same iteration written in the log domain, for costs whose exp(-M/eps)
 * would overflow FP64:
 *   f_i = -eps LSE_j((g_j - M_ij)/eps)
 *   S_j = sum_i exp((f_i + g_j - M_ij)/eps),  resid = max_j |S_j - 1|
 *   g_j = -eps LSE_i((f_i - M_ij)/eps)
 * g carries the warm start in and the duals out (f is output only). */
int oracle_lot_log(const double *M, int n, double eps, double tol, int max_iter,
                   double *f, double *g, double *Q, double *resid_out)
{
    int it = 0;
    double resid = INFINITY;
    while (it < max_iter) {
        for (int i = 0; i < n; ++i) {
            double m = -INFINITY;
            for (int j = 0; j < n; ++j) { double x = (g[j] - M[IDX(i, j, n)]) / eps; if (x > m) m = x; }
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += exp((g[j] - M[IDX(i, j, n)]) / eps - m);
            f[i] = -eps * (m + log(s));
        }
        resid = 0.0;
        for (int j = 0; j < n; ++j) {
            double m = -INFINITY;
            for (int i = 0; i < n; ++i) { double x = (f[i] - M[IDX(i, j, n)]) / eps; if (x > m) m = x; }
            double s = 0.0;
            for (int i = 0; i < n; ++i) s += exp((f[i] - M[IDX(i, j, n)]) / eps - m);
            double S = exp(g[j] / eps + m) * s; /* column sum before the column scaling */
            double d = fabs(S - 1.0);
            if (d > resid || d != d) resid = d;
            g[j] = -eps * (m + log(s));
        }
        ++it;
        if (resid < tol) break;
    }
    if (Q)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) Q[IDX(i, j, n)] = exp((f[i] + g[j] - M[IDX(i, j, n)]) / eps);
    if (resid_out) *resid_out = resid;
    return it;
}

/* Row scaling of the log-domain iteration on a block of rows of a large
 * single-precision cost (Mrows is nrows x n):  f_r = -eps LSE_j((g_j - M_rj)/eps). */
void oracle_lot_rows_f32(const float *Mrows, int nrows, int n, const float *g, double eps, double *f_out)
{
    for (int r = 0; r < nrows; ++r) {
        const float *mi = Mrows + IDX(r, 0, n);
        double m = -INFINITY;
        for (int j = 0; j < n; ++j) { double x = ((double)g[j] - (double)mi[j]) / eps; if (x > m) m = x; }
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += exp(((double)g[j] - (double)mi[j]) / eps - m);
        f_out[r] = -eps * (m + log(s));
    }
}

/* Column sums S_c = sum_i exp((f_i + g_c - M_ic)/eps) on a block of columns
 * (Mcols is n x ncols, row-major: Mcols[i][c] = M[i][column c]). */
void oracle_lot_colsums_f32(const float *Mcols, int n, int ncols, const float *f, const float *gcols, double eps,
                            double *S_out)
{
    for (int c = 0; c < ncols; ++c) {
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            s += exp(((double)f[i] + (double)gcols[c] - (double)Mcols[IDX(i, c, ncols)]) / eps);
        S_out[c] = s;
    }
}

/* ------------------------------------------------------------------ */
/* step size, Alg. 3 step 3                                             */
/* ------------------------------------------------------------------ */

/* phi(alpha) = f(alpha P + (1-alpha) Q) = f(Q) + b alpha + a alpha^2 with
 * E = P - Q:  a = tr(A^T E B E^T),  b = tr(A^T E B Q^T) + tr(A^T Q B E^T).
 * Using tr(A^T X B Y^T) = <A X, Y B>_F the three traces are formed from the
 * products A E, A Q, E B and Q B.  maximize = 1 picks argmax over [0,1]
 * (graph matching), 0 picks argmin (QAP).  Returns alpha (paper's notation:
 * the weight of P in the update). */
double oracle_step_size(const double *A, const double *B, const double *P, const double *Q, int n, int maximize,
                        double *a_out, double *b_out)
{
    size_t nn = (size_t)n * (size_t)n;
    double *E = alloc_mat(n), *AE = alloc_mat(n), *AQ = alloc_mat(n), *Bt = alloc_mat(n), *T = alloc_mat(n),
           *XB = alloc_mat(n), *Xt = alloc_mat(n);
    for (size_t t = 0; t < nn; ++t) E[t] = P[t] - Q[t];
    matmul(A, E, n, AE);
    matmul(A, Q, n, AQ);
    transpose(B, n, Bt);
    /* E B = (B^T E^T)^T */
    transpose(E, n, Xt);
    matmul(Bt, Xt, n, T);
    transpose(T, n, XB); /* XB = E B */
    double a = frob_inner(AE, XB, n);           /* tr(A^T E B E^T) = <A E, E B> */
    double b = frob_inner(AQ, XB, n);           /* tr(A^T Q B E^T) = <A Q, E B> */
    transpose(Q, n, Xt);
    matmul(Bt, Xt, n, T);
    transpose(T, n, XB); /* XB = Q B */
    b += frob_inner(AE, XB, n);                 /* tr(A^T E B Q^T) = <A E, Q B> */

    double alpha;
    if (maximize) {
        if (a < 0.0) {
            alpha = -b / (2.0 * a);
            if (alpha < 0.0) alpha = 0.0;
            if (alpha > 1.0) alpha = 1.0;
        } else {
            /* convex in alpha: the maximum is at an end point; phi(0) - phi(1) = -(a + b) */
            alpha = (a + b < 0.0) ? 0.0 : 1.0;
        }
    } else {
        if (a > 0.0) {
            alpha = -b / (2.0 * a);
            if (alpha < 0.0) alpha = 0.0;
            if (alpha > 1.0) alpha = 1.0;
        } else {
            alpha = (a + b > 0.0) ? 0.0 : 1.0;
        }
    }
    if (a_out) *a_out = a;
    if (b_out) *b_out = b;
    free(E); free(AE); free(AQ); free(Bt); free(T); free(XB); free(Xt);
    return alpha;
}

/* ------------------------------------------------------------------ */
/* linear assignment: Hungarian method with potentials (Kuhn-Munkres,  */
/* in its shortest-augmenting-path form, O(n^3))                        */
/* ------------------------------------------------------------------ */

/* Minimises sum_i C[i][perm[i]] over permutations.  Rows are inserted one
 * at a time; for each new row a Dijkstra search over reduced costs
 * C_ij - u_i - v_j >= 0 grows a tree of tight edges until it reaches a free
 * column, the potentials are shifted by the tree distances, and the matching
 * is flipped along the path.  Writes perm and the final potentials (u, v may
 * be NULL).  Returns the optimal cost. */
double oracle_lap_min(const double *C, int n, int *perm, double *u_out, double *v_out)
{
    /* column index n is a virtual root column that holds the row being inserted */
    double *u = (double *)calloc((size_t)n, sizeof(double));
    double *v = (double *)calloc((size_t)n + 1, sizeof(double));
    double *dist = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    int *owner = (int *)malloc(sizeof(int) * ((size_t)n + 1)); /* owner[j] = row matched to column j, -1 free */
    int *pred = (int *)malloc(sizeof(int) * ((size_t)n + 1));  /* previous column on the shortest path */
    char *in_tree = (char *)malloc((size_t)n + 1);
    for (int j = 0; j <= n; ++j) owner[j] = -1;

    for (int r = 0; r < n; ++r) {
        const int root = n;
        owner[root] = r;
        for (int j = 0; j <= n; ++j) { dist[j] = INFINITY; in_tree[j] = 0; pred[j] = -1; }
        int col = root;
        for (;;) {
            in_tree[col] = 1;
            int row = owner[col];
            double best = INFINITY;
            int best_col = -1;
            for (int j = 0; j < n; ++j) {
                if (in_tree[j]) continue;
                double reduced = C[IDX(row, j, n)] - u[row] - v[j];
                if (reduced < dist[j]) { dist[j] = reduced; pred[j] = col; }
                if (dist[j] < best) { best = dist[j]; best_col = j; }
            }
            /* shift potentials so that the newly reached column becomes tight */
            for (int j = 0; j <= n; ++j) {
                if (in_tree[j]) {
                    u[owner[j]] += best;
                    v[j] -= best;
                } else {
                    dist[j] -= best;
                }
            }
            col = best_col;
            if (owner[col] < 0) break; /* reached a free column: augment */
        }
        while (col != root) {
            int prev = pred[col];
            owner[col] = owner[prev];
            col = prev;
        }
    }
    double cost = 0.0;
    for (int j = 0; j < n; ++j) perm[owner[j]] = j;
    for (int i = 0; i < n; ++i) cost += C[IDX(i, perm[i], n)];
    if (u_out) memcpy(u_out, u, sizeof(double) * (size_t)n);
    if (v_out) memcpy(v_out, v, sizeof(double) * (size_t)n);
    free(u); free(v); free(dist); free(owner); free(pred); free(in_tree);
    return cost;
}

/* maximize = 1: argmax_{perm} sum_i C[i][perm i] (Alg. 1/3 return line);
 * 0: argmin.  Returns the optimal objective in the caller's sense. */
double oracle_lap(const double *C, int n, int maximize, int *perm)
{
    if (!maximize) return oracle_lap_min(C, n, perm, NULL, NULL);
    size_t nn = (size_t)n * (size_t)n;
    double *neg = (double *)malloc(sizeof(double) * nn);
    for (size_t t = 0; t < nn; ++t) neg[t] = -C[t];
    oracle_lap_min(neg, n, perm, NULL, NULL);
    free(neg);
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += C[IDX(i, perm[i], n)];
    return s;
}

/* Same on a single-precision matrix (values converted exactly to FP64). */
double oracle_lap_f32(const float *C, int n, int maximize, int *perm)
{
    size_t nn = (size_t)n * (size_t)n;
    double *D = (double *)malloc(sizeof(double) * nn);
    for (size_t t = 0; t < nn; ++t) D[t] = (double)C[t];
    double s = oracle_lap(D, n, maximize, perm);
    free(D);
    return s;
}

/* Cost of a given assignment on a single-precision matrix, summed in FP64 in
 * row order (the fixed order used whenever two assignments are compared). */
double oracle_assignment_cost_f32(const float *C, int n, const int *perm)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += (double)C[IDX(i, perm[i], n)];
    return s;
}

/* LP duality check for the maximisation LAP on a single-precision matrix:
 * given an assignment perm and duals (u, v), reports
 *   max_violation = max_{i,j} (C_ij - u_i - v_j)    (<= 0 when the duals are feasible)
 *   gap           = sum_i u_i + sum_j v_j - sum_i C[i][perm i]   (>= 0 by weak duality)
 * A feasible dual with zero gap certifies that perm is optimal. */
void oracle_lap_certificate_f32(const float *C, int n, const int *perm, const double *u, const double *v,
                                double *max_violation, double *gap)
{
    double viol = -INFINITY;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double d = (double)C[IDX(i, j, n)] - u[i] - v[j];
            if (d > viol) viol = d;
        }
    double dual = 0.0, primal = 0.0;
    for (int i = 0; i < n; ++i) dual += u[i];
    for (int j = 0; j < n; ++j) dual += v[j];
    for (int i = 0; i < n; ++i) primal += (double)C[IDX(i, perm[i], n)];
    *max_violation = viol;
    *gap = dual - primal;
}

/* ------------------------------------------------------------------ */
/* random starting points (Sec. 3.4)                                    */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood 2014): the k-th output of the generator
 * seeded with `seed` is the mix of seed + (k + 1) * 0x9E3779B97F4A7C15. */
uint64_t oracle_splitmix64_output(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The paper's random start P0 = (J + K) / 2, J = 11^T / n, with K the
 * Sinkhorn-Knopp scaling of the noise U_ij = ((output k >> 40) + 1) / 2^24,
 * k = (q << 32) | (i n + j), for problem q. */
void oracle_random_start(int n, uint64_t seed, int q, double *P0)
{
    double *U = alloc_mat(n), *K = alloc_mat(n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            uint64_t k = ((uint64_t)q << 32) | (uint64_t)((uint32_t)i * (uint32_t)n + (uint32_t)j);
            U[IDX(i, j, n)] = (double)((oracle_splitmix64_output(seed, k) >> 40) + 1u) / 16777216.0;
        }
    oracle_sinkhorn_knopp(U, n, 1e-12, 100000, NULL, K, NULL, NULL, NULL);
    for (size_t t = 0; t < (size_t)n * (size_t)n; ++t) P0[t] = 0.5 / (double)n + 0.5 * K[t];
    free(U); free(K);
}

/* ------------------------------------------------------------------ */
/* learned warm start: node features and the network (no counterpart in */
/* the paper; written from their definitions)                           */
/* ------------------------------------------------------------------ */

static void line_stats(const double *x, int n, int stride, double scale, double *mean, double *mx, double *sd,
                       double *mn)
{
    double s = 0.0, s2 = 0.0, hi = -INFINITY, lo = INFINITY;
    for (int k = 0; k < n; ++k) {
        double v = x[(size_t)k * (size_t)stride] * scale;
        s += v;
        s2 += v * v;
        if (v > hi) hi = v;
        if (v < lo) lo = v;
    }
    *mean = s / n;
    double var = s2 / n - (*mean) * (*mean);
    *sd = var > 0.0 ? sqrt(var) : 0.0;
    *mx = hi;
    *mn = lo;
}

/* feats (2n x 8): nodes 0..n-1 are the rows of G, n..2n-1 its columns:
 * degree / mean degree, 2-hop degree / its mean, mean, max, std, min of the
 * node's line of G over eps, side, ln(n)/10. */
void oracle_dual_features(const double *G, const double *A, const double *B, int n, double eps, double *feats)
{
    double *deg = (double *)calloc(2 * (size_t)n, sizeof(double));
    double *hop = (double *)calloc(2 * (size_t)n, sizeof(double));
    double sdA = 0, sdB = 0, shA = 0, shB = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) { deg[i] += A[IDX(i, j, n)]; deg[n + i] += B[IDX(i, j, n)]; }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) { hop[i] += A[IDX(i, k, n)] * deg[k]; hop[n + i] += B[IDX(i, k, n)] * deg[n + k]; }
    for (int i = 0; i < n; ++i) { sdA += deg[i]; sdB += deg[n + i]; shA += hop[i]; shB += hop[n + i]; }
    for (int v = 0; v < 2 * n; ++v) {
        int side = v >= n, idx = side ? v - n : v;
        double *o = feats + (size_t)v * 8;
        double md = (side ? sdB : sdA) / n, mh = (side ? shB : shA) / n;
        o[0] = md > 0 ? deg[v] / md : 0.0;
        o[1] = mh > 0 ? hop[v] / mh : 0.0;
        if (!side) line_stats(G + IDX(idx, 0, n), n, 1, 1.0 / eps, &o[2], &o[3], &o[4], &o[5]);
        else line_stats(G + idx, n, n, 1.0 / eps, &o[2], &o[3], &o[4], &o[5]);
        o[6] = side;
        o[7] = log((double)n) / 10.0;
    }
    free(deg); free(hop);
}

/* The warm-start network y = w2 . tanh(W1 x + b1) + b2 (hidden width 64, 8
 * inputs; packed parameters W1 [64][8] at 0, b1 at 512, w2 at 576, b2 at 640)
 * and the mean squared error L = (1/N) sum_s (y_s - t_s)^2 with its gradient
 * by the chain rule.  y_out (nullable) gets the outputs.  Returns L. */
double oracle_mlp_loss_grad(const double *prm, const double *x, const double *t, int N, double *grad, double *y_out)
{
    double L = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * 641);
    for (int s = 0; s < N; ++s) {
        const double *xs = x + (size_t)s * 8;
        double h[64], y = prm[640];
        for (int k = 0; k < 64; ++k) {
            double z = prm[512 + k];
            for (int d = 0; d < 8; ++d) z += prm[k * 8 + d] * xs[d];
            h[k] = tanh(z);
            y += prm[576 + k] * h[k];
        }
        if (y_out) y_out[s] = y;
        double e = y - t[s];
        L += e * e / N;
        if (grad) {
            double dy = 2.0 * e / N;
            grad[640] += dy;
            for (int k = 0; k < 64; ++k) {
                grad[576 + k] += dy * h[k];
                double dz = dy * prm[576 + k] * (1.0 - h[k] * h[k]);
                grad[512 + k] += dz;
                for (int d = 0; d < 8; ++d) grad[k * 8 + d] += dz * xs[d];
            }
        }
    }
    return L;
}

/* ------------------------------------------------------------------ */
/* brute force over all n! permutations (n <= 10)                       */
/* ------------------------------------------------------------------ */

/* Advances perm to the next permutation in lexicographic order; returns 0
 * after the last one. */
static int next_permutation(int *p, int n)
{
    int i = n - 2;
    while (i >= 0 && p[i] >= p[i + 1]) --i;
    if (i < 0) return 0;
    int j = n - 1;
    while (p[j] <= p[i]) --j;
    int t = p[i]; p[i] = p[j]; p[j] = t;
    for (int a = i + 1, b = n - 1; a < b; ++a, --b) { t = p[a]; p[a] = p[b]; p[b] = t; }
    return 1;
}

/* Best sum_i C[i][perm i] over all permutations; counts how many attain it
 * (exact comparison) and returns the first optimum found in perm_best. */
double oracle_brute_lap(const double *C, int n, int maximize, int *perm_best, int *n_optimal)
{
    int p[16];
    for (int i = 0; i < n; ++i) p[i] = i;
    double best = maximize ? -INFINITY : INFINITY;
    int count = 0;
    do {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += C[IDX(i, p[i], n)];
        int better = maximize ? (s > best) : (s < best);
        if (better) { best = s; count = 1; memcpy(perm_best, p, sizeof(int) * (size_t)n); }
        else if (s == best) ++count;
    } while (next_permutation(p, n));
    if (n_optimal) *n_optimal = count;
    return best;
}

/* Best f(Pi) = sum_ij A_ij B[pi i][pi j] over all permutations (eq. QAP / GM). */
double oracle_brute_qap(const double *A, const double *B, int n, int maximize, int *perm_best)
{
    int p[16];
    for (int i = 0; i < n; ++i) p[i] = i;
    double best = maximize ? -INFINITY : INFINITY;
    do {
        double s = oracle_objective_perm(A, B, n, p);
        int better = maximize ? (s > best) : (s < best);
        if (better) { best = s; memcpy(perm_best, p, sizeof(int) * (size_t)n); }
    } while (next_permutation(p, n));
    return best;
}

/* ------------------------------------------------------------------ */
/* GOAT (Alg. 3) and FAQ (Alg. 1)                                       */
/* ------------------------------------------------------------------ */

typedef struct {
    int iters;            /* Frank-Wolfe iterations run                          */
    int converged;        /* 1 if ||P_new - P||_F / sqrt(n) < tol ended the loop */
    double objective;     /* f at the returned permutation                      */
} oracle_stats;

/* Runs GOAT (use_lap = 0) or FAQ (use_lap = 1) on A, B, optionally seeded.
 *   m             seeds: vertex i of A is known to match vertex i of B for i < m
 *                 (Fishkind et al.'s seeded graph matching, which Sec. 4 applies
 *                 to both methods).  The iterate keeps the form P = I_m (+) P22,
 *                 each direction is found on the unseeded block of the gradient
 *                 (the derivative of f with respect to P22) and padded with I_m,
 *                 and the final assignment is solved on that block; m = 0 is
 *                 the unseeded method.
 *   P0            initial doubly stochastic P (NULL: I_m (+) the barycenter of
 *                 the unseeded block, 11^T / (n - m)); with seeds it must have the
 *                 I_m (+) P22 form
 *   eps_rel       entropic weight per iteration: eps = eps_rel * max|grad f(P)| over
 *                 the unseeded block
 *   max_iter, tol Frank-Wolfe limits;  sk_tol, sk_max_iter  Sinkhorn limits
 *   maximize      1: graph matching (max f), 0: QAP (min f)
 *   project_on_grad  0: final LAP on P (closest permutation); 1: on grad f(P)
 * Outputs perm (perm[i] = vertex of B matched to vertex i of A), the final
 * relaxed P (nullable), per-iteration step sizes in the paper's notation and
 * Sinkhorn iteration counts (nullable, max_iter entries each). */
int oracle_goat_seeded(const double *A, const double *B, int n, int m, const double *P0, double eps_rel,
                       int max_iter, double tol, double sk_tol, int sk_max_iter, int use_lap, int maximize,
                       int project_on_grad, int *perm, double *P_out, double *alpha_trace, int *sk_iters_trace,
                       oracle_stats *stats)
{
    if (m < 0 || m > n) return -1;
    size_t nn = (size_t)n * (size_t)n;
    int n2 = n - m; /* unseeded vertices */
    double *P = alloc_mat(n), *grad = alloc_mat(n), *Q = alloc_mat(n);
    double *M = alloc_mat(n2 > 0 ? n2 : 1), *Q2 = alloc_mat(n2 > 0 ? n2 : 1);
    int *qperm = (int *)malloc(sizeof(int) * (size_t)(n2 > 0 ? n2 : 1));
    if (P0) {
        memcpy(P, P0, sizeof(double) * nn);
    } else {
        for (int i = 0; i < m; ++i) P[IDX(i, i, n)] = 1.0;
        for (int i = m; i < n; ++i)
            for (int j = m; j < n; ++j) P[IDX(i, j, n)] = 1.0 / (double)n2;
    }

    int it = 0, converged = 0;
    while (n2 > 0 && it < max_iter) {
        /* step 1: gradient */
        oracle_gradient(A, B, P, n, grad);
        /* step 2: direction on the unseeded block.  Maximising tr(Q^T grad) is the
         * rLAP with cost -grad. */
        double gmax = 0.0;
        for (int i = 0; i < n2; ++i)
            for (int j = 0; j < n2; ++j) {
                double v = grad[IDX(m + i, m + j, n)];
                M[IDX(i, j, n2)] = maximize ? -v : v;
                if (fabs(v) > gmax) gmax = fabs(v);
            }
        int sk_it = 0;
        if (use_lap) {
            oracle_lap_min(M, n2, qperm, NULL, NULL);
            memset(Q2, 0, sizeof(double) * (size_t)n2 * (size_t)n2);
            for (int i = 0; i < n2; ++i) Q2[IDX(i, qperm[i], n2)] = 1.0;
        } else {
            double eps = eps_rel * gmax;
            if (eps <= 0.0) eps = 1.0; /* grad == 0: every doubly stochastic Q is optimal */
            sk_it = oracle_lot(M, n2, eps, sk_tol, sk_max_iter, NULL, Q2, NULL, NULL, NULL);
        }
        memset(Q, 0, sizeof(double) * nn);
        for (int i = 0; i < m; ++i) Q[IDX(i, i, n)] = 1.0;
        for (int i = 0; i < n2; ++i)
            for (int j = 0; j < n2; ++j) Q[IDX(m + i, m + j, n)] = Q2[IDX(i, j, n2)];
        /* step 3: step size (alpha weights P) */
        double alpha = oracle_step_size(A, B, P, Q, n, maximize, NULL, NULL);
        /* step 4: update, and the stopping test on the change of P */
        double change = 0.0;
        for (size_t t = 0; t < nn; ++t) {
            double pn = alpha * P[t] + (1.0 - alpha) * Q[t];
            double d = pn - P[t];
            change += d * d;
            P[t] = pn;
        }
        if (alpha_trace) alpha_trace[it] = alpha;
        if (sk_iters_trace) sk_iters_trace[it] = sk_it;
        ++it;
        if (sqrt(change) / sqrt((double)n) < tol) { converged = 1; break; }
    }

    /* projection onto the permutations that keep the seeds */
    for (int i = 0; i < m; ++i) perm[i] = i;
    if (n2 > 0) {
        const double *X = P;
        if (project_on_grad) {
            oracle_gradient(A, B, P, n, grad);
            X = grad;
        }
        for (int i = 0; i < n2; ++i)
            for (int j = 0; j < n2; ++j) M[IDX(i, j, n2)] = X[IDX(m + i, m + j, n)];
        oracle_lap(M, n2, project_on_grad ? maximize : 1, qperm);
        for (int i = 0; i < n2; ++i) perm[m + i] = m + qperm[i];
    }
    if (P_out) memcpy(P_out, P, sizeof(double) * nn);
    if (stats) {
        stats->iters = it;
        stats->converged = converged;
        stats->objective = oracle_objective_perm(A, B, n, perm);
    }
    free(P); free(grad); free(M); free(Q); free(Q2); free(qperm);
    return 0;
}

/* The unseeded method (m = 0). */
int oracle_goat(const double *A, const double *B, int n, const double *P0, double eps_rel, int max_iter,
                double tol, double sk_tol, int sk_max_iter, int use_lap, int maximize, int project_on_grad,
                int *perm, double *P_out, double *alpha_trace, int *sk_iters_trace, oracle_stats *stats)
{
    return oracle_goat_seeded(A, B, n, 0, P0, eps_rel, max_iter, tol, sk_tol, sk_max_iter, use_lap, maximize,
                              project_on_grad, perm, P_out, alpha_trace, sk_iters_trace, stats);
}
