// goat_internal.h -- declarations shared by the translation units of libgoat.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/goat.h"

namespace goat {

enum { GEMM_OUT_F32 = 0, GEMM_OUT_BF16_TERMS = 1 };

// One "D = scale * X Y^T" launch (see goat_gemm.cu).  X: x_rows rows, row
// stride x_stride, read at k mod kx_period; Y: y_rows rows, row stride
// y_stride, K extent k_total.  Both BF16, 16-byte aligned, K-major.
struct GemmCall {
    const void *X;           // BF16, or E4M3 bytes when fp8
    int x_rows;
    long long x_stride;      // elements
    int kx_period;
    const void *Y;
    int y_rows;
    long long y_stride;
    int k_total;             // multiple of 64 (BF16) or 128 (E4M3) elements
    int M, N;
    int fp8;                 // operands E4M3 (kind::f8f6f4), else BF16 (kind::f16)
    float scale;
    const float *scale_dev;  // device factor on top of scale (nullable)
    int mode;
    float *out_f32;
    long long ld_out;
    __nv_bfloat16 *out_b16;
    int out_terms;
    long long term_stride;
    long long row_stride;
    int out_rows, out_cols;
    int *err;
    int k_begin;             // this launch covers K positions [k_begin, k_begin + k_total) (multiple of the stage K)
    const float *addend;     // FP32 matrix added to the result in the epilogue (nullable; may be out_f32 itself)
    long long ld_addend;
    int addend_cols;         // columns of the addend (later output columns add nothing)
    // mixed launch (X8 non-null): after the BF16 K range above, K8 more positions of
    // E4M3 operands X8 (period kx8_period, row stride x8_stride) and Y8 (row stride
    // y8_stride) into the same accumulator; BF16 only above, no k_begin or addend
    const void *X8;
    long long x8_stride;
    int kx8_period;
    const void *Y8;
    long long y8_stride;
    int k8_total;            // multiple of 128
};

int gemm_xyT(const GemmCall &c, cudaStream_t stream);

// Grouped mode: many independent problems in one launch.  X and Y are stacked
// row-wise (one 2-D tensor map each, inner extent k_extent); a problem's tiles
// read rows from its own offsets (rows past its end belong to the next problem
// and are masked on store).
struct GemmGroupDesc {
    long long x_row0, y_row0;  // first row of the problem in the stacked X / Y
    int num_kb;                // K blocks: ceil(n / 64)
    int M, N;                  // valid output rows / columns
    int out_cols;              // columns written; [N, out_cols) are written as zero
    int pad;
    float *out_f32;
    long long ld_out;
    __nv_bfloat16 *out_b16;
    long long row_stride;
};

struct GemmGroupCall {
    const __nv_bfloat16 *X;
    long long x_rows, x_stride;
    const __nv_bfloat16 *Y;
    long long y_rows, y_stride;
    int k_extent;
    const int4 *items;
    int num_items;
    const GemmGroupDesc *descs;
    float scale;
    int mode;
    int *err;
};

int gemm_grouped(const GemmGroupCall &c, cudaStream_t stream);

// Kernel launches issued by this host thread (every launch site reports here).
void note_launches(int k);
long long launches_so_far();

struct DevState;

// goat_fw.cu
// An adjacency matrix in device memory: element type GOAT_DTYPE_*, leading dimension ld.
struct AdjView {
    const void *p;
    long long ld;
    int dtype;
};
// The rows x cols window at (r0, c0) -> operand rows of `width` elements (zero
// beyond cols), `stride` elements apart; deg (nullable) gets the window's row sums.
int adj_to_bf16(const AdjView &v, int r0, int c0, int rows, int cols, __nv_bfloat16 *dst, int width, long long stride,
                float *deg, cudaStream_t s);
int adj_to_e4m3(const AdjView &v, int r0, int c0, int rows, int cols, uint8_t *dst, int width, long long stride,
                cudaStream_t s);
// The same for the window's transpose (dst row c = window column c, width >= rows).
int adj_to_bf16_t(const AdjView &v, int r0, int c0, int rows, int cols, __nv_bfloat16 *dst, int width,
                  long long stride, cudaStream_t s);
int adj_to_e4m3_t(const AdjView &v, int r0, int c0, int rows, int cols, uint8_t *dst, int width, long long stride,
                  cudaStream_t s);
int adj_col_sums(const AdjView &v, int r0, int c0, int rows, int cols, float *out, cudaStream_t s);
// The split intermediate's lo term -> E4M3 (and its hi term scaled to match) for the
// second product of GOAT_PREC_BF16_SPLIT8; inv_scale (device) receives 1/s.
int split_lo_to_e4m3(__nv_bfloat16 *C1, int rows, int ld, int parts, uint8_t *C8, int w8, unsigned *amax_bits,
                     float *inv_scale, cudaStream_t s);
int bf16_to_e4m3(const __nv_bfloat16 *X, int rows, int ld_src, uint8_t *X8, int ld8, unsigned *amax_bits,
                 float *inv_scale, cudaStream_t s);
int count_asym(const void *A, int dtype, int n, int *count_dev, cudaStream_t s);
void f32_to_terms(const float *X, int n, long long ldx, __nv_bfloat16 *Xb, int ld16, int terms, cudaStream_t s);
// G = scale (dA dB^T + eA eB^T) [+ C], P = J (nullable); eA/eB and C nullable.
void barycenter(const float *dA, const float *dB, const float *eA, const float *eB, int n, float scale,
                const float *C, float *G, float *P, DevState *st, cudaStream_t s);
void add_f32(float *X, const float *C, long long total, cudaStream_t s);  // X, C 16-byte aligned
void seed_perm(int32_t *perm, int n, int m, cudaStream_t s);
void embed_block(const float *P22, int n, int m, float *out, cudaStream_t s);
void absmax(const float *X, long long total, unsigned *out, cudaStream_t s);
int ls_blocks(int n);
// Q for the step size and the update: from the LOT duals f, g (non-null: recomputed
// in FP32 from G, Q_ij = 2^(c (f_i + g_j - G_ij)) with st->c), else the BF16 split
// terms Qb, else FP32 Qf.
void line_search(const float *G, const float *GQ, const float *P, const __nv_bfloat16 *Qb, int ldq, int terms,
                 const float *Qf, const float *f, const float *g, int n, double *partial, DevState *st,
                 cudaStream_t s);
void fw_update(float *P, float *G, const float *GQ, const __nv_bfloat16 *Qb, int ldq, int terms, const float *Qf,
               const float *f, const float *g, int n, const DevState *st, float alpha_value, unsigned *gmax_out,
               cudaStream_t s);
void fw_roll(DevState *st, cudaStream_t s);
// Blocks of the FP64 objective sums (a fixed grid, so the sums are reproducible);
// objective() takes 3 * kObjBlocks doubles of scratch in fpart, and fsum, fA, fB
// must be consecutive doubles.
constexpr int kObjBlocks = 512;
int objective(const void *A, const void *B, int dtype, int n, const int32_t *perm, unsigned long long *isum,
              double *fsum, unsigned long long *nA, unsigned long long *nB, double *fA, double *fB, int *bad,
              double *fpart, cudaStream_t s);

// goat_sinkhorn.cu
// Smallest n the fused single-read Sinkhorn iteration runs at (below it the row and
// column passes run, which are faster there: the fused form's cost per row is
// mostly fixed); sinkhorn_partial_elems covers both.
constexpr int kSkFusedMinN = 20480;
long long sinkhorn_partial_elems(int n);
void sinkhorn_begin(DevState *st, float eps, float tol, float *g_zero, int n, cudaStream_t s);
int sinkhorn_solve(const float *G, int n, long long ld, float *f, float *g, double *partial, DevState *st,
                   int max_iter, int check_every, int *host_flag, cudaStream_t s);
void sinkhorn_queue_fixed(const float *G, int n, long long ld, float *f, float *g, double *partial, DevState *st,
                          int max_iter, cudaStream_t s);
// FAQ's first direction at the barycenter, exactly: perm pairs the k-th largest FP64
// degree of A with the k-th largest of B (grad f(J) is rank one).  scratch holds
// rearrangement_scratch_bytes(n) bytes (8-byte aligned).
size_t rearrangement_scratch_bytes(int n);
int rearrangement_perm(const void *A, const void *B, int dtype, int n, int maximize, void *scratch, int32_t *perm,
                       cudaStream_t s);
// Zeroes the operand buffer and writes the permutation matrix of perm into it (FAQ's Q).
int write_perm_q(const int32_t *perm, int n, __nv_bfloat16 *Qb, int ldq, int terms, cudaStream_t s);
void write_q(const float *G, int n, long long ld, const float *f, const float *g, const DevState *st,
             __nv_bfloat16 *Qb, int ldq, int terms, float *Qf, long long ldf, cudaStream_t s);

// goat_warmstart.cu
size_t mlp_warm_start_scratch_bytes(int n);
int mlp_warm_start_g(const float *G, const void *A, const void *B, int n, int dtype, float eps,
                     const __nv_bfloat16 *w, float *g, float *scratch, cudaStream_t s);

// goat_lap.cu
int lap_chunks(int n);
size_t lap_bytes(int n, int nchunks);
// Controls of the projection's schedule (negative: the built-in default).
struct LapControl {
    int max_rounds;        // Jacobi rounds over all phases
    int head_rounds;       // Jacobi rounds per phase before the sequential steps
    long long tail_bids;   // Gauss-Seidel bids per phase
    long long tail_stall;  // bids without the queue shrinking that end the Gauss-Seidel tail
    long long sap_pops;    // row scans the augmenting-path searches may do per phase (0: none)
    int sap_step;          // columns a search settles per parallel step
    int head_stall;        // Jacobi rounds without fewer bidders that end a phase's rounds
    int sap_every_phase;   // 1: the searches complete every phase; 0: only the last
};
void lap_default_control(LapControl *c);
struct LapReport {
    int phases, rounds, sap_rows, filled;
    long long tail_bids, sap_pops, sap_epochs;
    double ms_head, ms_tail, ms_sap;
};
int lap_solve(const float *M, int n, int maximize, int32_t *perm_out, void *lap_ws, DevState *st,
              const LapControl &ctl, double *cost_dev, int *host_pinned, double *gap_host, LapReport *rep,
              cudaStream_t s);

}  // namespace goat
