// goat_api.cu -- the C ABI of libgoat and the Frank-Wolfe driver of GOAT (Alg. 3).
//
// goat_match runs, stream-ordered and with one host synchronisation per
// Frank-Wolfe step (the stop test) plus the Sinkhorn polls:
//   operands   A, B -> BF16 (exact for 0/1), degrees, symmetry check; with seeds
//              the unseeded block and the seeds' constant share of the gradient
//   init       P = J and G = -grad f(J) in closed form from the degrees, or G from the GEMMs
//   loop       eps = eps_rel max|G|; Sinkhorn (warm or cold duals); Q -> BF16 terms;
//              C1 = B Q^T; G_Q = -2 A C1^T (directed graphs: -(A Q B^T + A^T Q B));
//              line search (b, a, alpha, stop test);
//              P += alpha (Q - P), G += alpha (G_Q - G)   (grad f is linear)
//   project    auction + certification on P (or on grad f(P))
//   objective  f(perm) and the disagreement count, exact for 0/1 inputs
//
// Minimising f (QAP, maximize = 0) runs the same iteration on G = +grad f: every
// step maximises the linearisation of -f.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

enum : int { NEED_GEMM = 1, NEED_FW = 2, NEED_SK = 4, NEED_LAP = 8, NEED_HOSTCOPY = 16 };

// Shape of one solve: n_full vertices, the first m of them seeds (vertex i of A
// known to match vertex i of B), so the iteration runs on the n = n_full - m
// unseeded ones; dir = 1 for general (directed) graphs, whose gradient needs four
// products instead of two.
struct Shape {
    int n_full, m, dir;
};

struct Plan {
    size_t state, A16, B16, Xq, C1, GQ, P, G, f, g, deg, partial, lap, perm, Ad, Bd, Id, cost, objpart, mlp, rearr;
    size_t A8, B8, Q8, C8, f8s;  // E4M3 operands and their scales (8-bit form)
    size_t SX, SY, Cs;           // seeded: the seed term's BF16 operands and its FP32 value
    size_t total;
    int n, m, n_full, dir;
    int ld;     // K extent of one operand part (multiple of 64; of 128 for directed graphs)
    int terms;  // BF16 terms of Q (2 in the FP32-accurate form)
    int tc;     // BF16 terms of C1 (2 in the FP32-accurate and the split-intermediate forms)
    bool q8;    // first product in E4M3 (B and Q), second in BF16 over C1's two terms
    bool lo8;   // second product: C1's hi term in BF16, its lo term in E4M3 against A in E4M3
    int ld8;    // E4M3 row width of Q (multiple of 128; equal to ld for directed graphs)
    int parts;  // 1, or 2 for directed graphs: A16 = [A | A^T], B16 = [B | B^T], C1 = [C1 | C1']
    int ldm;    // K extent of the seed term (multiple of 64)
    bool fp8;
};

static Plan make_plan(const Shape &sh, int dtype, int precision, int need) {
    Plan w;
    std::memset(&w, 0, sizeof(w));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (size_t)round_up((int64_t)std::max<size_t>(bytes, 1), 256);
        return o;
    };
    const int n = sh.n_full - sh.m;
    const size_t nn = (size_t)n * (size_t)n;
    w.n = n;
    w.m = sh.m;
    w.n_full = sh.n_full;
    w.dir = sh.dir;
    w.parts = sh.dir ? 2 : 1;
    w.ld = sh.dir ? (int)round_up(n, 128) : operand_ld(n);
    w.ld8 = (int)round_up(n, 128);  // an E4M3 stage holds 128 elements of K
    w.terms = precision == GOAT_PREC_FP32 ? 2 : 1;
    w.tc = (precision == GOAT_PREC_FP32 || precision == GOAT_PREC_BF16_SPLIT || precision == GOAT_PREC_FP8_SPLIT ||
            precision == GOAT_PREC_BF16_SPLIT8)
               ? 2
               : 1;
    w.q8 = precision == GOAT_PREC_FP8_SPLIT;  // 8-bit first product only
    w.fp8 = precision == GOAT_PREC_FP8;
    w.lo8 = precision == GOAT_PREC_BF16_SPLIT8;  // second product's low term in E4M3
    w.ldm = sh.m > 0 ? (int)round_up((int64_t)sh.m * w.parts, 64) : 0;
    w.state = take(sizeof(DevState));
    w.cost = take(16 * sizeof(double));  // [0,3) u64 sums, [3,6) f64 sums, [6] assignment cost, [7,10) LAP bound
    w.objpart = take(3 * kObjBlocks * sizeof(double));  // per-block partials of the FP64 objective sums
    if (need & (NEED_GEMM | NEED_FW)) {
        w.A16 = take((size_t)n * w.parts * w.ld * 2);
        w.B16 = take((size_t)n * w.parts * w.ld * 2);
        w.Xq = take((size_t)n * w.terms * w.ld * 2);
        w.C1 = take((size_t)n * w.parts * w.tc * w.ld * 2);
        if (w.fp8 || w.q8) {
            const size_t row8 = sh.dir ? 2 * (size_t)w.ld : (size_t)w.ld8;
            w.A8 = take((size_t)n * row8);
            w.B8 = take((size_t)n * row8);
            w.Q8 = take((size_t)n * w.ld8);
            w.C8 = take((size_t)n * row8);
            w.f8s = take(4 * sizeof(float));  // [0] max|Q| bits, [1] 1/s_Q, [2] max|C1| bits, [3] 1/s_C1
        }
        if (w.lo8) {
            // A in E4M3 and the low term of C1 in E4M3, both K-major over [A | A^T]
            const size_t row8 = sh.dir ? 2 * (size_t)w.ld : (size_t)w.ld8;
            w.A8 = take((size_t)n * row8);
            w.C8 = take((size_t)n * row8);
            w.f8s = take(4 * sizeof(float));  // [2] max|C1| bits, [3] 1/s
        }
        w.deg = take((size_t)4 * n * 4);  // out-degrees of A, B, in-degrees of A, B (directed)
        if (sh.m > 0) {
            w.SX = take((size_t)n * w.ldm * 2);
            w.SY = take((size_t)n * w.ldm * 2);
            w.Cs = take(nn * 4);
        }
    }
    if (need & NEED_FW) {
        w.GQ = take(nn * 4);
        w.P = take(nn * 4);
        w.G = take(nn * 4);
        w.f = take((size_t)n * 4);
        w.g = take((size_t)n * 4);
        // the network's features (only plain solves take network weights)
        if (sh.m == 0 && !sh.dir) w.mlp = take(mlp_warm_start_scratch_bytes(n));
        w.rearr = take(rearrangement_scratch_bytes(n));
    }
    if (need & (NEED_SK | NEED_FW)) {
        const size_t sk = (size_t)sinkhorn_partial_elems(std::max(n, 1)) * 8;
        const size_t ls = (size_t)ls_blocks(std::max(n, 1)) * 3 * 8;
        w.partial = take(std::max(sk, ls));
    }
    if (need & (NEED_LAP | NEED_FW)) {
        w.lap = take(lap_bytes(std::max(n, 1), lap_chunks(n)));
        w.perm = take((size_t)sh.n_full * 4);
    }
    if (need & NEED_HOSTCOPY) {
        const size_t es = dtype == GOAT_DTYPE_U8 ? 1 : 4;
        const size_t nf2 = (size_t)sh.n_full * (size_t)sh.n_full;
        w.Ad = take(nf2 * es);
        w.Bd = take(nf2 * es);
        w.Id = take(nf2 * 4);
    }
    w.total = off;
    return w;
}

// ---------------------------------------------------------------- helpers

static thread_local long long t_launches = 0;
void note_launches(int k) { t_launches += k; }
long long launches_so_far() { return t_launches; }

static int device_ok() {
    static int status = 1;  // 1 = unknown
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (status != 1) return status;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return GOAT_ERR_CUDA;  // not cached: the context may come later
    }
    status = (prop.major == 10 && prop.minor == 3) ? GOAT_OK : GOAT_ERR_UNSUPPORTED;
    return status;
}

// Pinned host words for polling device flags (one set per host thread).
static int *pinned_words() {
    thread_local int *p = nullptr;
    if (!p) {
        if (cudaMallocHost(&p, 64 * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    return p;
}

struct Scratch {
    uint8_t *base = nullptr;
    bool owned = false;
    cudaStream_t s = 0;
    int acquire(void *user, size_t user_bytes, size_t need, cudaStream_t stream) {
        s = stream;
        if (user) {
            if (user_bytes < need) return GOAT_ERR_OUT_OF_MEMORY;
            if (reinterpret_cast<uintptr_t>(user) & 255) return GOAT_ERR_INVALID_ARG;
            base = (uint8_t *)user;
            return GOAT_OK;
        }
        if (cudaMallocAsync((void **)&base, need, stream) != cudaSuccess) {
            cudaGetLastError();
            return GOAT_ERR_OUT_OF_MEMORY;
        }
        owned = true;
        return GOAT_OK;
    }
    template <typename T>
    T *at(size_t off) const {
        return reinterpret_cast<T *>(base + off);
    }
    ~Scratch() {
        if (owned) cudaFreeAsync(base, s);
    }
};

__global__ void k_state_init(DevState *st, float eps_rel, int maximize, float fw_tol, int stop_n) {
    st->eps_rel = eps_rel;
    st->maximize = maximize;
    st->fw_tol = fw_tol;
    st->stop_n = stop_n;
    st->eps = 1.0f;
    st->c = 1.4426950408889634f;
}

static int init_state(DevState *st, float eps_rel, int maximize, float fw_tol, cudaStream_t s, int stop_n = 0) {
    if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess) return GOAT_ERR_CUDA;
    k_state_init<<<1, 1, 0, s>>>(st, eps_rel, maximize, fw_tol, stop_n);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? GOAT_OK : GOAT_ERR_CUDA;
}

#define GOAT_TRY(x)                    \
    do {                               \
        const int _st = (x);           \
        if (_st != GOAT_OK) return _st; \
    } while (0)

static int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GOAT_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GOAT_ERR_OUT_OF_MEMORY : GOAT_ERR_CUDA;
}

// The 8-bit form of the products: Q (BF16 in Xq) and then C1 = B Q^T (with C1' = B^T Q^T
// beside it for directed graphs) are each rounded to E4M3 under a power-of-two scale;
// the GEMM epilogues undo the scales.  scale2 is the factor of the second product.
static int gradient_fp8(const Plan &w, const Scratch &ws, float scale2, float *G_out, int *err, cudaStream_t s,
                        cudaEvent_t between) {
    const int n = w.n;
    const long long row8 = w.dir ? 2LL * w.ld : w.ld8;  // row stride of A8, B8, C8
    const long long cs = (long long)w.parts * w.ld;     // row stride of C1 (one term)
    float *sc = ws.at<float>(w.f8s);
    unsigned *amax = reinterpret_cast<unsigned *>(sc);
    GOAT_TRY(bf16_to_e4m3(ws.at<__nv_bfloat16>(w.Xq), n, w.ld, ws.at<uint8_t>(w.Q8), w.ld8, amax, sc + 1, s));
    GemmCall c1;
    std::memset(&c1, 0, sizeof(c1));
    c1.fp8 = 1;
    c1.X = ws.at<uint8_t>(w.B8);
    c1.x_rows = n;
    c1.x_stride = row8;
    c1.kx_period = w.ld8;
    c1.Y = ws.at<uint8_t>(w.Q8);
    c1.y_rows = n;
    c1.y_stride = w.ld8;
    c1.k_total = w.ld8;
    c1.M = n;
    c1.N = n;
    c1.scale = 1.0f;
    c1.scale_dev = sc + 1;
    c1.mode = GEMM_OUT_BF16_TERMS;
    c1.out_b16 = ws.at<__nv_bfloat16>(w.C1);
    c1.out_terms = 1;
    c1.term_stride = cs;
    c1.row_stride = cs;
    c1.out_rows = n;
    c1.out_cols = w.ld;  // the padding columns receive zeros
    c1.err = err;
    GOAT_TRY(gemm_xyT(c1, s));
    if (w.dir) {  // C1' = B^T Q^T beside C1 (for directed graphs ld == ld8)
        GemmCall c1t = c1;
        c1t.X = ws.at<uint8_t>(w.B8) + w.ld;
        c1t.out_b16 = ws.at<__nv_bfloat16>(w.C1) + w.ld;
        GOAT_TRY(gemm_xyT(c1t, s));
    }
    if (between) cudaEventRecord(between, s);
    GOAT_TRY(bf16_to_e4m3(ws.at<__nv_bfloat16>(w.C1), n, (int)cs, ws.at<uint8_t>(w.C8), (int)row8,
                          reinterpret_cast<unsigned *>(sc + 2), sc + 3, s));
    GemmCall c2 = c1;
    c2.X = ws.at<uint8_t>(w.A8);
    c2.x_stride = row8;
    c2.kx_period = (int)row8;
    c2.Y = ws.at<uint8_t>(w.C8);
    c2.y_stride = row8;
    c2.k_total = (int)row8;
    c2.scale = scale2;
    c2.scale_dev = sc + 3;
    c2.mode = GEMM_OUT_F32;
    c2.out_f32 = G_out;
    c2.ld_out = n;
    c2.out_b16 = nullptr;
    c2.out_cols = n;
    return gemm_xyT(c2, s);
}

// K positions per launch of the FP32-accurate form's products.  The tensor core
// accumulates in FP32 with truncation, so the error of one accumulation grows with
// its number of (nonzero) K steps; longer products are split into chunks of at
// most this length whose partial sums are added in round-to-nearest FP32 by the
// next chunk's epilogue.
constexpr int kFp32ChunkK = 16384;

// Runs the product c (mode F32 or BF16 terms) as K chunks of at most kFp32ChunkK:
// every chunk but the last writes FP32 into tmp (n x n, ld n), adding the previous
// chunk's sum; the last adds tmp and writes c's own output.  One chunk: c as is.
static int gemm_chunked(const GemmCall &c, float *tmp, int n, cudaStream_t s) {
    const int chunks = (int)ceil_div(c.k_total, kFp32ChunkK);
    if (chunks <= 1) return gemm_xyT(c, s);
    const int len = (int)round_up(ceil_div(c.k_total, chunks), 64);
    int k0 = 0;
    for (int k = 0; k0 < c.k_total; ++k) {
        const int kl = std::min(len, c.k_total - k0);
        const bool last = k0 + kl >= c.k_total;
        GemmCall ck = c;
        ck.k_begin = k0;
        ck.k_total = kl;
        if (k > 0) {
            ck.addend = tmp;
            ck.ld_addend = n;
            ck.addend_cols = n;
        }
        if (!last) {  // FP32 partial sum into tmp (in place after the first chunk)
            ck.mode = GEMM_OUT_F32;
            ck.out_f32 = tmp;
            ck.ld_out = n;
            ck.out_b16 = nullptr;
            ck.out_cols = n;
        }
        GOAT_TRY(gemm_xyT(ck, s));
        k0 += kl;
    }
    return GOAT_OK;
}

// The BF16 / FP32-accurate form, X (Q or P) already in the split-term buffer Xq:
//   C1 = B X^T [and C1' = B^T X^T],  out = scale2 * ([A | A^T] [C1 | C1']^T)
// with the split terms of X and C1 accumulated along K (X re-read per term).
static int gradient_bf16(const Plan &w, const Scratch &ws, float scale2, float *G_out, int *err, cudaStream_t s,
                         cudaEvent_t between) {
    const int n = w.n;
    // the FP32-accurate form accumulates long K in chunks; G_out holds the partial
    // sums of product 1 (it is written only by product 2)
    // (only the FP32-accurate form, terms = 2, needs the chunks: in the other forms the
    // operands' rounding is far larger than the accumulation's)
    auto run = [&](const GemmCall &c) { return w.terms > 1 ? gemm_chunked(c, G_out, n, s) : gemm_xyT(c, s); };
    const long long xs = (long long)w.parts * w.ld;         // row stride of A16, B16
    const long long cs = (long long)w.parts * w.tc * w.ld;  // row stride of C1
    GemmCall c1;
    std::memset(&c1, 0, sizeof(c1));
    c1.X = ws.at<__nv_bfloat16>(w.B16);
    c1.x_rows = n;
    c1.x_stride = xs;
    c1.kx_period = w.ld;
    c1.Y = ws.at<__nv_bfloat16>(w.Xq);
    c1.y_rows = n;
    c1.y_stride = (long long)w.terms * w.ld;
    c1.k_total = w.terms * w.ld;
    c1.M = n;
    c1.N = n;
    c1.scale = 1.0f;
    c1.mode = GEMM_OUT_BF16_TERMS;
    c1.out_b16 = ws.at<__nv_bfloat16>(w.C1);
    c1.out_terms = w.tc;
    c1.term_stride = (long long)w.parts * w.ld;  // [C1_hi | C1'_hi | C1_lo | C1'_lo]
    c1.row_stride = cs;
    c1.out_rows = n;
    c1.out_cols = w.ld;  // the padding columns receive zeros
    c1.err = err;
    if (w.q8) {
        // first product in E4M3: B exact, Q rounded under one power-of-two scale; its
        // output C1 still goes out as two BF16 terms for the BF16 second product
        float *sc = ws.at<float>(w.f8s);
        GOAT_TRY(bf16_to_e4m3(ws.at<__nv_bfloat16>(w.Xq), n, w.ld, ws.at<uint8_t>(w.Q8), w.ld8,
                              reinterpret_cast<unsigned *>(sc), sc + 1, s));
        c1.fp8 = 1;
        c1.X = ws.at<uint8_t>(w.B8);
        c1.x_stride = w.dir ? 2LL * w.ld : w.ld8;
        c1.kx_period = w.ld8;
        c1.Y = ws.at<uint8_t>(w.Q8);
        c1.y_stride = w.ld8;
        c1.k_total = w.ld8;
        c1.scale_dev = sc + 1;
    }
    GOAT_TRY(run(c1));
    if (w.dir) {
        GemmCall c1t = c1;
        c1t.X = w.q8 ? (const void *)(ws.at<uint8_t>(w.B8) + w.ld8) : (const void *)(ws.at<__nv_bfloat16>(w.B16) + w.ld);
        c1t.out_b16 = ws.at<__nv_bfloat16>(w.C1) + w.ld;
        GOAT_TRY(run(c1t));
    }
    if (between) cudaEventRecord(between, s);

    if (w.lo8) {
        // C1's lo term to E4M3 (hi scaled by the same power of two); the scale's inverse
        // goes to the second product's epilogue
        float *sc = ws.at<float>(w.f8s);
        GOAT_TRY(split_lo_to_e4m3(ws.at<__nv_bfloat16>(w.C1), n, w.ld, w.parts, ws.at<uint8_t>(w.C8),
                                  w.dir ? w.ld : w.ld8, reinterpret_cast<unsigned *>(sc + 2), sc + 3, s));
    }

    // K runs over [A | A^T] (period parts*ld) against C1's row: term t, part p at
    // offset (t * parts + p) ld, so position k meets A for p = 0 and A^T for p = 1
    GemmCall c2 = c1;
    c2.fp8 = 0;
    c2.scale_dev = nullptr;
    c2.X = ws.at<__nv_bfloat16>(w.A16);
    c2.x_stride = xs;
    c2.kx_period = w.parts * w.ld;
    c2.Y = ws.at<__nv_bfloat16>(w.C1);
    c2.y_stride = cs;
    c2.k_total = (int)cs;
    c2.scale = scale2;
    c2.mode = GEMM_OUT_F32;
    c2.out_f32 = G_out;
    c2.ld_out = n;
    c2.out_b16 = nullptr;
    c2.out_cols = n;
    if (w.lo8) {
        // BF16 over the hi term, then E4M3 over the lo term against A in E4M3
        const long long row8 = w.dir ? 2LL * w.ld : w.ld8;
        c2.k_total = w.parts * w.ld;
        c2.scale_dev = ws.at<float>(w.f8s) + 3;
        c2.X8 = ws.at<uint8_t>(w.A8);
        c2.x8_stride = row8;
        c2.kx8_period = (int)row8;
        c2.Y8 = ws.at<uint8_t>(w.C8);
        c2.y8_stride = row8;
        c2.k8_total = (int)row8;
    }
    return run(c2);
}

// G_out = -sigma grad f(X) on the solved block, X in Xq (sigma = +1: maximise f,
// -1: minimise), plus the seeds' constant share (already carrying the sign).
static int gradient_from_terms(const Plan &w, const Scratch &ws, float sigma, float *G_out, int *err, cudaStream_t s,
                               cudaEvent_t between = nullptr) {
    const float scale2 = -sigma * (w.dir ? 1.0f : 2.0f);
    GOAT_TRY(w.fp8 ? gradient_fp8(w, ws, scale2, G_out, err, s, between)
                   : gradient_bf16(w, ws, scale2, G_out, err, s, between));
    if (w.m > 0) add_f32(G_out, ws.at<float>(w.Cs), (long long)w.n * w.n, s);
    return GOAT_OK;
}

// The unseeded block of A and B (rows and columns m..n_full-1) as GEMM operands,
// the block's degrees (with_deg), and the symmetry check the two-product form
// relies on.  deg: out-degrees of A, of B, in-degrees of A, of B (n each).
static int prepare_operands(const AdjView &A, const AdjView &B, const Plan &w, const Scratch &ws, DevState *st,
                            bool with_deg, int *pinned, cudaStream_t s) {
    const int n = w.n, m = w.m;
    if (n > 0) {
        const long long xs = (long long)w.parts * w.ld;
        float *deg = with_deg ? ws.at<float>(w.deg) : nullptr;
        __nv_bfloat16 *A16 = ws.at<__nv_bfloat16>(w.A16), *B16 = ws.at<__nv_bfloat16>(w.B16);
        GOAT_TRY(adj_to_bf16(A, m, m, n, n, A16, w.ld, xs, deg, s));
        GOAT_TRY(adj_to_bf16(B, m, m, n, n, B16, w.ld, xs, deg ? deg + n : nullptr, s));
        if (w.dir) {
            GOAT_TRY(adj_to_bf16_t(A, m, m, n, n, A16 + w.ld, w.ld, xs, s));
            GOAT_TRY(adj_to_bf16_t(B, m, m, n, n, B16 + w.ld, w.ld, xs, s));
            if (deg) {
                GOAT_TRY(adj_col_sums(A, m, m, n, n, deg + 2 * (size_t)n, s));
                GOAT_TRY(adj_col_sums(B, m, m, n, n, deg + 3 * (size_t)n, s));
            }
        }
        if (w.fp8 || w.q8 || w.lo8) {
            const int width = w.dir ? w.ld : w.ld8;
            const long long row8 = w.dir ? 2LL * w.ld : w.ld8;
            GOAT_TRY(adj_to_e4m3(A, m, m, n, n, ws.at<uint8_t>(w.A8), width, row8, s));
            if (!w.lo8) GOAT_TRY(adj_to_e4m3(B, m, m, n, n, ws.at<uint8_t>(w.B8), width, row8, s));
            if (w.dir) {
                GOAT_TRY(adj_to_e4m3_t(A, m, m, n, n, ws.at<uint8_t>(w.A8) + w.ld, w.ld, row8, s));
                if (!w.lo8) GOAT_TRY(adj_to_e4m3_t(B, m, m, n, n, ws.at<uint8_t>(w.B8) + w.ld, w.ld, row8, s));
            }
        }
    }
    if (w.dir) return GOAT_OK;
    GOAT_TRY(count_asym(A.p, A.dtype, w.n_full, &st->asym_count, s));
    GOAT_TRY(count_asym(B.p, B.dtype, w.n_full, &st->asym_count, s));
    GOAT_TRY(cuda_status(cudaMemcpyAsync(pinned, &st->asym_count, sizeof(int), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    return pinned[0] == 0 ? GOAT_OK : GOAT_ERR_INVALID_ARG;
}

// Seeded matching: with P = I_m (+) P22 the unseeded block of grad f(P) is
//   A21 B21^T + A12^T B12 + A22 P22 B22^T + A22^T P22 B22
// (A21 = rows m.., columns ..m-1 of A; A12 its transposed counterpart), so the seeds
// add the constant C = A21 B21^T + A12^T B12 (2 A21 B21^T for symmetric graphs).
// Cs = -sigma C, one product over K = [A21 | A12^T] x [B21 | B12^T], once per solve.
static int seed_term(const AdjView &A, const AdjView &B, const Plan &w, const Scratch &ws, float sigma, int *err,
                     cudaStream_t s) {
    const int n = w.n, m = w.m;
    __nv_bfloat16 *SX = ws.at<__nv_bfloat16>(w.SX), *SY = ws.at<__nv_bfloat16>(w.SY);
    GOAT_TRY(adj_to_bf16(A, m, 0, n, m, SX, w.dir ? m : w.ldm, w.ldm, nullptr, s));
    GOAT_TRY(adj_to_bf16(B, m, 0, n, m, SY, w.dir ? m : w.ldm, w.ldm, nullptr, s));
    if (w.dir) {
        GOAT_TRY(adj_to_bf16_t(A, 0, m, m, n, SX + m, w.ldm - m, w.ldm, s));
        GOAT_TRY(adj_to_bf16_t(B, 0, m, m, n, SY + m, w.ldm - m, w.ldm, s));
    }
    GemmCall c;
    std::memset(&c, 0, sizeof(c));
    c.X = SX;
    c.x_rows = n;
    c.x_stride = w.ldm;
    c.kx_period = w.ldm;
    c.Y = SY;
    c.y_rows = n;
    c.y_stride = w.ldm;
    c.k_total = w.ldm;
    c.M = n;
    c.N = n;
    c.scale = -sigma * (w.dir ? 1.0f : 2.0f);
    c.mode = GEMM_OUT_F32;
    c.out_f32 = ws.at<float>(w.Cs);
    c.ld_out = n;
    c.out_rows = n;
    c.out_cols = n;
    c.err = err;
    return gemm_xyT(c, s);
}

static int read_error(DevState *st, int *pinned, cudaStream_t s) {
    GOAT_TRY(cuda_status(cudaMemcpyAsync(pinned, &st->error, sizeof(int), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    return pinned[0];
}

static int match_impl(const AdjView &A, const AdjView &B, const float *init, float eps_rel, int max_iter, float tol,
                      const goat_params &prm, int32_t *perm_out, double *objective_out, goat_stats *stats,
                      const Plan &w, const Scratch &ws, cudaStream_t s) {
    int *pinned = pinned_words();
    if (!pinned) return GOAT_ERR_CUDA;
    const int n = w.n, m = w.m, nf = w.n_full;
    const int dtype = A.dtype;
    const float sigma = prm.maximize ? 1.0f : -1.0f;
    DevState *st = ws.at<DevState>(w.state);
    float *P = ws.at<float>(w.P), *G = ws.at<float>(w.G), *GQ = ws.at<float>(w.GQ);
    float *f = ws.at<float>(w.f), *g = ws.at<float>(w.g);
    float *deg = ws.at<float>(w.deg);
    double *partial = ws.at<double>(w.partial);
    __nv_bfloat16 *Xq = ws.at<__nv_bfloat16>(w.Xq);
    int32_t *perm_dev = ws.at<int32_t>(w.perm);
    int32_t *perm_blk = perm_dev + m;  // the unseeded block's assignment (block indices)
    const long long nn = (long long)n * n;

    cudaEvent_t ev[4];
    for (auto &e : ev) cudaEventCreate(&e);
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int k = 0; k < 4; ++k) cudaEventDestroy(e[k]);
        }
    } evg{ev};
    cudaEventRecord(ev[0], s);

    const long long launches0 = launches_so_far();
    GOAT_TRY(init_state(st, eps_rel, 1, tol, s, nf));
    GOAT_TRY(prepare_operands(A, B, w, ws, st, true, pinned, s));
    if (m > 0 && n > 0) GOAT_TRY(seed_term(A, B, w, ws, sigma, &st->error, s));
    const float *Cs = (m > 0 && n > 0) ? ws.at<float>(w.Cs) : nullptr;

    if (n > 0) {
        if (!init) {
            // G = -sigma grad f(J) in closed form from the block's degrees (plus the seeds' share)
            if (w.dir)
                barycenter(deg, deg + n, deg + 2 * (size_t)n, deg + 3 * (size_t)n, n, -sigma / (float)n, Cs, G, P, st,
                           s);
            else
                barycenter(deg, deg + n, nullptr, nullptr, n, -2.0f * sigma / (float)n, Cs, G, P, st, s);
        } else {
            // the unseeded block of the caller's start (which has the form I_m (+) P22)
            GOAT_TRY(cuda_status(cudaMemcpy2DAsync(P, (size_t)n * 4, init + ((size_t)m * nf + m), (size_t)nf * 4,
                                                   (size_t)n * 4, (size_t)n, cudaMemcpyDeviceToDevice, s)));
            f32_to_terms(P, n, n, Xq, w.ld, w.terms, s);
            GOAT_TRY(gradient_from_terms(w, ws, sigma, G, &st->error, s));
            absmax(G, nn, &st->gmax_bits, s);
        }
        GOAT_TRY(cuda_status(cudaMemsetAsync(g, 0, (size_t)n * 4, s)));
    }
    GOAT_TRY(cuda_status(cudaGetLastError()));
    cudaEventRecord(ev[1], s);

    const bool prof = prm.profile != 0;
    cudaEvent_t pe[6] = {};  // s0 | sinkhorn | s1 | write_q | g0 | gemm1 | g1 | gemm2 | g2 | step | u1
    if (prof)
        for (auto &e : pe) cudaEventCreate(&e);
    struct ProfGuard {
        cudaEvent_t *e;
        bool on;
        ~ProfGuard() {
            if (on)
                for (int k = 0; k < 6; ++k) cudaEventDestroy(e[k]);
        }
    } pg{pe, prof};
    float ms_gemm = 0.f, ms_sk = 0.f, ms_step = 0.f;
    int gemm_launches = 0;

    // the LAP schedule: FAQ's per-iteration directions and the final projection
    LapControl ctl;
    lap_default_control(&ctl);
    ctl.max_rounds = prm.lap_max_rounds;
    const bool faq = prm.direction == GOAT_DIR_LAP;

    int it = 0, converged = 0;
    for (; n > 0 && it < max_iter; ++it) {
        if (prof) cudaEventRecord(pe[0], s);
        if (faq) {
            // FAQ (Alg. 1): Q = argmax over permutations of <Pi, grad f(P)> = argmin <Pi, G>;
            // an uncertified assignment is still a permutation, so it is used
            if (it == 0 && !init && !w.dir && m == 0) {
                // at the barycenter grad f(J) of symmetric graphs is rank one: the
                // assignment is the rearrangement pairing of the degrees, solved exactly
                GOAT_TRY(rearrangement_perm(A.p, B.p, dtype, n, prm.maximize, ws.at<void>(w.rearr), perm_blk, s));
            } else {
                LapReport drep{};
                double dgap = 0.0;
                const int dst = lap_solve(G, n, 0, perm_blk, ws.at<void>(w.lap), st, ctl,
                                          ws.at<double>(w.cost) + 6, pinned, &dgap, &drep, s);
                if (dst != GOAT_OK && dst != GOAT_ERR_NOT_CONVERGED) return dst;
            }
            if (prof) cudaEventRecord(pe[1], s);
            GOAT_TRY(write_perm_q(perm_blk, n, Xq, w.ld, w.terms, s));
        } else {
            // GOAT (Alg. 3): Q = LOT(-grad f(P)) (Alg. 2)
            const bool learned = it == 0 && prm.mlp_weights;
            if (learned) {
                // the learned warm start needs this step's eps on the host: eps_rel * max|G|
                GOAT_TRY(cuda_status(
                    cudaMemcpyAsync(pinned, &st->gmax_bits, sizeof(unsigned), cudaMemcpyDeviceToHost, s)));
                GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
                float gm;
                std::memcpy(&gm, pinned, sizeof(float));
                float e0 = eps_rel * gm;
                if (!(e0 > 0.f)) e0 = 1.0f;
                GOAT_TRY(mlp_warm_start_g(G, A.p, B.p, n, dtype, e0, (const __nv_bfloat16 *)prm.mlp_weights, g,
                                          ws.at<float>(w.mlp), s));
            }
            sinkhorn_begin(st, -1.0f, prm.sk_tol, (prm.sk_warm_start || learned) ? nullptr : g, n, s);
            GOAT_TRY(sinkhorn_solve(G, n, n, f, g, partial, st, prm.sk_max_iter, prm.sk_check_every, pinned, s));
            if (learned) {
                // fallback: a learned start that does not reach the tolerance is redone cold
                GOAT_TRY(
                    cuda_status(cudaMemcpyAsync(pinned, &st->sk_resid, sizeof(float), cudaMemcpyDeviceToHost, s)));
                GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
                float r;
                std::memcpy(&r, pinned, sizeof(float));
                if (!(r < prm.sk_tol)) {
                    sinkhorn_begin(st, -1.0f, prm.sk_tol, g, n, s);
                    GOAT_TRY(
                        sinkhorn_solve(G, n, n, f, g, partial, st, prm.sk_max_iter, prm.sk_check_every, pinned, s));
                }
            }
            if (prof) cudaEventRecord(pe[1], s);
            write_q(G, n, n, f, g, st, Xq, w.ld, w.terms, nullptr, 0, s);
        }
        if (prof) cudaEventRecord(pe[2], s);
        GOAT_TRY(gradient_from_terms(w, ws, sigma, GQ, &st->error, s, prof ? pe[3] : nullptr));
        if (prof) cudaEventRecord(pe[4], s);
        // the LOT direction enters the step size and the update in FP32, recomputed from
        // its duals (the products took it rounded); FAQ's permutation is exact in Xq
        const float *fq = faq ? nullptr : f, *gq = faq ? nullptr : g;
        line_search(G, GQ, P, Xq, w.ld, w.terms, nullptr, fq, gq, n, partial, st, s);
        fw_update(P, G, GQ, Xq, w.ld, w.terms, nullptr, fq, gq, n, st, 0.0f, &st->gmax_next, s);
        fw_roll(st, s);
        if (prof) cudaEventRecord(pe[5], s);
        GOAT_TRY(cuda_status(cudaMemcpyAsync(pinned, &st->fw_done, sizeof(int), cudaMemcpyDeviceToHost, s)));
        GOAT_TRY(cuda_status(cudaMemcpyAsync(pinned + 1, &st->error, sizeof(int), cudaMemcpyDeviceToHost, s)));
        GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
        if (prof) {
            float a = 0.f, b = 0.f, c = 0.f, d = 0.f, e = 0.f;
            cudaEventElapsedTime(&a, pe[0], pe[1]);
            cudaEventElapsedTime(&b, pe[1], pe[2]);
            cudaEventElapsedTime(&c, pe[2], pe[3]);
            cudaEventElapsedTime(&d, pe[3], pe[4]);
            cudaEventElapsedTime(&e, pe[4], pe[5]);
            ms_sk += a;
            ms_step += b + e;
            ms_gemm += c + d;
            gemm_launches += 2;
        }
        if (pinned[1]) return pinned[1];
        if (pinned[0]) {
            converged = 1;
            ++it;
            break;
        }
    }
    cudaEventRecord(ev[2], s);

    // projection onto the permutations (of the unseeded block; the seeds keep their match)
    double gap = 0.0;
    LapReport rep{};
    if (n > 0) {
        int lst;
        if (prm.project_on_grad) {
            // argmax tr(Pi^T grad f(P)) (argmin when minimising) = argmin <Pi, G>
            lst = lap_solve(G, n, 0, perm_blk, ws.at<void>(w.lap), st, ctl, ws.at<double>(w.cost) + 6, pinned,
                            &gap, &rep, s);
        } else {
            lst = lap_solve(P, n, 1, perm_blk, ws.at<void>(w.lap), st, ctl, ws.at<double>(w.cost) + 6, pinned,
                            &gap, &rep, s);
        }
        if (lst != GOAT_OK && lst != GOAT_ERR_NOT_CONVERGED) return lst;
    }
    if (m > 0) seed_perm(perm_dev, nf, m, s);
    if (prm.relaxed_out) {
        if (m == 0)
            GOAT_TRY(cuda_status(cudaMemcpyAsync(prm.relaxed_out, P, (size_t)nn * 4, cudaMemcpyDeviceToDevice, s)));
        else
            embed_block(P, n, m, prm.relaxed_out, s);
    }
    cudaEventRecord(ev[3], s);

    // objective and disagreements at the returned permutation
    unsigned long long *isums = ws.at<unsigned long long>(w.cost);
    double *fsums = ws.at<double>(w.cost) + 3;
    GOAT_TRY(cuda_status(cudaMemsetAsync(isums, 0, 6 * sizeof(double), s)));
    GOAT_TRY(objective(A.p, B.p, dtype, nf, perm_dev, isums, fsums, isums + 1, isums + 2, fsums + 1, fsums + 2,
                       &st->bad_perm, ws.at<double>(w.objpart), s));
    unsigned long long hi[3];
    double hf[3];
    GOAT_TRY(cuda_status(cudaMemcpyAsync(hi, isums, sizeof(hi), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaMemcpyAsync(hf, fsums, sizeof(hf), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaMemcpyAsync(perm_out, perm_dev, (size_t)nf * 4, cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    double fobj, dis;
    if (dtype == GOAT_DTYPE_U8) {
        fobj = (double)hi[0];
        dis = (double)hi[1] + (double)hi[2] - 2.0 * (double)hi[0];
    } else {
        fobj = hf[0];
        dis = hf[1] + hf[2] - 2.0 * hf[0];
    }
    if (objective_out) *objective_out = fobj;
    if (stats) {
        DevState hs;
        GOAT_TRY(cuda_status(cudaMemcpy(&hs, st, sizeof(DevState), cudaMemcpyDeviceToHost)));
        std::memset(stats, 0, sizeof(*stats));
        stats->fw_iters = it;
        stats->converged = converged;
        const int m = std::min(it, GOAT_TRACE_MAX);
        for (int k = 0; k < m; ++k) {
            stats->sk_iters[k] = hs.tr_sk_iters[k];
            stats->sk_resid[k] = hs.tr_sk_resid[k];
            stats->alpha[k] = hs.tr_alpha[k];
            stats->sk_iters_total += hs.tr_sk_iters[k];
        }
        stats->objective = fobj;
        stats->disagreements = dis;
        stats->lap_gap = gap;
        stats->lap_rounds = rep.rounds;
        stats->lap_tail_bids = rep.tail_bids;
        stats->lap_sap_rows = rep.sap_rows;
        stats->lap_sap_pops = rep.sap_pops;
        stats->lap_ms_head = (float)rep.ms_head;
        stats->lap_ms_tail = (float)rep.ms_tail;
        stats->lap_ms_sap = (float)rep.ms_sap;
        cudaEventElapsedTime(&stats->ms_total, ev[0], ev[3]);
        cudaEventElapsedTime(&stats->ms_fw, ev[1], ev[2]);
        cudaEventElapsedTime(&stats->ms_project, ev[2], ev[3]);
        stats->ms_gemm = ms_gemm;
        stats->gemm_launches = gemm_launches;
        stats->ms_sinkhorn = ms_sk;
        stats->ms_step = ms_step;
        stats->launches = launches_so_far() - launches0;
    }
    return GOAT_OK;  // an uncertified projection still returns its (eps-optimal) assignment
}

static goat_params resolve_params(const goat_params *p) {
    goat_params d;
    goat_default_params(&d);
    if (!p) return d;
    goat_params r = *p;
    if (r.sk_max_iter <= 0) r.sk_max_iter = d.sk_max_iter;
    if (!(r.sk_tol > 0.0f)) r.sk_tol = d.sk_tol;
    if (r.sk_check_every <= 0) r.sk_check_every = d.sk_check_every;
    if (r.lap_max_rounds <= 0) r.lap_max_rounds = d.lap_max_rounds;
    return r;
}

static bool valid_precision(int p) {
    return p == GOAT_PREC_BF16 || p == GOAT_PREC_FP32 || p == GOAT_PREC_FP8 || p == GOAT_PREC_BF16_SPLIT ||
           p == GOAT_PREC_FP8_SPLIT || p == GOAT_PREC_BF16_SPLIT8;
}

// The solve's shape from its parameters; false if they do not fit n.
static bool match_shape(const goat_params &p, int n, Shape *sh) {
    if (p.seeds < 0 || p.seeds > n || (p.directed != 0 && p.directed != 1) || (p.maximize != 0 && p.maximize != 1))
        return false;
    // the learned warm start is trained on unseeded symmetric problems
    if (p.mlp_weights && (p.seeds > 0 || p.directed)) return false;
    sh->n_full = n;
    sh->m = p.seeds;
    sh->dir = p.directed;
    return true;
}
static bool valid_direction(int d) { return d == GOAT_DIR_LOT || d == GOAT_DIR_LAP; }
static bool valid_dtype(int d) { return d == GOAT_DTYPE_U8 || d == GOAT_DTYPE_F32; }

}  // namespace goat

using namespace goat;

// ===================================================================== C ABI

extern "C" {

void goat_default_params(goat_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->precision = GOAT_PREC_BF16;
    p->sk_max_iter = 500;
    p->sk_tol = 1e-3f;
    p->sk_warm_start = 1;
    p->sk_check_every = 8;
    p->project_on_grad = 0;
    p->lap_max_rounds = 1 << 20;
    p->direction = GOAT_DIR_LOT;
    p->maximize = 1;
    p->seeds = 0;
    p->directed = 0;
    p->relaxed_out = nullptr;
}

const char *goat_strerror(int status) {
    switch (status) {
        case GOAT_OK: return "ok";
        case GOAT_ERR_INVALID_ARG: return "invalid argument";
        case GOAT_ERR_NOT_CONVERGED: return "iteration cap reached before convergence";
        case GOAT_ERR_CUDA: return "CUDA runtime error";
        case GOAT_ERR_OUT_OF_MEMORY: return "out of device memory or workspace too small";
        case GOAT_ERR_NAN: return "non-finite value in the iteration";
        case GOAT_ERR_TIMEOUT: return "a bounded device-side wait ran out";
        case GOAT_ERR_UNSUPPORTED: return "device is not compute capability 10.3 (sm_103)";
        default: return "unknown status";
    }
}

size_t goat_workspace_bytes(int n, int dtype_AB, int precision) {
    if (n < 1 || !valid_dtype(dtype_AB) || !valid_precision(precision)) return 0;
    return make_plan(Shape{n, 0, 0}, dtype_AB, precision, NEED_FW).total;
}

size_t goat_workspace_bytes_host(int n, int dtype_AB, int precision) {
    if (n < 1 || !valid_dtype(dtype_AB) || !valid_precision(precision)) return 0;
    return make_plan(Shape{n, 0, 0}, dtype_AB, precision, NEED_FW | NEED_HOSTCOPY).total;
}

size_t goat_workspace_bytes_ex(int n, int dtype_AB, int precision, int directed, int seeds, int host) {
    if (n < 1 || !valid_dtype(dtype_AB) || !valid_precision(precision) || seeds < 0 || seeds > n ||
        (directed != 0 && directed != 1))
        return 0;
    return make_plan(Shape{n, seeds, directed}, dtype_AB, precision, NEED_FW | (host ? NEED_HOSTCOPY : 0)).total;
}

int goat_match(const void *A, const void *B, int n, int dtype_AB, const float *init, float eps_rel, int max_iter,
               float tol, const goat_params *p, int32_t *perm_out, double *objective_out, goat_stats *stats,
               void *workspace, size_t workspace_bytes, goat_stream_t stream) {
    if (!A || !B || !perm_out || n < 1 || !valid_dtype(dtype_AB) || max_iter < 0 || !(eps_rel > 0.0f) ||
        !(tol >= 0.0f) || max_iter > (1 << 20))
        return GOAT_ERR_INVALID_ARG;
    const goat_params prm = resolve_params(p);
    Shape sh;
    if (!valid_precision(prm.precision) || !valid_direction(prm.direction) || !match_shape(prm, n, &sh))
        return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    cudaStream_t s = (cudaStream_t)stream;
    const Plan w = make_plan(sh, dtype_AB, prm.precision, NEED_FW);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    return match_impl(AdjView{A, n, dtype_AB}, AdjView{B, n, dtype_AB}, init, eps_rel, max_iter, tol, prm, perm_out,
                      objective_out, stats, w, ws, s);
}

int goat_match_host(const void *A_host, const void *B_host, int n, int dtype_AB, const float *init_host,
                    float eps_rel, int max_iter, float tol, const goat_params *p, int32_t *perm_out,
                    double *objective_out, goat_stats *stats, void *workspace, size_t workspace_bytes,
                    goat_stream_t stream) {
    if (!A_host || !B_host || !perm_out || n < 1 || !valid_dtype(dtype_AB) || max_iter < 0 || !(eps_rel > 0.0f) ||
        !(tol >= 0.0f))
        return GOAT_ERR_INVALID_ARG;
    const goat_params prm = resolve_params(p);
    Shape sh;
    if (!valid_precision(prm.precision) || !valid_direction(prm.direction) || !match_shape(prm, n, &sh))
        return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    cudaStream_t s = (cudaStream_t)stream;
    // the device copies sit after the goat_match layout, so a goat_match-sized
    // workspace is not enough here: size = goat_workspace_bytes + copies
    const Plan w = make_plan(sh, dtype_AB, prm.precision, NEED_FW | NEED_HOSTCOPY);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    const size_t es = dtype_AB == GOAT_DTYPE_U8 ? 1 : 4;
    const size_t bytes = (size_t)n * n * es;
    GOAT_TRY(cuda_status(cudaMemcpyAsync(ws.at<void>(w.Ad), A_host, bytes, cudaMemcpyHostToDevice, s)));
    GOAT_TRY(cuda_status(cudaMemcpyAsync(ws.at<void>(w.Bd), B_host, bytes, cudaMemcpyHostToDevice, s)));
    const float *init_dev = nullptr;
    if (init_host) {
        GOAT_TRY(cuda_status(
            cudaMemcpyAsync(ws.at<void>(w.Id), init_host, (size_t)n * n * 4, cudaMemcpyHostToDevice, s)));
        init_dev = ws.at<float>(w.Id);
    }
    return match_impl(AdjView{ws.at<void>(w.Ad), n, dtype_AB}, AdjView{ws.at<void>(w.Bd), n, dtype_AB}, init_dev,
                      eps_rel, max_iter, tol, prm, perm_out, objective_out, stats, w, ws, s);
}

int goat_gradient_ex(const void *A, const void *B, int n, int dtype_AB, const float *P, float *G_out, int precision,
                     int directed, void *workspace, size_t workspace_bytes, goat_stream_t stream) {
    if (!A || !B || !P || !G_out || n < 1 || !valid_dtype(dtype_AB) || !valid_precision(precision) ||
        (directed != 0 && directed != 1))
        return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    int *pinned = pinned_words();
    if (!pinned) return GOAT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const Plan w = make_plan(Shape{n, 0, directed}, dtype_AB, precision, NEED_GEMM);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    DevState *st = ws.at<DevState>(w.state);
    GOAT_TRY(init_state(st, 0.03f, 1, 0.0f, s));
    GOAT_TRY(prepare_operands(AdjView{A, n, dtype_AB}, AdjView{B, n, dtype_AB}, w, ws, st, false, pinned, s));
    f32_to_terms(P, n, n, ws.at<__nv_bfloat16>(w.Xq), w.ld, w.terms, s);
    GOAT_TRY(gradient_from_terms(w, ws, 1.0f, G_out, &st->error, s));
    const int e = read_error(st, pinned, s);
    return e;
}

int goat_gradient(const void *A, const void *B, int n, int dtype_AB, const float *P, float *G_out, int precision,
                  void *workspace, size_t workspace_bytes, goat_stream_t stream) {
    return goat_gradient_ex(A, B, n, dtype_AB, P, G_out, precision, 0, workspace, workspace_bytes, stream);
}

int goat_sinkhorn(const float *G, int n, float eps, float tol, int max_iter, float *f_out, float *g_io,
                  float *Q_out, int *iters_out, float *resid_out, void *workspace, size_t workspace_bytes,
                  goat_stream_t stream) {
    if (!G || !f_out || !g_io || n < 1 || !(eps > 0.0f) || !(tol >= 0.0f) || max_iter < 1)
        return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    int *pinned = pinned_words();
    if (!pinned) return GOAT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const Plan w = make_plan(Shape{n, 0, 0}, GOAT_DTYPE_U8, GOAT_PREC_BF16, NEED_SK);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    DevState *st = ws.at<DevState>(w.state);
    GOAT_TRY(init_state(st, 0.03f, 1, 0.0f, s));
    sinkhorn_begin(st, eps, tol, nullptr, n, s);
    GOAT_TRY(sinkhorn_solve(G, n, n, f_out, g_io, ws.at<double>(w.partial), st, max_iter, 8, pinned, s));
    if (Q_out) write_q(G, n, n, f_out, g_io, st, nullptr, (int)round_up(n, 8), 1, Q_out, n, s);
    DevState hs;
    GOAT_TRY(cuda_status(cudaMemcpyAsync(&hs, st, offsetof(DevState, tr_sk_iters), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    if (iters_out) *iters_out = hs.sk_iters;
    if (resid_out) *resid_out = hs.sk_resid;
    return hs.error;
}

int goat_line_search(const float *G, const float *G_Q, const float *P, const float *Q, int n, int maximize,
                     double *alpha_out, double *a_out, double *b_out, void *workspace, size_t workspace_bytes,
                     goat_stream_t stream) {
    if (!G || !G_Q || !P || !Q || !alpha_out || n < 1) return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    cudaStream_t s = (cudaStream_t)stream;
    const Plan w = make_plan(Shape{n, 0, 0}, GOAT_DTYPE_U8, GOAT_PREC_BF16, NEED_SK);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    DevState *st = ws.at<DevState>(w.state);
    GOAT_TRY(init_state(st, 0.03f, maximize ? 1 : 0, 0.0f, s));
    line_search(G, G_Q, P, nullptr, 0, 1, Q, nullptr, nullptr, n, ws.at<double>(w.partial), st, s);
    DevState hs;
    GOAT_TRY(cuda_status(cudaMemcpyAsync(&hs, st, offsetof(DevState, tr_sk_iters), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    *alpha_out = hs.alpha;
    if (a_out) *a_out = hs.ls_a;
    if (b_out) *b_out = hs.ls_b;
    return hs.error;
}

int goat_entropic_eps(const float *G, int n, float eps_rel, float *eps_out, goat_stream_t stream) {
    if (!G || !eps_out || n < 1 || !(eps_rel > 0.0f)) return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    cudaStream_t s = (cudaStream_t)stream;
    int *pinned = pinned_words();
    if (!pinned) return GOAT_ERR_CUDA;
    unsigned *bits = nullptr;
    GOAT_TRY(cuda_status(cudaMallocAsync((void **)&bits, sizeof(unsigned), s)));
    cudaMemsetAsync(bits, 0, sizeof(unsigned), s);
    absmax(G, (long long)n * n, bits, s);
    cudaMemcpyAsync(pinned, bits, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(bits, s);
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    float gm;
    std::memcpy(&gm, pinned, sizeof(float));
    if (!(gm == gm) || std::isinf(gm)) return GOAT_ERR_NAN;
    // the rule of k_sk_begin: eps_rel max|G|, and 1 when G == 0 (every doubly
    // stochastic Q is then optimal)
    float e = eps_rel * gm;
    if (!(e > 0.0f)) e = 1.0f;
    *eps_out = e;
    return GOAT_OK;
}

int goat_fw_update(float *P, float *G, const float *Q, const float *G_Q, int n, double alpha, goat_stream_t stream) {
    if (!P || !G || !Q || !G_Q || n < 1 || !(alpha >= 0.0 && alpha <= 1.0)) return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    cudaStream_t s = (cudaStream_t)stream;
    fw_update(P, G, G_Q, nullptr, 0, 1, Q, nullptr, nullptr, n, nullptr, (float)alpha, nullptr, s);
    return cuda_status(cudaGetLastError());
}

void goat_lap_default_options(goat_lap_options *o) {
    if (!o) return;
    LapControl c;
    lap_default_control(&c);
    o->max_rounds = c.max_rounds;
    o->head_rounds = c.head_rounds;
    o->tail_bids = c.tail_bids;
    o->tail_stall = c.tail_stall;
    o->sap_pops = c.sap_pops;
    o->head_stall = c.head_stall;
    o->sap_every_phase = c.sap_every_phase;
}

int goat_project_ex(const float *M, int n, int maximize, const goat_lap_options *opts, int32_t *perm_out,
                    double *cost_out, double *gap_out, goat_lap_info *info, void *workspace, size_t workspace_bytes,
                    goat_stream_t stream) {
    if (!M || !perm_out || n < 1) return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    int *pinned = pinned_words();
    if (!pinned) return GOAT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    LapControl ctl;
    lap_default_control(&ctl);
    if (opts) {
        if (opts->max_rounds > 0) ctl.max_rounds = opts->max_rounds;
        if (opts->head_rounds >= 0) ctl.head_rounds = opts->head_rounds;
        ctl.tail_bids = opts->tail_bids;
        ctl.tail_stall = opts->tail_stall;
        ctl.sap_pops = opts->sap_pops;
        if (opts->head_stall > 0) ctl.head_stall = opts->head_stall;
        if (opts->sap_every_phase >= 0) ctl.sap_every_phase = opts->sap_every_phase;
    }
    const Plan w = make_plan(Shape{n, 0, 0}, GOAT_DTYPE_U8, GOAT_PREC_BF16, NEED_LAP);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    DevState *st = ws.at<DevState>(w.state);
    GOAT_TRY(init_state(st, 0.03f, maximize ? 1 : 0, 0.0f, s));
    double gap = 0.0;
    LapReport rep{};
    const int r = lap_solve(M, n, maximize ? 1 : 0, perm_out, ws.at<void>(w.lap), st, ctl, ws.at<double>(w.cost) + 6,
                            pinned, &gap, &rep, s);
    if (r != GOAT_OK && r != GOAT_ERR_NOT_CONVERGED) return r;
    double cost = 0.0;
    GOAT_TRY(cuda_status(
        cudaMemcpyAsync(&cost, ws.at<double>(w.cost) + 6, sizeof(double), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    if (cost_out) *cost_out = cost;
    if (gap_out) *gap_out = gap;
    if (info) {
        info->phases = rep.phases;
        info->rounds = rep.rounds;
        info->tail_bids = rep.tail_bids;
        info->sap_rows = rep.sap_rows;
        info->sap_pops = rep.sap_pops;
        info->sap_steps = rep.sap_epochs;
        info->filled = rep.filled;
        info->ms_head = rep.ms_head;
        info->ms_tail = rep.ms_tail;
        info->ms_sap = rep.ms_sap;
    }
    return r;
}

int goat_project(const float *M, int n, int maximize, int32_t *perm_out, double *cost_out, double *gap_out,
                 void *workspace, size_t workspace_bytes, goat_stream_t stream) {
    return goat_project_ex(M, n, maximize, nullptr, perm_out, cost_out, gap_out, nullptr, workspace, workspace_bytes,
                           stream);
}

int goat_objective(const void *A, const void *B, int n, int dtype_AB, const int32_t *perm, double *objective_out,
                   double *disagreements_out, void *workspace, size_t workspace_bytes, goat_stream_t stream) {
    if (!A || !B || !perm || n < 1 || !valid_dtype(dtype_AB)) return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    cudaStream_t s = (cudaStream_t)stream;
    const Plan w = make_plan(Shape{n, 0, 0}, dtype_AB, GOAT_PREC_BF16, 0);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    DevState *st = ws.at<DevState>(w.state);
    GOAT_TRY(init_state(st, 0.03f, 1, 0.0f, s));
    unsigned long long *isums = ws.at<unsigned long long>(w.cost);
    double *fsums = ws.at<double>(w.cost) + 3;
    GOAT_TRY(cuda_status(cudaMemsetAsync(isums, 0, 6 * sizeof(double), s)));
    GOAT_TRY(objective(A, B, dtype_AB, n, perm, isums, fsums, isums + 1, isums + 2, fsums + 1, fsums + 2,
                       &st->bad_perm, ws.at<double>(w.objpart), s));
    unsigned long long hi[3];
    double hf[3];
    int bad = 0;
    GOAT_TRY(cuda_status(cudaMemcpyAsync(hi, isums, sizeof(hi), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaMemcpyAsync(hf, fsums, sizeof(hf), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaMemcpyAsync(&bad, &st->bad_perm, sizeof(int), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    if (bad) return GOAT_ERR_INVALID_ARG;
    if (dtype_AB == GOAT_DTYPE_U8) {
        if (objective_out) *objective_out = (double)hi[0];
        if (disagreements_out) *disagreements_out = (double)hi[1] + (double)hi[2] - 2.0 * (double)hi[0];
    } else {
        if (objective_out) *objective_out = hf[0];
        if (disagreements_out) *disagreements_out = hf[1] + hf[2] - 2.0 * hf[0];
    }
    return GOAT_OK;
}

int goat_gemm_bf16_xyT(const void *X, int x_rows, int x_stride, int kx_period, const void *Y, int y_rows,
                       int y_stride, int k_total, float scale, float *out, int ld_out, int out_rows, int out_cols,
                       goat_stream_t stream) {
    if (!X || !Y || !out || x_rows < 1 || y_rows < 1 || out_rows < 1 || out_cols < 1 || ld_out < out_cols)
        return GOAT_ERR_INVALID_ARG;
    if ((k_total % 64) || (kx_period % 64) || kx_period < 1 || k_total < 1 || x_stride < kx_period ||
        y_stride < k_total)
        return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    int *pinned = pinned_words();
    if (!pinned) return GOAT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int *err = nullptr;
    GOAT_TRY(cuda_status(cudaMallocAsync((void **)&err, sizeof(int), s)));
    cudaMemsetAsync(err, 0, sizeof(int), s);
    GemmCall c;
    std::memset(&c, 0, sizeof(c));
    c.X = (const __nv_bfloat16 *)X;
    c.x_rows = x_rows;
    c.x_stride = x_stride;
    c.kx_period = kx_period;
    c.Y = (const __nv_bfloat16 *)Y;
    c.y_rows = y_rows;
    c.y_stride = y_stride;
    c.k_total = k_total;
    c.M = out_rows;
    c.N = out_cols;
    c.scale = scale;
    c.mode = GEMM_OUT_F32;
    c.out_f32 = out;
    c.ld_out = ld_out;
    c.out_rows = out_rows;
    c.out_cols = out_cols;
    c.err = err;
    int r = gemm_xyT(c, s);
    if (r == GOAT_OK) {
        cudaMemcpyAsync(pinned, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) r = GOAT_ERR_CUDA;
        else r = pinned[0];
    }
    cudaFreeAsync(err, s);
    return r;
}

}  // extern "C"
