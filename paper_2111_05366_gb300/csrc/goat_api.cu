// goat_api.cu -- the C ABI of libgoat and the Frank-Wolfe driver of GOAT (Alg. 3).
//
// goat_match runs, stream-ordered and with one host synchronisation per
// Frank-Wolfe step (the stop test) plus the Sinkhorn polls:
//   operands   A, B -> BF16 (exact for 0/1), degrees, symmetry check
//   init       P = J and G = -grad f(J) = -(2/n) d_A d_B^T in closed form, or G from the GEMMs
//   loop       eps = eps_rel max|G|; Sinkhorn (warm or cold duals); Q -> BF16 terms;
//              C1 = B Q^T; G_Q = -2 A C1^T; line search (b, a, alpha, stop test);
//              P += alpha (Q - P), G += alpha (G_Q - G)   (grad f is linear)
//   project    auction + certification on P (or on grad f(P))
//   objective  f(perm) and the disagreement count, exact for 0/1 inputs
#include <algorithm>
#include <cstring>
#include <mutex>

#include "goat_common.cuh"
#include "goat_internal.h"

namespace goat {

enum : int { NEED_GEMM = 1, NEED_FW = 2, NEED_SK = 4, NEED_LAP = 8, NEED_HOSTCOPY = 16 };

struct Plan {
    size_t state, A16, B16, Xq, C1, GQ, P, G, f, g, deg, partial, lap, perm, Ad, Bd, Id, cost, objpart, mlp, rearr, total;
    size_t A8, B8, Q8, C8, f8s;  // E4M3 operands and their scales (8-bit form)
    int ld, terms, ld8;
    bool fp8;
};

static Plan make_plan(int n, int dtype, int precision, int need) {
    Plan w;
    std::memset(&w, 0, sizeof(w));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (size_t)round_up((int64_t)std::max<size_t>(bytes, 1), 256);
        return o;
    };
    const size_t nn = (size_t)n * (size_t)n;
    w.ld = operand_ld(n);
    w.ld8 = (int)round_up(n, 128);  // an E4M3 stage holds 128 elements of K
    w.terms = precision == GOAT_PREC_FP32 ? 2 : 1;
    w.fp8 = precision == GOAT_PREC_FP8;
    w.state = take(sizeof(DevState));
    w.cost = take(16 * sizeof(double));  // [0,3) u64 sums, [3,6) f64 sums, [6] assignment cost, [7,10) LAP bound
    w.objpart = take(3 * kObjBlocks * sizeof(double));  // per-block partials of the FP64 objective sums
    if (need & (NEED_GEMM | NEED_FW)) {
        w.A16 = take((size_t)n * w.ld * 2);
        w.B16 = take((size_t)n * w.ld * 2);
        w.Xq = take((size_t)n * w.terms * w.ld * 2);
        w.C1 = take((size_t)n * w.terms * w.ld * 2);
        if (w.fp8) {
            w.A8 = take((size_t)n * w.ld8);
            w.B8 = take((size_t)n * w.ld8);
            w.Q8 = take((size_t)n * w.ld8);
            w.C8 = take((size_t)n * w.ld8);
            w.f8s = take(4 * sizeof(float));  // [0] max|Q| bits, [1] 1/s_Q, [2] max|C1| bits, [3] 1/s_C1
        }
    }
    if (need & NEED_FW) {
        w.GQ = take(nn * 4);
        w.P = take(nn * 4);
        w.G = take(nn * 4);
        w.f = take((size_t)n * 4);
        w.g = take((size_t)n * 4);
        w.deg = take((size_t)2 * n * 4);
        w.mlp = take(mlp_warm_start_scratch_bytes(n));
        w.rearr = take(rearrangement_scratch_bytes(n));
    }
    if (need & (NEED_SK | NEED_FW)) {
        const size_t sk = (size_t)sinkhorn_partial_elems(n) * 8;
        const size_t ls = (size_t)ls_blocks(n) * 3 * 8;
        w.partial = take(std::max(sk, ls));
    }
    if (need & (NEED_LAP | NEED_FW)) {
        w.lap = take(lap_bytes(n, lap_chunks(n)));
        w.perm = take((size_t)n * 4);
    }
    if (need & NEED_HOSTCOPY) {
        const size_t es = dtype == GOAT_DTYPE_U8 ? 1 : 4;
        w.Ad = take(nn * es);
        w.Bd = take(nn * es);
        w.Id = take(nn * 4);
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

__global__ void k_state_init(DevState *st, float eps_rel, int maximize, float fw_tol) {
    st->eps_rel = eps_rel;
    st->maximize = maximize;
    st->fw_tol = fw_tol;
    st->eps = 1.0f;
    st->c = 1.4426950408889634f;
}

static int init_state(DevState *st, float eps_rel, int maximize, float fw_tol, cudaStream_t s) {
    if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess) return GOAT_ERR_CUDA;
    k_state_init<<<1, 1, 0, s>>>(st, eps_rel, maximize, fw_tol);
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

// The 8-bit form of the two products: Q (BF16 in Xq) and then C1 = B Q^T are each
// rounded to E4M3 under a power-of-two scale; the GEMM epilogues undo the scales.
static int gradient_fp8(const Plan &w, const Scratch &ws, int n, float *G_out, int *err, cudaStream_t s,
                        cudaEvent_t between) {
    float *sc = ws.at<float>(w.f8s);
    unsigned *amax = reinterpret_cast<unsigned *>(sc);
    GOAT_TRY(bf16_to_e4m3(ws.at<__nv_bfloat16>(w.Xq), n, w.ld, ws.at<uint8_t>(w.Q8), w.ld8, amax, sc + 1, s));
    GemmCall c1;
    std::memset(&c1, 0, sizeof(c1));
    c1.fp8 = 1;
    c1.X = ws.at<uint8_t>(w.B8);
    c1.x_rows = n;
    c1.x_stride = w.ld8;
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
    c1.term_stride = w.ld;
    c1.row_stride = w.ld;
    c1.out_rows = n;
    c1.out_cols = w.ld;  // the padding columns receive zeros
    c1.err = err;
    GOAT_TRY(gemm_xyT(c1, s));
    if (between) cudaEventRecord(between, s);
    GOAT_TRY(bf16_to_e4m3(ws.at<__nv_bfloat16>(w.C1), n, w.ld, ws.at<uint8_t>(w.C8), w.ld8,
                          reinterpret_cast<unsigned *>(sc + 2), sc + 3, s));
    GemmCall c2 = c1;
    c2.X = ws.at<uint8_t>(w.A8);
    c2.Y = ws.at<uint8_t>(w.C8);
    c2.scale = -2.0f;
    c2.scale_dev = sc + 3;
    c2.mode = GEMM_OUT_F32;
    c2.out_f32 = G_out;
    c2.ld_out = n;
    c2.out_b16 = nullptr;
    c2.out_cols = n;
    return gemm_xyT(c2, s);
}

// -grad f(X) = -2 A X B for symmetric A, B, with X already in the split-term buffer Xq.
static int gradient_from_terms(const Plan &w, const Scratch &ws, int n, float *G_out, int *err, cudaStream_t s,
                               cudaEvent_t between = nullptr) {
    if (w.fp8) return gradient_fp8(w, ws, n, G_out, err, s, between);
    GemmCall c1;
    std::memset(&c1, 0, sizeof(c1));
    c1.X = ws.at<__nv_bfloat16>(w.B16);
    c1.x_rows = n;
    c1.x_stride = w.ld;
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
    c1.out_terms = w.terms;
    c1.term_stride = w.ld;
    c1.row_stride = (long long)w.terms * w.ld;
    c1.out_rows = n;
    c1.out_cols = w.ld;  // the padding columns receive zeros
    c1.err = err;
    GOAT_TRY(gemm_xyT(c1, s));
    if (between) cudaEventRecord(between, s);

    GemmCall c2 = c1;
    c2.X = ws.at<__nv_bfloat16>(w.A16);
    c2.Y = ws.at<__nv_bfloat16>(w.C1);
    c2.scale = -2.0f;
    c2.mode = GEMM_OUT_F32;
    c2.out_f32 = G_out;
    c2.ld_out = n;
    c2.out_b16 = nullptr;
    c2.out_cols = n;
    return gemm_xyT(c2, s);
}

static int prepare_operands(const void *A, const void *B, int n, int dtype, const Plan &w, const Scratch &ws,
                            DevState *st, float *degA, float *degB, int *pinned, cudaStream_t s) {
    GOAT_TRY(adj_to_bf16(A, dtype, n, ws.at<__nv_bfloat16>(w.A16), w.ld, degA, s));
    GOAT_TRY(adj_to_bf16(B, dtype, n, ws.at<__nv_bfloat16>(w.B16), w.ld, degB, s));
    if (w.fp8) {
        GOAT_TRY(adj_to_e4m3(A, dtype, n, ws.at<uint8_t>(w.A8), w.ld8, s));
        GOAT_TRY(adj_to_e4m3(B, dtype, n, ws.at<uint8_t>(w.B8), w.ld8, s));
    }
    GOAT_TRY(count_asym(A, dtype, n, &st->asym_count, s));
    GOAT_TRY(count_asym(B, dtype, n, &st->asym_count, s));
    GOAT_TRY(cuda_status(cudaMemcpyAsync(pinned, &st->asym_count, sizeof(int), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    return pinned[0] == 0 ? GOAT_OK : GOAT_ERR_INVALID_ARG;
}

static int read_error(DevState *st, int *pinned, cudaStream_t s) {
    GOAT_TRY(cuda_status(cudaMemcpyAsync(pinned, &st->error, sizeof(int), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    return pinned[0];
}

static int match_impl(const void *A, const void *B, int n, int dtype, const float *init, float eps_rel,
                      int max_iter, float tol, const goat_params &prm, int32_t *perm_out, double *objective_out,
                      goat_stats *stats, const Plan &w, const Scratch &ws, cudaStream_t s) {
    int *pinned = pinned_words();
    if (!pinned) return GOAT_ERR_CUDA;
    DevState *st = ws.at<DevState>(w.state);
    float *P = ws.at<float>(w.P), *G = ws.at<float>(w.G), *GQ = ws.at<float>(w.GQ);
    float *f = ws.at<float>(w.f), *g = ws.at<float>(w.g);
    float *degA = ws.at<float>(w.deg), *degB = degA + n;
    double *partial = ws.at<double>(w.partial);
    __nv_bfloat16 *Xq = ws.at<__nv_bfloat16>(w.Xq);
    int32_t *perm_dev = ws.at<int32_t>(w.perm);
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
    GOAT_TRY(init_state(st, eps_rel, 1, tol, s));
    GOAT_TRY(prepare_operands(A, B, n, dtype, w, ws, st, degA, degB, pinned, s));

    if (!init) {
        barycenter(degA, degB, n, G, P, st, s);
    } else {
        GOAT_TRY(cuda_status(cudaMemcpyAsync(P, init, nn * 4, cudaMemcpyDeviceToDevice, s)));
        f32_to_terms(P, n, n, Xq, w.ld, w.terms, s);
        GOAT_TRY(gradient_from_terms(w, ws, n, G, &st->error, s));
        absmax(G, nn, &st->gmax_bits, s);
    }
    GOAT_TRY(cuda_status(cudaMemsetAsync(g, 0, (size_t)n * 4, s)));
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
    for (; it < max_iter; ++it) {
        if (prof) cudaEventRecord(pe[0], s);
        if (faq) {
            // FAQ (Alg. 1): Q = argmax over permutations of <Pi, grad f(P)> = argmin <Pi, G>;
            // an uncertified assignment is still a permutation, so it is used
            if (it == 0 && !init) {
                // at the barycenter grad f(J) is rank one: the assignment is the
                // rearrangement pairing of the degrees, solved exactly
                GOAT_TRY(rearrangement_perm(A, B, dtype, n, ws.at<void>(w.rearr), perm_dev, s));
            } else {
                LapReport drep{};
                double dgap = 0.0;
                const int dst = lap_solve(G, n, 0, perm_dev, ws.at<void>(w.lap), st, ctl,
                                          ws.at<double>(w.cost) + 6, pinned, &dgap, &drep, s);
                if (dst != GOAT_OK && dst != GOAT_ERR_NOT_CONVERGED) return dst;
            }
            if (prof) cudaEventRecord(pe[1], s);
            GOAT_TRY(write_perm_q(perm_dev, n, Xq, w.ld, w.terms, s));
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
                GOAT_TRY(mlp_warm_start_g(G, A, B, n, dtype, e0, (const __nv_bfloat16 *)prm.mlp_weights, g,
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
        GOAT_TRY(gradient_from_terms(w, ws, n, GQ, &st->error, s, prof ? pe[3] : nullptr));
        if (prof) cudaEventRecord(pe[4], s);
        line_search(G, GQ, P, Xq, w.ld, w.terms, nullptr, n, partial, st, s);
        fw_update(P, G, GQ, Xq, w.ld, w.terms, nullptr, n, st, 0.0f, &st->gmax_next, s);
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

    // projection onto the permutations
    double gap = 0.0;
    LapReport rep{};
    int lst;
    if (prm.project_on_grad) {
        // argmax tr(Pi^T grad f(P)) = argmin <Pi, G>
        lst = lap_solve(G, n, 0, perm_dev, ws.at<void>(w.lap), st, ctl, ws.at<double>(w.cost) + 6, pinned, &gap,
                        &rep, s);
    } else {
        lst = lap_solve(P, n, 1, perm_dev, ws.at<void>(w.lap), st, ctl, ws.at<double>(w.cost) + 6, pinned, &gap,
                        &rep, s);
    }
    if (lst != GOAT_OK && lst != GOAT_ERR_NOT_CONVERGED) return lst;
    cudaEventRecord(ev[3], s);

    // objective and disagreements at the returned permutation
    unsigned long long *isums = ws.at<unsigned long long>(w.cost);
    double *fsums = ws.at<double>(w.cost) + 3;
    GOAT_TRY(cuda_status(cudaMemsetAsync(isums, 0, 6 * sizeof(double), s)));
    GOAT_TRY(objective(A, B, dtype, n, perm_dev, isums, fsums, isums + 1, isums + 2, fsums + 1, fsums + 2,
                       &st->bad_perm, ws.at<double>(w.objpart), s));
    unsigned long long hi[3];
    double hf[3];
    GOAT_TRY(cuda_status(cudaMemcpyAsync(hi, isums, sizeof(hi), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaMemcpyAsync(hf, fsums, sizeof(hf), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaMemcpyAsync(perm_out, perm_dev, (size_t)n * 4, cudaMemcpyDeviceToHost, s)));
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

static bool valid_precision(int p) { return p == GOAT_PREC_BF16 || p == GOAT_PREC_FP32 || p == GOAT_PREC_FP8; }
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
    return make_plan(n, dtype_AB, precision, NEED_FW).total;
}

size_t goat_workspace_bytes_host(int n, int dtype_AB, int precision) {
    if (n < 1 || !valid_dtype(dtype_AB) || !valid_precision(precision)) return 0;
    return make_plan(n, dtype_AB, precision, NEED_FW | NEED_HOSTCOPY).total;
}

int goat_match(const void *A, const void *B, int n, int dtype_AB, const float *init, float eps_rel, int max_iter,
               float tol, const goat_params *p, int32_t *perm_out, double *objective_out, goat_stats *stats,
               void *workspace, size_t workspace_bytes, goat_stream_t stream) {
    if (!A || !B || !perm_out || n < 1 || !valid_dtype(dtype_AB) || max_iter < 0 || !(eps_rel > 0.0f) ||
        !(tol >= 0.0f) || max_iter > (1 << 20))
        return GOAT_ERR_INVALID_ARG;
    const goat_params prm = resolve_params(p);
    if (!valid_precision(prm.precision) || !valid_direction(prm.direction)) return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    cudaStream_t s = (cudaStream_t)stream;
    const Plan w = make_plan(n, dtype_AB, prm.precision, NEED_FW);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    return match_impl(A, B, n, dtype_AB, init, eps_rel, max_iter, tol, prm, perm_out, objective_out, stats, w, ws,
                      s);
}

int goat_match_host(const void *A_host, const void *B_host, int n, int dtype_AB, const float *init_host,
                    float eps_rel, int max_iter, float tol, const goat_params *p, int32_t *perm_out,
                    double *objective_out, goat_stats *stats, void *workspace, size_t workspace_bytes,
                    goat_stream_t stream) {
    if (!A_host || !B_host || !perm_out || n < 1 || !valid_dtype(dtype_AB) || max_iter < 0 || !(eps_rel > 0.0f) ||
        !(tol >= 0.0f))
        return GOAT_ERR_INVALID_ARG;
    const goat_params prm = resolve_params(p);
    if (!valid_precision(prm.precision) || !valid_direction(prm.direction)) return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    cudaStream_t s = (cudaStream_t)stream;
    // the device copies sit after the goat_match layout, so a goat_match-sized
    // workspace is not enough here: size = goat_workspace_bytes + copies
    const Plan w = make_plan(n, dtype_AB, prm.precision, NEED_FW | NEED_HOSTCOPY);
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
    return match_impl(ws.at<void>(w.Ad), ws.at<void>(w.Bd), n, dtype_AB, init_dev, eps_rel, max_iter, tol, prm,
                      perm_out, objective_out, stats, w, ws, s);
}

int goat_gradient(const void *A, const void *B, int n, int dtype_AB, const float *P, float *G_out, int precision,
                  void *workspace, size_t workspace_bytes, goat_stream_t stream) {
    if (!A || !B || !P || !G_out || n < 1 || !valid_dtype(dtype_AB) || !valid_precision(precision))
        return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    int *pinned = pinned_words();
    if (!pinned) return GOAT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const Plan w = make_plan(n, dtype_AB, precision, NEED_GEMM);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    DevState *st = ws.at<DevState>(w.state);
    GOAT_TRY(init_state(st, 0.03f, 1, 0.0f, s));
    GOAT_TRY(prepare_operands(A, B, n, dtype_AB, w, ws, st, nullptr, nullptr, pinned, s));
    f32_to_terms(P, n, n, ws.at<__nv_bfloat16>(w.Xq), w.ld, w.terms, s);
    GOAT_TRY(gradient_from_terms(w, ws, n, G_out, &st->error, s));
    const int e = read_error(st, pinned, s);
    return e;
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
    const Plan w = make_plan(n, GOAT_DTYPE_U8, GOAT_PREC_BF16, NEED_SK);
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
    const Plan w = make_plan(n, GOAT_DTYPE_U8, GOAT_PREC_BF16, NEED_SK);
    Scratch ws;
    GOAT_TRY(ws.acquire(workspace, workspace_bytes, w.total, s));
    DevState *st = ws.at<DevState>(w.state);
    GOAT_TRY(init_state(st, 0.03f, maximize ? 1 : 0, 0.0f, s));
    line_search(G, G_Q, P, nullptr, 0, 1, Q, n, ws.at<double>(w.partial), st, s);
    DevState hs;
    GOAT_TRY(cuda_status(cudaMemcpyAsync(&hs, st, offsetof(DevState, tr_sk_iters), cudaMemcpyDeviceToHost, s)));
    GOAT_TRY(cuda_status(cudaStreamSynchronize(s)));
    *alpha_out = hs.alpha;
    if (a_out) *a_out = hs.ls_a;
    if (b_out) *b_out = hs.ls_b;
    return hs.error;
}

int goat_fw_update(float *P, float *G, const float *Q, const float *G_Q, int n, double alpha, goat_stream_t stream) {
    if (!P || !G || !Q || !G_Q || n < 1 || !(alpha >= 0.0 && alpha <= 1.0)) return GOAT_ERR_INVALID_ARG;
    GOAT_TRY(device_ok());
    cudaStream_t s = (cudaStream_t)stream;
    fw_update(P, G, G_Q, nullptr, 0, 1, Q, n, nullptr, (float)alpha, nullptr, s);
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
    }
    const Plan w = make_plan(n, GOAT_DTYPE_U8, GOAT_PREC_BF16, NEED_LAP);
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
    const Plan w = make_plan(n, dtype_AB, GOAT_PREC_BF16, 0);
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
