"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the paper's
worked example, brute force over all permutations, closed forms, a library
routine (scipy's linear_sum_assignment) on the same special case, invariants,
and identities between independently coded routines.  Together they are chosen
so that a dropped term, a sign error, a swapped index or a transposed operand in
any oracle routine fails at least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic


def rand_graph(n, p, seed, directed=False, weighted=False):
    rng = np.random.default_rng(seed)
    A = (rng.random((n, n)) < p).astype(np.float64)
    np.fill_diagonal(A, 0.0)
    if not directed:
        A = np.triu(A, 1)
        A = A + A.T
    if weighted:
        A = A * rng.lognormal(0.0, 1.0, size=(n, n))
    return A


def random_ds(n, seed):
    """A random doubly stochastic matrix (convex mix of permutation matrices)."""
    rng = np.random.default_rng(seed)
    P = np.zeros((n, n))
    w = rng.random(5)
    w /= w.sum()
    for k in range(5):
        P[np.arange(n), rng.permutation(n)] += w[k]
    return P


# --------------------------------------------------------------- objective

def test_objective_perm_matches_trace_and_brute_force():
    # eq. (QAP): f(P) = tr(A^T P B P^T); at a permutation it is sum A_ij B[pi i, pi j]
    for seed in range(5):
        n = 6
        A = rand_graph(n, 0.5, seed, directed=True, weighted=True)
        B = rand_graph(n, 0.5, seed + 100, directed=True, weighted=True)
        for perm in itertools.islice(itertools.permutations(range(n)), 0, 720, 97):
            perm = np.array(perm)
            P = np.zeros((n, n)); P[np.arange(n), perm] = 1.0
            direct = sum(A[i, j] * B[perm[i], perm[j]] for i in range(n) for j in range(n))
            assert oracle.objective_perm(A, B, perm) == pytest.approx(direct, rel=1e-13)
            assert oracle.objective(A, B, P) == pytest.approx(direct, rel=1e-13)
            # written out from the definition with numpy's matmul
            assert np.trace(A.T @ P @ B @ P.T) == pytest.approx(direct, rel=1e-13)


def test_gm_is_negated_qap():
    # Sec. 2.2: ||A - P B P^T||_F^2 = ||A||^2 + ||B||^2 - 2 tr(A^T P B P^T) at permutations,
    # so minimising disagreements = maximising f (the printed "+2 tr(...)" is a sign garble).
    rng = np.random.default_rng(3)
    n = 7
    A = rand_graph(n, 0.4, 1)
    B = rand_graph(n, 0.4, 2)
    for _ in range(20):
        perm = rng.permutation(n)
        P = np.zeros((n, n)); P[np.arange(n), perm] = 1.0
        dis = np.sum((A - P @ B @ P.T) ** 2)
        f = oracle.objective_perm(A, B, perm)
        assert dis == pytest.approx(A.sum() + B.sum() - 2 * f, abs=1e-12)
    # brute force: the argmax of f has the fewest disagreements
    fbest, pbest = oracle.brute_qap(A, B, maximize=True)
    best_dis = min(np.sum((A - B[np.ix_(p, p)]) ** 2) for p in map(np.array, itertools.permutations(range(n))))
    assert A.sum() + B.sum() - 2 * fbest == pytest.approx(best_dis)


def test_brute_qap_isomorphic_pair_reaches_edge_count():
    # rho = 1 pair: the hidden correspondence attains f = ||A||^2, the largest possible value
    gp = synthetic.rho_er_pair(7, 0.5, 1.0, seed=11)
    A, B = gp.A.astype(float), gp.B.astype(float)
    fbest, _ = oracle.brute_qap(A, B)
    assert fbest == A.sum()
    assert oracle.objective_perm(A, B, gp.truth) == A.sum()


# --------------------------------------------------------------- gradient

def test_gradient_closed_form_at_barycenter():
    # grad f(J) = A J B^T + A^T J B = (d_out(A) d_out(B)^T + d_in(A) d_in(B)^T) / n, J = 11^T/n
    n = 23
    A = rand_graph(n, 0.3, 5, directed=True, weighted=True)
    B = rand_graph(n, 0.3, 6, directed=True, weighted=True)
    J = np.full((n, n), 1.0 / n)
    G = oracle.gradient(A, B, J)
    expect = (np.outer(A.sum(1), B.sum(1)) + np.outer(A.sum(0), B.sum(0))) / n
    np.testing.assert_allclose(G, expect, rtol=1e-13, atol=1e-13)


def test_gradient_index_form_at_permutation():
    # at P = Pi: (A Pi B^T)_ij = sum_k A_ik B[j, pi k] and (A^T Pi B)_ij = sum_k A_ki B[pi k, j]
    n = 17
    A = rand_graph(n, 0.3, 7, directed=True)
    B = rand_graph(n, 0.3, 8, directed=True)
    perm = np.random.default_rng(9).permutation(n)
    P = np.zeros((n, n)); P[np.arange(n), perm] = 1.0
    G = oracle.gradient(A, B, P)
    expect = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            expect[i, j] = sum(A[i, k] * B[j, perm[k]] + A[k, i] * B[perm[k], j] for k in range(n))
    np.testing.assert_array_equal(G, expect)  # integer matrix, exact


def test_gradient_euler_and_central_difference():
    # f is a homogeneous quadratic: <grad f(P), P> = 2 f(P), and the central
    # difference f(P + tD) - f(P - tD) = 2 t <grad f(P), D> holds exactly.
    n = 15
    for seed in range(3):
        A = rand_graph(n, 0.4, seed, directed=True, weighted=True)
        B = rand_graph(n, 0.4, seed + 50, directed=True, weighted=True)
        rng = np.random.default_rng(seed)
        P = rng.random((n, n))
        D = rng.standard_normal((n, n))
        G = oracle.gradient(A, B, P)
        assert np.sum(G * P) == pytest.approx(2 * oracle.objective(A, B, P), rel=1e-12)
        t = 0.25
        cd = oracle.objective(A, B, P + t * D) - oracle.objective(A, B, P - t * D)
        assert cd == pytest.approx(2 * t * np.sum(G * D), rel=1e-10, abs=1e-9)


def test_gradient_rows_match_full_gradient():
    n = 40
    A = rand_graph(n, 0.2, 1, directed=True)
    B = rand_graph(n, 0.2, 2, directed=True)
    P = random_ds(n, 3).astype(np.float32)
    G = oracle.gradient(A, B, P.astype(np.float64))
    rows = np.array([0, 5, 39, 17])
    Gr = oracle.gradient_rows(A.astype(np.uint8), B.astype(np.uint8), P, rows)
    np.testing.assert_allclose(Gr, G[rows], rtol=1e-13, atol=1e-13)
    Aw = rand_graph(n, 0.2, 1, directed=True, weighted=True).astype(np.float32)
    Gw = oracle.gradient(Aw.astype(np.float64), B, P.astype(np.float64))
    Grw = oracle.gradient_rows(Aw, B.astype(np.float32), P, rows)
    np.testing.assert_allclose(Grw, Gw[rows], rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------- Sinkhorn / LOT

def test_sinkhorn_marginals_tight():
    # Sec. 3.3: the LOT direction lies in D, rows and columns summing to 1 (within 1e-9)
    n = 60
    M = -np.random.default_rng(1).random((n, n)) * 10
    eps = 0.03 * np.abs(M).max()
    Q, f, g, it, resid = oracle.lot(M, eps, 1e-12, 100000)
    assert resid < 1e-12
    np.testing.assert_allclose(Q.sum(1), 1.0, atol=1e-9)
    np.testing.assert_allclose(Q.sum(0), 1.0, atol=1e-9)
    assert (Q > 0).all()
    # dual form: Q_ij = exp((f_i + g_j - M_ij)/eps)
    np.testing.assert_allclose(Q, np.exp((f[:, None] + g[None, :] - M) / eps), rtol=1e-10)


def test_sinkhorn_separable_cost_gives_barycenter():
    # K = exp(-(a_i + b_j)/eps) has rank one, so the doubly stochastic scaling is J = 11^T/n
    n = 9
    rng = np.random.default_rng(2)
    a, b = rng.random(n) * 3, rng.random(n) * 5
    M = a[:, None] + b[None, :]
    Q, *_ = oracle.lot(M, 0.7, 1e-13, 1000)
    np.testing.assert_allclose(Q, np.full((n, n), 1.0 / n), atol=1e-12)
    Qc, *_ = oracle.lot(np.full((n, n), 4.2), 0.1, 1e-13, 1000)
    np.testing.assert_allclose(Qc, np.full((n, n), 1.0 / n), atol=1e-12)


def test_sinkhorn_two_by_two_closed_form():
    # For n = 2, D = {[[t, 1-t], [1-t, t]]}; minimising <Q, M> + eps sum Q log Q gives
    # t = 1 / (1 + exp(Delta / (2 eps))), Delta = M00 + M11 - M01 - M10.
    rng = np.random.default_rng(3)
    for _ in range(10):
        M = rng.standard_normal((2, 2)) * 2
        eps = float(rng.uniform(0.3, 3))
        delta = M[0, 0] + M[1, 1] - M[0, 1] - M[1, 0]
        t = 1.0 / (1.0 + np.exp(delta / (2 * eps)))
        Q, *_ = oracle.lot(M, eps, 1e-14, 100000)
        np.testing.assert_allclose(Q, [[t, 1 - t], [1 - t, t]], atol=1e-12)
        Ql, *_ = oracle.lot_log(M, eps, 1e-14, 100000)
        np.testing.assert_allclose(Ql, [[t, 1 - t], [1 - t, t]], atol=1e-12)


def test_log_and_scaling_domain_agree_with_warm_start():
    n = 30
    rng = np.random.default_rng(4)
    M = -rng.random((n, n)) * 20
    eps = 0.03 * np.abs(M).max()
    g0 = rng.standard_normal(n) * eps
    Q1, f1, g1, it1, r1 = oracle.lot(M, eps, 1e-3, 7, g_init=g0)
    Q2, f2, g2, it2, r2 = oracle.lot_log(M, eps, 1e-3, 7, g_init=g0)
    assert it1 == it2
    np.testing.assert_allclose(Q1, Q2, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(f1, f2, atol=1e-10 * eps)
    np.testing.assert_allclose(g1, g2, atol=1e-10 * eps)
    assert r1 == pytest.approx(r2, rel=1e-8, abs=1e-14)
    # block-row / block-column forms agree with one full iteration
    rows = np.array([0, 7, 29])
    M32, g32 = M.astype(np.float32), g0.astype(np.float32)
    fr = oracle.lot_rows(M32[rows], g32, eps)
    _, fl, gl, _, _ = oracle.lot_log(M32.astype(np.float64), eps, 0.0, 1, g_init=g32.astype(np.float64))
    np.testing.assert_allclose(fr, fl[rows], atol=1e-12 * eps)
    # column sums of the row-scaled Q (before the column scaling) give g_new = g - eps log S
    f32 = fl.astype(np.float32)
    S = oracle.lot_colsums(M32[:, rows], f32, g32[rows], eps)
    Sfull = np.exp((f32.astype(np.float64)[:, None] + g32.astype(np.float64)[None, :] - M32.astype(np.float64)) / eps).sum(0)
    np.testing.assert_allclose(S, Sfull[rows], rtol=1e-12)


def test_sinkhorn_small_eps_recovers_unique_lap_optimum():
    # as eps -> 0 the entropic solution tends to the LAP optimum (unique here)
    n = 8
    M = np.random.default_rng(5).random((n, n))
    _, perm_b, nopt = oracle.brute_lap(M, maximize=False)
    assert nopt == 1
    Q, *_ = oracle.lot_log(M, 0.002, 1e-10, 200000)
    assert (Q.argmax(1) == perm_b).all()
    assert np.sum(Q * M) == pytest.approx(M[np.arange(n), perm_b].sum(), abs=1e-3)


def test_lemma1_tie_gives_midpoint(golden):
    # Sec. 3.1 + Lemma 1: the tied optima P1, P2 of the worked example; every convex
    # combination is optimal over D, and the entropic solution at small eps is the
    # maximum-entropy point of that optimal face, the midpoint (P1 + P2)/2.
    g = golden("paper_4x4_tie.txt")
    M = np.array(g["matrix"])
    P1 = np.zeros((4, 4)); P1[np.arange(4), np.array(g["P1"], int)] = 1
    P2 = np.zeros((4, 4)); P2[np.arange(4), np.array(g["P2"], int)] = 1
    for lam in np.linspace(0, 1, 11):
        assert np.sum((lam * P1 + (1 - lam) * P2) * M) == pytest.approx(g["value"][0])
    # The next-best permutation costs 1 more, so the entropic bias is of order
    # exp(-1/eps); Sinkhorn converges only sublinearly on this tied problem,
    # hence the long run at a moderate eps.
    Q, _, _, it, resid = oracle.lot_log(M, 0.1, 1e-13, 2_000_000)
    assert resid < 1e-12
    np.testing.assert_allclose(Q, 0.5 * (P1 + P2), atol=2 * np.exp(-1 / 0.1))


# --------------------------------------------------------------- linear assignment

def test_lap_paper_example(golden):
    g = golden("paper_4x4_tie.txt")
    M = np.array(g["matrix"])
    ties = {tuple(int(x) for x in g["P1"]), tuple(int(x) for x in g["P2"])}
    for key in ("P1", "P2"):
        p = np.array(g[key], int)
        assert M[np.arange(4), p].sum() == g["value"][0]
    cost, perm, nopt = oracle.brute_lap(M, maximize=False)
    assert cost == g["value"][0] and nopt == 2
    perm_h, cost_h = oracle.lap(M, maximize=False)
    assert cost_h == g["value"][0] and tuple(perm_h) in ties
    # the maximum (not printed by the paper): brute force and Hungarian agree
    cmax, _, nmax = oracle.brute_lap(M, maximize=True)
    _, cost_hmax = oracle.lap(M, maximize=True)
    assert cost_hmax == cmax == 183 and nmax == 2


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_lap_vs_brute_force(n):
    for seed in range(30):
        rng = np.random.default_rng(seed)
        C = rng.integers(0, 5, size=(n, n)).astype(float) if seed % 2 else rng.standard_normal((n, n))
        for mx in (True, False):
            cb, _, _ = oracle.brute_lap(C, maximize=mx)
            perm, ch = oracle.lap(C, maximize=mx)
            assert sorted(perm) == list(range(n))
            assert ch == pytest.approx(cb, abs=1e-12)


def test_lap_vs_scipy_and_duals():
    scipy_opt = pytest.importorskip("scipy.optimize")
    for n, seed in [(50, 0), (137, 1), (300, 2)]:
        rng = np.random.default_rng(seed)
        C = rng.uniform(100, 150, size=(n, n))   # Fig. 1 cost distribution
        r, c = scipy_opt.linear_sum_assignment(C)
        perm, cost, u, v = oracle.lap_min_with_duals(C)
        assert cost == pytest.approx(C[r, c].sum(), rel=1e-13)
        red = C - u[:, None] - v[None, :]
        assert red.min() > -1e-9                                      # dual feasible
        assert np.abs(red[np.arange(n), perm]).max() < 1e-9           # complementary slackness
        _, cmax = oracle.lap(C, maximize=True)
        r, c = scipy_opt.linear_sum_assignment(C, maximize=True)
        assert cmax == pytest.approx(C[r, c].sum(), rel=1e-13)


def test_lap_certificate_detects_suboptimal():
    n = 20
    C = np.random.default_rng(1).random((n, n)).astype(np.float32)
    perm, cost = oracle.lap(C.astype(np.float64), maximize=True)
    # duals of the max problem from the min problem on -C
    p2, c2, u, v = oracle.lap_min_with_duals(-C.astype(np.float64))
    viol, gap = oracle.lap_certificate(C, p2, -u, -v)
    assert viol < 1e-12 and abs(gap) < 1e-9
    bad = p2.copy(); bad[[0, 1]] = bad[[1, 0]]
    _, gap_bad = oracle.lap_certificate(C, bad, -u, -v)
    assert gap_bad > 1e-6 or C[0, p2[1]] + C[1, p2[0]] == C[0, p2[0]] + C[1, p2[1]]


# --------------------------------------------------------------- step size

def test_step_size_coefficients_from_objective():
    # f(alpha P + (1-alpha) Q) = f(Q) + b alpha + a alpha^2; three objective values fix (a, b)
    n = 14
    for seed in range(4):
        A = rand_graph(n, 0.4, seed, directed=bool(seed % 2))
        B = rand_graph(n, 0.4, seed + 9, directed=bool(seed % 2))
        P, Q = random_ds(n, seed), random_ds(n, seed + 20)
        alpha, a, b = oracle.step_size(A, B, P, Q)
        f0 = oracle.objective(A, B, Q)
        fh = oracle.objective(A, B, 0.5 * P + 0.5 * Q)
        f1 = oracle.objective(A, B, P)
        a_fit = 2 * (f1 - 2 * fh + f0)
        b_fit = f1 - f0 - a_fit
        assert a == pytest.approx(a_fit, rel=1e-9, abs=1e-9)
        assert b == pytest.approx(b_fit, rel=1e-9, abs=1e-9)


def test_step_size_is_grid_optimal_in_unit_interval():
    n = 12
    grid = np.linspace(0, 1, 10001)
    for seed in range(8):
        A = rand_graph(n, 0.5, seed)
        B = rand_graph(n, 0.5, seed + 3)
        P, Q = random_ds(n, seed), random_ds(n, seed + 40)
        for mx in (True, False):
            alpha, a, b = oracle.step_size(A, B, P, Q, maximize=mx)
            assert 0.0 <= alpha <= 1.0
            phi = lambda t: oracle.objective(A, B, t * P + (1 - t) * Q)
            vals = b * grid + a * grid ** 2
            best = vals.max() if mx else vals.min()
            got = b * alpha + a * alpha ** 2
            if mx:
                assert got >= best - 1e-9
                assert phi(alpha) >= phi(1.0) - 1e-9   # never worse than staying at P
            else:
                assert got <= best + 1e-9
                assert phi(alpha) <= phi(1.0) + 1e-9


# --------------------------------------------------------------- end to end

def test_goat_recovers_isomorphic_pairs():
    # rho = 1: GOAT finds the exact correspondence (Sec. 4.2 / Fig. 2 claim of exact recovery)
    for seed in range(5):
        gp = synthetic.rho_er_pair(100, 0.1, 1.0, seed=seed)
        r = oracle.goat(gp.A, gp.B)
        assert (r["perm"] == gp.truth).all()
        assert r["objective"] == gp.A.sum()


def test_goat_relaxed_iterates_stay_doubly_stochastic_and_improve():
    gp = synthetic.rho_er_pair(60, 0.15, 0.8, seed=4)
    A, B = gp.A.astype(float), gp.B.astype(float)
    f_prev = oracle.objective(A, B, np.full((60, 60), 1 / 60))
    P = None
    for it in range(1, 6):
        r = oracle.goat(A, B, max_iter=it, tol=0.0, sk_tol=1e-8, sk_max_iter=5000)
        P = r["P"]
        f_now = oracle.objective(A, B, P)
        assert f_now >= f_prev - 1e-9       # the line search never decreases the objective
        f_prev = f_now
        np.testing.assert_allclose(P.sum(0), 1, atol=1e-7)
        np.testing.assert_allclose(P.sum(1), 1, atol=1e-7)
        assert (r["alphas"] >= 0).all() and (r["alphas"] <= 1).all()


def test_goat_small_pairs_reach_brute_force_optimum_on_isomorphic_graphs():
    hits = 0
    for seed in range(6):
        gp = synthetic.rho_er_pair(8, 0.4, 1.0, seed=seed)
        A, B = gp.A.astype(float), gp.B.astype(float)
        fbest, _ = oracle.brute_qap(A, B)
        r = oracle.goat(A, B)
        assert r["objective"] <= fbest
        hits += r["objective"] == fbest
    assert hits >= 4


def test_goat_at_least_faq_on_sbm():
    # Sec. 4.3: on rho-SBM pairs (n=150, k=3) GOAT's match ratio is >= FAQ's
    Pb = [[0.2, 0.01, 0.01], [0.01, 0.1, 0.01], [0.01, 0.01, 0.2]]
    acc_g, acc_f = [], []
    for seed in range(6):
        gp = synthetic.rho_sbm_pair([50, 50, 50], Pb, 0.8, seed=seed)
        rg = oracle.goat(gp.A, gp.B)
        rf = oracle.faq(gp.A, gp.B)
        acc_g.append((rg["perm"] == gp.truth).mean())
        acc_f.append((rf["perm"] == gp.truth).mean())
    assert np.mean(acc_g) >= np.mean(acc_f)


def test_faq_first_direction_is_the_degree_rearrangement():
    # at J the gradient is (2/n) d_A d_B^T, so FAQ's first direction maximises
    # sum_i d_A(i) d_B(pi(i)): by the rearrangement inequality it pairs the vertices
    # of equal degree rank (unique when the weighted degrees are distinct); the
    # first step's relaxed iterate then projects back onto that pairing
    for n, seed in [(60, 1), (150, 8)]:
        gp = synthetic.rho_er_pair(n, 0.1, 0.8, seed=seed, weighted=True)
        A, B = gp.A.astype(np.float64), gp.B.astype(np.float64)
        dA, dB = A.sum(1), B.sum(1)
        assert np.diff(np.sort(dA)).min() > 0 and np.diff(np.sort(dB)).min() > 0
        r = oracle.faq(A, B, max_iter=1, tol=1e-4)
        want = np.empty(n, dtype=np.int32)
        want[np.argsort(dA)] = np.argsort(dB)
        np.testing.assert_array_equal(r["perm"], want)
        assert 0.0 <= r["alphas"][0] < 1.0  # a real step towards the direction (paper's alpha weights P)


def test_lot_objective_within_half_percent_of_lap_on_fig1_costs():
    # Sec. 3.3, Fig. 1: Uniform(100, 150) costs, lambda >= 100; LOT's relaxed
    # objective <Q, M> stays within 0.5 % of the LAP optimum.  Below it only by the
    # marginal error of an inexact Q (Birkhoff: the LP attains the LAP optimum).
    for n, seed in [(100, 1), (250, 2)]:
        M = synthetic.uniform_costs(n, 100, 150, seed)
        _, lap_cost = oracle.lap(M, maximize=False)
        Q, _, _, _, resid = oracle.lot_log(M, 0.01, 1e-3, 20000)
        assert resid < 1e-3
        ofv = float((Q * M).sum())
        assert abs(lap_cost - ofv) / lap_cost < 5e-3
        assert ofv >= lap_cost * (1 - 2e-3)


# --------------------------------------------------------------- seeded matching

def _align_seeds(gp, m):
    """Relabels B so that vertex i of A matches vertex i of B for i < m; returns (B, truth)."""
    n = gp.A.shape[0]
    head = [int(v) for v in gp.truth[:m]]
    taken = set(head)
    order = np.array(head + [v for v in range(n) if v not in taken])
    inv = np.empty(n, dtype=np.int64)
    inv[order] = np.arange(n)
    return gp.B[np.ix_(order, order)], inv[gp.truth]


def test_seeded_gradient_block_is_the_seeded_objective_gradient():
    # with P = I_m (+) P22 and symmetric graphs, f = tr(A11 B11) + 2 tr(P22^T A21 B21^T)
    # + tr(A22 P22 B22 P22^T), whose gradient in P22 is 2 A21 B21^T + 2 A22 P22 B22:
    # the unseeded block of the full gradient, which the seeded method steps along
    gp = synthetic.rho_er_pair(40, 0.2, 0.8, seed=4)
    A, B = gp.A.astype(np.float64), gp.B.astype(np.float64)
    m = 9
    P22 = random_ds(40 - m, 3)
    P = np.zeros((40, 40))
    P[:m, :m] = np.eye(m)
    P[m:, m:] = P22
    want = 2 * A[m:, :m] @ B[m:, :m].T + 2 * A[m:, m:] @ P22 @ B[m:, m:]
    np.testing.assert_allclose(oracle.gradient(A, B, P)[m:, m:], want, rtol=1e-12, atol=1e-12)
    f_blocks = (np.trace(A[:m, :m] @ B[:m, :m]) + 2 * np.sum(P22 * (A[m:, :m] @ B[m:, :m].T))
                + np.trace(A[m:, m:] @ P22 @ B[m:, m:] @ P22.T))
    assert oracle.objective(A, B, P) == pytest.approx(f_blocks, rel=1e-12)


def test_seeds_are_kept_and_full_seeding_is_the_identity():
    gp = synthetic.rho_er_pair(30, 0.2, 0.7, seed=5)
    for m in (0, 1, 12, 29, 30):
        for lap in (False, True):
            r = oracle.goat(gp.A, gp.B, seeds=m, use_lap=lap)
            np.testing.assert_array_equal(r["perm"][:m], np.arange(m))
            assert sorted(r["perm"]) == list(range(30))
            if m >= 29:  # at most one free vertex: nothing to solve
                np.testing.assert_array_equal(r["perm"], np.arange(30))
    assert oracle.goat(gp.A, gp.B, seeds=30)["iters"] == 0


def test_seeded_small_pairs_against_brute_force():
    # the seeded result never beats the best seed-respecting permutation, and reaches
    # it on isomorphic pairs
    n, m = 7, 3
    for seed in range(4):
        gp = synthetic.rho_er_pair(n, 0.5, 1.0, seed=seed)
        B, truth = _align_seeds(gp, m)
        A64, B64 = gp.A.astype(np.float64), B.astype(np.float64)
        best = max(oracle.objective_perm(A64, B64, np.array(list(range(m)) + [m + q for q in rest]))
                   for rest in itertools.permutations(range(n - m)))
        assert oracle.objective_perm(A64, B64, truth) == best
        for lap in (False, True):
            r = oracle.goat(A64, B64, seeds=m, use_lap=lap)
            assert r["objective"] <= best + 1e-9
        assert oracle.goat(A64, B64, seeds=m)["objective"] == best


def test_seeds_recover_sbm_pairs():
    # Sec. 4 (seeded experiment, after Fishkind et al.): on rho-SBM pairs with the
    # paper's block matrix, a few seeds turn a failed unseeded match into an exact one
    # (rho = 0.6), and GOAT matches at least as many vertices as FAQ with seeds (rho = 0.3)
    Pb = [[0.7, 0.3, 0.4], [0.3, 0.7, 0.3], [0.4, 0.3, 0.7]]
    acc = {}
    for rho, m in ((0.6, 0), (0.6, 10), (0.3, 30)):
        g, f = [], []
        for seed in range(2):
            gp = synthetic.rho_sbm_pair([40, 40, 40], Pb, rho, seed=seed)
            B, truth = _align_seeds(gp, m)
            g.append((oracle.goat(gp.A, B, seeds=m)["perm"] == truth).mean())
            f.append((oracle.faq(gp.A, B, seeds=m)["perm"] == truth).mean())
        acc[rho, m] = (np.mean(g), np.mean(f))
    assert acc[0.6, 0][0] < 0.1 and acc[0.6, 10][0] == 1.0
    assert acc[0.3, 30][0] >= acc[0.3, 30][1]


def test_projection_on_gradient_variant_runs():
    gp = synthetic.rho_er_pair(50, 0.2, 1.0, seed=2)
    r = oracle.goat(gp.A, gp.B, project_on_grad=True)
    assert (r["perm"] == gp.truth).all()


# --------------------------------------------------------------- random starts

def test_splitmix64_published_first_output():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 0: the first output is 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF


def test_random_start_is_half_barycenter_half_scaled_noise():
    # Sec. 3.4: P0 = (J + K)/2 with K doubly stochastic, so P0 is doubly stochastic and >= 1/(2n)
    for n, q in [(5, 0), (40, 3), (123, 17)]:
        P0 = oracle.random_start(n, 99, q)
        np.testing.assert_allclose(P0.sum(0), 1, atol=1e-10)
        np.testing.assert_allclose(P0.sum(1), 1, atol=1e-10)
        assert P0.min() >= 0.5 / n - 1e-15
        K = 2 * P0 - 1.0 / n
        # K is the Sinkhorn-Knopp scaling of the noise: K_ij / U_ij = u_i v_j has rank one
        U = np.array([[((oracle.splitmix64(99, (q << 32) | (i * n + j)) >> 40) + 1) / 2 ** 24
                       for j in range(n)] for i in range(n)])
        R = K / U
        np.testing.assert_allclose(R / R[:, :1] / (R[:1, :] / R[0, 0]), 1.0, rtol=1e-8)
    assert not np.allclose(oracle.random_start(30, 1, 0), oracle.random_start(30, 1, 1))


# --------------------------------------------------------------- learned warm start (definitions)

def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    prm = rng.standard_normal(641) * 0.3
    x = rng.standard_normal((37, 8))
    t = rng.standard_normal(37)
    L, grad, y = oracle.mlp_loss_grad(prm, x, t)
    h = 1e-6
    for k in list(range(0, 512, 53)) + [512, 530, 575, 576, 600, 639, 640]:
        e = np.zeros(641); e[k] = h
        Lp, _, _ = oracle.mlp_loss_grad(prm + e, x, t)
        Lm, _, _ = oracle.mlp_loss_grad(prm - e, x, t)
        assert grad[k] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6, abs=1e-9)
    # outputs from the definition with numpy
    W1, b1, w2, b2 = prm[:512].reshape(64, 8), prm[512:576], prm[576:640], prm[640]
    np.testing.assert_allclose(y, np.tanh(x @ W1.T + b1) @ w2 + b2, rtol=1e-12)
    assert L == pytest.approx(np.mean((y - t) ** 2), rel=1e-12)


def test_dual_features_closed_form_at_barycenter():
    # at the barycenter G = -(2/n) d_A d_B^T: row i is -(2/n) d_A(i) d_B, column j is -(2/n) d_B(j) d_A
    gp = synthetic.rho_er_pair(60, 0.2, 0.8, seed=3)
    A, B = gp.A.astype(float), gp.B.astype(float)
    n = 60
    dA, dB = A.sum(1), B.sum(1)
    G = -2.0 / n * np.outer(dA, dB)
    eps = 0.03 * np.abs(G).max()
    F = oracle.dual_features(G, A, B, eps)
    c = -2.0 / n / eps
    np.testing.assert_allclose(F[:n, 2], c * dA * dB.mean(), rtol=1e-12)
    np.testing.assert_allclose(F[:n, 3], c * dA * dB.min(), rtol=1e-12)
    np.testing.assert_allclose(F[:n, 5], c * dA * dB.max(), rtol=1e-12)
    np.testing.assert_allclose(F[:n, 4], -c * dA * dB.std(), rtol=1e-9)
    np.testing.assert_allclose(F[n:, 2], c * dB * dA.mean(), rtol=1e-12)
    np.testing.assert_allclose(F[:n, 0], dA / dA.mean(), rtol=1e-12)
    np.testing.assert_allclose(F[n:, 1], (B @ dB) / (B @ dB).mean(), rtol=1e-12)
    assert (F[:n, 6] == 0).all() and (F[n:, 6] == 1).all()
    np.testing.assert_allclose(F[:, 7], np.log(n) / 10)
