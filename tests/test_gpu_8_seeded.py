"""Seeded graph matching on the GPU (Sec. 4's seeded experiment, after Fishkind et
al.): vertex i of A is known to match vertex i of B for i < m.  The iterate keeps
the form I_m (+) P22; the library solves on the unseeded block, the seeds entering
as the constant term A21 B21^T + A12^T B12 of the block's gradient.  Compared with
the oracle's seeded GOAT and FAQ (pinned in the CPU suite), on rho-SBM pairs with
the paper's block matrix.  Trajectory checks use a cold-started Sinkhorn to marginal
tolerance 1e-5 and a fixed number of steps, as in the directed tests."""
import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402

PB = [[0.7, 0.3, 0.4], [0.3, 0.7, 0.3], [0.4, 0.3, 0.7]]
TIGHT = dict(sk_warm_start=0, sk_tol=1e-5, sk_max_iter=5000)


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def align_seeds(gp, m):
    """Relabels B so that vertex i of A matches vertex i of B for i < m; returns (B, truth)."""
    n = gp.A.shape[0]
    head = [int(v) for v in gp.truth[:m]]
    taken = set(head)
    order = np.array(head + [v for v in range(n) if v not in taken])
    inv = np.empty(n, dtype=np.int64)
    inv[order] = np.arange(n)
    return np.ascontiguousarray(gp.B[np.ix_(order, order)]), inv[gp.truth]


def solve(A, B, max_iter=30, tol=0.03, **prm):
    n = A.shape[0]
    P = torch.empty((n, n), dtype=torch.float32, device="cuda")
    params = goat.default_params(relaxed_out=P, **prm)
    perm, obj, st = goat.goat_match(cuda(A), cuda(B), eps_rel=0.03, max_iter=max_iter, tol=tol, params=params)
    return perm, obj, st, P.cpu().double().numpy()


@pytest.mark.parametrize("m", [10, 37])
def test_seeded_goat_follows_oracle(m):
    gp = synthetic.rho_sbm_pair([40, 40, 40], PB, 0.6, seed=1)
    B, truth = align_seeds(gp, m)
    perm, obj, st, P = solve(gp.A, B, 6, 0.0, precision=goat.GOAT_PREC_FP32, seeds=m, **TIGHT)
    ro = oracle.goat(gp.A, B, eps_rel=0.03, max_iter=6, tol=0.0, sk_tol=1e-5, sk_max_iter=5000, seeds=m)
    np.testing.assert_array_equal(perm[:m], np.arange(m))
    assert sorted(perm) == list(range(120))
    assert st["fw_iters"] == ro["iters"] == 6
    np.testing.assert_allclose(st["alpha"], 1.0 - ro["alphas"], atol=1e-4)
    np.testing.assert_allclose(P, ro["P"], atol=1e-4)
    assert obj == oracle.objective_perm(gp.A, B, perm)
    best = ro["P"][np.arange(120), ro["perm"]].sum()
    assert ro["P"][np.arange(120), perm].sum() >= best - 120 * 1e-4


def test_seeds_turn_a_failed_match_exact():
    # the oracle pin of the seeded experiment, on the GPU: rho = 0.6, no seeds -> chance
    # level; 10 seeds -> every vertex matched
    for seed in range(2):
        gp = synthetic.rho_sbm_pair([40, 40, 40], PB, 0.6, seed=seed)
        perm0, _, _, _ = solve(gp.A, gp.B)
        assert (perm0 == gp.truth).mean() < 0.1
        B, truth = align_seeds(gp, 10)
        for precision in (goat.GOAT_PREC_FP32, goat.GOAT_PREC_BF16, goat.GOAT_PREC_FP8):
            perm, _, _, _ = solve(gp.A, B, precision=precision, seeds=10)
            np.testing.assert_array_equal(perm, truth)


def test_seeded_faq_follows_oracle():
    # weighted graphs: FAQ's assignments are unique, so the two runs take the same steps
    gp = synthetic.rho_sbm_pair([40, 40, 40], PB, 0.5, seed=3, weighted=True)
    A = torch.from_numpy(gp.A).to(torch.bfloat16).float().numpy()
    Bw = torch.from_numpy(gp.B).to(torch.bfloat16).float().numpy()
    gp_w = synthetic.GraphPair(A=A, B=Bw, truth=gp.truth, n=gp.n, seed=gp.seed)
    B, truth = align_seeds(gp_w, 20)
    perm, obj, st, _ = solve(A, B, 20, 1e-4, precision=goat.GOAT_PREC_FP32, seeds=20, direction=goat.GOAT_DIR_LAP)
    ro = oracle.faq(A.astype(np.float64), B.astype(np.float64), max_iter=20, tol=1e-4, seeds=20)
    np.testing.assert_array_equal(perm, ro["perm"])
    assert st["fw_iters"] == ro["iters"]
    np.testing.assert_allclose(st["alpha"], 1.0 - np.asarray(ro["alphas"]), atol=1e-5)
    assert obj == pytest.approx(ro["objective"], rel=1e-9)


def test_full_and_near_full_seeding_is_the_identity():
    gp = synthetic.rho_er_pair(50, 0.2, 0.7, seed=5)
    for m in (49, 50):
        perm, obj, st, P = solve(gp.A, gp.B, seeds=m)
        np.testing.assert_array_equal(perm, np.arange(50))
        assert obj == oracle.objective_perm(gp.A, gp.B, np.arange(50))
        np.testing.assert_array_equal(P, np.eye(50))
    assert solve(gp.A, gp.B, seeds=50)[2]["fw_iters"] == 0


def test_seeded_directed_follows_oracle():
    gp = synthetic.rho_er_digraph_pair(130, 0.12, 0.7, seed=9)
    B, truth = align_seeds(gp, 15)
    perm, obj, st, P = solve(gp.A, B, 5, 0.0, precision=goat.GOAT_PREC_FP32, seeds=15, directed=1, **TIGHT)
    ro = oracle.goat(gp.A, B, eps_rel=0.03, max_iter=5, tol=0.0, sk_tol=1e-5, sk_max_iter=5000, seeds=15)
    np.testing.assert_allclose(st["alpha"], 1.0 - ro["alphas"], atol=1e-4)
    np.testing.assert_allclose(P, ro["P"], atol=1e-4)
    np.testing.assert_array_equal(perm[:15], np.arange(15))
    assert obj == oracle.objective_perm(gp.A, B, perm)


def test_seeded_workspace_and_bad_seed_counts():
    n, m = 64, 10
    # the plan is laid out for the unseeded block: at least its FP32 G, P and the step's
    # gradient, plus the seeds' constant term; a seeded solve runs in exactly that room
    wb = goat.workspace_bytes(n, seeds=m)
    assert wb >= 4 * 4 * (n - m) ** 2
    assert goat.workspace_bytes(n, seeds=n + 1) == 0
    gp = synthetic.rho_er_pair(n, 0.2, 0.9, seed=2)
    ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
    perm, obj, _ = goat.goat_match(cuda(gp.A), cuda(gp.B), params=goat.default_params(seeds=m), workspace=ws)
    np.testing.assert_array_equal(perm[:m], np.arange(m))
    assert obj == oracle.objective_perm(gp.A, gp.B, perm)
    with pytest.raises(goat.GoatError):
        goat.goat_match(cuda(gp.A), cuda(gp.B), params=goat.default_params(seeds=n + 1))
