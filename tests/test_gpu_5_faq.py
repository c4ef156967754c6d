"""FAQ (Alg. 1) on the GPU: goat_match with the exact linear-assignment direction
(params.direction = GOAT_DIR_LAP), against the oracle's FAQ (the same Frank-Wolfe
loop with the Hungarian method as the direction step).

FAQ's directions are argmax problems with ties on 0/1 graphs (Sec. 3.1), and a
tie settled differently sends the two runs apart.  The parity cases therefore use
weighted graphs (lognormal weights), whose directions are unique once the
weighted degrees are distinct: the first step, where grad f(J) = (2/n) d_A d_B^T
is rank one and the assignment is the rearrangement pairing of the degrees (the
library solves it exactly from FP64 degrees), and isomorphic pairs, which FAQ
solves in a few steps.  The weights are drawn representable in BF16, the format
the products take adjacency values in, so that the FP32 form computes the
gradient exactly and the step sizes agree with the FP64 oracle to rounding."""
import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402


def _weighted_pair(n, rho, seed):
    gp = synthetic.rho_er_pair(n, 0.1, rho, seed=seed, weighted=True)
    A = torch.from_numpy(gp.A).to(torch.bfloat16).float().numpy()
    B = torch.from_numpy(gp.B).to(torch.bfloat16).float().numpy()
    return A, B, gp.truth


def _faq_gpu(A, B, precision, **kw):
    prm = goat.default_params(precision=precision, direction=goat.GOAT_DIR_LAP)
    return goat.goat_match(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), params=prm, **kw)


def _distinct_degrees(A, B):
    dA, dB = A.astype(np.float64).sum(1), B.astype(np.float64).sum(1)
    return np.unique(dA).size == dA.size and np.unique(dB).size == dB.size


@pytest.mark.parametrize("n,seed", [(60, 1), (150, 8), (150, 4), (300, 9)])
def test_faq_first_step_matches_oracle(n, seed):
    # distinct weighted degrees: the first assignment is unique, and the GPU's must be
    # the oracle Hungarian's, exactly; the step size must be the oracle's for it
    A, B, _ = _weighted_pair(n, 0.8, seed)
    assert _distinct_degrees(A, B)
    perm, obj, st = _faq_gpu(A, B, goat.GOAT_PREC_FP32, max_iter=1, tol=1e-4)
    assert st["fw_iters"] == 1 and st["sk_iters"][0] == 0
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    J = np.full((n, n), 1.0 / n)
    grad = oracle.gradient(A64, B64, J)
    # alpha > 0, so P = (1 - alpha) J + alpha Pi projects onto the direction Pi itself
    assert st["alpha"][0] > 0
    ref, _ = oracle.lap(grad, maximize=True)
    np.testing.assert_array_equal(perm, ref)
    Pi = np.zeros((n, n))
    Pi[np.arange(n), perm] = 1.0
    alpha_paper, _, _ = oracle.step_size(A64, B64, J, Pi)
    # the oracle's alpha weights P (the paper's notation), the library's weights Q
    assert st["alpha"][0] == pytest.approx(1.0 - alpha_paper, abs=1e-5)
    assert obj == pytest.approx(oracle.objective_perm(A64, B64, perm), rel=1e-9)


def test_faq_first_step_with_tied_degrees_is_an_optimum():
    # two vertices of equal weighted degree: several first assignments are optimal
    # (Sec. 3.1's ties); the GPU's must reach the Hungarian optimum's value
    A, B, _ = _weighted_pair(300, 1.0, 6)
    assert not _distinct_degrees(A, B)
    perm, _, st = _faq_gpu(A, B, goat.GOAT_PREC_FP32, max_iter=1, tol=1e-4)
    grad = oracle.gradient(A.astype(np.float64), B.astype(np.float64), np.full((300, 300), 1.0 / 300))
    _, best = oracle.lap(grad, maximize=True)
    mine = float(grad[np.arange(300), perm].sum())
    assert mine == pytest.approx(best, rel=1e-12)


@pytest.mark.parametrize("n,seed", [(100, 5), (300, 9), (300, 2)])
def test_faq_recovers_weighted_isomorphic_pairs(n, seed):
    A, B, truth = _weighted_pair(n, 1.0, seed)
    assert _distinct_degrees(A, B)
    perm, obj, st = _faq_gpu(A, B, goat.GOAT_PREC_FP32, max_iter=30, tol=1e-4)
    ro = oracle.faq(A.astype(np.float64), B.astype(np.float64), max_iter=30, tol=1e-4)
    assert (ro["perm"] == truth).all()
    np.testing.assert_array_equal(perm, truth)
    assert st["converged"] and ro["converged"]
    # the same directions as the oracle's, hence the same number of steps and step sizes
    assert st["fw_iters"] == ro["iters"]
    np.testing.assert_allclose(st["alpha"], 1.0 - np.asarray(ro["alphas"]), atol=1e-5)
    assert obj == pytest.approx(ro["objective"], rel=1e-6)


def test_faq_is_deterministic_on_tied_inputs():
    # 0/1 graphs: many tied assignments at every step; two runs must return the same
    # permutation, the same step sizes and the same number of steps
    gp = synthetic.rho_er_pair(400, 0.05, 0.7, seed=21)
    runs = [_faq_gpu(gp.A, gp.B, goat.GOAT_PREC_BF16, max_iter=15, tol=1e-4) for _ in range(3)]
    for perm, obj, st in runs[1:]:
        np.testing.assert_array_equal(perm, runs[0][0])
        assert obj == runs[0][1]
        assert st["fw_iters"] == runs[0][2]["fw_iters"]
        assert st["alpha"] == runs[0][2]["alpha"]


@pytest.mark.parametrize("precision", [goat.GOAT_PREC_FP8, goat.GOAT_PREC_BF16, goat.GOAT_PREC_FP32])
def test_faq_every_form_returns_an_exact_objective(precision):
    # 0/1 inputs: the permutation direction is exact in every operand format
    # (1 in BF16, and 1 x 2^8 in E4M3 under the 8-bit form's scale)
    gp = synthetic.rho_er_pair(200, 0.1, 0.9, seed=11)
    perm, obj, st = _faq_gpu(gp.A, gp.B, precision, max_iter=10, tol=1e-4)
    assert sorted(perm) == list(range(200))
    assert obj == oracle.objective_perm(gp.A, gp.B, perm)
    assert st["fw_iters"] >= 1 and all(k == 0 for k in st["sk_iters"][:st["fw_iters"]])
    assert all(0.0 <= a <= 1.0 for a in st["alpha"][:st["fw_iters"]])


def test_goat_matches_more_vertices_than_faq_on_sbm():
    # Sec. 4.3 on rho-SBM pairs (n = 150, 3 blocks, rho = 0.8): the oracle gives
    # GOAT 1.0 and FAQ 0.06 mean match ratio over these six seeds
    Pb = [[0.2, 0.01, 0.01], [0.01, 0.1, 0.01], [0.01, 0.01, 0.2]]
    acc_g, acc_f = [], []
    for seed in range(6):
        gp = synthetic.rho_sbm_pair([50, 50, 50], Pb, 0.8, seed=seed)
        A, B = torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda()
        pg, _, _ = goat.goat_match(A, B, params=goat.default_params(precision=goat.GOAT_PREC_FP32))
        pf, _, _ = goat.goat_match(A, B, params=goat.default_params(precision=goat.GOAT_PREC_FP32,
                                                                    direction=goat.GOAT_DIR_LAP))
        acc_g.append((pg == gp.truth).mean())
        acc_f.append((pf == gp.truth).mean())
    assert np.mean(acc_g) >= 0.9, acc_g
    assert np.mean(acc_g) >= np.mean(acc_f) + 0.3, (acc_g, acc_f)
