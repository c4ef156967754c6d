"""Directed graphs and QAP minimisation through goat_match (Alg. 1 / Alg. 3 with no
symmetry shortcut, and eq. QAP's minimisation), against the FP64 oracle, which
assumes no symmetry and takes `maximize`.

For general graphs grad f(P) = A P B^T + A^T P B needs four products; the library
computes C1 = B P^T and C1' = B^T P^T, then [A | A^T] [C1 | C1']^T in one
tensor-core accumulation.  Minimising f runs the same iteration on G = +grad f.

Trajectory checks run both sides with a cold-started Sinkhorn to a tight marginal
tolerance (1e-5) and no stop test (tol = 0, a fixed number of steps), so each
direction is the same entropic optimum up to FP32 rounding: the step sizes and the
relaxed iterate then agree to about 1e-5.  The inputs are 0/1 graphs or weights
drawn representable in BF16 (the format the products take adjacency values in)."""
import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def bf16_exact(x):
    return torch.from_numpy(x).to(torch.bfloat16).float().numpy()


def random_ds(n, seed, k=4):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, n))
    for w in rng.random(k) + 0.1:
        P[np.arange(n), rng.permutation(n)] += w
    P /= P.sum(1, keepdims=True)
    return P


def rel_err(G, ref):
    return float(np.linalg.norm(G - ref) / np.linalg.norm(ref))


def solve(A, B, max_iter, tol, **prm):
    n = A.shape[0]
    P = torch.empty((n, n), dtype=torch.float32, device="cuda")
    params = goat.default_params(relaxed_out=P, **prm)
    perm, obj, st = goat.goat_match(cuda(A), cuda(B), eps_rel=0.03, max_iter=max_iter, tol=tol, params=params)
    return perm, obj, st, P.cpu().double().numpy()


TIGHT = dict(sk_warm_start=0, sk_tol=1e-5, sk_max_iter=5000)


@pytest.mark.parametrize("n", [300, 777])
@pytest.mark.parametrize("precision,bound", [(goat.GOAT_PREC_FP32, 1e-5), (goat.GOAT_PREC_BF16, 2e-2),
                                             (goat.GOAT_PREC_FP8, 2e-2)])
def test_directed_gradient_matches_oracle(n, precision, bound):
    # at the directions the method computes: the Sinkhorn Q of -grad f(J) (Alg. 2), and
    # for the 16- and 32-bit forms also a mixture of permutations (the 8-bit form's
    # error there is the structured case of test_gradient_fp8_form_on_permutation_mixtures)
    gp = synthetic.rho_er_digraph_pair(n, 0.1, 0.8, seed=n)
    assert (gp.A != gp.A.T).any()
    A, B = cuda(gp.A), cuda(gp.B)
    J = torch.full((n, n), 1.0 / n, dtype=torch.float32, device="cuda")
    G0 = goat.goat_gradient(A, B, J, precision=goat.GOAT_PREC_FP32, directed=True)
    _, _, Q, _, _ = goat.goat_sinkhorn(G0, 0.03 * float(G0.abs().max()), 1e-3, 500, want_Q=True)
    inputs = [Q.cpu().numpy()]
    if precision != goat.GOAT_PREC_FP8:
        inputs.append(random_ds(n, 1).astype(np.float32))
    for P in inputs:
        G = goat.goat_gradient(A, B, cuda(P), precision=precision, directed=True)
        ref = -oracle.gradient(gp.A.astype(np.float64), gp.B.astype(np.float64), P.astype(np.float64))
        assert rel_err(G.cpu().double().numpy(), ref) <= bound


def test_directed_gradient_weighted_inputs():
    gp = synthetic.rho_er_digraph_pair(257, 0.12, 0.7, seed=3, weighted=True)
    A, B = bf16_exact(gp.A), bf16_exact(gp.B)
    P = random_ds(257, 2).astype(np.float32)
    G = goat.goat_gradient(cuda(A), cuda(B), cuda(P), precision=goat.GOAT_PREC_FP32, directed=True)
    ref = -oracle.gradient(A.astype(np.float64), B.astype(np.float64), P.astype(np.float64))
    assert rel_err(G.cpu().double().numpy(), ref) <= 1e-5


def test_general_form_equals_symmetric_form_on_symmetric_graphs():
    gp = synthetic.rho_er_pair(400, 0.08, 0.8, seed=2)
    P = cuda(random_ds(400, 5).astype(np.float32))
    for precision in (goat.GOAT_PREC_FP32, goat.GOAT_PREC_BF16):
        G2 = goat.goat_gradient(cuda(gp.A), cuda(gp.B), P, precision=precision)
        G4 = goat.goat_gradient(cuda(gp.A), cuda(gp.B), P, precision=precision, directed=True)
        assert rel_err(G4.cpu().double().numpy(), G2.cpu().double().numpy()) <= 1e-6


def test_directed_match_follows_oracle():
    gp = synthetic.rho_er_digraph_pair(150, 0.1, 0.85, seed=7)
    perm, obj, st, P = solve(gp.A, gp.B, 6, 0.0, precision=goat.GOAT_PREC_FP32, directed=1, **TIGHT)
    ro = oracle.goat(gp.A, gp.B, eps_rel=0.03, max_iter=6, tol=0.0, sk_tol=1e-5, sk_max_iter=5000)
    assert st["fw_iters"] == ro["iters"] == 6
    np.testing.assert_allclose(st["alpha"], 1.0 - ro["alphas"], atol=1e-4)
    np.testing.assert_allclose(P, ro["P"], atol=1e-4)
    assert obj == oracle.objective_perm(gp.A, gp.B, perm)
    # the projection is an optimum of the oracle's relaxed P to within the iterates' difference
    best = ro["P"][np.arange(150), ro["perm"]].sum()
    assert ro["P"][np.arange(150), perm].sum() >= best - 150 * 1e-4


@pytest.mark.parametrize("precision", [goat.GOAT_PREC_FP32, goat.GOAT_PREC_BF16, goat.GOAT_PREC_FP8])
def test_directed_match_recovers_isomorphic_pairs(precision):
    gp = synthetic.rho_er_digraph_pair(200, 0.1, 1.0, seed=11)
    perm, obj, st, _ = solve(gp.A, gp.B, 30, 1e-3, precision=precision, directed=1)
    np.testing.assert_array_equal(perm, gp.truth)
    assert obj == gp.A.sum()


def test_symmetric_solve_rejects_directed_input_unless_asked():
    gp = synthetic.rho_er_digraph_pair(64, 0.2, 0.9, seed=1)
    with pytest.raises(goat.GoatError) as e:
        goat.goat_match(cuda(gp.A), cuda(gp.B))
    assert e.value.status == goat.GOAT_ERR_INVALID_ARG


@pytest.mark.parametrize("directed", [0, 1])
def test_qap_minimisation_follows_oracle(directed):
    if directed:
        gp = synthetic.rho_er_digraph_pair(120, 0.15, 0.5, seed=4, weighted=True)
    else:
        gp = synthetic.rho_er_pair(120, 0.15, 0.5, seed=4, weighted=True)
    A, B = bf16_exact(gp.A), bf16_exact(gp.B)
    perm, obj, st, P = solve(A, B, 6, 0.0, precision=goat.GOAT_PREC_FP32, maximize=0, directed=directed, **TIGHT)
    ro = oracle.goat(A.astype(np.float64), B.astype(np.float64), eps_rel=0.03, max_iter=6, tol=0.0, sk_tol=1e-5,
                     sk_max_iter=5000, maximize=False)
    assert st["fw_iters"] == ro["iters"] == 6
    np.testing.assert_allclose(st["alpha"], 1.0 - ro["alphas"], atol=1e-4)
    np.testing.assert_allclose(P, ro["P"], atol=1e-4)
    assert obj == pytest.approx(oracle.objective_perm(A.astype(np.float64), B.astype(np.float64), perm), rel=1e-12)
    # minimising: the result is far below the maximising solve's objective
    _, obj_max, _, _ = solve(A, B, 6, 0.0, precision=goat.GOAT_PREC_FP32, directed=directed, **TIGHT)
    assert obj < obj_max


def test_faq_minimisation_first_step_is_the_reversed_rearrangement():
    # grad f(J) = (2/n) d_A d_B^T: the minimising assignment pairs the largest degree of
    # A with the smallest of B (the rearrangement inequality's other extreme)
    gp = synthetic.rho_er_pair(150, 0.1, 0.8, seed=8, weighted=True)
    A, B = bf16_exact(gp.A).astype(np.float64), bf16_exact(gp.B).astype(np.float64)
    assert np.unique(A.sum(1)).size == 150 and np.unique(B.sum(1)).size == 150
    prm = goat.default_params(precision=goat.GOAT_PREC_FP32, direction=goat.GOAT_DIR_LAP, maximize=0)
    perm, _, st = goat.goat_match(cuda(A.astype(np.float32)), cuda(B.astype(np.float32)), max_iter=1, tol=1e-4,
                                  params=prm)
    grad = oracle.gradient(A, B, np.full((150, 150), 1.0 / 150))
    ref, _ = oracle.lap(grad, maximize=False)
    assert st["alpha"][0] > 0
    np.testing.assert_array_equal(perm, ref)
    ro = oracle.faq(A, B, max_iter=8, tol=1e-4, maximize=False)
    perm8, obj8, st8 = goat.goat_match(cuda(A.astype(np.float32)), cuda(B.astype(np.float32)), max_iter=8, tol=1e-4,
                                       params=prm)
    assert st8["fw_iters"] == ro["iters"]
    np.testing.assert_allclose(st8["alpha"], 1.0 - np.asarray(ro["alphas"]), atol=1e-5)
    assert obj8 == pytest.approx(ro["objective"], rel=1e-9)
