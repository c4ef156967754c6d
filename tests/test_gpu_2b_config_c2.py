"""The precision forms against the FP64 oracle at the n = 2000 plain-vs-precision
workload (correlated ER, p = 0.05, rho = 0.8, B vertex-permuted; eps = 0.03 max|G|;
Sinkhorn to marginal tolerance 1e-3, cold-started as the oracle's is), over the
first four Frank-Wolfe steps of Alg. 3: every form must take the oracle's steps
(the same Sinkhorn iteration counts and step sizes), and the relaxed iterate's
elementwise error against the oracle's is stated per form and bounded for the
two forms that match the oracle's accuracy (FP32-accurate and split-intermediate
BF16).  The method does not recover this pair from the barycenter (the oracle
matches 2 % of the vertices), so the accuracy comparison runs on the Sec. 4.3
workload instead (test_gpu_9_accuracy.py)."""
import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402

N, STEPS = 2000, 4


@pytest.fixture(scope="module")
def c2():
    gp = synthetic.rho_er_pair(N, 0.05, 0.8, seed=2000)
    ro = oracle.goat(gp.A, gp.B, eps_rel=0.03, max_iter=STEPS, tol=0.0, sk_tol=1e-3, sk_max_iter=500)
    return gp, ro


# (form, bound on max |P - P_oracle| / max P_oracle, or None: stated only)
FORMS = [(goat.GOAT_PREC_FP32, 1e-4), (goat.GOAT_PREC_BF16_SPLIT, 1e-2), (goat.GOAT_PREC_BF16_SPLIT8, 1e-2),
         (goat.GOAT_PREC_BF16, None),
         (goat.GOAT_PREC_FP8, None)]


@pytest.mark.timeout(900)
@pytest.mark.parametrize("precision,bound", FORMS)
def test_c2_forms_take_the_oracle_steps(c2, precision, bound):
    gp, ro = c2
    P = torch.empty((N, N), dtype=torch.float32, device="cuda")
    prm = goat.default_params(precision=precision, sk_warm_start=0, sk_tol=1e-3, sk_max_iter=500, relaxed_out=P)
    perm, obj, st = goat.goat_match(torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda(), eps_rel=0.03,
                                    max_iter=STEPS, tol=0.0, params=prm)
    assert st["fw_iters"] == STEPS
    assert st["sk_iters"] == list(ro["sinkhorn_iters"])
    np.testing.assert_allclose(st["alpha"], 1.0 - ro["alphas"], atol=1e-6)
    err = float(np.abs(P.cpu().double().numpy() - ro["P"]).max() / ro["P"].max())
    print(f"C2 precision {precision}: max |P - P_oracle| / max P = {err:.3e}, objective {obj:.0f} "
          f"(oracle {ro['objective']:.0f})")
    assert obj == oracle.objective_perm(gp.A, gp.B, perm)
    if bound is not None:
        assert err <= bound
