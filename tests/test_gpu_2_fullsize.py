"""Parity at the benchmark size (n = 32768, the 3-block SBM pair bench.py times),
in the launch configuration bench.py uses: sampled outputs the FP64 oracle can
compute one by one, and properties that hold at any size."""
import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402

N = 32768
ROWS = [0, 12345, N - 1]


@pytest.fixture(scope="module")
def pair():
    gp = synthetic.large_sbm_pair(N, seed=3000)
    return gp, torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda()


def _half_perm_start(n, seed):
    # (J + Pi) / 2: doubly stochastic, every entry in {1/(2n), 1/(2n) + 1/2}
    P = torch.full((n, n), 0.5 / n, dtype=torch.float32, device="cuda")
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(n)).cuda()
    P[torch.arange(n, device="cuda"), perm] += 0.5
    return P


@pytest.mark.timeout(900)
def test_fullsize_gradient_rows_match_oracle(pair):
    gp, A, B = pair
    P = _half_perm_start(N, 1)
    ref = -oracle.gradient_rows(gp.A, gp.B, P.cpu().numpy(), ROWS)
    for prec, tol in ((goat.GOAT_PREC_FP8, 2e-2), (goat.GOAT_PREC_BF16, 5e-3), (goat.GOAT_PREC_FP32, 1e-5)):
        G = goat.goat_gradient(A, B, P, precision=prec)
        got = G[ROWS].cpu().double().numpy()
        del G
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= tol, (prec, err)


@pytest.mark.timeout(900)
def test_fullsize_sinkhorn_marginals(pair):
    gp, A, B = pair
    J = torch.full((N, N), 1.0 / N, dtype=torch.float32, device="cuda")
    G = goat.goat_gradient(A, B, J, precision=goat.GOAT_PREC_FP32)
    del J
    eps = 0.03 * float(G.abs().max())
    f, g, _, it, resid = goat.goat_sinkhorn(G, eps, 1e-3, 500)
    assert resid < 1e-3 and it < 500
    fh, gh = f.cpu().numpy(), g.cpu().numpy()
    cols = [1, 20000, N - 2]
    # the last column scaling makes these columns' sums 1 (FP64 oracle on the GPU's duals)
    csum = oracle.lot_colsums(G[:, cols].cpu().numpy(), fh, gh[cols], eps)
    np.testing.assert_allclose(csum, 1.0, atol=1e-4)
    # the rows are within the stop tolerance of 1
    rows = G[ROWS].cpu().numpy()
    f_ref = oracle.lot_rows(rows, gh, eps)  # f that would make these rows sum to 1 exactly
    rsum = np.exp((fh[ROWS] - f_ref) / eps)  # = sum_j Q_ij with the GPU's f
    np.testing.assert_allclose(rsum, 1.0, atol=5e-3)


@pytest.mark.timeout(900)
def test_fullsize_match_objective_exact_and_projection_certified(pair):
    gp, A, B = pair
    prm = goat.default_params(precision=goat.GOAT_PREC_FP8, sk_warm_start=1, sk_tol=1e-3, sk_max_iter=500)
    perm, obj, st = goat.goat_match(A, B, eps_rel=0.03, max_iter=30, tol=1e-4, params=prm)
    assert sorted(perm.tolist()) == list(range(N))
    assert obj == oracle.objective_perm(gp.A, gp.B, perm)
    assert st["lap_gap"] == 0.0  # the projection's LP duality certificate
