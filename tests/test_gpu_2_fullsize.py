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
ROWS = [0, 4321, 12345, 20000, 27777, N - 1]


@pytest.fixture(scope="module")
def pair():
    gp = synthetic.large_sbm_pair(N, seed=3000)
    return gp, torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda()


@pytest.fixture(scope="module")
def directions(pair):
    """The operands the timed solve feeds the products: the LOT direction Q at the
    barycenter (the first step's Sinkhorn solution), and the relaxed iterate P after
    three Frank-Wolfe steps of the 8-bit form (host float32 copies)."""
    gp, A, B = pair
    J = torch.full((N, N), 1.0 / N, dtype=torch.float32, device="cuda")
    G = goat.goat_gradient(A, B, J, precision=goat.GOAT_PREC_FP32)
    del J
    _, _, Q, _, _ = goat.goat_sinkhorn(G, 0.03 * float(G.abs().max()), 1e-3, 500, want_Q=True)
    del G
    Qh = Q.cpu().numpy()
    P3 = Q  # reused as the relaxed-iterate output
    prm = goat.default_params(precision=goat.GOAT_PREC_FP8, sk_warm_start=1, sk_tol=1e-3, sk_max_iter=500,
                              relaxed_out=P3)
    goat.goat_match(A, B, eps_rel=0.03, max_iter=3, tol=0.0, params=prm)
    P3h = P3.cpu().numpy()
    del P3, Q
    torch.cuda.empty_cache()
    return {"Q": Qh, "P3": P3h}


@pytest.mark.timeout(1200)
@pytest.mark.parametrize("which", ["Q", "P3"])
def test_fullsize_gradient_rows_match_oracle(pair, directions, which):
    gp, A, B = pair
    X = directions[which]
    # doubly stochastic (within the Sinkhorn tolerance), with many distinct values per
    # row (Q at the barycenter takes one value per distinct degree)
    np.testing.assert_allclose(X[ROWS].sum(1), 1.0, atol=2e-3)
    assert np.unique(X[ROWS[0]]).size > 100
    ref = -oracle.gradient_rows(gp.A, gp.B, X, ROWS)
    Xd = torch.from_numpy(X).cuda()
    rows = {}
    for prec, tol in ((goat.GOAT_PREC_FP8, 2e-2), (goat.GOAT_PREC_BF16, 5e-3), (goat.GOAT_PREC_FP32, 1e-5),
                      (goat.GOAT_PREC_BF16_SPLIT, 5e-3), (goat.GOAT_PREC_BF16_SPLIT8, 5e-3)):
        G = goat.goat_gradient(A, B, Xd, precision=prec)
        got = G[ROWS].cpu().double().numpy()
        del G
        rows[prec] = got
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"n={N} {which} precision {prec}: gradient rows rel. error {err:.3e}")
        assert err <= tol, (prec, err)
    # the 8-bit lo term of the timed form adds about 2^-12 to the split form's error
    a, b = rows[goat.GOAT_PREC_BF16_SPLIT8], rows[goat.GOAT_PREC_BF16_SPLIT]
    assert np.linalg.norm(a - b) / np.linalg.norm(ref) <= 4e-4


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
