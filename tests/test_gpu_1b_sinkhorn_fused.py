"""The single-read Sinkhorn iteration (Alg. 2; used from n = 20480 up to n = 32768,
n a multiple of 16, for every iteration after the first): a cluster of four CTAs
streams each row of G once, forms the row scaling f_i = -eps LSE_j((g_j - G_ij)/eps)
and adds the row-scaled entries to its column sums two rows later.  Against the
oracle's log-domain LOT run for the same number of iterations from the same warm
start, at the smallest size it takes, at a size whose quarter rows (6148 columns)
leave the threads' last column group ragged, and at the largest.  The costs are the
paper's Fig. 1 law, i.i.d. Uniform(100, 150)."""
import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402


@pytest.mark.timeout(900)
@pytest.mark.parametrize("n,iters", [(20480, 3), (24592, 3), (32768, 2)])
def test_fused_sinkhorn_matches_oracle(n, iters):
    M = synthetic.uniform_costs(n, 100.0, 150.0, 7 * n, np.float32)
    eps = 0.5  # far from converged after `iters` iterations, so the residuals compare
    g0 = (np.random.default_rng(n).standard_normal(n) * eps).astype(np.float32)
    f, g, Q, it, resid = goat.goat_sinkhorn(torch.from_numpy(M).cuda(), eps, 0.0, iters,
                                            g_init=torch.from_numpy(g0).cuda(), want_Q=True)
    Qo, fo, go, ito, ro = oracle.lot_log(M.astype(np.float64), eps, 0.0, iters, g_init=g0.astype(np.float64))
    assert it == ito == iters
    np.testing.assert_allclose(f.cpu().double().numpy(), fo, atol=2e-3 * eps, rtol=0)
    np.testing.assert_allclose(g.cpu().double().numpy(), go, atol=2e-3 * eps, rtol=0)
    Qg = Q.cpu().double().numpy()
    del Q
    np.testing.assert_allclose(Qg, Qo, rtol=1e-3, atol=1e-9)
    # FP32 column sums carry an absolute error near the residual floor of 1.5e-5 that
    # both the two-pass and the fused iteration reach on these costs at eps = 0.5
    # (exponents of magnitude ~100 in base 2); three iterations leave ~1e-3 above it
    assert resid == pytest.approx(ro, rel=1e-2, abs=3e-5)
    # the GPU's Q: columns sum to 1 after the column scaling
    np.testing.assert_allclose(Qg.sum(0), 1.0, atol=1e-4)


@pytest.mark.timeout(900)
def test_fused_sinkhorn_converges_at_the_bench_size():
    # n = 32768: converges to the tolerance, and the oracle recomputes the column sums
    # of sampled columns from the GPU's duals (row sums within the tolerance)
    n = 32768
    M = torch.from_numpy(synthetic.uniform_costs(n, 100.0, 150.0, 11, np.float32)).cuda()
    eps = 1.5
    f, g, _, it, resid = goat.goat_sinkhorn(M, eps, 1e-4, 500)
    assert resid < 1e-4 and it < 500
    cols = [0, 777, 8191, 8192, 16384, n - 1]
    fh, gh = f.cpu().numpy(), g.cpu().numpy()
    csum = oracle.lot_colsums(M[:, cols].cpu().numpy(), fh, gh[cols], eps)
    np.testing.assert_allclose(csum, 1.0, atol=2e-4)
    rows = [0, 12345, n - 1]
    f_ref = oracle.lot_rows(M[rows].cpu().numpy(), gh, eps)
    np.testing.assert_allclose(np.exp((fh[rows] - f_ref) / eps), 1.0, atol=5e-4)
