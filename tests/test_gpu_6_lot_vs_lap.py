"""LOT against exact linear assignment on the workload of the paper's Fig. 1
(Sec. 3.3): i.i.d. Uniform(100, 150) costs, n = 250 ... 3000, lambda = 100
(eps = 1/lambda = 0.01 in cost units).  The relaxed objective <Q, M> of LOT's
doubly stochastic Q stays within 0.5 % of the LAP optimum.  The optimum comes
from the GPU's certified projection (checked against the oracle's Hungarian at
n = 250), and LOT's objective is checked against the oracle's own LOT at n = 250."""
import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402

EPS = 0.01      # lambda = 100, the paper's lower bound on lambda
SK_TOL = 1e-3   # max |column sum - 1| of the row-scaled Q


def _costs(n, seed):
    return synthetic.uniform_costs(n, 100, 150, seed, np.float32)


def _lot_objective(M):
    f, g, Q, it, resid = goat.goat_sinkhorn(torch.from_numpy(M).cuda(), EPS, SK_TOL, 5000, want_Q=True)
    assert resid < SK_TOL, (it, resid)
    Qd = Q.double()
    # the last half-step scales the columns (rows then within the tolerance); at
    # this eps the FP32 exponent (f_i + g_j - M_ij) log2(e) / eps alone carries a
    # relative error of about ulp(150) / eps ~ 1e-3 per entry
    assert float((Qd.sum(0) - 1).abs().max()) < 5e-3
    assert float((Qd.sum(1) - 1).abs().max()) < 5e-3
    return float((Qd * torch.from_numpy(M).cuda().double()).sum()), it


@pytest.mark.parametrize("n", [250, 1000, 3000])
def test_lot_objective_within_half_percent_of_lap(n):
    for seed in range(2):
        M = _costs(n, 1000 * n + seed)
        perm, cost_lap, _ = goat.goat_project(torch.from_numpy(M).cuda(), maximize=False)
        p = perm.cpu().numpy()
        assert sorted(p) == list(range(n))
        if n <= 250:
            _, cost_o = oracle.lap(M, maximize=False)
            assert abs(cost_lap - cost_o) <= n * 2.0 ** -52 * 150.0 * 4
        ofv, it = _lot_objective(M)
        rel = (cost_lap - ofv) / cost_lap
        assert abs(rel) < 5e-3, (n, seed, cost_lap, ofv, it)


def test_lot_objective_matches_oracle_lot():
    n = 250
    M = _costs(n, 77)
    ofv, _ = _lot_objective(M)
    Qo, _, _, _, ro = oracle.lot_log(M.astype(np.float64), EPS, SK_TOL, 100000)
    ofv_o = float((Qo * M.astype(np.float64)).sum())
    assert ro < SK_TOL
    assert abs(ofv - ofv_o) <= 1e-4 * ofv_o, (ofv, ofv_o)
