"""The split form with an 8-bit low term (GOAT_PREC_BF16_SPLIT8): the second
product runs the hi term of C1 = B Q^T in BF16 and its lo term in E4M3 (both under
one power-of-two scale) in one accumulator (Alg. 3 step 1).  Against the FP64
oracle's gradient on the directions the method computes (the Sinkhorn Q at the
barycenter), next to the all-BF16 split form: the 8-bit lo term may only add what
its 3 mantissa bits lose, about 2^-12 of the gradient, on 0/1 and weighted graphs,
undirected (padded 8-bit rows) and directed ([A | A^T] layout)."""
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


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# n = 300: K blocks of the hi term (320) and the lo term (384, zero padded) differ;
# n = 1000: several 128 x 256 tiles with a ragged edge
@pytest.mark.parametrize("n,weighted,directed", [(300, False, False), (700, True, False), (1000, False, False),
                                                 (300, False, True), (260, True, True)])
def test_split8_gradient_follows_the_split_form(n, weighted, directed):
    make = synthetic.rho_er_digraph_pair if directed else synthetic.rho_er_pair
    gp = make(n, 0.1, 0.8, seed=n + 7, weighted=weighted)
    A, B = cuda(gp.A), cuda(gp.B)
    J = torch.full((n, n), 1.0 / n, dtype=torch.float32, device="cuda")
    G = goat.goat_gradient(A, B, J, precision=goat.GOAT_PREC_FP32, directed=int(directed))
    _, _, Q, _, _ = goat.goat_sinkhorn(G, 0.03 * float(G.abs().max()), 1e-3, 500, want_Q=True)
    ref = -oracle.gradient(gp.A, gp.B, Q.cpu().double().numpy())
    g_split = goat.goat_gradient(A, B, Q, precision=goat.GOAT_PREC_BF16_SPLIT, directed=int(directed))
    g_8 = goat.goat_gradient(A, B, Q, precision=goat.GOAT_PREC_BF16_SPLIT8, directed=int(directed))
    e_split = rel_fro(g_split.cpu().double().numpy(), ref)
    e_8 = rel_fro(g_8.cpu().double().numpy(), ref)
    d = rel_fro(g_8.cpu().double().numpy(), g_split.cpu().double().numpy())
    print(f"n={n} weighted={weighted} directed={directed}: split {e_split:.2e}, split8 {e_8:.2e}, apart {d:.2e}")
    assert e_split <= 5e-3 and e_8 <= 5e-3
    # the lo term is at most 2^-8 of hi; E4M3 keeps it to 2^-4 (plus A's E4M3
    # rounding for weighted graphs): the two forms differ by about 2^-12
    assert d <= 4e-4, d


def test_split8_match_objective_is_exact():
    gp = synthetic.rho_er_pair(400, 0.08, 0.9, seed=4)
    prm = goat.default_params(precision=goat.GOAT_PREC_BF16_SPLIT8)
    perm, obj, st = goat.goat_match(cuda(gp.A), cuda(gp.B), params=prm)
    assert sorted(perm.tolist()) == list(range(400))
    assert obj == oracle.objective_perm(gp.A, gp.B, perm)


@pytest.mark.parametrize("directed,seeds", [(1, 0), (0, 30), (1, 20)])
def test_split8_seeded_and_directed_solves_are_exact(directed, seeds):
    # the whole solve in the split8 form on the other operand layouts: [A | A^T] rows
    # (directed) and the unseeded block (seeds); the permutation keeps the seeds and
    # its objective is the oracle's exact value
    n = 260
    make = synthetic.rho_er_digraph_pair if directed else synthetic.rho_er_pair
    gp = make(n, 0.08, 0.9, seed=31 + seeds)
    prm = goat.default_params(precision=goat.GOAT_PREC_BF16_SPLIT8, directed=directed, seeds=seeds,
                              sk_warm_start=1)
    perm, obj, st = goat.goat_match(cuda(gp.A), cuda(gp.B), params=prm)
    assert sorted(perm.tolist()) == list(range(n))
    np.testing.assert_array_equal(perm[:seeds], np.arange(seeds))
    assert obj == oracle.objective_perm(gp.A, gp.B, perm)
    assert st["fw_iters"] >= 1
