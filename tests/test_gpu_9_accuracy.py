"""Matching accuracy of the precision forms against the FP64 oracle where the method
works: the paper's Sec. 4.3 rho-SBM at n = 1500 (3 equal blocks, block matrix
[[0.2, 0.01, 0.01], [0.01, 0.1, 0.01], [0.01, 0.01, 0.2]]), rho = 0.9 and 0.95,
20 seeds each, with the parameters of the timed solve.  The oracle's accuracies are
stored in tests/golden/sbm1500_oracle.txt by the committed script beside it.

The bar (the benchmark spec's): mean accuracy within 1 percentage point of the oracle's.
The FP32-accurate form and the split-intermediate BF16 form (Q in BF16, Q B in two
BF16 terms) meet it, cold- or warm-started.  The plain BF16 form (Q B rounded to
BF16, which the second product sums over only the degree) and the 8-bit form (Q and
Q B in E4M3) do not: their gradient errors, amplified by 1/eps = 1/(0.03 max|G|) in
the entropic step, change the matches (bench.py reports every form's accuracy)."""
import os

import numpy as np
import pytest

from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402

PB = [[0.2, 0.01, 0.01], [0.01, 0.1, 0.01], [0.01, 0.01, 0.2]]
SEEDS = range(1, 21)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sbm1500_oracle.txt")


def oracle_accuracy():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        rho, seed, acc, _, _ = line.split()
        out[(float(rho), int(seed))] = float(acc)
    return out


@pytest.fixture(scope="module")
def pairs():
    return {rho: [synthetic.rho_sbm_pair([500, 500, 500], PB, rho, seed=s) for s in SEEDS] for rho in (0.9, 0.95)}


def mean_accuracy(pairs, precision, warm):
    prm = goat.default_params(precision=precision, sk_warm_start=warm, sk_tol=1e-3, sk_max_iter=500)
    accs = []
    for gp in pairs:
        perm, obj, _ = goat.goat_match(torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda(), eps_rel=0.03,
                                       max_iter=30, tol=1e-4, params=prm)
        accs.append((perm == gp.truth).mean())
    return float(np.mean(accs))


@pytest.mark.parametrize("precision", [goat.GOAT_PREC_FP32, goat.GOAT_PREC_BF16_SPLIT, goat.GOAT_PREC_BF16_SPLIT8])
@pytest.mark.parametrize("warm", [0, 1])
def test_accurate_forms_within_one_point_of_oracle(pairs, precision, warm):
    ref = oracle_accuracy()
    for rho, ps in pairs.items():
        mine = mean_accuracy(ps, precision, warm)
        theirs = float(np.mean([ref[(rho, s)] for s in SEEDS]))
        assert abs(mine - theirs) <= 0.01, (rho, mine, theirs)
