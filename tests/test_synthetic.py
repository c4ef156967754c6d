"""The seeded rho-correlated SBM / ER generator: structure and moments."""
import numpy as np

from paper_2111_05366_gb300 import synthetic


def test_pair_structure_and_truth():
    gp = synthetic.rho_er_pair(300, 0.1, 0.9, seed=5)
    A, B, t = gp.A, gp.B, gp.truth
    assert A.dtype == np.uint8 and A.shape == (300, 300)
    assert (A == A.T).all() and (B == B.T).all()
    assert A.diagonal().sum() == 0 and B.diagonal().sum() == 0
    assert sorted(t) == list(range(300))
    # B relabelled back through the truth is the correlated copy of A
    Bp = B[np.ix_(t, t)]
    agree = (A & Bp).sum() / max(A.sum(), 1)
    assert agree > 0.85
    # rho = 1: exact isomorphism through the truth
    g1 = synthetic.rho_er_pair(200, 0.1, 1.0, seed=3)
    assert (g1.A == g1.B[np.ix_(g1.truth, g1.truth)]).all()


def test_edge_density_and_correlation_moments():
    n, p, rho = 1200, 0.05, 0.7
    gp = synthetic.rho_er_pair(n, p, rho, seed=1)
    iu = np.triu_indices(n, 1)
    a = gp.A[iu].astype(float)
    b = gp.B[np.ix_(gp.truth, gp.truth)][iu].astype(float)
    m = a.size
    for x in (a, b):
        se = np.sqrt(p * (1 - p) / m)
        assert abs(x.mean() - p) < 4 * se
    r = np.corrcoef(a, b)[0, 1]
    assert abs(r - rho) < 4 * np.sqrt((1 - rho ** 2) ** 2 / m) + 0.01


def test_sbm_block_probabilities():
    Pb = np.array([[0.2, 0.01, 0.01], [0.01, 0.1, 0.01], [0.01, 0.01, 0.2]])
    gp = synthetic.rho_sbm_pair([200, 200, 200], Pb, 0.9, seed=2)
    A = gp.A.astype(float)
    for r in range(3):
        for c in range(3):
            blk = A[r * 200:(r + 1) * 200, c * 200:(c + 1) * 200]
            cnt = 200 * 199 if r == c else 200 * 200
            est = blk.sum() / cnt
            se = np.sqrt(Pb[r, c] * (1 - Pb[r, c]) / (cnt / (2 if r == c else 1)))
            assert abs(est - Pb[r, c]) < 5 * se


def test_weighted_pairs_share_weights_on_common_edges():
    gp = synthetic.rho_er_pair(200, 0.1, 0.8, seed=9, weighted=True)
    A, B = gp.A, gp.B
    assert A.dtype == np.float32 and (A == A.T).all()
    Bp = B[np.ix_(gp.truth, gp.truth)]
    common = (A > 0) & (Bp > 0)
    assert common.sum() > 0
    np.testing.assert_array_equal(A[common], Bp[common])


def test_large_sbm_sizes_and_determinism():
    sizes = synthetic.sbm3_block_sizes(32768)
    assert sizes == [13107, 11468, 8193] and sum(sizes) == 32768
    g1 = synthetic.rho_er_pair(100, 0.1, 0.5, seed=4)
    g2 = synthetic.rho_er_pair(100, 0.1, 0.5, seed=4)
    assert (g1.A == g2.A).all() and (g1.B == g2.B).all() and (g1.truth == g2.truth).all()


def test_directed_pair_density_correlation_and_truth():
    n, p, rho = 900, 0.06, 0.75
    gp = synthetic.rho_er_digraph_pair(n, p, rho, seed=3)
    A, B, t = gp.A, gp.B, gp.truth
    assert A.dtype == np.uint8 and (A != A.T).any()
    assert A.diagonal().sum() == 0 and B.diagonal().sum() == 0
    assert sorted(t) == list(range(n))
    off = ~np.eye(n, dtype=bool)
    a = A[off].astype(float)
    b = B[np.ix_(t, t)][off].astype(float)
    m = a.size
    for x in (a, b):
        assert abs(x.mean() - p) < 4 * np.sqrt(p * (1 - p) / m)
    assert abs(np.corrcoef(a, b)[0, 1] - rho) < 4 * np.sqrt((1 - rho ** 2) ** 2 / m) + 0.01
    g1 = synthetic.rho_er_digraph_pair(150, 0.1, 1.0, seed=4, weighted=True)
    assert g1.A.dtype == np.float32
    np.testing.assert_array_equal(g1.A, g1.B[np.ix_(g1.truth, g1.truth)])
