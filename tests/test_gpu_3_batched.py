"""Batched GOAT (many pairs of uneven n, random restarts, CUDA-graph FW loop) vs the oracle."""
import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402


def _pairs(specs, seed0):
    return [synthetic.rho_er_pair(n, p, rho, seed=seed0 + k) for k, (n, p, rho) in enumerate(specs)]


def test_batched_random_starts_and_their_projection_match_oracle():
    # max_iter = 0: every problem's relaxed P is its starting point (J, or the random
    # start (J + K)/2 of Sec. 3.4), and the returned permutation is the projection of
    # the best restart's start: an optimum of the oracle's Hungarian on that matrix
    specs = [(40, 0.2, 0.9), (77, 0.1, 0.8), (130, 0.1, 0.7)]
    gps = _pairs(specs, 100)
    seed, R = 12345, 3
    prm = goat.default_params(sk_tol=1e-3, sk_max_iter=500)
    perms, obj, best, its, rel = goat.goat_match_batched([g.A for g in gps], [g.B for g in gps], restarts=R,
                                                         seed=seed, max_iter=0, params=prm, want_relaxed=True)
    for p, gp in enumerate(gps):
        n = gp.n
        for r in range(R):
            q = p * R + r
            P0 = np.full((n, n), 1.0 / n) if r == 0 else oracle.random_start(n, seed, q)
            np.testing.assert_allclose(rel[q], P0, rtol=1e-5, atol=1e-7)
        q = p * R + int(best[p])
        assert sorted(perms[p]) == list(range(n))
        Pg = rel[q]
        _, opt = oracle.lap(Pg, maximize=True)
        got = oracle.assignment_cost_f32(Pg, perms[p])
        assert abs(got - opt) <= n * 2.0 ** -52 * float(np.abs(Pg).max()) * 4
        assert obj[p] == oracle.objective_perm(gp.A, gp.B, perms[p])


def test_batched_matches_oracle_best_of_restarts():
    specs = [(60, 0.15, 0.9), (96, 0.1, 0.85), (128, 0.1, 1.0), (150, 0.08, 0.8), (203, 0.06, 0.9),
             (77, 0.2, 0.7), (255, 0.05, 0.95), (111, 0.12, 0.75)]
    gps = _pairs(specs, 500)
    seed, R = 7, 2
    prm = goat.default_params(sk_tol=1e-3, sk_max_iter=500)
    perms, obj, best, its = goat.goat_match_batched([g.A for g in gps], [g.B for g in gps], restarts=R, seed=seed,
                                                    max_iter=30, tol=1e-3, params=prm)
    acc, acc_o = [], []
    for p, gp in enumerate(gps):
        n = gp.n
        assert obj[p] == oracle.objective_perm(gp.A, gp.B, perms[p])
        runs = []
        for r in range(R):
            P0 = None if r == 0 else oracle.random_start(n, seed, p * R + r)
            runs.append(oracle.goat(gp.A, gp.B, P0=P0, eps_rel=0.03, max_iter=30, tol=1e-3, sk_tol=1e-3,
                                    sk_max_iter=500))
        ref = max(runs, key=lambda x: x["objective"])
        acc.append((perms[p] == gp.truth).mean())
        acc_o.append((ref["perm"] == gp.truth).mean())
    assert abs(np.mean(acc) - np.mean(acc_o)) <= 0.02, (acc, acc_o)


@pytest.mark.parametrize("steps", [1, 2])
def test_batched_iterates_follow_the_oracle_per_problem(steps):
    # every problem's relaxed P after `steps` Frank-Wolfe iterations (tol 0: no early
    # stop) against the oracle's run from the same start.  From the barycenter the
    # first gradient is exact up to a uniform scale (BF16 rounding of 1/n), which eps
    # absorbs, so the first direction matches; the step size uses grad f(Q) from a
    # BF16 product (about 1e-3 relative), which moves P by about that much.  Later
    # gradients carry the BF16 rounding of Q and Q B, which the entropic step
    # amplifies by about 1/0.03
    specs = [(64, 0.15, 0.9), (97, 0.1, 0.8), (150, 0.08, 0.85)]
    gps = _pairs(specs, 900)
    seed, R = 99, 2
    prm = goat.default_params(sk_tol=1e-4, sk_max_iter=2000)
    perms, obj, best, its, rel = goat.goat_match_batched([g.A for g in gps], [g.B for g in gps], restarts=R,
                                                         seed=seed, max_iter=steps, tol=0.0, params=prm,
                                                         want_relaxed=True)
    for p, gp in enumerate(gps):
        n = gp.n
        assert its[p] == steps
        for r in range(R):
            q = p * R + r
            P0 = None if r == 0 else oracle.random_start(n, seed, q)
            ro = oracle.goat(gp.A, gp.B, P0=P0, eps_rel=0.03, max_iter=steps, tol=0.0, sk_tol=1e-4, sk_max_iter=2000)
            err = float(np.abs(rel[q] - ro["P"]).max() / ro["P"].max())
            rows = np.abs(rel[q].sum(1) - 1.0).max()
            print(f"pair {p} (n={n}) restart {r}, {steps} step(s): max |P - P_oracle| / max P = {err:.2e}")
            assert rows <= 2e-3  # still doubly stochastic (rows exact up to the Sinkhorn tolerance)
            bound = 5e-3 if (steps == 1 and r == 0) else 5e-2
            assert err <= bound, (p, r, steps, err)
        assert obj[p] == oracle.objective_perm(gp.A, gp.B, perms[p])


def test_batched_rejects_oversized_problems():
    A = np.zeros((2049, 2049), np.uint8)
    with pytest.raises(goat.GoatError) as e:
        goat.goat_match_batched([A], [A], restarts=1)
    assert e.value.status == goat.GOAT_ERR_INVALID_ARG
