"""The learned Sinkhorn warm start: feature, inference and training kernels vs the
FP64 oracle, and what the trained network gains over a cold start."""
import numpy as np
import pytest

import oracle
from paper_2111_05366_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402
from paper_2111_05366_gb300 import warmstart  # noqa: E402


def _bf16_params(seed):
    rng = np.random.default_rng(seed)
    w = (rng.standard_normal(goat.GOAT_MLP_PARAMS) * 0.4).astype(np.float32)
    wb = torch.from_numpy(w).cuda().to(torch.bfloat16)
    return wb, wb.float().cpu().double().numpy()  # the exact BF16 values, for the oracle


# n = 211: scalar column loads, a ragged last group of columns; n = 1028: float4 loads,
# two 1024-column tiles (the second holds one group), several row chunks
@pytest.mark.parametrize("n,weighted", [(211, False), (211, True), (1028, True)])
def test_features_match_oracle(n, weighted):
    gp = synthetic.rho_er_pair(n, 0.1, 0.8, seed=9, weighted=weighted)
    A, B = torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda()
    rng = np.random.default_rng(1)
    P = np.zeros((n, n), np.float32)
    for w in rng.random(4) + 0.1:
        P[np.arange(n), rng.permutation(n)] += w
    P /= P.sum(1, keepdims=True)
    G = goat.goat_gradient(A, B, torch.from_numpy(P).cuda(), precision=goat.GOAT_PREC_FP32)
    eps = 0.03 * float(G.abs().max())
    F = goat.goat_dual_features(G, A, B, eps).cpu().double().numpy()
    Fo = oracle.dual_features(G.cpu().double().numpy(), gp.A.astype(float), gp.B.astype(float), eps)
    np.testing.assert_allclose(F, Fo, rtol=1e-4, atol=1e-4)


def test_forward_matches_oracle():
    wb, wd = _bf16_params(2)
    x = torch.from_numpy(np.random.default_rng(3).standard_normal((1000, 8)).astype(np.float32)).cuda()
    y = goat.goat_mlp_forward(wb, x).cpu().double().numpy()
    _, _, yo = oracle.mlp_loss_grad(wd, x.cpu().double().numpy(), np.zeros(1000))
    np.testing.assert_allclose(y, yo, rtol=1e-4, atol=1e-4)


def test_gradient_matches_oracle():
    wb, wd = _bf16_params(4)
    rng = np.random.default_rng(5)
    N = 3000
    x = torch.from_numpy(rng.standard_normal((N, 8)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).cuda()
    master = wb.float().clone()
    adam = torch.zeros(2 * goat.GOAT_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss, grad = goat.goat_mlp_train_step(master, adam, wb, x, t, lr=0.0, step=1)
    Lo, go, _ = oracle.mlp_loss_grad(wd, x.cpu().double().numpy(), t.cpu().double().numpy())
    assert float(loss.item()) == pytest.approx(Lo, rel=1e-4)
    g = grad.cpu().double().numpy()
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-4


def test_first_adam_step_closed_form():
    # after one step from zero moments, the bias-corrected Adam update is lr * g / (|g| + 1e-8)
    wb, wd = _bf16_params(6)
    rng = np.random.default_rng(7)
    x = torch.from_numpy(rng.standard_normal((500, 8)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal(500).astype(np.float32)).cuda()
    master = wb.float().clone()
    before = master.cpu().double().numpy()
    adam = torch.zeros(2 * goat.GOAT_MLP_PARAMS, dtype=torch.float32, device="cuda")
    lr = 1e-3
    _, grad = goat.goat_mlp_train_step(master, adam, wb, x, t, lr=lr, step=1)
    g = grad.cpu().double().numpy()
    np.testing.assert_allclose(master.cpu().double().numpy() - before, -lr * g / (np.abs(g) + 1e-8),
                               rtol=1e-3, atol=1e-9)
    np.testing.assert_array_equal(wb.float().cpu().numpy(), master.to(torch.bfloat16).float().cpu().numpy())


def test_trained_network_beats_cold_start_on_held_out_problems():
    X, T = warmstart.collect(warmstart.default_training_pairs(14, seed=11, nmin=300, nmax=900), fw_steps=2)
    master, adam, wb, losses = warmstart.train(X, T, steps=800, batch=4096, lr=3e-3, seed=0)
    base = float(((T - T.mean()) ** 2).mean())
    assert losses[-1] < 0.25 * base, (losses[-1], base)
    cold, warm = [], []
    for gp in warmstart.default_training_pairs(3, seed=99, nmin=500, nmax=900):
        A, B = torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda()
        J = torch.full((gp.n, gp.n), 1.0 / gp.n, dtype=torch.float32, device="cuda")
        G = goat.goat_gradient(A, B, J)
        eps = 0.03 * float(G.abs().max())
        _, _, _, it_c, r_c = goat.goat_sinkhorn(G, eps, 1e-4, 5000)
        g0 = goat.goat_mlp_warm_start(G, A, B, eps, wb)
        _, _, _, it_w, r_w = goat.goat_sinkhorn(G, eps, 1e-4, 5000, g_init=g0)
        assert r_c < 1e-4 and r_w < 1e-4
        cold.append(it_c)
        warm.append(it_w)
    assert np.mean(warm) < np.mean(cold), (cold, warm)
    # goat_match takes the network as its first warm start and still returns an exact objective
    gp = synthetic.rho_er_pair(300, 0.1, 0.9, seed=3)
    prm = goat.default_params(mlp_weights=wb)
    perm, obj, st = goat.goat_match(torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda(), params=prm)
    assert obj == oracle.objective_perm(gp.A, gp.B, perm)


def test_entropic_eps_and_dual_targets_follow_their_definitions():
    # eps = eps_rel max|G| (float32 product, as the solve computes it), 1 for G = 0;
    # targets = duals over eps with each side's mean removed
    rng = np.random.default_rng(8)
    n = 333
    G = rng.standard_normal((n, n)).astype(np.float32) * 7.0
    e = goat.goat_entropic_eps(torch.from_numpy(G).cuda(), 0.03)
    assert e == float(np.float32(0.03) * np.float32(np.abs(G).max()))
    assert goat.goat_entropic_eps(torch.zeros((n, n), dtype=torch.float32, device="cuda"), 0.03) == 1.0
    f = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32) + 5.0
    t = goat.goat_dual_targets(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), 0.25).cpu().double().numpy()
    tf, tg = f.astype(np.float64) / 0.25, g.astype(np.float64) / 0.25
    np.testing.assert_allclose(t, np.concatenate([tf - tf.mean(), tg - tg.mean()]), rtol=0, atol=1e-5)
