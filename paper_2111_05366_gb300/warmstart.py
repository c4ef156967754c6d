"""Training the learned Sinkhorn warm start on duals the method itself produces.

The data: for graph pairs drawn from `synthetic`, run a few Frank-Wolfe steps of
GOAT through the library (goat_gradient, goat_sinkhorn at a tight tolerance,
goat_line_search, goat_fw_update); at every step record the node features
(goat_dual_features) and the converged duals over eps, each side's mean removed
(the duals are defined up to f + c, g - c).  Training runs the library's own
kernels (goat_mlp_train_step: forward, backward, Adam); this module only moves
tensors between those calls.
"""
from __future__ import annotations

import numpy as np

from . import (GOAT_MLP_PARAMS, goat_dual_features, goat_dual_targets, goat_entropic_eps, goat_fw_update,
               goat_gradient, goat_line_search, goat_mlp_train_step, goat_sinkhorn)
from . import synthetic


def _torch():
    import torch
    return torch


def collect(pairs, fw_steps: int = 3, eps_rel: float = 0.03, sk_tol: float = 1e-5, sk_max_iter: int = 3000):
    """Features and dual targets from converged LOT solves along short GOAT runs.

    pairs: iterable of synthetic.GraphPair.  Returns (X [N x 8], T [N]) device tensors."""
    torch = _torch()
    xs, ts = [], []
    for gp in pairs:
        A = torch.from_numpy(gp.A).cuda()
        B = torch.from_numpy(gp.B).cuda()
        n = gp.n
        P = torch.full((n, n), 1.0 / n, dtype=torch.float32, device="cuda")
        G = goat_gradient(A, B, P)
        for _ in range(fw_steps):
            eps = goat_entropic_eps(G, eps_rel)  # the rule goat_match applies
            f, g, Q, it, res = goat_sinkhorn(G, eps, sk_tol, sk_max_iter, want_Q=True)
            xs.append(goat_dual_features(G, A, B, eps))
            ts.append(goat_dual_targets(f, g, eps))
            GQ = goat_gradient(A, B, Q)
            alpha, _, _ = goat_line_search(G, GQ, P, Q)
            goat_fw_update(P, G, Q, GQ, alpha)
    return torch.cat(xs), torch.cat(ts)


def default_training_pairs(count: int, seed: int, nmin: int = 500, nmax: int = 2000, weighted_frac: float = 0.5):
    """Correlated ER / 3-block SBM pairs with n in [nmin, nmax], some with lognormal weights."""
    rng = np.random.default_rng(seed)
    for k in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        rho = float(rng.uniform(0.6, 1.0))
        weighted = bool(rng.random() < weighted_frac)
        if rng.random() < 0.5:
            p = float(rng.uniform(0.02, 0.1))
            yield synthetic.rho_er_pair(n, p, rho, seed=seed * 1000 + k, weighted=weighted)
        else:
            sizes = synthetic.sbm3_block_sizes(n)
            Pb = np.full((3, 3), float(rng.uniform(0.002, 0.01)))
            np.fill_diagonal(Pb, float(rng.uniform(0.02, 0.08)))
            yield synthetic.rho_sbm_pair(sizes, Pb, rho, seed=seed * 1000 + k, weighted=weighted)


def init_weights(seed: int = 0):
    """(master FP32, Adam state, BF16 weights) with small seeded random initial values."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    w = np.zeros(GOAT_MLP_PARAMS, dtype=np.float32)
    w[:512] = rng.standard_normal(512) * (1.0 / np.sqrt(8.0))
    w[576:640] = rng.standard_normal(64) * (1.0 / np.sqrt(64.0))
    master = torch.from_numpy(w).cuda()
    adam = torch.zeros(2 * GOAT_MLP_PARAMS, dtype=torch.float32, device="cuda")
    return master, adam, master.to(torch.bfloat16)


def train(X, T, steps: int = 2000, batch: int = 8192, lr: float = 3e-3, seed: int = 0, weights=None):
    """Adam on the mean squared error with the library's kernels.  Returns
    (master, adam_state, bf16 weights, list of losses)."""
    torch = _torch()
    master, adam, wb = weights if weights is not None else init_weights(seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    grad = torch.empty(GOAT_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    losses = []
    N = X.shape[0]
    for step in range(1, steps + 1):
        idx = torch.randint(0, N, (min(batch, N),), device="cuda", generator=gen)
        xb = X[idx].contiguous()
        tb = T[idx].contiguous()
        goat_mlp_train_step(master, adam, wb, xb, tb, lr, step, grad=grad, loss=loss)
        if step % 100 == 0 or step == steps:
            losses.append(float(loss.item()))
    return master, adam, wb, losses
