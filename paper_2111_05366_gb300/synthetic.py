"""Seeded synthetic inputs for graph matching (numpy only).

This module generates inputs and nothing else: it holds none of the matching
method's arithmetic, and both the GPU path's tests/benchmarks and the CPU
oracle's tests draw their inputs from it.

The rho-correlated stochastic block model (Sec. 4.1 of the paper, sampler in the
style of graspologic's): for every vertex pair {i, j}, i < j, in blocks (r, c)
with edge probability p = Pb[r, c]

    A_ij ~ Bernoulli(p)
    B'_ij | A_ij = 1 ~ Bernoulli(p + rho (1 - p))
    B'_ij | A_ij = 0 ~ Bernoulli(p (1 - rho))

so both graphs are Bernoulli(p) with edge correlation rho; rho = 1 gives
isomorphic graphs, rho = 0 independent ones.  The Erdos-Renyi model is the
single-block case.  B is then B' with its vertices relabelled by a seeded
permutation sigma (B[a, b] = B'[sigma a, sigma b]) so that no method can profit
from the input order (the paper shuffles B for the same reason), and the
hidden correspondence is truth[i] = sigma^{-1}(i): vertex i of A is vertex
truth[i] of B.

Pairs are sampled sparsely (binomial edge counts, distinct uniform pairs), so
n = 32768 pairs take seconds; dense byte matrices are assembled at the end.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class GraphPair:
    A: np.ndarray          # n x n, uint8 (0/1) or float32 (weighted), symmetric, zero diagonal
    B: np.ndarray          # same shape and dtype as A
    truth: np.ndarray      # int32 [n]: vertex i of A corresponds to vertex truth[i] of B
    n: int
    seed: int


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _distinct_uniform(rng, count: int, total: int) -> np.ndarray:
    """`count` distinct integers drawn uniformly from [0, total)."""
    if count <= 0:
        return np.zeros(0, dtype=np.int64)
    if count > total // 2:
        return np.sort(rng.choice(total, size=count, replace=False)).astype(np.int64)
    got = np.zeros(0, dtype=np.int64)
    while got.size < count:
        extra = rng.integers(0, total, size=int((count - got.size) * 1.1) + 16, dtype=np.int64)
        got = np.unique(np.concatenate([got, extra]))
    if got.size > count:
        got = np.sort(rng.choice(got, size=count, replace=False))
    return got


def _bernoulli_pairs(rng, rows: np.ndarray, cols: np.ndarray, same_block: bool, p: float):
    """Independent Bernoulli(p) draw over the vertex pairs of one block pair.

    rows/cols hold the global vertex ids of the two blocks.  For a diagonal
    block the pairs are the unordered {i, j}, i < j.  Returns (i, j) arrays of
    global ids with i < j."""
    mr, mc = rows.size, cols.size
    if same_block:
        total = mr * (mr - 1) // 2
    else:
        total = mr * mc
    if total == 0 or p <= 0.0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    k = int(rng.binomial(total, min(p, 1.0)))
    idx = _distinct_uniform(rng, k, total)
    if same_block:
        # unordered pair index t -> (a, b), a < b, row-major over the strict upper
        # triangle: row a starts at S[a] = a (2 mr - a - 1) / 2
        ar = np.arange(mr, dtype=np.int64)
        S = ar * (2 * mr - ar - 1) // 2
        a = np.searchsorted(S, idx, side="right") - 1
        b = idx - S[a] + a + 1
        i, j = rows[a], rows[b]
    else:
        i, j = rows[idx // mc], cols[idx % mc]
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    return lo.astype(np.int64), hi.astype(np.int64)


def rho_sbm_edges(block_sizes, block_p, rho: float, seed: int):
    """Edge lists (i < j) of a rho-correlated SBM pair in A's vertex order.

    Returns (n, eA, eB) with eA, eB int64 arrays of shape [m, 2]."""
    rng = _rng(seed)
    sizes = [int(s) for s in block_sizes]
    n = int(sum(sizes))
    Pb = np.asarray(block_p, dtype=np.float64)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    eA, eB = [], []
    for r in range(len(sizes)):
        for c in range(r, len(sizes)):
            p = float(Pb[r, c])
            rows = np.arange(starts[r], starts[r + 1], dtype=np.int64)
            cols = np.arange(starts[c], starts[c + 1], dtype=np.int64)
            same = r == c
            ai, aj = _bernoulli_pairs(rng, rows, cols, same, p)
            # B' on A's edges: keep with probability p + rho (1 - p)
            keep = rng.random(ai.size) < (p + rho * (1.0 - p))
            # B' on A's non-edges: Bernoulli(p (1 - rho)) restricted to non-edges of A
            ni, nj = _bernoulli_pairs(rng, rows, cols, same, p * (1.0 - rho))
            if ni.size:
                codeA = ai * n + aj
                codeN = ni * n + nj
                fresh = ~np.isin(codeN, codeA)
                ni, nj = ni[fresh], nj[fresh]
            eA.append(np.stack([ai, aj], 1))
            eB.append(np.concatenate([np.stack([ai[keep], aj[keep]], 1), np.stack([ni, nj], 1)], 0))
    eA = np.concatenate(eA, 0) if eA else np.zeros((0, 2), np.int64)
    eB = np.concatenate(eB, 0) if eB else np.zeros((0, 2), np.int64)
    return n, eA, eB


def _dense(n: int, edges: np.ndarray, weights=None, dtype=np.uint8) -> np.ndarray:
    M = np.zeros((n, n), dtype=dtype)
    if edges.size:
        val = 1 if weights is None else weights
        M[edges[:, 0], edges[:, 1]] = val
        M[edges[:, 1], edges[:, 0]] = val
    return M


def rho_sbm_pair(block_sizes, block_p, rho: float, seed: int, weighted: bool = False) -> GraphPair:
    """A rho-correlated SBM pair with B vertex-permuted by a seeded sigma.

    weighted=True puts lognormal(0, 1) weights on A's edges; an edge present in
    both graphs carries the same weight in B, an edge only in B draws a fresh
    weight.  Matrices are then float32."""
    n, eA, eB = rho_sbm_edges(block_sizes, block_p, rho, seed)
    rng = _rng(seed + 7_777_777)
    sigma = rng.permutation(n).astype(np.int64)     # B[a, b] = B'[sigma a, sigma b]
    sigma_inv = np.empty(n, dtype=np.int64)
    sigma_inv[sigma] = np.arange(n)
    eBp = sigma_inv[eB]                              # B' edge (i, j) -> B edge (sigma^-1 i, sigma^-1 j)
    if weighted:
        wA = rng.lognormal(0.0, 1.0, size=eA.shape[0]).astype(np.float32)
        codeA = eA[:, 0] * n + eA[:, 1]
        codeB = eB[:, 0] * n + eB[:, 1]
        order = np.argsort(codeA)
        pos = np.searchsorted(codeA[order], codeB)
        pos = np.minimum(pos, max(codeA.size - 1, 0))
        shared = (codeA.size > 0) & (codeA[order][pos] == codeB) if codeA.size else np.zeros(codeB.size, bool)
        wB = rng.lognormal(0.0, 1.0, size=eB.shape[0]).astype(np.float32)
        if codeA.size:
            wB[shared] = wA[order][pos[shared]]
        A = _dense(n, eA, wA, np.float32)
        B = _dense(n, eBp, wB, np.float32)
    else:
        A = _dense(n, eA)
        B = _dense(n, eBp)
    return GraphPair(A=A, B=B, truth=sigma_inv.astype(np.int32), n=n, seed=seed)


def rho_er_pair(n: int, p: float, rho: float, seed: int, weighted: bool = False) -> GraphPair:
    """A rho-correlated Erdos-Renyi pair (the one-block SBM)."""
    return rho_sbm_pair([n], [[p]], rho, seed, weighted=weighted)


def rho_er_digraph_pair(n: int, p: float, rho: float, seed: int, weighted: bool = False) -> GraphPair:
    """A rho-correlated directed Erdos-Renyi pair: every ordered pair (i, j), i != j,
    is an arc of A with probability p; B' keeps an arc of A with probability
    p + rho (1 - p) and adds one where A has none with probability p (1 - rho), so
    each graph has density p and arc correlation rho; B = B' relabelled by a seeded
    sigma.  Dense sampling (n up to a few thousand).  weighted=True: lognormal(0, 1)
    weights on A's arcs, shared arcs carry A's weight in B, new arcs fresh ones."""
    rng = _rng(seed + 31_337)
    a = rng.random((n, n)) < p
    u = rng.random((n, n))
    b = np.where(a, u < p + rho * (1.0 - p), u < p * (1.0 - rho))
    np.fill_diagonal(a, False)
    np.fill_diagonal(b, False)
    sigma = rng.permutation(n).astype(np.int64)
    sigma_inv = np.empty(n, dtype=np.int64)
    sigma_inv[sigma] = np.arange(n)
    if weighted:
        wa = rng.lognormal(0.0, 1.0, size=(n, n)).astype(np.float32)
        wb = np.where(a, wa, rng.lognormal(0.0, 1.0, size=(n, n)).astype(np.float32))
        A = np.where(a, wa, 0.0).astype(np.float32)
        Bp = np.where(b, wb, 0.0).astype(np.float32)
    else:
        A = a.astype(np.uint8)
        Bp = b.astype(np.uint8)
    B = np.ascontiguousarray(Bp[np.ix_(sigma, sigma)])  # B[x, y] = B'[sigma x, sigma y]
    return GraphPair(A=np.ascontiguousarray(A), B=B, truth=sigma_inv.astype(np.int32), n=n, seed=seed)


def sbm3_block_sizes(n: int, fractions=(0.40, 0.35, 0.25)):
    """Block sizes for the 3-block SBM: floor of each fraction, remainder to the last block."""
    sizes = [int(np.floor(f * n)) for f in fractions[:-1]]
    sizes.append(n - sum(sizes))
    return sizes


def large_sbm_pair(n: int = 32768, p_in: float = 0.02, p_out: float = 0.004, rho: float = 0.7,
                   seed: int = 3000) -> GraphPair:
    """The large single-pair workload: 3-block SBM (40/35/25 %), p_in on the diagonal blocks."""
    sizes = sbm3_block_sizes(n)
    Pb = np.full((3, 3), p_out)
    np.fill_diagonal(Pb, p_in)
    return rho_sbm_pair(sizes, Pb, rho, seed)


def uniform_noise(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """U[0, 1) noise of shape n x n (the raw material of a random doubly stochastic init)."""
    return _rng(seed).random((n, n)).astype(dtype)


def uniform_costs(n: int, low: float, high: float, seed: int, dtype=np.float64) -> np.ndarray:
    """Cost matrix with i.i.d. Uniform(low, high) entries (the paper's LAP-vs-LOT inputs)."""
    return _rng(seed).uniform(low, high, size=(n, n)).astype(dtype)


def random_permutation(n: int, seed: int) -> np.ndarray:
    return _rng(seed).permutation(n).astype(np.int32)
