"""The allocation-free Sinkhorn entry point against the regular one.

goat_sinkhorn_noalloc exists for callers that cannot allocate device memory
during the call (for example code running under an allocator it does not own or
within a fixed memory budget); it keeps its scratch in one static device array.
This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It also runs alone in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2111_05366_gb300 as goat  # noqa: E402
from paper_2111_05366_gb300 import synthetic  # noqa: E402


def _cost(n, seed):
    gp = synthetic.rho_er_pair(n, 0.1, 0.8, seed=seed)
    rng = np.random.default_rng(seed)
    P = np.zeros((n, n), np.float32)
    for w in rng.random(4) + 0.1:
        P[np.arange(n), rng.permutation(n)] += w
    P /= P.sum(1, keepdims=True)
    G = goat.goat_gradient(torch.from_numpy(gp.A).cuda(), torch.from_numpy(gp.B).cuda(), torch.from_numpy(P).cuda(),
                           precision=goat.GOAT_PREC_FP32)
    return G


def test_noalloc_matches_regular_entry_on_two_calls_in_a_row():
    # two consecutive calls with different sizes and inputs: the second must not see the first's state
    for n, seed, iters, tol in [(300, 1, 40, 1e-4), (1000, 2, 60, 1e-5)]:
        G = _cost(n, seed)
        eps = 0.03 * float(G.abs().max())
        g0 = torch.from_numpy((np.random.default_rng(seed).standard_normal(n) * eps).astype(np.float32)).cuda()
        f_r, g_r, _, it_r, res_r = goat.goat_sinkhorn(G, eps, tol, iters, g_init=g0)
        f_n, g_n, it_n, res_n = goat.goat_sinkhorn_noalloc(G, eps, tol, iters, g_init=g0)
        torch.cuda.synchronize()
        assert int(it_n.item()) == it_r
        assert float(res_n.item()) == pytest.approx(res_r, rel=1e-6, abs=1e-9)
        np.testing.assert_allclose(f_n.cpu().numpy(), f_r.cpu().numpy(), atol=2e-3 * eps, rtol=0)
        np.testing.assert_allclose(g_n.cpu().numpy(), g_r.cpu().numpy(), atol=2e-3 * eps, rtol=0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n = goat.NOALLOC_MAX_N + 1
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = goat.load().goat_sinkhorn_noalloc(p, n, 1.0, 1e-3, 10, p, p, None, None,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == goat.GOAT_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        goat.goat_sinkhorn_noalloc(torch.zeros((n, n), dtype=torch.float32, device="cuda"), 1.0, 1e-3, 10)
