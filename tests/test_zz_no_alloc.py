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


def _raw_call(G, eps, tol, iters, f, g, it, res, status):
    """goat_sinkhorn_noalloc through the C ABI with caller-owned device outputs."""
    n = G.shape[0]
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    return goat.load().goat_sinkhorn_noalloc(vp(G), n, float(eps), float(tol), int(iters), vp(f), vp(g), vp(it),
                                             vp(res), vp(status),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_regular_entry_on_two_calls_in_a_row():
    # two consecutive calls with different sizes and inputs: the second must not see the first's state
    for n, seed, iters, tol in [(300, 1, 40, 1e-4), (1000, 2, 60, 1e-5)]:
        G = _cost(n, seed)
        eps = 0.03 * float(G.abs().max())
        g0 = torch.from_numpy((np.random.default_rng(seed).standard_normal(n) * eps).astype(np.float32)).cuda()
        f_r, g_r, _, it_r, res_r = goat.goat_sinkhorn(G, eps, tol, iters, g_init=g0)
        f_n, g_n, it_n, res_n, st_n = goat.goat_sinkhorn_noalloc(G, eps, tol, iters, g_init=g0)
        torch.cuda.synchronize()
        assert int(st_n.item()) == goat.GOAT_OK
        assert int(it_n.item()) == it_r
        assert float(res_n.item()) == pytest.approx(res_r, rel=1e-6, abs=1e-9)
        np.testing.assert_allclose(f_n.cpu().numpy(), f_r.cpu().numpy(), atol=2e-3 * eps, rtol=0)
        np.testing.assert_allclose(g_n.cpu().numpy(), g_r.cpu().numpy(), atol=2e-3 * eps, rtol=0)


def test_noalloc_call_allocates_no_device_memory():
    # preallocated inputs and outputs, one warm-up call (it looks up the static
    # array's address), then the device's free memory must not move across a call
    n = 4096
    G = _cost(n, 3)
    eps = 0.03 * float(G.abs().max())
    f = torch.empty(n, dtype=torch.float32, device="cuda")
    g = torch.zeros(n, dtype=torch.float32, device="cuda")
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    res = torch.zeros(1, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _raw_call(G, eps, 1e-4, 50, f, g, it, res, status) == goat.GOAT_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    g.zero_()
    assert _raw_call(G, eps, 1e-4, 50, f, g, it, res, status) == goat.GOAT_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
    assert int(status.item()) == goat.GOAT_OK and int(it.item()) >= 1


def test_noalloc_reports_a_non_finite_cost_in_its_status():
    n = 256
    G = _cost(n, 4)
    eps = 0.03 * float(G.abs().max())
    G[7, 11] = float("-inf")  # exp(-G/eps) overflows: the residual is not finite
    _, _, _, res, status = goat.goat_sinkhorn_noalloc(G, eps, 1e-4, 20)
    torch.cuda.synchronize()
    assert int(status.item()) == goat.GOAT_ERR_NAN
    assert not np.isfinite(float(res.item()))
    # the next call on finite input starts clean
    G[7, 11] = -1.0
    _, _, _, _, status = goat.goat_sinkhorn_noalloc(G, eps, 1e-4, 20)
    torch.cuda.synchronize()
    assert int(status.item()) == goat.GOAT_OK


def test_noalloc_rejects_sizes_beyond_its_scratch_and_queue():
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = goat.load()
    n = goat.NOALLOC_MAX_N + 1
    assert lib.goat_sinkhorn_noalloc(p, n, 1.0, 1e-3, 10, p, p, None, None, None, stream) == goat.GOAT_ERR_INVALID_ARG
    assert (lib.goat_sinkhorn_noalloc(p, 2, 1.0, 1e-3, goat.NOALLOC_MAX_ITER + 1, p, p, None, None, None, stream)
            == goat.GOAT_ERR_INVALID_ARG)
    with pytest.raises(ValueError):
        goat.goat_sinkhorn_noalloc(torch.zeros((n, n), dtype=torch.float32, device="cuda"), 1.0, 1e-3, 10)
