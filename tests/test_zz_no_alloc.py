"""GPU test of fcgno_solve_noalloc, the solve entry point for callers that cannot allocate
device memory (a fixed, pre-reserved memory budget, or a context where the CUDA allocator
must not be entered). Its Krylov state lives in the library's fixed 8 MiB device array.

This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import math

import numpy as np
import pytest

from oracle import fcgno_oracle as O
from paper_2402_05598_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_solve_matches_solve_on_two_calls_in_a_row(lib, dev):
    """Two consecutive calls (different shapes, windows and grid paths) agree with
    fcgno_solve (identity preconditioner) to the FP64 parity tolerance of the other tests.
    The first call runs 20 fixed iterations and is also compared with the FP64 oracle's
    iterate (CG, Algorithm 1 with B = I) within 10x the oracle's own rounding sensitivity;
    the second solves to 1e-8. The second call leaves free device memory unchanged."""
    import torch
    cases = [(48, 3, 1, 2000, True), (100, 2, 3, 2100, False)]  # fused (N <= 90) and tiled paths
    for call, (N, B, m, seed, fixed) in enumerate(cases):
        k, f = I.make_batch(N, range(seed, seed + B))
        x0 = np.random.default_rng(seed).standard_normal((B, N, N))
        op = lib.Operator(torch.from_numpy(k).to(dev))
        fb = torch.from_numpy(f).to(dev)
        xa = torch.from_numpy(x0).to(dev)
        xb = xa.clone()
        iters = 20 if fixed else 3000
        ia = lib.solve(op, None, fb, xa, tol=1e-8, m_max=m, max_iter=iters, fixed_iters=fixed, prec="fp64")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        ib = lib.solve_noalloc(op, fb, xb, tol=1e-8, m_max=m, max_iter=iters, fixed_iters=fixed)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        assert [i["iters"] for i in ib] == [i["iters"] for i in ia]
        assert [i["status"] for i in ib] == [i["status"] for i in ia] == [lib.FCGNO_OK] * B
        if fixed:
            # 20 fixed iterations: the two paths sum the dot products of Algorithm 1 in different
            # orders (one CTA per instance or a cluster of bands), and the recurrences amplify
            # that rounding; both are held to 10x the oracle's own sensitivity to the order
            xs, xas = xb.cpu().numpy(), xa.cpu().numpy()
            for b in range(B):
                run = lambda d: O.fcg(lambda u: O.apply_A(k[b], u), lambda r: r, f[b], x0[b], m, iters,
                                      **({} if d is None else {"dot": d}))["u"]
                ref = run(None)
                sens = rel(run(lambda a_, b_: math.fsum(np.ravel(a_ * b_))), ref)
                tol = max(1e-10, 10.0 * sens)
                assert ib[b]["iters"] == iters
                assert rel(xs[b], ref) < tol
                assert rel(xs[b], xas[b]) < tol
                assert abs(ib[b]["relres"] - ia[b]["relres"]) <= tol * max(ia[b]["relres"], 1e-300) + 1e-14
        else:
            for b in range(B):
                assert abs(ib[b]["relres"] - ia[b]["relres"]) <= 1e-10 * max(ia[b]["relres"], 1e-300) + 1e-14
            assert rel(xb.cpu().numpy(), xa.cpu().numpy()) < 1e-10


def test_noalloc_solve_rejects_problems_beyond_its_fixed_scratch(lib, dev):
    import torch
    N, B = 128, 16  # 16 x 128 x 128 unknowns need more than 8 MiB of Krylov state
    k, f = I.make_batch(N, range(B))
    op = lib.Operator(torch.from_numpy(k).to(dev))
    x = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
    with pytest.raises(lib.FcgnoError) as ei:
        lib.solve_noalloc(op, torch.from_numpy(f).to(dev), x, tol=1e-6)
    assert ei.value.code == lib.FCGNO_EINVAL
    assert "8 MiB" in str(ei.value)
