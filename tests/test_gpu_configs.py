"""GPU parity at the sizes of the configured workloads beyond the benchmark's own:
resolution transfer (128..512 grids, 64 instances), large single solves (1024 x 1024 with 8
instances, 2048 x 2048 with 2, 16 x 16 modes, sigma 2, length 0.05), and the precision
acceptance of the 16-bit preconditioner (iteration count within 15 % of the FP64 one).
Outputs the oracle can compute one by one are sampled; the rest is checked through
properties that hold at any size."""
import numpy as np
import pytest

from oracle import fcgno_oracle as O
from paper_2402_05598_gb300 import inputs as I

from test_gpu_parity import ELEM_TOL, batch, elem_check, model_pair, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,M,B,sigma,ell,sample", [
    (512, 12, 64, 2.0, 0.1, (0, 31, 63)),     # resolution transfer, largest grid
    (1024, 16, 8, 2.0, 0.05, (0, 7)),         # large single solves
    (2048, 16, 2, 2.0, 0.05, (1,)),
])
def test_preconditioner_at_workload_sizes_sampled(lib, dev, N, M, B, sigma, ell, sample):
    """BF16 tensor-core preconditioner on the whole batch; sampled instances against the FP64
    oracle (2e-2 relative), all outputs finite."""
    import torch
    k, r = batch(N, B, 7000 + N, sigma, ell)
    desc, P, model, _w = model_pair(lib, dev, 32, M)
    op = lib.Operator(to_dev(k, dev))
    z = torch.empty((B, N, N), dtype=torch.float64, device=dev)
    lib.precond_apply(model, op, to_dev(r, dev), z, prec="bf16")
    zs = z.cpu().numpy()
    assert np.all(np.isfinite(zs))
    for b in sample:
        ref = O.no_forward(P, desc, r[b], np.log(k[b]))
        err = rel(zs[b], ref)
        assert err < 2e-2, (b, err)
        elem_check(zs[b], ref, ELEM_TOL["bf16"], ("bf16", N, b))


@pytest.mark.parametrize("N,B,prec", [(1024, 8, "bf16"), (2048, 2, "bf16"), (256, 4, "fp64")])
def test_large_solve_recursive_residual_is_the_true_residual(lib, dev, N, B, prec):
    """Six FCG-NO iterations (m = 5) on the large-solve grids through the tiled FCG kernels:
    the recursively updated residual of Algorithm 1 (reported relres) equals the true residual
    b - A x of the returned iterate (computed by the oracle's stencil) up to rounding. This
    holds at any size and fails for a wrong alpha, update or stencil. (The residual norm itself
    need not fall: FCG minimises the energy norm of the error, and the oracle's own run of the
    same case grows ||r|| by 5-20 % over these iterations.) The FP64 case is also compared with
    the oracle's iterate on one instance."""
    import torch
    k, f = batch(N, B, 7100 + N, 2.0, 0.05)
    desc, P, model, _w = model_pair(lib, dev, 32, 16 if N >= 1024 else 12)
    op = lib.Operator(to_dev(k, dev))
    x = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
    info = lib.solve(op, model, to_dev(f, dev), x, m_max=5, max_iter=6, fixed_iters=True, prec=prec)
    xs = x.cpu().numpy()
    for b in range(B):
        assert info[b]["iters"] == 6
        r0 = np.linalg.norm(f[b])
        assert abs(info[b]["r0norm"] - r0) <= 1e-12 * r0
        true = np.linalg.norm(f[b] - O.apply_A(k[b], xs[b])) / r0
        assert abs(true - info[b]["relres"]) <= 1e-9, (b, true, info[b]["relres"])
    if prec == "fp64":
        ref = O.fcg(lambda u: O.apply_A(k[0], u), lambda r: O.no_forward(P, desc, r, np.log(k[0])), f[0],
                    np.zeros((N, N)), 5, 6)
        assert rel(xs[0], ref["u"]) < 1e-10
        elem_check(xs[0], ref["u"], 1e-10, ("fp64 iterate", N), "global")


def test_bf16_iterations_within_15_percent_of_fp64(lib, dev):
    """Precision acceptance: with a preconditioner trained briefly on Krylov vectors (64 x 64,
    width 32, 12 x 12 modes), FCG-NO with the BF16 tensor-core preconditioner reaches relative
    residual 1e-6 on every held-out instance, and its true residual agrees. Its mean iteration
    count over the batch is at most 15 % above that of the same solves with the FP64
    preconditioner; per instance (where 16-bit rounding sends a nonlinear preconditioner's
    iteration down another path) it stays within 1.5 x + 2."""
    import torch
    from paper_2402_05598_gb300 import train as T
    N, B = 64, 16
    desc_np = I.ModelDesc(width=32, layers=4, modes=12, proj_width=32)
    blob = to_dev(I.xavier_weights(desc_np, 0), dev)
    model = lib.Model(lib.make_desc(32, 4, 12, 32), blob)
    T.train(model, N, range(0, 64), K=100, batch=32, lr=1e-3, steps=1500)
    k, f = batch(N, B, 10000)
    u0 = np.stack([np.random.default_rng(s + 777).standard_normal((N, N)) for s in range(10000, 10000 + B)])
    op = lib.Operator(to_dev(k, dev))
    its = {}
    for prec in ("fp64", "bf16"):
        x = to_dev(u0, dev)
        info = lib.solve(op, model, to_dev(f, dev), x, tol=1e-6, m_max=1, max_iter=400, prec=prec)
        xs = x.cpu().numpy()
        its[prec] = [i["iters"] for i in info]
        for b in range(B):
            assert info[b]["status"] == lib.FCGNO_OK and info[b]["relres"] <= 1e-6, (prec, b, info[b])
            r0 = np.linalg.norm(f[b] - O.apply_A(k[b], u0[b]))
            assert np.linalg.norm(f[b] - O.apply_A(k[b], xs[b])) / r0 <= 2e-6
    assert np.mean(its["bf16"]) <= 1.15 * np.mean(its["fp64"]), its
    for b in range(B):
        assert its["bf16"][b] <= 1.5 * its["fp64"][b] + 2, (b, its)


def test_fine_tuning_step_on_the_large_grid_recomputes_and_matches(lib, dev):
    """A fine-tuning step of the large-solve configuration (1024 x 1024, 8 instances, width 32,
    16 x 16 modes) on Krylov vectors of CG (with a coarse CG solution as u*, which only sets
    the error vectors e_i = u* - u_i): in the automatic mode the step rebuilds the
    pre-activations (they would take 4 GiB) and returns exactly the loss and gradient of the
    step that keeps them; both are finite and the loss (a ratio of energy norms) is positive."""
    import torch
    N, B = 1024, 8
    k, f = batch(N, B, 7300, 2.0, 0.05)
    desc, P, model, wdev = model_pair(lib, dev, 32, 16)
    op = lib.Operator(to_dev(k, dev))
    fb = to_dev(f, dev)
    x0 = to_dev(np.random.default_rng(5).standard_normal((B, N, N)), dev)
    ustar = torch.zeros_like(fb)
    lib.solve(op, None, fb, ustar, tol=1e-4, m_max=1, max_iter=2000, prec="fp64", check_every=64)
    K = 3
    r_out = torch.empty((K, B, N, N), dtype=torch.float64, device=dev)
    e_out = torch.empty_like(r_out)
    lib.krylov_harvest(op, fb, x0, ustar, K, r_out, e_out)
    r, e = r_out[K - 1].contiguous(), e_out[K - 1].contiguous()
    out = {}
    for mode in ("auto", "never"):
        model.set_train_recompute(mode)
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        grad = torch.zeros(wdev.numel(), dtype=torch.float32, device=dev)
        lib.train_step(model, op, r, e, loss, grad, prec="fp32")
        torch.cuda.synchronize()
        out[mode] = (loss.clone(), grad.clone())
    assert torch.isfinite(out["auto"][1]).all() and np.isfinite(out["auto"][0].item())
    assert torch.equal(out["auto"][0], out["never"][0]) and torch.equal(out["auto"][1], out["never"][1])
    assert out["auto"][0].item() > 0.0
