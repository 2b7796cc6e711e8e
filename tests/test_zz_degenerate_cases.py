"""Degenerate cases of the solve. Shapes the 16-bit (tensor-core) preconditioner does not
support are argument errors: the solve and the preconditioner application return
FCGNO_EINVAL before any launch and leave their outputs untouched; the CUDA-core
preconditioners take the same shape. A preconditioner that returns zero makes
(p_0, A p_0) = 0: every instance stops at iteration 0 with FCGNO_EBREAKDOWN (Algorithm 1
cannot take a step), as the oracle does, and x is left as it was. A NaN in one instance's
input fails that instance alone. A bounded device wait that runs out is reported as
FCGNO_ETIMEOUT and leaves the context usable."""
import numpy as np
import pytest

from paper_2402_05598_gb300 import inputs as I


@pytest.mark.gpu
def test_unsupported_16bit_shape_is_rejected_before_any_launch(lib, dev):
    import torch
    N, B, C, M = 48, 2, 32, 12  # N is neither 32, 64 nor a multiple of 128
    k, f = I.make_batch(N, [3, 4])
    desc = I.ModelDesc(width=C, layers=4, modes=M, proj_width=C)
    w = torch.from_numpy(I.xavier_weights(desc, 0)).to(dev)
    model = lib.Model(lib.make_desc(C, 4, M, C), w)
    op = lib.Operator(torch.from_numpy(k).to(dev))
    fb = torch.from_numpy(f).to(dev)
    x = torch.full((B, N, N), 0.5, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    for prec in ("bf16", "fp16"):
        n0 = lib.launch_count()
        with pytest.raises(lib.FcgnoError) as ei:
            lib.solve(op, model, fb, x, tol=1e-6, m_max=1, max_iter=10, prec=prec)
        assert ei.value.code == lib.FCGNO_EINVAL and "16-bit" in str(ei.value)
        with pytest.raises(lib.FcgnoError) as ei:
            lib.precond_apply(model, op, fb, x, prec=prec)
        assert ei.value.code == lib.FCGNO_EINVAL and "16-bit" in str(ei.value)
        assert lib.launch_count() == n0
    torch.cuda.synchronize()
    assert bool(torch.all(x == 0.5))
    x.zero_()
    info = lib.solve(op, model, fb, x, tol=1e-6, m_max=1, max_iter=3, prec="fp64", fixed_iters=True)
    assert all(i["iters"] == 3 for i in info)
    assert np.isfinite(x.cpu().numpy()).all()


@pytest.mark.gpu
@pytest.mark.parametrize("N,prec", [(32, "fp64"), (32, "bf16"), (128, "bf16")])
def test_zero_preconditioner_breaks_down_at_the_first_step(lib, dev, N, prec):
    import torch
    from oracle import fcgno_oracle as O
    B, C, M = 2, 32, 12
    k, f = I.make_batch(N, [7, 8])
    desc = I.ModelDesc(width=C, layers=4, modes=M, proj_width=C)
    w = torch.zeros(I.weight_count(desc), dtype=torch.float32, device=dev)
    model = lib.Model(lib.make_desc(C, 4, M, C), w)
    op = lib.Operator(torch.from_numpy(k).to(dev))
    x0 = np.random.default_rng(3).standard_normal((B, N, N))
    x = torch.from_numpy(x0).to(dev)
    info = lib.solve(op, model, torch.from_numpy(f).to(dev), x, tol=1e-6, m_max=5, max_iter=50, prec=prec)
    P = O.unpack_weights(np.zeros(I.weight_count(desc)), desc)
    for b in range(B):
        ref = O.fcg(lambda u: O.apply_A(k[b], u), lambda r: O.no_forward(P, desc, r, np.log(k[b])), f[b], x0[b],
                    5, 50, tol=1e-6)
        assert ref["status"] == O.STATUS_BREAKDOWN and ref["iterations"] == 0
        assert info[b]["status"] == lib.FCGNO_EBREAKDOWN and info[b]["iters"] == 0, info[b]
    assert np.array_equal(x.cpu().numpy(), x0)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["bf16", "fp64"])
def test_a_nan_input_fails_only_its_own_instance(lib, dev, prec):
    """A NaN in one instance's right-hand side makes its (p_0, A p_0) non-finite: that
    instance stops at iteration 0 with FCGNO_EBREAKDOWN and x unchanged, and the other
    instances give bit for bit the results they give when that right-hand side is clean (no
    kernel mixes instances: the mode-mixing GEMM's rows are independent and every reduction
    is per instance in a fixed order; the instances keep their positions in the batch)."""
    import torch
    N, C, M = 64, 32, 12
    k, f = I.make_batch(N, [21, 22, 23])
    f_bad = f.copy()
    f_bad[1, 5, 7] = np.nan
    desc = I.ModelDesc(width=C, layers=4, modes=M, proj_width=C)
    w = torch.from_numpy(I.xavier_weights(desc, 1)).to(dev)
    model = lib.Model(lib.make_desc(C, 4, M, C), w)
    x0 = np.random.default_rng(4).standard_normal((3, N, N))
    op3 = lib.Operator(torch.from_numpy(k).to(dev))
    x3 = torch.from_numpy(x0).to(dev)
    info3 = lib.solve(op3, model, torch.from_numpy(f_bad).to(dev), x3, tol=1e-6, m_max=5, max_iter=24, prec=prec)
    x_clean = torch.from_numpy(x0).to(dev)
    info_clean = lib.solve(op3, model, torch.from_numpy(f).to(dev), x_clean, tol=1e-6, m_max=5, max_iter=24,
                           prec=prec)
    assert info3[1]["status"] == lib.FCGNO_EBREAKDOWN and info3[1]["iters"] == 0
    assert info_clean[1]["status"] != lib.FCGNO_EBREAKDOWN and info_clean[1]["iters"] > 0
    xs3, xs_clean = x3.cpu().numpy(), x_clean.cpu().numpy()
    assert np.array_equal(xs3[1], x0[1])
    for b in (0, 2):
        assert info3[b]["iters"] == info_clean[b]["iters"] and info3[b]["status"] == info_clean[b]["status"]
        assert np.array_equal(xs3[b], xs_clean[b])


@pytest.mark.gpu
@pytest.mark.parametrize("limit", [2e-6, 5e-5])
def test_bounded_wait_gives_up_and_the_context_stays_usable(lib, dev, limit):
    """Failure detection without a GPU fault: a wait (the tensor-core kernels' bounded mbarrier
    wait) on a barrier phase that nothing completes gives up after the caller's limit of a few
    microseconds, and the call reports FCGNO_ETIMEOUT through the operator's timeout flag. The
    flag is cleared by that report, and a BF16 solve on the same operator and context then
    matches the FP64 oracle's preconditioner and iterate as in the parity tests."""
    import torch
    from oracle import fcgno_oracle as O
    from test_gpu_parity import ELEM_TOL, batch, elem_check, model_pair, rel, to_dev
    N, B = 32, 2
    k, f = batch(N, B, 9300)
    desc, P, model, _w = model_pair(lib, dev, 16, 8)
    op = lib.Operator(to_dev(k, dev))
    assert lib.wait_selftest(op, limit) == lib.FCGNO_ETIMEOUT
    assert "bounded device wait" in lib.last_error()
    z = torch.empty((B, N, N), dtype=torch.float64, device=dev)
    lib.precond_apply(model, op, to_dev(f, dev), z, prec="bf16")
    x = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
    info = lib.solve(op, model, to_dev(f, dev), x, m_max=1, max_iter=4, fixed_iters=True, prec="fp64")
    zs, xs = z.cpu().numpy(), x.cpu().numpy()
    for b in range(B):
        ref = O.no_forward(P, desc, f[b], np.log(k[b]))
        assert rel(zs[b], ref) < 2e-2
        elem_check(zs[b], ref, ELEM_TOL["bf16"], ("after time-out", b))
        it = O.fcg(lambda u: O.apply_A(k[b], u), lambda r: O.no_forward(P, desc, r, np.log(k[b])), f[b],
                   np.zeros((N, N)), 1, 4)
        assert info[b]["status"] == lib.FCGNO_OK and rel(xs[b], it["u"]) < 1e-10
