"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle on the same
seeded inputs. Sizes span several tiles and ragged tails; tolerances are stated per test."""
import math

import numpy as np
import pytest

from oracle import fcgno_oracle as O
from paper_2402_05598_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# Element-wise bounds (beside the 2-norm ones). FP64 paths: the stated tolerance itself, as a
# fraction of max|oracle|. 16-bit tensor-core preconditioner: every operand is rounded to 8
# (BF16) or 11 (FP16) significant bits, unit roundoff u = 2^-9 / 2^-12, and each of the four
# layers adds roughly u times the field's scale through its contractions (FP32 accumulation),
# so the error of one grid point stays within a few times 4u of max|z|: 4u = 7.8e-3 (BF16),
# 9.8e-4 (FP16). The bounds below are 5e-2 (BF16) and 1e-2 (FP16) of max|z|.
ELEM_TOL = {"fp64": 1e-12, "fp32": 1e-4, "bf16": 5e-2, "fp16": 1e-2}


def elem_check(z, ref, tol, what="", edge_scale="own"):
    """max |z - ref| <= tol * max|ref| over the whole grid, and on each grid edge (q = 0,
    q = N-1, p = 0, p = N-1) relative to that edge's own max|ref| (edge_scale "own"), so
    that one wrong grid point, a wrong tile edge or a wrong boundary column cannot hide in a
    norm. Iterates of the Dirichlet problem are small next to the walls while their rounding
    spreads at the field's scale: for them (edge_scale "global") each edge is held to
    tol * max|ref| over the whole grid, which still fails a wrong boundary column."""
    z, ref = np.asarray(z, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    assert z.shape == ref.shape and z.ndim == 2
    err = np.abs(z - ref)
    scale = float(np.max(np.abs(ref)))
    worst = np.unravel_index(int(np.argmax(err)), err.shape)
    assert err.max() <= tol * scale, (what, "max", float(err.max() / max(scale, 1e-300)), worst)
    edges = {"q=0": (0, slice(None)), "q=N-1": (-1, slice(None)), "p=0": (slice(None), 0),
             "p=N-1": (slice(None), -1)}
    for name, sl in edges.items():
        es = float(err[sl].max())
        ss = float(np.max(np.abs(ref[sl]))) if edge_scale == "own" else scale
        assert es <= tol * ss, (what, name, es / max(ss, 1e-300))


def to_dev(x, dev, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev)


def exact_dot(a, b):
    return math.fsum(np.ravel(a * b))


def rounding_tol(run, floor=1e-10):
    """Tolerance for an FP64 iterate: 10x the change of the oracle's own result when its dot
    products are exactly rounded instead of pairwise-summed (the recurrences of Algorithm 1
    amplify rounding; a GPU reduction order is one more valid rounding)."""
    a, b = run(None), run(exact_dot)
    return max(floor, 10.0 * rel(b, a))


def batch(N, B, seed0, sigma=1.0, ell=0.1):
    return I.make_batch(N, range(seed0, seed0 + B), sigma, ell)


def model_pair(lib, dev, C, M, L=4, seed=0, wscale=1.0, out_scale=0):
    """Seeded Xavier weights (times `wscale`, which drives the GELUs further from their
    linear range) with nonzero biases; returns (desc, oracle weights, library model, blob)."""
    desc_np = I.ModelDesc(width=C, layers=L, modes=M, proj_width=C, output_scale=out_scale)
    blob = I.xavier_weights(desc_np, seed) * np.float32(wscale)
    # give the biases nonzero values so that every parameter is exercised
    off = I.weight_offsets(desc_np)
    rng = np.random.default_rng(seed + 77)
    for name in ["lift_b", "proj1_b", "proj2_b"] + [f"b{l}" for l in range(L)]:
        o, s = off[name]
        blob[o:o + s] = rng.uniform(-0.3, 0.3, s)
    wdev = to_dev(blob, dev)
    model = lib.Model(lib.make_desc(C, L, M, C, output_scale=out_scale), wdev)
    return desc_np, O.unpack_weights(blob, desc_np), model, wdev


# ------------------------------------------------------------------------------- stencil
@pytest.mark.parametrize("N,B", [(8, 3), (33, 2), (64, 2), (130, 1)])
def test_stencil_matches_oracle(lib, dev, N, B):
    import torch
    k, f = batch(N, B, 100 + N)
    op = lib.Operator(to_dev(k, dev))
    y = torch.empty_like(to_dev(f, dev))
    op.apply(to_dev(f, dev), y)
    torch.cuda.synchronize()
    for b in range(B):
        ref = O.apply_A(k[b], f[b])
        assert rel(y[b].cpu().numpy(), ref) < 1e-14
        elem_check(y[b].cpu().numpy(), ref, 1e-14, ("stencil", b))


@pytest.mark.parametrize("N,axis,j", [(64, 1, 3), (130, 0, 2), (33, 1, 1)])
def test_stencil_layered_coefficient_closed_form(lib, dev, N, axis, j):
    """The CUDA stencil against the flux-balance closed form of a layered coefficient (no
    oracle involved): harmonic-mean interior faces, boundary faces at k of the node, 1/h^2."""
    import torch
    import closed_forms as CF
    k, u, Au = CF.layered_flux_field(N, axis=axis, j=j, seed=N)
    op = lib.Operator(to_dev(k[None], dev))
    y = torch.empty((1, N, N), dtype=torch.float64, device=dev)
    op.apply(to_dev(u[None], dev), y)
    torch.cuda.synchronize()
    elem_check(y[0].cpu().numpy(), Au, 1e-12, "layered")


@pytest.mark.parametrize("N,B", [(20, 2), (130, 1)])
def test_residual_pair_matches_oracle(lib, dev, N, B):
    """fcgno_residual_pair (the random-residual training pairs): r = b - A u against the
    oracle's stencil element by element (1e-14 of max|r|), e = u_star - u exactly."""
    import torch
    k, f = batch(N, B, 9500 + N)
    rng = np.random.default_rng(N)
    u, us = rng.standard_normal((B, N, N)), rng.standard_normal((B, N, N))
    op = lib.Operator(to_dev(k, dev))
    r = torch.empty((B, N, N), dtype=torch.float64, device=dev)
    e = torch.empty_like(r)
    op.residual_pair(to_dev(f, dev), to_dev(u, dev), to_dev(us, dev), r, e)
    rs, es = r.cpu().numpy(), e.cpu().numpy()
    for b in range(B):
        elem_check(rs[b], f[b] - O.apply_A(k[b], u[b]), 1e-14, ("residual pair", b))
        assert np.array_equal(es[b], us[b] - u[b])


# ------------------------------------------------------------------------------- CG / FCG(B=I)
@pytest.mark.parametrize("N,B,m", [(33, 2, 1), (64, 3, 5), (100, 2, 1), (130, 1, 3)])
def test_identity_preconditioned_iterates_match_oracle(lib, dev, N, B, m):
    """Fused path (N <= 80) and tiled path (N > 80): 20 fixed iterations of Algorithm 1 with
    B = I, iterate compared with the oracle within max(1e-10, 10x the oracle's own rounding
    sensitivity)."""
    import torch
    k, f = batch(N, B, 200 + N)
    x0 = np.random.default_rng(N).standard_normal((B, N, N))
    op = lib.Operator(to_dev(k, dev))
    x = to_dev(x0, dev)
    info = lib.solve(op, None, to_dev(f, dev), x, m_max=m, max_iter=20, fixed_iters=True, prec="fp64")
    xs = x.cpu().numpy()
    for b in range(B):
        ref = O.fcg(lambda u: O.apply_A(k[b], u), lambda r: r, f[b], x0[b], m, 20)
        tol = rounding_tol(lambda d: O.fcg(lambda u: O.apply_A(k[b], u), lambda r: r, f[b], x0[b], m, 20,
                                           **({} if d is None else {"dot": d}))["u"])
        assert info[b]["iters"] == 20
        assert rel(xs[b], ref["u"]) < tol
        elem_check(xs[b], ref["u"], tol, ("iterate", b), "global")
        assert abs(info[b]["relres"] - ref["relres"][-1]) <= 1e-8 * ref["relres"][-1]


def test_identity_solve_to_tolerance_and_zero_rhs(lib, dev):
    """A zero right-hand side converges at iteration 0 while its batch-mates iterate on."""
    N, B = 48, 3
    k, f = batch(N, B, 300)
    f[1] = 0.0
    op = lib.Operator(to_dev(k, dev))
    x = to_dev(np.zeros((B, N, N)), dev)
    info = lib.solve(op, None, to_dev(f, dev), x, tol=1e-8, m_max=1, max_iter=3000, prec="fp64")
    assert info[1]["iters"] == 0 and info[1]["status"] == lib.FCGNO_OK
    xs = x.cpu().numpy()
    for b in (0, 2):
        ref = O.fcg(lambda u: O.apply_A(k[b], u), lambda r: r, f[b], np.zeros((N, N)), 1, 3000, tol=1e-8)
        assert info[b]["status"] == lib.FCGNO_OK
        # several hundred iterations: rounding order may move the stopping iteration by ~1%
        assert abs(info[b]["iters"] - ref["iterations"]) <= max(2, ref["iterations"] // 100)
        assert info[b]["relres"] <= 1e-8
        true_res = np.linalg.norm(f[b] - O.apply_A(k[b], xs[b])) / np.linalg.norm(f[b])
        assert true_res <= 1e-7


# ------------------------------------------------------------------------------- preconditioner
@pytest.mark.parametrize("N,C,M,B,out_scale", [(32, 16, 8, 2, 0), (20, 8, 5, 3, 0), (64, 32, 12, 2, 0),
                                               (32, 16, 8, 2, 1), (20, 8, 5, 2, 1)])
def test_fp64_preconditioner_matches_oracle(lib, dev, N, C, M, B, out_scale):
    import torch
    k, r = batch(N, B, 400 + N, 2.0 if out_scale else 1.0)
    desc, P, model, _w = model_pair(lib, dev, C, M, out_scale=out_scale)
    op = lib.Operator(to_dev(k, dev))
    z = torch.empty((B, N, N), dtype=torch.float64, device=dev)
    lib.precond_apply(model, op, to_dev(r, dev), z, prec="fp64")
    zs = z.cpu().numpy()
    for b in range(B):
        ref = O.no_forward(P, desc, r[b], np.log(k[b]))
        assert rel(zs[b], ref) < 1e-12
        elem_check(zs[b], ref, ELEM_TOL["fp64"], ("fp64 NO", b))


@pytest.mark.parametrize("N,C,M,B", [(32, 16, 8, 2), (64, 32, 12, 2)])
def test_fp32_preconditioner_matches_oracle(lib, dev, N, C, M, B):
    import torch
    k, r = batch(N, B, 500 + N)
    desc, P, model, _w = model_pair(lib, dev, C, M)
    op = lib.Operator(to_dev(k, dev))
    z = torch.empty((B, N, N), dtype=torch.float64, device=dev)
    lib.precond_apply(model, op, to_dev(r, dev), z, prec="fp32")
    zs = z.cpu().numpy()
    for b in range(B):
        ref = O.no_forward(P, desc, r[b], np.log(k[b]))
        assert rel(zs[b], ref) < 2e-5
        elem_check(zs[b], ref, ELEM_TOL["fp32"], ("fp32 NO", b))


def test_fcg_no_fp64_thirty_iterations_match_oracle(lib, dev):
    """Plain FCG-NO parity workload: N = 32, one instance, k = exp(GRF(0.1, 1)), f ~ N(0,1),
    x0 = 0, NO width 16, 4 layers, 8 modes, Xavier seed 0, m = 1; 30 fixed iterations,
    iterate within 1e-10 of the oracle; then an identity-preconditioned solve to 1e-8."""
    import torch
    N = 32
    k, f = I.make_problem(N, 1000)
    k, f = k[None], f[None]
    desc = I.ModelDesc(width=16, layers=4, modes=8, proj_width=16)
    blob = I.xavier_weights(desc, 0)
    P = O.unpack_weights(blob, desc)
    wdev = to_dev(blob, dev)
    model = lib.Model(lib.make_desc(16, 4, 8, 16), wdev)
    op = lib.Operator(to_dev(k, dev))
    x = torch.zeros((1, N, N), dtype=torch.float64, device=dev)
    info = lib.solve(op, model, to_dev(f, dev), x, m_max=1, max_iter=30, fixed_iters=True, prec="fp64")
    ref = O.fcg(lambda u: O.apply_A(k[0], u), lambda r: O.no_forward(P, desc, r, np.log(k[0])), f[0],
                np.zeros((N, N)), 1, 30)
    assert info[0]["iters"] == 30
    assert rel(x[0].cpu().numpy(), ref["u"]) < 1e-10
    elem_check(x[0].cpu().numpy(), ref["u"], 1e-10, "30 iterations", "global")
    x.zero_()
    info = lib.solve(op, None, to_dev(f, dev), x, tol=1e-8, m_max=1, max_iter=5000, prec="fp64")
    ref = O.fcg(lambda u: O.apply_A(k[0], u), lambda r: r, f[0], np.zeros((N, N)), 1, 5000, tol=1e-8)
    assert info[0]["status"] == lib.FCGNO_OK
    assert abs(info[0]["iters"] - ref["iterations"]) <= max(2, ref["iterations"] // 100)
    assert rel(x[0].cpu().numpy(), ref["u"]) < 1e-7


@pytest.mark.parametrize("N,m", [(40, 5), (96, 2)])
def test_fcg_no_fp64_window_matches_oracle(lib, dev, N, m):
    """Truncation window m > 1 on the fused (N = 40) and tiled (N = 96) paths."""
    import torch
    B = 2
    k, f = batch(N, B, 600 + N)
    desc, P, model, _w = model_pair(lib, dev, 8, 4, L=2, seed=5)
    op = lib.Operator(to_dev(k, dev))
    x = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
    lib.solve(op, model, to_dev(f, dev), x, m_max=m, max_iter=12, fixed_iters=True, prec="fp64")
    xs = x.cpu().numpy()
    for b in range(B):
        ref = O.fcg(lambda u: O.apply_A(k[b], u), lambda r: O.no_forward(P, desc, r, np.log(k[b])), f[b],
                    np.zeros((N, N)), m, 12)
        assert rel(xs[b], ref["u"]) < 1e-10
        elem_check(xs[b], ref["u"], 1e-10, ("window", b), "global")


def test_solve_host_matches_device_solve(lib, dev):
    import torch
    N, B = 24, 2
    k, f = batch(N, B, 700)
    x_host = np.zeros((B, N, N))
    info_h = lib.solve_host(k, f, x_host, None, tol=1e-9, m_max=1, max_iter=2000, prec="fp64")
    op = lib.Operator(to_dev(k, dev))
    x = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
    info_d = lib.solve(op, None, to_dev(f, dev), x, tol=1e-9, m_max=1, max_iter=2000, prec="fp64")
    assert [i["iters"] for i in info_h] == [i["iters"] for i in info_d]
    assert np.array_equal(x_host, x.cpu().numpy())


def test_solve_host_reuses_its_device_state_across_problems(lib, dev):
    """fcgno_solve_host keeps the device buffers and the operator of a shape between calls:
    a second call with different k, f and u_0 of the same shape (re-assembled in place, same
    captured graphs), a call of another shape in between, and a call after releasing the state
    each equal a device solve of their own problem, bit for bit."""
    import torch
    desc, P, model, _w = model_pair(lib, dev, 32, 12, out_scale=1)

    def both(N, B, seed):
        k, f = batch(N, B, seed)
        x0 = np.random.default_rng(seed).standard_normal((B, N, N))
        xh = x0.copy()
        ih = lib.solve_host(k, f, xh, model, tol=1e-6, m_max=5, max_iter=60, prec="bf16")
        op = lib.Operator(to_dev(k, dev))
        x = to_dev(x0, dev)
        idv = lib.solve(op, model, to_dev(f, dev), x, tol=1e-6, m_max=5, max_iter=60, prec="bf16")
        assert [i["iters"] for i in ih] == [i["iters"] for i in idv]
        assert np.array_equal(xh, x.cpu().numpy())

    both(64, 3, 710)
    both(64, 3, 720)   # same shape, new problem: cached state re-assembled
    both(32, 2, 730)   # another shape
    both(64, 3, 740)
    lib.solve_host_release()
    both(64, 3, 750)


def test_krylov_harvest_matches_oracle_cg(lib, dev):
    """Eq. (9): residuals r_i and errors e_i = u* - u_i of CG from u_0 ~ N(0, 1)."""
    import torch
    N, B, K = 16, 2, 6
    k, f = batch(N, B, 800)
    x0 = np.random.default_rng(3).standard_normal((B, N, N))
    ustar = np.stack([np.linalg.solve(O.dense_A(k[b]), f[b].ravel()).reshape(N, N) for b in range(B)])
    op = lib.Operator(to_dev(k, dev))
    r_out = torch.empty((K, B, N, N), dtype=torch.float64, device=dev)
    e_out = torch.empty_like(r_out)
    lib.krylov_harvest(op, to_dev(f, dev), to_dev(x0, dev), to_dev(ustar, dev), K, r_out, e_out)
    rs, es = r_out.cpu().numpy(), e_out.cpu().numpy()
    for b in range(B):
        ref = O.fcg(lambda u: O.apply_A(k[b], u), lambda r: r, f[b], x0[b], 1, K, record=True)
        for i in range(K):
            assert rel(rs[i, b], ref["rs"][i + 1]) < 1e-11
            assert rel(es[i, b], ustar[b] - ref["us"][i + 1]) < 1e-11
            elem_check(rs[i, b], ref["rs"][i + 1], 1e-11, ("harvest r", i, b))
            elem_check(es[i, b], ustar[b] - ref["us"][i + 1], 1e-11, ("harvest e", i, b))


# ------------------------------------------------------------------------------- tensor cores
@pytest.mark.parametrize("N,C,M,B,prec,tol,sigma,wscale", [
    (32, 16, 8, 2, "bf16", 2e-2, 1.0, 1.0),
    (64, 32, 12, 3, "bf16", 2e-2, 1.0, 1.0),
    (64, 32, 12, 2, "fp16", 4e-3, 1.0, 1.0),
    (128, 32, 12, 2, "bf16", 2e-2, 1.0, 1.0),
    (64, 32, 16, 2, "bf16", 2e-2, 1.0, 1.0),
    (64, 32, 12, 2, "bf16", 2e-2, 2.0, 1.0),   # the high-contrast coefficient family
    (32, 16, 8, 2, "bf16", 2e-2, 2.0, 2.5),    # and weights far into the GELUs' nonlinear range
    (256, 32, 12, 1, "bf16", 2e-2, 0.5, 2.5),
    (64, 32, 12, 2, "bf16", 2e-2, 2.0, -1.0),  # output scaled by 1/k (wscale < 0 marks output_scale 1)
    (128, 32, 12, 2, "fp16", 4e-3, 1.0, -1.0),
])
def test_tensor_core_preconditioner_matches_oracle(lib, dev, N, C, M, B, prec, tol, sigma, wscale):
    """tcgen05 BF16/FP16 preconditioner (FP32 accumulation) against the FP64 oracle:
    relative 2-norm error per instance within 2e-2 (BF16) / 4e-3 (FP16), and element by
    element (including each grid edge) within ELEM_TOL of max|z|."""
    import torch
    k, r = batch(N, B, 900 + N + M, sigma)
    desc, P, model, _w = model_pair(lib, dev, C, M, wscale=abs(wscale), out_scale=int(wscale < 0))
    op = lib.Operator(to_dev(k, dev))
    z = torch.empty((B, N, N), dtype=torch.float64, device=dev)
    lib.precond_apply(model, op, to_dev(r, dev), z, prec=prec)
    zs = z.cpu().numpy()
    for b in range(B):
        ref = O.no_forward(P, desc, r[b], np.log(k[b]))
        if desc.output_scale:
            # the 16-bit arithmetic produces the network output; the pointwise factor 1/k is
            # applied after it in FP64. The bounds hold for the network output (z k); z itself
            # weights each point's error by 1/k, which at sigma 2 concentrates the norm on the
            # few points of smallest k, so its norm-wise error is bounded at 2.5x the tolerance
            assert rel(zs[b], ref) < 2.5 * tol, (b, rel(zs[b], ref))
            zs_b, ref = zs[b] * k[b], ref * k[b]
        else:
            zs_b = zs[b]
        err = rel(zs_b, ref)
        assert err < tol, (b, err)
        elem_check(zs_b, ref, ELEM_TOL[prec], (prec, b))


@pytest.mark.parametrize("N,C,M,B,sample", [
    (64, 32, 12, 256, range(0, 256, 37)),   # the benchmark's launch configuration
    (32, 16, 8, 130, (0, 64, 127, 128, 129)),  # crosses the 128-instance block of the mode mixing
    (1024, 32, 16, 1, (0,)),                # the large-solve grid and mode count
])
def test_tensor_core_preconditioner_full_size_sampled(lib, dev, N, C, M, B, sample):
    """The BF16 tensor-core preconditioner at full launch sizes: every kernel runs on the
    whole batch, and sampled instances are compared with the FP64 oracle (2e-2 relative);
    the rest must be finite and zero exactly where r is."""
    import torch
    k, r = batch(N, B, 5000 + N)
    r[B - 1] = 0.0 if B > 1 else r[B - 1]
    desc, P, model, _w = model_pair(lib, dev, C, M)
    op = lib.Operator(to_dev(k, dev))
    z = torch.empty((B, N, N), dtype=torch.float64, device=dev)
    lib.precond_apply(model, op, to_dev(r, dev), z, prec="bf16")
    zs = z.cpu().numpy()
    assert np.all(np.isfinite(zs))
    if B > 1:
        assert not np.any(zs[B - 1])
    for b in sample:
        if b == B - 1 and B > 1:
            continue
        ref = O.no_forward(P, desc, r[b], np.log(k[b]))
        err = rel(zs[b], ref)
        assert err < 2e-2, (b, err)
        elem_check(zs[b], ref, ELEM_TOL["bf16"], ("bf16 full size", b))


def test_tensor_core_preconditioner_inside_solve(lib, dev):
    """Algorithm 1 with the BF16 preconditioner: every iterate keeps the exact line-search
    property (monotone energy error), and instances that stop leave their batch-mates intact."""
    import torch
    N, B = 64, 3
    k, f = batch(N, B, 1200)
    f[2] = 0.0
    desc, P, model, _w = model_pair(lib, dev, 32, 12)
    op = lib.Operator(to_dev(k, dev))
    x = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
    info = lib.solve(op, model, to_dev(f, dev), x, m_max=1, max_iter=15, fixed_iters=True, prec="bf16")
    assert info[2]["iters"] == 0
    for b in range(2):
        assert info[b]["iters"] == 15 and np.isfinite(info[b]["relres"])
        ustar = O.fcg(lambda u: O.apply_A(k[b], u), lambda r: r, f[b], np.zeros((N, N)), 1, 4000, tol=1e-12)["u"]
        e15 = O.energy_norm(k[b], ustar - x[b].cpu().numpy())
        e0 = O.energy_norm(k[b], ustar)
        assert e15 <= e0


# ------------------------------------------------------------------------------- training step
@pytest.mark.parametrize("prec,tol,out_scale", [("fp64", 1e-6, 0), ("fp32", 2e-4, 0), ("fp64", 1e-6, 1),
                                               ("fp32", 2e-4, 1)])
def test_train_step_matches_oracle_gradient(lib, dev, prec, tol, out_scale):
    """Energy-norm loss (Eq. (11)) and its gradient w.r.t. the whole weight blob, from the
    hand-written CUDA backward, against the oracle's reverse mode (itself pinned by finite
    differences), for both output scales. Relative 2-norm error of the gradient: 1e-6 (FP64
    arithmetic, FP32 output), 2e-4 (FP32)."""
    check_train_step(lib, dev, prec, tol, "energy", out_scale)


@pytest.mark.parametrize("kind,out_scale", [("energy", 0), ("energy", 1), ("l2", 0)])
def test_fp64_output_train_step_matches_oracle_gradient_to_1e8(lib, dev, kind, out_scale):
    """fcgno_train_step_f64 (FP64 arithmetic, loss and gradient stored in FP64) against the
    oracle's reverse mode: loss within 1e-12 relative, the whole gradient within 1e-8 relative
    (2-norm), and every parameter group element by element within 1e-8 of its largest entry.
    Both sides are FP64 throughout and differ only in summation order."""
    import torch
    N, B, C, M = 32, 3, 16, 8
    k, f = batch(N, B, 1300)
    es = np.stack([np.linalg.solve(O.dense_A(k[b]), f[b].ravel()).reshape(N, N) for b in range(B)])
    desc, P, model, wdev = model_pair(lib, dev, C, M, L=4, seed=2, out_scale=out_scale)
    op = lib.Operator(to_dev(k, dev))
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.full((wdev.numel(),), float("nan"), dtype=torch.float64, device=dev)
    lib.train_step_f64(model, op, to_dev(f, dev), to_dev(es, dev), loss, grad, loss_kind=kind)
    ref = O.notay_loss_and_grad if kind == "energy" else O.l2_loss_and_grad
    L_ref, g_ref = ref(P, desc, list(k), list(f), list(es))
    assert abs(float(loss.item()) - L_ref) <= 1e-12 * L_ref
    g = grad.cpu().numpy()
    assert rel(g, g_ref) < 1e-8, rel(g, g_ref)
    off = I.weight_offsets(desc)
    for name, (o, s_) in off.items():
        if name != "_total":
            gg, rr = g[o:o + s_], g_ref[o:o + s_]
            assert np.max(np.abs(gg - rr)) <= 1e-8 * np.max(np.abs(rr)), name


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("fp32", 2e-4)])
def test_l2_train_step_matches_oracle_gradient(lib, dev, prec, tol):
    """The L2 ablation loss (2-norm in error form) and its gradient against the oracle's
    reverse mode (pinned by finite differences), same tolerances as Eq. (11)."""
    check_train_step(lib, dev, prec, tol, "l2")


def check_train_step(lib, dev, prec, tol, kind, out_scale=0):
    import torch
    N, B, C, M = 32, 3, 16, 8
    k, f = batch(N, B, 1300)
    es = np.stack([np.linalg.solve(O.dense_A(k[b]), f[b].ravel()).reshape(N, N) for b in range(B)])
    desc, P, model, wdev = model_pair(lib, dev, C, M, L=4, seed=2, out_scale=out_scale)
    op = lib.Operator(to_dev(k, dev))
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    grad = torch.zeros(wdev.numel(), dtype=torch.float32, device=dev)
    lib.train_step(model, op, to_dev(f, dev), to_dev(es, dev), loss, grad, prec=prec, loss_kind=kind)
    ref = O.notay_loss_and_grad if kind == "energy" else O.l2_loss_and_grad
    L_ref, g_ref = ref(P, desc, list(k), list(f), list(es))
    assert abs(float(loss.item()) - L_ref) <= max(tol, 1e-6) * L_ref
    g = grad.double().cpu().numpy()
    assert rel(g, g_ref) < tol
    # every parameter group is exercised
    off = I.weight_offsets(desc)
    for name, (o, s) in off.items():
        if name != "_total":
            assert rel(g[o:o + s], g_ref[o:o + s]) < max(tol * 10, 1e-7), name


# BF16 training step (Fourier layers forward and backward on the tensor cores, FP32
# accumulation, FP32 master weights). Every activation, pre-activation and gradient image is
# rounded to 8 significant bits (u = 2^-9) between layers, so the gradient carries a few times
# 4u of relative error, like the 16-bit preconditioner's output. Bounds (loss, gradient 2-norm,
# worst parameter group in 2-norm and in max|g - g_ref| / max|g_ref|): twice the largest error
# measured over these cases.
BF16_TRAIN_TOL = {"energy": (1e-2, 2e-2, 5e-2, 5e-2), "l2": (1e-2, 3e-2, 8e-2, 1e-1)}


@pytest.fixture(scope="module")
def trained_pair(lib, dev):
    """A preconditioner trained briefly (600 BF16 steps on Krylov vectors of 64 x 64 problems,
    sigma in {0.5, 1, 2}): weights no longer Xavier, GELUs away from their linear range. Returns
    (desc, oracle weights, model, blob); the oracle weights are the trained blob's."""
    from paper_2402_05598_gb300 import train as T
    desc, _P, model, wdev = model_pair(lib, dev, 32, 12, seed=11, out_scale=1)
    T.train(model, 64, range(0, 96), K=40, batch=32, lr=1e-3, steps=600, prec="bf16", sigma=(0.5, 1.0, 2.0))
    return desc, O.unpack_weights(wdev.double().cpu().numpy(), desc), model, wdev


@pytest.mark.parametrize("prec,tol", [("bf16", 2e-2), ("fp16", 4e-3), ("fp64", 1e-12)])
@pytest.mark.parametrize("sigma", [0.5, 2.0])
def test_trained_preconditioner_matches_oracle(lib, dev, trained_pair, prec, tol, sigma):
    """The preconditioner with trained weights on held-out fields of low and high contrast,
    against the oracle with the same weights: relative 2-norm error of the network output
    (z k, output_scale 1) within 2e-2 (BF16), 4e-3 (FP16), 1e-12 (FP64), and element by element
    (every grid edge included) within ELEM_TOL of max|z k|. The residuals are those a solve
    sees: r = f - A u for a random u."""
    import torch
    desc, P, model, _w = trained_pair
    N, B = 64, 3
    k, f = batch(N, B, 4400 + int(10 * sigma), sigma)
    u = np.random.default_rng(5).standard_normal((B, N, N))
    r = np.stack([f[b] - O.apply_A(k[b], u[b]) for b in range(B)])
    op = lib.Operator(to_dev(k, dev))
    z = torch.empty((B, N, N), dtype=torch.float64, device=dev)
    lib.precond_apply(model, op, to_dev(r, dev), z, prec=prec)
    zs = z.cpu().numpy()
    for b in range(B):
        ref = O.no_forward(P, desc, r[b], np.log(k[b])) * k[b]
        zk = zs[b] * k[b]
        assert rel(zk, ref) < tol, (b, rel(zk, ref))
        elem_check(zk, ref, ELEM_TOL[prec], ("trained " + prec, sigma, b))


@pytest.mark.parametrize("N,B,C,M,seed,out_scale,kind", [
    (32, 3, 16, 8, 2, 0, "energy"),
    (32, 3, 16, 8, 2, 1, "energy"),
    (32, 3, 16, 8, 2, 0, "l2"),
    (64, 2, 32, 12, 4, 1, "energy"),   # the training configuration's width and modes
    (128, 1, 32, 12, 5, 1, "energy"),  # tiles of one grid column (N >= 128)
])
def test_bf16_train_step_matches_oracle_gradient(lib, dev, N, B, C, M, seed, out_scale, kind):
    """fcgno_train_step with FCGNO_BF16 against the oracle's reverse mode (pinned by finite
    differences): loss, whole gradient and every parameter group element-wise; a second call
    returns the identical loss and gradient (no order-dependent reduction)."""
    import torch
    k, f = batch(N, B, 1300 + N)
    if N <= 32:
        es = np.stack([np.linalg.solve(O.dense_A(k[b]), f[b].ravel()).reshape(N, N) for b in range(B)])
    else:
        es = np.stack([O.fcg(lambda u, b=b: O.apply_A(k[b], u), lambda r: r, f[b], np.zeros((N, N)), 1, 20 * N * N,
                             tol=1e-13)["u"] for b in range(B)])
    desc, P, model, wdev = model_pair(lib, dev, C, M, L=4, seed=seed, out_scale=out_scale)
    op = lib.Operator(to_dev(k, dev))
    ref = O.notay_loss_and_grad if kind == "energy" else O.l2_loss_and_grad
    L_ref, g_ref = ref(P, desc, list(k), list(f), list(es))
    tl, tg, tgrp, tmax = BF16_TRAIN_TOL[kind]
    runs = []
    for _ in range(2):
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        grad = torch.full((wdev.numel(),), float("nan"), dtype=torch.float32, device=dev)
        lib.train_step(model, op, to_dev(f, dev), to_dev(es, dev), loss, grad, prec="bf16", loss_kind=kind)
        runs.append((loss.clone(), grad.clone()))
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
    loss, grad = runs[0]
    assert abs(float(loss.item()) - L_ref) <= tl * L_ref
    g = grad.double().cpu().numpy()
    assert np.all(np.isfinite(g))
    assert rel(g, g_ref) < tg
    off = I.weight_offsets(desc)
    for name, (o, s) in off.items():
        if name == "_total":
            continue
        gg, rr = g[o:o + s], g_ref[o:o + s]
        assert rel(gg, rr) < tgrp, name
        assert np.max(np.abs(gg - rr)) <= tmax * np.max(np.abs(rr)), name


def test_bf16_training_interleaves_with_solves(lib, dev):
    """A BF16 training step between two BF16 preconditioner applications: the step refreshes
    the weight images from the master blob, so after an in-place weight change the
    preconditioner follows the new weights (as after fcgno_model_sync), and an FP16 training
    step is rejected before any launch."""
    import torch
    N, B = 32, 2
    k, f = batch(N, B, 1320)
    desc, P, model, wdev = model_pair(lib, dev, 16, 8, L=4, seed=6)
    op = lib.Operator(to_dev(k, dev))
    r = to_dev(f, dev)
    z0 = torch.empty((B, N, N), dtype=torch.float64, device=dev)
    lib.precond_apply(model, op, r, z0, prec="bf16")
    wdev.mul_(0.5)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    grad = torch.zeros(wdev.numel(), dtype=torch.float32, device=dev)
    lib.train_step(model, op, r, r, loss, grad, prec="bf16")
    z1 = torch.empty_like(z0)
    lib.precond_apply(model, op, r, z1, prec="bf16")
    P2 = O.unpack_weights(wdev.double().cpu().numpy(), desc)
    for b in range(B):
        ref = O.no_forward(P2, desc, f[b], np.log(k[b]))
        assert rel(z1[b].cpu().numpy(), ref) < 2e-2
        elem_check(z1[b].cpu().numpy(), ref, ELEM_TOL["bf16"], ("after bf16 step", b))
    with pytest.raises(RuntimeError):
        lib.train_step(model, op, r, r, loss, grad, prec="fp16")


@pytest.mark.parametrize("kind", ["energy", "l2"])
def test_autograd_loss_gives_the_library_gradient(lib, dev, kind):
    """The training loss as a torch.autograd.Function: loss.backward() leaves exactly the
    hand-written gradient of fcgno_train_step in weights.grad (scaled by the upstream
    gradient), and the forward value is the library's loss."""
    import torch
    from paper_2402_05598_gb300 import train as T
    N, B, C, M = 32, 3, 16, 8
    k, f = batch(N, B, 1300)
    es = np.stack([np.linalg.solve(O.dense_A(k[b]), f[b].ravel()).reshape(N, N) for b in range(B)])
    desc, P, model, wdev = model_pair(lib, dev, C, M, L=4, seed=2)
    op = lib.Operator(to_dev(k, dev))
    r, e = to_dev(f, dev), to_dev(es, dev)
    loss0 = torch.zeros(1, dtype=torch.float32, device=dev)
    grad0 = torch.zeros(wdev.numel(), dtype=torch.float32, device=dev)
    lib.train_step(model, op, r, e, loss0, grad0, prec="fp32", loss_kind=kind)
    wdev.requires_grad_(True)
    loss = T.preconditioner_loss(model, op, r, e, prec="fp32", loss_kind=kind)
    (2.5 * loss).backward()
    assert loss.item() == loss0.item()
    assert torch.equal(wdev.grad, 2.5 * grad0)
    wdev.requires_grad_(False)


@pytest.mark.parametrize("prec,kind", [("fp32", "energy"), ("fp64", "energy"), ("fp32", "l2"), ("bf16", "energy"),
                                       ("bf16", "l2")])
def test_training_with_recomputed_preactivations_is_bit_identical(lib, dev, prec, kind):
    """Activation checkpointing: a training step that rebuilds every layer's pre-activation
    in the backward returns exactly the loss and gradient of the step that keeps them."""
    import torch
    N, B, C, M = 32, 3, 16, 8
    k, f = batch(N, B, 1350)
    es = np.stack([np.linalg.solve(O.dense_A(k[b]), f[b].ravel()).reshape(N, N) for b in range(B)])
    desc, P, model, wdev = model_pair(lib, dev, C, M, L=4, seed=3)
    op = lib.Operator(to_dev(k, dev))
    out = {}
    for mode in ("never", "always"):
        model.set_train_recompute(mode)
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        grad = torch.zeros(wdev.numel(), dtype=torch.float32, device=dev)
        lib.train_step(model, op, to_dev(f, dev), to_dev(es, dev), loss, grad, prec=prec, loss_kind=kind)
        out[mode] = (loss.clone(), grad.clone())
    assert torch.equal(out["never"][0], out["always"][0])
    assert torch.equal(out["never"][1], out["always"][1])


@pytest.mark.parametrize("N,B,steps,m", [(32, 2, 4, 1), (100, 2, 3, 2)])
def test_jacobi_preconditioned_iterates_match_oracle(lib, dev, N, B, steps, m):
    """Algorithm 1 with the Jacobi(k) preconditioner of Eq. (15), fused (N <= 80) and tiled
    paths: 15 fixed iterations against the oracle within its rounding sensitivity."""
    k, f = batch(N, B, 1400 + N)
    x0 = np.random.default_rng(7).standard_normal((B, N, N))
    op = lib.Operator(to_dev(k, dev))
    x = to_dev(x0, dev)
    info = lib.solve_jacobi(op, steps, to_dev(f, dev), x, m_max=m, max_iter=15, fixed_iters=True)
    xs = x.cpu().numpy()
    for b in range(B):
        run = lambda d: O.fcg(lambda u: O.apply_A(k[b], u), lambda r: O.jacobi_precond(k[b], r, steps), f[b], x0[b],
                              m, 15, **({} if d is None else {"dot": d}))["u"]
        assert info[b]["iters"] == 15
        assert rel(xs[b], run(None)) < rounding_tol(run)


def test_workspace_bytes_counts_what_a_solve_allocates(lib, dev):
    """fcgno_workspace_bytes (the figure serving admits against) against the device memory a
    first BF16 solve actually takes (operator, Krylov workspace, 16-bit activations): not
    below it, and above it by no more than allocation rounding and the model's per-grid
    tables and weight images (96 MiB). At 512 x 512 x 32 one FP64 vector is 64 MiB, so
    leaving out even one buffer of the workspace would fail the test."""
    import torch
    N, B, m = 512, 32, 5
    k, f = batch(N, B, 9100)
    kd, fd = to_dev(k, dev), to_dev(f, dev)
    x = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
    desc, P, model, _w = model_pair(lib, dev, 32, 12)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    op = lib.Operator(kd)
    lib.solve(op, model, fd, x, m_max=m, max_iter=1, fixed_iters=True, prec="bf16")
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    predicted = lib.workspace_bytes(N, B, m, lib.make_desc(32, 4, 12, 32), "bf16")
    assert predicted - (1 << 20) <= used <= predicted + (96 << 20), (used, predicted)
    op.close()


def test_stopped_instances_do_not_change_the_others(lib, dev):
    """200 instances at 64 x 64 in the wide launch shape, where the analysis runs as persistent
    blocks that walk two instances each: with every third instance stopped at iteration 0 (zero
    right-hand side, so the kernels skip it), every other instance's iterate after 6 BF16
    FCG-NO iterations is bit-identical to the run in which all 200 are active. Every step works
    per instance (the mode mixing per row of its 128-instance tile), so the batch around an
    instance must not change it."""
    import torch
    N, B = 64, 200
    k, f = batch(N, B, 4700)
    desc, P, model, _w = model_pair(lib, dev, 32, 12, out_scale=1)
    op = lib.Operator(to_dev(k, dev))
    fa = to_dev(f, dev)
    fz = fa.clone()
    fz[::3] = 0.0
    lib.set_launch_shape("wide")
    try:
        xa = torch.zeros_like(fa)
        lib.solve(op, model, fa, xa, m_max=5, max_iter=6, fixed_iters=True, prec="bf16")
        xz = torch.zeros_like(fa)
        info = lib.solve(op, model, fz, xz, m_max=5, max_iter=6, fixed_iters=True, prec="bf16")
    finally:
        lib.set_launch_shape("auto")
    keep = [b for b in range(B) if b % 3 != 0]
    assert all(info[b]["iters"] == 0 for b in range(0, B, 3))
    assert all(info[b]["iters"] == 6 for b in keep)
    assert torch.equal(xz[keep], xa[keep])


@pytest.mark.parametrize("N,C,M", [(64, 32, 12), (32, 16, 8), (100, 16, 8)])
def test_narrow_launch_shapes_match_the_wide_ones(lib, dev, N, C, M):
    """Once few instances are still running, replayed iterations switch to the narrow launch
    shapes: the FCG step splits each instance over a cluster of CTAs (16-row bands, halo rows
    and partial sums through distributed shared memory) and the 16-bit synthesis uses
    narrower grid-column chunks. With 3 instances every replay is narrow; the same solve run
    iteration by iteration runs the wide shapes. FP64 preconditioner: the two iterates agree
    within 10x the oracle's own rounding sensitivity (only the summation order differs; the
    nonlinear preconditioner amplifies it over the iterations). BF16: in both shapes the
    recursively updated residual equals the true residual b - A x of the returned iterate
    and the energy error has not grown (exact line search), for these untrained weights."""
    import torch
    B, iters = 3, 17
    k, f = batch(N, B, 9400 + N)
    desc, P, model, _w = model_pair(lib, dev, C, M, out_scale=1)
    op = lib.Operator(to_dev(k, dev))
    xs = {}
    for check in (1, 8):  # 1: no replay (wide shapes); 8: replayed graphs, narrow with 3 running instances
        x = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
        info = lib.solve(op, model, to_dev(f, dev), x, m_max=5, max_iter=iters, fixed_iters=True, prec="fp64",
                         check_every=check)
        assert all(i["iters"] == iters for i in info)
        xs[check] = x.cpu().numpy()
    for b in range(B):
        run = lambda d: O.fcg(lambda u: O.apply_A(k[b], u), lambda r: O.no_forward(P, desc, r, np.log(k[b])), f[b],
                              np.zeros((N, N)), 5, iters, **({} if d is None else {"dot": d}))["u"]
        tol = rounding_tol(run)
        elem_check(xs[8][b], xs[1][b], tol, ("narrow fp64", b), "global")
    if not lib.precision_supported(N, lib.make_desc(C, 4, M, C), "bf16"):
        return
    for check in (1, 8):
        x = torch.zeros((B, N, N), dtype=torch.float64, device=dev)
        info = lib.solve(op, model, to_dev(f, dev), x, m_max=5, max_iter=24, fixed_iters=True, prec="bf16",
                         check_every=check)
        xh = x.cpu().numpy()
        for b in range(B):
            r0 = np.linalg.norm(f[b])
            true = np.linalg.norm(f[b] - O.apply_A(k[b], xh[b])) / r0
            assert abs(true - info[b]["relres"]) <= 1e-9, (check, b, true, info[b]["relres"])
            ustar = np.linalg.solve(O.dense_A(k[b]), f[b].ravel()).reshape(N, N) if N <= 32 else None
            if ustar is not None:
                assert O.energy_norm(k[b], ustar - xh[b]) <= O.energy_norm(k[b], ustar)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["bf16", None])
def test_host_check_cadence_does_not_change_the_solve(lib, dev, trained_pair, prec):
    """Each instance stops on the device at its own convergence (Algorithm 1's test on
    ||r_i||), so how often the host reads the convergence counter changes neither an iterate
    nor an iteration count. Checked with the launch shape held wide: iteration by iteration
    (check_every 1, no graph), and replayed 8- or 16-iteration graphs that drop to
    2-iteration replays once 32 or fewer of the 48 instances run. BF16 FCG-NO at 64 x 64 with
    the briefly trained preconditioner (m = 5, tol 1e-6, cap 400: some instances converge, the
    others stop at the cap) and plain CG at 32 x 32 (tol 1e-8, 198 to 512 iterations in the
    oracle): bit-identical iterates and the same per-instance iteration counts and statuses."""
    import torch
    N, B = (64, 48) if prec else (32, 48)
    k, f = batch(N, B, 5100 + N)
    model = trained_pair[2] if prec else None
    op = lib.Operator(to_dev(k, dev))
    fd = to_dev(f, dev)
    tol = 1e-6 if prec else 1e-8
    out = {}
    lib.set_launch_shape("wide")
    try:
        for check in (1, 8, 16):
            x = torch.zeros_like(fd)
            info = lib.solve(op, model, fd, x, tol=tol, m_max=5 if prec else 1, max_iter=400 if prec else 2000,
                             prec=prec or "fp64", check_every=check)
            out[check] = (x.cpu(), [(i["iters"], i["status"]) for i in info])
    finally:
        lib.set_launch_shape("auto")
    its = [t[0] for t in out[1][1]]
    if not prec:
        assert all(t[1] == lib.FCGNO_OK for t in out[1][1]), out[1][1]
    assert sum(t[1] == lib.FCGNO_OK for t in out[1][1]) >= 8, out[1][1]
    assert max(its) > min(its), its  # the instances stop at different iterations
    for check in (8, 16):
        assert out[check][1] == out[1][1], check
        assert torch.equal(out[check][0], out[1][0]), check


@pytest.mark.parametrize("N,C,M,B,prec", [(64, 32, 12, 5, "bf16"), (32, 16, 8, 130, "bf16"), (64, 32, 12, 3, "fp16")])
def test_narrow_shape_preconditioner_matches_oracle(lib, dev, N, C, M, B, prec):
    """The narrow launch shape (fcgno_set_launch_shape forces it) runs the 16-bit analysis in
    16-column chunks (the mixing sums twice as many 16-bit partial coefficients) and the
    synthesis in 8-column chunks. Its output meets the same bounds against the FP64 oracle as
    the wide shape's (2-norm and element-wise, on the network output z k), and the two shapes
    agree within that 16-bit tolerance."""
    import torch
    k, r = batch(N, B, 9600 + N)
    desc, P, model, _w = model_pair(lib, dev, C, M, out_scale=1)
    op = lib.Operator(to_dev(k, dev))
    z = {}
    try:
        for mode in ("wide", "narrow"):
            lib.set_launch_shape(mode)
            zz = torch.empty((B, N, N), dtype=torch.float64, device=dev)
            lib.precond_apply(model, op, to_dev(r, dev), zz, prec=prec)
            z[mode] = zz.cpu().numpy()
    finally:
        lib.set_launch_shape("auto")
    tol = 2e-2 if prec == "bf16" else 4e-3
    for b in sorted({0, B // 2, B - 1}):
        ref = O.no_forward(P, desc, r[b], np.log(k[b])) * k[b]
        for mode in ("wide", "narrow"):
            assert rel(z[mode][b] * k[b], ref) < tol, (mode, b)
            elem_check(z[mode][b] * k[b], ref, ELEM_TOL[prec], (mode, b))
        assert rel(z["narrow"][b] * k[b], z["wide"][b] * k[b]) < tol
