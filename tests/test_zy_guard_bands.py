"""Guard bands around output buffers (out-of-bounds writes; compute-sanitizer is not available
for this). Every output a call writes sits inside a larger buffer whose 512 bytes before and
after it hold a sentinel value; after the call, and a synchronisation, the bands must be
intact. Sizes are ragged or tile-edge cases, so a kernel that rounds its last tile up and
writes past the end would be caught even where the parity tests cannot see it (a write past
the last instance lands outside the tensor). The 512-byte bands keep the buffers' alignment."""
import numpy as np
import pytest

from paper_2402_05598_gb300 import inputs as I

SENTINEL = 7.25
PAD_BYTES = 512


def guarded(shape, dtype, dev):
    import torch
    esz = torch.tensor([], dtype=dtype).element_size()
    pad = PAD_BYTES // esz
    n = int(np.prod(shape))
    buf = torch.full((pad + n + pad,), SENTINEL, dtype=dtype, device=dev)
    return buf, buf[pad:pad + n].view(*shape), pad, n


def bands_intact(buf, pad, n):
    import torch
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    return bool(np.all(b[:pad] == SENTINEL) and np.all(b[pad + n:] == SENTINEL))


def model_for(lib, dev, C, M, seed=0):
    import torch
    desc = I.ModelDesc(width=C, layers=4, modes=M, proj_width=C)
    w = torch.from_numpy(I.xavier_weights(desc, seed)).to(dev)
    return lib.Model(lib.make_desc(C, 4, M, C), w), w


@pytest.mark.gpu
@pytest.mark.parametrize("N,B", [(33, 3), (100, 2)])
def test_apply_A_and_harvest_write_inside_their_outputs(lib, dev, N, B):
    import torch
    k, f = I.make_batch(N, list(range(40, 40 + B)))
    op = lib.Operator(torch.from_numpy(k).to(dev))
    x = torch.from_numpy(np.random.default_rng(1).standard_normal((B, N, N))).to(dev)
    buf, y, pad, n = guarded((B, N, N), torch.float64, dev)
    op.apply(x, y)
    assert bands_intact(buf, pad, n)
    K = 4
    rb, r_out, rpad, rn = guarded((K, B, N, N), torch.float64, dev)
    eb, e_out, epad, en = guarded((K, B, N, N), torch.float64, dev)
    fb = torch.from_numpy(f).to(dev)
    ustar = torch.zeros_like(fb)
    lib.krylov_harvest(op, fb, torch.zeros_like(fb), ustar, K, r_out, e_out)
    assert bands_intact(rb, rpad, rn) and bands_intact(eb, epad, en)


@pytest.mark.gpu
@pytest.mark.parametrize("N,B,C,M,prec", [(20, 3, 8, 5, "fp64"), (64, 3, 32, 12, "bf16"),
                                          (128, 2, 32, 12, "bf16"), (32, 1, 16, 8, "fp16")])
def test_preconditioner_writes_inside_z(lib, dev, N, B, C, M, prec):
    import torch
    k, r = I.make_batch(N, list(range(60, 60 + B)))
    model, _w = model_for(lib, dev, C, M)
    op = lib.Operator(torch.from_numpy(k).to(dev))
    buf, z, pad, n = guarded((B, N, N), torch.float64, dev)
    lib.precond_apply(model, op, torch.from_numpy(r).to(dev), z, prec=prec)
    assert bands_intact(buf, pad, n)
    assert np.isfinite(z.cpu().numpy()).all()


@pytest.mark.gpu
@pytest.mark.parametrize("N,B,C,M,prec", [(64, 3, 32, 12, "bf16"), (100, 2, 8, 5, "fp64"), (128, 2, 32, 12, "bf16")])
def test_solve_writes_inside_x(lib, dev, N, B, C, M, prec):
    import torch
    k, f = I.make_batch(N, list(range(80, 80 + B)))
    model, _w = model_for(lib, dev, C, M)
    op = lib.Operator(torch.from_numpy(k).to(dev))
    buf, x, pad, n = guarded((B, N, N), torch.float64, dev)
    x.zero_()
    info = lib.solve(op, model, torch.from_numpy(f).to(dev), x, tol=1e-6, m_max=5, max_iter=12, prec=prec,
                     fixed_iters=True)
    assert all(i["iters"] == 12 for i in info)
    assert bands_intact(buf, pad, n)


@pytest.mark.gpu
def test_train_step_writes_inside_loss_and_grad(lib, dev):
    import torch
    N, B, C, M = 32, 2, 16, 8
    k, f = I.make_batch(N, [90, 91])
    model, w = model_for(lib, dev, C, M, seed=4)
    op = lib.Operator(torch.from_numpy(k).to(dev))
    fb = torch.from_numpy(f).to(dev)
    e = torch.from_numpy(np.random.default_rng(2).standard_normal((B, N, N))).to(dev)
    lb, loss, lpad, ln = guarded((1,), torch.float32, dev)
    gb, grad, gpad, gn = guarded((w.numel(),), torch.float32, dev)
    lib.train_step(model, op, fb, e, loss, grad, prec="fp32")
    assert bands_intact(lb, lpad, ln) and bands_intact(gb, gpad, gn)
    assert np.isfinite(grad.cpu().numpy()).all() and float(loss.item()) > 0
