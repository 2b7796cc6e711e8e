"""The FP64 multiply-add rate kernel behind the FP64 roof the Krylov kernels are measured
against: it must do every multiply-add it claims (its output equals the chain's closed form
x_K = a^K x_0 + c (1 - a^K) / (1 - a)), and its argument checks reject bad sizes before any
launch."""
import numpy as np
import pytest


@pytest.mark.gpu
@pytest.mark.parametrize("blocks,steps", [(1, 1), (3, 1000), (152 * 8, 2048)])
def test_fp64_fma_rate_kernel_matches_the_closed_form(lib, dev, blocks, steps):
    import torch
    a, c = 1.0 - 2.0 ** -10, 2.0 ** -12
    out = torch.full((blocks * 256,), float("nan"), dtype=torch.float64, device=dev)
    fmas = lib.fp64_fma_rate(blocks, steps, a, c, out)
    torch.cuda.synchronize()
    assert fmas == blocks * 256 * 8 * steps
    aK = a ** steps
    x0 = 1.0 + 0.0625 * np.arange(8)
    expect = float(np.sum(aK * x0 + c * (1.0 - aK) / (1.0 - a)))
    got = out.cpu().numpy()
    # each step rounds once: the relative error stays below steps * 2^-52 of the terms
    assert np.all(np.abs(got - expect) <= 8 * steps * 2.0 ** -52 * 8.0 + 1e-15)


@pytest.mark.gpu
def test_fp64_fma_rate_rejects_bad_sizes(lib, dev):
    import torch
    out = torch.zeros(256, dtype=torch.float64, device=dev)
    for blocks, steps in [(0, 10), (1, 0), (1 << 21, 1), (1, (1 << 24) + 1)]:
        with pytest.raises(lib.FcgnoError) as ei:
            lib.fp64_fma_rate(blocks, steps, 1.0, 0.0, out)
        assert ei.value.code == lib.FCGNO_EINVAL
