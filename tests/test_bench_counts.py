"""The bench's algorithmic work counts (host logic, no GPU): the truncation window it uses to
count FP64 multiply-adds is the oracle's rule of Algorithm 1, the FMA count of the fused FCG
step follows from it, and the synthesis byte count matches the tensor sizes it names."""
import importlib.util
import os

import pytest

from oracle import fcgno_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_window_rule_is_algorithm_1(bench):
    for m in (1, 2, 5, 8):
        assert [bench.window_m(i, m) for i in range(40)] == [O.truncation_window(i, m) for i in range(40)]


def test_fcg_step_fma_count(bench):
    # m = 5: windows 0, 1, 2, 3, 4, 5, 1, 1, 2 for iterations 0..8
    n = 7
    assert bench.fcg_step_fmas([1], n, 5) == n * 10
    assert bench.fcg_step_fmas([9], n, 5) == n * (10 * 9 + 2 * (0 + 1 + 2 + 3 + 4 + 5 + 1 + 1 + 2))
    # instances add independently; one that stopped at iteration 0 did no work
    assert bench.fcg_step_fmas([3, 0, 2], n, 1) == bench.fcg_step_fmas([3], n, 1) + bench.fcg_step_fmas([2], n, 1)
    assert bench.fcg_step_fmas([], n, 5) == 0


def test_synthesis_bytes(bench):
    N, C, M, L = 64, 32, 12, 4
    n = N * N
    # hidden layer: read the 16-bit input and the mixed coefficients, write the 16-bit output
    hidden = n * C * 2 + M * C * 4 * M * 2 + n * C * 2
    # last layer: read input and coefficients, write z in FP64
    last = n * C * 2 + M * C * 4 * M * 2 + n * 8
    assert hidden == 561_152 and last == 331_776
    total, launches = bench.roofline_synthesis([256, 200, 3], N, C, M, L)
    assert launches == 3 * L
    assert total == (256 + 200 + 3) * ((L - 1) * hidden + last)
    # output_scale 1: the last layer also reads the pointwise 1/k in FP64
    total1, _ = bench.roofline_synthesis([256, 200, 3], N, C, M, L, output_scale=1)
    assert total1 == total + (256 + 200 + 3) * n * 8


def test_fcg_step_bytes(bench):
    # per active unknown and iteration: 72 + 16 m_i bytes; m = 5 windows 0, 1, 2 for i = 0, 1, 2
    n = 5
    assert bench.fcg_step_bytes([3], n, 5) == n * (72 * 3 + 16 * (0 + 1 + 2))
    assert bench.fcg_step_bytes([0, 1], n, 1) == n * 72
    assert bench.fcg_step_bytes([], n, 5) == 0


def test_synthesis_flops(bench):
    N, C, M, L, Cp = 64, 32, 12, 4, 32
    n = N * N
    per_unknown = 16 * M * M * C / N + 4 * M * C + 2 * C * C
    assert per_unknown == 4736
    total = bench.synthesis_flops([256, 7], N, C, M, L, Cp)
    assert total == (256 + 7) * n * (L * per_unknown + 2 * C * Cp + 2 * Cp)


def test_rate_and_frac(bench):
    assert bench.rate_and_frac(2e12, 1000.0, 1e12, 4.0) == (2.0, 0.5)
    assert bench.rate_and_frac(1.0, 0.0, 1.0, 1.0) == (None, None)
    assert bench.rate_and_frac(5e9, 1.0, 1e9, None) == (5000.0, None)
