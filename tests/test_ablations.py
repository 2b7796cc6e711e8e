"""Ablation runner (Sections 3.4-3.5): host logic on the CPU, data and a short run on the GPU."""
import numpy as np
import pytest

from paper_2402_05598_gb300 import inputs as I


def test_dataset_registry_is_deterministic_and_matches_generators():
    for name in I.DATASETS:
        k1, f1 = I.dataset_problem(name, 16, 3)
        k2, f2 = I.dataset_problem(name, 16, 3)
        assert k1.shape == f1.shape == (16, 16)
        assert np.array_equal(k1, k2) and np.array_equal(f1, f2)
        assert np.all(k1 > 0)
        g = I.dataset_rhs(name, 16, np.random.default_rng(0))
        assert g.shape == (16, 16) and np.all(np.isfinite(g))
    assert np.array_equal(I.dataset_problem("poisson", 16, 5)[1], I.poisson_problem(16, 5)[1])
    assert np.array_equal(I.dataset_problem("diffusion", 16, 5)[0], I.diffusion_problem(16, 5)[0])
    with pytest.raises(ValueError):
        I.dataset_problem("nope", 16, 0)


def test_ablation_table_shape():
    pytest.importorskip("torch")
    from paper_2402_05598_gb300 import ablations as A
    rows = [{"dataset": "poisson", "grid": 32, "variant": v, "iterations": {"0.001": 4.0, "1e-06": 9.0, "1e-12": None}}
            for v in A.VARIANTS]
    t = A.format_table(rows).splitlines()
    assert len(t) == 3
    assert t[2].startswith("| poisson | 32 |")
    assert t[2].count("---") == len(A.VARIANTS)
    assert A.VARIANTS["l2_krylov"] == ("l2", "krylov") and A.VARIANTS["notay_random"] == ("energy", "random")


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["krylov", "random"])
def test_training_pairs_satisfy_A_e_equals_r(lib, dev, kind):
    """Both data kinds give e = A^{-1} r: Krylov pairs (Eq. (9)) and random residuals
    (Section 3.5: r = f - A u, e = A^{-1} f - u)."""
    import torch
    from paper_2402_05598_gb300 import train as T
    Data = T.KrylovData if kind == "krylov" else T.RandomResidualData
    d = Data(32, list(range(4)), 5, dev, dataset="diffusion")
    Ae = torch.empty_like(d.e[0])
    for i in range(5):
        d.op.apply(d.e[i].contiguous(), Ae)
        err = float(torch.linalg.norm(Ae - d.r[i]) / torch.linalg.norm(d.r[i]))
        assert err < 1e-8, (kind, i, err)


@pytest.mark.gpu
def test_short_ablation_run(lib, dev):
    from paper_2402_05598_gb300 import ablations as A
    for v in A.VARIANTS:
        row = A.run_variant("poisson", 32, v, steps=10, eval_instances=4, device=dev)
        assert row["steps"] == 10 and row["variant"] == v
        assert set(row["iterations"]) == {f"{t:g}" for t in A.FACTORS}
        assert row["iterations"]["0.001"] is not None and row["iterations"]["0.001"] > 0
