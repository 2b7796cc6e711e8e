"""Ablations of Sections 3.4-3.5 (Tables 2 and 3): the loss and the training data.

Three variants of the preconditioner are trained on the paper's Poisson and Diffusion
datasets (Section 3.2) with N_train = grid instances and 100 samples per instance, then used
in FCG (Algorithm 1) on held-out instances; the table reports the mean number of iterations
needed to reduce ||r_i|| / ||r_0|| below 1e-3, 1e-6 and 1e-12:
  notay_krylov  Eq. (11) loss on Krylov residuals (Eq. (9))        -- the method
  l2_krylov     L2 loss in error form on Krylov residuals          -- Table 2, right half
  notay_random  Eq. (11) loss on random residuals r = f - A u       -- Table 3, right half
An entry is None when some held-out instance did not reach the factor within max_iter
(the paper's "---").

Run: python -m paper_2402_05598_gb300.ablations --out results.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import fcgno as F
from . import inputs as I
from . import train as T

VARIANTS = {
    "notay_krylov": ("energy", "krylov"),
    "l2_krylov": ("l2", "krylov"),
    "notay_random": ("energy", "random"),
}
FACTORS = (1e-3, 1e-6, 1e-12)


def evaluate(model, dataset: str, N: int, seeds, prec: str = "bf16", m_max: int = 5, max_iter: int = 2000,
             factors=FACTORS, detail: dict | None = None) -> dict:
    """Mean FCG-NO iterations to each residual-reduction factor over the given instances
    (u_0 ~ N(0, 1)); None where an instance did not get there within max_iter. ``detail``
    (optional) receives per factor the outcome counts by status and the best relative
    residual reached."""
    import torch
    dev = model.weights.device
    pairs = [I.dataset_problem(dataset, N, s) for s in seeds]
    k = torch.from_numpy(np.ascontiguousarray(np.stack([p[0] for p in pairs]))).to(dev)
    f = torch.from_numpy(np.ascontiguousarray(np.stack([p[1] for p in pairs]))).to(dev)
    x0 = torch.from_numpy(np.random.default_rng(4242).standard_normal((len(seeds), N, N))).to(dev)
    op = F.Operator(k)
    out = {}
    for tol in factors:
        x = x0.clone()
        info = F.solve(op, model, f, x, tol=tol, m_max=m_max, max_iter=max_iter, prec=prec, check_every=8)
        ok = all(i["status"] == F.FCGNO_OK for i in info)
        out[f"{tol:g}"] = float(np.mean([i["iters"] for i in info])) if ok else None
        if detail is not None:
            counts = {}
            for i in info:
                name = F.status_str(i["status"])
                counts[name] = counts.get(name, 0) + 1
            detail[f"{tol:g}"] = {"status": counts, "min_relres": float(min(i["relres"] for i in info)),
                                  "max_relres": float(max(i["relres"] for i in info))}
    op.close()
    return out


def run_variant(dataset: str, N: int, variant: str, steps: int, width: int = 32, layers: int = 4, modes: int = 12,
                eval_instances: int = 32, m_max: int = 5, seed: int = 0, device=None, output_scale: int = 1) -> dict:
    """Trains one variant from Xavier weights (seed) and evaluates it."""
    import torch
    dev = device or torch.device("cuda:0")
    loss_kind, data = VARIANTS[variant]
    desc = I.ModelDesc(width=width, layers=layers, modes=modes, proj_width=width, output_scale=output_scale)
    w = torch.from_numpy(I.xavier_weights(desc, seed)).to(dev)
    model = F.Model(F.make_desc(width, layers, modes, width, output_scale=output_scale), w)
    t0 = time.perf_counter()
    res = T.train(model, N, range(N), K=100, batch=32, lr=1e-3, steps=steps, dataset=dataset, data=data,
                  loss_kind=loss_kind, log_every=max(1, steps // 4))
    secs = time.perf_counter() - t0
    detail = {}
    its = evaluate(model, dataset, N, range(30000, 30000 + eval_instances), m_max=m_max, detail=detail)
    model.close()
    return {"dataset": dataset, "grid": N, "variant": variant, "loss": loss_kind, "data": data, "steps": res.steps,
            "output_scale": output_scale,
            "train_seconds": round(secs, 2), "harvest_seconds": round(res.harvest_seconds, 2),
            "loss_log": [(s, round(v, 4)) for s, v in res.losses], "iterations": its, "outcomes": detail}


def format_table(rows) -> str:
    """Markdown table in the shape of Tables 2 and 3 (one row per dataset and grid)."""
    keys = [f"{t:g}" for t in FACTORS]
    head = "| Dataset | grid | " + " | ".join(f"{v} {k}" for v in VARIANTS for k in keys) + " |"
    sep = "|" + "---|" * (2 + len(VARIANTS) * len(keys))
    lines = [head, sep]
    cells = {}
    for r in rows:
        cells[(r["dataset"], r["grid"], r["variant"])] = r["iterations"]
    for ds, grid in sorted({(r["dataset"], r["grid"]) for r in rows}):
        vals = []
        for v in VARIANTS:
            its = cells.get((ds, grid, v), {})
            for k in keys:
                x = its.get(k)
                vals.append("---" if x is None else f"{x:.1f}")
        lines.append(f"| {ds} | {grid} | " + " | ".join(vals) + " |")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--datasets", default="poisson,diffusion")
    ap.add_argument("--grids", default="32,64")
    ap.add_argument("--variants", default=",".join(VARIANTS))
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--output-scale", type=int, default=1, choices=[0, 1])
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    rows = []
    for ds in args.datasets.split(","):
        for N in (int(g) for g in args.grids.split(",")):
            for v in args.variants.split(","):
                rows.append(run_variant(ds, N, v, args.steps, output_scale=args.output_scale))
                print(json.dumps(rows[-1]), flush=True)
    print(format_table(rows))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump({"rows": rows, "table": format_table(rows)}, fh, indent=1)


if __name__ == "__main__":
    main()
