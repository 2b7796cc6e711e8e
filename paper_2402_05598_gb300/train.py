"""Training the neural-operator preconditioner (Section 3.1, Fig. 2(a)-(b)).

Data (Eq. (9)): for every training instance, u_0 ~ N(0, 1); CG (Algorithm 1 with B = I)
runs K iterations and every iterate gives a residual r_i and an error e_i = u* - u_i, where
u* is the same problem solved to a relative residual of 1e-12. The loss is Eq. (11),
mean ||NO(r) - e||_A / ||e||_A, and its gradient comes from the library's hand-written
backward (fcgno_train_step). PyTorch's Adam updates the FP32 master blob.

Ablations (Sections 3.4-3.5): the L2 loss in error form instead of Eq. (11)
(``loss_kind="l2"``), and random residuals instead of Krylov vectors (``data="random"``):
u_i ~ N(0, I), f_i ~ p_f, r_i = f_i - A u_i, e_i = A^{-1} f_i - u_i.

Batches hold one sample from each instance of a group of ``batch`` instances (one
assembled operator per group); the sample index inside each instance's Krylov sequence is
drawn at random every step.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import fcgno as F
from . import inputs as I


@dataclass
class TrainResult:
    """Outcome of train(): steps taken, wall time (and the Krylov harvest's share), (step, loss) log."""
    steps: int
    seconds: float
    harvest_seconds: float
    losses: list = field(default_factory=list)


class KrylovData:
    """Harvested (r_i, e_i) pairs of one group of instances, resident on the device."""

    def __init__(self, N, seeds, K, device, sigma=1.0, ell=0.1, x0_seed=12345, stream=None, dataset="grf"):
        import torch
        k, f = _problems(dataset, N, seeds, sigma, ell)
        B = len(seeds)
        self.B, self.N, self.K = B, N, K
        self.k = torch.from_numpy(k).to(device)
        self.op = F.Operator(self.k, stream)
        fb = torch.from_numpy(f).to(device)
        ustar = torch.zeros_like(fb)
        F.solve(self.op, None, fb, ustar, tol=1e-12, m_max=1, max_iter=20 * N * N, prec="fp64", check_every=64,
                stream=stream)
        x0 = torch.from_numpy(np.random.default_rng(x0_seed).standard_normal((B, N, N))).to(device)
        self.r = torch.empty((K, B, N, N), dtype=torch.float64, device=device)
        self.e = torch.empty_like(self.r)
        F.krylov_harvest(self.op, fb, x0, ustar, K, self.r, self.e, stream)


class RandomResidualData:
    """Random residuals (the ablation of Section 3.5): for sample i of each instance,
    u_i ~ N(0, I) and f_i ~ p_f of the dataset (k stays the instance's); r_i = f_i - A u_i and
    e_i = A^{-1} f_i - u_i, with A^{-1} f_i from CG to a relative residual of 1e-12."""

    def __init__(self, N, seeds, K, device, sigma=1.0, ell=0.1, x0_seed=12345, stream=None, dataset="grf"):
        import torch
        k, _ = _problems(dataset, N, seeds, sigma, ell)
        B = len(seeds)
        self.B, self.N, self.K = B, N, K
        self.k = torch.from_numpy(k).to(device)
        self.op = F.Operator(self.k, stream)
        rng = np.random.default_rng(x0_seed)
        self.r = torch.empty((K, B, N, N), dtype=torch.float64, device=device)
        self.e = torch.empty_like(self.r)
        for i in range(K):
            f = torch.from_numpy(np.ascontiguousarray(np.stack([I.dataset_rhs(dataset, N, rng) for _ in range(B)])))
            f = f.to(device)
            u = torch.from_numpy(rng.standard_normal((B, N, N))).to(device)
            x = torch.zeros_like(f)
            F.solve(self.op, None, f, x, tol=1e-12, m_max=1, max_iter=20 * N * N, prec="fp64", check_every=64,
                    stream=stream)
            # r_i = f_i - A u_i and e_i = A^-1 f_i - u_i, formed by the library
            self.op.residual_pair(f, u, x, self.r[i], self.e[i], stream)


class PreconditionerLoss(torch.autograd.Function):
    """The training loss of the neural preconditioner as an autograd node: Eq. (11) (energy
    norm, loss_kind "energy") or the L2 ablation loss. The forward and the backward run in one
    library call (fcgno_train_step: the reverse mode is hand-written in CUDA): the forward
    computes the loss and the weight gradient together and keeps the gradient, which the
    backward scales by the incoming gradient."""

    @staticmethod
    def forward(ctx, weights, model, op, r, e, prec, loss_kind):
        loss = torch.zeros(1, dtype=torch.float32, device=weights.device)
        grad = torch.empty_like(weights)
        F.train_step(model, op, r, e, loss, grad, prec=prec, loss_kind=loss_kind)
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None, None, None, None


def preconditioner_loss(model: "F.Model", op: "F.Operator", r, e, prec: str = "fp32", loss_kind: str = "energy"):
    """Scalar loss tensor of a batch (r, e) with ``model.weights`` as its autograd input:
    ``preconditioner_loss(...).backward()`` fills ``model.weights.grad``."""
    return PreconditionerLoss.apply(model.weights, model, op, r, e, prec, loss_kind)


def _problems(dataset, N, seeds, sigma, ell):
    if dataset == "grf":
        return I.make_batch(N, seeds, sigma, ell)
    pairs = [I.dataset_problem(dataset, N, s) for s in seeds]
    return (np.ascontiguousarray(np.stack([p[0] for p in pairs])),
            np.ascontiguousarray(np.stack([p[1] for p in pairs])))


def train(model: "F.Model", N: int, train_seeds, K: int = 100, batch: int = 32, lr: float = 1e-3,
          steps: int = 1000, seconds: float | None = None, prec: str = "fp32", seed: int = 0,
          sigma=1.0, ell: float = 0.1, log_every: int = 0, decay_at=(0.5, 0.75),
          dataset: str = "grf", data: str = "krylov", loss_kind: str = "energy",
          weight_decay: float = 0.0) -> TrainResult:
    """Trains ``model.weights`` in place; returns the loss history. The learning rate is
    halved at the given fractions of ``steps`` (the paper halves it on a fixed schedule,
    Table 6). ``data``: "krylov" (Eq. (9)) or "random" (Section 3.5); ``loss_kind``: "energy"
    (Eq. (11)) or "l2". ``sigma`` is the GRF standard deviation of the coefficient fields, or
    a sequence of them: group g of ``batch`` instances then uses sigma[g % len(sigma)], so
    that the training distribution covers every coefficient contrast it will be served.
    ``weight_decay`` > 0 applies decoupled weight decay (AdamW) of that rate (Table 6 lists
    1e-2)."""
    import torch
    dev = model.weights.device
    t0 = time.perf_counter()
    groups = []
    seeds = list(train_seeds)
    Data = KrylovData if data == "krylov" else RandomResidualData
    sigmas = tuple(sigma) if isinstance(sigma, (tuple, list)) else (sigma,)
    for gi, g0 in enumerate(range(0, len(seeds) - batch + 1, batch)):
        groups.append(Data(N, seeds[g0:g0 + batch], K, dev, sigmas[gi % len(sigmas)], ell, x0_seed=1000 + g0,
                           dataset=dataset))
    torch.cuda.synchronize()
    t_h = time.perf_counter() - t0
    param = model.weights
    param.requires_grad_(True)
    opt = (torch.optim.AdamW([param], lr=lr, weight_decay=weight_decay) if weight_decay > 0
           else torch.optim.Adam([param], lr=lr))
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    ar = torch.arange(batch, device=dev)
    losses = []
    t1 = time.perf_counter()
    step = 0
    decay_steps = {int(f * steps) for f in decay_at}
    while step < steps and (seconds is None or time.perf_counter() - t1 < seconds):
        if step in decay_steps:
            for pg in opt.param_groups:
                pg["lr"] *= 0.5
        d = groups[step % len(groups)]
        idx = torch.randint(0, K, (batch,), generator=gen, device=dev)
        r = d.r[idx, ar].contiguous()
        e = d.e[idx, ar].contiguous()
        opt.zero_grad(set_to_none=True)
        loss = preconditioner_loss(model, d.op, r, e, prec=prec, loss_kind=loss_kind)
        loss.backward()
        opt.step()
        if prec == "fp64":
            model.sync()
        if log_every and step % log_every == 0:
            losses.append((step, float(loss.item())))
        step += 1
    param.requires_grad_(False)
    param.grad = None
    model.sync()
    torch.cuda.synchronize()
    return TrainResult(steps=step, seconds=time.perf_counter() - t1, harvest_seconds=t_h, losses=losses)
