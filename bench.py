"""Benchmark: FCG-NO solves/s to relative residual 1e-6 on one GB300 (or N replicas).

Workload (the training-plus-solve configuration on a 64 x 64 grid): 256 held-out diffusion
instances (seeds 10000 + 256*rank + i), k = exp(GRF(length 0.1, sigma 1)), f iid N(0, 1),
u_0 iid N(0, 1) (Algorithm 1), FNO preconditioner of width 32, 4 Fourier layers, 12 x 12
modes, trained in the setup phase with the energy-norm loss on Krylov vectors harvested
from CG on 512 seeded training instances. One step = assembling the batch's operator from k
(fcgno_reassemble) and one batched solve of all 256 instances to ||r_i|| <= 1e-6 ||r_0||
(truncation m = 5) with the BF16 tensor-core preconditioner and the FP64 Krylov loop. Inputs
are resident in HBM when a timed step starts; L2 is flushed (256 MB write) between timed
steps. The timed steps run untraced; the roofline comes from a traced copy of the same step.

Beside the headline: m = 1; the all-FP64 GPU FCG-NO, CG and Jacobi(4)-PCG on the same 256
instances (CUDA events, same protocol); the resolution-transfer configuration (128..512 grids,
sigma in {0.5, 1, 2}); the large single solves (1024 x 1024 x 8, 2048 x 2048 x 2 to 1e-8); the
serving stream; the end-to-end call on host buffers; the FP64 CPU oracle on a bounded sample.

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_GRID = 64
WIDTH, LAYERS, MODES = 32, 4, 12
EVAL_BATCH = 256
TOL = 1e-6
METRIC = "solves/s to rel-residual 1e-6 (BF16-NO FCG, FP64 Krylov loop)"
UNIT = "solves/s"


# --------------------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------------- oracle
def _oracle_worker(args):
    """One instance of the workload solved by the FP64 CPU oracle (runs in a spawned process)."""
    N, seed, blob, m_max, max_iter, fixed_iters, out_scale = args
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import fcgno_oracle as O
    from paper_2402_05598_gb300 import inputs as I
    desc = I.ModelDesc(width=WIDTH, layers=LAYERS, modes=MODES, proj_width=WIDTH, output_scale=out_scale)
    P = O.unpack_weights(blob, desc)
    k, f = I.make_problem(N, seed)
    u0 = np.random.default_rng(seed + 777).standard_normal((N, N))
    lk = np.log(k)
    t = time.perf_counter()
    out = O.fcg(lambda u: O.apply_A(k, u), lambda r: O.no_forward(P, desc, r, lk), f, u0, m_max, max_iter,
                tol=None if fixed_iters else TOL)
    return time.perf_counter() - t, out["iterations"]


def workload_name(m: int) -> str:
    return (f"FCG-NO eval: {EVAL_BATCH} instances/GPU, {N_GRID}x{N_GRID} diffusion (k=exp(GRF 0.1, 1)), "
            f"FNO width {WIDTH}, {LAYERS} layers, {MODES}x{MODES} modes, m={m}, tol {TOL}")


def oracle_sample(blob: np.ndarray, n_inst: int, iters: int, cores: int, m_max: int = 5, out_scale: int = 1):
    """Times the oracle FCG-NO on n_inst instances, `iters` fixed iterations each, in a pool of
    `cores` spawned single-threaded processes. Returns (wall seconds, total iterations)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    env_old = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_old:
        os.environ[k] = "1"
    try:
        jobs = [(N_GRID, 10000 + i, blob, m_max, iters, True, out_scale) for i in range(n_inst)]
        t = time.perf_counter()
        with ctx.Pool(processes=cores) as pool:
            res = pool.map(_oracle_worker, jobs)
        wall = time.perf_counter() - t
    finally:
        for k, v in env_old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return wall, sum(r[1] for r in res)


# --------------------------------------------------------------------------------------- helpers
def roofline_synthesis(active_per_iter, N, C, M, layers, output_scale=0):
    """Algorithmic HBM bytes of all synthesis launches: per active instance and layer, read
    the layer input (n*C*2 B) and the mixed coefficients (M*C*4M*2 B); hidden layers write
    the next activation (n*C*2 B), the last layer writes z (n*8 B) and, with output_scale 1,
    reads the pointwise 1/k (n*8 B)."""
    n = N * N
    chat = M * C * 4 * M * 2
    hidden = 2 * n * C * 2 + chat
    last = n * C * 2 + chat + n * 8 + (n * 8 if output_scale else 0)
    per_inst = (layers - 1) * hidden + last
    return float(sum(active_per_iter)) * per_inst, int(len(active_per_iter)) * layers


def window_m(i, m_max):
    """Truncation window m_i of Algorithm 1 at iteration i (0-based)."""
    return min(i, max(1, i % (m_max + 1)))


def fcg_step_fmas(iters_per_instance, n, m_max):
    """Algorithmic FP64 multiply-adds of the fused FCG step over a solve: per active instance
    and iteration i, n (10 + 2 m_i) -- m_i window dots and m_i direction updates, the 5-point
    stencil (5), the dots (p, s) and (p, r), the updates of u and r and ||r||^2."""
    return float(sum(n * (10 + 2 * window_m(i, m_max)) for it in iters_per_instance for i in range(it)))


def fcg_step_bytes(iters_per_instance, n, m_max):
    """Algorithmic HBM bytes of the fused FCG step over a solve: per active instance and
    iteration i, n (72 + 16 m_i) -- read w and the m_i vectors s_k and p_k, write p and s, read
    the two face-coefficient arrays, read and write u and r (the stored diagonal, a
    convenience of this implementation, is not counted)."""
    return float(sum(n * (72 + 16 * window_m(i, m_max)) for it in iters_per_instance for i in range(it)))


def synthesis_flops(active_per_iter, N, C, M, layers, Cp):
    """Algorithmic FLOPs of all synthesis launches: per active instance and layer, stage 1
    (16 M^2 C N: the inverse transform over x1 of the 2M x M x C complex coefficients for every
    column), stage 2 (4 M C N^2: the inverse transform over x2, real part) and the pointwise
    path W v (2 C^2 N^2); the last layer adds the decoder (2 C Cp + 2 Cp per point)."""
    n = N * N
    layer = 16 * M * M * C * N + 4 * M * C * n + 2 * C * C * n
    last = layer + (2 * C * Cp + 2 * Cp) * n
    return float(sum(active_per_iter)) * ((layers - 1) * layer + last)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine() or "unknown"


def rate_and_frac(amount, ms, scale, peak):
    """(amount per second / scale, that over peak); (None, None) without a positive time."""
    if not ms or ms <= 0:
        return None, None
    rate = amount / (ms / 1000.0) / scale
    return rate, (rate / peak if peak else None)


# GB300's nominal dense FP64 rate (TFLOP/s). The FMA-chain kernel below reaches about 84 % of
# it (ncu: FP64 pipe active 84 % of cycles at 2.07 GHz), which is the measured roof.
FP64_NOMINAL_TFLOPS = 1.25


def measure_fp64_roof(dev, stream, repeats=5):
    """FP64 multiply-add rate of this GPU, measured with the library's FMA-chain kernel on
    every SM (8 CTAs of 256 threads per SM, 2048 steps of 8 chains per thread); CUDA events on
    the launching stream, best and median of `repeats` launches after two warm-ups."""
    import torch
    from paper_2402_05598_gb300 import fcgno as F
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 8
    out = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
    a, c = 1.0 - 2.0 ** -10, 2.0 ** -12
    for _ in range(2):
        F.fp64_fma_rate(blocks, 2048, a, c, out, stream)
    ms = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fmas = F.fp64_fma_rate(blocks, 2048, a, c, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    best, med = min(ms), float(np.median(ms))
    return {"tflops": 2.0 * fmas / (best / 1000.0) / 1e12, "tflops_median": 2.0 * fmas / (med / 1000.0) / 1e12,
            "fmas_per_launch": fmas, "blocks": blocks,
            "how": "fcgno_fp64_fma_rate: independent FP64 FMA chains on every SM; best of %d launches" % repeats}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one tc_synthesis_kernel launch
# per active instance, mean of the four layers of an iteration, measured by ncu on this
# kernel at 64 x 64, 256 instances, width 32, 12 x 12 modes, output_scale 1. Scaled by the
# active instances per launch; None when the kernel has changed since the last capture.
SYN_TRAFFIC_PER_INSTANCE = 364_695


SERVE_SIZES = {64: 0.40, 128: 0.25, 256: 0.20, 512: 0.10, 1024: 0.05}
SERVE_SIGMAS = (0.5, 1.0, 2.0)


def run_serving(args, model, desc_np, dev, rate, n_req, budget_gb=80.0):
    """Serving stream of the configured mix through the device-driven server (admission and
    retirement on the device every iteration): exponential inter-arrival times (mean 1/rate,
    seed 5), grid sizes drawn with the configured probabilities, sigma uniform in
    {0.5, 1, 2}, ell = 0.1; every request has its own problem (k, f iid N(0,1), u_0 iid
    N(0,1), seed 50000 + request index), generated and made resident before the run. Bucket
    capacities split the HBM budget in proportion to each size's share of the offered
    unknowns. Each request's solution is delivered into its own output tensor."""
    import torch
    from paper_2402_05598_gb300 import fcgno as F
    from paper_2402_05598_gb300 import inputs as I
    from paper_2402_05598_gb300 import serve as S
    rng = np.random.default_rng(5)
    sizes = list(SERVE_SIZES)
    probs = np.array([SERVE_SIZES[N] for N in sizes])
    gaps = rng.exponential(1.0 / rate, n_req)
    arrivals = np.cumsum(gaps) - gaps[0]
    Ns = rng.choice(sizes, size=n_req, p=probs / probs.sum())
    sis = rng.integers(0, len(SERVE_SIGMAS), n_req)
    t_gen = time.perf_counter()
    reqs = []
    for i in range(n_req):
        N, sg = int(Ns[i]), SERVE_SIGMAS[int(sis[i])]
        kk, ff = I.make_problem(N, 50000 + i, sigma=sg, ell=0.1)
        x0 = np.random.default_rng(50000 + i + 777).standard_normal((N, N))
        kd, fd, xd = (torch.from_numpy(a).to(dev) for a in (kk, ff, x0))
        reqs.append(S.Request(i, float(arrivals[i]), N, kd, fd, xd, out=torch.empty_like(xd)))
    t_gen = time.perf_counter() - t_gen
    m = args.serve_m
    mdesc = F.make_desc(WIDTH, LAYERS, MODES, WIDTH, output_scale=args.output_scale)
    caps = S.plan_capacities(SERVE_SIZES, int(budget_gb * 2**30), m, mdesc, args.prec, max_slots=1 << 16)
    srv = S.DeviceServer(model, caps, prec=args.prec, m_max=m, tol=TOL, max_iter=args.max_iter, iters_per_step=8)
    # warm every bucket once (first steps run eagerly and allocate), outside the measurement
    warm = [S.Request(1_000_000_000 + j, 0.0, N,
                      *(torch.from_numpy(a).to(dev) for a in (*I.make_problem(N, 1), np.zeros((N, N)))))
            for j, N in enumerate(sizes)]
    srv.run(warm, S.ServeStats())
    stats = S.ServeStats(offered_rate=rate)
    stats.bucket_bytes = sum(cap * S.slot_bytes(N, m, mdesc, args.prec) for N, cap in caps.items())
    srv.run(reqs, stats)
    srv.close()
    out = stats.summary()
    out.update({"capacities": {str(N): c for N, c in caps.items()}, "budget_gb": budget_gb,
                "sizes": {str(N): p for N, p in SERVE_SIZES.items()}, "tol": TOL, "m": m,
                "max_iter": args.max_iter, "problem_generation_s": round(t_gen, 1),
                "iterations_mean_by_size": {str(N): float(np.mean([r.iters for r in reqs if r.N == N] or [0]))
                                            for N in sizes},
                # requests that reached the tolerance, per grid size and coefficient contrast
                "converged_by_size_sigma": {f"{N}/{sg}": [sum(1 for r, s_ in zip(reqs, sis)
                                                              if r.N == N and SERVE_SIGMAS[s_] == sg and r.status == F.FCGNO_OK),
                                                          sum(1 for r, s_ in zip(reqs, sis)
                                                              if r.N == N and SERVE_SIGMAS[s_] == sg)]
                                            for N in sizes for sg in SERVE_SIGMAS}})
    return out


TRANSFER_SIZES = (128, 256, 512)
TRANSFER_SIGMAS = (0.5, 1.0, 2.0)


def run_transfer(args, model, dev, flush, stream):
    """Resolution transfer: the 64 x 64-trained preconditioner at N in {128, 256, 512}, 64
    instances per (N, sigma), sigma in {0.5, 1, 2}, length 0.1, f and u_0 iid N(0, 1), tol 1e-6,
    truncation m. Per cell: the BF16 preconditioner with the FP64 Krylov loop on all 64
    instances; the all-FP64 FCG-NO (CUDA-core FP64 preconditioner, same weights) and the BF16
    path on the first `fp64_instances` of them (like for like); Jacobi(4)-PCG on all 64. Each
    timed with CUDA events after a warm-up solve."""
    import torch
    from paper_2402_05598_gb300 import fcgno as F
    from paper_2402_05598_gb300 import inputs as I
    out = {}
    for N in TRANSFER_SIZES:
        for si, sg in enumerate(TRANSFER_SIGMAS):
            seeds = range(20000 + 1000 * si + 100 * int(np.log2(N)), 20000 + 1000 * si + 100 * int(np.log2(N)) + 64)
            k_np, f_np = I.make_batch(N, seeds, sg, 0.1)
            u0_np = np.stack([np.random.default_rng(s_ + 777).standard_normal((N, N)) for s_ in seeds])
            cell = {}
            for label, nb in (("all", 64), ("sub", args.transfer_fp64_instances)):
                k = torch.from_numpy(np.ascontiguousarray(k_np[:nb])).to(dev)
                f = torch.from_numpy(np.ascontiguousarray(f_np[:nb])).to(dev)
                u0 = torch.from_numpy(np.ascontiguousarray(u0_np[:nb])).to(dev)
                op = F.Operator(k)
                x = torch.empty_like(u0)

                def step(prec, cap, jac=0):
                    def fn():
                        op.reassemble(k)
                        x.copy_(u0)
                        if jac:
                            return F.solve_jacobi(op, jac, f, x, tol=TOL, m_max=1, max_iter=cap, check_every=32)
                        return F.solve(op, model, f, x, tol=TOL, m_max=args.m, max_iter=cap, prec=prec,
                                       check_every=8 if prec == "bf16" else 16)
                    return fn

                if label == "all":
                    ms, res = timed_steps(step("bf16", args.transfer_max_iter), 1, 1, flush, stream,
                                          warm_fn=step("bf16", 16))
                    cell["bf16"] = solve_summary(ms, res, F)
                    ms, res = timed_steps(step("fp64", 20000, jac=4), 1, 1, flush, stream,
                                          warm_fn=step("fp64", 64, jac=4))
                    cell["jacobi4_pcg"] = solve_summary(ms, res, F)
                else:
                    ms, res = timed_steps(step("bf16", args.transfer_max_iter), 1, 1, flush, stream,
                                          warm_fn=step("bf16", 16))
                    cell["bf16_subset"] = solve_summary(ms, res, F)
                    cap = int(1.3 * cell["bf16_subset"]["iterations"]["max"]) + 16
                    ms, res = timed_steps(step("fp64", cap), 1, 0, flush, stream)
                    cell["fp64_no_subset"] = dict(solve_summary(ms, res, F), max_iter=cap)
                del op
            out[f"{N}/{sg}"] = cell
    return out


LARGE_CASES = ((1024, 8), (2048, 2))


def run_train_leg(args, desc_np, dev, eval_fn):
    """Training throughput (Eq. (11) steps, batch 32 on the 64 x 64 grid, the training
    configuration's shape): BF16 on the tensor cores (FP32 accumulation, FP32 master weights)
    against FP32 on CUDA cores, each timed with CUDA events over `train_bench_steps` library
    steps on one harvested batch; then two models trained from the same seed on the same data
    for the same number of steps, one per precision, and their eval iterations (the
    headline's instances and protocol)."""
    import torch
    from paper_2402_05598_gb300 import fcgno as F
    from paper_2402_05598_gb300 import inputs as I
    from paper_2402_05598_gb300 import train as T
    data = T.KrylovData(N_GRID, list(range(0, 32)), 100, dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    idx = torch.randint(0, 100, (32,), generator=gen, device=dev)
    ar = torch.arange(32, device=dev)
    r, e = data.r[idx, ar].contiguous(), data.e[idx, ar].contiguous()

    def fresh(seed=0):
        blob = torch.from_numpy(I.xavier_weights(desc_np, seed)).to(dev)
        return F.Model(F.make_desc(WIDTH, LAYERS, MODES, WIDTH, output_scale=args.output_scale), blob)

    out = {"batch": 32, "grid": N_GRID, "timed_steps": args.train_bench_steps,
           "what": "one fcgno_train_step (forward, loss, backward, every weight gradient); Adam excluded"}
    for prec in ("fp32", "bf16"):
        m = fresh()
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        grad = torch.zeros(m.weights.numel(), dtype=torch.float32, device=dev)
        for _ in range(5):
            F.train_step(m, data.op, r, e, loss, grad, prec=prec)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.train_bench_steps):
            F.train_step(m, data.op, r, e, loss, grad, prec=prec)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.train_bench_steps
        out[prec] = {"ms_per_step": round(ms, 4), "steps_per_s": round(1000.0 / ms, 1),
                     "samples_per_s": round(32 * 1000.0 / ms, 1)}
    out["bf16_speedup"] = round(out["fp32"]["ms_per_step"] / out["bf16"]["ms_per_step"], 3)
    if args.train_compare_steps > 0:
        cmp_ = {"steps": args.train_compare_steps, "instances": args.train_instances, "seed": 0}
        for prec in ("fp32", "bf16"):
            m = fresh()
            tr = T.train(m, N_GRID, range(0, args.train_instances), K=100, batch=32, lr=1e-3,
                         steps=args.train_compare_steps, prec=prec)
            its, conv = eval_fn(m)
            cmp_[prec] = {"train_seconds": round(tr.seconds, 2), "steps_per_s": round(tr.steps / tr.seconds, 1),
                          "eval_iterations": {"mean": float(np.mean(its)), "max": int(max(its)), "converged": conv}}
        cmp_["mean_iterations_ratio_bf16_over_fp32"] = round(
            cmp_["bf16"]["eval_iterations"]["mean"] / cmp_["fp32"]["eval_iterations"]["mean"], 4)
        out["same_steps_models"] = cmp_
    return out


def run_large(args, dev, flush, stream):
    """Large single solves: 1024 x 1024 x 8 and 2048 x 2048 x 2, k = exp(GRF(length 0.05,
    sigma 2)), f and u_0 iid N(0, 1), tol 1e-8, m = 5. The model (width 32, 16 x 16 modes) is
    trained at 64 x 64 on the same coefficient family, then fine-tuned at 1024 x 1024 on Krylov
    vectors of that grid, where the training step rebuilds its pre-activations (activation
    checkpointing). Reports the fine-tuning steps and, per grid, the BF16 FCG-NO solve and
    Jacobi(4)-PCG on the same instances (CUDA events, one warm-up each)."""
    import torch
    from paper_2402_05598_gb300 import fcgno as F
    from paper_2402_05598_gb300 import inputs as I
    from paper_2402_05598_gb300 import train as T
    M = 16
    desc = I.ModelDesc(width=WIDTH, layers=LAYERS, modes=M, proj_width=WIDTH, output_scale=args.output_scale)
    blob = torch.from_numpy(I.xavier_weights(desc, 1)).to(dev)
    model = F.Model(F.make_desc(WIDTH, LAYERS, M, WIDTH, output_scale=args.output_scale), blob)
    tr = T.train(model, N_GRID, range(0, args.train_instances), K=100, batch=32, lr=1e-3,
                 steps=args.large_train_steps, sigma=2.0, ell=0.05, prec=args.train_prec)
    out = {"model": {"modes": M, "train_steps_64": tr.steps, "train_seconds_64": round(tr.seconds, 2),
                     "train_prec_64": args.train_prec}}
    # fine-tuning at 1024 x 1024 (8 instances): Krylov vectors of CG from u_0 ~ N(0, 1), u* from
    # Jacobi(4)-PCG to 1e-10; Adam steps on Eq. (11) with recomputed pre-activations
    Nf, Bf = LARGE_CASES[0]
    seeds = range(41000, 41000 + Bf)
    k_np, f_np = I.make_batch(Nf, seeds, 2.0, 0.05)
    kf = torch.from_numpy(k_np).to(dev)
    ff = torch.from_numpy(f_np).to(dev)
    opf = F.Operator(kf)
    ustar = torch.zeros_like(ff)
    F.solve_jacobi(opf, 4, ff, ustar, tol=1e-10, m_max=1, max_iter=50000, check_every=64)
    x0 = torch.from_numpy(np.random.default_rng(41).standard_normal((Bf, Nf, Nf))).to(dev)
    K = args.large_finetune_k
    r_out = torch.empty((K, Bf, Nf, Nf), dtype=torch.float64, device=dev)
    e_out = torch.empty_like(r_out)
    F.krylov_harvest(opf, ff, x0, ustar, K, r_out, e_out)
    model.set_train_recompute("always")
    opt = torch.optim.Adam([blob.requires_grad_(True)], lr=args.large_finetune_lr)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(args.large_finetune_steps):
        i = it % K
        opt.zero_grad(set_to_none=True)
        loss = T.preconditioner_loss(model, opf, r_out[i].contiguous(), e_out[i].contiguous(), prec=args.train_prec)
        loss.backward()
        opt.step()
        if it % max(1, args.large_finetune_steps // 10) == 0 or it == args.large_finetune_steps - 1:
            losses.append((it, round(float(loss.item()), 4)))
    blob.requires_grad_(False)
    blob.grad = None
    model.sync()
    torch.cuda.synchronize()
    out["finetune"] = {"grid": Nf, "instances": Bf, "krylov_K": K, "steps": args.large_finetune_steps,
                       "prec": args.train_prec, "lr": args.large_finetune_lr,
                       "seconds": round(time.perf_counter() - t0, 2), "losses": losses,
                       "recompute": "always (every layer's pre-activation rebuilt in the backward)"}
    del opf, r_out, e_out, ustar
    for N, B in LARGE_CASES:
        seeds = range(42000 + N, 42000 + N + B)
        k_np, f_np = I.make_batch(N, seeds, 2.0, 0.05)
        u0_np = np.stack([np.random.default_rng(s_ + 777).standard_normal((N, N)) for s_ in seeds])
        k = torch.from_numpy(k_np).to(dev)
        f = torch.from_numpy(f_np).to(dev)
        u0 = torch.from_numpy(u0_np).to(dev)
        op = F.Operator(k)
        x = torch.empty_like(u0)

        def bf16_step(cap=None):
            op.reassemble(k)
            x.copy_(u0)
            return F.solve(op, model, f, x, tol=1e-8, m_max=5, max_iter=cap or args.large_max_iter, prec="bf16",
                           check_every=16)

        def jac_step(cap=None):
            op.reassemble(k)
            x.copy_(u0)
            return F.solve_jacobi(op, 4, f, x, tol=1e-8, m_max=1, max_iter=cap or 50000, check_every=64)

        cell = {}
        ms, res = timed_steps(bf16_step, 1, 1, flush, stream, warm_fn=lambda: bf16_step(32))
        cell["bf16"] = solve_summary(ms, res, F)
        # the true residual of the returned iterates, from the library's own stencil
        Ax = torch.empty_like(x)
        op.apply(x, Ax)
        r_true = (f - Ax).flatten(1).norm(dim=1) / (f - _apply(op, u0)).flatten(1).norm(dim=1)
        cell["bf16"]["true_relres_max"] = float(r_true.max())
        ms, res = timed_steps(jac_step, 1, 1, flush, stream, warm_fn=lambda: jac_step(128))
        cell["jacobi4_pcg"] = solve_summary(ms, res, F)
        out[f"{N}x{B}"] = cell
        del op
    return out


def _apply(op, u):
    import torch
    y = torch.empty_like(u)
    op.apply(u, y)
    return y


def timed_steps(fn, steps, warmup, flush, stream, warm_fn=None):
    """Runs `warm_fn` (default fn) `warmup` times, then fn() `steps` times with L2 flushed
    before each, timing each call with CUDA events on `stream`. Returns (per-step ms,
    per-step results)."""
    import torch
    for _ in range(warmup):
        (warm_fn or fn)()
    torch.cuda.synchronize()
    ms, res = [], []
    for s_ in range(steps):
        flush.fill_(float(s_))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res.append(fn())
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms, res


def solve_summary(ms, infos, F):
    """solves/s (converged solves only), ms per step, iteration and residual statistics of the
    timed solves."""
    its = [i["iters"] for inf in infos for i in inf]
    rr = [i["relres"] for inf in infos for i in inf]
    conv = sum(1 for inf in infos for i in inf if i["status"] == F.FCGNO_OK)
    return {"value": conv / (sum(ms) / 1000.0), "unit": UNIT, "ms_per_step": float(np.mean(ms)), "steps": len(ms),
            "instances": len(infos[0]), "iterations": {"mean": float(np.mean(its)), "max": int(max(its))},
            "converged": conv, "solves": len(its), "relres_max": float(max(rr)),
            "relres_median": float(np.median(rr))}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2402_05598_gb300 import inputs as I
    cores = min(16, os.cpu_count() or 1)
    desc = I.ModelDesc(width=WIDTH, layers=LAYERS, modes=MODES, proj_width=WIDTH)
    blob = I.xavier_weights(desc, 0)
    iters = args.ref_iters
    vals = []
    for s in range(args.warmup + args.steps):
        wall, tot_it = oracle_sample(blob, cores, iters, cores, args.m, args.output_scale)
        if s >= args.warmup:
            vals.append((wall, tot_it))
    wall = sum(v[0] for v in vals)
    n_inst = cores * args.steps
    value = n_inst / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.m), "grid": N_GRID, "instances_per_gpu": EVAL_BATCH},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": cores,
                             "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                             "sample": f"{cores} instances per step, {iters} FCG-NO iterations each (the GPU arm's "
                                       f"iterations per solve), one single-threaded process per core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp16"])
    ap.add_argument("--m", type=int, default=5, help="truncation m of Algorithm 1 for the headline (5; m = 1 is "
                                                     "measured alongside)")
    ap.add_argument("--m-alt", type=int, default=1, help="second truncation reported next to the headline (0 = none)")
    ap.add_argument("--train-steps", type=int, default=48000)
    ap.add_argument("--train-prec", default="bf16", choices=["bf16", "fp32"],
                    help="arithmetic of the models' training steps (BF16 tensor cores or FP32 CUDA cores)")
    ap.add_argument("--train-leg", type=int, default=1, help="run the training-throughput leg (BF16 vs FP32)")
    ap.add_argument("--train-bench-steps", type=int, default=50)
    ap.add_argument("--train-compare-steps", type=int, default=4000,
                    help="steps of the two same-seed models (BF16, FP32) compared by eval iterations (0 = skip)")
    ap.add_argument("--train-instances", type=int, default=512)
    ap.add_argument("--max-iter", type=int, default=400,
                    help="iteration cap (CG needs ~400 on this workload); capped instances are not counted")
    ap.add_argument("--ref-iters", type=int, default=15,
                    help="FCG-NO iterations per oracle solve in the reference arm (the GPU arm measures a mean "
                         "of 14.7 at m = 5 on this workload)")
    ap.add_argument("--cpu-baseline", type=int, default=1)
    ap.add_argument("--transfer", type=int, default=1, help="run the resolution-transfer leg (128..512 grids)")
    ap.add_argument("--large", type=int, default=1, help="run the large-solve leg (1024^2 x 8, 2048^2 x 2, tol 1e-8)")
    ap.add_argument("--large-max-iter", type=int, default=3000)
    ap.add_argument("--large-train-steps", type=int, default=4000)
    ap.add_argument("--large-finetune-steps", type=int, default=600)
    ap.add_argument("--large-finetune-k", type=int, default=16)
    ap.add_argument("--large-finetune-lr", type=float, default=2e-4)
    ap.add_argument("--output-scale", type=int, default=1, choices=[0, 1],
                    help="model output scale: 0 = h^2 rms(r), 1 = h^2 rms(r) / k")
    ap.add_argument("--transfer-max-iter", type=int, default=2000)
    ap.add_argument("--transfer-fp64-instances", type=int, default=4,
                    help="instances per transfer cell solved by the all-FP64 FCG-NO (and the BF16 path, like for like)")
    ap.add_argument("--comparators", type=int, default=1,
                    help="time the all-FP64 FCG-NO, CG and Jacobi(4)-PCG on the headline's instances")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests in the serving stream (0 = skip the serving measurement)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="mean arrival rate of the serving stream (1/s)")
    ap.add_argument("--serve-m", type=int, default=1, help="truncation m of the served solves")
    ap.add_argument("--serve-requests-light", type=int, default=500, help="requests of the lighter stream")
    ap.add_argument("--mix-train-steps", type=int, default=16000)
    ap.add_argument("--mix-train-instances", type=int, default=768)
    ap.add_argument("--serve-rate-light", type=float, default=50.0,
                    help="arrival rate of a second, lighter serving stream (0 = skip)")
    ap.add_argument("--profile", type=int, default=0,
                    help="profiling mode: no training, two solves of --profile-iters fixed iterations")
    ap.add_argument("--profile-iters", type=int, default=8)
    ap.add_argument("--profile-grid", type=int, default=N_GRID, help="grid side of the profiling workload")
    ap.add_argument("--profile-batch", type=int, default=EVAL_BATCH, help="instances of the profiling workload")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world, device_id=dev)
    from paper_2402_05598_gb300 import fcgno as F
    from paper_2402_05598_gb300 import inputs as I
    from paper_2402_05598_gb300 import train as T
    from paper_2402_05598_gb300 import replicas as R

    # ---- setup: model, training (untimed)
    desc_np = I.ModelDesc(width=WIDTH, layers=LAYERS, modes=MODES, proj_width=WIDTH, output_scale=args.output_scale)
    blob = torch.from_numpy(I.xavier_weights(desc_np, 0)).to(dev)
    model = F.Model(F.make_desc(WIDTH, LAYERS, MODES, WIDTH, output_scale=args.output_scale), blob)
    tr = None
    if args.profile:
        # short fixed-iteration solves with every instance active (the ncu capture workload)
        seeds = range(10000, 10000 + args.profile_batch)
        k_np, f_np = I.make_batch(args.profile_grid, seeds)
        op = F.Operator(torch.from_numpy(k_np).to(dev))
        f = torch.from_numpy(f_np).to(dev)
        x = torch.zeros_like(f)
        for rep in range(2):
            x.zero_()
            info = F.solve(op, model, f, x, tol=TOL, m_max=args.m, max_iter=args.profile_iters, prec=args.prec,
                           fixed_iters=True, check_every=args.profile_iters)
        torch.cuda.synchronize()
        print(json.dumps({"profile": True, "iters": info[0]["iters"], "instances": args.profile_batch,
                          "grid": args.profile_grid, "launches": F.launch_count()}))
        return
    if args.train_steps > 0:
        tr = T.train(model, N_GRID, range(0, args.train_instances), K=100, batch=32, lr=1e-3, steps=args.train_steps,
                     log_every=1000, prec=args.train_prec)

    # ---- eval inputs (resident)
    seeds = R.rank_seeds(rank, EVAL_BATCH)
    k_np, f_np = I.make_batch(N_GRID, seeds)
    u0_np = np.stack([np.random.default_rng(s + 777).standard_normal((N_GRID, N_GRID)) for s in seeds])
    k = torch.from_numpy(k_np).to(dev)
    f = torch.from_numpy(f_np).to(dev)
    u0 = torch.from_numpy(u0_np).to(dev)
    op = F.Operator(k)
    x = torch.empty_like(u0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def solve_once(m=None, prec=None, model_=model):
        # one step: the operator assembled from k (in place), u_0 copied in, the batched solve
        op.reassemble(k)
        x.copy_(u0)
        return F.solve(op, model_, f, x, tol=TOL, m_max=args.m if m is None else m, max_iter=args.max_iter,
                       prec=args.prec if prec is None else prec, check_every=8)

    for _ in range(args.warmup):
        info = solve_once()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    # ---- timed region (untraced)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    launches0 = F.launch_count()
    step_ms, infos = timed_steps(solve_once, args.steps, 0, flush, stream)
    launches = F.launch_count() - launches0
    clk = clocks.stop()
    solved = sum(sum(1 for i in inf if i["status"] == F.FCGNO_OK) for inf in infos)
    total_ms, solved_all = R.reduce_timing(float(sum(step_ms)), solved, dev)
    iters = [i["iters"] for i in infos[-1]]
    # only solves that reached the tolerance count (capped instances are reported, not counted)
    value = solved_all / (total_ms / 1000.0)

    # ---- the synthesis launches of the same step, traced with CUDA events on their stream
    F.trace_set("tc_synthesis")
    F.trace_collect()
    trace_steps = 2
    for s_ in range(trace_steps):
        flush.fill_(float(s_))
        solve_once()
    syn_ms, syn_launches = F.trace_collect()
    trace_note = F.last_error() if "trace" in F.last_error() else ""
    F.trace_set("")

    # ---- the other configured truncation, same protocol (fewer timed steps)
    alt = None
    if args.m_alt and args.m_alt != args.m:
        alt_ms, alt_infos = timed_steps(lambda: solve_once(m=args.m_alt), 3, 2, flush, stream)
        alt_solved = sum(sum(1 for i in inf if i["status"] == F.FCGNO_OK) for inf in alt_infos)
        alt_total, alt_solved = R.reduce_timing(float(sum(alt_ms)), alt_solved, dev)
        alt_its = [i["iters"] for i in alt_infos[-1]]
        alt = {"m": args.m_alt, "value": alt_solved / (alt_total / 1000.0), "unit": UNIT, "steps": 3,
               "ms_per_step": alt_total / 3, "iterations": {"mean": float(np.mean(alt_its)), "max": int(max(alt_its))}}

    # ---- roofline of the dominant kernel (synthesis): algorithmic bytes / traced device time
    max_it = max(iters)
    active = [sum(1 for it in iters if it > i) for i in range(max_it)]
    alg_bytes_one, syn_per_step = roofline_synthesis(active, N_GRID, WIDTH, MODES, LAYERS, args.output_scale)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6800.0, "fallback"
    bf16_peak, bf16_src = 1700.0, "fallback (sustained)"
    if os.path.exists(peaks_path):
        with open(peaks_path) as fh:
            peaks = json.load(fh)
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
        if "bf16_tflops_sustained" in peaks:
            bf16_peak, bf16_src = float(peaks["bf16_tflops_sustained"]), "measured (sustained)"
    syn_avg_ms = syn_ms / max(syn_launches, 1)
    active_per_launch = float(sum(active)) * LAYERS * trace_steps / max(syn_launches, 1)
    traffic = SYN_TRAFFIC_PER_INSTANCE * active_per_launch if SYN_TRAFFIC_PER_INSTANCE else None
    achieved = alg_bytes_one * trace_steps / (syn_ms / 1000.0) / 1e9 if syn_ms > 0 else None
    # the same launches against the tensor pipe (the NO's work is dense contractions)
    syn_flops_one = synthesis_flops(active, N_GRID, WIDTH, MODES, LAYERS, WIDTH)
    t_ach, t_frac = rate_and_frac(syn_flops_one * trace_steps, syn_ms, 1e12, bf16_peak)
    intensity = syn_flops_one / alg_bytes_one if alg_bytes_one else None
    ceiling = intensity * peak / 1e3 if intensity else None  # TFLOP/s at the measured copy peak
    tensor_roofline = {"kernel": "tc_synthesis_kernel", "bound": "tensor", "unit": "TFLOP/s", "achieved": t_ach,
                       "peak": bf16_peak, "peak_source": bf16_src, "frac": t_frac,
                       "flops_per_launch": syn_flops_one * trace_steps / max(syn_launches, 1),
                       "intensity_flop_per_byte": intensity, "ceiling_at_hbm_peak": ceiling,
                       "frac_of_ceiling": (t_ach / ceiling) if (t_ach and ceiling) else None,
                       "note": "the activations pass through HBM, so the HBM roof caps the tensor pipe at "
                               "ceiling_at_hbm_peak"}

    # ---- kernel shares over one more (untimed) step per family
    shares, raw = {}, {}
    for fam in ("tc_synthesis", "tc_analysis", "tc_mix", "tc_lift", "fcg_fused"):
        F.trace_set(fam)
        F.trace_collect()
        solve_once()
        ms, cnt = F.trace_collect()
        shares[fam] = {"ms": round(ms, 3), "launches": cnt}
        raw[fam] = (ms, cnt)
    F.trace_set("")

    # ---- the fused FCG step against the FP64 roof (measured here; no vendor figure exists).
    # Step average: the traced step above, whose late launches hold few active instances.
    # Full occupancy: a traced solve of 2 (m + 1) fixed iterations, every instance active.
    fp64 = measure_fp64_roof(dev, stream)
    n_pts = N_GRID * N_GRID
    fused_ms, fused_cnt = raw["fcg_fused"]
    step_flops = 2.0 * fcg_step_fmas(iters, n_pts, args.m)
    k_full = 2 * (args.m + 1)
    F.trace_set("fcg_fused")
    F.trace_collect()
    x.copy_(u0)
    F.solve(op, model, f, x, tol=TOL, m_max=args.m, max_iter=k_full, prec=args.prec, fixed_iters=True,
            check_every=8)
    full_ms, full_cnt = F.trace_collect()
    F.trace_set("")
    full_flops = 2.0 * fcg_step_fmas([k_full] * EVAL_BATCH, n_pts, args.m)
    step_bytes = fcg_step_bytes(iters, n_pts, args.m)
    full_bytes = fcg_step_bytes([k_full] * EVAL_BATCH, n_pts, args.m)

    def fp64_leg(flops, nbytes, ms, cnt):
        ach = flops / (ms / 1000.0) / 1e12 if ms > 0 else None
        gbs, gfrac = rate_and_frac(nbytes, ms, 1e9, peak)
        return {"achieved": ach, "frac": (ach / fp64["tflops"]) if ach else None,
                "frac_of_nominal": (ach / FP64_NOMINAL_TFLOPS) if ach else None, "launches": cnt,
                "avg_launch_ms": ms / max(cnt, 1), "flops_per_launch": flops / max(cnt, 1),
                "hbm_gbs": gbs, "hbm_frac": gfrac, "bytes_per_launch": nbytes / max(cnt, 1)}

    fp64_roofline = {"kernel": "fused_step_kernel", "bound": "fp64", "unit": "TFLOP/s", "peak": fp64["tflops"],
                     "peak_source": "measured here (" + fp64["how"] + ")", "peak_median": fp64["tflops_median"],
                     "peak_nominal": FP64_NOMINAL_TFLOPS,
                     "flops_per_unknown": "2 (10 + 2 m_i) per active instance and iteration",
                     "bytes_per_unknown": "72 + 16 m_i per active instance and iteration (hbm_frac: of the "
                                          "measured copy peak)",
                     "step_average": fp64_leg(step_flops, step_bytes, fused_ms, fused_cnt),
                     "full_occupancy": dict(fp64_leg(full_flops, full_bytes, full_ms, full_cnt), iterations=k_full)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if args.prec == "bf16" else "f16", "data": "synthetic",
            "config": {"workload": workload_name(args.m), "grid": N_GRID, "instances_per_gpu": EVAL_BATCH,
                       "l2": "flushed (256 MB write) between timed steps",
                       "training": None if tr is None else {"steps": tr.steps, "batch": 32, "instances":
                                                            args.train_instances, "krylov_K": 100,
                                                            "prec": args.train_prec,
                                                            "seconds": round(tr.seconds, 2),
                                                            "loss_log": [(s_, round(l_, 4)) for s_, l_ in tr.losses]},
                       "max_iter": args.max_iter,
                       "parallelism": f"replicas x{world}"},
            "iterations": {"mean": float(np.mean(iters)), "max": int(max(iters)), "converged": solved,
                           "solves": EVAL_BATCH * args.steps},
            "unknowns_iterations_per_s": float(np.sum(iters)) * N_GRID * N_GRID * world / (step_ms[-1] / 1000.0),
            "gpu_launches": int(launches),
            "clocks": clk,
            "roofline": {"kernel": "tc_synthesis_kernel", "bound": "hbm", "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "traffic_note": "ncu dram read+write per active instance x active instances per launch",
                         "algorithmic_bytes_per_launch": alg_bytes_one * trace_steps / max(syn_launches, 1),
                         "avg_launch_ms": syn_avg_ms, "launches": syn_launches,
                         "note": trace_note or None},
            "kernel_ms_one_step": shares,
            "fp64_roofline": fp64_roofline,
            "tensor_roofline": tensor_roofline,
            "other_truncation": alt}

    # ---- comparison paths on the same 256 instances, same protocol (assembly + solve per step,
    # CUDA events on the launching stream, L2 flushed before each timed step)
    if rank == 0 and args.comparators:
        def fp64_step():
            return solve_once(prec="fp64")

        def cg_step():
            op.reassemble(k)
            x.copy_(u0)
            return F.solve(op, None, f, x, tol=TOL, m_max=1, max_iter=20000, prec="fp64", check_every=16)

        def jac_step():
            op.reassemble(k)
            x.copy_(u0)
            return F.solve_jacobi(op, 4, f, x, tol=TOL, m_max=1, max_iter=20000, check_every=16)

        ms, res = timed_steps(fp64_step, 1, 1, flush, stream)
        line["fp64_no"] = dict(solve_summary(ms, res, F), m=args.m, preconditioner="FP64 CUDA-core NO (same weights)")
        ms, res = timed_steps(cg_step, 2, 1, flush, stream)
        line["cg"] = dict(solve_summary(ms, res, F), m=1, preconditioner="identity")
        # Jacobi(4)-preconditioned CG (Eq. (15), the Jacobi column of Table 1)
        ms, res = timed_steps(jac_step, 2, 1, flush, stream)
        line["jacobi4_pcg"] = dict(solve_summary(ms, res, F), m=1, preconditioner="Jacobi(4), Eq. (15)")

    # ---- training throughput, BF16 tensor cores against FP32 CUDA cores
    if rank == 0 and args.train_leg:
        def eval_iters(m_):
            res = solve_once(model_=m_)
            return [i["iters"] for i in res], sum(1 for i in res if i["status"] == F.FCGNO_OK)
        line["train"] = run_train_leg(args, desc_np, dev, eval_iters)

    # ---- the model served and transferred: trained at 64 x 64 on the sigma mixture the
    # serving stream and the transfer configuration draw (0.5, 1, 2)
    model_mix, tr_mix = None, None
    if rank == 0 and (args.transfer or args.serve_requests > 0):
        blob_mix = torch.from_numpy(I.xavier_weights(desc_np, 2)).to(dev)
        model_mix = F.Model(F.make_desc(WIDTH, LAYERS, MODES, WIDTH, output_scale=args.output_scale), blob_mix)
        tr_mix = T.train(model_mix, N_GRID, range(0, args.mix_train_instances), K=100, batch=32, lr=1e-3,
                         steps=args.mix_train_steps, sigma=SERVE_SIGMAS, prec=args.train_prec)
        line["config"]["training_mix"] = {"steps": tr_mix.steps, "batch": 32, "instances": args.mix_train_instances,
                                          "sigmas": list(SERVE_SIGMAS), "seconds": round(tr_mix.seconds, 2),
                                          "prec": args.train_prec}
    # ---- resolution transfer (128..512 grids, sigma 0.5 / 1 / 2)
    if rank == 0 and args.transfer:
        line["transfer"] = run_transfer(args, model_mix, dev, flush, stream)
    # ---- large single solves (1024^2 x 8, 2048^2 x 2, sigma 2, length 0.05, tol 1e-8)
    if rank == 0 and args.large:
        line["large"] = run_large(args, dev, flush, stream)

    # ---- serving stream: continuous batching over size buckets (latency incl. queueing)
    if rank == 0 and args.serve_requests > 0:
        # the configured stream (offered load above what one GPU sustains: latency grows with
        # the queue) and a lighter stream that the GPU keeps up with
        line["serve"] = run_serving(args, model_mix, desc_np, dev, args.serve_rate, args.serve_requests)
        if args.serve_rate_light > 0:
            line["serve_light"] = run_serving(args, model_mix, desc_np, dev, args.serve_rate_light,
                                              args.serve_requests_light)

    # ---- end to end through the host-buffer entry point
    kh = torch.from_numpy(k_np).pin_memory()
    fh = torch.from_numpy(f_np).pin_memory()
    xh = torch.from_numpy(u0_np).pin_memory()
    e2e_t = 0.0
    for s in range(args.e2e_steps + 1):
        xh.copy_(torch.from_numpy(u0_np))
        t0 = time.perf_counter()
        F.solve_host(kh.numpy(), fh.numpy(), xh.numpy(), model, tol=TOL, m_max=args.m, max_iter=args.max_iter,
                     prec=args.prec, check_every=4)
        if s > 0:
            e2e_t += time.perf_counter() - t0
    vec = EVAL_BATCH * N_GRID * N_GRID * 8
    line["e2e"] = {"value": EVAL_BATCH * world * args.e2e_steps / e2e_t, "unit": UNIT,
                   "h2d_bytes_per_step": 3 * vec, "d2h_bytes_per_step": vec}

    # ---- CPU oracle baseline (bounded sample)
    if rank == 0 and args.cpu_baseline:
        cores = min(16, os.cpu_count() or 1)
        it_solve = max(1, int(round(np.mean(iters))))
        # the oracle's cost per iteration does not depend on the weight values: it runs the seeded
        # initial weights (no value produced by the CUDA path enters the oracle)
        wall, tot_it = oracle_sample(I.xavier_weights(desc_np, 0), cores, it_solve, cores, args.m, args.output_scale)
        line["cpu_baseline"] = {"kind": "oracle", "value": cores / wall, "unit": UNIT, "cores": cores,
                                "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                                "sample": f"{cores} instances, {it_solve} FCG-NO iterations each (the GPU solve's "
                                          f"mean iterations per solve), FP64 numpy oracle, one single-threaded "
                                          f"process per core"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
