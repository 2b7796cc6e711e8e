"""Request loop for serving FCG-NO solves (continuous batching over size buckets).

Requests (grid size N, coefficient field k, right-hand side f, initial guess u_0) arrive
over time. Each grid size has one resident bucket (``fcgno.Bucket``) whose capacity was
admitted against an HBM budget when the server started. With the 16-bit preconditioner
every bucket runs on its own CUDA stream, so the steps of different grid sizes overlap on
the GPU and a small solve does not wait behind a large one. The loop repeatedly
  1. admits every arrived request whose bucket has a free slot (first come, first served;
     the others wait in their bucket's queue),
  2. starts one step (a few FCG-NO iterations, replayed as one CUDA graph) of every bucket
     that has running slots and no step in flight,
  3. for every bucket whose step has finished (an event query, no waiting), reads the slot
     states and retires finished slots (converged, breakdown, or capped): each retired
     slot's iterate is copied into its request's output tensor, and the request completes
     once that copy has finished.
Latency = completion time - arrival time (queueing and delivery of the result included). A request the library rejects
at admission (FcgnoError: bad input, no memory) completes at once with that status and its
slot stays free; when a bucket's poll reports FCGNO_ETIMEOUT (a bounded device wait gave up
during its step) every solve running in that bucket completes with that status and the
bucket goes on serving. Other library errors stop the loop.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import fcgno as F


@dataclass
class Request:
    """One solve request: arrival time, grid size, device inputs; the loop fills in the outcome."""
    rid: int
    arrival: float          # seconds from the start of the run
    N: int
    k: object               # device [N][N] float64
    f: object
    x0: object
    out: object = None      # device [N][N] float64 receiving the solution (None: written into x0)
    done: float = -1.0
    iters: int = 0
    status: int = -1
    relres: float = 0.0


@dataclass
class ServeStats:
    """Latencies and counts of one serving run."""
    latencies_ms: list = field(default_factory=list)
    completed: int = 0
    converged: int = 0
    wall_s: float = 0.0
    offered_rate: float = 0.0
    bucket_bytes: int = 0
    failed: int = 0

    def summary(self) -> dict:
        """p50/p99/mean latency (ms), served and offered rates, counts."""
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": self.completed, "converged": self.converged, "failed": self.failed,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "solves_per_s": self.completed / max(self.wall_s, 1e-9),
                "offered_per_s": self.offered_rate, "wall_s": self.wall_s, "bucket_bytes": self.bucket_bytes}


def slot_bytes(N: int, m_max: int, desc, prec: str) -> int:
    """Device bytes one resident solve of an N x N grid needs (solver state and operator)."""
    return F.workspace_bytes(N, 1, m_max, desc, prec) + 2 * 8 * N * N  # + iterate and right-hand side


def plan_capacities(sizes_weights: dict, budget_bytes: int, m_max: int, desc, prec: str, max_slots: int = 256) -> dict:
    """Split an HBM budget across buckets in proportion to each size's share of the offered
    unknowns (weight x N^2), capped at max_slots slots per bucket."""
    tot = sum(w * N * N for N, w in sizes_weights.items())
    caps = {}
    for N, w in sizes_weights.items():
        share = budget_bytes * (w * N * N) / tot
        caps[N] = int(max(1, min(max_slots, share // slot_bytes(N, m_max, desc, prec))))
    return caps


class Server:
    """``bucket_factory`` (default ``fcgno.Bucket``) and ``cuda`` (default ``torch.cuda``: Stream,
    Event, current_stream, synchronize) can be replaced, e.g. by host-side fakes that test the
    scheduling without a GPU."""

    def __init__(self, model, capacities: dict, prec="bf16", m_max=1, tol=1e-6, max_iter=400, iters_per_step=8,
                 bucket_factory=None, cuda=None):
        if cuda is None:
            import torch
            cuda = torch.cuda
        self.cuda = cuda
        bucket_factory = bucket_factory or F.Bucket
        # The CUDA-core FP64/FP32 preconditioner keeps its activations in the model, so its
        # buckets share one stream; the 16-bit path keeps them per operator (per bucket).
        concurrent = prec in ("bf16", "fp16")
        shared = cuda.Stream()
        self.streams = {N: (cuda.Stream() if concurrent else shared) for N in capacities}
        self.buckets = {N: bucket_factory(N, cap, model, prec=prec, m_max=m_max, tol=tol, max_iter=max_iter,
                                          iters_per_step=iters_per_step, stream=self.streams[N])
                        for N, cap in capacities.items()}
        self.slots = {N: [None] * cap for N, cap in capacities.items()}
        self.queues = {N: deque() for N in capacities}
        self.inflight = {N: None for N in capacities}  # event recorded after the bucket's last step

    @staticmethod
    def _complete(r, status, iters, relres, tnow, stats):
        r.done, r.iters, r.status, r.relres = tnow, int(iters), int(status), float(relres)
        stats.latencies_ms.append(1000.0 * (r.done - r.arrival))
        stats.completed += 1
        stats.converged += int(r.status == F.FCGNO_OK)

    def run(self, requests: list, stats: ServeStats) -> ServeStats:
        """Serves the requests (sorted by arrival) and returns latency statistics."""
        cuda = self.cuda
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        # requests reference device tensors made on the current stream: order the buckets'
        # streams after them
        for s_ in set(self.streams.values()):
            s_.wait_stream(cuda.current_stream())
        t0 = time.perf_counter()
        outstanding = len(pending)
        while outstanding:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                self.queues[r.N].append(r)
            # admit into free slots (ordered after the bucket's step in flight, if any)
            for N, q in self.queues.items():
                slots = self.slots[N]
                for i in range(len(slots)):
                    if not q:
                        break
                    if slots[i] is None:
                        r = q.popleft()
                        try:
                            self.buckets[N].admit(i, r.k, r.f, r.x0, stream=self.streams[N])
                        except F.FcgnoError as e:
                            # rejected by the library: completes now, the slot stays free
                            self._complete(r, e.code, 0, 0.0, time.perf_counter() - t0, stats)
                            stats.failed += 1
                            outstanding -= 1
                            continue
                        slots[i] = r
            # start a step of every bucket with running slots and no step in flight
            busy = [N for N, slots in self.slots.items() if any(s is not None for s in slots)]
            for N in busy:
                if self.inflight[N] is None:
                    self.buckets[N].step(stream=self.streams[N])
                    ev = cuda.Event()
                    ev.record(self.streams[N])
                    self.inflight[N] = ev
            # retire the slots of every bucket whose step has finished
            progressed = False
            for N, ev in self.inflight.items():
                if ev is None or not ev.query():
                    continue
                self.inflight[N] = None
                progressed = True
                try:
                    st, it, rr = self.buckets[N].poll(stream=self.streams[N])
                except F.FcgnoError as e:
                    if e.code != F.FCGNO_ETIMEOUT:
                        raise
                    # this bucket's step is invalid: its running solves complete with the status
                    tnow = time.perf_counter() - t0
                    for i, r in enumerate(self.slots[N]):
                        if r is not None:
                            self.buckets[N].take(i, stream=self.streams[N])
                            self._complete(r, e.code, 0, 0.0, tnow, stats)
                            stats.failed += 1
                            self.slots[N][i] = None
                            outstanding -= 1
                    continue
                retired = [i for i, r in enumerate(self.slots[N]) if r is not None and st[i] != -1]
                for i in retired:
                    r = self.slots[N][i]
                    self.buckets[N].take(i, r.out if r.out is not None else r.x0, stream=self.streams[N])
                if retired:
                    self.streams[N].synchronize()  # the results have been delivered
                tnow = time.perf_counter() - t0
                for i in retired:
                    self._complete(self.slots[N][i], st[i], it[i], rr[i], tnow, stats)
                    self.slots[N][i] = None
                    outstanding -= 1
            if not progressed:
                if not busy and pending:  # idle until the next arrival
                    time.sleep(max(0.0, min(0.001, pending[0].arrival - (time.perf_counter() - t0))))
                elif busy:
                    time.sleep(2e-5)
        cuda.synchronize()
        stats.wall_s = time.perf_counter() - t0
        return stats

    def close(self):
        for b in self.buckets.values():
            b.close()


class DeviceServer:
    """Continuous batching with admission and retirement on the device
    (``fcgno_bucket_serve_enable``): every iteration of every step retires the slots whose
    solve stopped (their iterate copied into the request's output, then the result published)
    and admits queued requests into free slots. The host only
      1. appends every arrived request to its bucket's queue (mapped host memory, no CUDA call;
         a full queue keeps the request waiting on the host),
      2. keeps up to ``depth`` steps in flight on each bucket that has unfinished requests,
      3. collects published results (mapped host memory) and completes their requests.
    It never waits for a step. Latency = time the host reads the result - arrival time.
    ``bucket_factory`` and ``cuda`` can be replaced by host-side fakes (tests)."""

    def __init__(self, model, capacities: dict, prec="bf16", m_max=1, tol=1e-6, max_iter=400, iters_per_step=4,
                 queue_capacity=None, depth=2, bucket_factory=None, cuda=None, stall_s=120.0):
        self.stall_s = stall_s
        if cuda is None:
            import torch
            cuda = torch.cuda
        self.cuda = cuda
        bucket_factory = bucket_factory or F.Bucket
        concurrent = prec in ("bf16", "fp16")
        shared = cuda.Stream()
        self.streams = {N: (cuda.Stream() if concurrent else shared) for N in capacities}
        self.buckets = {}
        for N, cap in capacities.items():
            bk = bucket_factory(N, cap, model, prec=prec, m_max=m_max, tol=tol, max_iter=max_iter,
                                iters_per_step=iters_per_step, stream=self.streams[N])
            qcap = queue_capacity or max(64, 4 * cap)
            bk.serve_enable(qcap, qcap + cap)
            self.buckets[N] = bk
        self.depth = depth
        self.inflight = {N: deque() for N in capacities}

    def run(self, requests: list, stats: ServeStats) -> ServeStats:
        """Serves the requests (sorted by arrival) and returns latency statistics."""
        cuda = self.cuda
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        for s_ in set(self.streams.values()):
            s_.wait_stream(cuda.current_stream())
        waiting = {N: deque() for N in self.buckets}
        queued = {N: 0 for N in self.buckets}    # enqueued, result not yet collected
        by_tag = {}
        t0 = time.perf_counter()
        outstanding = len(pending)
        last_result = t0
        while outstanding:
            now = time.perf_counter() - t0
            if any(queued.values()) and time.perf_counter() - last_result > self.stall_s:
                raise RuntimeError(f"serving: no result for {self.stall_s} s with requests queued: "
                                   f"queued={queued}, in flight={ {N: len(v) for N, v in self.inflight.items()} }")
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                waiting[r.N].append(r)
            progressed = False
            for N, bk in self.buckets.items():
                w = waiting[N]
                while w:
                    r = w[0]
                    try:
                        ok = bk.enqueue(r.k, r.f, r.x0, r.out if r.out is not None else r.x0, r.rid)
                    except F.FcgnoError as e:
                        w.popleft()
                        Server._complete(r, e.code, 0, 0.0, time.perf_counter() - t0, stats)
                        stats.failed += 1
                        outstanding -= 1
                        continue
                    if not ok:
                        break
                    w.popleft()
                    by_tag[r.rid] = r
                    queued[N] += 1
                    progressed = True
            for N, bk in self.buckets.items():
                inf = self.inflight[N]
                while inf and inf[0].query():
                    inf.popleft()
                if queued[N] > 0 and len(inf) < self.depth:
                    bk.step(stream=self.streams[N])
                    ev = cuda.Event()
                    ev.record(self.streams[N])
                    inf.append(ev)
                    progressed = True
            for N, bk in self.buckets.items():
                res = bk.results()
                if res:
                    last_result = time.perf_counter()
                    tnow = last_result - t0
                    for tag, st, it, rr in res:
                        r = by_tag.pop(tag)
                        Server._complete(r, st, it, rr, tnow, stats)
                        queued[N] -= 1
                        outstanding -= 1
                    progressed = True
            if not progressed:
                time.sleep(2e-5 if any(queued.values()) else max(0.0, min(0.001, (pending[0].arrival - now)
                                                                       if pending else 0.001)))
        cuda.synchronize()
        stats.wall_s = time.perf_counter() - t0
        return stats

    def close(self):
        self.cuda.synchronize()
        for b in self.buckets.values():
            b.close()
