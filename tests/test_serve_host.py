"""Host logic of the serving loop (no GPU): admission into free slots, first come first
served per grid size, retirement at each solve's own stop, one completion per request, and
the HBM-budget split of the bucket capacities. The buckets and the CUDA stream/event API
are host-side fakes with the same calls as fcgno.Bucket and torch.cuda."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def S():
    """The serve module (it loads the library: build it first, host-only)."""
    from paper_2402_05598_gb300 import build
    build.build()
    from paper_2402_05598_gb300 import serve
    return serve


class FakeStream:
    def wait_stream(self, other):
        pass

    def synchronize(self):
        pass


class FakeEvent:
    def record(self, stream):
        pass

    def query(self):
        return True


class FakeCuda:
    Stream = FakeStream
    Event = FakeEvent

    @staticmethod
    def current_stream():
        return FakeStream()

    @staticmethod
    def synchronize():
        pass


class FakeBucket:
    """A slot runs for the number of iterations its request asks for (stored in `k`), in
    steps of iters_per_step, or stops at max_iter; status -1 = running."""
    log = []

    def __init__(self, N, cap, model, prec, m_max, tol, max_iter, iters_per_step, stream):
        self.N, self.cap, self.max_iter, self.g = N, cap, max_iter, iters_per_step
        self.need = [0] * cap
        self.it = [0] * cap
        self.state = ["free"] * cap

    def admit(self, slot, k, f, x0, stream=None):
        assert self.state[slot] == "free", "slot admitted twice"
        self.state[slot] = "run"
        self.need[slot], self.it[slot] = int(k), 0
        self.owner = getattr(self, "owner", [None] * self.cap)
        self.owner[slot] = x0
        FakeBucket.log.append(("admit", self.N, int(f)))

    def step(self, stream=None):
        for s in range(self.cap):
            if self.state[s] == "run":
                self.it[s] = min(self.it[s] + self.g, self.need[s], self.max_iter)
                if self.it[s] >= self.need[s] or self.it[s] >= self.max_iter:
                    self.state[s] = "done"

    def poll(self, stream=None):
        st = np.array([-1 if x == "run" else (0 if self.it[i] >= self.need[i] else 4) if x == "done" else 0
                       for i, x in enumerate(self.state)], dtype=np.int32)
        return st, np.array(self.it, dtype=np.int32), np.zeros(self.cap)

    def take(self, slot, x_out=None, stream=None):
        assert self.state[slot] == "done"
        # a retired solve's iterate is delivered into its own request's buffer (x0 here)
        assert x_out is not None and x_out == self.owner[slot]
        FakeBucket.log.append(("take", self.N, x_out[1]))
        self.state[slot] = "free"

    def close(self):
        pass


def test_serve_loop_admits_retires_and_completes_each_request_once(S):
    rng = np.random.default_rng(0)
    FakeBucket.log = []
    sizes = (64, 128)
    reqs = []
    for i in range(60):
        N = int(rng.choice(sizes))
        need = int(rng.integers(1, 40)) if i != 7 else 10_000  # one request runs into max_iter
        reqs.append(S.Request(i, 0.0002 * i, N, need, i, ("x0", i)))
    srv = S.Server(None, {64: 3, 128: 2}, prec="bf16", max_iter=200, iters_per_step=8,
                   bucket_factory=FakeBucket, cuda=FakeCuda)
    stats = srv.run(reqs, S.ServeStats())
    assert stats.completed == len(reqs) and len(stats.latencies_ms) == len(reqs)
    assert stats.converged == len(reqs) - 1
    for r in reqs:
        assert r.done >= r.arrival and r.status in (0, 4)
        assert r.iters == (min(r.k, 200) if r.status == 0 else 200)
    assert reqs[7].status == 4
    # every request's result was delivered exactly once
    taken = sorted(rid for kind, n, rid in FakeBucket.log if kind == "take")
    assert taken == list(range(len(reqs)))
    # first come, first served within each grid size
    for N in sizes:
        order = [rid for kind, n, rid in FakeBucket.log if kind == "admit" and n == N]
        assert order == sorted(order) and len(order) == sum(1 for r in reqs if r.N == N)


def test_capacity_plan_respects_the_budget_and_the_offered_mix(S):
    from paper_2402_05598_gb300 import fcgno as F
    desc = F.make_desc(32, 4, 12, 32)
    mix = {64: 0.40, 128: 0.25, 256: 0.20, 512: 0.10, 1024: 0.05}
    budget = 8 * 2**30
    caps = S.plan_capacities(mix, budget, 1, desc, "bf16", max_slots=10_000)
    used = sum(cap * S.slot_bytes(N, 1, desc, "bf16") for N, cap in caps.items())
    assert used <= budget and all(c >= 1 for c in caps.values())
    # each size's share of the budget follows its share of the offered unknowns (within one slot)
    tot = sum(w * N * N for N, w in mix.items())
    for N, cap in caps.items():
        share = budget * mix[N] * N * N / tot
        assert cap * S.slot_bytes(N, 1, desc, "bf16") <= share < (cap + 1) * S.slot_bytes(N, 1, desc, "bf16")
    capped = S.plan_capacities(mix, budget, 1, desc, "bf16", max_slots=16)
    assert max(capped.values()) <= 16


class FaultyBucket(FakeBucket):
    """FakeBucket with host-injected faults: admitting request 13 fails with FCGNO_ENOMEM, and
    the third poll of the 128 x 128 bucket reports FCGNO_ETIMEOUT (its running solves are
    recorded in `timed_out`)."""
    polls = {}
    timed_out = set()

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.rid = [None] * self.cap

    def admit(self, slot, k, f, x0, stream=None):
        from paper_2402_05598_gb300 import fcgno as F
        if int(f) == 13:
            raise F.FcgnoError(F.FCGNO_ENOMEM, "fcgno_bucket_admit")
        super().admit(slot, k, f, x0, stream)
        self.rid[slot] = int(f)

    def poll(self, stream=None):
        from paper_2402_05598_gb300 import fcgno as F
        n = FaultyBucket.polls.get(self.N, 0) + 1
        FaultyBucket.polls[self.N] = n
        if self.N == 128 and n == 3:
            FaultyBucket.timed_out |= {self.rid[s] for s in range(self.cap) if self.state[s] != "free"}
            raise F.FcgnoError(F.FCGNO_ETIMEOUT, "fcgno_bucket_poll")
        return super().poll(stream)

    def take(self, slot, x_out=None, stream=None):
        self.state[slot] = "free"
        self.rid[slot] = None


def test_serve_loop_survives_host_injected_faults(S):
    """A rejected admission completes that request with its status and leaves the slot free; a
    timed-out step completes the bucket's running solves with FCGNO_ETIMEOUT; every other
    request is served as usual and each completes exactly once."""
    from paper_2402_05598_gb300 import fcgno as F
    rng = np.random.default_rng(1)
    FakeBucket.log = []
    FaultyBucket.polls, FaultyBucket.timed_out = {}, set()
    reqs = [S.Request(i, 0.0002 * i, int(rng.choice((64, 128))), int(rng.integers(1, 30)), i, None)
            for i in range(50)]
    srv = S.Server(None, {64: 3, 128: 2}, prec="bf16", max_iter=200, iters_per_step=8,
                   bucket_factory=FaultyBucket, cuda=FakeCuda)
    stats = srv.run(reqs, S.ServeStats())
    assert stats.completed == len(reqs) and len(stats.latencies_ms) == len(reqs)
    timed_out = FaultyBucket.timed_out
    assert timed_out and 13 not in timed_out
    assert reqs[13].status == F.FCGNO_ENOMEM and reqs[13].iters == 0
    for r in reqs:
        if r.rid in timed_out:
            assert r.status == F.FCGNO_ETIMEOUT and r.N == 128
        elif r.rid != 13:
            assert r.status == 0 and r.iters == r.k
    assert stats.failed == 1 + len(timed_out)
    assert stats.converged == len(reqs) - stats.failed
    # the 128 x 128 bucket went on serving after its timed-out step
    late = [r for r in reqs if r.N == 128 and r.rid not in timed_out and r.done > min(
        reqs[i].done for i in timed_out)]
    assert late and all(r.status == 0 for r in late)


class FakeServeBucket:
    """Host model of a device-driven bucket: at every iteration boundary, slots whose request
    reached its iteration count (stored in `k`) or max_iter publish a result and free up, then
    free slots take queued requests in order; running slots advance one iteration."""
    admitted = []

    def __init__(self, N, cap, model, prec, m_max, tol, max_iter, iters_per_step, stream):
        self.N, self.cap, self.max_iter, self.g = N, cap, max_iter, iters_per_step
        self.slots = [None] * cap  # [tag, need, iters]

    def serve_enable(self, qcap, dcap):
        from collections import deque
        self.qcap, self.queue, self.out = qcap, deque(), []

    def enqueue(self, k, f, x0, x_out, tag):
        if len(self.queue) >= self.qcap:
            return False
        self.queue.append((tag, int(k)))
        return True

    def step(self, stream=None):
        for _ in range(self.g):
            for i, s in enumerate(self.slots):
                if s is not None and (s[2] >= s[1] or s[2] >= self.max_iter):
                    self.out.append((s[0], 0 if s[2] >= s[1] else 4, s[2], 0.0))
                    self.slots[i] = None
            for i in range(self.cap):
                if self.slots[i] is None and self.queue:
                    tag, need = self.queue.popleft()
                    FakeServeBucket.admitted.append((self.N, tag))
                    self.slots[i] = [tag, need, 0]
            for s in self.slots:
                if s is not None:
                    s[2] += 1

    def results(self):
        out, self.out = self.out, []
        return out

    def close(self):
        pass


def test_device_server_enqueues_collects_and_completes_each_request_once(S):
    """The device-driven loop: requests are appended to their bucket's queue (a small queue
    keeps some waiting on the host), steps are issued only while a bucket has unfinished
    requests, and every result is collected once; admission is first in, first out per size."""
    rng = np.random.default_rng(3)
    FakeServeBucket.admitted = []
    reqs = []
    for i in range(80):
        N = int(rng.choice((64, 128)))
        need = int(rng.integers(1, 40)) if i != 11 else 10_000
        reqs.append(S.Request(i, 0.0001 * i, N, need, i, ("x0", i)))
    srv = S.DeviceServer(None, {64: 3, 128: 2}, prec="bf16", max_iter=200, iters_per_step=4, queue_capacity=4,
                         bucket_factory=FakeServeBucket, cuda=FakeCuda)
    stats = srv.run(reqs, S.ServeStats())
    assert stats.completed == len(reqs) and len(stats.latencies_ms) == len(reqs)
    assert reqs[11].status == 4 and reqs[11].iters == 200
    for r in reqs:
        assert r.done >= r.arrival
        if r.rid != 11:
            assert r.status == 0 and r.iters == r.k
    for N in (64, 128):
        order = [tag for n, tag in FakeServeBucket.admitted if n == N]
        assert order == sorted(order) and len(order) == sum(1 for r in reqs if r.N == N)
