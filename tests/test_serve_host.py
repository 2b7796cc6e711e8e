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
        reqs.append(S.Request(i, 0.0002 * i, N, need, i, None))
    srv = S.Server(None, {64: 3, 128: 2}, prec="bf16", max_iter=200, iters_per_step=8,
                   bucket_factory=FakeBucket, cuda=FakeCuda)
    stats = srv.run(reqs, S.ServeStats())
    assert stats.completed == len(reqs) and len(stats.latencies_ms) == len(reqs)
    assert stats.converged == len(reqs) - 1
    for r in reqs:
        assert r.done >= r.arrival and r.status in (0, 4)
        assert r.iters == (min(r.k, 200) if r.status == 0 else 200)
    assert reqs[7].status == 4
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
