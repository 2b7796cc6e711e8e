"""Serving buckets (continuous batching): a solve's result does not depend on the other
slots of its bucket, on when it was admitted, or on slots admitted and retired around it."""
import numpy as np
import pytest

from oracle import fcgno_oracle as O
from paper_2402_05598_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def dev_arrays(N, seed, dev):
    import torch
    k, f = I.make_problem(N, seed)
    x0 = np.random.default_rng(seed + 777).standard_normal((N, N))
    return tuple(torch.from_numpy(a).to(dev) for a in (k, f, x0))


def run_alone(lib, dev, model, N, seed, prec, steps, **kw):
    import torch
    bk = lib.Bucket(N, 4, model, prec=prec, iters_per_step=8, **kw)
    k, f, x0 = dev_arrays(N, seed, dev)
    bk.admit(0, k, f, x0)
    for _ in range(steps):
        bk.step()
    st, it, rr = bk.poll()
    x = torch.empty((N, N), dtype=torch.float64, device=dev)
    bk.take(0, x)
    torch.cuda.synchronize()
    return x.cpu().numpy(), int(it[0]), float(rr[0]), int(st[0])


def run_in_mix(lib, dev, model, N, seed, prec, steps, **kw):
    """The same request admitted into slot 2 after two steps of other traffic; another
    request joins one step later and one leaves while ours runs."""
    import torch
    bk = lib.Bucket(N, 4, model, prec=prec, iters_per_step=8, **kw)
    a = dev_arrays(N, seed + 1, dev)
    c = dev_arrays(N, seed + 2, dev)
    d = dev_arrays(N, seed + 3, dev)
    bk.admit(1, *a)
    bk.step()
    bk.admit(3, *d)
    bk.step()
    k, f, x0 = dev_arrays(N, seed, dev)
    bk.admit(2, k, f, x0)
    for s in range(steps):
        bk.step()
        if s == 0:
            bk.admit(0, *c)
        if s == 1:
            bk.take(3)  # a neighbour retires early
    st, it, rr = bk.poll()
    x = torch.empty((N, N), dtype=torch.float64, device=dev)
    bk.take(2, x)
    torch.cuda.synchronize()
    return x.cpu().numpy(), int(it[2]), float(rr[2]), int(st[2])


@pytest.mark.parametrize("prec,C,M,N", [("bf16", 32, 12, 64), ("fp64", 16, 8, 32)])
def test_result_is_the_same_alone_and_in_the_mix(lib, dev, prec, C, M, N):
    import torch
    desc = I.ModelDesc(width=C, layers=4, modes=M, proj_width=C)
    w = torch.from_numpy(I.xavier_weights(desc, 4)).to(dev)
    model = lib.Model(lib.make_desc(C, 4, M, C), w)
    xa, ia, ra, sa = run_alone(lib, dev, model, N, 3000, prec, 3, max_iter=24)
    xb, ib, rb, sb = run_in_mix(lib, dev, model, N, 3000, prec, 3, max_iter=24)
    assert ia == ib == 24 and sa == sb == lib.FCGNO_ENOCONV
    assert np.array_equal(xa, xb)
    assert ra == rb


def test_bucket_slot_matches_oracle_cg_and_stops_itself(lib, dev):
    """Identity preconditioner: a slot converges on its own (status FCGNO_OK), with the
    oracle's iteration count, while a neighbour keeps running."""
    import torch
    N = 24
    bk = lib.Bucket(N, 3, None, prec="fp64", tol=1e-8, max_iter=5000, iters_per_step=8)
    k, f, x0 = dev_arrays(N, 3100, dev)
    other = dev_arrays(N, 3101, dev)
    bk.admit(1, *other)
    bk.step()
    bk.admit(0, k, f, x0)
    for _ in range(400):
        bk.step()
        st, it, rr = bk.poll()
        if st[0] != -1:
            break
    assert st[0] == lib.FCGNO_OK
    x = torch.empty((N, N), dtype=torch.float64, device=dev)
    bk.take(0, x)
    kn, fn, x0n = (t.cpu().numpy() for t in (k, f, x0))
    ref = O.fcg(lambda u: O.apply_A(kn, u), lambda r: r, fn, x0n, 1, 5000, tol=1e-8)
    assert abs(int(it[0]) - ref["iterations"]) <= max(2, ref["iterations"] // 100)
    assert rr[0] <= 1e-8
    true_res = np.linalg.norm(fn - O.apply_A(kn, x.cpu().numpy())) / np.linalg.norm(fn - O.apply_A(kn, x0n))
    assert true_res < 1e-7


def test_concurrent_buckets_sharing_a_model_match_alone(lib, dev):
    """Buckets of two grid sizes that share one BF16 model step concurrently on their own
    streams (as the serving loop runs them): each slot's result equals its result when its
    bucket runs alone. The preconditioner's activations belong to each bucket's operator, so
    the concurrent steps cannot overwrite each other's."""
    import torch
    C, M = 32, 12
    desc = I.ModelDesc(width=C, layers=4, modes=M, proj_width=C)
    w = torch.from_numpy(I.xavier_weights(desc, 5)).to(dev)
    model = lib.Model(lib.make_desc(C, 4, M, C), w)
    sizes = (64, 128)
    alone = {N: run_alone(lib, dev, model, N, 3300 + N, "bf16", 3, max_iter=24) for N in sizes}
    streams = {N: torch.cuda.Stream() for N in sizes}
    bks = {N: lib.Bucket(N, 4, model, prec="bf16", iters_per_step=8, max_iter=24, stream=streams[N]) for N in sizes}
    for N in sizes:
        streams[N].wait_stream(torch.cuda.current_stream())
        bks[N].admit(0, *dev_arrays(N, 3300 + N, dev), stream=streams[N])
    for _ in range(3):
        for N in sizes:
            bks[N].step(stream=streams[N])
    for N in sizes:
        st, it, rr = bks[N].poll(stream=streams[N])
        x = torch.empty((N, N), dtype=torch.float64, device=dev)
        with torch.cuda.stream(streams[N]):
            bks[N].take(0, x, stream=streams[N])
        streams[N].synchronize()
        xa, ia, ra, sa = alone[N]
        assert int(it[0]) == ia == 24 and int(st[0]) == sa
        assert np.array_equal(x.cpu().numpy(), xa)
        assert float(rr[0]) == ra


def test_server_delivers_each_result_as_solved_alone(lib, dev):
    """The request loop copies every retired solve's iterate into its request's output
    tensor: each delivered result equals the same request solved alone in its own bucket,
    bit for bit, although the requests shared buckets of two sizes and overlapped in time."""
    import torch
    from paper_2402_05598_gb300 import serve as S
    C, M = 32, 12
    desc = I.ModelDesc(width=C, layers=4, modes=M, proj_width=C)
    w = torch.from_numpy(I.xavier_weights(desc, 6)).to(dev)
    model = lib.Model(lib.make_desc(C, 4, M, C), w)
    reqs = []
    for i in range(6):
        N = (64, 128)[i % 2]
        k, f, x0 = dev_arrays(N, 3400 + i, dev)
        out = torch.full((N, N), float("nan"), dtype=torch.float64, device=dev)
        reqs.append(S.Request(i, 0.002 * i, N, k, f, x0, out=out))
    srv = S.Server(model, {64: 2, 128: 2}, prec="bf16", max_iter=24, iters_per_step=8)
    stats = srv.run(reqs, S.ServeStats())
    srv.close()
    assert stats.completed == len(reqs)
    for i, r in enumerate(reqs):
        xa, ia, ra, sa = run_alone(lib, dev, model, r.N, 3400 + i, "bf16", 3, max_iter=24)
        assert r.iters == ia == 24 and r.status == sa == lib.FCGNO_ENOCONV
        assert np.array_equal(r.out.cpu().numpy(), xa), i


def test_device_driven_serving_matches_solves_alone(lib, dev):
    """Admission and retirement on the device (fcgno_bucket_serve_enable): requests of two grid
    sizes, more than the slots, queued through the mapped queue while steps run; every result
    equals the same request solved alone in a host-driven bucket, bit for bit (the admission
    assembles and forms r_0 with the same arithmetic, and a slot's solve does not depend on
    the others), and is published only after its x_out holds the iterate."""
    import torch
    from paper_2402_05598_gb300 import serve as S
    C, M = 32, 12
    desc = I.ModelDesc(width=C, layers=4, modes=M, proj_width=C, output_scale=1)
    w = torch.from_numpy(I.xavier_weights(desc, 7)).to(dev)
    model = lib.Model(lib.make_desc(C, 4, M, C, output_scale=1), w)
    reqs = []
    for i in range(9):
        N = (64, 128)[i % 2]
        k, f, x0 = dev_arrays(N, 3500 + i, dev)
        out = torch.full((N, N), float("nan"), dtype=torch.float64, device=dev)
        reqs.append(S.Request(i, 0.001 * i, N, k, f, x0, out=out))
    srv = S.DeviceServer(model, {64: 2, 128: 2}, prec="bf16", max_iter=24, iters_per_step=8)
    stats = srv.run(reqs, S.ServeStats())
    srv.close()
    assert stats.completed == len(reqs)
    for i, r in enumerate(reqs):
        xa, ia, ra, sa = run_alone(lib, dev, model, r.N, 3500 + i, "bf16", 3, max_iter=24)
        assert r.iters == ia == 24 and r.status == lib.FCGNO_ENOCONV, (i, r.iters, r.status)
        assert np.array_equal(r.out.cpu().numpy(), xa), i
        assert r.relres == ra


def test_device_driven_identity_solves_match_oracle_cg_and_queue_limits(lib, dev):
    """Identity preconditioner through the device queue: each request converges on its own with
    the oracle's CG iteration count (within 1 %) and true residual; a full queue refuses the
    next request until the device has taken some."""
    import torch
    N = 24
    bk = lib.Bucket(N, 2, None, prec="fp64", tol=1e-8, max_iter=5000, iters_per_step=8)
    bk.serve_enable(3, 8)
    probs = [dev_arrays(N, 3600 + i, dev) for i in range(4)]
    outs = [torch.empty((N, N), dtype=torch.float64, device=dev) for _ in probs]
    assert all(bk.enqueue(*probs[i], outs[i], i) for i in range(3))
    assert not bk.enqueue(*probs[3], outs[3], 3)  # queue of 3 is full until a step takes requests
    done = {}
    pending3 = True
    for _ in range(2000):
        bk.step()
        torch.cuda.synchronize()
        for tag, st, it, rr in bk.results():
            done[tag] = (st, it, rr)
        if pending3 and bk.enqueue(*probs[3], outs[3], 3):
            pending3 = False
        if len(done) == 4:
            break
    assert len(done) == 4
    for i in range(4):
        kn, fn, x0n = (t.cpu().numpy() for t in probs[i])
        st, it, rr = done[i]
        ref = O.fcg(lambda u: O.apply_A(kn, u), lambda r: r, fn, x0n, 1, 5000, tol=1e-8)
        assert st == lib.FCGNO_OK and abs(it - ref["iterations"]) <= max(2, ref["iterations"] // 100)
        true = np.linalg.norm(fn - O.apply_A(kn, outs[i].cpu().numpy())) / np.linalg.norm(fn - O.apply_A(kn, x0n))
        assert true < 1e-7 and rr <= 1e-8
    bk.close()
