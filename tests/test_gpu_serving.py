"""Serving form of the solver (continuous batching of Newton-step requests).

* every result is bit-identical whether its instance runs alone or mixed with
  other instances on other streams (each instance computes on its own buffers
  with fixed reduction orders);
* admission by device bytes: with a budget that holds one instance, a second
  instance waits until the first one is freed, and both finish;
* an instance larger than the whole budget is rejected at submit;
* eviction under memory pressure: an idle instance is evicted to the host and
  rebuilt from its saved state, and its results do not change;
* cancellation: a cancelled request completes with FSI_E_CANCELLED without
  advancing its instance, and the instance's other results do not change.
"""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1709_05660_gb300.workloads import Problem, SolverOpts, noise, problem_3d  # noqa: E402

# parameters inside the range where plain Newton with this smoother converges
# on these coarse meshes (U <= 0.3; the oracle fails at U >= 0.6 on 3 levels)
INSTANCES = [
    (11, Problem(levels=3, mu_s=1e5, U=0.3), SolverOpts(tile=(2, 2), precision=1)),
    (12, Problem(levels=3, mu_s=8e5, U=0.2), SolverOpts(tile=(2, 2), precision=0)),
    (13, Problem(levels=4, mu_s=3e4, U=0.15), SolverOpts(tile=(2, 2), precision=1)),
    (14, problem_3d(levels=2, mu_s=5e5, U=0.2), SolverOpts(tile=(2, 2, 2), precision=1)),
]
STEPS = 3


def _fsi():
    from paper_1709_05660_gb300 import fsi
    return fsi


def _n(prob):
    from paper_1709_05660_gb300 import fsi
    s = fsi.FSI(prob, SolverOpts(), plan_only=True)
    n = int(s.N[-1])
    s.close()
    return n


def _run(server, instances, order):
    """Submits STEPS requests per instance in the given interleaving."""
    tickets = {}
    sizes = {iid: _n(p) for iid, p, _ in instances}
    step = {iid: 0 for iid, _, _ in instances}
    spec = {iid: (p, o) for iid, p, o in instances}
    for iid in order:
        p, o = spec[iid]
        k = step[iid]
        tickets[(iid, k)] = server.submit(iid, p, o, noise=noise(sizes[iid], iid) if k == 0 else None,
                                          last=(k == STEPS - 1), keep_dx=True)
        step[iid] += 1
    server.drain()
    out = {}
    for key, t in tickets.items():
        dx = np.empty(sizes[key[0]])
        res = server.poll(t, dx)
        assert res is not None and res["status"] == 0, res
        out[key] = (dx, res)
    return out


def test_alone_vs_mixed_bitwise():
    fsi = _fsi()
    torch.cuda.set_device(0)
    order = [iid for _ in range(STEPS) for iid, _, _ in INSTANCES]     # round-robin interleaving
    srv = fsi.Server(hbm_budget_bytes=0, max_slots=len(INSTANCES))
    mixed = _run(srv, INSTANCES, order)
    srv.close()
    for inst in INSTANCES:
        srv = fsi.Server(hbm_budget_bytes=0, max_slots=1)
        alone = _run(srv, [inst], [inst[0]] * STEPS)
        srv.close()
        for k in range(STEPS):
            a, _ = alone[(inst[0], k)]
            m, res = mixed[(inst[0], k)]
            assert np.array_equal(a, m), (inst[0], k, np.max(np.abs(a - m)))
            assert res["rel_res"] <= inst[2].rtol
    # Newton converges across the 3 steps of each instance
    for iid, _, _ in INSTANCES:
        assert mixed[(iid, STEPS - 1)][1]["rel_step"] < mixed[(iid, 0)][1]["rel_step"]


def test_admission_by_device_bytes():
    fsi = _fsi()
    p, o = Problem(levels=3), SolverOpts(tile=(2, 2), precision=1)
    plan = fsi.FSI(p, o, plan_only=True)
    one = plan.hbm_bytes
    n = int(plan.N[-1])
    plan.close()
    srv = fsi.Server(hbm_budget_bytes=int(one * 1.5), max_slots=2)
    t1 = srv.submit(1, p, o, noise=noise(n, 1), last=True)
    t2 = srv.submit(2, p, o, noise=noise(n, 2), last=True)
    srv.drain()
    r1, r2 = srv.poll(t1), srv.poll(t2)
    assert r1["status"] == 0 and r2["status"] == 0
    # the second instance could only start after the first was freed
    assert r2["queue_ms"] >= r1["run_ms"] * 0.5 or r1["queue_ms"] >= r2["run_ms"] * 0.5
    assert srv.resident_bytes() == 0
    with pytest.raises(fsi.FSIError):
        srv.submit(3, replace(p, levels=5), o, noise=noise(313860, 3))
    srv.close()


def test_rebound_streams_overlap():
    """Two instances built on the same stream and then rebound to two streams
    (fsi_set_stream) overlap on the device when driven from two threads: the
    sum of their device times (CUDA events on each stream) exceeds the wall
    time, and the concurrent run is faster than running them one after the
    other.  Results are bit-identical to the sequential run."""
    import threading
    import time
    fsi = _fsi()
    torch.cuda.set_device(0)
    s0 = torch.cuda.Stream()
    p, o = Problem(levels=3, mu_s=5e5, U=0.2), SolverOpts(tile=(2, 2), precision=1)
    inst = [fsi.FSI(p, o, stream=s0.cuda_stream) for _ in range(2)]
    n = int(inst[0].N[-1])
    y0 = []
    for k, s in enumerate(inst):
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        s.initial_state(torch.tensor(noise(n, 40 + k), dtype=torch.float64, device="cuda"), y)
        y0.append(y)
    steps = 6

    def run(k, out, stream=None):
        s = inst[k]
        dx = torch.empty(n, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = stream or s0
        e0.record(st)
        for _ in range(steps):
            s.set_state(y0[k])
            s.newton_step(dx)
        e1.record(st)
        e1.synchronize()
        out[k] = (dx.cpu().numpy(), e0.elapsed_time(e1))

    seq = {}
    for k in range(2):
        run(k, seq)                    # warm-up (records the V-cycle graphs)
    t0 = time.perf_counter()
    for k in range(2):
        run(k, seq)
    t_seq = time.perf_counter() - t0
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k in range(2):
        inst[k].set_stream(streams[k].cuda_stream)
    par = {}
    th = [threading.Thread(target=run, args=(k, par, streams[k])) for k in range(2)]
    t0 = time.perf_counter()
    for t in th:
        t.start()
    for t in th:
        t.join()
    t_par = time.perf_counter() - t0
    for k in range(2):
        assert np.array_equal(par[k][0], seq[k][0])
    dev_sum_ms = par[0][1] + par[1][1]
    assert dev_sum_ms > 1.1 * t_par * 1e3, (dev_sum_ms, t_par)
    assert t_par < 0.9 * t_seq, (t_par, t_seq)
    for s in inst:
        s.close()


def test_failed_instance_completes_its_queued_requests():
    """An instance whose first step fails (a non-finite state) is freed; its
    queued follow-up requests complete at once with the same error instead of
    rebuilding the hierarchy, and nothing stays resident."""
    fsi = _fsi()
    p, o = Problem(levels=3, mu_s=5e5, U=0.2), SolverOpts(tile=(2, 2), precision=1)
    n = _n(p)
    bad = np.full(n, np.nan)
    srv = fsi.Server(hbm_budget_bytes=0, max_slots=2)
    tickets = [srv.submit(7, p, o, noise=bad if k == 0 else None, last=(k == 3)) for k in range(4)]
    good = srv.submit(8, p, o, noise=noise(n, 8), last=True)
    srv.drain()
    res = [srv.poll(t) for t in tickets]
    assert res[0]["status"] in (-6, -7), res[0]
    for r in res[1:]:
        assert r["status"] == res[0]["status"]
        assert r["run_ms"] < 50.0, r
    assert srv.poll(good)["status"] == 0
    assert srv.resident_bytes() == 0
    srv.close()


def test_factor_batch_is_bitwise_the_individual_factorisation():
    """fsi_factor_schwarz_batch over instances of different shapes (2D at 3
    and 4 levels, whose blocks take the 32-column panel, and 3D at 2 levels,
    whose 784-unknown blocks take the 24-column one): the Newton corrections
    after the batched factorisation equal, bit for bit, those after each
    instance's own fsi_factor_schwarz."""
    fsi = _fsi()
    torch.cuda.set_device(0)
    s0 = torch.cuda.Stream()
    specs = [(Problem(levels=3, mu_s=1e5, U=0.3), SolverOpts(tile=(2, 2), precision=1)),
             (Problem(levels=4, mu_s=3e4, U=0.15), SolverOpts(tile=(2, 2), precision=1)),
             (problem_3d(levels=2, mu_s=5e5, U=0.2), SolverOpts(tile=(2, 2, 2), precision=1))]
    inst, y0 = [], []
    for k, (p, o) in enumerate(specs):
        s = fsi.FSI(p, o, stream=s0.cuda_stream)
        n = int(s.N[-1])
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        s.initial_state(torch.tensor(noise(n, 60 + k), dtype=torch.float64, device="cuda"), y)
        inst.append(s)
        y0.append(y)

    def run(batched):
        out = []
        for s, y in zip(inst, y0):
            s.set_state(y)
            s.assemble()
        if batched:
            fsi.factor_batch(inst)
        else:
            for s in inst:
                s.factor()
        for s, y in zip(inst, y0):
            dx = torch.empty_like(y)
            s.newton_solve_update(dx)
            out.append(dx.cpu().numpy())
        return out

    ref = run(False)
    got = run(True)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    for s in inst:
        s.close()


def _wait(srv, tickets, n, deadline_s=600.0):
    """Polls the tickets until all are done (a stuck request fails the test
    instead of blocking it)."""
    import time
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for k, t in tickets.items():
            if k in out:
                continue
            dx = np.empty(n)
            r = srv.poll(t, dx)
            if r is not None:
                out[k] = (dx, r)
        assert time.time() - t0 < deadline_s, f"requests still pending: {sorted(set(tickets) - set(out))}"
        time.sleep(0.01)
    return out


def test_eviction_and_readmission_keep_results():
    """A budget that holds one instance, two instances with two steps each,
    the second submitted while the first is resident and idle: the first is
    evicted (state to the host, hierarchy freed), the second runs; the first's
    next (last) request evicts the second and rebuilds the first from its
    saved state; the second's next request then rebuilds the second, which
    fits once the first has ended.  Every correction equals, bit for bit, that
    of the instance served alone."""
    fsi = _fsi()
    p, o = Problem(levels=3, mu_s=1e5, U=0.3), SolverOpts(tile=(2, 2), precision=1)
    plan = fsi.FSI(p, o, plan_only=True)
    one, n = plan.hbm_bytes, int(plan.N[-1])
    plan.close()
    ref = {}
    for iid in (1, 2):
        srv = fsi.Server(hbm_budget_bytes=0, max_slots=1)
        ts = {(iid, 0): srv.submit(iid, p, o, noise=noise(n, iid), keep_dx=True),
              (iid, 1): srv.submit(iid, p, o, last=True, keep_dx=True)}
        ref.update(_wait(srv, ts, n))
        srv.close()
    srv = fsi.Server(hbm_budget_bytes=int(one * 1.5), max_slots=2)
    got = _wait(srv, {(1, 0): srv.submit(1, p, o, noise=noise(n, 1), keep_dx=True)}, n)
    got.update(_wait(srv, {(2, 0): srv.submit(2, p, o, noise=noise(n, 2), keep_dx=True)}, n))
    assert srv.evictions() == 1
    got.update(_wait(srv, {(1, 1): srv.submit(1, p, o, last=True, keep_dx=True)}, n))
    assert srv.evictions() == 2
    got.update(_wait(srv, {(2, 1): srv.submit(2, p, o, last=True, keep_dx=True)}, n))
    assert srv.evictions() == 2
    for key, (dx, r) in got.items():
        assert r["status"] == 0, (key, r)
        assert np.array_equal(dx, ref[key][0]), (key, np.max(np.abs(dx - ref[key][0])))
    assert srv.resident_bytes() == 0
    srv.close()


def test_cancelled_requests_leave_the_other_results_unchanged():
    """One worker, instance 1 with three queued steps and instance 2 with
    three: cancelling instance 1's last step ends it after its second (nothing
    stays resident), cancelling instance 2's first step hands the initial-state
    noise to its second, which builds it.  The cancelled requests complete with
    FSI_E_CANCELLED; every other correction equals, bit for bit, the
    corresponding step of the instance served alone."""
    fsi = _fsi()
    p, o = Problem(levels=3, mu_s=1e5, U=0.3), SolverOpts(tile=(2, 2), precision=1)
    n = _n(p)
    ref = {}
    for iid in (1, 2):
        srv = fsi.Server(hbm_budget_bytes=0, max_slots=1)
        ts = {(iid, 0): srv.submit(iid, p, o, noise=noise(n, iid), keep_dx=True),
              (iid, 1): srv.submit(iid, p, o, last=True, keep_dx=True)}
        ref.update(_wait(srv, ts, n))
        srv.close()
    srv = fsi.Server(hbm_budget_bytes=0, max_slots=1)
    ts = {}
    for iid in (1, 2):
        for k in range(3):
            ts[(iid, k)] = srv.submit(iid, p, o, noise=noise(n, iid) if k == 0 else None, last=(k == 2),
                                      keep_dx=True)
    # the single worker is still building instance 1 for its first step
    assert srv.cancel(ts[(1, 2)]) and srv.cancel(ts[(2, 0)])
    srv.drain()
    assert srv.cancel(ts[(1, 0)]) is False
    got = _wait(srv, ts, n)
    for key in ((1, 2), (2, 0)):
        assert got[key][1]["status"] == -9, got[key][1]
    for key, refkey in (((1, 0), (1, 0)), ((1, 1), (1, 1)), ((2, 1), (2, 0)), ((2, 2), (2, 1))):
        dx, r = got[key]
        assert r["status"] == 0, (key, r)
        assert np.array_equal(dx, ref[refkey][0]), key
    assert srv.resident_bytes() == 0
    with pytest.raises(fsi.FSIError):
        srv.cancel(ts[(1, 0)])
    srv.close()
