"""Host logic of the serving loop (paper_1707_03581_gb300/serving.py) on the CPU,
with a stand-in for the library's Solver: admission, slot reuse and, under a tight
HBM budget, the closing of idle slots of other machines (least recently used
first). The device work itself is covered by tests/test_gpu_serving.py."""

import types

import numpy as np
import pytest


class FakeSolver:
    made, closed, live = 0, 0, set()
    sizes = {}

    def __init__(self, device, own_stream=False):
        FakeSolver.made += 1
        self.steps_left = 0

    fail_names = set()

    def set_machine(self, m, precision="mixed"):
        self.m = m
        self.n = m.n_dof
        FakeSolver.live.add(id(self))
        if m.name in FakeSolver.fail_names:  # a forced allocation failure
            raise RuntimeError("SDC_ERR_CUDA: out of memory (forced)")

    def set_graph_branches(self, on):
        pass

    def footprint(self):
        return FakeSolver.sizes[self.m.name]

    def set_temperature(self, T, t0=0.0):
        self.T = np.full(self.n, 20.0)

    def poll(self):
        return True

    def step_async(self, k):
        self.T = self.T + k

    def synchronize(self):
        pass

    def temperature(self):
        return self.T.copy()

    def close(self):
        FakeSolver.closed += 1
        FakeSolver.live.discard(id(self))


def _machine(name, n):
    sc = types.SimpleNamespace(dt=1.0, M=3, P=20, nodes="lobatto")
    return types.SimpleNamespace(name=name, n_dof=n, scheme=sc, t0=0.0, T0=20.0)


@pytest.fixture
def server(monkeypatch):
    pytest.importorskip("torch")
    from paper_1707_03581_gb300 import binding, serving

    monkeypatch.setattr(binding, "Solver", FakeSolver)
    FakeSolver.made, FakeSolver.closed, FakeSolver.live = 0, 0, set()
    FakeSolver.fail_names = set()
    machines = [_machine(f"m{i}", 10 + i) for i in range(4)]
    FakeSolver.sizes = {m.name: 100 for m in machines}

    def make(budget):
        srv = serving.LookAheadServer(machines, device=0, hbm_budget_bytes=budget, chunk=4, keep_results=True)
        srv.state = [object()] * len(machines)  # resident states exist (no device here)
        return srv, serving

    return make


def test_slots_are_reused_and_every_request_finishes(server):
    srv, serving = server(10_000)
    reqs = [serving.Request(0.0, 10.0, i % 2) for i in range(6)]
    srv.run(reqs)
    assert all(r.t_done is not None for r in reqs)
    assert all(np.all(r.result == 20.0 + 10) for r in reqs)
    assert srv.slots_made <= 6 and FakeSolver.closed == 0
    srv.close()


def test_tight_budget_closes_idle_slots_of_other_machines(server):
    srv, serving = server(250)  # room for two slots of 100 bytes
    reqs = [serving.Request(0.001 * k, 4.0, k % 4) for k in range(8)]
    srv.run(reqs)
    assert all(r.t_done is not None for r in reqs)
    assert srv.footprint <= 250
    assert FakeSolver.closed >= 2  # four machines through two slots' worth of memory
    assert len(FakeSolver.live) <= 2
    srv.close()
    assert not FakeSolver.live


def test_least_recently_idle_slot_goes_first(server):
    srv, serving = server(250)
    srv.run([serving.Request(0.0, 1.0, 0)])
    srv.run([serving.Request(0.0, 1.0, 1)])
    srv.run([serving.Request(0.0, 1.0, 0)])  # machine 0's slot is reused and idle again, last
    assert [j for j, _ in srv.idle] == [1, 0]
    srv.run([serving.Request(0.0, 1.0, 2)])  # makes room by closing machine 1's slot
    assert srv.free_slots[1] == [] and len(srv.free_slots[0]) == 1 and len(srv.free_slots[2]) == 1
    srv.close()


def test_cancelled_requests_leave_and_the_others_are_unchanged(server):
    srv, serving = server(10_000)
    reqs = [serving.Request(0.0, 6.0, k % 2) for k in range(4)]
    queued = serving.Request(0.01, 6.0, 0, cancel_at_s=0.0)     # cancelled on arrival
    running = serving.Request(0.0, 1e6, 1, cancel_at_s=0.05)    # cancelled while its steps run
    srv.run(reqs + [queued, running])
    assert queued.status == "cancelled" and queued.t_admit is None
    assert running.status == "cancelled" and running.t_admit is not None
    assert all(r.status == "done" and np.all(r.result == 26.0) for r in reqs)
    stats = serving.summarize(reqs + [queued, running], srv.machines, [m.n_dof for m in srv.machines])
    assert (stats["requests"], stats["cancelled"], stats["failed"]) == (4, 2, 0)
    # the cancelled request's slot went back to the pool and serves the next request
    more = serving.Request(0.0, 3.0, 1)
    srv.run([more])
    assert more.status == "done" and np.all(more.result == 23.0)
    srv.close()


def test_a_failed_admission_fails_alone(server):
    srv, serving = server(10_000)
    FakeSolver.fail_names = {"m3"}
    reqs = [serving.Request(0.001 * k, 5.0, k % 4) for k in range(8)]
    srv.run(reqs)
    for r in reqs:
        if r.machine_index == 3:
            assert r.status == "failed" and "out of memory" in r.error
        else:
            assert r.status == "done" and np.all(r.result == 25.0)
    assert FakeSolver.closed == 2  # each failed slot was closed at once
    stats = serving.summarize(reqs, srv.machines, [m.n_dof for m in srv.machines])
    assert (stats["requests"], stats["failed"]) == (6, 2)
    srv.close()
    assert not FakeSolver.live



class SlowSolver(FakeSolver):
    """A stand-in whose enqueued steps stay in flight for a number of polls, so that
    slots of several machines are active at once."""

    polls_busy = 30

    def step_async(self, k):
        super().step_async(k)
        self.busy = SlowSolver.polls_busy

    def poll(self):
        if getattr(self, "busy", 0) > 0:
            self.busy -= 1
            return False
        return True


def test_admission_never_exceeds_the_budget_while_slots_are_active(server, monkeypatch):
    from paper_1707_03581_gb300 import binding

    monkeypatch.setattr(binding, "Solver", SlowSolver)
    srv, serving = server(250)  # room for two slots of 100 bytes
    seen = []
    orig = srv._slot

    def watched(i):
        s = orig(i)
        seen.append(srv.footprint)
        assert srv.footprint <= srv.budget, (i, srv.footprint)
        return s

    srv._slot = watched
    reqs = [serving.Request(0.0, 8.0, k % 4) for k in range(8)]  # four machines at once
    srv.run(reqs)
    assert all(r.status == "done" and np.all(r.result == 28.0) for r in reqs)
    assert max(seen) <= 250 and srv.peak_footprint <= 250
    srv.close()
    assert not FakeSolver.live


def test_an_underestimated_first_slot_is_closed_and_its_request_waits(server, monkeypatch):
    # machine 3's slot has twice the bytes per DOF of the others: its estimate (scaled
    # from them) is short, so the slot made while two others run is closed again at once
    from paper_1707_03581_gb300 import binding

    monkeypatch.setattr(binding, "Solver", SlowSolver)
    srv, serving = server(350)
    FakeSolver.sizes["m3"] = 200  # estimate 13 DOF x 10 bytes = 130
    reqs = [serving.Request(0.0, 8.0, 0), serving.Request(0.0, 8.0, 1), serving.Request(0.0, 8.0, 3)]
    srv.run(reqs)
    assert all(r.status == "done" for r in reqs)
    assert srv.peak_footprint <= 350
    assert FakeSolver.made > srv.slots_made  # the oversized attempt was made, then closed
    srv.close()
    assert not FakeSolver.live
