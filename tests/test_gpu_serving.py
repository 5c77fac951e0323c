"""Serving loop: every forecast served in the mix equals the same forecast run alone.

Requests for three machines arrive while others run; their slots, streams and
step graphs overlap on the device. Slots keep their own state and reductions
have a fixed order, so the comparison is bitwise.
"""

import numpy as np
import pytest

from synth import machine_config, tiny_machine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_results_in_the_mix_equal_results_alone(torch, precision):
    from paper_1707_03581_gb300 import Solver
    from paper_1707_03581_gb300.serving import LookAheadServer, Request, summarize

    machines = [machine_config(0), tiny_machine(z0=0.37, amp=0.21, period=1.7),
                tiny_machine(z0=0.40, amp=0.15, period=3.1, q0=3.0e4)]
    rng = np.random.default_rng(3)
    server = LookAheadServer(machines, precision=precision, max_active=4, chunk=2, keep_results=True)
    # a warm-start state that differs from the uniform initial field for machine 0
    warm = 20.0 + 0.5 * rng.standard_normal(machines[0].n_dof)
    server.set_state(0, warm)
    reqs = [Request(0.002 * k, float(rng.integers(2, 7)), int(k % 3)) for k in range(9)]
    server.run(reqs)
    stats = summarize(reqs, machines, [m.n_dof for m in machines])
    assert stats["requests"] == 9 and stats["latency_s"]["p99"] > 0
    assert server.slots_made <= len(reqs)
    for r in reqs:
        assert r.t_done >= r.t_admit >= 0
        s = Solver(0, own_stream=True)
        s.set_machine(machines[r.machine_index], precision=precision,
                      T0=warm if r.machine_index == 0 else None)
        s.run_horizon(r.n_steps)
        assert np.array_equal(s.temperature(), r.result), r
        s.close()
    server.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_pool_machines_in_the_mix_equal_results_alone(torch, precision):
    # the machines serving draws from: batch members of stand resolution 16, 24 and 32
    # (12,902 to 95,434 DOF), with their own strokes and friction fluxes
    from paper_1707_03581_gb300 import Solver
    from paper_1707_03581_gb300.serving import LookAheadServer, Request
    from synth.machines import batch_resolutions

    first = batch_resolutions()
    machines = machine_config(3, select={first[16], first[24], first[32]})
    rng = np.random.default_rng(4)
    server = LookAheadServer(machines, precision=precision, max_active=6, chunk=2, keep_results=True)
    reqs = [Request(0.001 * k, float(rng.integers(2, 6)), int(k % 3)) for k in range(9)]
    server.run(reqs)
    assert all(r.status == "done" for r in reqs)
    for r in reqs:
        s = Solver(0, own_stream=True)
        s.set_machine(machines[r.machine_index], precision=precision)
        s.run_horizon(r.n_steps)
        assert np.array_equal(s.temperature(), r.result), (r.machine_index, r.n_steps)
        s.close()
    server.close()
