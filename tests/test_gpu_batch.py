"""Batches (sdc_batch_*): machines stepped concurrently equal each machine stepped alone.

Members share no state and every reduction has a fixed order, so the
comparison is bitwise, in both precisions.
"""

import numpy as np
import pytest

from synth import machine_config, tiny_machine
from synth.machines import with_scheme

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _machines():
    base = machine_config(0)
    return [base,
            with_scheme(tiny_machine(z0=0.37, amp=0.21, period=1.7), nodes="radau_right", M=3, P=8, sweeps=2),
            tiny_machine(z0=0.40, amp=0.15, period=3.1, q0=3.0e4)]


def _solver(torch, mach, precision, own=True):
    from paper_1707_03581_gb300 import Solver

    s = Solver(0, own_stream=True) if own else Solver(0, stream=torch.cuda.Stream())
    s.set_machine(mach, precision=precision)
    return s


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_members_alone(torch, precision):
    from paper_1707_03581_gb300 import Batch

    machines = _machines()
    steps = [5, 3, 4]
    alone = []
    for mach, k in zip(machines, steps):
        s = _solver(torch, mach, precision)
        s.run_horizon(k)
        alone.append(s.temperature())
        s.close()
    members = [_solver(torch, m, precision, own=(i != 1)) for i, m in enumerate(machines)]
    b = Batch(0)
    for s in members:
        b.add(s)
    assert len(b) == 3
    b.step([2, 1, 2], wait=False)
    b.step([3, 2, 2], wait=True)
    for s, ref in zip(members, alone):
        assert s.poll()
        assert np.array_equal(s.temperature(), ref)
    b.remove(members[1])
    assert len(b) == 2
    b.step(None, wait=True)
    b.close()
    for s in members:
        s.close()


def test_batch_rejects_shared_stream_and_unready_member(torch):
    from paper_1707_03581_gb300 import Batch, SdcError, Solver

    stream = torch.cuda.Stream()
    a = Solver(0, stream=stream)
    a.set_machine(machine_config(0))
    c = Solver(0, stream=stream)
    c.set_machine(machine_config(0))
    b = Batch(0)
    b.add(a)
    with pytest.raises(SdcError):
        b.add(c)
    with pytest.raises(SdcError):
        b.add(a)
    fresh = Solver(0, stream=torch.cuda.Stream())
    with pytest.raises(SdcError):
        b.add(fresh)
    b.close()
    for s in (a, c, fresh):
        s.close()


def test_batch_of_large_machines_equals_members_alone(torch):
    # Members large enough that their CG kernels take several waves of blocks,
    # stepped concurrently: blocks of one launch start at different times.
    from paper_1707_03581_gb300 import Batch

    machines = machine_config(3, truncate=12)
    alone = []
    for mach in machines:
        s = _solver(torch, mach, "mixed")
        s.run_horizon(2)
        alone.append(s.temperature())
        s.close()
    members = [_solver(torch, m, "mixed") for m in machines]
    b = Batch(0)
    for s in members:
        b.add(s)
    b.step([2] * len(members), wait=True)
    for s, ref in zip(members, alone):
        assert np.array_equal(s.temperature(), ref)
    b.close()
    for s in members:
        s.close()


def test_fused_batch_equals_members_alone(torch):
    # The block-diagonal form (sdc_batch_set_fused): the FP32 inner CG of the qualifying
    # members (mixed precision, deferred-dot grids) runs as one launch per kernel over all of
    # them. Members of four resolutions of the batched workload (12,902 to 313,646 DOF) and
    # a machine of another scheme; an FP64 member does not qualify and keeps its own graph.
    from paper_1707_03581_gb300 import Batch, SdcError
    from synth.machines import batch_resolutions

    first = batch_resolutions()
    pool = machine_config(3, select={first[16], first[24], first[32], first[48]})
    cases = [(m, "mixed") for m in pool] + [(machine_config(0), "mixed"), (pool[0], "fp64")]
    steps = 3
    alone = []
    for mach, prec in cases:
        s = _solver(torch, mach, prec)
        s.run_horizon(steps)
        alone.append(s.temperature())
        s.close()
    members = [_solver(torch, mach, prec) for mach, prec in cases]
    b = Batch(0)
    for s in members:
        b.add(s)
    b.set_fused(True)
    assert b.fused_size() == 5  # the mixed members; machine_config(0) shares their scheme
    b.step([1] * len(members), wait=False)
    b.step([2] * len(members), wait=True)
    for s, ref, (mach, prec) in zip(members, alone, cases):
        assert np.array_equal(s.temperature(), ref), (mach.name, prec)
    # fused members step together
    with pytest.raises(SdcError):
        b.step([1, 2, 1, 1, 1, 1], wait=True)
    # and the batch goes on after fusion is switched off, still equal to members alone
    b.set_fused(False)
    assert b.fused_size() == 0
    b.step([1] * len(members), wait=True)
    for s, (mach, prec) in zip(members, cases):
        r = _solver(torch, mach, prec)
        r.run_horizon(steps + 1)
        assert np.array_equal(s.temperature(), r.temperature()), (mach.name, prec)
        r.close()
    b.close()
    for s in members:
        s.close()
