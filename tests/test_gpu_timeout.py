"""The contact loop's bounded waits give up cleanly (SDC_ERR_TIMEOUT) and the context stays usable.

A wait budget of one poll (sdc_set_wait_limit) makes the exchange waits of the contact
substep loop give up on copies that are still on their way, so the give-up path runs
without any fault: the CTA whose wait gave up stops exchanging, drains the copies still
addressed to it and reports SDC_ERR_TIMEOUT (the protocol is checked on the host in
test_contact_exchange_model.py). With global replicas the wait that gives up is the one for
the CTA's own copy of the replica into shared memory: the CTA issues no further copy and
drains that one before exit. In the grid-wide loop (placement 3) it is a wait of the grid
barrier: the CTA goes on (every later wait is bounded too) and no copy is in flight.
Afterwards the default budget restores normal steps, bitwise equal to a context that never
timed out.
"""

import numpy as np
import pytest

from synth.machines import batch_resolutions, machine_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("precision,placement",
                         [("fp64", 0), ("mixed", 0), ("fp64", 1), ("mixed", 1), ("fp64", 3), ("mixed", 3)])
def test_wait_budget_of_one_poll_times_out_and_context_recovers(torch, precision, placement):
    from paper_1707_03581_gb300 import SdcError, Solver

    # a 16-CTA loop cluster: the r = 24 machine of the batch (about a thousand contact DOFs)
    # in FP64; in mixed precision, whose FP32 copies are half the size and land sooner, the
    # 313,646-DOF machine (3,950 contact DOFs)
    if precision == "fp64":
        (mach,) = machine_config(3, select={batch_resolutions()[24]})
    else:
        mach = machine_config(1)
    # placement 1: global replicas, staged into shared memory after every substep; the wait
    # that gives up is the one for the CTA's own staging copy
    s = Solver(0)
    s.set_machine(mach, precision=precision)
    s.set_contact_replicas(placement)
    ref = Solver(0)
    ref.set_machine(mach, precision=precision)
    ref.set_contact_replicas(placement)
    s.set_wait_limit(1)
    timed_out = False
    for _ in range(20):
        try:
            rep = s.step(report=True)
        except SdcError as e:
            assert "SDC_ERR_TIMEOUT" in str(e), str(e)
            timed_out = True
            break
        assert rep["contact_cluster"] > 1
    assert timed_out
    # the device is fine and the context usable: the default budget gives normal steps again
    s.set_wait_limit(0)
    s.set_temperature(np.full(s.n, mach.T0), t0=mach.t0)
    for _ in range(2):
        ra = s.step(report=True)
        rb = ref.step(report=True)
        assert ra["status"] == 0 and rb["status"] == 0
    assert np.array_equal(s.temperature(), ref.temperature())
    with pytest.raises(SdcError):
        s.set_wait_limit(-1)
    s.close()
    ref.close()
