"""The autotuner (sdc_autotune) and the launch options it picks.

Its options (CG loop pairs, FP32 update grid, contact cluster cap, replica placement,
graph side branches) must leave every result bitwise unchanged, the tuning must leave the
context's state as it was (it times trial steps from a saved copy and restores it), and a
second context of the same shape must take the cached picks without trials.
"""

import numpy as np
import pytest

from synth import machine_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _solver(mach, precision):
    from paper_1707_03581_gb300 import Solver

    s = Solver(0)
    s.set_machine(mach, precision=precision)
    return s


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tuned_context_is_bitwise_equal_and_state_is_kept(torch, precision):
    mach = machine_config(0)
    a = _solver(mach, precision)
    a.step(report=True)  # a state other than the start
    T1 = a.temperature()
    h1 = a.heat_totals()
    rep = a.autotune(trial_steps=2)
    assert rep["cached"] == 0 and rep["trials"] >= 2 and rep["ms_tuned"] > 0
    assert rep["ms_tuned"] <= rep["ms_default"]
    assert 1 <= rep["cg_unroll"] <= 8 and rep["contact_cluster"] >= 1
    # the trial steps left no trace
    assert np.array_equal(a.temperature(), T1)
    h = a.heat_totals()
    assert h["t"] == h1["t"] and h["friction_in"] == h1["friction_in"]
    b = _solver(mach, precision)
    b.step(report=True)
    for _ in range(3):
        ra = a.step(report=True)
        rb = b.step(report=True)
    assert np.array_equal(a.temperature(), b.temperature())
    assert ra["cg_iters_total"] == rb["cg_iters_total"] and ra["t"] == rb["t"]
    # a context of the same shape takes the cached picks
    c = _solver(mach, precision)
    rc = c.autotune()
    assert rc["cached"] == 1 and rc["trials"] == 0
    assert (rc["cg_unroll"], rc["update_blocks_per_sm"], rc["contact_cluster_cap"], rc["graph_branches"]) == (
        rep["cg_unroll"], rep["update_blocks_per_sm"], rep["contact_cluster_cap"], rep["graph_branches"])
    for s in (a, b, c):
        s.close()


def test_update_grid_is_bitwise_neutral(torch):
    # the FP32 update's one-wave grid at 2, 3 and the default (as many as fit) blocks a SM
    from paper_1707_03581_gb300 import SdcError

    mach = machine_config(1)
    ref = None
    for bps in (0, 2, 3):
        s = _solver(mach, "mixed")
        s.set_update_blocks(bps)
        for _ in range(2):
            rep = s.step(report=True)
        T = s.temperature()
        if ref is None:
            ref, iters = T, rep["cg_iters_total"]
        assert np.array_equal(T, ref), bps
        assert rep["cg_iters_total"] == iters
        if bps == 3:
            with pytest.raises(SdcError):
                s.set_update_blocks(33)
        s.close()


def test_autotune_refuses_eager_execution(torch):
    from paper_1707_03581_gb300 import SdcError

    s = _solver(machine_config(0), "fp64")
    s.set_execution(True)
    with pytest.raises(SdcError) as e:
        s.autotune()
    assert "SDC_ERR_STATE" in str(e.value)
    s.close()
