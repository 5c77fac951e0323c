"""The mixed path's implicit solves against their FP64 definition, and its drift over a full horizon.

The mixed-precision solve refines x in FP64 but carries its residual with the FP32
operator: r = (b - A x0) - A32 (x - x0), with b - A x0 formed in FP64. Its stop test
(||r|| <= 1e-12 ||b||) is therefore applied to that carried residual. These tests check
what it means for the FP64 system (Algorithms 1 and 2, the implicit stage
(diag(m) + dtau K) x = b):
  * the true residual ||b - (m x + dtau K x)|| / ||b||, with the FP64 K and the FP64
    iterate (sdc_set_diagnostics bit 1), stays below TRUE_RES_BOUND in every solve of
    every macro step over the 313,646-DOF workload's 600 s horizon;
  * over that horizon the mixed temperature stays within the stated 1e-6 bar of the FP64
    path (pinned to the oracle at 1e-10 per step in test_gpu_parity.py), on T and on the
    rise T - T0, every 50 steps;
  * the diagnostic changes nothing: results are bitwise equal with it on or off.
"""

import numpy as np
import pytest

from synth import machine_config

pytestmark = pytest.mark.gpu

REL_MIXED = 1e-6
# the carried residual stops at 1e-12 ||b||; the FP32 operator error of the correction
# term is ~6e-8 ||A (x - x0)||, and ||A (x - x0)|| is a small part of ||b|| (the 20 degC
# field dominates b); measured below 1e-10 on this workload
TRUE_RES_BOUND = 1e-9


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_true_residual_and_drift_over_600_s(torch):
    from paper_1707_03581_gb300 import Solver

    mach = machine_config(1)
    a = Solver(0)
    a.set_machine(mach, precision="mixed")
    a.set_diagnostics(False, true_residual=True)
    b = Solver(0)
    b.set_machine(mach, precision="fp64")
    worst_true, worst_rel, worst_rise = 0.0, 0.0, 0.0
    for k in range(1, 601):
        ra = a.step(report=True)
        rb = b.step(report=(k % 50 == 0))
        assert ra["status"] == 0 and ra["true_residual_max"] >= 0.0
        worst_true = max(worst_true, ra["true_residual_max"])
        if k % 50 == 0:
            assert rb["true_residual_max"] == -1.0  # FP64 solves have no carried residual
            Ta, Tb = a.temperature(), b.temperature()
            rel = np.linalg.norm(Ta - Tb) / np.linalg.norm(Tb)
            rise = np.linalg.norm(Ta - Tb) / np.linalg.norm(Tb - mach.T0)
            worst_rel, worst_rise = max(worst_rel, rel), max(worst_rise, rise)
            assert rel <= REL_MIXED and rise <= REL_MIXED, (k, rel, rise)
    print(f"true residual max {worst_true:.3e}, rel {worst_rel:.3e}, rise {worst_rise:.3e}")
    assert worst_true <= TRUE_RES_BOUND, worst_true
    a.close()
    b.close()


def test_true_residual_diagnostic_changes_nothing(torch):
    from paper_1707_03581_gb300 import Solver

    mach = machine_config(0)
    a = Solver(0)
    a.set_machine(mach, precision="mixed")
    a.set_diagnostics(False, true_residual=True)
    b = Solver(0)
    b.set_machine(mach, precision="mixed")
    for _ in range(3):
        ra = a.step(report=True)
        rb = b.step(report=True)
    assert np.array_equal(a.temperature(), b.temperature())
    assert 0.0 <= ra["true_residual_max"] <= TRUE_RES_BOUND and rb["true_residual_max"] == -1.0
    assert ra["cg_iters_total"] == rb["cg_iters_total"]
    a.close()
    b.close()
