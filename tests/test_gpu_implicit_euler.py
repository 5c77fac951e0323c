"""Fully implicit Euler with the contact coupling in the matrix (the comparison
method of Sec. 1 and Sec. 5, sdc_set_stepper) on the GPU, against
oracle.mrsdc.implicit_euler_step (a sparse direct solve of the same system)."""

import numpy as np
import pytest

from oracle.machine import MachineProblem
from oracle.mrsdc import implicit_euler_step
from synth import machine_config, tiny_machine
from synth.machines import with_scheme

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _solver(mach, precision="fp64", T0=None):
    from paper_1707_03581_gb300 import Solver

    s = Solver(0)
    s.set_machine(mach, precision=precision, T0=T0)
    s.set_stepper("implicit_euler")
    return s


def _parity(mach, n_steps, precision, T0=None):
    prob = MachineProblem(mach)
    dt = mach.scheme.dt
    X = np.full(prob.n, mach.T0) if T0 is None else np.array(T0, dtype=np.float64)
    start = X.copy()
    s = _solver(mach, precision, T0)
    for n in range(n_steps):
        rep = s.step(report=True)
        assert rep["status"] == 0
        assert rep["sweeps"] == 0 and rep["cg_iters_total"] > 0
        X = implicit_euler_step(prob, X, mach.t0 + n * dt, dt)
        got = s.temperature()
        # the solve is FP64 Jacobi-PCG in both precisions
        rel = np.linalg.norm(got - X) / np.linalg.norm(X)
        rise = np.linalg.norm(got - X) / np.linalg.norm(X - start)
        assert rel <= 1e-10 and rise <= 1e-8, (n, rel, rise)
    T = s.temperature()
    s.close()
    return T


def test_config0_both_precisions_agree_with_the_oracle(torch):
    # the 1,876-DOF machine (seeded stroke), 6 steps of the scheme's dt
    mach = machine_config(0)
    a = _parity(mach, 6, "fp64")
    b = _parity(mach, 6, "mixed")
    assert np.linalg.norm(a - b) / np.linalg.norm(a) <= 1e-12


@pytest.mark.parametrize("dt", [0.2, 0.8, 5.0])
def test_moving_contact_on_tiny_machine(torch, dt):
    mach = with_scheme(tiny_machine(z0=0.37, amp=0.21, period=1.7), dt=dt)
    rng = np.random.default_rng(21)
    T0 = 20.0 + rng.standard_normal(mach.n_dof)
    _parity(mach, 4, "fp64", T0=T0)


def test_insulated_heat_is_conserved_and_friction_ledger(torch):
    # insulated, frictionless: the coupling only moves heat between the bodies
    mach = tiny_machine(z0=0.37, amp=0.25, period=np.inf, q0=0.0)
    mach.stand.h = 0.0
    mach.stock.h = 0.0
    rng = np.random.default_rng(9)
    T0 = 20.0 + 3.0 * rng.standard_normal(mach.n_dof)
    s = _solver(mach, T0=T0)
    h0 = s.heat_totals()
    for _ in range(5):
        s.step(report=True)
    h1 = s.heat_totals()
    Q0 = h0["stored_stand"] + h0["stored_stock"]
    Q1 = h1["stored_stand"] + h1["stored_stock"]
    assert abs(Q1 - Q0) <= 1e-12 * abs(Q0)
    assert abs(h1["friction_in"]) <= 1e-8
    s.close()
    # resting stock, constant flux: the ledger books q0 * area * dt per step
    mach = tiny_machine(z0=0.37, amp=0.25, period=np.inf, q0=2.0e4)
    s = _solver(mach)
    for _ in range(3):
        s.step(report=True)
    h = s.heat_totals()
    assert abs(h["friction_in"] - 3 * 2.0e4 * 0.06 * 1.0) <= 1e-9 * 3 * 2.0e4 * 0.06
    s.close()


def test_eager_equals_graph_and_no_diagnostics(torch):
    from paper_1707_03581_gb300 import SdcError

    mach = machine_config(0)
    a = _solver(mach, "mixed")
    b = _solver(mach, "mixed")
    b.set_execution(True)
    for _ in range(3):
        ra = a.step(report=True)
        rb = b.step(report=True)
    assert np.array_equal(a.temperature(), b.temperature())
    assert ra["kernel_launches"] == rb["kernel_launches"]
    with pytest.raises(SdcError):
        a.set_diagnostics(True)
    # back to MRSDC on the same context: the oracle's MRSDC step from the same state
    from oracle.mrsdc import mrsdc_step
    from oracle.weights import mrsdc_weights

    a.set_stepper("mrsdc")
    T = a.temperature()
    t = mach.t0 + 3 * mach.scheme.dt
    a.set_temperature(T, t0=t)
    a.step(report=True)
    sc = mach.scheme
    X, _ = mrsdc_step(MachineProblem(mach), T, t, sc.dt, mrsdc_weights(sc.nodes, sc.M, sc.P, sc.window), sc.sweeps)
    assert np.linalg.norm(a.temperature() - X) / np.linalg.norm(X) <= 1e-6
    a.close()
    b.close()
