"""Single-rate semi-implicit SDC (Sec. 3, sdc_set_stepper) on the GPU
against oracle.mrsdc.sisdc_step."""

import numpy as np
import pytest

from oracle.machine import MachineProblem
from oracle.mrsdc import sisdc_step
from oracle.weights import mrsdc_weights
from synth import machine_config, tiny_machine
from synth.machines import with_scheme

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _solver(mach, precision, T0=None):
    from paper_1707_03581_gb300 import Solver

    s = Solver(0)
    s.set_machine(mach, precision=precision, T0=T0)
    s.set_stepper("sisdc")
    return s


def _parity(mach, n_steps, precision, T0=None):
    prob = MachineProblem(mach)
    sc = mach.scheme
    W = mrsdc_weights(sc.nodes, sc.M, sc.P, sc.window)
    X = np.full(prob.n, mach.T0) if T0 is None else np.array(T0, dtype=np.float64)
    start = X.copy()
    s = _solver(mach, precision, T0)
    worst = 0.0
    for n in range(n_steps):
        rep = s.step(report=True)
        assert rep["status"] == 0
        X, _ = sisdc_step(prob, X, mach.t0 + n * sc.dt, sc.dt, W, sc.sweeps)
        got = s.temperature()
        rel = np.linalg.norm(got - X) / np.linalg.norm(X)
        rise = np.linalg.norm(got - X) / np.linalg.norm(X - start)
        if precision == "fp64":
            assert rel <= 1e-10 and rise <= 1e-8, (n, rel, rise)
        else:
            assert rel <= 1e-6 and rise <= 1e-6, (n, rel, rise)
        worst = max(worst, rel)
    s.close()
    return worst


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config0_lobatto(torch, precision):
    # the 1,876-DOF machine, Lobatto M=3, 3 sweeps; P = 1 (single-rate uses the end slots)
    mach = with_scheme(machine_config(0), P=1, window=0)
    _parity(mach, 6, precision)


@pytest.mark.parametrize("nodes,M,K", [("radau_right", 3, 2), ("equi_noleft", 4, 3), ("lobatto", 4, 0)])
def test_schemes_on_tiny_machine(torch, nodes, M, K):
    mach = with_scheme(tiny_machine(z0=0.37, amp=0.21, period=1.7), nodes=nodes, M=M, P=2, sweeps=K,
                       window=0, dt=0.8)
    rng = np.random.default_rng(11)
    T0 = 20.0 + rng.standard_normal(mach.n_dof)
    _parity(mach, 4, "fp64", T0=T0)


def test_eager_equals_graph_and_no_diagnostics(torch):
    from paper_1707_03581_gb300 import SdcError

    mach = with_scheme(machine_config(0), P=1, window=0)
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
    a.close()
    b.close()
