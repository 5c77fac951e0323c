"""GPU stationary initial state (Sec. 5, sdc_set_stationary_state) against the
oracle and the closed form, and MRSDC steps from it."""

import numpy as np
import pytest

from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step
from oracle.weights import mrsdc_weights
from synth.machines import build_machine
from test_oracle_stationary import _two_face_machine, linear_profile

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


def _floor_machine():
    # 8x8x20 + 4x4x6 (1,876 DOF) whose stand stands on a 40 degC floor (h = 500)
    return build_machine("floor", (8, 8, 20), (4, 4, 6), floor=(500.0, 40.0))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_robin_faces_linear_profile(torch, precision):
    mach = _two_face_machine()
    s = _solver(mach, precision)
    iters = s.set_stationary_state(t0=0.0, rtol=1e-14)
    assert iters > 0
    T = s.temperature()
    nf = mach.stand.mesh.n_nodes
    np.testing.assert_allclose(T[:nf], linear_profile(mach), rtol=1e-11)
    np.testing.assert_allclose(T[nf:], mach.stock.T_env, rtol=1e-12)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stationary_state_matches_oracle_and_steps_from_it(torch, precision):
    mach = _floor_machine()
    prob = MachineProblem(mach)
    T_or = prob.stationary_state()
    s = _solver(mach, precision)
    s.set_stationary_state(t0=mach.t0, rtol=1e-13)
    T = s.temperature()
    rise = T_or - 20.0
    assert np.linalg.norm(T - T_or) / np.linalg.norm(T_or) <= 1e-12
    assert np.linalg.norm(T - T_or) / np.linalg.norm(rise) <= 1e-10
    # MRSDC from the stationary start: both sides from the oracle's state
    s.set_temperature(T_or, t0=mach.t0)
    sc = mach.scheme
    W = mrsdc_weights(sc.nodes, sc.M, sc.P, sc.window)
    X = T_or.copy()
    bar = 1e-10 if precision == "fp64" else 1e-6
    for n in range(2):
        rep = s.step(report=True)
        assert rep["status"] == 0
        X, _ = mrsdc_step(prob, X, mach.t0 + n * sc.dt, sc.dt, W, sc.sweeps)
        got = s.temperature()
        assert np.linalg.norm(got - X) / np.linalg.norm(X) <= bar
        assert np.linalg.norm(got - X) / np.linalg.norm(X - T_or) <= 1e2 * bar
    s.close()


def test_iteration_cap_is_reported_and_context_stays_usable(torch):
    from paper_1707_03581_gb300 import SdcError

    mach = _floor_machine()
    s = _solver(mach, "fp64")
    with pytest.raises(SdcError) as e:
        s.set_stationary_state(t0=0.0, rtol=1e-14, max_iter=2)
    assert "NOT_CONVERGED" in str(e.value)
    assert s.set_stationary_state(t0=0.0, rtol=1e-13) > 2
    s.step(report=True)
    s.close()
