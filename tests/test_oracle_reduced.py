"""The oracle's interface-only form (oracle.mrsdc.mrsdc_step_reduced), the fairer CPU baseline.

Off the contact f^E vanishes, so the P embedded substeps of an interval add up to one update
of the bulk (Algorithms 1 and 2 with sum_p S~[m,p,j] = S[m,j], sum_p S_emb[m,p,q] = S^[m,q]),
and only the interface DOFs need every substep. The reduced form must give the literal
step (mrsdc_step, itself pinned by test_oracle_stepper.py and test_oracle_bruteforce.py) to
rounding, on several node families, sweep counts and moving contacts; its f^E on the
interface must be the literal f^E restricted there, and the literal f^E must vanish off it.
"""

import numpy as np
import pytest

from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step, mrsdc_step_reduced, predictor_interval, predictor_interval_reduced
from oracle.weights import mrsdc_weights
from synth import machine_config, tiny_machine
from synth.machines import with_scheme


def _machines():
    return [
        with_scheme(tiny_machine(z0=0.37, amp=0.2, period=2.5), nodes="lobatto", M=3, P=6, sweeps=2),
        with_scheme(tiny_machine(z0=0.40, amp=0.15, period=3.1, q0=3.0e4), nodes="radau_right", M=2, P=5,
                    sweeps=3),
        with_scheme(machine_config(0), nodes="lobatto", M=3, P=8, sweeps=1),
    ]


@pytest.mark.parametrize("k", range(3))
def test_fE_on_the_interface_is_the_literal_fE_there(k):
    mach = _machines()[k]
    prob = MachineProblem(mach)
    rng = np.random.default_rng(k)
    T = 20.0 + rng.standard_normal(prob.n)
    for t in (0.0, 0.3, 1.1):
        full = prob.fE(T, t)
        red = prob.fE_iface(T[prob.iface], t)
        assert np.allclose(red, full[prob.iface], rtol=1e-14, atol=1e-12 * np.abs(full).max())
        off = np.ones(prob.n, dtype=bool)
        off[prob.iface] = False
        assert np.all(full[off] == 0.0)


@pytest.mark.parametrize("k", range(3))
def test_reduced_step_equals_literal_step(k):
    mach = _machines()[k]
    s = mach.scheme
    prob = MachineProblem(mach)
    W = mrsdc_weights(s.nodes, s.M, s.P, s.window)
    rng = np.random.default_rng(10 + k)
    T = mach.T0 + 0.5 * rng.standard_normal(prob.n)
    Ta, Tb = T.copy(), T.copy()
    for n in range(3):
        t = mach.t0 + n * s.dt
        Ta, _ = mrsdc_step(prob, Ta, t, s.dt, W, s.sweeps)
        Tb = mrsdc_step_reduced(prob, Tb, t, s.dt, W, s.sweeps)
        rise = np.linalg.norm(Ta - T)
        assert np.linalg.norm(Tb - Ta) <= 1e-12 * max(rise, 1.0), (n, np.linalg.norm(Tb - Ta), rise)


def test_reduced_predictor_interval_equals_literal():
    mach = _machines()[0]
    s = mach.scheme
    prob = MachineProblem(mach)
    W = mrsdc_weights(s.nodes, s.M, s.P, s.window)
    T = np.full(prob.n, mach.T0) + np.linspace(0.0, 1.0, prob.n)
    m = 1
    tau = [mach.t0 + s.dt * c for c in W["c"]]
    emb = [mach.t0 + s.dt * e for e in W["emb"][m]]
    Temb, it_a = predictor_interval(prob, T, tau[m], tau[m + 1], emb)
    T_m, Ti, it_b = predictor_interval_reduced(prob, T, tau[m], tau[m + 1], emb)
    assert it_a == it_b
    assert np.allclose(T_m, Temb[-1], rtol=1e-14, atol=0.0)
    for p in range(len(Ti)):
        assert np.allclose(Ti[p], Temb[p][prob.iface], rtol=1e-14, atol=0.0)
    # a bounded sample stops after the requested substeps
    T_none, Ti3, _ = predictor_interval_reduced(prob, T, tau[m], tau[m + 1], emb, n_substeps=3)
    assert T_none is None and len(Ti3) == 4
