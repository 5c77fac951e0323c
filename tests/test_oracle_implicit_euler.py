"""Pins for oracle.mrsdc.implicit_euler_step, fully implicit Euler with the
contact coupling in the matrix (the comparison method of Sec. 1 and Sec. 5).

Checked against: first order on the scalar equation y' = ls y + a cos(om t) y
with both terms implicit, the closed form of one scalar step, implicit Euler
written out when f^E = 0 (MRSDC's predictor with one Radau node), exact
conservation of total heat for insulated, frictionless bodies, and the
operator E(t) against f^E evaluated directly.
"""

import dataclasses

import numpy as np
import scipy.sparse as sp

from oracle.machine import MachineProblem
from oracle.mrsdc import implicit_euler_step, mrsdc_step
from oracle.weights import mrsdc_weights
from synth import tiny_machine
from test_oracle_stepper import ScalarIMEX


class ScalarLinear(ScalarIMEX):
    def fI_matrix(self):
        return sp.csr_matrix([[self.ls]])

    def contact_matrix(self, t):
        return sp.csr_matrix([[self.a * np.cos(self.om * t)]]), np.zeros(1)


def test_scalar_closed_form_and_first_order():
    pr = ScalarLinear()
    y1 = implicit_euler_step(pr, np.array([1.3]), 0.2, 0.1)
    exact_step = 1.3 / (1.0 - 0.1 * (pr.ls + pr.a * np.cos(pr.om * 0.3)))
    assert abs(y1[0] - exact_step) <= 1e-15 * abs(exact_step)

    def err(n):
        y, dt = np.ones(1), 1.0 / n
        for i in range(n):
            y = implicit_euler_step(pr, y, i * dt, dt)
        return abs(y[0] - pr.exact(1.0))

    assert abs(np.log2(err(256) / err(512)) - 1.0) < 0.05


def test_without_contact_it_is_implicit_euler():
    prob = MachineProblem(tiny_machine(), solver="dense", with_contact=False)
    rng = np.random.default_rng(4)
    T_n = 20.0 + rng.standard_normal(prob.n)
    a = implicit_euler_step(prob, T_n, 0.0, 25.0)
    b, _ = mrsdc_step(prob, T_n, 0.0, 25.0, mrsdc_weights("radau_right", 1, 1), 0)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


def test_contact_matrix_reproduces_fE_and_heat_is_conserved():
    mach = tiny_machine(z0=0.37, amp=0.21, period=1.7, q0=0.0)
    mach = dataclasses.replace(mach, stand=dataclasses.replace(mach.stand, h=0.0),
                               stock=dataclasses.replace(mach.stock, h=0.0))
    prob = MachineProblem(mach)
    rng = np.random.default_rng(9)
    T = 20.0 + 3.0 * rng.standard_normal(prob.n)
    E, e = prob.contact_matrix(0.6)
    np.testing.assert_allclose(E @ T + e, prob.fE(T, 0.6), rtol=1e-12, atol=1e-9)
    heat0 = prob.mass @ T
    for n in range(3):
        T = implicit_euler_step(prob, T, 0.6 + 0.5 * n, 0.5)
    assert abs(prob.mass @ T - heat0) <= 1e-12 * abs(heat0)


def test_coupling_is_symmetric_and_negative_semidefinite():
    # Reading of the implicit Euler operator: L_E(t) is symmetric (both bodies' exchange uses one
    # overlap quadrature) and negative semidefinite (it only exchanges heat), so that
    # m + dt (K - L_E) is SPD and Jacobi-PCG applies. Checked at several stroke positions.
    mach = tiny_machine(z0=0.37, amp=0.21, period=1.7)
    prob = MachineProblem(mach)
    for t in (0.0, 0.3, 0.9, 1.4):
        E, _ = prob.contact_matrix(t)
        Ed = E.toarray()
        assert np.abs(Ed - Ed.T).max() <= 1e-12 * np.abs(Ed).max()
        assert np.abs(Ed).max() > 0.0
        lam = np.linalg.eigvalsh(0.5 * (Ed + Ed.T))
        assert lam.max() <= 1e-10 * np.abs(lam).max()
        # rows sum to zero: a uniform temperature exchanges no heat
        np.testing.assert_allclose(Ed.sum(axis=1), 0.0, atol=1e-10 * np.abs(Ed).max())
        A = np.diag(prob.mass) - 5.0 * prob.fI_matrix().toarray() - 5.0 * Ed
        assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0.0
