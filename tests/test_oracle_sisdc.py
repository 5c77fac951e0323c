"""Pins for oracle.mrsdc.sisdc_step, single-rate semi-implicit SDC (Sec. 3).

Checked against: the exact solution of the scalar IMEX equation (order
min(M, k+1) with M equidistant nodes), the directly solved collocation system
with f^E at the standard nodes (the sweeps' fixed point), IMEX Euler written
out node by node (the predictor), and MRSDC when f^E = 0 (both are then
implicit SDC).
"""

import numpy as np
import pytest

from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step, sisdc_step
from oracle.weights import mrsdc_weights
from synth import tiny_machine
from test_oracle_stepper import ScalarIMEX


def _scalar_error(W, sweeps, n):
    pr = ScalarIMEX(ls=-4.0, a=3.0, om=7.0)
    y = np.ones(1)
    dt = 1.0 / n
    for i in range(n):
        y, _ = sisdc_step(pr, y, i * dt, dt, W, sweeps)
    return abs(y[0] - pr.exact(1.0))


@pytest.mark.parametrize("K", [0, 1, 2, 3])
def test_scalar_order_is_min_M_k_plus_1(K):
    # measured 1.00, 1.97, 2.96, 3.93 between 128 and 256 steps
    W = mrsdc_weights("equi_noleft", 5, 1)
    e1, e2 = _scalar_error(W, K, 128), _scalar_error(W, K, 256)
    assert abs(np.log2(e1 / e2) - min(5, K + 1)) < 0.15, (e1, e2)


def test_sweeps_converge_to_the_standard_collocation_solution():
    pr = ScalarIMEX(ls=-2.0, a=1.5, om=3.0)
    W = mrsdc_weights("radau_right", 3, 1)
    t_n, dt, y_n = 0.3, 0.2, 1.7
    y, _ = sisdc_step(pr, np.array([y_n]), t_n, dt, W, 60)
    # y_m = y_n + sum_j q_{m,j} (ls + a cos(om tau_j)) y_j, q_{m,j} = sum_{i <= m} s_{i,j}
    M = W["M"]
    Q = np.cumsum(dt * np.asarray(W["S"]), axis=0)
    tau = t_n + dt * np.asarray(W["c"][1:])
    lam = pr.ls + pr.a * np.cos(pr.om * tau)
    ys = np.linalg.solve(np.eye(M) - Q * lam[None, :], np.full(M, y_n))
    assert abs(y[0] - ys[-1]) <= 1e-13 * abs(ys[-1])


def test_predictor_is_imex_euler_node_to_node():
    pr = ScalarIMEX()
    W = mrsdc_weights("radau_right", 3, 1)
    t_n, dt, y = 0.1, 0.25, 1.3
    tau = t_n + dt * np.asarray(W["c"])
    for m in range(3):
        dtau = tau[m + 1] - tau[m]
        y = (y + dtau * pr.a * np.cos(pr.om * tau[m]) * y) / (1.0 - dtau * pr.ls)
    got, _ = sisdc_step(pr, np.array([1.3]), t_n, dt, W, 0)
    assert abs(got[0] - y) <= 1e-15 * abs(y)


@pytest.mark.parametrize("K", [0, 2])
def test_without_contact_it_is_mrsdc(K):
    # f^E = 0: both methods are implicit Euler predictor + implicit SDC sweeps
    prob = MachineProblem(tiny_machine(), solver="dense", with_contact=False)
    W = mrsdc_weights("radau_right", 3, 4)
    rng = np.random.default_rng(8)
    T_n = 20.0 + rng.standard_normal(prob.n)
    a, _ = sisdc_step(prob, T_n, 0.0, 30.0, W, K)
    b, _ = mrsdc_step(prob, T_n, 0.0, 30.0, W, K)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=0)
