"""Pins for oracle.mrsdc and oracle.linsolve (Sec. 3, Algorithms 1 and 2).

Checked against: the exact solution of the scalar IMEX equation
y' = lambda_s y + lambda_f(t) y (order min(M, P, k+1), property (ii)), the
directly solved collocation system (property (i): the sweeps converge to it),
implicit Euler and single-rate implicit SDC written out independently for
f^E = 0, exact conservation of total heat, and a dense Cholesky solve.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.linsolve import dense_solve, pcg
from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step
from oracle.weights import mrsdc_weights
from synth import machine_config, tiny_machine


class ScalarIMEX:
    """y' = ls y + a cos(om t) y; implicit part ls y, explicit part a cos(om t) y."""

    def __init__(self, ls=-1.0, a=1.0, om=5.0):
        self.ls, self.a, self.om = ls, a, om
        self.mass = np.ones(1)

    def fI(self, y):
        return self.ls * y

    def g(self, t):
        return np.zeros(1)

    def fE(self, y, t):
        return self.a * np.cos(self.om * t) * y

    def solve(self, dtau, rhs, x0):
        return rhs / (1.0 - dtau * self.ls), 0

    def exact(self, t):
        return np.exp(self.ls * t + self.a / self.om * np.sin(self.om * t))


def _scalar_error(W, sweeps, n):
    pr = ScalarIMEX()
    y = np.ones(1)
    dt = 1.0 / n
    for i in range(n):
        y, _ = mrsdc_step(pr, y, i * dt, dt, W, sweeps)
    return abs(y[0] - pr.exact(1.0))


@pytest.mark.parametrize("M,P,K", [(3, 2, k) for k in range(5)] + [(3, 8, k) for k in range(5)]
                         + [(5, 8, 0), (5, 8, 1), (5, 8, 2), (5, 8, 4)])
def test_scalar_imex_order(M, P, K):
    # the paper's experiment of property (ii): equidistant no-left nodes, literal weights
    W = mrsdc_weights("equi_noleft", M, P, window=P)
    e1, e2 = _scalar_error(W, K, 32), _scalar_error(W, K, 64)
    expected = min(M, P, K + 1)
    assert abs(np.log2(e1 / e2) - expected) < 0.2, (e1, e2, expected)


def _linear_ops(prob, t):
    """Dense L_I, L_E(t), e(t) with f^I = L_I T, f^E = L_E T + e (g folded into e_I)."""
    n = prob.n
    LI = -prob.K.toarray()
    E, e = prob.coupling_operator(t)
    return LI, E, e


def test_sweeps_converge_to_collocation_solution():
    # property (i): for a linear problem the fixed point of Algorithm 2 is the
    # solution of the discrete node-to-node equations (standard + embedded)
    mach = tiny_machine(z0=0.37, amp=0.2, period=3.0)
    prob = MachineProblem(mach, solver="dense")
    W = mrsdc_weights("radau_right", 2, 3, window=3)
    M, P = 2, 3
    dt, t_n = 5.0, 0.7
    n = prob.n
    rng = np.random.default_rng(0)
    T_n = 20.0 + rng.standard_normal(n)
    LI = -prob.K.toarray()
    g = prob.genv
    tau = [t_n + dt * c for c in W["c"]]
    tau_emb = [[t_n + dt * e for e in row] for row in W["emb"]]
    ops = [[prob.coupling_operator(tau_emb[m][q + 1]) for q in range(P)] for m in range(M)]
    # unknowns: U[m, p] = T_{m,p}, p = 1..P (T_m = U[m, P])
    N = M * P * n
    A = np.zeros((N, N))
    b = np.zeros(N)

    def idx(m, p):
        return (m * P + (p - 1)) * n

    mass = prob.mass
    for m in range(M):
        for p in range(1, P + 1):
            r = idx(m, p)
            A[r:r + n, r:r + n] += np.diag(mass)
            if p > 1:
                A[r:r + n, idx(m, p - 1):idx(m, p - 1) + n] -= np.diag(mass)
            elif m > 0:
                A[r:r + n, idx(m - 1, P):idx(m - 1, P) + n] -= np.diag(mass)
            else:
                b[r:r + n] += mass * T_n
            for j in range(M):
                w = dt * W["Stil"][m, p - 1, j]
                A[r:r + n, idx(j, P):idx(j, P) + n] -= w * LI
                b[r:r + n] += w * g
            for q in range(P):
                w = dt * W["Semb"][m, p - 1, q]
                E, e = ops[m][q]
                A[r:r + n, idx(m, q + 1):idx(m, q + 1) + n] -= w * E
                b[r:r + n] += w * e
    U = np.linalg.solve(A, b)
    T_coll = U[idx(M - 1, P):idx(M - 1, P) + n]
    T_sdc, res = mrsdc_step(prob, T_n, t_n, dt, W, 40, want_residuals=True)
    assert np.abs(T_sdc - T_coll).max() < 1e-11 * np.abs(T_coll).max()
    assert res.residuals[-1] < 1e-9 * res.residuals[0]
    assert res.residuals[3] < res.residuals[1] < res.residuals[0]


def test_no_contact_predictor_is_implicit_euler_and_sweeps_are_implicit_sdc():
    mach = tiny_machine()
    prob = MachineProblem(mach, solver="dense", with_contact=False)
    W = mrsdc_weights("radau_right", 3, 4)
    dt, t_n = 40.0, 0.0
    rng = np.random.default_rng(2)
    T_n = 20.0 + rng.standard_normal(prob.n)
    mass, K, g = prob.mass, prob.K.toarray(), prob.genv
    c = W["c"]
    # implicit Euler node to node
    T = T_n.copy()
    T_pred = []
    for m in range(3):
        dtau = dt * (c[m + 1] - c[m])
        T = np.linalg.solve(np.diag(mass) + dtau * K, mass * T + dtau * g)
        T_pred.append(T)
    _, r0 = mrsdc_step(prob, T_n, t_n, dt, W, 0, keep_nodes=True)
    for m in range(3):
        np.testing.assert_allclose(r0.T_std[m + 1], T_pred[m], rtol=1e-13, atol=0)
    # two single-rate implicit SDC sweeps (Eq. sdc_sweep with f^E = 0)
    Tk = list(T_pred)
    for _ in range(2):
        F = [-(K @ Tk[j]) + g for j in range(3)]
        new = []
        prev = T_n
        for m in range(3):
            dtau = dt * (c[m + 1] - c[m])
            I = sum(dt * W["S"][m, j] * F[j] for j in range(3))
            rhs = mass * prev - dtau * (-(K @ Tk[m])) + I
            prev = np.linalg.solve(np.diag(mass) + dtau * K, rhs)
            new.append(prev)
        Tk = new
    _, r2 = mrsdc_step(prob, T_n, t_n, dt, W, 2, keep_nodes=True)
    for m in range(3):
        np.testing.assert_allclose(r2.T_std[m + 1], Tk[m], rtol=1e-12, atol=0)


def test_conservation_insulated_no_friction():
    mach = machine_config(0)
    mach.stand.h = 0.0
    mach.stock.h = 0.0
    mach.q0 = 0.0
    prob = MachineProblem(mach)
    W = mrsdc_weights("lobatto", 3, 20)
    xyz = np.concatenate([mach.stand.mesh.xyz, mach.stock.mesh.xyz])
    T = 20.0 + 5.0 * np.sin(3.0 * xyz[:, 2]) + (np.arange(prob.n) >= prob.n_fix) * 8.0
    Q0 = sum(prob.heat(T))
    for i in range(3):
        T, _ = mrsdc_step(prob, T, float(i), 1.0, W, 3)
    Q1 = sum(prob.heat(T))
    assert abs(Q1 - Q0) < 1e-13 * Q0
    # heat did move from the hot stock into the stand
    assert prob.heat(T)[0] > 0


def test_pcg_matches_cholesky():
    prob = MachineProblem(machine_config(0))
    rng = np.random.default_rng(4)
    b = prob.mass * (20.0 + rng.standard_normal(prob.n))
    A = sp.diags(prob.mass) + 0.5 * prob.K
    dinv = 1.0 / A.diagonal()
    x, it, ok = pcg(lambda v: A @ v, b, np.zeros(prob.n), dinv, 1e-12, 500)
    xd = dense_solve(A.toarray(), b)
    assert ok and it > 0
    assert np.abs(x - xd).max() < 1e-10 * np.abs(xd).max()


def test_hand_trace_scalar_one_step():
    # M = 1 standard node (c = 1), P = 2 literal embedded nodes; predictor and one
    # sweep written out by hand for y' = ls y + a cos(om t) y. The explicit Euler
    # step takes f^E at the left embedded node (Algorithm 1), the quadrature at
    # tau_{m,q}, q = 1..P (Eq. embedded_quad).
    pr = ScalarIMEX(ls=-0.7, a=1.3, om=2.0)
    W = mrsdc_weights("equi_noleft", 1, 2, window=2)
    dt, t0, y0 = 0.4, 0.25, 1.5
    lam = lambda t: pr.a * np.cos(pr.om * t)
    t1, t2 = t0 + dt / 2, t0 + dt
    # predictor
    ys = y0 / (1 + 0.7 * dt)
    fs = -0.7 * ys
    y1 = y0 + dt / 2 * (fs + lam(t0) * y0)
    y2 = y1 + dt / 2 * (fs + lam(t1) * y1)
    got, _ = mrsdc_step(pr, np.array([y0]), t0, dt, W, 0)
    assert abs(got[0] - y2) < 1e-15
    # one sweep: s_{1,1} = dt; embedded Lagrange basis on the nodes t1, t2 is
    # l_1 = (t2 - t)/h, l_2 = (t - t1)/h with h = dt/2, integrated by hand:
    h = dt / 2
    s11 = (h * 1.5, -h * 0.5)       # int over [t0, t1] of (l_1, l_2)
    s12 = (h * 0.5, h * 0.5)        # int over [t1, t2]
    F_I = -0.7 * y2
    fe1, fe2 = lam(t1) * y1, lam(t2) * y2
    I1 = h * F_I + s11[0] * fe1 + s11[1] * fe2
    I2 = h * F_I + s12[0] * fe1 + s12[1] * fe2
    Istd = dt * F_I + (s11[0] + s12[0]) * fe1 + (s11[1] + s12[1]) * fe2
    ys = (y0 - dt * (-0.7 * y2) + Istd) / (1 + 0.7 * dt)
    fs = -0.7 * ys - (-0.7 * y2)
    z1 = y0 + h * fs + h * (lam(t0) * y0 - lam(t0) * y0) + I1
    z2 = z1 + h * fs + h * (lam(t1) * z1 - lam(t1) * y1) + I2
    got, _ = mrsdc_step(pr, np.array([y0]), t0, dt, W, 1)
    assert abs(got[0] - z2) < 1e-14
