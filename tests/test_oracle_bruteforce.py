"""Whole-system pin: dense matrix-exponential brute force on a <= 200-DOF machine.

With the stock at rest (period = inf: constant position, constant friction
flux q0) the coupled system of Eq. coupledFEM is linear time-invariant,
M T' = L T + c with L = -K + E symmetric. Its exact solution is
T(t) = T_inf + M^{-1/2} V exp(t Lambda) V^T M^{1/2} (T0 - T_inf) from the
symmetric eigendecomposition of M^{-1/2} L M^{-1/2}. Converged MRSDC must
reproduce it up to the collocation error.
"""

import numpy as np

from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step
from oracle.weights import mrsdc_weights
from synth import tiny_machine


def test_resting_stock_matches_matrix_exponential():
    mach = tiny_machine(z0=0.37, amp=0.25, period=np.inf, q0=3.0e4)
    assert mach.n_dof <= 200
    prob = MachineProblem(mach, solver="dense")
    E, e = prob.coupling_operator(0.0)
    L = -prob.K.toarray() + E
    assert np.abs(L - L.T).max() < 1e-9 * np.abs(L).max()
    cvec = prob.genv + e
    m = prob.mass
    T_inf = np.linalg.solve(-L, cvec)
    S = L / np.sqrt(m)[:, None] / np.sqrt(m)[None, :]
    lam, V = np.linalg.eigh(0.5 * (S + S.T))
    assert lam.max() < 0

    xyz = np.concatenate([mach.stand.mesh.xyz, mach.stock.mesh.xyz])
    T0 = 20.0 + 2.0 * np.cos(4.0 * xyz[:, 2]) + (np.arange(prob.n) >= prob.n_fix) * 3.0
    t_end, dt = 40.0, 2.0

    def exact(t):
        y0 = V.T @ (np.sqrt(m) * (T0 - T_inf))
        return T_inf + (V @ (np.exp(lam * t) * y0)) / np.sqrt(m)

    for kind, M, P, K in (("radau_right", 3, 4, 8), ("lobatto", 3, 5, 6)):
        W = mrsdc_weights(kind, M, P)
        T = T0.copy()
        for i in range(int(t_end / dt)):
            T, _ = mrsdc_step(prob, T, i * dt, dt, W, K)
        ref = exact(t_end)
        rise = np.abs(ref - T0).max()
        assert rise > 0.1
        assert np.abs(T - ref).max() < 1e-8 * rise, (kind, np.abs(T - ref).max(), rise)
