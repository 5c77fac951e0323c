"""IMEX multi-rate SDC, Algorithms 1 and 2 taken literally, and for comparison
single-rate semi-implicit SDC (Sec. 3) and fully implicit Euler with the
coupling in the matrix (Sec. 1, Sec. 5) (oracle; test infrastructure only).

Problem interface (any object with):
    mass           (N,) diagonal of M (lumped)
    fI(T)          the slow, linear, implicit term f^I(T)
    g(t)           the slow source g(t)
    fE(T, t)       the fast explicit term f^E(T, t)
    solve(dtau, rhs, x0) -> (x, iters)   solves  mass * x - dtau * fI(x) = rhs

One macro step [t_n, t_n + dt] with standard nodes tau_m = t_n + dt c_m and
embedded nodes tau_{m,p} (see oracle.weights):

Algorithm 1 (predictor), for m = 1..M:
    solve  M T*_m = M T_{m-1} + dtau_m (f^I(T*_m) + g(tau_m))
    f*_m = f^I(T*_m) + g(tau_m)
    T_{m,0} = T_{m-1};  for p = 1..P:
        M T_{m,p} = M T_{m,p-1} + dt_{m,p} (f*_m + f^E(T_{m,p-1}, tau_{m,p-1}))
    T_m = T_{m,P}

Algorithm 2 (sweep k -> k+1): build I_{m-1}^m (Eq. standard_quad) and
I_{m,p-1}^p (Eq. embedded_quad) from iterate k; T_0 = T(t_n); for m = 1..M:
    solve  M T*_m = M T^{k+1}_{m-1} + dtau_m (f^I(T*_m) - f^I(T^k_m)) + I_{m-1}^m
    f*_m = f^I(T*_m) - f^I(T^k_m)
    T_{m,0} = T^{k+1}_{m-1};  for p = 1..P:
        M T_{m,p} = M T_{m,p-1} + dt_{m,p} f*_m
                    + dt_{m,p} (f^E(T^{k+1}_{m,p-1}, tau_{m,p-1}) - f^E(T^k_{m,p-1}, tau_{m,p-1}))
                    + I_{m,p-1}^p
    T^{k+1}_m = T^{k+1}_{m,P}

Full vectors are kept at every embedded node; nothing is specialised to the
location of the contact, so the fast library path (which runs the P substeps
only on contact DOFs) is checked against this plain form. mrsdc_step_reduced
and predictor_interval_reduced take the substeps on the interface only (the
fairer CPU baseline); they are pinned to the literal form by
tests/test_oracle_reduced.py and serve no parity test.

Residual (Eq. residual, with the sum index read as j, i.e. sum_{j<=m} I_{j-1}^j):
    r^k = max_m || M T^k_m - M T(t_n) - sum_{j=1}^m I_{j-1}^j ||_inf
computed from iterate k (and its own quadrature).

Readings: g is evaluated at tau_m in the predictor (Algorithm 1 includes it
in f*); the explicit Euler step uses f^E at the left embedded node
tau_{m,p-1}; quadratures use f^E at tau_{m,q}, q = 1..P. A zero-length
interval (Lobatto, m = 1) is run as written: its solve returns T_{m-1} and
its substeps have zero length.

Parity: pinned by tests/test_oracle_stepper.py (order min(M, w, k+1) on the
scalar IMEX equation, convergence of the sweeps to the directly solved
collocation system, equality with implicit Euler / implicit SDC when f^E = 0,
conservation of total heat) and tests/test_oracle_bruteforce.py (matrix
exponential of a <= 200-DOF machine).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class StepResult:
    def __init__(self):
        self.residuals = []
        self.cg_iters = []
        self.T_std = None
        self.T_emb = None


def _quadratures(prob, T_std, T_emb, tau, tau_emb, W, dt):
    """F^I_j, f^E at embedded nodes and the integrals I_{m-1}^m, I_{m,p-1}^p of one iterate."""
    M, P = W["M"], W["P"]
    FI = [prob.fI(T_std[j + 1]) + prob.g(tau[j + 1]) for j in range(M)]
    FE = [[prob.fE(T_emb[m][q], tau_emb[m][q]) for q in range(P + 1)] for m in range(M)]
    I_std = []
    I_emb = []
    for m in range(M):
        acc = np.zeros_like(T_std[0])
        for j in range(M):
            acc = acc + dt * W["S"][m, j] * FI[j]
        for q in range(P):
            acc = acc + dt * W["Shat"][m, q] * FE[m][q + 1]
        I_std.append(acc)
        row = []
        for p in range(P):
            acc = np.zeros_like(T_std[0])
            for j in range(M):
                acc = acc + dt * W["Stil"][m, p, j] * FI[j]
            for q in range(P):
                acc = acc + dt * W["Semb"][m, p, q] * FE[m][q + 1]
            row.append(acc)
        I_emb.append(row)
    return FI, FE, I_std, I_emb


def _residual(prob, T_n, T_std, I_std):
    M = len(I_std)
    cum = np.zeros_like(T_n)
    r = 0.0
    for m in range(M):
        cum = cum + I_std[m]
        res = prob.mass * T_std[m + 1] - prob.mass * T_n - cum
        r = max(r, float(np.max(np.abs(res))))
    return r


def predictor_interval(prob, T_left, tau_left, tau_right, tau_emb_m, n_substeps=None):
    """Algorithm 1 on one interval [tau_{m-1}, tau_m]: the implicit solve for T*_m, f*_m, then
    the explicit substeps T_{m,p}, p = 1..P, on the embedded nodes tau_emb_m[0..P]. Returns
    ([T_{m,0}, ..., T_{m,P}], CG iterations). n_substeps < P stops after that many substeps
    (a bounded sample of the interval's work; the list then ends at T_{m,n_substeps})."""
    mass = prob.mass
    P = len(tau_emb_m) - 1
    dtau = tau_right - tau_left
    rhs = mass * T_left + dtau * prob.g(tau_right)
    Tstar, it = prob.solve(dtau, rhs, T_left)
    fstar = prob.fI(Tstar) + prob.g(tau_right)
    T_emb = [T_left.copy()]
    for p in range(1, (P if n_substeps is None else min(P, n_substeps)) + 1):
        dtp = tau_emb_m[p] - tau_emb_m[p - 1]
        incr = dtp * (fstar + prob.fE(T_emb[p - 1], tau_emb_m[p - 1]))
        T_emb.append(T_emb[p - 1] + incr / mass)
    return T_emb, it


def mrsdc_step(prob, T_n, t_n, dt, W, sweeps, want_residuals=False, keep_nodes=False):
    """One macro step; returns (T(t_n + dt), StepResult)."""
    M, P = W["M"], W["P"]
    c, emb = W["c"], W["emb"]
    tau = [t_n + dt * c[m] for m in range(M + 1)]          # tau[0] = t_n
    tau_emb = [[t_n + dt * emb[m][p] for p in range(P + 1)] for m in range(M)]
    mass = prob.mass
    res = StepResult()

    # ---------------- Algorithm 1: predictor ----------------
    T_std = [T_n.copy()] + [None] * M
    T_emb = [None] * M
    for m in range(M):
        T_emb[m], it = predictor_interval(prob, T_std[m], tau[m], tau[m + 1], tau_emb[m])
        res.cg_iters.append(it)
        T_std[m + 1] = T_emb[m][P]

    # ---------------- Algorithm 2: sweeps ----------------
    for k in range(sweeps):
        FI, FE, I_std, I_emb = _quadratures(prob, T_std, T_emb, tau, tau_emb, W, dt)
        if want_residuals:
            res.residuals.append(_residual(prob, T_n, T_std, I_std))
        new_std = [T_n.copy()] + [None] * M
        new_emb = [[None] * (P + 1) for _ in range(M)]
        for m in range(M):
            dtau = tau[m + 1] - tau[m]
            fI_old = FI[m] - prob.g(tau[m + 1])            # f^I(T^k_m)
            rhs = mass * new_std[m] - dtau * fI_old + I_std[m]
            Tstar, it = prob.solve(dtau, rhs, T_std[m + 1])
            res.cg_iters.append(it)
            fstar = prob.fI(Tstar) - fI_old
            new_emb[m][0] = new_std[m].copy()
            for p in range(1, P + 1):
                dtp = tau_emb[m][p] - tau_emb[m][p - 1]
                fe_new = prob.fE(new_emb[m][p - 1], tau_emb[m][p - 1])
                fe_old = FE[m][p - 1]                       # f^E(T^k_{m,p-1}, tau_{m,p-1})
                incr = dtp * fstar + dtp * (fe_new - fe_old) + I_emb[m][p - 1]
                new_emb[m][p] = new_emb[m][p - 1] + incr / mass
            new_std[m + 1] = new_emb[m][P]
        T_std, T_emb = new_std, new_emb

    if want_residuals:
        _, _, I_std, _ = _quadratures(prob, T_std, T_emb, tau, tau_emb, W, dt)
        res.residuals.append(_residual(prob, T_n, T_std, I_std))
    if keep_nodes:
        res.T_std, res.T_emb = T_std, T_emb
    return T_std[M].copy(), res


# ---------------------------------------------------------------------------
# The same step with the embedded substeps taken on the interface only (the fairer CPU
# baseline). Off the contact f^E vanishes, so there the P substeps of an interval add up to
#   M T_m = M T_{m-1} + dtau_m f*_m + I_{m-1}^m
# (sum_p dt_{m,p} = dtau_m; sum_p S~[m,p,j] = S[m,j] and sum_p S_emb[m,p,q] = S^[m,q], and the
# f^E terms of I_{m-1}^m are zero there), and only the interface DOFs (prob.iface, with
# prob.fE_iface) need every substep. Equal to mrsdc_step up to the order of rounding.
# The problem object also provides iface (sorted interface DOFs) and fE_iface(Ti, t).


def predictor_interval_reduced(prob, T_left, tau_left, tau_right, tau_emb_m, n_substeps=None):
    """predictor_interval with the substeps on the interface: returns (T_m, the interface
    temperatures [T_{m,0}, ..., T_{m,P}] there, CG iterations). n_substeps < P stops after that
    many interface substeps (a bounded sample; T_m is then None)."""
    mass, I = prob.mass, prob.iface
    P = len(tau_emb_m) - 1
    dtau = tau_right - tau_left
    rhs = mass * T_left + dtau * prob.g(tau_right)
    Tstar, it = prob.solve(dtau, rhs, T_left)
    fstar = prob.fI(Tstar) + prob.g(tau_right)
    Ti = [T_left[I].copy()]
    mi, fi = mass[I], fstar[I]
    for p in range(1, (P if n_substeps is None else min(P, n_substeps)) + 1):
        dtp = tau_emb_m[p] - tau_emb_m[p - 1]
        Ti.append(Ti[p - 1] + dtp * (fi + prob.fE_iface(Ti[p - 1], tau_emb_m[p - 1])) / mi)
    if len(Ti) < P + 1:
        return None, Ti, it
    T_m = T_left + dtau * fstar / mass
    T_m[I] = Ti[P]
    return T_m, Ti, it


def mrsdc_step_reduced(prob, T_n, t_n, dt, W, sweeps):
    """One macro step as mrsdc_step, substeps on the interface only; returns T(t_n + dt)."""
    M, P = W["M"], W["P"]
    c, emb = W["c"], W["emb"]
    tau = [t_n + dt * c[m] for m in range(M + 1)]
    tau_emb = [[t_n + dt * emb[m][p] for p in range(P + 1)] for m in range(M)]
    mass, I = prob.mass, prob.iface
    mi = mass[I]

    # Algorithm 1, and f^E of the predictor at every embedded node of the interface
    T_std = [T_n.copy()] + [None] * M
    FE = [None] * M
    for m in range(M):
        T_std[m + 1], Ti, _ = predictor_interval_reduced(prob, T_std[m], tau[m], tau[m + 1], tau_emb[m])
        FE[m] = [prob.fE_iface(Ti[q], tau_emb[m][q]) for q in range(P + 1)]

    # Algorithm 2
    for k in range(sweeps):
        FI = [prob.fI(T_std[j + 1]) + prob.g(tau[j + 1]) for j in range(M)]
        new_std = [T_n.copy()] + [None] * M
        new_FE = [None] * M
        for m in range(M):
            dtau = tau[m + 1] - tau[m]
            I_std = np.zeros_like(T_n)
            for j in range(M):
                I_std = I_std + dt * W["S"][m, j] * FI[j]
            for q in range(P):
                I_std[I] = I_std[I] + dt * W["Shat"][m, q] * FE[m][q + 1]
            fI_old = FI[m] - prob.g(tau[m + 1])
            rhs = mass * new_std[m] - dtau * fI_old + I_std
            Tstar, _ = prob.solve(dtau, rhs, T_std[m + 1])
            fstar = prob.fI(Tstar) - fI_old
            # off the contact: the substeps' sum
            T_m = new_std[m] + (dtau * fstar + I_std) / mass
            # on the contact: every substep
            Ti = new_std[m][I].copy()
            fe_row = [prob.fE_iface(Ti, tau_emb[m][0])]
            for p in range(1, P + 1):
                dtp = tau_emb[m][p] - tau_emb[m][p - 1]
                I_emb = np.zeros(I.size)
                for j in range(M):
                    I_emb = I_emb + dt * W["Stil"][m, p - 1, j] * FI[j][I]
                for q in range(P):
                    I_emb = I_emb + dt * W["Semb"][m, p - 1, q] * FE[m][q + 1]
                fe_new = fe_row[p - 1]
                Ti = Ti + (dtp * fstar[I] + dtp * (fe_new - FE[m][p - 1]) + I_emb) / mi
                fe_row.append(prob.fE_iface(Ti, tau_emb[m][p]))
            T_m[I] = Ti
            new_std[m + 1] = T_m
            new_FE[m] = fe_row
        T_std, FE = new_std, new_FE
    return T_std[M].copy()


def sisdc_step(prob, T_n, t_n, dt, W, sweeps, want_residuals=False):
    """One macro step of single-rate semi-implicit SDC (Sec. 3), the method MRSDC
    extends; returns (T(t_n + dt), StepResult). f^E is evaluated only at the
    standard nodes:

    predictor (IMEX Euler from node to node), for m = 1..M:
        M T_m = M T_{m-1} + dtau_m (f^I(T_m) + g(tau_m)) + dtau_m f^E(T_{m-1}, tau_{m-1})
    sweep (Eq. sdc_sweep), for m = 1..M:
        M T^{k+1}_m = M T^{k+1}_{m-1} + dtau_m (f^I(T^{k+1}_m) - f^I(T^k_m))
                      + dtau_m (f^E(T^{k+1}_{m-1}, tau_{m-1}) - f^E(T^k_{m-1}, tau_{m-1}))
                      + I_{m-1}^m,
        I_{m-1}^m = sum_j s_{m,j} F(T^k_j, tau_j),  F = f^I + g + f^E.

    The residual (Eq. residual) uses this I_{m-1}^m."""
    M = W["M"]
    c = W["c"]
    tau = [t_n + dt * c[m] for m in range(M + 1)]          # tau[0] = t_n
    mass = prob.mass
    res = StepResult()

    def quadrature(T):
        F = [prob.fI(T[j + 1]) + prob.g(tau[j + 1]) + prob.fE(T[j + 1], tau[j + 1]) for j in range(M)]
        I = []
        for m in range(M):
            acc = np.zeros_like(T_n)
            for j in range(M):
                acc = acc + dt * W["S"][m, j] * F[j]
            I.append(acc)
        return I

    T = [T_n.copy()] + [None] * M
    for m in range(M):
        dtau = tau[m + 1] - tau[m]
        rhs = mass * T[m] + dtau * (prob.g(tau[m + 1]) + prob.fE(T[m], tau[m]))
        T[m + 1], it = prob.solve(dtau, rhs, T[m])
        res.cg_iters.append(it)
    for k in range(sweeps):
        I = quadrature(T)
        if want_residuals:
            res.residuals.append(_residual(prob, T_n, T, I))
        fe_left_old = [prob.fE(T[m], tau[m]) for m in range(M)]   # f^E(T^k_{m-1}, tau_{m-1})
        new = [T_n.copy()] + [None] * M
        for m in range(M):
            dtau = tau[m + 1] - tau[m]
            fI_old = prob.fI(T[m + 1])                            # f^I(T^k_m)
            rhs = (mass * new[m] - dtau * fI_old
                   + dtau * (prob.fE(new[m], tau[m]) - fe_left_old[m]) + I[m])
            new[m + 1], it = prob.solve(dtau, rhs, T[m + 1])
            res.cg_iters.append(it)
        T = new
    if want_residuals:
        res.residuals.append(_residual(prob, T_n, T, quadrature(T)))
    return T[M].copy(), res


def implicit_euler_step(prob, T_n, t_n, dt):
    """One step of fully implicit Euler with the contact coupling in the matrix, the
    comparison method of Sec. 1 and Sec. 5 (oracle):

        M T_{n+1} = M T_n + dt (f^I(T_{n+1}) + g(t_{n+1}) + f^E(T_{n+1}, t_{n+1})),

    with f^I = L_I T and f^E(T, t) = E(t) T + e(t) affine in T, i.e. the sparse direct
    solve of (M - dt L_I - dt E(t_{n+1})) T_{n+1} = M T_n + dt (g(t_{n+1}) + e(t_{n+1}))."""
    t1 = t_n + dt
    E, e = prob.contact_matrix(t1)
    A = sp.diags(prob.mass) - dt * prob.fI_matrix() - dt * E
    rhs = prob.mass * T_n + dt * (prob.g(t1) + e)
    return spla.spsolve(sp.csc_matrix(A), rhs)


def run(prob, T0, t0, dt, W, sweeps, n_steps, callback=None):
    """n_steps macro steps from (T0, t0); t_n = t0 + n dt (no accumulated sum)."""
    T = np.array(T0, dtype=np.float64, copy=True)
    for n in range(n_steps):
        T, r = mrsdc_step(prob, T, t0 + n * dt, dt, W, sweeps)
        if callback is not None:
            callback(n, T, r)
    return T
