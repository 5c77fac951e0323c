"""The reduced problem of Sec. 4 (synth.slab_machine) on the GPU: parity with
the oracle, and the two properties Sec. 4 demonstrates with it.

(i)  The SDC residual decays with the sweep count k: every sweep divides it by a
     factor proportional to dt (so after k sweeps it carries dt^k).
(ii) The measured order of MRSDC with k sweeps is min(M, P, k + 1), for
     (M, P) = (5, 8) and (5, 2) with the literal embedded weights.

The slab's diffusion and contact rates are about 0.1/s and 1.6/s, so a 2 s
horizon resolves the orders well above the solver tolerance.
"""

import os

import numpy as np
import pytest

from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step
from oracle.weights import mrsdc_weights
from synth.machines import Scheme, slab_machine

pytestmark = pytest.mark.gpu

T_END = 2.0


def _expected_orders():
    # tests/golden/orders_sec4.txt: the orders the figure of Sec. 4 states, by (M, P, k)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "orders_sec4.txt")
    with open(path) as f:
        rows = [line.split() for line in f if line.strip() and not line.startswith("#")]
    return {(int(M), int(P), int(k)): int(q) for M, P, k, q in rows}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _slab(M, P, K, dt, ny=4, nz=16, capacity_ratio=1e12):
    return slab_machine(ny, nz, scheme=Scheme("equi_noleft", M, P, K, P, dt, 1e-14, 4000), rho=10.0, c=1000.0,
                        capacity_ratio=capacity_ratio)


def _gpu_run(mach, T0, n_steps, precision="fp64", residuals=False):
    from paper_1707_03581_gb300 import Solver

    s = Solver(0)
    s.set_machine(mach, precision=precision, T0=T0, residuals=residuals)
    reps = [s.step(report=True) for _ in range(n_steps)]
    T = s.temperature()
    s.close()
    return T, reps


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab_matches_oracle(torch, precision):
    mach, T0 = _slab(5, 8, 2, 0.5)
    prob = MachineProblem(mach)
    sc = mach.scheme
    W = mrsdc_weights(sc.nodes, sc.M, sc.P, sc.window)
    X = T0.copy()
    for n in range(3):
        X, _ = mrsdc_step(prob, X, mach.t0 + n * sc.dt, sc.dt, W, sc.sweeps)
    T, reps = _gpu_run(mach, T0, 3, precision)
    assert all(r["status"] == 0 for r in reps)
    rel = np.linalg.norm(T - X) / np.linalg.norm(X)
    rise = np.linalg.norm(T - X) / np.linalg.norm(X - T0)
    if precision == "fp64":
        assert rel <= 1e-10 and rise <= 1e-8, (rel, rise)
    else:
        assert rel <= 1e-6 and rise <= 1e-6, (rel, rise)


def _stand_error(T, ref, T0, nf):
    return np.linalg.norm(T[:nf] - ref[:nf]) / np.linalg.norm(ref[:nf] - T0[:nf])


@pytest.fixture(scope="module")
def reference(torch):
    # the solution at T_END from a step many times smaller: (M, P) = (5, 8), 8 sweeps
    mach, T0 = _slab(5, 8, 8, T_END / 256)
    T, _ = _gpu_run(mach, T0, 256)
    return T, T0, mach.stand.mesh.n_nodes


# Errors below this are at the floor set by the reference and by the source
# crossing element edges (the overlap, hence f^E, is only piecewise smooth in t).
ERR_FLOOR = 1e-9


@pytest.mark.parametrize("M,P", [(5, 8), (5, 2)])
def test_measured_order_is_min_M_P_k_plus_1(torch, reference, M, P):
    ref, T0, nf = reference
    for k in range(5):
        steps = (4, 8, 16)
        errs = []
        for n in steps:
            mach, _ = _slab(M, P, k, T_END / n)
            T, _ = _gpu_run(mach, T0, n)
            errs.append(_stand_error(T, ref, T0, nf))
        # the order from the smallest pair of steps still above the floor
        pairs = [i for i in range(len(steps) - 1) if errs[i + 1] >= ERR_FLOOR]
        assert pairs, (M, P, k, errs)
        i = pairs[-1]
        order = np.log2(errs[i] / errs[i + 1])
        expected = _expected_orders()[(M, P, k)]
        assert order >= expected - 0.35, (M, P, k, errs, order)
        assert order <= expected + 1.0, (M, P, k, errs, order)


def test_residual_decays_like_dt_to_the_k(torch):
    # Residual of the first macro step after k sweeps, for dt = T_END/5, /10, /20. It
    # is measured in units of M T over all rows, so the source here holds 1e6 (not 1e12)
    # times the stand's heat capacity: its rounding then stays far below the residuals.
    res = {}
    for n in (5, 10, 20):
        mach, T0 = _slab(5, 8, 4, T_END / n, capacity_ratio=1e6)
        _, reps = _gpu_run(mach, T0, 1, residuals=True)
        res[n] = np.asarray(reps[0]["residual"])
    # above the floor that the source's rounding sets (about 1e-7 of the first residual)
    def resolved(n, k):
        return res[n][k] > 1e-6 * res[n][0]

    for n in res:
        for k in range(1, 5):
            if resolved(n, k):
                # each sweep divides the residual by a factor that shrinks with dt
                assert res[n][k] < 0.05 * res[n][k - 1], (n, k, res[n])
    for k in range(0, 5):
        # halving dt divides the k-th residual by at least 2^(k + 1) (measured: 2^(k + 2))
        for a, b in ((5, 10), (10, 20)):
            if resolved(b, k):
                assert res[b][k] <= res[a][k] / 2.0 ** (k + 1), (k, a, b, res[a][k], res[b][k])
    assert all(resolved(n, 2) for n in res)
