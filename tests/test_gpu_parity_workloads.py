"""GPU parity on the configurations the benchmark and the batch run, against the oracle.

* Per-hex conductivity, the defining input of the 5,751,586-DOF workload (one k per
  hexahedron, log-uniform in [40, 60] W/(m K), both bodies), with that workload's
  scheme (Radau IIA M = 4, 4 sweeps, P = 40) on smaller meshes that the oracle can step:
  the assembled K and lumped mass, then three macro steps in both precisions.
* One macro step of the first batch machine of every stand resolution r in
  {16, 24, 32, 48, 64} (12,902 to 733,586 DOF), in both precisions. The r = 64 machine
  runs the large-grid FP32 CG (more than 2048 SpMV blocks: last-block reduction in the
  SpMV) that the 5.75M-DOF workload also takes.

Tolerances as in test_gpu_parity.py: FP64 rel-L2 <= 1e-10 on T and <= 1e-8 on the rise
T - T0 per macro step; mixed precision <= 1e-6 on both (the stated bar).
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step
from oracle.weights import mrsdc_weights
from synth.machines import batch_resolutions, machine_config, per_hex_machine

pytestmark = pytest.mark.gpu

REL_T, REL_RISE = 1e-10, 1e-8
REL_MIXED = 1e-6


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _solver(mach, **kw):
    from paper_1707_03581_gb300 import Solver

    s = Solver(0)
    s.set_machine(mach, **kw)
    return s


def _rel(got, ref, T0):
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    rise = float(np.linalg.norm(got - ref) / np.linalg.norm(ref - T0))
    return rel, rise


def _oracle_steps(mach, n_steps):
    prob = MachineProblem(mach)
    sc = mach.scheme
    W = mrsdc_weights(sc.nodes, sc.M, sc.P, sc.window)
    T = np.full(prob.n, mach.T0)
    out = []
    for n in range(n_steps):
        T, _ = mrsdc_step(prob, T, mach.t0 + n * sc.dt, sc.dt, W, sc.sweeps)
        out.append(T.copy())
    return prob, out


@pytest.mark.parametrize("stand_n,stock_n", [((8, 8, 20), (4, 4, 6)), ((24, 24, 60), (12, 12, 18))])
def test_per_hex_conductivity_system_and_steps(torch, stand_n, stock_n):
    mach = per_hex_machine("per-hex", stand_n, stock_n, seed=3)
    assert mach.stand.k_per_hex.min() >= 40.0 and mach.stand.k_per_hex.max() <= 60.0
    prob, ref = _oracle_steps(mach, 3)
    for precision in ("fp64", "mixed"):
        s = _solver(mach, precision=precision)
        rp, col, val, mass, genv = s.system()
        K = sp.csr_matrix((val, col, rp), shape=(s.n, s.n))
        assert abs(K - prob.K).max() <= 1e-13 * abs(prob.K).max()
        np.testing.assert_allclose(mass, prob.mass, rtol=1e-14)
        np.testing.assert_allclose(genv, prob.genv, rtol=1e-13, atol=1e-13 * abs(prob.genv).max())
        tol_t, tol_r = (REL_T, REL_RISE) if precision == "fp64" else (REL_MIXED, REL_MIXED)
        for n in range(3):
            rep = s.step(report=True)
            assert rep["status"] == 0
            rel, rise = _rel(s.temperature(), ref[n], mach.T0)
            assert rel <= tol_t and rise <= tol_r, (precision, n, rel, rise)
        s.close()
    # the per-hex field is what was assembled: a uniform-k machine differs
    uni = MachineProblem(_uniform_twin(mach))
    assert abs(uni.K - prob.K).max() > 1e-3 * abs(prob.K).max()


def _uniform_twin(mach):
    import copy

    m = copy.deepcopy(mach)
    m.stand.k_per_hex = None
    m.stock.k_per_hex = None
    return m


BATCH_R = batch_resolutions()


@pytest.mark.parametrize("r", [16, 24, 32, 48, 64])
def test_batch_member_of_each_resolution_one_macro_step(torch, r):
    i = BATCH_R[r]
    (mach,) = machine_config(3, select={i})
    assert mach.name == f"c4-m{i}-r{r}"
    _, (ref,) = _oracle_steps(mach, 1)
    for precision, tol_t, tol_r in (("fp64", REL_T, REL_RISE), ("mixed", REL_MIXED, REL_MIXED)):
        s = _solver(mach, precision=precision)
        rep = s.step(report=True)
        assert rep["status"] == 0
        rel, rise = _rel(s.temperature(), ref, mach.T0)
        assert rel <= tol_t and rise <= tol_r, (r, precision, rel, rise)
        if precision == "mixed" and r == 64:
            # the large-grid FP32 CG: one block (k_mx_dots) takes the SpMV's dots
            s.set_execution(True)
            s.set_kernel_timing(True)
            s.step(report=True)
            kt = s.kernel_times()
            assert kt["k_mx_dots"][0] > 0 and kt["k_mx_update_red"][0] > 0 and "k_mx_update" not in kt
        s.close()
