"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 path rel-L2 <= 1e-10 per macro step on the temperature
(the stated bar), plus the stricter rel-L2 of the rise T - T0 <= 1e-8, since
the 20 degC offset makes the first metric lenient. Component checks use
1e-12..1e-13 (rounding-order differences of FP64 sums only).
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import contact as ct
from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step
from oracle.weights import mrsdc_weights
from synth import machine_config, tiny_machine
from synth.machines import with_scheme

pytestmark = pytest.mark.gpu

REL_T = 1e-10
REL_RISE = 1e-8


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


def _compare(got, ref, T0, tag, rel_t=REL_T, rel_rise=REL_RISE):
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    d = np.linalg.norm(ref - T0)
    rise = np.linalg.norm(got - ref) / d if d > 0 else np.linalg.norm(got - ref)
    assert rel <= rel_t, (tag, rel)
    assert rise <= rel_rise, (tag, rise)
    return rel, rise


def test_assembled_system_matches_oracle(torch):
    mach = machine_config(0)
    s = _solver(mach)
    prob = MachineProblem(mach)
    rp, col, val, mass, genv = s.system()
    K = sp.csr_matrix((val, col, rp), shape=(s.n, s.n))
    diff = abs(K - prob.K)
    assert diff.max() <= 1e-13 * abs(prob.K).max()
    np.testing.assert_allclose(mass, prob.mass, rtol=1e-14)
    np.testing.assert_allclose(genv, prob.genv, rtol=1e-13, atol=1e-13 * abs(prob.genv).max())
    # the library keeps structurally present entries that sum to exactly zero
    # (edge neighbours on cube cells); scipy drops them from the oracle's pattern
    assert s.n_stand == mach.stand.mesh.n_nodes and s.nnz >= prob.K.nnz


def test_operator_solve_and_contact_components(torch):
    mach = machine_config(0)
    s = _solver(mach)
    prob = MachineProblem(mach)
    rng = np.random.default_rng(11)
    x = 20.0 + rng.standard_normal(s.n)
    for dtau in (0.0, 0.5, 0.123):
        y = s.apply_operator(dtau, x).cpu().numpy()
        ref = prob.mass * x + dtau * (prob.K @ x)
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    b = prob.mass * (20.0 + rng.standard_normal(s.n))
    xs, it = s.solve(0.5, b, np.full(s.n, 20.0))
    A = (sp.diags(prob.mass) + 0.5 * prob.K).toarray()
    xd = np.linalg.solve(A, b)
    assert it > 0
    assert np.abs(xs.cpu().numpy() - xd).max() <= 1e-10 * np.abs(xd).max()
    T = 20.0 + rng.standard_normal(s.n)
    for t in (0.0, 0.37, 1.0, 1.5, 7.31):
        fe = s.contact_flux(T, t).cpu().numpy()
        ref = prob.fE(T, t)
        assert np.abs(fe - ref).max() <= 1e-12 * np.abs(ref).max(), t


def _run_parity(mach, n_steps, residuals=False, T0=None, precision="fp64", rel_t=REL_T, rel_rise=REL_RISE):
    s = _solver(mach, residuals=residuals, T0=T0, precision=precision)
    prob = MachineProblem(mach)
    sc = mach.scheme
    W = mrsdc_weights(sc.nodes, sc.M, sc.P, sc.window)
    T = np.full(prob.n, mach.T0) if T0 is None else np.array(T0, dtype=np.float64)
    start = T.copy()
    worst = (0.0, 0.0)
    for n in range(n_steps):
        rep = s.step(report=True)
        T, r = mrsdc_step(prob, T, mach.t0 + n * sc.dt, sc.dt, W, sc.sweeps, want_residuals=residuals)
        got = s.temperature()
        rel, rise = _compare(got, T, start, f"step {n}", rel_t, rel_rise)
        worst = (max(worst[0], rel), max(worst[1], rise))
        assert rep["status"] == 0
        if residuals:
            scale = max(r.residuals[0], 1e-300)
            np.testing.assert_allclose(rep["residual"], r.residuals, rtol=1e-6, atol=1e-9 * scale)
        h = s.heat_totals()
        hs, hk = prob.heat(got)
        assert abs(h["stored_stand"] - hs) <= 1e-12 * abs(hs)
        assert abs(h["stored_stock"] - hk) <= 1e-12 * abs(hk)
    s.close()
    return worst


def test_config0_full_horizon_lobatto(torch):
    # 8x8x20 + 4x4x6, Lobatto M=3, 3 sweeps, P=20, dt = 1 s, 60 macro steps
    mach = machine_config(0)
    _run_parity(mach, 60)


@pytest.mark.parametrize("nodes,M,P,K,window", [("radau_right", 4, 8, 4, 0), ("equi_noleft", 3, 2, 2, 2),
                                                 ("equi_noleft", 5, 8, 3, 8), ("lobatto", 2, 1, 1, 0),
                                                 ("radau_right", 1, 5, 0, 0), ("lobatto", 4, 40, 2, 0)])
def test_schemes_on_tiny_machine_with_residuals(torch, nodes, M, P, K, window):
    mach = with_scheme(tiny_machine(z0=0.37, amp=0.21, period=1.7), nodes=nodes, M=M, P=P, sweeps=K,
                       window=window, dt=0.8)
    rng = np.random.default_rng(5)
    T0 = 20.0 + rng.standard_normal(mach.n_dof)
    _run_parity(mach, 4, residuals=True, T0=T0)


def test_resting_stock_and_insulated_conservation(torch):
    mach = tiny_machine(z0=0.37, amp=0.25, period=np.inf, q0=0.0)
    mach.stand.h = 0.0
    mach.stock.h = 0.0
    rng = np.random.default_rng(9)
    T0 = 20.0 + 3.0 * rng.standard_normal(mach.n_dof)
    s = _solver(mach, T0=T0)
    h0 = s.heat_totals()
    Q0 = h0["stored_stand"] + h0["stored_stock"]
    for _ in range(5):
        s.step(report=True)
    h1 = s.heat_totals()
    Q1 = h1["stored_stand"] + h1["stored_stock"]
    assert abs(Q1 - Q0) <= 1e-12 * abs(Q0)
    # no friction: the ledger only sees the rounding of exchange terms that cancel
    assert abs(h1["friction_in"]) <= 1e-8


def test_friction_energy_ledger(torch):
    # resting stock, constant flux: friction energy per step = q0 * area * dt
    mach = tiny_machine(z0=0.37, amp=0.25, period=np.inf, q0=2.0e4)
    s = _solver(mach)
    for _ in range(3):
        s.step(report=True)
    h = s.heat_totals()
    assert abs(h["friction_in"] - 3 * 2.0e4 * 0.06 * 1.0) <= 1e-9 * 3 * 2.0e4 * 0.06


def test_deterministic_and_horizon_equals_steps(torch):
    mach = machine_config(0)
    a = _solver(mach)
    for _ in range(4):
        a.step(report=False)
    a.synchronize()
    Ta = a.temperature()
    b = _solver(mach)
    rep = b.run_horizon(4)
    Tb = b.temperature()
    assert np.array_equal(Ta, Tb)
    assert abs(rep["t"] - 4.0) < 1e-12


def test_config1_two_macro_steps(torch):
    # 48x48x120 + 24x24x36 (313,646 DOF), seeded stroke: the benchmark workload
    mach = machine_config(1)
    _run_parity(mach, 2)


def test_errors_are_reported_not_fatal(torch):
    from paper_1707_03581_gb300 import Solver
    from paper_1707_03581_gb300.binding import SdcError

    s = Solver(0)
    with pytest.raises(SdcError) as e:
        s.step()
    assert "SDC_ERR_STATE" in str(e.value)
    mach = machine_config(0)
    bad = mach.stand.mesh.hex8.copy()
    bad[0, 0] = 10 ** 9
    s.set_body(0, mach.stand.mesh.xyz, bad, 50.0, 7850.0, 460.0)
    s.set_body(1, mach.stock.mesh.xyz, mach.stock.mesh.hex8, 50.0, 7850.0, 460.0)
    s.set_contact(mach.stand_contact, mach.stock_contact, 2000.0, 5e4)
    s.set_motion((0, 0, 1), 0.35, 0.25, 2.0)
    with pytest.raises(SdcError) as e:
        s.assemble()
    assert "SDC_ERR_ARG" in str(e.value)
    # a cap of one CG iteration cannot reach 1e-12: the step reports it
    s2 = _solver(with_scheme(machine_config(0), cg_max_iter=1))
    rng = np.random.default_rng(0)
    s2.set_temperature(20.0 + rng.standard_normal(s2.n))
    with pytest.raises(SdcError) as e:
        s2.step(report=True)
    assert "NOT_CONVERGED" in str(e.value)
    # the context stays usable
    s2.set_scheme("lobatto", 3, 20, 3, 0, 1.0, 1e-12, 2000)
    s2.set_temperature(None, 20.0, 0.0)
    s2.step(report=True)


def test_eager_execution_matches_graph(torch):
    mach = machine_config(0)
    a = _solver(mach)
    b = _solver(mach)
    b.set_execution(True)
    for _ in range(3):
        ra = a.step(report=True)
        rb = b.step(report=True)
    assert np.array_equal(a.temperature(), b.temperature())
    assert ra["cg_iters_total"] == rb["cg_iters_total"]
    assert ra["kernel_launches"] == rb["kernel_launches"]


def test_eager_kernel_timing_counts_every_launch(torch):
    mach = machine_config(0)
    s = _solver(mach)
    s.set_execution(True)
    s.set_kernel_timing(True)
    rep = s.step(report=True)
    kt = s.kernel_times()
    assert sum(n for n, _ in kt.values()) == rep["kernel_launches"]
    # one SpMV per update plus the one whose residual test stops each solve; loop
    # bodies of small grids hold three (SpMV, update) pairs, whose pairs after the
    # stop return at once
    assert kt["k_cg_spmv"][0] == kt["k_cg_update"][0]
    assert kt["k_cg_spmv"][0] % 3 == 0
    assert rep["cg_iters_total"] + rep["n_solves"] <= kt["k_cg_spmv"][0] <= rep["cg_iters_total"] + 3 * rep["n_solves"]
    loops = sum(n for name, (n, _) in kt.items() if name.startswith("k_iface_loop"))
    assert loops == rep["n_solves"]
    assert all(ms > 0 for _, ms in kt.values())
    assert rep["contact_cluster"] >= 1
    s.close()


# Mixed precision (FP32 inner CG inside FP64 iterative refinement). The stated
# bar is rel-L2 <= 1e-6 against the FP64 oracle per macro step; the FP64 outer
# residual to cg_rtol keeps the result far inside it, so the rise metric is
# checked at 1e-6 as well.
REL_MIXED = 1e-6


def test_mixed_config0_full_horizon(torch):
    mach = machine_config(0)
    worst = _run_parity(mach, 60, precision="mixed", rel_t=REL_MIXED, rel_rise=REL_MIXED)
    assert worst[0] <= REL_MIXED


@pytest.mark.parametrize("nodes,M,P,K,window", [("radau_right", 4, 8, 4, 0), ("lobatto", 3, 20, 3, 0),
                                                 ("equi_noleft", 3, 2, 2, 2)])
def test_mixed_schemes_on_tiny_machine(torch, nodes, M, P, K, window):
    mach = with_scheme(tiny_machine(z0=0.37, amp=0.21, period=1.7), nodes=nodes, M=M, P=P, sweeps=K,
                       window=window, dt=0.8)
    rng = np.random.default_rng(6)
    T0 = 20.0 + rng.standard_normal(mach.n_dof)
    _run_parity(mach, 4, residuals=True, T0=T0, precision="mixed", rel_t=REL_MIXED, rel_rise=REL_MIXED)


def test_mixed_solve_component_and_refinement(torch):
    mach = machine_config(0)
    s = _solver(mach, precision="mixed")
    prob = MachineProblem(mach)
    rng = np.random.default_rng(12)
    b = prob.mass * (20.0 + rng.standard_normal(s.n))
    xs, it = s.solve(0.5, b, np.full(s.n, 20.0))
    A = (sp.diags(prob.mass) + 0.5 * prob.K).toarray()
    xd = np.linalg.solve(A, b)
    assert it > 0
    # The refinement carries r = b - A x0 - A (x - x0): b - A x0 exactly in FP64, the
    # correction term with the FP32 operator. The solution is therefore exact to FP32
    # rounding of the correction (here O(1 K) on a 20 degC field), not of the field.
    x0 = np.full(s.n, 20.0)
    err = np.abs(xs.cpu().numpy() - xd).max()
    assert err <= 1e-6 * np.abs(xd - x0).max(), err
    assert err <= 1e-7 * np.abs(xd).max(), err
    rep = s.step(report=True)
    assert rep["refinements_total"] >= rep["n_solves"] - 1
    s.close()


def test_mixed_config1_two_macro_steps(torch):
    mach = machine_config(1)
    _run_parity(mach, 2, precision="mixed", rel_t=REL_MIXED, rel_rise=REL_MIXED)


def test_mixed_eager_matches_graph(torch):
    mach = machine_config(0)
    a = _solver(mach, precision="mixed")
    b = _solver(mach, precision="mixed")
    b.set_execution(True)
    b.set_kernel_timing(True)
    for _ in range(3):
        ra = a.step(report=True)
        rb = b.step(report=True)
    assert np.array_equal(a.temperature(), b.temperature())
    assert ra["cg_iters_total"] == rb["cg_iters_total"]
    assert ra["refinements_total"] == rb["refinements_total"]
    assert ra["kernel_launches"] == rb["kernel_launches"]
    kt = b.kernel_times()
    assert kt["k_mx_spmv"][0] == kt["k_mx_update"][0] > 0 and "k_cg_spmv" not in kt


def test_mixed_large_grid_matches_fp64(torch):
    # 733,586 DOFs: grids above the deferred-dot limit, where one block (k_mx_dots) sums the
    # SpMV's partials; the FP64 path is the oracle-pinned one
    mach = machine_config(3, truncate=1)[0]
    a = _solver(mach, precision="mixed")
    b = _solver(mach, precision="fp64")
    c = _solver(mach, precision="mixed")
    c.set_execution(True)
    for _ in range(2):
        a.step(report=True)
        b.step(report=True)
        c.step(report=True)
    Ta, Tb = a.temperature(), b.temperature()
    assert np.linalg.norm(Ta - Tb) / np.linalg.norm(Tb) <= 1e-9
    assert np.linalg.norm(Ta - Tb) / np.linalg.norm(Tb - mach.T0) <= REL_MIXED
    # eager execution: the same results as the graph, and the same launches (one timed step)
    assert np.array_equal(Ta, c.temperature())
    c.set_kernel_timing(True)
    ra = a.step(report=True)
    rc = c.step(report=True)
    assert np.array_equal(a.temperature(), c.temperature())
    assert ra["kernel_launches"] == rc["kernel_launches"]
    kt = c.kernel_times()
    assert sum(n for n, _ in kt.values()) == rc["kernel_launches"]
    # the large-grid FP32 CG: SpMV, one block for its dots, update of four rows a thread
    assert kt["k_mx_spmv"][0] == kt["k_mx_dots"][0] == kt["k_mx_update_red"][0] > 0 and "k_mx_update" not in kt
    assert kt["k_mx_refine"][0] == rc["refinements_total"]
    a.close()
    b.close()
    c.close()


def test_config2_full_size_mixed_matches_fp64(torch):
    # The 5,751,586-DOF machine (128x128x320 + 64x64x96, per-hex conductivity, Radau M=4,
    # 4 sweeps, P=40), in the launch configuration bench.py times. The oracle cannot take
    # a step of it; the FP64 path is the oracle-pinned one (smaller machines above), and
    # the mixed path must stay within the 1e-6 bar of it on the full size, with the large-grid
    # FP32 CG and the global-replica contact loop that only this size uses.
    mach = machine_config(2)
    a = _solver(mach, precision="mixed")
    b = _solver(mach, precision="fp64")
    ra = a.step(report=True)
    rb = b.step(report=True)
    assert ra["status"] == 0 and rb["status"] == 0
    Ta, Tb = a.temperature(), b.temperature()
    assert np.all(np.isfinite(Ta))
    assert np.linalg.norm(Ta - Tb) / np.linalg.norm(Tb) <= 1e-9
    assert np.linalg.norm(Ta - Tb) / np.linalg.norm(Tb - mach.T0) <= REL_MIXED
    # the contact heats the bodies: the step is not trivial
    assert np.linalg.norm(Tb - mach.T0) > 0.0
    a.close()
    b.close()


def test_mixed_eager_kernel_timing_counts_every_launch(torch):
    mach = machine_config(0)
    s = _solver(mach, precision="mixed")
    s.set_execution(True)
    s.step(report=True)
    s.set_kernel_timing(True)
    rep = s.step(report=True)
    kt = s.kernel_times()
    assert sum(n for n, _ in kt.values()) == rep["kernel_launches"]
    # one SpMV per update, and one whose dots stop each inner solve; loop bodies of
    # small grids hold three (SpMV, update) pairs, whose pairs after the stop return
    # at once
    n_pass = rep["refinements_total"]
    assert kt["k_mx_spmv"][0] == kt["k_mx_update"][0]
    assert kt["k_mx_spmv"][0] % 3 == 0
    assert rep["cg_iters_total"] + n_pass <= kt["k_mx_spmv"][0] <= rep["cg_iters_total"] + 3 * n_pass
    assert kt["k_mx_refine"][0] == n_pass and "k_mx_inner_init" not in kt
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_side_branches_equal_one_chain(torch, precision):
    # geometry and k_iface_prep beside the implicit solves, or all in one chain
    mach = machine_config(0)
    a = _solver(mach, precision=precision)
    b = _solver(mach, precision=precision)
    b.set_graph_branches(False)
    for _ in range(3):
        ra = a.step(report=True)
        rb = b.step(report=True)
    assert np.array_equal(a.temperature(), b.temperature())
    assert ra["kernel_launches"] == rb["kernel_launches"]
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cg_loop_pairs_are_bitwise_equal(torch, precision):
    # 1, 2, 5 and the default 3 (SpMV, update) pairs per CG loop body, graph and eager
    mach = machine_config(0)
    ref = None
    for pairs, eager in ((0, False), (1, False), (2, True), (5, False), (5, True)):
        s = _solver(mach, precision=precision)
        s.set_cg_unroll(pairs)
        s.set_execution(eager)
        for _ in range(3):
            rep = s.step(report=True)
        T = s.temperature()
        if ref is None:
            ref, iters = T, rep["cg_iters_total"]
        assert np.array_equal(T, ref), (pairs, eager)
        assert rep["cg_iters_total"] == iters
        s.close()
    from paper_1707_03581_gb300 import SdcError

    s = _solver(mach, precision=precision)
    with pytest.raises(SdcError):
        s.set_cg_unroll(9)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_contact_cluster_sizes_are_bitwise_equal(torch, precision):
    # the automatic size and forced 16-, 2- and 1-CTA clusters of the substep loop
    mach = machine_config(0)
    ref = None
    for cs in (0, 16, 2, 1):
        s = _solver(mach, precision=precision)
        s.set_contact_cluster(cs)
        for _ in range(3):
            rep = s.step(report=True)
        if cs:
            assert 1 <= rep["contact_cluster"] <= cs
        T = s.temperature()
        if ref is None:
            ref = T
        else:
            assert np.array_equal(T, ref), cs
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("placement", [1, 2, 3])
def test_global_replica_loop_equals_shared_memory_loop(torch, precision, placement):
    # the loop forms for interfaces too large for shared memory, forced on a small machine:
    # staged into shared memory after every substep (1), gathered from global memory (2), or
    # the grid-wide loop with one contact DOF a thread (3)
    mach = machine_config(0)
    a = _solver(mach, precision=precision)
    b = _solver(mach, precision=precision)
    b.set_contact_replicas(placement)
    for _ in range(3):
        a.step(report=True)
        b.step(report=True)
    assert np.array_equal(a.temperature(), b.temperature())
    b.set_execution(True)
    b.set_kernel_timing(True)
    b.step(report=True)
    suffix = {1: "_gls", 2: "_gl", 3: "_grid"}[placement]
    assert any(k.endswith(suffix) for k in b.kernel_times())


def test_mixed_loop_forms_are_bitwise_equal_on_a_large_interface(torch):
    # 3,950 contact DOFs: 16 CTAs give one DOF a thread (k_iface_loop_mx1), 4 CTAs two
    # (k_iface_loop_mx), 2 CTAs too many for shared memory forms (global replicas staged in
    # shared memory after every substep: k_iface_loop_mx_gls; a cluster cap keeps the loop off
    # the grid-wide form that an uncapped interface this large for shared memory takes)
    mach = machine_config(1)
    ref = None
    for cap, form in ((0, "k_iface_loop_mx1"), (4, "k_iface_loop_mx"), (2, "k_iface_loop_mx_gls")):
        s = _solver(mach, precision="mixed")
        s.set_contact_cluster(cap)
        for _ in range(2):
            s.step(report=True)
        s.set_execution(True)
        s.set_kernel_timing(True)
        s.step(report=True)
        loops = [k for k in s.kernel_times() if k.startswith("k_iface_loop")]
        assert loops == [form], (cap, loops)
        T = s.temperature()
        if ref is None:
            ref = T
        assert np.array_equal(T, ref), cap
        s.close()
