"""Column forms of the stored matrix K (sdc_set_matrix_columns).

Every SpMV of the path (CG, f^I, bulk endpoints, refinement) reads K through the sliced
ELL. Its columns are stored as 16-bit offsets from each 32-row slice's smallest column
when every slice spans at most 65,535 columns, else as 32-bit columns; and the FP32 copy
of the mixed-precision solves has implied columns when the matrix allows them (each
slice's rows share one increasing table of relative columns, absent neighbours hold 0).
Every form sums the same products of a row in the same order, so:
  * the forms give bitwise equal steps, in both precisions, also on the 733,586-DOF machine
    whose FP32 CG runs three launches an iteration;
  * a node numbering whose slices span more columns (a random renumbering of the stand)
    takes 32-bit columns and no implied columns by itself, and gives the steps of the
    natural numbering, permuted, to rounding (the rows' entries are then summed in another
    order).
"""

from dataclasses import replace

import numpy as np
import pytest

from synth import machine_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _solver(mach, precision, bits):
    from paper_1707_03581_gb300 import Solver

    s = Solver(0)
    s.set_matrix_columns(bits)
    s.set_machine(mach, precision=precision)
    return s


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("idx", [0, 1])
def test_column_forms_are_bitwise_equal(torch, precision, idx):
    mach = machine_config(idx)
    a = _solver(mach, precision, 0)
    b = _solver(mach, precision, 16)
    c = _solver(mach, precision, 32)
    assert a.matrix_columns() == 16 and b.matrix_columns() == 16 and c.matrix_columns() == 32
    assert a.matrix_implied() and not b.matrix_implied() and not c.matrix_implied()
    for _ in range(3):
        ra = a.step(report=True)
        rb = b.step(report=True)
        rc = c.step(report=True)
    assert np.array_equal(a.temperature(), b.temperature())
    assert np.array_equal(a.temperature(), c.temperature())
    assert ra["cg_iters_total"] == rb["cg_iters_total"] == rc["cg_iters_total"]
    assert ra["refinements_total"] == rb["refinements_total"] == rc["refinements_total"]
    for s in (a, b, c):
        s.close()


def test_implied_columns_bitwise_on_the_large_grid_machine(torch):
    # the first machine of the 64-machine batch: 733,586 DOF, 2,866 blocks, so its FP32 CG
    # runs the three-launch form (k_mx_spmv, k_mx_dots, k_mx_update_red4)
    mach = machine_config(3)[0]
    a = _solver(mach, "mixed", 0)
    b = _solver(mach, "mixed", 16)
    assert a.n == 733586 and a.matrix_implied() and not b.matrix_implied()
    ra = a.step(report=True)
    rb = b.step(report=True)
    assert np.array_equal(a.temperature(), b.temperature())
    assert ra["cg_iters_total"] == rb["cg_iters_total"] and ra["refinements_total"] == rb["refinements_total"]
    a.close()
    b.close()


def _renumber_stand(mach, perm):
    """The same machine with stand node j the old node perm[j]."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    st = mach.stand
    mesh = replace(st.mesh, xyz=st.mesh.xyz[perm], hex8=inv[st.mesh.hex8])
    extra = tuple((inv[q], h, T) for q, h, T in st.robin_extra)
    stand = replace(st, mesh=mesh, robin_quads=inv[st.robin_quads], robin_extra=extra)
    return replace(mach, stand=stand, stand_contact=inv[mach.stand_contact])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_scrambled_numbering_takes_32_bit_columns(torch, precision):
    mach = machine_config(1)
    nf = mach.stand.mesh.n_nodes
    perm = np.random.default_rng(5).permutation(nf)
    scr = _renumber_stand(mach, perm)
    a = _solver(mach, precision, 0)
    b = _solver(scr, precision, 0)
    assert a.matrix_columns() == 16 and b.matrix_columns() == 32
    assert a.matrix_implied() and not b.matrix_implied()
    for _ in range(2):
        a.step(report=True)
        b.step(report=True)
    Ta, Tb = a.temperature(), b.temperature()
    Tb_nat = Tb.copy()
    Tb_nat[perm] = Tb[:nf]
    rise = np.linalg.norm(Ta - mach.T0)
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.linalg.norm(Tb_nat - Ta) <= tol * rise, np.linalg.norm(Tb_nat - Ta) / rise
    a.close()
    b.close()


def test_matrix_columns_argument_checks(torch):
    from paper_1707_03581_gb300 import SdcError, Solver

    s = Solver(0)
    with pytest.raises(SdcError):
        s.matrix_columns()  # before assembly
    with pytest.raises(SdcError):
        s.matrix_implied()
    for bad in (8, 24, -1):
        with pytest.raises(SdcError):
            s.set_matrix_columns(bad)
    for ok in (0, 16, 32):
        s.set_matrix_columns(ok)
    s.close()


@pytest.mark.parametrize("case", ["tiny", "slab"])
def test_implied_columns_bitwise_on_small_machines(torch, case):
    # machines of a few hundred DOF, where a larger share of the slices meet the ends of the
    # numbering and clamp their columns
    from paper_1707_03581_gb300 import Solver
    from synth import tiny_machine
    from synth.machines import slab_machine

    if case == "tiny":
        mach, T0 = tiny_machine(z0=0.37, amp=0.2, period=2.5), None
    else:
        mach, T0 = slab_machine()
    out = []
    for bits in (0, 16):
        s = Solver(0)
        s.set_matrix_columns(bits)
        s.set_machine(mach, precision="mixed", T0=T0)
        assert s.matrix_implied() == (bits == 0)
        reps = [s.step(report=True) for _ in range(3)]
        assert all(r["status"] == 0 for r in reps)
        out.append((s.temperature(), [r["cg_iters_total"] for r in reps]))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
