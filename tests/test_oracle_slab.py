"""The reduced problem of Sec. 4 as a one-hexahedron-thick slab with a
constant-temperature source (synth.slab_machine), checked on the oracle.

- 2D reduction: with both x faces insulated, the nodal temperatures on the two
  faces stay equal (the trilinear model is the bilinear one extruded).
- Constant source: the source's heat capacity is 1e12 times the stand's, so
  its temperature stays at T_source.
- Heat balance: with no environment and no friction, the heat the stand gains
  is the heat the source loses (to the solves' tolerance).
"""

import numpy as np

from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step
from oracle.weights import mrsdc_weights
from synth.machines import Scheme, slab_machine


def _run(mach, T0, n_steps):
    prob = MachineProblem(mach)
    sc = mach.scheme
    W = mrsdc_weights(sc.nodes, sc.M, sc.P, sc.window)
    T = T0.copy()
    for n in range(n_steps):
        T, _ = mrsdc_step(prob, T, mach.t0 + n * sc.dt, sc.dt, W, sc.sweeps)
    return prob, T


def test_slab_reduces_to_2d_with_a_constant_source():
    mach, T0 = slab_machine(4, 16, scheme=Scheme("equi_noleft", 5, 8, 2, 8, 0.5, 1e-14, 4000),
                            rho=10.0, c=1000.0)
    prob, T = _run(mach, T0, 3)
    nf = prob.n_fix
    xyz = mach.stand.mesh.xyz
    front = np.where(np.isclose(xyz[:, 0], 0.0))[0]
    back = np.where(~np.isclose(xyz[:, 0], 0.0))[0]
    # match nodes of the two faces by their (y, z)
    order_f = np.lexsort((xyz[front, 2], xyz[front, 1]))
    order_b = np.lexsort((xyz[back, 2], xyz[back, 1]))
    Ts = T[:nf]
    np.testing.assert_allclose(Ts[front[order_f]], Ts[back[order_b]], rtol=0, atol=1e-11)
    # the stand has warmed under the source, and nowhere below its start
    assert Ts.max() > 50.0 and Ts.min() >= 20.0 - 1e-9
    np.testing.assert_allclose(T[nf:], 100.0, rtol=1e-10)


def test_slab_heat_balance():
    # with a source of 1e6 times the stand's capacity its temperature change is
    # resolvable in FP64 (at 1e12 it is ~1e-10 K, below the resolution of 100 degC)
    mach, T0 = slab_machine(4, 16, scheme=Scheme("equi_noleft", 5, 8, 2, 8, 0.5, 1e-14, 4000),
                            rho=10.0, c=1000.0, capacity_ratio=1e6)
    prob, T = _run(mach, T0, 3)
    nf = prob.n_fix
    m = prob.mass
    gain = m[:nf] @ (T[:nf] - T0[:nf])
    loss = m[nf:] @ (T0[nf:] - T[nf:])
    assert gain > 100.0
    assert abs(gain - loss) <= 1e-8 * gain
