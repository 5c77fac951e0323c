"""Pins of the oracle's stationary initial state (Sec. 5: 0 = f^I(T0) + g, i.e.
K T0 = b_env for the machine at rest), against closed forms.

- One environment temperature per body: K 1 = B_env 1 (the stiffness of a
  constant vanishes) and b_env = T_env B_env 1, so T0 = T_env on every node.
- A body whose only Robin faces are its two y faces, with different h and
  T_env, is a 1D conduction problem: T(y) = A + B y with the flux k B equal on
  both faces. Trilinear hexahedra reproduce a field linear in y exactly, and
  T is constant on each Robin face, so the FEM nodal values are the exact ones.
  A wrong coefficient, sign or temperature of either Robin group breaks it.
"""

import dataclasses

import numpy as np

from oracle.machine import MachineProblem
from synth import machine_config, tiny_machine


def test_one_environment_temperature_per_body_gives_uniform_state():
    mach = machine_config(0)
    mach = dataclasses.replace(mach, stock=dataclasses.replace(mach.stock, T_env=35.0))
    prob = MachineProblem(mach)
    T0 = prob.stationary_state()
    nf = prob.n_fix
    np.testing.assert_allclose(T0[:nf], 20.0, rtol=1e-12)
    np.testing.assert_allclose(T0[nf:], 35.0, rtol=1e-12)


def _two_face_machine(h0=50.0, T0=10.0, h1=200.0, T1=90.0):
    """tiny_machine whose stand exchanges heat only through its y = ymin face
    (h0, T0) and its whole y = ymax face (h1, T1, rail included)."""
    mach = tiny_machine()
    st = mach.stand
    ymin, _, _ = st.mesh.side_quads("ymin")
    ymax, _, _ = st.mesh.side_quads("ymax")
    stand = dataclasses.replace(st, robin_quads=ymin, h=h0, T_env=T0, robin_extra=((ymax, h1, T1),))
    return dataclasses.replace(mach, stand=stand)


def linear_profile(mach, h0=50.0, T0=10.0, h1=200.0, T1=90.0):
    """Exact stationary temperature of the stand nodes of _two_face_machine:
    k T'(y0) = h0 (T(y0) - T0) and -k T'(y1) = h1 (T(y1) - T1), T'' = 0."""
    st = mach.stand
    y = st.mesh.xyz[:, 1]
    y0, y1 = y.min(), y.max()
    k = st.k
    B = (T1 - T0) / (k / h0 + k / h1 + (y1 - y0))
    A = T0 + k * B / h0
    return A + B * (y - y0)


def test_two_robin_faces_give_the_exact_linear_profile():
    mach = _two_face_machine()
    prob = MachineProblem(mach)
    T0 = prob.stationary_state()
    nf = prob.n_fix
    exact = linear_profile(mach)
    np.testing.assert_allclose(T0[:nf], exact, rtol=1e-11)
    np.testing.assert_allclose(T0[nf:], mach.stock.T_env, rtol=1e-12)
    # the profile is not trivial: it spans tens of kelvin
    assert exact.max() - exact.min() > 1.0


def test_floor_group_splits_the_stand_face():
    # build_machine(floor=...) takes the stand's y = ymin face out of the main group
    m = machine_config(0)
    from synth.machines import build_machine

    f = build_machine("floor", (8, 8, 20), (4, 4, 6), floor=(500.0, 40.0))
    n_main = len(m.stand.robin_quads)
    quads, h, T = f.stand.robin_extra[0]
    assert (h, T) == (500.0, 40.0)
    assert len(f.stand.robin_quads) + len(quads) == n_main
    prob = MachineProblem(f)
    T0 = prob.stationary_state()
    nf = prob.n_fix
    # the stand sits between 20 degC air and the 40 degC floor; the stock is at 20 degC
    assert 20.0 < T0[:nf].min() and T0[:nf].max() < 40.0
    np.testing.assert_allclose(T0[nf:], 20.0, rtol=1e-12)
