"""Pins for oracle.fem: trilinear mass, stiffness and Robin terms (Sec. 2).

Checked against: the unit-cube element matrix integrated exactly with sympy,
zero row sums of the Neumann stiffness, the linear patch test, total mass and
area, and h^2 convergence to the decaying cosine mode of the heat equation.
"""

import numpy as np
import pytest

from oracle import fem
from oracle.mrsdc import mrsdc_step
from oracle.weights import mrsdc_weights
from synth import box_mesh, machine_config


def _exact_unit_cube_stiffness():
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    corners = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    phis = []
    for cx, cy, cz in corners:
        fx = x if cx else 1 - x
        fy = y if cy else 1 - y
        fz = z if cz else 1 - z
        phis.append(fx * fy * fz)
    K = np.zeros((8, 8))
    Mass = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            ga = [sympy.diff(phis[a], v) for v in (x, y, z)]
            gb = [sympy.diff(phis[b], v) for v in (x, y, z)]
            integrand = sum(p * q for p, q in zip(ga, gb))
            K[a, b] = float(sympy.integrate(integrand, (x, 0, 1), (y, 0, 1), (z, 0, 1)))
            Mass[a, b] = float(sympy.integrate(phis[a] * phis[b], (x, 0, 1), (y, 0, 1), (z, 0, 1)))
    return K, Mass


def test_unit_cube_element_against_exact_integration():
    Kx, Mx = _exact_unit_cube_stiffness()
    X = np.array([[[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                   [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]]], dtype=float)
    Ke, me = fem.element_matrices(X, np.array([1.0]), 1.0)
    np.testing.assert_allclose(Ke[0], Kx, atol=1e-14)
    # lumped mass = row sums of the consistent mass (1/8 each on the unit cube)
    np.testing.assert_allclose(me[0], Mx.sum(axis=1), atol=1e-15)
    # textbook values: diagonal 1/3, face diagonal -1/12, edge neighbour 0
    assert abs(Kx[0, 0] - 1 / 3) < 1e-15 and abs(Kx[0, 2] + 1 / 12) < 1e-15 and abs(Kx[0, 1]) < 1e-15


def test_scaled_element_and_face():
    # a 2 x 3 x 5 box element with k = 7: K scales per direction, mass = rho c V / 8
    X = np.array([[[0, 0, 0], [2, 0, 0], [2, 3, 0], [0, 3, 0],
                   [0, 0, 5], [2, 0, 5], [2, 3, 5], [0, 3, 5]]], dtype=float)
    Ke, me = fem.element_matrices(X, np.array([7.0]), 11.0)
    np.testing.assert_allclose(me[0], np.full(8, 11.0 * 30 / 8))
    np.testing.assert_allclose(Ke[0].sum(axis=1), 0.0, atol=1e-13)
    # energy of the linear field u = x: k * V * |grad u|^2 = 7 * 30 * 1
    u = X[0, :, 0]
    assert abs(u @ Ke[0] @ u - 7.0 * 30.0) < 1e-11
    Fe, fe = fem.face_integrals(X[0], np.array([[0, 1, 2, 3]]))
    np.testing.assert_allclose(fe[0], np.full(4, 6.0 / 4))
    np.testing.assert_allclose(Fe[0].sum(), 6.0)
    # consistent face mass of a rectangle: area/9 * [4 2 1 2] pattern / 4
    np.testing.assert_allclose(Fe[0][0], 6.0 / 36 * np.array([4, 2, 1, 2]))


def test_row_sums_mass_area_and_patch():
    mach = machine_config(0)
    st = mach.stand
    K, m = fem.assemble_body(st.mesh.xyz, st.mesh.hex8, st.k, st.rho, st.c)
    np.testing.assert_allclose(K @ np.ones(K.shape[0]), 0.0, atol=1e-9)
    assert abs(m.sum() - st.rho * st.c * 0.4 * 0.4 * 1.0) < 1e-6 * m.sum()
    # patch test: interior rows of K annihilate linear fields
    xyz = st.mesh.xyz
    u = 1.0 + 2.0 * xyz[:, 0] - 3.0 * xyz[:, 1] + 0.5 * xyz[:, 2]
    r = K @ u
    interior = ((xyz[:, 0] > 1e-9) & (xyz[:, 0] < 0.4 - 1e-9) & (xyz[:, 1] > 1e-9)
                & (xyz[:, 1] < 0.4 - 1e-9) & (xyz[:, 2] > 1e-9) & (xyz[:, 2] < 1 - 1e-9))
    assert np.abs(r[interior]).max() < 1e-10
    # Robin: sum of entries = h * area, b_env = h * T_env * int phi
    B, b = fem.robin_terms(xyz, st.robin_quads, st.h, st.T_env)
    area = 2 * (0.4 * 1.0) * 2 + 2 * 0.4 * 0.4 - 0.2 * 1.0   # rail strip is not Robin
    assert abs(B.sum() - st.h * area) < 1e-10
    assert abs(b.sum() - st.h * st.T_env * area) < 1e-9
    np.testing.assert_allclose(B @ np.ones(B.shape[0]) * st.T_env, b, atol=1e-12)


def _cosine_mode_error(n, t_end=0.02, dt=0.005):
    mesh = box_mesh((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (n, n, n))
    K, m = fem.assemble_body(mesh.xyz, mesh.hex8, 1.0, 1.0, 1.0)
    x, y, z = mesh.xyz.T
    mode = np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
    Kd = K.toarray()

    class Heat:
        mass = m

        def fI(self, T):
            return -(K @ T)

        def g(self, t):
            return np.zeros_like(m)

        def fE(self, T, t):
            return np.zeros_like(m)

        def solve(self, dtau, rhs, x0):
            return np.linalg.solve(np.diag(m) + dtau * Kd, rhs), 0

    W = mrsdc_weights("radau_right", 3, 2)
    T = mode.copy()
    steps = int(round(t_end / dt))
    for i in range(steps):
        T, _ = mrsdc_step(Heat(), T, i * dt, dt, W, 4)
    exact = np.exp(-3 * np.pi ** 2 * t_end) * mode
    return np.sqrt(np.sum(m * (T - exact) ** 2))


def test_h2_convergence_cosine_mode():
    e4, e8 = _cosine_mode_error(4), _cosine_mode_error(8)
    rate = np.log2(e4 / e8)
    assert 1.8 < rate < 2.3, (e4, e8, rate)
