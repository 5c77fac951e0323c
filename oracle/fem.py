"""Trilinear finite elements for the heat equation (oracle; test infrastructure only).

Follows Sec. 2 of the paper: the weak forms Eq. femContFix / femContMov and
the matrices defined after Eq. femDiscr:

* M_X = int rho c phi_i phi_j, replaced by its row-sum lumped diagonal
  m_i = int rho c phi_i (the lumping stated after Eq. coupledFEM). rho c is
  kept in M because it multiplies d_t T on the left of Eq. femContFix;
* A_X = -int k grad phi_i . grad phi_j;
* B_X,env = -int_{Gamma_env} h phi_i phi_j (consistent, not lumped);
* b_X,env = int_{Gamma_env} h T_env phi_i.

The oracle returns K = -(A + B_env), which is symmetric positive definite, so
that f^I(T) = -K T and g = b_env.

Element integrals use 2x2x2 Gauss points on the isoparametric trilinear hex
(2x2 on bilinear faces); on affine (box) elements these rules are exact.
Hexahedra list corners bottom face counter-clockwise, then the top face;
reference corner a has coordinates (+-1, +-1, +-1) in that order.

Parity: pinned by tests/test_oracle_fem.py (closed-form unit-cube element
matrix, zero row sums without Robin terms, linear patch test, total mass and
area, h^2 convergence to a decaying cosine mode).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

CORNERS = np.array(
    [[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
     [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)
QUAD_CORNERS = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], dtype=np.float64)
G = 1.0 / np.sqrt(3.0)


def hex_shape(xi):
    """Trilinear shape functions N[8] and reference gradients dN[8, 3] at xi."""
    s = 1.0 + CORNERS * xi[None, :]            # (8, 3) factors (1 + xi_a xi)
    N = 0.125 * s[:, 0] * s[:, 1] * s[:, 2]
    dN = np.empty((8, 3))
    dN[:, 0] = 0.125 * CORNERS[:, 0] * s[:, 1] * s[:, 2]
    dN[:, 1] = 0.125 * CORNERS[:, 1] * s[:, 0] * s[:, 2]
    dN[:, 2] = 0.125 * CORNERS[:, 2] * s[:, 0] * s[:, 1]
    return N, dN


def quad_shape(xi):
    """Bilinear shape functions N[4] and reference gradients dN[4, 2] at xi."""
    s = 1.0 + QUAD_CORNERS * xi[None, :]
    N = 0.25 * s[:, 0] * s[:, 1]
    dN = np.empty((4, 2))
    dN[:, 0] = 0.25 * QUAD_CORNERS[:, 0] * s[:, 1]
    dN[:, 1] = 0.25 * QUAD_CORNERS[:, 1] * s[:, 0]
    return N, dN


def element_matrices(X, k_hex, rho_c):
    """Stiffness k int grad phi_a . grad phi_b and lumped mass for a batch of hexes.

    X: (n, 8, 3) corner coordinates; k_hex: (n,) conductivities.
    Returns Ke (n, 8, 8) and me (n, 8).
    """
    n = X.shape[0]
    Ke = np.zeros((n, 8, 8))
    me = np.zeros((n, 8))
    for gx in (-G, G):
        for gy in (-G, G):
            for gz in (-G, G):
                N, dN = hex_shape(np.array([gx, gy, gz]))
                J = np.einsum("ad,nai->ndi", dN, X)            # J[n, d, i] = dx_i / dxi_d
                det = np.linalg.det(J)
                if np.any(det <= 0):
                    raise ValueError("inverted or degenerate hexahedron")
                Jinv = np.linalg.inv(J)                          # Jinv[n, i, d]
                grad = np.einsum("ad,nid->nai", dN, Jinv)        # physical gradients
                Ke += (k_hex * det)[:, None, None] * np.einsum("nai,nbi->nab", grad, grad)
                me += (rho_c * det)[:, None] * N[None, :]
    return Ke, me


def assemble_body(xyz, hex8, k, rho, c, k_per_hex=None, chunk=400_000):
    """Stiffness (CSR) and lumped mass of one body, without boundary terms."""
    n_nodes = xyz.shape[0]
    kh = np.full(hex8.shape[0], float(k)) if k_per_hex is None else np.asarray(k_per_hex, float)
    rows, cols, vals = [], [], []
    m = np.zeros(n_nodes)
    for s in range(0, hex8.shape[0], chunk):
        h = hex8[s:s + chunk]
        Ke, me = element_matrices(xyz[h], kh[s:s + chunk], rho * c)
        rows.append(np.repeat(h, 8, axis=1).ravel())
        cols.append(np.tile(h, (1, 8)).ravel())
        vals.append(Ke.ravel())
        np.add.at(m, h.ravel(), me.ravel())
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_nodes, n_nodes)).tocsr()
    K.sum_duplicates()
    return K, m


def face_integrals(xyz, quads):
    """For a batch of bilinear faces: Fe[n,4,4] = int phi_a phi_b dS, fe[n,4] = int phi_a dS."""
    X = xyz[quads]                                   # (n, 4, 3)
    Fe = np.zeros((quads.shape[0], 4, 4))
    fe = np.zeros((quads.shape[0], 4))
    for gx in (-G, G):
        for gy in (-G, G):
            N, dN = quad_shape(np.array([gx, gy]))
            t1 = np.einsum("a,nai->ni", dN[:, 0], X)
            t2 = np.einsum("a,nai->ni", dN[:, 1], X)
            dS = np.linalg.norm(np.cross(t1, t2), axis=1)
            Fe += dS[:, None, None] * np.outer(N, N)[None]
            fe += dS[:, None] * N[None, :]
    return Fe, fe


def robin_terms(xyz, quads, h, T_env):
    """-B_env = h int phi phi (CSR, SPD part of K) and b_env = h T_env int phi."""
    n_nodes = xyz.shape[0]
    if quads is None or len(quads) == 0 or h == 0.0:
        return sp.csr_matrix((n_nodes, n_nodes)), np.zeros(n_nodes)
    Fe, fe = face_integrals(xyz, quads)
    rows = np.repeat(quads, 4, axis=1).ravel()
    cols = np.tile(quads, (1, 4)).ravel()
    B = sp.coo_matrix((h * Fe.ravel(), (rows, cols)), shape=(n_nodes, n_nodes)).tocsr()
    b = np.zeros(n_nodes)
    np.add.at(b, quads.ravel(), (h * T_env * fe).ravel())
    return B, b


def body_system(xyz, hex8, k, rho, c, robin_quads, h, T_env, k_per_hex=None, robin_extra=()):
    """K = -(A + B_env), lumped mass m and g = b_env of one body. B_env and b_env
    sum over the Robin groups: (robin_quads, h, T_env) and each (quads, h, T_env)
    of robin_extra."""
    A_neg, m = assemble_body(xyz, hex8, k, rho, c, k_per_hex)
    B_neg, b = robin_terms(xyz, robin_quads, h, T_env)
    for quads, hg, Tg in robin_extra:
        Bg, bg = robin_terms(xyz, quads, hg, Tg)
        B_neg = B_neg + Bg
        b = b + bg
    return (A_neg + B_neg).tocsr(), m, b
