"""The coupled stand/stock problem of Sec. 2 as an oracle problem object (test infrastructure only).

Builds Eq. coupledFEM for two independently meshed bodies: block-diagonal
lumped mass M and K = -(A + B_env), constant g = b_env (the environment
temperature is static), and the explicit term f^E(T, t) of oracle.contact.
DOFs are numbered stand first, then stock.

    f^I(T) = -K T,   g(t) = b_env,   f^E(T, t) = contact flux at time t

Parity: inherits the pins of oracle.fem and oracle.contact; the assembled
coupled system is additionally pinned by tests/test_oracle_bruteforce.py.
fE_iface (f^E on the interface DOFs only, for the interface-only form of the
stepper) is pinned to fE by tests/test_oracle_reduced.py.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import contact as ct
from . import fem
from .linsolve import dense_solve, pcg


class MachineProblem:
    def __init__(self, machine, rtol=None, max_iter=None, solver="pcg", with_contact=True):
        st, sk = machine.stand, machine.stock
        Kf, mf, bf = fem.body_system(st.mesh.xyz, st.mesh.hex8, st.k, st.rho, st.c,
                                     st.robin_quads, st.h, st.T_env, st.k_per_hex,
                                     getattr(st, "robin_extra", ()))
        Km, mm, bm = fem.body_system(sk.mesh.xyz, sk.mesh.hex8, sk.k, sk.rho, sk.c,
                                     sk.robin_quads, sk.h, sk.T_env, sk.k_per_hex,
                                     getattr(sk, "robin_extra", ()))
        self.n_fix = st.mesh.n_nodes
        self.n = st.mesh.n_nodes + sk.mesh.n_nodes
        self.K = sp.block_diag([Kf, Km], format="csr")
        self.mass = np.concatenate([mf, mm])
        self.genv = np.concatenate([bf, bm])
        self.diagK = self.K.diagonal()
        self.rtol = machine.scheme.cg_rtol if rtol is None else rtol
        self.max_iter = machine.scheme.cg_max_iter if max_iter is None else max_iter
        self.solver = solver
        self.with_contact = with_contact
        self.h_c, self.q0 = machine.h_c, machine.q0
        self.motion = (machine.motion_dir, machine.z0, machine.amp, machine.period)
        self.fix_quads = np.asarray(machine.stand_contact, dtype=np.int64)
        self.mov_quads = np.asarray(machine.stock_contact, dtype=np.int64) + self.n_fix
        self.fix_rect = ct.contact_rectangles(st.mesh.xyz, machine.stand_contact)
        self.mov_rect = ct.contact_rectangles(sk.mesh.xyz, machine.stock_contact)
        if self.fix_rect["normal"] != self.mov_rect["normal"]:
            raise ValueError("stand and stock contact faces lie in different planes")
        self.fe_calls = 0
        self.cg_total = 0
        # the interface: every DOF of a contact face, the only DOFs where f^E can be nonzero
        self.iface = np.unique(np.concatenate([self.fix_quads.ravel(), self.mov_quads.ravel()]))
        self._fix_local = np.searchsorted(self.iface, self.fix_quads)
        self._mov_local = np.searchsorted(self.iface, self.mov_quads)

    # ---- the stationary initial state of Sec. 5 ----
    def stationary_state(self):
        """T0 with 0 = f^I(T0) + g: the machine at rest, exchanging heat only with
        the environment and cooling equipment (the contact term is not part of the
        slow split), i.e. the sparse direct solve of K T0 = b_env."""
        return spla.spsolve(self.K.tocsc(), self.genv)

    # ---- the split of Eq. ivp ----
    def fI(self, T):
        return -(self.K @ T)

    def g(self, t):
        return self.genv

    def offset(self, t):
        d, z0, amp, per = self.motion
        return ct.stock_offset(t, d, z0, amp, per, self.fix_rect["u"], self.fix_rect["v"])

    def flux_q(self, t):
        return ct.friction_flux(t, self.q0, self.motion[3])

    def fE(self, T, t):
        self.fe_calls += 1
        if not self.with_contact:
            return np.zeros(self.n)
        du, dv = self.offset(t)
        return ct.contact_flux(T, self.fix_quads, self.mov_quads, self.fix_rect, self.mov_rect,
                               du, dv, self.h_c, self.flux_q(t), self.n)

    def fE_iface(self, Ti, t):
        """f^E on the interface DOFs (self.iface order) from the temperatures Ti there: the
        same contact integrals as fE with the faces' nodes numbered within the interface."""
        self.fe_calls += 1
        if not self.with_contact:
            return np.zeros(self.iface.size)
        du, dv = self.offset(t)
        return ct.contact_flux(Ti, self._fix_local, self._mov_local, self.fix_rect, self.mov_rect,
                               du, dv, self.h_c, self.flux_q(t), self.iface.size)

    def solve(self, dtau, rhs, x0):
        if dtau == 0.0:
            return rhs / self.mass, 0
        if self.solver == "dense":
            A = (sp.diags(self.mass) + dtau * self.K).toarray()
            return dense_solve(A, rhs), 0
        A = sp.diags(self.mass) + dtau * self.K
        dinv = 1.0 / (self.mass + dtau * self.diagK)
        x, it, ok = pcg(lambda v: A @ v, rhs, x0, dinv, self.rtol, self.max_iter)
        if not ok:
            raise RuntimeError("oracle PCG did not converge")
        self.cg_total += it
        return x, it

    # ---- diagnostics ----
    def heat(self, T):
        """Stored heat sum_i m_i T_i per body (J relative to 0 degC)."""
        q = self.mass * T
        return float(q[: self.n_fix].sum()), float(q[self.n_fix:].sum())

    def fI_matrix(self):
        """f^I(T) = L_I T with L_I = -K (sparse)."""
        return -self.K

    def contact_matrix(self, t):
        """Sparse E and e with f^E(T, t) = E T + e: f^E is affine in T and depends only on
        the temperatures of the contact nodes, so E is formed column by column from
        f^E of unit vectors on those nodes."""
        e = self.fE(np.zeros(self.n), t)
        nodes = np.unique(np.concatenate([self.fix_quads.ravel(), self.mov_quads.ravel()]))
        rows, cols, vals = [], [], []
        for j in nodes:
            unit = np.zeros(self.n)
            unit[j] = 1.0
            col = self.fE(unit, t) - e
            nz = np.nonzero(col)[0]
            rows.append(nz)
            cols.append(np.full(nz.size, j))
            vals.append(col[nz])
        E = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n, self.n))
        return E, e

    def coupling_operator(self, t):
        """Dense matrix E and vector e with f^E(T, t) = E T + e (small problems only)."""
        e = self.fE(np.zeros(self.n), t)
        E = np.empty((self.n, self.n))
        for j in range(self.n):
            unit = np.zeros(self.n)
            unit[j] = 1.0
            E[:, j] = self.fE(unit, t) - e
        return E, e
