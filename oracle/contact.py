"""Explicit contact term f^E(T, t) on the moving interface (oracle; test infrastructure only).

Follows Sec. 2: with Gamma_R(t) the part of the stand's rail covered by the
stock at time t, the coupling and friction terms of Eq. femContFix /
femContMov give, for a stand test function phi_fix,

    f^E_fix,i = int_{Gamma_R(t)} ( alpha (T_mov - T_fix) + q(t)/2 ) phi_fix,i dS

and the same with fix <-> mov for stock test functions. This equals
M_B T + C_B T + b(t) in the paper's matrix notation (the definitions of
b_X(t), M_B and C_B), evaluated matrix-free.

The integral over Gamma_R(t) is split over every pair (stand face, stock face)
whose rectangles overlap at the current stock displacement. Each overlap is an
axis-aligned rectangle on which both integrands are products of bilinear
functions, so 2x2 Gauss points integrate them exactly. Pairs are found by
brute force over all stand x stock face pairs (the intersection step that the
paper delegates to a grid-glue library).

Readings: faces are planar axis-aligned rectangles in one common contact
plane; the stock moves rigidly by d(t) = dir * (z0 + A sin(2 pi t / Per)),
with dir in the plane; the friction flux q(t) = q0 |cos(2 pi t / Per)| is the
total generated flux, of which each body receives q/2 (the "eta(t)/2" of
Sec. 2). Per = inf gives a resting stock with constant flux q0.

Parity: pinned by tests/test_oracle_contact.py (uniform field gives zero
coupling, total flux equals q times the covered area, closed-form exchange
for linear fields, fine Riemann sums of the overlap integrals).
"""

from __future__ import annotations

import numpy as np

GP = 1.0 / np.sqrt(3.0)


def contact_rectangles(xyz, quads):
    """Describe planar axis-aligned quads as rectangles in their plane.

    Returns dict with normal axis, in-plane axes (u, v), lo/hi extents (n, 2)
    and corner_code (n, 4): for each listed node, bit 0 = at high u,
    bit 1 = at high v.
    """
    X = xyz[quads]                                  # (n, 4, 3)
    spread = X.max(axis=(0, 1)) - X.min(axis=(0, 1))
    normal = int(np.argmin(spread))
    if spread[normal] > 1e-12 * max(1.0, spread.max()):
        raise ValueError("contact faces are not in one axis-aligned plane")
    u, v = [a for a in range(3) if a != normal]
    lo = X[:, :, [u, v]].min(axis=1)
    hi = X[:, :, [u, v]].max(axis=1)
    code = ((np.isclose(X[:, :, u], hi[:, None, 0])).astype(np.int64)
            | (np.isclose(X[:, :, v], hi[:, None, 1]).astype(np.int64) << 1))
    for row in code:
        if sorted(row.tolist()) != [0, 1, 2, 3]:
            raise ValueError("contact face is not an axis-aligned rectangle")
    return {"normal": normal, "u": u, "v": v, "lo": lo, "hi": hi, "code": code,
            "plane": float(X[0, 0, normal])}


def _bilinear(code, lo, hi, pu, pv):
    """Value of the corner basis function `code` of rectangle [lo, hi] at (pu, pv)."""
    wu = hi[..., 0] - lo[..., 0]
    wv = hi[..., 1] - lo[..., 1]
    fu = np.where(code & 1, (pu - lo[..., 0]) / wu, (hi[..., 0] - pu) / wu)
    fv = np.where(code & 2, (pv - lo[..., 1]) / wv, (hi[..., 1] - pv) / wv)
    return fu * fv


def stock_offset(t, motion_dir, z0, amp, period, u_axis, v_axis):
    """In-plane (du, dv) displacement of the stock at time t."""
    s = z0 + amp * np.sin(2.0 * np.pi * t / period)
    d = np.asarray(motion_dir, dtype=np.float64) * s
    return d[u_axis], d[v_axis]


def friction_flux(t, q0, period):
    """q(t) = q0 |cos(2 pi t / Per)| (the |v| / max|v| scaling of the motion law)."""
    return q0 * abs(np.cos(2.0 * np.pi * t / period))


def overlap_pairs(fix, mov, du, dv):
    """All (stand face, stock face) pairs whose rectangles overlap with positive area."""
    ua = np.maximum(fix["lo"][:, None, 0], mov["lo"][None, :, 0] + du)
    ub = np.minimum(fix["hi"][:, None, 0], mov["hi"][None, :, 0] + du)
    va = np.maximum(fix["lo"][:, None, 1], mov["lo"][None, :, 1] + dv)
    vb = np.minimum(fix["hi"][:, None, 1], mov["hi"][None, :, 1] + dv)
    f, s = np.nonzero((ub > ua) & (vb > va))
    return f, s, ua[f, s], ub[f, s], va[f, s], vb[f, s]


def contact_flux(T, fix_quads, mov_quads, fix, mov, du, dv, h_c, q, n_dof):
    """f^E on all DOFs (zero away from the contact) for field T.

    fix_quads / mov_quads hold global DOF ids; fix / mov are the rectangle
    descriptions from `contact_rectangles`, with stock rectangles given in the
    stock's reference position (shifted here by (du, dv)).
    """
    out = np.zeros(n_dof)
    f, s, ua, ub, va, vb = overlap_pairs(fix, mov, du, dv)
    if f.size == 0:
        return out
    cu, cv = 0.5 * (ua + ub), 0.5 * (va + vb)
    hu, hv = 0.5 * (ub - ua), 0.5 * (vb - va)
    wgt = hu * hv                               # area / 4 per Gauss point
    flo, fhi = fix["lo"][f], fix["hi"][f]
    mlo = mov["lo"][s] + np.array([du, dv])
    mhi = mov["hi"][s] + np.array([du, dv])
    fcode, mcode = fix["code"][f], mov["code"][s]
    fnod, mnod = fix_quads[f], mov_quads[s]
    for gu in (-GP, GP):
        for gv in (-GP, GP):
            pu, pv = cu + gu * hu, cv + gv * hv
            phi_f = np.stack([_bilinear(fcode[:, a], flo, fhi, pu, pv) for a in range(4)], axis=1)
            phi_m = np.stack([_bilinear(mcode[:, a], mlo, mhi, pu, pv) for a in range(4)], axis=1)
            Tf = np.sum(phi_f * T[fnod], axis=1)
            Tm = np.sum(phi_m * T[mnod], axis=1)
            flux_f = h_c * (Tm - Tf) + 0.5 * q
            flux_m = h_c * (Tf - Tm) + 0.5 * q
            np.add.at(out, fnod.ravel(), (wgt[:, None] * flux_f[:, None] * phi_f).ravel())
            np.add.at(out, mnod.ravel(), (wgt[:, None] * flux_m[:, None] * phi_m).ravel())
    return out


def covered_area(fix, mov, du, dv):
    """Area of Gamma_R(t): sum of the overlap rectangles."""
    _, _, ua, ub, va, vb = overlap_pairs(fix, mov, du, dv)
    return float(np.sum((ub - ua) * (vb - va)))
