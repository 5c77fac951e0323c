"""Pins for oracle.contact: the explicit contact/friction term f^E (Sec. 2).

Checked against: zero exchange for a uniform field, total input equal to the
friction flux times the covered area, closed-form integrals of linear fields
(value and first moment), an independent fine midpoint-rule integration with
its own interpolation, and continuity through exactly aligned positions.
"""

import numpy as np

from oracle import contact as ct
from oracle.machine import MachineProblem
from synth import machine_config, tiny_machine


def _setup(mach):
    prob = MachineProblem(mach)
    return prob, prob.fix_rect, prob.mov_rect


def test_uniform_field_no_friction_gives_zero():
    prob, fix, mov = _setup(tiny_machine(z0=0.37))
    T = np.full(prob.n, 23.5)
    for s in (0.0, 0.11, 0.37, 0.5, 0.7):
        f = ct.contact_flux(T, prob.fix_quads, prob.mov_quads, fix, mov, 0.0, s, 2000.0, 0.0, prob.n)
        assert np.abs(f).max() < 1e-10


def test_total_input_is_friction_times_area():
    prob, fix, mov = _setup(machine_config(0))
    rng = np.random.default_rng(1)
    T = 20.0 + rng.standard_normal(prob.n)
    for s in (0.1, 0.2345, 0.6):
        q = 3.7e4
        f = ct.contact_flux(T, prob.fix_quads, prob.mov_quads, fix, mov, 0.0, s, 2000.0, q, prob.n)
        # the whole stock face (0.2 m x 0.3 m) is always on the rail
        assert abs(ct.covered_area(fix, mov, 0.0, s) - 0.06) < 1e-14
        assert abs(f.sum() - q * 0.06) < 1e-8 * q * 0.06


def test_linear_fields_closed_form():
    mach = tiny_machine(z0=0.37)
    prob, fix, mov = _setup(mach)
    xyz_fix = mach.stand.mesh.xyz
    xyz_mov = mach.stock.mesh.xyz
    s = 0.4133
    a, bx, bz = 21.0, 3.0, -2.0       # T_fix = a + bx x + bz z (world)
    c, dx, dz = 24.0, -1.0, 5.0       # T_mov = c + dx x + dz z (world, stock moved by s)
    T = np.concatenate([a + bx * xyz_fix[:, 0] + bz * xyz_fix[:, 2],
                        c + dx * xyz_mov[:, 0] + dz * (xyz_mov[:, 2] + s)])
    h_c, q = 1500.0, 2.0e4
    f = ct.contact_flux(T, prob.fix_quads, prob.mov_quads, fix, mov, 0.0, s, h_c, q, prob.n)
    u0, u1, v0, v1 = 0.1, 0.3, s, s + 0.3
    area = (u1 - u0) * (v1 - v0)
    Iu = (u1 ** 2 - u0 ** 2) / 2 * (v1 - v0)
    Iv = (v1 ** 2 - v0 ** 2) / 2 * (u1 - u0)
    Iuu = (u1 ** 3 - u0 ** 3) / 3 * (v1 - v0)
    Iuv = (u1 ** 2 - u0 ** 2) / 2 * (v1 ** 2 - v0 ** 2) / 2
    # flux into the stand: h_c (T_mov - T_fix) + q/2 = alpha + beta_u u + beta_v v
    alpha = h_c * (c - a) + q / 2
    bu, bv = h_c * (dx - bx), h_c * (dz - bz)
    fix_total = alpha * area + bu * Iu + bv * Iv
    n_fix = prob.n_fix
    assert abs(f[:n_fix].sum() - fix_total) < 1e-9 * abs(fix_total)
    # first moment: sum_i f_i x_i = int flux * x
    moment = alpha * Iu + bu * Iuu + bv * Iuv
    assert abs(f[:n_fix] @ xyz_fix[:, 0] - moment) < 1e-9 * abs(moment)
    # the stock side receives the opposite exchange plus its own q/2
    mov_total = -h_c * ((c - a) * area + (dx - bx) * Iu + (dz - bz) * Iv) + q / 2 * area
    assert abs(f[n_fix:].sum() - mov_total) < 1e-9 * abs(mov_total)


def _grid_interp(xs, zs, vals, px, pz):
    """Independent bilinear interpolation on a tensor grid (vals[iz, ix])."""
    ix = np.clip(np.searchsorted(xs, px, side="right") - 1, 0, len(xs) - 2)
    iz = np.clip(np.searchsorted(zs, pz, side="right") - 1, 0, len(zs) - 2)
    tx = (px - xs[ix]) / (xs[ix + 1] - xs[ix])
    tz = (pz - zs[iz]) / (zs[iz + 1] - zs[iz])
    w = [((1 - tx) * (1 - tz), iz, ix), (tx * (1 - tz), iz, ix + 1),
         ((1 - tx) * tz, iz + 1, ix), (tx * tz, iz + 1, ix + 1)]
    return w


def test_against_fine_midpoint_rule():
    mach = tiny_machine(z0=0.37)
    prob, fix, mov = _setup(mach)
    rng = np.random.default_rng(7)
    T = 20.0 + rng.standard_normal(prob.n)
    s, h_c, q = 0.2871, 1800.0, 1.0e4
    f = ct.contact_flux(T, prob.fix_quads, prob.mov_quads, fix, mov, 0.0, s, h_c, q, prob.n)

    # stand rail grid: nodes on y = 0.4 with x in [0.1, 0.3]
    xf, yf, zf = mach.stand.mesh.xyz.T
    sel = np.isclose(yf, 0.4) & (xf > 0.1 - 1e-12) & (xf < 0.3 + 1e-12)
    xs_f, zs_f = np.unique(xf[sel]), np.unique(zf[sel])
    gid_f = np.full((len(zs_f), len(xs_f)), -1)
    for i in np.nonzero(sel)[0]:
        gid_f[np.searchsorted(zs_f, zf[i]), np.searchsorted(xs_f, xf[i])] = i
    xm, ym, zm = mach.stock.mesh.xyz.T
    selm = np.isclose(ym, 0.4)
    xs_m, zs_m0 = np.unique(xm[selm]), np.unique(zm[selm])
    zs_m = zs_m0 + s
    gid_m = np.full((len(zs_m), len(xs_m)), -1)
    for i in np.nonzero(selm)[0]:
        gid_m[np.searchsorted(zs_m0, zm[i]), np.searchsorted(xs_m, xm[i])] = i + prob.n_fix
    assert (gid_f >= 0).all() and (gid_m >= 0).all()

    n = 400
    px = 0.1 + (np.arange(n) + 0.5) * 0.2 / n
    pz = s + (np.arange(n) + 0.5) * 0.3 / n
    PX, PZ = np.meshgrid(px, pz)
    PX, PZ = PX.ravel(), PZ.ravel()
    dA = 0.2 * 0.3 / (n * n)
    wf = _grid_interp(xs_f, zs_f, None, PX, PZ)
    wm = _grid_interp(xs_m, zs_m, None, PX, PZ)
    nid_f = [gid_f[iz, ix] for _, iz, ix in wf]
    nid_m = [gid_m[iz, ix] for _, iz, ix in wm]
    Tf = sum(w * T[ids] for (w, _, _), ids in zip(wf, nid_f))
    Tm = sum(w * T[ids] for (w, _, _), ids in zip(wm, nid_m))
    ref = np.zeros(prob.n)
    for (w, _, _), ids in zip(wf, nid_f):
        np.add.at(ref, ids, (h_c * (Tm - Tf) + q / 2) * w * dA)
    for (w, _, _), ids in zip(wm, nid_m):
        np.add.at(ref, ids, (h_c * (Tf - Tm) + q / 2) * w * dA)
    scale = np.abs(ref).max()
    assert np.abs(f - ref).max() < 2e-4 * scale


def test_continuity_through_aligned_positions():
    prob, fix, mov = _setup(machine_config(0))
    rng = np.random.default_rng(3)
    T = 20.0 + rng.standard_normal(prob.n)
    # stock and stand z-grids coincide at s = 0.35 (both spacings are 0.05)
    f0 = ct.contact_flux(T, prob.fix_quads, prob.mov_quads, fix, mov, 0.0, 0.35, 2000.0, 5e4, prob.n)
    for eps in (1e-13, -1e-13, 1e-9):
        f1 = ct.contact_flux(T, prob.fix_quads, prob.mov_quads, fix, mov, 0.0, 0.35 + eps, 2000.0,
                             5e4, prob.n)
        assert np.abs(f1 - f0).max() < 1e3 * abs(eps) * np.abs(f0).max() + 1e-9


def test_motion_law_and_resting_stock():
    assert ct.stock_offset(0.5, (0, 0, 1), 0.35, 0.25, 2.0, 0, 2) == (0.0, 0.35 + 0.25)
    assert ct.friction_flux(0.5, 5e4, 2.0) < 1e-10 * 5e4          # turning point: |v| = 0
    assert ct.friction_flux(1.0, 5e4, 2.0) == 5e4                 # centre of stroke: |v| max
    assert ct.stock_offset(123.0, (0, 0, 1), 0.35, 0.25, np.inf, 0, 2) == (0.0, 0.35)
    assert ct.friction_flux(123.0, 5e4, np.inf) == 5e4
