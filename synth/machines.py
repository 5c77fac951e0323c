"""Box-shaped stand/stock machines of the kind simulated in Sec. 2 and Sec. 5.

The paper's own machine geometry and material table are not available, so
the workloads are synthetic boxes of the same physics:

* the fixed *stand* is the box [0,0.4] x [0,0.4] x [0,1] m;
* the moving *stock* is the box [0.1,0.3] x [0.4,0.6] x [0,0.3] m in its
  reference position and slides along +z by the displacement
  s(t) = z0 + A sin(2 pi t / Per) (motion law of Sec. 5, with the
  configuration's own z0, A, Per);
* the contact (Gamma_R in Sec. 2) is the stand face y = 0.4 restricted to
  the rail strip x in [0.1, 0.3] against the stock face y = 0.4;
* the rail strip is insulated where the stock does not cover it; every other
  outer face of both bodies carries one Robin condition (h, T_env).

Everything returned here is plain input data: coordinates, connectivity,
boundary quadrilaterals, material constants, motion and scheme parameters,
and seeded random draws. No finite-element or time-stepping arithmetic lives
in this module.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

STAND_SIZE = (0.4, 0.4, 1.0)
STOCK_ORIGIN = (0.1, 0.4, 0.0)
STOCK_SIZE = (0.2, 0.2, 0.3)
RAIL_X = (0.1, 0.3)

STEEL_RHO = 7850.0   # kg/m^3
STEEL_C = 460.0      # J/(kg K)
STEEL_K = 50.0       # W/(m K)


@dataclass
class BoxMesh:
    """Structured hexahedral mesh of an axis-aligned box.

    Node (i, j, k) has id i + (nx+1) * (j + (ny+1) * k) (x fastest); hexahedron
    (i, j, k) has id i + nx * (j + ny * k) and lists its corners in the usual
    trilinear order: the bottom face (k) counter-clockwise, then the top face.
    """

    origin: tuple
    size: tuple
    n: tuple
    xyz: np.ndarray = field(repr=False)
    hex8: np.ndarray = field(repr=False)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_hex(self) -> int:
        return int(self.hex8.shape[0])

    def node_id(self, i, j, k):
        nx, ny, _ = self.n
        return np.asarray(i) + (nx + 1) * (np.asarray(j) + (ny + 1) * np.asarray(k))

    def side_quads(self, side: str):
        """Quadrilateral faces on one side of the box.

        Returns (quads[n, 4] node ids, cell_lo[n, 3] float coordinates of the
        face's lower corner, cell_hi[n, 3]). Corners go around the face.
        """
        nx, ny, nz = self.n
        axis = "xyz".index(side[0])
        at_max = side[1:] == "max"
        dims = [nx, ny, nz]
        a, b = [d for d in range(3) if d != axis]
        ia, ib = np.meshgrid(np.arange(dims[a]), np.arange(dims[b]), indexing="ij")
        ia = ia.ravel(order="F")
        ib = ib.ravel(order="F")
        fixed = dims[axis] if at_max else 0
        corners = []
        for da, db in ((0, 0), (1, 0), (1, 1), (0, 1)):
            idx = [None, None, None]
            idx[axis] = np.full_like(ia, fixed)
            idx[a] = ia + da
            idx[b] = ib + db
            corners.append(self.node_id(*idx))
        quads = np.stack(corners, axis=1).astype(np.int64)
        lo = self.xyz[quads[:, 0]]
        hi = self.xyz[quads[:, 2]]
        return quads, lo, hi


def box_mesh(origin, size, n) -> BoxMesh:
    """Uniform nx x ny x nz hexahedral mesh of the box origin + [0, size]."""
    nx, ny, nz = (int(v) for v in n)
    xs = origin[0] + size[0] * np.arange(nx + 1) / nx
    ys = origin[1] + size[1] * np.arange(ny + 1) / ny
    zs = origin[2] + size[2] * np.arange(nz + 1) / nz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()

    def nid(ii, jj, kk):
        return ii + (nx + 1) * (jj + (ny + 1) * kk)

    hex8 = np.stack(
        [
            nid(i, j, k), nid(i + 1, j, k), nid(i + 1, j + 1, k), nid(i, j + 1, k),
            nid(i, j, k + 1), nid(i + 1, j, k + 1), nid(i + 1, j + 1, k + 1), nid(i, j + 1, k + 1),
        ],
        axis=1,
    ).astype(np.int64)
    return BoxMesh(tuple(origin), tuple(size), (nx, ny, nz), xyz, hex8)


@dataclass
class Body:
    """One body: mesh, material constants and its Robin boundary faces."""

    mesh: BoxMesh
    k: float
    rho: float
    c: float
    robin_quads: np.ndarray
    h: float
    T_env: float
    k_per_hex: Optional[np.ndarray] = None
    # further Robin groups (quads, h, T_env): floor, cooling equipment ...
    robin_extra: tuple = ()


@dataclass
class Scheme:
    """Time-stepping parameters of one MRSDC run (Sec. 3)."""

    nodes: str = "lobatto"          # 'lobatto' | 'radau_right' | 'equi_noleft'
    M: int = 3
    P: int = 20
    sweeps: int = 3
    window: int = 0                 # 0 -> min(M, P); P -> the paper's literal weights
    dt: float = 1.0
    cg_rtol: float = 1e-12
    cg_max_iter: int = 2000


@dataclass
class Machine:
    """A stand/stock machine: two bodies, their contact and the stock motion."""

    name: str
    stand: Body
    stock: Body
    stand_contact: np.ndarray      # (n, 4) stand-local node ids (rail strip)
    stock_contact: np.ndarray      # (n, 4) stock-local node ids
    h_c: float
    q0: float
    motion_dir: tuple
    z0: float
    amp: float
    period: float
    scheme: Scheme
    T0: float = 20.0
    t0: float = 0.0
    horizon: float = 60.0

    @property
    def n_dof(self) -> int:
        return self.stand.mesh.n_nodes + self.stock.mesh.n_nodes


def build_machine(
    name: str,
    stand_n,
    stock_n,
    *,
    z0: float = 0.35,
    amp: float = 0.25,
    period: float = 2.0,
    h_c: float = 2000.0,
    q0: float = 5e4,
    h: float = 10.0,
    T_env: float = 20.0,
    k: float = STEEL_K,
    rho: float = STEEL_RHO,
    c: float = STEEL_C,
    k_per_hex_stand: Optional[np.ndarray] = None,
    k_per_hex_stock: Optional[np.ndarray] = None,
    scheme: Optional[Scheme] = None,
    T0: float = 20.0,
    horizon: float = 60.0,
    floor: Optional[tuple] = None,
) -> Machine:
    """Assemble the input arrays of one synthetic machine.

    stand_n must have nx divisible by 4 so that the rail strip x in [0.1, 0.3]
    lies on mesh lines of the stand. floor = (h, T): the stand's y = 0 face
    exchanges heat with a floor at T through h, as a Robin group of its own.
    """
    stand_n = tuple(int(v) for v in stand_n)
    stock_n = tuple(int(v) for v in stock_n)
    if stand_n[0] % 4:
        raise ValueError("stand nx must be divisible by 4 (rail strip on mesh lines)")
    stand = box_mesh((0.0, 0.0, 0.0), STAND_SIZE, stand_n)
    stock = box_mesh(STOCK_ORIGIN, STOCK_SIZE, stock_n)

    # Stand: rail strip on y = 0.4 (ymax) is the contact; the rest of ymax and
    # all other sides are Robin faces.
    robin_stand = []
    stand_extra = ()
    rail = None
    for side in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax"):
        quads, lo, hi = stand.side_quads(side)
        if side == "ymin" and floor is not None:
            stand_extra = ((quads, float(floor[0]), float(floor[1])),)
            continue
        if side == "ymax":
            on_rail = (lo[:, 0] >= RAIL_X[0] - 1e-12) & (hi[:, 0] <= RAIL_X[1] + 1e-12)
            rail = quads[on_rail]
            quads = quads[~on_rail]
        robin_stand.append(quads)
    robin_stand = np.concatenate(robin_stand, axis=0)

    # Stock: its y = 0.4 face (ymin) touches the rail; every other side is Robin.
    robin_stock = []
    contact_stock = None
    for side in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax"):
        quads, _, _ = stock.side_quads(side)
        if side == "ymin":
            contact_stock = quads
            continue
        robin_stock.append(quads)
    robin_stock = np.concatenate(robin_stock, axis=0)

    return Machine(
        name=name,
        stand=Body(stand, k, rho, c, robin_stand, h, T_env, k_per_hex_stand, stand_extra),
        stock=Body(stock, k, rho, c, robin_stock, h, T_env, k_per_hex_stock),
        stand_contact=rail,
        stock_contact=contact_stock,
        h_c=h_c,
        q0=q0,
        motion_dir=(0.0, 0.0, 1.0),
        z0=z0,
        amp=amp,
        period=period,
        scheme=scheme if scheme is not None else Scheme(),
        T0=T0,
        horizon=horizon,
    )


def tiny_machine(**kw) -> Machine:
    """A <= 200-DOF machine (stand 4x2x4 hexes, stock 2x2x2: 102 DOF)."""
    return build_machine("tiny", (4, 2, 4), (2, 2, 2), **kw)


def _res_machine(name, r, **kw):
    """Stand r x r x 2.5r hexes, stock at half resolution (same spacing)."""
    return build_machine(name, (r, r, int(round(2.5 * r))),
                         (r // 2, r // 2, int(round(0.75 * r))), **kw)


def machine_config(idx: int, seed: int = 0, truncate: Optional[int] = None, select=None):
    """The five synthetic workloads, as Machine objects (a list for index 3).

    0: 8x8x20 stand + 4x4x6 stock (1,876 DOF), Lobatto M=3, 3 sweeps, P=20,
       dt = 1 s, 60 s, z(t) = 0.35 + 0.25 sin(2 pi t / 2 s).
    1: 48x48x120 + 24x24x36 (313,646 DOF), amplitude ~ U(0.1, 0.3) m and
       period ~ U(1, 4) s drawn in that order from default_rng(seed); 600 s.
    2: 128x128x320 + 64x64x96 (5,751,586 DOF), per-hex conductivity
       exp(U(ln 40, ln 60)) drawn stand first then stock in hex order;
       Radau IIA M=4, 4 sweeps, P=40, dt = 1 s, 60 s, motion as config 0.
    3: 64 machines; per machine r ~ {16,24,32,48,64}, then A, Per, q0 ~
       U(2.5e4, 7.5e4) W/m^2; scheme as config 0; 120 s each. `truncate`
       keeps only the first machines; `select` (indices) builds only those
       machines, in index order (the draws of all 64 are taken either way).
    4: the serving mix: machines are drawn like config 3 (see `serving_requests`).
    """
    if idx == 0:
        return build_machine("c1-8x8x20", (8, 8, 20), (4, 4, 6),
                             scheme=Scheme("lobatto", 3, 20, 3, 0, 1.0), horizon=60.0)
    if idx == 1:
        rng = np.random.default_rng(seed)
        amp = float(rng.uniform(0.1, 0.3))
        per = float(rng.uniform(1.0, 4.0))
        return build_machine("c2-48x48x120", (48, 48, 120), (24, 24, 36), amp=amp, period=per,
                             scheme=Scheme("lobatto", 3, 20, 3, 0, 1.0), horizon=600.0)
    if idx == 2:
        rng = np.random.default_rng(seed)
        n_stand = 128 * 128 * 320
        n_stock = 64 * 64 * 96
        lo, hi = np.log(40.0), np.log(60.0)
        k_stand = np.exp(rng.uniform(lo, hi, n_stand))
        k_stock = np.exp(rng.uniform(lo, hi, n_stock))
        return build_machine("c3-128x128x320", (128, 128, 320), (64, 64, 96),
                             k_per_hex_stand=k_stand, k_per_hex_stock=k_stock,
                             scheme=Scheme("radau_right", 4, 40, 4, 0, 1.0), horizon=60.0)
    if idx == 3:
        rng = np.random.default_rng(seed)
        out = []
        n = 64 if truncate is None else int(truncate)
        for i in range(64):
            r = int(rng.choice([16, 24, 32, 48, 64]))
            amp = float(rng.uniform(0.1, 0.3))
            per = float(rng.uniform(1.0, 4.0))
            q0 = float(rng.uniform(2.5e4, 7.5e4))
            if i < n and (select is None or i in select):
                out.append(_res_machine(f"c4-m{i}-r{r}", r, amp=amp, period=per, q0=q0,
                                        scheme=Scheme("lobatto", 3, 20, 3, 0, 1.0),
                                        horizon=120.0))
        return out
    raise ValueError(f"no machine list for config index {idx}")


def per_hex_machine(name: str, stand_n, stock_n, seed: int = 0, scheme: Optional[Scheme] = None, **kw) -> Machine:
    """A machine with one conductivity per hexahedron, exp(U(ln 40, ln 60)) W/(m K), drawn
    from default_rng(seed) for the stand's hexes then the stock's, in hex order: the
    material recipe of config 2 at any mesh size (default scheme: config 2's Radau IIA
    M=4, 4 sweeps, P=40, dt = 1 s)."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(40.0), np.log(60.0)
    n_stand = int(np.prod(stand_n))
    n_stock = int(np.prod(stock_n))
    k_stand = np.exp(rng.uniform(lo, hi, n_stand))
    k_stock = np.exp(rng.uniform(lo, hi, n_stock))
    return build_machine(name, stand_n, stock_n, k_per_hex_stand=k_stand, k_per_hex_stock=k_stock,
                         scheme=scheme if scheme is not None else Scheme("radau_right", 4, 40, 4, 0, 1.0), **kw)


def batch_resolutions(seed: int = 0):
    """Index of the first machine of each stand resolution r in the batch of config 3:
    {r: index}, from the same draws as machine_config(3, seed)."""
    rng = np.random.default_rng(seed)
    first = {}
    for i in range(64):
        r = int(rng.choice([16, 24, 32, 48, 64]))
        rng.uniform(0.1, 0.3)
        rng.uniform(1.0, 4.0)
        rng.uniform(2.5e4, 7.5e4)
        first.setdefault(r, i)
    return first


def serving_requests(lam: float, n_requests: int = 500, seed: int = 0, pool: int = 64):
    """Poisson arrival schedule of look-ahead requests (config 4).

    Returns a list of dicts {arrival_s, horizon_s, machine_index} where
    machine_index points into the resident pool drawn like config 3.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out: List[dict] = []
    for _ in range(n_requests):
        t += float(rng.exponential(1.0 / lam))
        out.append({"arrival_s": t, "horizon_s": float(rng.uniform(30.0, 600.0)),
                    "machine_index": int(rng.integers(0, pool))})
    return out


CONFIGS = {
    0: "8x8x20 stand + 4x4x6 stock, Lobatto M=3, 3 sweeps, P=20, dt=1 s, 60 s",
    1: "48x48x120 stand + 24x24x36 stock, seeded stroke, Lobatto M=3, 3 sweeps, P=20, 600 s",
    2: "128x128x320 stand + 64x64x96 stock, per-hex k, Radau IIA M=4, 4 sweeps, P=40",
    3: "64 machines r in {16,24,32,48,64}, Lobatto M=3, 3 sweeps, P=20, 120 s",
    4: "Poisson serving of config-3 machines, horizons U(30,600) s",
}


def slab_machine(ny: int = 8, nz: int = 32, *, scheme: Optional[Scheme] = None, T_source: float = 100.0,
                 T_stand: float = 20.0, alpha: float = 2000.0, speed: float = 0.1, period: float = 80.0,
                 thickness: float = 0.05, height: float = 1.0, length: float = 4.0, source_len: float = 0.2,
                 capacity_ratio: float = 1e12, k: float = STEEL_K, rho: float = STEEL_RHO, c: float = STEEL_C):
    """The reduced problem of Sec. 4 as a two-body machine: a stand rectangle
    (length x height in z and y) whose top edge meets a small source of constant
    temperature T_source moving along it; every other edge insulated, no
    environment (g = 0), no friction.

    The rectangle is a slab one hexahedron thick in x with insulated faces, so
    the trilinear model reduces exactly to the bilinear one of Sec. 4 (nodal
    values equal on both faces). The source is a stock whose volumetric heat
    capacity is capacity_ratio times the stand's, so its temperature stays at
    T_source to ~1/capacity_ratio. The exchange alpha (T_source - T) on the
    overlap is the contact term with h_c = alpha. The source moves by the
    library's motion law, s(t) = z0 + A sin(2 pi t / period), with A set so that
    its speed at t = 0 is -speed (the paper moves it at a constant -0.1 m/s),
    starting with its centre at the middle of the top edge.

    Returns (machine, T0) with T0 the initial temperature vector (stand nodes
    first)."""
    stand = box_mesh((0.0, 0.0, 0.0), (thickness, height, length), (1, ny, nz))
    hz = length / nz
    ns = max(1, int(round(source_len / hz)))
    stock = box_mesh((0.0, height, 0.0), (thickness, height / ny, ns * hz), (1, 1, ns))
    top, _, _ = stand.side_quads("ymax")
    bottom, _, _ = stock.side_quads("ymin")
    none = np.zeros((0, 4), dtype=np.int64)
    amp = -speed * period / (2.0 * np.pi)
    z0 = 0.5 * length - 0.5 * ns * hz
    m = Machine(
        name=f"slab-{ny}x{nz}",
        stand=Body(stand, k, rho, c, none, 0.0, T_stand),
        stock=Body(stock, k, rho * capacity_ratio, c, none, 0.0, T_source),
        stand_contact=top,
        stock_contact=bottom,
        h_c=alpha,
        q0=0.0,
        motion_dir=(0.0, 0.0, 1.0),
        z0=z0,
        amp=amp,
        period=period,
        scheme=scheme if scheme is not None else Scheme("equi_noleft", 5, 8, 4, 8, 1.0, 1e-14, 4000),
        T0=T_stand,
        horizon=20.0,
    )
    T0 = np.concatenate([np.full(stand.n_nodes, T_stand), np.full(stock.n_nodes, T_source)])
    return m, T0


def with_scheme(machine: Machine, **kw) -> Machine:
    """A copy of `machine` with some scheme fields replaced."""
    return replace(machine, scheme=replace(machine.scheme, **kw))
