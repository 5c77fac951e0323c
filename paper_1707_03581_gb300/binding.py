"""Thin ctypes binding of libsdcheat (the C ABI in include/sdcheat.h).

Argument marshalling only: every step of the simulation runs in the
library's CUDA kernels. PyTorch provides the device, the stream and, through
the allocator hook, the device memory. There is no CPU fallback: if the
library is missing or no GPU is present, calls raise.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsdcheat.so")

SDC_OK = 0
STATUS_NAMES = {0: "SDC_OK", -1: "SDC_ERR_ARG", -2: "SDC_ERR_OOM", -3: "SDC_ERR_CUDA",
                -4: "SDC_ERR_NOT_CONVERGED", -5: "SDC_ERR_TIMEOUT", -6: "SDC_ERR_STATE"}
NODES = {"equi_noleft": 0, "radau_right": 1, "lobatto": 2}
PRECISION = {"fp64": 0, "mixed": 1}
MAX_SWEEPS = 15

_i64p = C.POINTER(C.c_int64)
_f64p = C.POINTER(C.c_double)
_vp = C.c_void_p


class StepReport(C.Structure):
    _fields_ = [("t", C.c_double), ("sweeps", C.c_int32), ("n_solves", C.c_int32),
                ("cg_iters_total", C.c_int32), ("cg_iters_max", C.c_int32),
                ("refinements_total", C.c_int32), ("status", C.c_int32), ("kernel_launches", C.c_int32),
                ("residual", C.c_double * (MAX_SWEEPS + 1)),
                ("heat_stand", C.c_double), ("heat_stock", C.c_double),
                ("contact_cluster", C.c_int32), ("pad_", C.c_int32), ("true_residual_max", C.c_double)]

    def as_dict(self):
        return {"t": self.t, "sweeps": self.sweeps, "n_solves": self.n_solves,
                "cg_iters_total": self.cg_iters_total, "cg_iters_max": self.cg_iters_max,
                "refinements_total": self.refinements_total, "status": self.status,
                "kernel_launches": self.kernel_launches,
                "residual": [r for r in self.residual[: self.sweeps + 1]],
                "heat_stand": self.heat_stand, "heat_stock": self.heat_stock,
                "contact_cluster": self.contact_cluster, "true_residual_max": self.true_residual_max}


class TuneReport(C.Structure):
    _fields_ = [("cg_unroll", C.c_int32), ("update_blocks_per_sm", C.c_int32), ("contact_cluster_cap", C.c_int32),
                ("contact_cluster", C.c_int32), ("contact_global", C.c_int32), ("graph_branches", C.c_int32),
                ("trials", C.c_int32), ("cached", C.c_int32), ("skipped", C.c_int32), ("pad_", C.c_int32),
                ("ms_default", C.c_double), ("ms_tuned", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad_"}


class Heat(C.Structure):
    _fields_ = [("stored_stand", C.c_double), ("stored_stock", C.c_double),
                ("friction_in", C.c_double), ("t", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(_vp, C.c_size_t, _vp)
FREE_FN = C.CFUNCTYPE(None, _vp, _vp)

_SIGS = {
    "sdc_create": (C.c_int, [C.POINTER(_vp), C.c_int, _vp]),
    "sdc_create_own_stream": (C.c_int, [C.POINTER(_vp), C.c_int]),
    "sdc_get_stream": (C.c_int, [_vp, C.POINTER(_vp)]),
    "sdc_destroy": (None, [_vp]),
    "sdc_scheme_weights": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int] + [C.POINTER(C.c_double)] * 6),
    "sdc_last_error": (C.c_char_p, [_vp]),
    "sdc_set_allocator": (C.c_int, [_vp, ALLOC_FN, FREE_FN, _vp]),
    "sdc_set_body": (C.c_int, [_vp, C.c_int, _f64p, C.c_int64, _i64p, C.c_int64, _f64p,
                               C.c_double, C.c_double, C.c_double]),
    "sdc_set_robin": (C.c_int, [_vp, C.c_int, _i64p, C.c_int64, C.c_double, C.c_double]),
    "sdc_add_robin": (C.c_int, [_vp, C.c_int, _i64p, C.c_int64, C.c_double, C.c_double]),
    "sdc_set_stepper": (C.c_int, [_vp, C.c_int]),
    "sdc_set_cg_unroll": (C.c_int, [_vp, C.c_int]),
    "sdc_set_stationary_state": (C.c_int, [_vp, C.c_double, C.c_double, C.c_int32, C.POINTER(C.c_int32)]),
    "sdc_set_contact": (C.c_int, [_vp, _i64p, C.c_int64, _i64p, C.c_int64, C.c_double, C.c_double]),
    "sdc_set_motion": (C.c_int, [_vp, _f64p, C.c_double, C.c_double, C.c_double]),
    "sdc_assemble": (C.c_int, [_vp]),
    "sdc_set_scheme": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                 C.c_double, C.c_int, C.c_int]),
    "sdc_set_diagnostics": (C.c_int, [_vp, C.c_int]),
    "sdc_set_execution": (C.c_int, [_vp, C.c_int]),
    "sdc_set_kernel_timing": (C.c_int, [_vp, C.c_int]),
    "sdc_set_contact_replicas": (C.c_int, [_vp, C.c_int]),
    "sdc_set_contact_cluster": (C.c_int, [_vp, C.c_int]),
    "sdc_set_graph_branches": (C.c_int, [_vp, C.c_int]),
    "sdc_get_kernel_times": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_char_p), C.POINTER(C.c_int32),
                                       _f64p, C.POINTER(C.c_int32)]),
    "sdc_set_temperature": (C.c_int, [_vp, _vp, C.c_double, C.c_double]),
    "sdc_step": (C.c_int, [_vp, C.POINTER(StepReport)]),
    "sdc_run_horizon": (C.c_int, [_vp, C.c_int64, C.POINTER(StepReport)]),
    "sdc_synchronize": (C.c_int, [_vp]),
    "sdc_get_sizes": (C.c_int, [_vp, _i64p, _i64p, _i64p, _i64p]),
    "sdc_set_matrix_columns": (C.c_int, [_vp, C.c_int]),
    "sdc_get_matrix_columns": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "sdc_get_matrix_implied": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "sdc_get_temperature": (C.c_int, [_vp, _vp, C.c_int64]),
    "sdc_get_temperature_device": (C.c_int, [_vp, C.POINTER(_vp)]),
    "sdc_get_heat_totals": (C.c_int, [_vp, C.POINTER(Heat)]),
    "sdc_get_system": (C.c_int, [_vp, _i64p, _i64p, _f64p, _f64p, _f64p]),
    "sdc_apply_operator": (C.c_int, [_vp, C.c_double, _vp, _vp]),
    "sdc_solve": (C.c_int, [_vp, C.c_double, _vp, _vp, C.POINTER(C.c_int32)]),
    "sdc_set_wait_limit": (C.c_int, [_vp, C.c_int64]),
    "sdc_set_update_blocks": (C.c_int, [_vp, C.c_int]),
    "sdc_autotune": (C.c_int, [_vp, C.c_int32, C.POINTER(TuneReport)]),
    "sdc_time_cg_iterations": (C.c_int, [_vp, C.c_double, C.c_int32, C.c_int32, C.POINTER(C.c_float),
                                         C.POINTER(C.c_float)]),
    "sdc_contact_flux": (C.c_int, [_vp, _vp, C.c_double, _vp]),
    "sdc_heat_totals_noalloc": (C.c_int, [_vp, _vp, _vp]),
    "sdc_poll": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "sdc_step_async": (C.c_int, [_vp, C.c_int64]),
    "sdc_get_footprint": (C.c_int, [_vp, _i64p]),
    "sdc_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int]),
    "sdc_batch_destroy": (None, [_vp]),
    "sdc_batch_last_error": (C.c_char_p, [_vp]),
    "sdc_batch_add": (C.c_int, [_vp, _vp, C.POINTER(C.c_int32)]),
    "sdc_batch_remove": (C.c_int, [_vp, _vp]),
    "sdc_batch_size": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "sdc_batch_step": (C.c_int, [_vp, _i64p, C.c_int]),
    "sdc_batch_synchronize": (C.c_int, [_vp]),
    "sdc_batch_set_fused": (C.c_int, [_vp, C.c_int]),
    "sdc_batch_fused_size": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
}

_LIB = None


NODES = {"equi_noleft": 0, "radau_right": 1, "lobatto": 2}


def scheme_weights(nodes: str, M: int, P: int, window: int = 0) -> dict:
    """The weight tables sdc_set_scheme forms (sdc_scheme_weights; host only, no GPU)."""
    import numpy as np

    lib = load_library()
    shapes = {"c": (M + 1,), "emb": (M, P + 1), "S": (M, M), "Shat": (M, P), "Stil": (M, P, M),
              "Semb": (M, P, P)}
    out = {k: np.zeros(v) for k, v in shapes.items()}
    ptr = [out[k].ctypes.data_as(C.POINTER(C.c_double)) for k in shapes]
    st = lib.sdc_scheme_weights(NODES[nodes], int(M), int(P), int(window), *ptr)
    if st != 0:
        raise SdcError(st, "sdc_scheme_weights refused the scheme")
    return out


def load_library(path: str = LIB_PATH):
    """Load libsdcheat.so and declare every exported signature."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class SdcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_i64p)


class Solver:
    """One simulation context on one GPU (wraps an sdc_ctx)."""

    def __init__(self, device: int = 0, stream=None, torch_allocator: bool = True, own_stream: bool = False):
        """stream: a torch.cuda.Stream to issue work on (default: the current stream);
        own_stream=True: the library creates a private non-blocking stream instead
        (PyTorch hands out pooled streams, which repeat after 32)."""
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (the library has no CPU path)")
        self._torch = torch
        self.lib = load_library()
        self.device = device
        h = _vp()
        if own_stream:
            self._check_plain(self.lib.sdc_create_own_stream(C.byref(h), device))
            ptr = _vp()
            st = self.lib.sdc_get_stream(h, C.byref(ptr))
            if st != SDC_OK:
                self.lib.sdc_destroy(h)
                raise SdcError(st, "sdc_get_stream failed")
            stream = torch.cuda.ExternalStream(ptr.value, device=device)
        else:
            if stream is None:
                stream = torch.cuda.current_stream(device)
            self._check_plain(self.lib.sdc_create(C.byref(h), device, _vp(stream.cuda_stream)))
        self.stream = stream
        self.h = h
        self._keep = []
        if torch_allocator:
            dev, sptr = device, stream.cuda_stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, sptr)
                except Exception:
                    return None

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(int(ptr))

            a, f = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [a, f]
            self._call("sdc_set_allocator", a, f, None)
        self.n = None

    # ---------------------------------------------------------------- plumbing
    def _check_plain(self, st):
        if st != SDC_OK:
            raise SdcError(st, "context creation failed")

    def _call(self, name, *args):
        st = getattr(self.lib, name)(self.h, *args)
        if st != SDC_OK:
            msg = self.lib.sdc_last_error(self.h)
            raise SdcError(st, msg.decode() if msg else "")
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.sdc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- problem
    def set_body(self, body, xyz, hex8, k, rho, c, k_per_hex=None):
        xyz, pxyz = _f64(xyz)
        hx, phx = _i64(hex8)
        if k_per_hex is not None:
            kh, pkh = _f64(k_per_hex)
        else:
            kh, pkh = None, None
        self._call("sdc_set_body", body, pxyz, xyz.shape[0], phx, hx.shape[0], pkh, k, rho, c)

    def set_robin(self, body, quads, h, T_env):
        q, pq = _i64(quads)
        self._call("sdc_set_robin", body, pq, q.shape[0], h, T_env)

    def add_robin(self, body, quads, h, T_env):
        """One more Robin group of the body (sdc_add_robin)."""
        q, pq = _i64(quads)
        self._call("sdc_add_robin", body, pq, q.shape[0], h, T_env)

    def set_stationary_state(self, t0: float = 0.0, rtol: float = 1e-12, max_iter: int = 50000) -> int:
        """Make the stationary state K T0 = b_env (Sec. 5) the temperature at t0; returns
        the CG iterations (sdc_set_stationary_state)."""
        it = C.c_int32()
        self._call("sdc_set_stationary_state", float(t0), float(rtol), int(max_iter), C.byref(it))
        return it.value

    def set_contact(self, stand_quads, stock_quads, h_c, q0):
        a, pa = _i64(stand_quads)
        b, pb = _i64(stock_quads)
        self._call("sdc_set_contact", pa, a.shape[0], pb, b.shape[0], h_c, q0)

    def set_motion(self, direction, z0, amp, period):
        d, pd = _f64(direction)
        self._call("sdc_set_motion", pd, z0, amp, period)

    def assemble(self):
        self._call("sdc_assemble")
        n, nf, nnz, ni = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        self._call("sdc_get_sizes", C.byref(n), C.byref(nf), C.byref(nnz), C.byref(ni))
        self.n, self.n_stand, self.nnz, self.n_contact = n.value, nf.value, nnz.value, ni.value

    def set_scheme(self, nodes="lobatto", M=3, P=20, sweeps=3, window=0, dt=1.0, cg_rtol=1e-12,
                   cg_max_iter=2000, precision="fp64"):
        self._call("sdc_set_scheme", NODES[nodes], M, P, sweeps, window, dt, cg_rtol, cg_max_iter,
                   PRECISION[precision])

    def set_execution(self, eager: bool):
        """True: plain kernel launches with host-driven CG loops (profiling/debugging)."""
        self._call("sdc_set_execution", 1 if eager else 0)

    def set_contact_replicas(self, global_memory):
        """Replica placement of the contact loop: False/0 automatic, True/1 global memory
        (staged in shared memory each substep when it fits), 2 global without staging, 3 the
        grid-wide loop (one contact DOF a thread, cooperative launch)."""
        self._call("sdc_set_contact_replicas", int(global_memory))

    STEPPERS = {"mrsdc": 0, "sisdc": 1, "implicit_euler": 2}

    def set_stepper(self, stepper: str):
        """Time stepper of step(): "mrsdc" (default), "sisdc" (single-rate semi-implicit
        SDC, Sec. 3) or "implicit_euler" (coupling in the matrix) (sdc_set_stepper)."""
        if stepper not in self.STEPPERS:
            raise ValueError(f"unknown stepper {stepper!r}")
        self._call("sdc_set_stepper", self.STEPPERS[stepper])

    def set_cg_unroll(self, pairs: int):
        """(SpMV, update) pairs per CG loop body, 1..8; 0 = by grid size (sdc_set_cg_unroll)."""
        self._call("sdc_set_cg_unroll", int(pairs))

    def set_matrix_columns(self, bits: int):
        """Column form of the stored matrix from the next assembly (set_machine): 0 automatic
        (16-bit offsets from each slice's base when they reach, and implied columns for the
        FP32 copy when the matrix allows them), 16 = the same without implied columns,
        32 = 32-bit columns."""
        self._call("sdc_set_matrix_columns", int(bits))

    def matrix_columns(self) -> int:
        """Bits of a column index in the assembled matrix (16 or 32)."""
        b = C.c_int32()
        self._call("sdc_get_matrix_columns", C.byref(b))
        return b.value

    def matrix_implied(self) -> bool:
        """Whether the assembled matrix's FP32 copy has implied columns (no stored column)."""
        b = C.c_int32()
        self._call("sdc_get_matrix_implied", C.byref(b))
        return bool(b.value)

    def set_graph_branches(self, on: bool):
        """Run solve-independent kernels beside the implicit solves (True) or in one chain."""
        self._call("sdc_set_graph_branches", 1 if on else 0)

    def set_contact_cluster(self, max_ctas: int):
        """Cap the CTAs of the contact substep loop's cluster (0: automatic)."""
        self._call("sdc_set_contact_cluster", int(max_ctas))

    def set_kernel_timing(self, on: bool):
        """Eager steps time every kernel launch with CUDA events (see sdc_set_kernel_timing)."""
        self._call("sdc_set_kernel_timing", 1 if on else 0)

    def kernel_times(self):
        """{kernel name: (launches, total device ms)} of the timed eager steps."""
        cap = 32
        names = (C.c_char_p * cap)()
        n = (C.c_int32 * cap)()
        ms = (C.c_double * cap)()
        k = C.c_int32()
        self._call("sdc_get_kernel_times", cap, names, n, ms, C.byref(k))
        return {names[i].decode(): (n[i], ms[i]) for i in range(min(k.value, cap))}

    def set_diagnostics(self, residuals: bool, true_residual: bool = False):
        """FP64 SDC residual of every sweep (Eq. residual) and/or the FP64 true residual of
        every mixed-precision solve (sdc_set_diagnostics)."""
        self._call("sdc_set_diagnostics", (1 if residuals else 0) | (2 if true_residual else 0))

    def set_temperature(self, T=None, T_uniform=20.0, t0=0.0):
        if T is None:
            self._call("sdc_set_temperature", None, T_uniform, t0)
        elif isinstance(T, np.ndarray):
            arr = np.ascontiguousarray(T, dtype=np.float64)
            self._call("sdc_set_temperature", _vp(arr.ctypes.data), 0.0, t0)
        else:
            t = T.contiguous().to(self._torch.float64)
            self._call("sdc_set_temperature", _vp(t.data_ptr()), 0.0, t0)

    def set_machine(self, m, precision="fp64", T0=None, residuals=False):
        """Feed a synth.Machine (mesh, materials, contact, motion, scheme, initial state)."""
        self.set_body(0, m.stand.mesh.xyz, m.stand.mesh.hex8, m.stand.k, m.stand.rho, m.stand.c,
                      m.stand.k_per_hex)
        self.set_body(1, m.stock.mesh.xyz, m.stock.mesh.hex8, m.stock.k, m.stock.rho, m.stock.c,
                      m.stock.k_per_hex)
        self.set_robin(0, m.stand.robin_quads, m.stand.h, m.stand.T_env)
        self.set_robin(1, m.stock.robin_quads, m.stock.h, m.stock.T_env)
        for b, body in enumerate((m.stand, m.stock)):
            for quads, h, T_env in getattr(body, "robin_extra", ()):
                self.add_robin(b, quads, h, T_env)
        self.set_contact(m.stand_contact, m.stock_contact, m.h_c, m.q0)
        self.set_motion(m.motion_dir, m.z0, m.amp, m.period)
        self.assemble()
        s = m.scheme
        self.set_scheme(s.nodes, s.M, s.P, s.sweeps, s.window, s.dt, s.cg_rtol, s.cg_max_iter, precision)
        self.set_diagnostics(residuals)
        if T0 is None:
            self.set_temperature(None, m.T0, m.t0)
        else:
            self.set_temperature(np.asarray(T0, dtype=np.float64), 0.0, m.t0)

    # ---------------------------------------------------------------- stepping
    def step(self, report: bool = True):
        if report:
            rep = StepReport()
            self._call("sdc_step", C.byref(rep))
            return rep.as_dict()
        self._call("sdc_step", None)
        return None

    def run_horizon(self, n_steps: int):
        rep = StepReport()
        self._call("sdc_run_horizon", int(n_steps), C.byref(rep))
        return rep.as_dict()

    def synchronize(self):
        self._call("sdc_synchronize")

    # ---------------------------------------------------------------- results
    def temperature(self, out=None):
        """T(t_n) as a numpy array (host) or into a given CUDA tensor."""
        if out is None:
            arr = np.empty(self.n, dtype=np.float64)
            self._call("sdc_get_temperature", _vp(arr.ctypes.data), self.n)
            return arr
        self._call("sdc_get_temperature", _vp(out.data_ptr()), self.n)
        return out

    def temperature_device_ptr(self) -> int:
        p = _vp()
        self._call("sdc_get_temperature_device", C.byref(p))
        return p.value

    def heat_totals(self):
        h = Heat()
        self._call("sdc_get_heat_totals", C.byref(h))
        return {"stored_stand": h.stored_stand, "stored_stock": h.stored_stock,
                "friction_in": h.friction_in, "t": h.t}

    def system(self):
        rp = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(self.nnz, dtype=np.int64)
        val = np.empty(self.nnz, dtype=np.float64)
        mass = np.empty(self.n, dtype=np.float64)
        genv = np.empty(self.n, dtype=np.float64)
        self._call("sdc_get_system", rp.ctypes.data_as(_i64p), col.ctypes.data_as(_i64p),
                   val.ctypes.data_as(_f64p), mass.ctypes.data_as(_f64p), genv.ctypes.data_as(_f64p))
        return rp, col, val, mass, genv

    # ---------------------------------------------------------------- components
    def _dev(self, x):
        torch = self._torch
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
        return x.to(device=f"cuda:{self.device}", dtype=torch.float64).contiguous()

    def apply_operator(self, dtau, x):
        x = self._dev(x)
        y = self._torch.empty_like(x)
        self._call("sdc_apply_operator", dtau, _vp(x.data_ptr()), _vp(y.data_ptr()))
        return y

    def set_update_blocks(self, blocks_per_sm: int):
        """Blocks a SM of the FP32 CG update's grid (0 = as many as fit; sdc_set_update_blocks)."""
        self._call("sdc_set_update_blocks", int(blocks_per_sm))

    def autotune(self, trial_steps: int = 3) -> dict:
        """Pick and set the launch options from timed trial steps (sdc_autotune); the state is
        left as it was. Returns the picks and the timings."""
        rep = TuneReport()
        self._call("sdc_autotune", int(trial_steps), C.byref(rep))
        return rep.as_dict()

    def set_wait_limit(self, polls: int):
        """Polls of each bounded exchange wait of the contact loop (0 = default; sdc_set_wait_limit)."""
        self._call("sdc_set_wait_limit", int(polls))

    def time_cg_iterations(self, dtau: float, n_iters: int, spmv_only: bool = False, per_spmv: bool = False):
        """Device milliseconds of n_iters consecutive CG iterations of the implicit stage in
        the scheme's precision, launched as one CUDA graph (sdc_time_cg_iterations); with
        per_spmv, also the summed durations of their SpMVs (events inside the graph)."""
        ms, ms_spmv = C.c_float(0.0), C.c_float(0.0)
        self._call("sdc_time_cg_iterations", float(dtau), int(n_iters), 1 if spmv_only else 0, C.byref(ms),
                   C.byref(ms_spmv) if per_spmv else None)
        return (float(ms.value), float(ms_spmv.value)) if per_spmv else float(ms.value)

    def solve(self, dtau, b, x0):
        b = self._dev(b)
        x = self._dev(x0).clone()
        it = C.c_int32()
        self._call("sdc_solve", dtau, _vp(b.data_ptr()), _vp(x.data_ptr()), C.byref(it))
        return x, it.value

    def contact_flux(self, T, t):
        T = self._dev(T)
        out = self._torch.empty_like(T)
        self._call("sdc_contact_flux", _vp(T.data_ptr()), float(t), _vp(out.data_ptr()))
        return out

    def step_async(self, n_steps: int = 1):
        """Enqueue n_steps macro steps on this solver's stream and return at once."""
        self._call("sdc_step_async", int(n_steps))

    def footprint(self) -> int:
        """Device bytes held by this context."""
        b = C.c_int64()
        self._call("sdc_get_footprint", C.byref(b))
        return b.value

    def poll(self) -> bool:
        """True once every step enqueued on this solver's stream has finished (non-blocking)."""
        idle = C.c_int()
        self._call("sdc_poll", C.byref(idle))
        return bool(idle.value)

    def heat_totals_noalloc(self, T_ptr: int, out):
        """Stored heat of stand and stock of the device field at T_ptr, into the
        2-element float64 CUDA tensor `out`, without any device allocation
        (see sdc_heat_totals_noalloc: fixed scratch, at most 8,388,608 DOF;
        concurrent calls on one device race)."""
        if not (getattr(out, "is_cuda", False) and out.device.index == self.device):
            raise ValueError(f"out must be a CUDA tensor on cuda:{self.device}")
        import torch

        if out.dtype != torch.float64 or out.numel() < 2 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 tensor of at least 2 elements")
        self._call("sdc_heat_totals_noalloc", _vp(int(T_ptr)), _vp(out.data_ptr()))
        return out


class Batch:
    """Several machines stepped concurrently on one GPU (wraps an sdc_batch).

    Each member is a Solver with its own stream; members keep their own state,
    so every result equals the member run alone. The batch does not own them."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        h = _vp()
        st = self.lib.sdc_batch_create(C.byref(h), device)
        if st != SDC_OK:
            raise SdcError(st, "batch creation failed")
        self.h = h
        self.members = []

    def _call(self, name, *args):
        st = getattr(self.lib, name)(self.h, *args)
        if st != SDC_OK:
            msg = self.lib.sdc_batch_last_error(self.h)
            raise SdcError(st, msg.decode() if msg else "")

    def add(self, solver: "Solver") -> int:
        idx = C.c_int32()
        self._call("sdc_batch_add", solver.h, C.byref(idx))
        self.members.append(solver)
        return idx.value

    def remove(self, solver: "Solver"):
        self._call("sdc_batch_remove", solver.h)
        self.members.remove(solver)

    def __len__(self):
        n = C.c_int32()
        self._call("sdc_batch_size", C.byref(n))
        return n.value

    def step(self, n_steps=None, wait: bool = True):
        """Enqueue n_steps[i] macro steps of member i (default one each), round-robin."""
        if n_steps is None:
            self._call("sdc_batch_step", None, 1 if wait else 0)
        else:
            arr, p = _i64(n_steps)
            self._call("sdc_batch_step", p, 1 if wait else 0)

    def synchronize(self):
        self._call("sdc_batch_synchronize")

    def set_fused(self, on: bool):
        """Block-diagonal form: qualifying members' FP32 CG as one launch (sdc_batch_set_fused)."""
        self._call("sdc_batch_set_fused", 1 if on else 0)

    def fused_size(self) -> int:
        n = C.c_int32()
        self._call("sdc_batch_fused_size", C.byref(n))
        return n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.sdc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

