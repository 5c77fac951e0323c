"""Benchmark: IMEX multi-rate SDC macro steps of the coupled stand/stock heat problem.

Workload (default): the largest single-GPU machine, 128x128x320 stand + 64x64x96
stock hexes (5,751,586 DOF, one conductivity per hexahedron), Radau IIA M=4,
4 sweeps, P=40 embedded substeps, dt = 1 s, CG to rel 1e-12. One "step" = one
macro step (Algorithm 1 + 4 x Algorithm 2). The 313,646-DOF machine (Lobatto
M=3, 3 sweeps, P=20) is measured beside it (`workload_313k`; --config 1 makes
it the headline).

  value  = DOF x substeps per second (N_dof x M' x P per macro step) of the
           mixed-precision path (FP32 SpMV/CG on the correction inside FP64
           iterative refinement; --precision fp64 times the plain FP64 path)
  eta    = simulated seconds per wall second (look-ahead factor)
  fp64   = the plain FP64 path on the same inputs, timed the same way, with
           the gain of the mixed path over it and the rel-L2 between the two;
           `accuracy` also holds the rel-L2 of each path against the CPU
           oracle's first macro step where the oracle takes one (313k)
  roofline / cg_iteration = the CG SpMV and the whole CG iteration (SpMV +
           update) against the measured HBM bandwidth, from CUDA events in live
           eager steps and in graph execution

Timing: W untimed warm-up steps; then K steps, each bracketed by CUDA events
on the solver's stream, with L2 flushed (256 MiB write) between steps
outside the timed intervals; barrier + synchronize around the region; the
maximum over ranks. `e2e` repeats the run through the public API with the
state coming from and going back to pinned host memory every step.

`--impl reference` times the FP64 CPU oracle on the host cores instead.
Multi-GPU (torchrun): independent replicas, one per GPU (weak scaling).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "look-ahead η & DOF·substeps/s, mixed vs FP64 at rel-L2≤1e-6; p99 latency"
UNIT = "DOF·substeps/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload(config_idx, member=None):
    from synth import machine_config

    m = machine_config(3, select={member})[0] if member is not None else machine_config(config_idx)
    s = m.scheme
    n_int = s.M - 1 if s.nodes == "lobatto" else s.M
    desc = (f"{m.name}: {m.stand.mesh.n[0]}x{m.stand.mesh.n[1]}x{m.stand.mesh.n[2]} stand + "
            f"{m.stock.mesh.n[0]}x{m.stock.mesh.n[1]}x{m.stock.mesh.n[2]} stock ({m.n_dof} DOF), "
            f"{s.nodes} M={s.M}, {s.sweeps} sweeps, P={s.P}, dt={s.dt} s, CG rtol {s.cg_rtol:g}")
    return m, n_int, desc


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _host_cpu():
    """Model name of the host CPU and its logical core count (os.cpu_count())."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform

    return {"model": model or platform.processor() or platform.machine(), "logical_cores": os.cpu_count(),
            "arch": platform.machine()}


def _oracle_env():
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    return env


# The oracle runs in a child process with one thread for BLAS (single-threaded numpy/scipy).
_ORACLE_STEPS = """
import os, sys, time, json, numpy as np
sys.path.insert(0, {root!r})
from synth import machine_config
from oracle.machine import MachineProblem
from oracle.mrsdc import mrsdc_step, mrsdc_step_reduced
from oracle.weights import mrsdc_weights
m = machine_config({idx}); s = m.scheme
t = time.perf_counter()
prob = MachineProblem(m)
W = mrsdc_weights(s.nodes, s.M, s.P, s.window)
asm = time.perf_counter() - t
T = np.full(prob.n, m.T0)
times = []
for n in range({warmup} + {steps}):
    t = time.perf_counter()
    if {reduced}:
        T = mrsdc_step_reduced(prob, T, m.t0 + n * s.dt, s.dt, W, s.sweeps)
    else:
        T, _ = mrsdc_step(prob, T, m.t0 + n * s.dt, s.dt, W, s.sweeps)
    if n >= {warmup}:
        times.append(time.perf_counter() - t)
if {save_to!r}:
    np.save({save_to!r}, T)
print(json.dumps({{"seconds": times, "n": prob.n, "assembly_s": asm}}))
"""

# A bounded sample of one macro step: Algorithm 1 on the first interval of positive length
# (its implicit solve, f*_m, then the first `substeps` of its P explicit substeps on the full
# vectors), with the oracle's own predictor code, repeated from the same start.
_ORACLE_SAMPLE = """
import os, sys, time, json, numpy as np
sys.path.insert(0, {root!r})
from synth import machine_config
from oracle.machine import MachineProblem
from oracle.mrsdc import predictor_interval, predictor_interval_reduced
from oracle.weights import mrsdc_weights
m = machine_config({idx}); s = m.scheme
t = time.perf_counter()
prob = MachineProblem(m)
W = mrsdc_weights(s.nodes, s.M, s.P, s.window)
asm = time.perf_counter() - t
c = W["c"]
k = next(j for j in range(s.M) if c[j + 1] > c[j])
tau_l, tau_r = m.t0 + s.dt * c[k], m.t0 + s.dt * c[k + 1]
emb = [m.t0 + s.dt * e for e in W["emb"][k]]
T = np.full(prob.n, m.T0)
times, it = [], 0
for n in range({warmup} + {reps}):
    t = time.perf_counter()
    if {reduced}:
        _, Temb, it = predictor_interval_reduced(prob, T, tau_l, tau_r, emb, n_substeps={substeps})
    else:
        Temb, it = predictor_interval(prob, T, tau_l, tau_r, emb, n_substeps={substeps})
    if n >= {warmup}:
        times.append(time.perf_counter() - t)
print(json.dumps({{"seconds": times, "n": prob.n, "assembly_s": asm, "interval": k + 1, "cg_iters": it,
                   "substeps": len(Temb) - 1}}))
"""


def _oracle_start(code):
    """Start an oracle child process (returns the Popen; read it with _oracle_finish)."""
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                            env=_oracle_env())


def _oracle_finish(proc, timeout=3600):
    out, err = proc.communicate(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError("oracle run failed: " + err[-2000:])
    return json.loads(out.strip().splitlines()[-1])


def _oracle_steps(config_idx, steps, warmup=0, save_to=None, reduced=False):
    """reduced: the oracle's interface-only form (substeps on the contact DOFs only)."""
    return _oracle_start(_ORACLE_STEPS.format(root=ROOT, idx=config_idx, steps=steps, warmup=warmup,
                                              save_to=save_to, reduced=reduced))


def _oracle_sample(config_idx, substeps, reps, warmup=0, reduced=False):
    return _oracle_start(_ORACLE_SAMPLE.format(root=ROOT, idx=config_idx, substeps=substeps, reps=reps,
                                               warmup=warmup, reduced=reduced))


# Workloads whose oracle macro step does not fit a bounded CPU sample: the sample is part of
# Algorithm 1 (first interval: its solve and the first SAMPLE_SUBSTEPS substeps).
SAMPLE_SUBSTEPS = {2: 8}
REFERENCE_SUBSTEPS = {2: 2}


def _sample_desc(m, n_int, substeps, res):
    return (f"Algorithm 1 on interval {res['interval']} of the first macro step of the {m.n_dof}-DOF workload: "
            f"its implicit solve ({res['cg_iters']} CG iterations from the uniform start), f*_m and the first "
            f"{substeps} of its P = {m.scheme.P} explicit substeps on the full vectors; credited "
            f"{substeps} x {m.n_dof} DOF-substeps per sample. A macro step runs {n_int} intervals of P substeps "
            f"and {m.scheme.sweeps} sweeps, whose quadratures and f^E differences the sample leaves out, so this "
            f"rate bounds the oracle's macro-step rate from above; single-threaded numpy/scipy "
            f"(oracle assembly, {res['assembly_s']:.0f} s, not timed)")


def _reduced_baseline(proc, m, n_int, config_idx, units_per_step):
    """The fairer CPU number: the oracle with the substeps on the interface only
    (oracle.mrsdc.*_reduced), on the same sample, credited the same DOF-substeps."""
    import numpy as np

    res = _oracle_finish(proc)
    if config_idx in SAMPLE_SUBSTEPS:
        S = SAMPLE_SUBSTEPS[config_idx]
        v = res["n"] * S / float(np.mean(res["seconds"]))
        sample = (f"the sample above with its {S} substeps on the {m.n_dof}-DOF workload's interface only and "
                  f"the interval's bulk update skipped (it follows the last substep)")
    else:
        v = units_per_step / float(np.mean(res["seconds"]))
        sample = "one macro step with every embedded substep on the interface only and one bulk update an interval"
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle, interface-only substeps", "sample": sample}


def _pool_worker(cfg, member, reduced, barrier, queue):
    """One oracle process of the multi-machine CPU baseline (spawned; BLAS threads = 1 from the
    environment the parent set): assemble machine `member` of workload `cfg`, wait for the
    others, run one macro step, report its DOF-substeps and monotonic start and end."""
    import threading

    import numpy as np

    sys.path.insert(0, ROOT)
    from oracle.machine import MachineProblem
    from oracle.mrsdc import mrsdc_step, mrsdc_step_reduced
    from oracle.weights import mrsdc_weights
    from synth import machine_config

    try:
        m = machine_config(cfg, select=[member])[0]
        sc = m.scheme
        prob = MachineProblem(m)
        W = mrsdc_weights(sc.nodes, sc.M, sc.P, sc.window)
        T = np.full(prob.n, m.T0)
        n_int = sum(1 for j in range(sc.M) if W["c"][j + 1] > W["c"][j])
        barrier.wait(timeout=1800)
        t0 = time.monotonic()
        if reduced:
            mrsdc_step_reduced(prob, T, m.t0, sc.dt, W, sc.sweeps)
        else:
            mrsdc_step(prob, T, m.t0, sc.dt, W, sc.sweeps)
        t1 = time.monotonic()
        queue.put({"member": member, "n": int(prob.n), "units": int(prob.n) * n_int * sc.P, "t0": t0, "t1": t1})
    except (Exception, threading.BrokenBarrierError) as e:  # reported, not raised: the parent waits on the queue
        barrier.abort()
        queue.put({"member": member, "error": repr(e)[:300]})


def _oracle_pool(cfg, members, reduced=False, timeout=1800):
    """The oracle across the host cores for a workload of many machines: one spawned process
    per machine (single-threaded numpy/scipy each), all assembled first, then one macro step
    each started together; value = their DOF-substeps / (last end - first start)."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    names = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {v: os.environ.get(v) for v in names}
    for v in names:
        os.environ[v] = "1"
    procs = []
    try:
        barrier, queue = ctx.Barrier(len(members)), ctx.Queue()
        procs = [ctx.Process(target=_pool_worker, args=(cfg, i, reduced, barrier, queue)) for i in members]
        for pr in procs:
            pr.start()
        res = [queue.get(timeout=timeout) for _ in procs]
        for pr in procs:
            pr.join(timeout=60)
    finally:
        for pr in procs:
            if pr.is_alive():
                pr.terminate()
        for v, x in saved.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x
    bad = [r for r in res if "error" in r]
    if bad:
        raise RuntimeError(f"oracle process failed: {bad[0]}")
    units = sum(r["units"] for r in res)
    secs = max(r["t1"] for r in res) - min(r["t0"] for r in res)
    dofs = sorted(r["n"] for r in res)
    return {"value": units / secs, "unit": UNIT, "cores": len(members), "kind": "oracle",
            "sample": (f"one macro step of each of {len(members)} machines of the workload ({dofs[0]}-{dofs[-1]} "
                       f"DOF, {sum(dofs)} in total){' with interface-only substeps' if reduced else ''}, one "
                       f"process per machine (single-threaded numpy/scipy), assembled first (not timed) and "
                       f"started together; {secs:.1f} s from the first start to the last end"),
            "host_cpu": _host_cpu()}


def _cpu_baseline_line(value, cores_note, sample, host):
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
            "threads": cores_note, "host_cpu": host}


def run_reference(args, rank, world):
    """The oracle on the host cores (the only reference: the paper ships no code), on the
    workload and metric of the GPU arm: K timed steps after W untimed ones, each a bounded
    sample of the workload (a full macro step where the oracle takes one in seconds, else
    part of Algorithm 1, see SAMPLE_SUBSTEPS)."""
    m, n_int, desc = _workload(args.config)
    if rank != 0:
        return
    host = _host_cpu()
    if args.config in REFERENCE_SUBSTEPS:
        S = REFERENCE_SUBSTEPS[args.config]
        res = _oracle_finish(_oracle_sample(args.config, S, args.steps, args.warmup))
        units = res["n"] * S * len(res["seconds"])
        sample = _sample_desc(m, n_int, S, res)
    else:
        res = _oracle_finish(_oracle_steps(args.config, args.steps, args.warmup))
        units = res["n"] * n_int * m.scheme.P * len(res["seconds"])
        sample = (f"{args.steps} macro steps of the workload after {args.warmup} untimed ones, "
                  f"single-threaded numpy/scipy")
    secs = float(sum(res["seconds"]))
    value = units / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "precision": "fp64", "l2": "n/a (CPU)"},
            "cpu_baseline": _cpu_baseline_line(value, "1 (BLAS threads = 1)", sample, host),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed_steps(s, stream, flush, steps, torch, reports=None):
    """Run `steps` macro steps, each bracketed by CUDA events on the solver's
    stream, with L2 flushed before each one outside the events; return ms per step.
    With a `reports` list, each step's report is appended to it."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        rep = s.step(report=reports is not None)
        ends[k].record(stream)
        if reports is not None:
            reports.append(rep)
        s.synchronize()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def _max_over_ranks(x, world, device="cpu"):
    """The maximum of a float over the job's ranks (x itself on one rank): the job's
    time is its slowest replica's."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _whole_job_rate(units_per_rank, seconds, world):
    """Units that all ranks processed per second of the slowest rank's time (weak
    scaling: every replica processes the same units)."""
    return units_per_rank * world / seconds


def _rel_l2(a, b):
    import numpy as np

    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _kernels_sha():
    import hashlib

    with open(os.path.join(ROOT, "paper_1707_03581_gb300", "csrc", "kernels.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _profile_traffic(kernel, n_dof):
    """DRAM bytes (read + written) per launch of `kernel` on the n_dof-DOF workload, from a
    kept ncu summary under profiles/: a line
        bench-traffic: kernel=<name> n_dof=<N> dram_bytes=<B> kernels_cu_sha256=<first 16 hex>
    Returns (bytes or None, note); None when no summary has the kernel and workload, or when
    kernels.cu changed since the capture (the counters then describe another kernel)."""
    import glob

    sha = _kernels_sha()
    stale = None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for ln in open(path):
            if not ln.startswith("bench-traffic:"):
                continue
            kv = dict(x.split("=", 1) for x in ln.split(":", 1)[1].split())
            if kv.get("kernel") != kernel or int(kv.get("n_dof", -1)) != n_dof:
                continue
            if kv.get("kernels_cu_sha256") != sha:
                stale = os.path.basename(path)
                continue
            return float(kv["dram_bytes"]), f"ncu summary {os.path.basename(path)} (kernels.cu {sha})"
    if stale:
        return None, f"kernels.cu changed since the capture in {stale}"
    return None, "no ncu summary of this kernel on this workload"


def _dominant_kernel(s, precision, kt, reps):
    """The CG SpMV of the timed path and its algorithmic bytes per launch that did work.

    Per SpMV: every nonzero's value and column (FP32 4 or FP64 8 bytes, and a 16-bit
    offset from its 32-row slice's base, 2 bytes, or a 32-bit column, 4 bytes; none for
    the FP32 copy with implied columns), the slices' 4-byte bases (or table positions),
    plus the row vectors it reads (u, r, m) and writes (w). The
    SpMVs that did work in the timed steps are the CG updates plus one stopping
    SpMV per inner solve (from the steps' reports); the loop bodies' later
    launches after a stop return at once, and their time stays in the total. On large
    grids the SpMV's dots are summed by a one-block kernel (k_mx_dots), whose time is
    counted with the SpMV's (its bytes, 12 B per 256 rows, are left out)."""
    n, nnz = s.n, s.nnz
    cb = s.matrix_columns() // 8
    bases = 4 * ((n + 31) // 32) if cb == 2 else 0
    iters = sum(r["cg_iters_total"] for r in reps)
    if precision == "mixed":
        if s.matrix_implied():  # the FP32 copy: values only, one 4-byte table position a slice
            cb, bases = 0, 4 * ((n + 31) // 32)
        name = "k_mx_spmv"
        upd = "k_mx_update" if "k_mx_update" in kt else "k_mx_update_red"
        work = iters + sum(r["refinements_total"] for r in reps)
        sp = kt.get(name, (0, 0.0))
        if "k_mx_dots" in kt:
            sp = (sp[0], sp[1] + kt["k_mx_dots"][1])
        return (name, upd, "FP32 sliced-ELL SpMV w = m u + dtau K u with (r,u), (w,u), (r,r)"
                + (" and its one-block dot sums (k_mx_dots)" if "k_mx_dots" in kt else ""),
                (4 + cb) * nnz + 16 * n + bases, 48 * n, work, sp, kt.get(upd, (0, 0.0)),
                f"{4 + cb} B/nnz + 16 B/row + 4 B per 32-row slice" if cb != 4 else f"{4 + cb} B/nnz + 16 B/row")
    work = iters + sum(r["n_solves"] for r in reps)
    return ("k_cg_spmv", "k_cg_update", "FP64 sliced-ELL SpMV w = m u + dtau K u with (r,u), (w,u), (r,r)",
            (8 + cb) * nnz + 32 * n + bases, 96 * n, work, kt.get("k_cg_spmv", (0, 0.0)),
            kt.get("k_cg_update", (0, 0.0)),
            f"{8 + cb} B/nnz + 32 B/row + 4 B per 32-row slice" if cb == 2 else f"{8 + cb} B/nnz + 32 B/row")


def _graph_cg(s, m, flush, n_iters=30, reps=3):
    """Device time of the CG iterations of the implicit stage in graph execution
    (sdc_time_cg_iterations): n_iters back-to-back (SpMV, update) iterations in one graph, L2
    flushed before each of `reps` graphs; the median per iteration, and the median duration
    of one SpMV inside those iterations (event records around every SpMV in the graph)."""
    dtau = 0.5 * m.scheme.dt
    pair, spmv = [], []
    for _ in range(reps):
        flush.fill_(1.0)
        pair.append(s.time_cg_iterations(dtau, n_iters) / n_iters)
        flush.fill_(2.0)
        spmv.append(s.time_cg_iterations(dtau, n_iters, per_spmv=True)[1] / n_iters)
    return statistics.median(pair), statistics.median(spmv)


def _stationary_start(m, local, torch):
    """The paper's initial state (Sec. 5): the same machine at rest with a 40 degC floor
    under the stand (h = 500 W/m^2K) besides the 20 degC environment, solved for
    K T0 = b_env on the device (FP64 Jacobi-PCG to 1e-12). Timed with CUDA events on the
    solver's stream around the call; its relative residual is checked on the host from
    the assembled system."""
    import numpy as np
    import scipy.sparse as sp

    from paper_1707_03581_gb300 import Solver
    from synth.machines import build_machine

    f = build_machine(m.name + "-floor", m.stand.mesh.n, m.stock.mesh.n, floor=(500.0, 40.0), scheme=m.scheme,
                      amp=m.amp, period=m.period, z0=m.z0, q0=m.q0, k_per_hex_stand=m.stand.k_per_hex,
                      k_per_hex_stock=m.stock.k_per_hex)
    s = Solver(local)
    s.set_machine(f, precision="fp64")
    st = s.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(st)
    iters = s.set_stationary_state(t0=f.t0, rtol=1e-12)
    ev[1].record(st)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    T = s.temperature()
    rp, col, val, _, genv = s.system()
    K = sp.csr_matrix((val, col, rp), shape=(s.n, s.n))
    res = float(np.linalg.norm(genv - K @ T) / np.linalg.norm(genv))
    nf = f.stand.mesh.n_nodes
    out = {"workload": f"{m.n_dof}-DOF machine at rest, stand on a 40 degC floor (h = 500 W/m^2K), "
                       "20 degC environment (h = 10 W/m^2K)",
           "ms": ms, "cg_iterations": iters, "ms_per_iteration": ms / max(iters, 1), "rel_residual": res,
           "T_stand_range": [float(T[:nf].min()), float(T[:nf].max())]}
    s.close()
    return out


def _vs_implicit_euler(m, local, torch, args):
    """Work against accuracy, the comparison of Sec. 5: MRSDC (k = 0..3 sweeps at the
    scheme's dt, and the scheme's sweeps at dt / 2 and dt / 4; the run's precision),
    single-rate SDC and fully implicit Euler with the coupling in the matrix (FP64 solve;
    dt / 1 .. dt / 32) over the same horizon of 8 macro steps from the same start. Error:
    ||T - T_ref|| / ||T_ref - T0|| at the horizon, T_ref from FP64 MRSDC with dt / 64 and
    the scheme's sweeps (its own error is estimated against dt / 32). eta = horizon /
    device time of run_horizon (CUDA events on the solver's stream; a second run from the
    same start, so the step graph exists; no L2 flush: consecutive steps, as a look-ahead
    runs them). Implicit Euler's eta at MRSDC's error is interpolated log-log between the
    two implicit Euler runs that bracket it (extrapolated from the last two, and marked,
    when none reaches it)."""
    import numpy as np

    from paper_1707_03581_gb300 import Solver
    from synth.machines import with_scheme

    n_macro = 8
    dt0 = m.scheme.dt
    horizon = n_macro * dt0

    def run(mach, precision, stepper, n, timed=True):
        s = Solver(local)
        s.set_machine(mach, precision=precision)
        if stepper != "mrsdc":
            s.set_stepper(stepper)
        rep = s.run_horizon(n)
        T = s.temperature()
        ms = None
        if timed:
            s.set_temperature(m.T0 * np.ones(s.n), t0=mach.t0)
            st = s.stream
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            ev[0].record(st)
            rep = s.run_horizon(n)
            ev[1].record(st)
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1])
            assert np.array_equal(T, s.temperature())
        s.close()
        assert rep["status"] == 0
        return T, ms

    T_ref, _ = run(with_scheme(m, dt=dt0 / 64), "fp64", "mrsdc", 64 * n_macro, timed=False)
    T_r32, _ = run(with_scheme(m, dt=dt0 / 32), "fp64", "mrsdc", 32 * n_macro, timed=False)
    rise = np.linalg.norm(T_ref - m.T0)

    def entry(T, ms, dt):
        return {"dt": dt, "rel_err": float(np.linalg.norm(T - T_ref) / rise), "ms": ms, "eta": horizon / (ms * 1e-3)}

    out = {"workload": f"{m.n_dof}-DOF machine, {n_macro} macro steps of {dt0:g} s from {m.T0:g} degC",
           "reference": f"FP64 MRSDC, dt / 64, {m.scheme.sweeps} sweeps",
           "reference_rel_err_estimate": float(np.linalg.norm(T_r32 - T_ref) / rise),
           "mrsdc": {}, "implicit_euler": []}
    for k in range(4):
        T, ms = run(with_scheme(m, sweeps=k), args.precision, "mrsdc", n_macro)
        out["mrsdc"][f"k={k}"] = entry(T, ms, dt0)
    K = m.scheme.sweeps
    for r in (2, 4):
        T, ms = run(with_scheme(m, dt=dt0 / r), args.precision, "mrsdc", r * n_macro)
        out["mrsdc"][f"k={K},dt/{r}"] = entry(T, ms, dt0 / r)
    T, ms = run(with_scheme(m, P=1), args.precision, "sisdc", n_macro)
    out["single_rate_sdc"] = entry(T, ms, dt0)
    for r in (1, 2, 4, 8, 16, 32):
        T, ms = run(with_scheme(m, dt=dt0 / r), args.precision, "implicit_euler", r * n_macro)
        out["implicit_euler"].append(entry(T, ms, dt0 / r))
    # implicit Euler at the error of MRSDC with the scheme's sweeps and dt
    target = out["mrsdc"][f"k={min(K, 3)}"]
    out["ie_at_mrsdc_error"] = _eta_at_error(out["implicit_euler"], target["rel_err"])
    out["eta_gain_mrsdc_vs_ie_at_equal_error"] = target["eta"] / out["ie_at_mrsdc_error"]["eta"]
    return out


def _eta_at_error(runs, err):
    """eta of a method at error `err`, from its runs ({"dt", "rel_err", "eta"}, step sizes
    falling): log eta linear in log error between the first two consecutive runs that
    bracket `err`, else extrapolated from the last two runs (marked)."""
    import numpy as np

    e = np.log([x["rel_err"] for x in runs])
    eta = np.log([x["eta"] for x in runs])
    lt = np.log(err)
    hit = [i for i in range(len(runs) - 1) if e[i] >= lt >= e[i + 1]]
    i = hit[0] if hit else len(runs) - 2
    w = (lt - e[i]) / (e[i + 1] - e[i])
    return {"rel_err": float(err), "eta": float(np.exp(eta[i] + w * (eta[i + 1] - eta[i]))),
            "between_dt": [runs[i]["dt"], runs[i + 1]["dt"]], "extrapolated": not hit}


def _single_rate(m, local, torch, args, flush):
    """Single-rate semi-implicit SDC (Sec. 3) on the same machine, nodes, sweeps and dt
    (mixed precision): f^E only at the standard nodes, no substeps. Timed like the
    headline (CUDA events around each step, L2 flushed between steps); and its relative
    difference from MRSDC after 5 macro steps from the same start, i.e. what resolving
    the contact term on the embedded nodes changes."""
    import numpy as np

    from paper_1707_03581_gb300 import Solver
    from synth.machines import with_scheme

    a = Solver(local)
    a.set_machine(with_scheme(m, P=1, window=0), precision=args.precision)
    a.set_stepper("sisdc")
    b = Solver(local)
    b.set_machine(m, precision=args.precision)
    for _ in range(5):
        a.step(report=False)
        b.step(report=False)
    Ta, Tb = a.temperature(), b.temperature()
    diff = float(np.linalg.norm(Ta - Tb) / np.linalg.norm(Tb))
    rise = float(np.linalg.norm(Ta - Tb) / np.linalg.norm(Tb - m.T0))
    b.close()
    st = a.stream
    with torch.cuda.stream(st):
        for _ in range(args.warmup):
            a.step(report=False)
        torch.cuda.synchronize()
        ms = _timed_steps(a, st, flush, args.steps, torch)
        rep = a.step(report=True)
    a.close()
    ms_step = float(sum(ms) / len(ms))
    return {"ms_per_step": ms_step, "eta": m.scheme.dt / (ms_step * 1e-3), "cg_iters_per_step": rep["cg_iters_total"],
            "rel_l2_vs_mrsdc_after_5_steps": diff, "rel_l2_rise_vs_mrsdc_after_5_steps": rise}


def _measure(m, n_int, args, local, torch, flush, world, precision, compare, e2e=True, clocks=True):
    """Macro steps of machine m timed in graph execution (the path in `precision`, and the
    plain FP64 path on the same inputs when `compare`), per-kernel event times of eager
    steps, the graph-mode CG iterations, and the end-to-end run through the public API."""
    import numpy as np

    from paper_1707_03581_gb300 import Solver

    tune = {}

    def make(prec):
        sv = Solver(local)
        sv.set_machine(m, precision=prec)
        if args.contact_replicas is not None:
            sv.set_contact_replicas(args.contact_replicas)
        if not args.no_tune and not args.eager:
            t = time.perf_counter()
            tune[prec] = sv.autotune(trial_steps=3)
            tune[prec]["seconds"] = time.perf_counter() - t
        if args.eager:
            sv.set_execution(True)
        return sv

    t_setup = time.perf_counter()
    s = make(precision)
    s64 = make("fp64") if compare else None
    t_setup = time.perf_counter() - t_setup
    stream = s.stream
    out = {"n": s.n, "nnz": s.nnz, "n_contact": s.n_contact, "setup_s": t_setup,
           "units_per_step": s.n * n_int * m.scheme.P, "autotune": tune}
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            s.step(report=True)
            if s64 is not None:
                s64.step(report=True)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        with ClockSampler(local) as clk:
            out["ms_steps"] = _timed_steps(s, stream, flush, args.steps, torch)
        out["clocks"] = clk.summary() if clocks else None
        out["rep"] = s.step(report=True)
        if s64 is not None:
            out["ms64"] = _timed_steps(s64, stream, flush, args.steps, torch)
            out["rep64"] = s64.step(report=True)
            Ta, Tb = s.temperature(), s64.temperature()
            out["rel_vs_fp64"] = _rel_l2(Ta, Tb)
            out["rel_rise_vs_fp64"] = _rel_l2(Ta - m.T0, Tb - m.T0)
            s64.close()
        # per-kernel device times of the same steps, each launch between CUDA events on the
        # solver's stream (plain launches; the CG loop is driven from the host one iteration ahead)
        s.set_execution(True)
        s.set_kernel_timing(True)
        out["eager_reps"] = []
        out["eager_ms"] = _timed_steps(s, stream, flush, args.steps, torch, out["eager_reps"])
        out["kt"] = s.kernel_times()
        s.set_kernel_timing(False)
        s.set_execution(bool(args.eager))
        out["graph_cg_ms"], out["graph_spmv_ms"] = _graph_cg(s, m, flush)
        if precision == "mixed":
            # the FP64 true residual of every implicit solve of one more step (diagnostic)
            s.set_diagnostics(False, true_residual=True)
            out["true_residual_max"] = s.step(report=True)["true_residual_max"]
            s.set_diagnostics(False, true_residual=False)
    out["total_ms"] = float(sum(out["ms_steps"]))
    if e2e:
        # end to end through the public API: host state in, host state out, every step
        pin_in = torch.empty(s.n, dtype=torch.float64).pin_memory()
        pin_out = torch.empty(s.n, dtype=torch.float64).pin_memory()
        pin_in.copy_(torch.from_numpy(s.temperature()))
        t_sim = m.t0
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.set_temperature(pin_in.numpy(), t0=t_sim)
            s.step(report=False)
            s.temperature(out=pin_out)
            t_sim += m.scheme.dt
        torch.cuda.synchronize()
        out["e2e_s"] = _max_over_ranks(time.perf_counter() - t0, world, f"cuda:{local}")
    out["solver"] = s
    return out


def _kernel_report(mres, precision, args, peak, peak_kind):
    """Roofline of the dominant kernel (the CG SpMV), the FP32/FP64 CG iteration in graph
    execution, and every kernel's share of the eager steps' kernel time."""
    s, kt, reps = mres["solver"], mres["kt"], mres["eager_reps"]
    name, upd, desc, sp_bytes, up_bytes, n_work, (n_launched, ms_spmv), (_, ms_upd), sp_note = _dominant_kernel(
        s, precision, kt, reps)
    ms_per_spmv = ms_spmv / max(n_work, 1)
    eager_achieved = sp_bytes / (ms_per_spmv * 1e-3) / 1e9 if n_work else 0.0
    traffic, traffic_note = _profile_traffic(name, s.n)
    g_spmv = mres["graph_spmv_ms"]
    g_iter = mres["graph_cg_ms"]
    it_bytes = sp_bytes + up_bytes
    achieved = sp_bytes / (g_spmv * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if peak else None, "traffic": traffic, "traffic_source": traffic_note,
            "kernel": f"{name} ({desc})", "algorithmic_bytes": sp_bytes, "bytes_note": sp_note,
            "ms_per_launch": g_spmv,
            "peak_kind": peak_kind,
            "timing": "CUDA events recorded inside a CUDA graph of 30 back-to-back CG iterations of the "
                      "step's kernels, grids and launch order, around every SpMV (sdc_time_cg_iterations), "
                      "on the solver's stream; L2 flushed before the graph; median of 3 graphs",
            "eager_cross_check": {"ms_per_launch": ms_per_spmv, "achieved": eager_achieved,
                                  "frac": eager_achieved / peak if peak else None,
                                  "launches_timed": n_launched, "launches_working": n_work,
                                  "timing": "CUDA events around each launch of live eager macro steps (host-driven "
                                            "CG loops; a launch that waits for the host counts that wait)"}}
    cg_it = {"kernels": f"{name} + {upd}", "algorithmic_bytes": it_bytes,
             "bytes_note": (f"SpMV {sp_bytes} ({sp_note}) + update {up_bytes} (48 B/row)" if precision == "mixed"
                            else f"SpMV {sp_bytes} ({sp_note}) + update {up_bytes} (96 B/row)"),
             "ms_graph": g_iter, "achieved": it_bytes / (g_iter * 1e-3) / 1e9,
             "frac": it_bytes / (g_iter * 1e-3) / 1e9 / peak, "peak_kind": peak_kind,
             "ms_eager": (ms_spmv + ms_upd) / max(n_work, 1),
             "timing": "30 back-to-back (SpMV, update) iterations in one CUDA graph of the step's kernels, "
                       "grids and launch order (sdc_time_cg_iterations), L2 flushed before; median of 3"}
    kern_total = sum(v[1] for v in kt.values())
    kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps,
                   "ms_per_launch": v[1] / max(v[0], 1), "share": v[1] / kern_total if kern_total else 0.0}
               for k, v in sorted(kt.items(), key=lambda kv: -kv[1][1])}
    return roof, cg_it, kernels


def _workload_summary(m, n_int, mres, args, precision):
    """Per-workload figures: the timed path, the FP64 comparison, the accuracy between them."""
    ms = mres["total_ms"] / args.steps
    units = mres["units_per_step"]
    srt = sorted(mres["ms_steps"])
    out = {"ms_per_step": ms, "value": units / (ms * 1e-3), "eta": m.scheme.dt / (ms * 1e-3),
           "step_latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))]},
           "cg_iters_per_step": mres["rep"]["cg_iters_total"],
           "refinements_per_step": mres["rep"]["refinements_total"],
           "contact_cluster": mres["rep"]["contact_cluster"],
           "eager_ms_per_step": sum(mres["eager_ms"]) / len(mres["eager_ms"]),
           "setup_s": mres["setup_s"],
           "autotune": mres["autotune"] or "off (--no-tune)"}
    if "true_residual_max" in mres:
        out["true_residual_max"] = {
            "value": mres["true_residual_max"],
            "definition": "largest ||b - (m x + dtau K x)|| / ||b|| with the FP64 K over the implicit solves of one "
                          "macro step (the mixed solves stop on a residual carried with the FP32 operator at 1e-12)"}
    if "ms64" in mres:
        ms64 = sum(mres["ms64"]) / args.steps
        out["fp64"] = {"value": units / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                       "eta": m.scheme.dt / (ms64 * 1e-3), "cg_iters_per_step": mres["rep64"]["cg_iters_total"]}
        out["gain_vs_fp64"] = ms64 / ms
        out["accuracy"] = {"rel_l2_mixed_vs_fp64": mres["rel_vs_fp64"],
                           "rel_l2_rise_mixed_vs_fp64": mres["rel_rise_vs_fp64"],
                           "after_steps": args.warmup + args.steps + 1}
    return out


def _oracle_accuracy(m, precision, compare, local, T_or):
    """rel-L2 of the GPU paths against the oracle's first macro step."""
    from paper_1707_03581_gb300 import Solver

    acc = {}
    for prec in ([precision, "fp64"] if compare else [precision]):
        g = Solver(local)
        g.set_machine(m, precision=prec)
        g.step(report=True)
        acc[f"rel_l2_{prec}_vs_oracle_step1"] = _rel_l2(g.temperature(), T_or)
        acc[f"rel_l2_rise_{prec}_vs_oracle_step1"] = _rel_l2(g.temperature() - m.T0, T_or - m.T0)
        g.close()
    return acc


def run_gpu(args, rank, world):
    import tempfile

    import numpy as np
    import torch

    from synth import machine_config

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    m, n_int, desc = _workload(args.config, args.member)
    compare = args.precision == "mixed" and not args.no_compare
    peak, peak_kind = _peaks()
    host = _host_cpu()
    cpu_on = not args.no_cpu_baseline and world == 1 and rank == 0 and args.member is None
    # The 313,646-DOF workload rides along with the 5.75M-DOF headline (labelled extra key); the
    # comparison rows (stationary start, single-rate SDC, implicit Euler) run on it there.
    side_idx = 1 if args.config == 2 and not args.no_extra and args.member is None else None
    tmp = tempfile.mkdtemp()
    oracle = {}
    if cpu_on:
        # the oracle runs in child processes on the host cores while the GPU work proceeds
        if args.config in SAMPLE_SUBSTEPS:
            oracle["main"] = _oracle_sample(args.config, SAMPLE_SUBSTEPS[args.config], reps=1)
            oracle["main_red"] = _oracle_sample(args.config, SAMPLE_SUBSTEPS[args.config], reps=1, reduced=True)
        else:
            oracle["main"] = _oracle_steps(args.config, 1, save_to=os.path.join(tmp, "main.npy"))
            oracle["main_red"] = _oracle_steps(args.config, 1, reduced=True)
        if side_idx is not None:
            oracle["side"] = _oracle_steps(side_idx, 1, save_to=os.path.join(tmp, "side.npy"))
            oracle["side_red"] = _oracle_steps(side_idx, 1, reduced=True)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    mres = _measure(m, n_int, args, local, torch, flush, world, args.precision, compare)
    t_max = _max_over_ranks(mres["total_ms"], world, f"cuda:{local}")
    roof, cg_it, kernels = _kernel_report(mres, args.precision, args, peak, peak_kind)
    summ = _workload_summary(m, n_int, mres, args, args.precision)
    units_per_step = mres["units_per_step"]
    s = mres["solver"]

    side = None
    if side_idx is not None:
        ms_, ni_, desc_ = _workload(side_idx)
        sres = _measure(ms_, ni_, args, local, torch, flush, world, args.precision, compare, e2e=False,
                        clocks=False)
        sroof, scg, skern = _kernel_report(sres, args.precision, args, peak, peak_kind)
        side = {"workload": desc_, **_workload_summary(ms_, ni_, sres, args, args.precision),
                "roofline": sroof, "cg_iteration": scg,
                "kernels_top": dict(list(skern.items())[:6])}
        sres["solver"].close()
    if rank != 0:
        return
    value = units_per_step * args.steps * world / (t_max * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": desc,
                   "precision": ("mixed: FP32 SpMV/CG on the correction inside FP64 iterative refinement, "
                                 "FP64 residuals, quadratures and state" if args.precision == "mixed"
                                 else "fp64 throughout"),
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MiB write); the step's working set exceeds L2",
                   "execution": "eager launches" if args.eager else "one CUDA graph per macro step"},
        "eta": args.steps * m.scheme.dt / (t_max * 1e-3),
        **{k: v for k, v in summ.items() if k not in ("ms_per_step", "value", "eta")},
        "e2e": {"value": units_per_step * args.steps * world / mres["e2e_s"], "unit": UNIT,
                "h2d_bytes_per_step": 8 * s.n, "d2h_bytes_per_step": 8 * s.n,
                "eta": args.steps * m.scheme.dt / mres["e2e_s"]},
        "gpu_launches": mres["rep"]["kernel_launches"] * args.steps,
        "roofline": roof,
        "cg_iteration": cg_it,
        "kernels": kernels,
        "clocks": mres["clocks"],
        "host_cpu": host,
    }
    if side is not None:
        line["workload_313k"] = side
    s.close()
    rows_m = machine_config(side_idx) if side_idx is not None else m
    if not args.no_stationary:
        line["stationary_start"] = _stationary_start(rows_m, local, torch)
    if not args.no_single_rate:
        line["single_rate"] = _single_rate(rows_m, local, torch, args, flush)
    if not args.no_ie and world == 1:
        small = machine_config(0)
        line["vs_implicit_euler"] = [_vs_implicit_euler(x, local, torch, args)
                                     for x in ([rows_m, small] if rows_m.n_dof != small.n_dof else [rows_m])]
    if cpu_on:
        try:
            res = _oracle_finish(oracle["main"])
            if args.config in SAMPLE_SUBSTEPS:
                S = SAMPLE_SUBSTEPS[args.config]
                v = res["n"] * S / float(np.mean(res["seconds"]))
                sample = _sample_desc(m, n_int, S, res)
            else:
                v = units_per_step / float(np.mean(res["seconds"]))
                sample = "one macro step of the same workload, single-threaded numpy/scipy"
                acc = line.setdefault("accuracy", {})
                acc.update(_oracle_accuracy(m, args.precision, compare, local, np.load(os.path.join(tmp, "main.npy"))))
            line["cpu_baseline"] = _cpu_baseline_line(v, "1 (BLAS threads = 1)", sample, host)
            line["cpu_baseline"]["reduced"] = _reduced_baseline(oracle["main_red"], m, n_int, args.config,
                                                                units_per_step)
        except Exception as e:  # reported, not fatal
            line["cpu_baseline"] = {"error": str(e)[:300]}
        if "side" in oracle:
            try:
                ms_, ni_, _ = _workload(side_idx)
                res = _oracle_finish(oracle["side"])
                side_units = ms_.n_dof * ni_ * ms_.scheme.P
                line["workload_313k"]["cpu_baseline"] = _cpu_baseline_line(
                    side_units / float(np.mean(res["seconds"])), "1 (BLAS threads = 1)",
                    "one full macro step of the 313,646-DOF workload, single-threaded numpy/scipy", host)
                line["workload_313k"]["cpu_baseline"]["reduced"] = _reduced_baseline(
                    oracle["side_red"], ms_, ni_, side_idx, side_units)
                line["workload_313k"].setdefault("accuracy", {}).update(
                    _oracle_accuracy(ms_, args.precision, compare, local, np.load(os.path.join(tmp, "side.npy"))))
            except Exception as e:
                line["workload_313k"]["cpu_baseline"] = {"error": str(e)[:300]}
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world):
    """Batched workload: the 64 synthetic machines (uneven sizes) stepped
    concurrently through one sdc_batch, each on its own stream; one "step" is
    one macro step of every machine. Also times the same machines one after
    another (each alone) for the gain of batching."""
    import numpy as np
    import torch

    from paper_1707_03581_gb300 import Batch, Solver
    from synth import machine_config

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    machines = machine_config(3, truncate=args.machines)
    sc = machines[0].scheme
    n_int = sc.M - 1 if sc.nodes == "lobatto" else sc.M
    t_setup = time.perf_counter()
    solvers = []
    tuned = {}
    for mach in machines:
        s = Solver(local, own_stream=True)
        s.set_machine(mach, precision=args.precision)
        if not args.no_tune:
            rep = s.autotune(trial_steps=3)
            if not rep["cached"]:
                tuned[f"{s.n} DOF"] = rep
        solvers.append(s)
    t_setup = time.perf_counter() - t_setup
    dofs = np.array([s.n for s in solvers])
    units_per_step = int(dofs.sum()) * n_int * sc.P
    b = Batch(local)
    for s in solvers:
        b.add(s)

    def timed(run, k):
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        start.record(torch.cuda.current_stream(local))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(k)
        ends = []
        for s in solvers:
            e = torch.cuda.Event(enable_timing=True)
            e.record(s.stream)
            ends.append(e)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        return max(start.elapsed_time(e) for e in ends), wall

    b.step([args.warmup] * len(solvers), wait=True)
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        ms, wall = timed(lambda k: b.step([k] * len(solvers), wait=False), args.steps)
    b.synchronize()
    ms = _max_over_ranks(ms, world, f"cuda:{local}")

    def sequential(k):
        for s in solvers:
            s.run_horizon(k)

    ms_seq, _ = timed(sequential, args.steps)

    # the block-diagonal form: the qualifying members' FP32 CG fused into single launches
    fused = None
    if not args.no_fused:
        b.set_fused(True)
        n_fused = b.fused_size()
        b.step([args.warmup] * len(solvers), wait=True)
        ms_f, _ = timed(lambda k: b.step([k] * len(solvers), wait=False), args.steps)
        b.synchronize()
        b.set_fused(False)
        ms_f = _max_over_ranks(ms_f, world, f"cuda:{local}")
        fused = {"value": units_per_step * args.steps * world / (ms_f * 1e-3), "ms_per_step": ms_f / args.steps,
                 "members_fused": n_fused,
                 "note": "members with grids of at most 2048 blocks (r <= 48) fused: one SpMV and one update "
                         "launch per CG iteration over all of them; the r = 64 members keep their own graphs"}
    best = "fused" if fused is not None and fused["ms_per_step"] < ms / args.steps else "concurrent"
    if rank != 0:
        return
    ms_best = ms if best == "concurrent" else fused["ms_per_step"] * args.steps
    line = {
        "metric": METRIC, "value": units_per_step * args.steps * world / (ms_best * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_best / args.steps,
        "form": best,
        "concurrent": {"value": units_per_step * args.steps * world / (ms * 1e-3), "ms_per_step": ms / args.steps,
                       "note": "every member its own step graph on its own stream, enqueued round-robin"},
        "fused": fused,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"{len(machines)} machines r in {{16,24,32,48,64}} (stand r x r x 2.5r, stock "
                               f"half resolution), {int(dofs.sum())} DOF in total ({int(dofs.min())}-"
                               f"{int(dofs.max())} each), {sc.nodes} M={sc.M}, {sc.sweeps} sweeps, P={sc.P}, "
                               f"dt={sc.dt} s", "precision": args.precision,
                   "parallelism": f"one sdc_batch, {len(machines)} streams, replicas x{world}",
                   "l2": "working set of all machines far larger than L2"},
        "eta": args.steps * sc.dt / (ms_best * 1e-3),
        "sequential": {"value": units_per_step * args.steps / (ms_seq * 1e-3), "ms_per_step": ms_seq / args.steps,
                       "note": "the same machines stepped one after another"},
        "gain_vs_sequential": ms_seq / ms_best,
        "host_wall_ms_per_step": 1e3 * wall / args.steps,
        "setup_s": t_setup,
        "autotune": tuned or "off (--no-tune)",
        "clocks": clk.summary(),
    }
    b.close()
    if not args.no_cpu_baseline and world == 1:
        # as many machines as the host has cores, one oracle process each
        try:
            line["cpu_baseline"] = _oracle_pool(3, list(range(min(len(machines), os.cpu_count() or 1))))
        except Exception as e:
            line["cpu_baseline"] = {"error": str(e)[:300]}
    print(json.dumps(line), flush=True)
    for s in solvers:
        s.close()


def run_orders(args, rank, world):
    """The reduced problem of Sec. 4 (synth.slab_machine: a stand rectangle under a moving
    source of constant temperature) on the GPU, FP64: the measured order of MRSDC with
    k = 0..4 sweeps for (M, P) = (5, 8) and (5, 2) with the literal embedded weights,
    against a reference from 256 steps of (5, 8) with 8 sweeps, and the SDC residual of
    the first macro step after k sweeps for three step sizes. Theory: order
    min(M, P, k + 1); every sweep divides the residual by a factor proportional to dt."""
    import numpy as np
    import torch

    from paper_1707_03581_gb300 import Solver
    from synth.machines import Scheme, slab_machine

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    t_end = 2.0

    def slab(M, P, K, dt, cap=1e12):
        return slab_machine(4, 16, scheme=Scheme("equi_noleft", M, P, K, P, dt, 1e-14, 4000), rho=10.0, c=1000.0,
                            capacity_ratio=cap)

    def run(mach, T0, n, residuals=False):
        s = Solver(local)
        s.set_machine(mach, precision="fp64", T0=T0, residuals=residuals)
        reps = [s.step(report=True) for _ in range(n)]
        T = s.temperature()
        s.close()
        return T, reps

    t0 = time.perf_counter()
    mach, T0 = slab(5, 8, 8, t_end / 256)
    ref, _ = run(mach, T0, 256)
    nf = mach.stand.mesh.n_nodes

    def err(T):
        return float(np.linalg.norm(T[:nf] - ref[:nf]) / np.linalg.norm(ref[:nf] - T0[:nf]))

    steps = (2, 4, 8, 16, 32)
    orders, errors, ratio = {}, {}, []
    for M, P in ((5, 8), (5, 2)):
        key = f"({M},{P})"
        orders[key], errors[key] = [], []
        for k in range(5):
            e = [err(run(slab(M, P, k, t_end / n)[0], T0, n)[0]) for n in steps]
            ok = [i for i in range(len(steps) - 1) if e[i + 1] >= 1e-9]
            i = ok[-1] if ok else 0
            order = float(np.log2(e[i] / e[i + 1]))
            orders[key].append(order)
            errors[key].append(e)
            ratio.append(order / min(M, P, k + 1))
    residuals = {}
    for n in (5, 10, 20, 40):
        m, Tr = slab(5, 8, 4, t_end / n, cap=1e6)
        residuals[f"dt={t_end / n:g}"] = [float(r) for r in run(m, Tr, 1, residuals=True)[1][0]["residual"]]
    wall = time.perf_counter() - t0
    if rank != 0:
        return
    line = {
        "metric": "measured order / min(M, P, k+1), MRSDC on the reduced problem of Sec. 4 (worst case)",
        "value": min(ratio), "unit": "ratio", "n_gpus": world, "steps": None, "warmup": 0, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"slab 1x4x16 hexes ({mach.n_dof} DOF) under a 100 degC source moving along its "
                               f"top edge, equidistant nodes without the left end point, literal embedded weights, "
                               f"t_end = {t_end} s",
                   "orders_from": "the smallest pair of step sizes whose errors stay above 1e-9"},
        "orders": orders, "expected": {"(5,8)": [1, 2, 3, 4, 5], "(5,2)": [1, 2, 2, 2, 2]},
        "errors_at_t_end": {"steps": list(steps), **errors},
        "residual_after_k_sweeps": residuals,
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def run_serving(args, rank, world):
    """Serving workload: Poisson arrivals (rate --lam) of look-ahead requests, each a
    machine of the 64-machine pool with horizon ~ U(30, 600) s from its resident
    state; continuous batching on one GPU. Mixed precision and plain FP64 serve
    the same request list; reports latency percentiles, per-request look-ahead
    factors and aggregate throughput."""
    import torch

    from paper_1707_03581_gb300.serving import LookAheadServer, Request, summarize
    from synth import machine_config
    from synth.machines import serving_requests

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    machines = machine_config(3)
    sched = serving_requests(args.lam, n_requests=args.requests, seed=0, pool=len(machines))
    out = {}
    precs = (args.precision,) if args.no_compare else ("mixed", "fp64")
    for prec in precs:
        server = LookAheadServer(machines, device=local, precision=prec, max_active=args.max_active)
        reqs = [Request(r["arrival_s"], round(r["horizon_s"]), r["machine_index"]) for r in sched]
        if world > 1:
            torch.distributed.barrier()
        with ClockSampler(local) as clk:
            server.run(reqs)
        n_dof = [m.n_dof for m in machines]
        st = summarize(reqs, machines, n_dof)
        st["slots"] = server.slots_made
        st["footprint_gb"] = server.footprint / 1e9
        st["clocks"] = clk.summary()
        # whole job: every rank serves the same request list, so the job's rate is the units
        # of all ranks over the slowest rank's makespan
        units = st["dof_substeps_per_s"] * st["makespan_s"]
        sim_s = st["simulated_s_per_s"] * st["makespan_s"]
        st["makespan_s"] = _max_over_ranks(st["makespan_s"], world, f"cuda:{local}")
        st["dof_substeps_per_s"] = _whole_job_rate(units, st["makespan_s"], world)
        st["simulated_s_per_s"] = _whole_job_rate(sim_s, st["makespan_s"], world)
        out[prec] = st
        server.close()
    if rank != 0:
        return
    # the line's own figures are those of the first precision served (mixed unless only FP64 ran)
    mx = out[precs[0]]
    f64 = out.get("fp64") if len(precs) == 2 else None
    line = {
        "metric": METRIC, "value": mx["dof_substeps_per_s"], "unit": UNIT, "n_gpus": world,
        "steps": sum(round(r["horizon_s"]) for r in sched), "warmup": 0,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if precs[0] == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"serving: {args.requests} Poisson arrivals at {args.lam}/s of look-ahead requests "
                               f"(horizon ~ U(30,600) s rounded to whole macro steps) on a pool of 64 machines "
                               f"(12.9k-734k DOF), warm-start state kept on the device",
                   "precision": "mixed vs fp64, same requests" if f64 else precs[0],
                   "parallelism": f"continuous batching, up to "
                   f"{args.max_active} requests in flight, replicas x{world}"},
        "latency_s": mx["latency_s"], "eta_per_request": mx["eta_per_request"],
        "offered_simulated_s_per_s": args.lam * world * sum(round(r["horizon_s"]) for r in sched) / len(sched),
        "served_simulated_s_per_s": mx["simulated_s_per_s"],
        **{p: out[p] for p in precs},
        "gain_vs_fp64": {"throughput": mx["dof_substeps_per_s"] / f64["dof_substeps_per_s"],
                         "p99_latency": f64["latency_s"]["p99"] / mx["latency_s"]["p99"],
                         "p50_latency": f64["latency_s"]["p50"] / mx["latency_s"]["p50"]} if f64 else None,
    }
    if not args.no_cpu_baseline and world == 1:
        # the serving pool's machines on the host cores, one oracle process each
        try:
            line["cpu_baseline"] = _oracle_pool(3, list(range(min(len(machines), os.cpu_count() or 1))))
        except Exception as e:
            line["cpu_baseline"] = {"error": str(e)[:300]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP64 comparison run of the mixed path (config 4: serve the requests in "
                         "--precision only)")
    ap.add_argument("--config", type=int, default=2,
                    help="0/1/2: one machine (2 = the headline workload, the largest single-GPU one); "
                         "3: the batch of 64 machines; "
                         "4: serving (Poisson arrivals); 5: convergence order and residual decay on the "
                         "reduced problem of Sec. 4")
    ap.add_argument("--machines", type=int, default=None, help="config 3: use only the first machines")
    ap.add_argument("--member", type=int, default=None,
                    help="config 3: time batch machine i alone, as a single-machine workload")
    ap.add_argument("--lam", type=float, default=10.0, help="config 4: arrival rate [requests/s]")
    ap.add_argument("--requests", type=int, default=32, help="config 4: number of requests")
    ap.add_argument("--max-active", type=int, default=64, help="config 4: requests in flight at most")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--contact-replicas", type=int, default=None, choices=[0, 1, 2, 3],
                    help="placement of the contact loop's replicas (sdc_set_contact_replicas); "
                         "default automatic")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch options (no sdc_autotune before timing)")
    ap.add_argument("--no-fused", action="store_true", help="config 3: skip the fused (block-diagonal) form")
    ap.add_argument("--no-extra", action="store_true",
                    help="config 2: skip the 313,646-DOF workload measured beside the headline")
    ap.add_argument("--no-single-rate", action="store_true",
                    help="skip the single-rate SDC comparison (Sec. 3) on the same machine")
    ap.add_argument("--no-ie", action="store_true",
                    help="skip the comparison with fully implicit Euler (work against accuracy)")
    ap.add_argument("--no-stationary", action="store_true",
                    help="skip the stationary-start measurement (Sec. 5 initial state)")
    ap.add_argument("--eager", action="store_true",
                    help="plain kernel launches with host-driven CG loops (for kernel-level profilers)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch

            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.config == 3 and args.member is None:
        run_batch(args, rank, world)
    elif args.config == 4:
        run_serving(args, rank, world)
    elif args.config == 5:
        run_orders(args, rank, world)
    else:
        run_gpu(args, rank, world)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
