"""Look-ahead serving on one GPU: continuous batching of forecast requests.

A request asks for the temperature field of one machine of a resident pool a
horizon ahead (the look-ahead of Sec. 1: simulated time faster than real
time). It starts from that machine's current state, which the server keeps on
the device (warm start), and runs horizon / dt macro steps of the machine's
scheme. The forecast does not change the resident state.

Scheduling (host loop over the C ABI; all simulation work runs in the
library's CUDA graphs):
  * requests are admitted in arrival order as soon as a slot is free: a
    context assembled for the request's machine, created on demand while
    the device bytes of all slots stay within the HBM budget, and reused
    once its request has finished. A slot's bytes are estimated before it
    is made (measured for a machine that had one, else scaled by DOF count
    from the slots made so far) and measured after; a new slot that leaves
    the total over the budget is closed again and its request waits for
    active slots to finish. To make room, idle slots of other machines are
    closed, least recently used first; a request that cannot fit even with
    every other slot idle and closed is an error;
  * every admitted request runs on its own stream; whenever that stream is
    idle the loop enqueues the next few macro steps, so requests that
    arrive while others run join the device work at once and their kernels
    overlap;
  * a request ends when its result is on the host ("done"). A request can be
    cancelled (Request.cancel_at_s, or LookAheadServer.cancel): it leaves the
    queue, or, once admitted, leaves between two enqueued batches of steps,
    with none of its steps in flight, and its slot is reused ("cancelled"). A
    request whose slot cannot be made (device memory, assembly) fails alone
    ("failed", with the error), and the others go on.

Each slot holds its own state and every reduction has a fixed order, so a
request's result equals the same forecast run alone.
"""

from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Request:
    arrival_s: float
    horizon_s: float
    machine_index: int
    # the client's cancellation time (relative to the start of the run), if any
    cancel_at_s: Optional[float] = None
    # filled by the server
    n_steps: int = 0
    status: str = "pending"  # then "done", "cancelled" or "failed"
    error: Optional[str] = None
    t_admit: Optional[float] = None
    t_done: Optional[float] = None
    result: Optional[np.ndarray] = field(default=None, repr=False)
    cancel_requested: bool = False

    def cancelled_by(self, now: float) -> bool:
        return self.cancel_requested or (self.cancel_at_s is not None and now >= self.cancel_at_s)

    @property
    def latency_s(self) -> float:
        return self.t_done - self.arrival_s

    @property
    def eta(self) -> float:
        """Look-ahead factor of this request: simulated seconds per second of latency."""
        return self.horizon_s / self.latency_s


class LookAheadServer:
    """Continuous-batching server over a pool of machines (synth.Machine inputs)."""

    def __init__(self, machines, device: int = 0, precision: str = "mixed",
                 hbm_budget_bytes: Optional[int] = None, max_active: int = 64, chunk: int = 4,
                 keep_results: bool = False):
        import torch

        self.torch = torch
        self.machines = list(machines)
        self.device = device
        self.precision = precision
        self.max_active = max_active
        self.chunk = chunk
        self.keep_results = keep_results
        if hbm_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget_bytes = int(0.8 * free)
        self.budget = hbm_budget_bytes
        self.footprint = 0
        self.peak_footprint = 0
        self.slots_made = 0
        self.free_slots = {i: [] for i in range(len(self.machines))}
        self.idle = deque()  # (machine index, slot) in the order the slots became idle
        self.slot_bytes = {}
        # resident warm-start states (device, FP64), initially each machine's uniform T0
        self.state = [None] * len(self.machines)

    # ------------------------------------------------------------------ state
    def set_state(self, i: int, T):
        """Replace machine i's resident state (host array or CUDA tensor of n_dof doubles)."""
        t = self.torch.as_tensor(np.asarray(T) if not self.torch.is_tensor(T) else T, dtype=self.torch.float64)
        self.state[i] = t.to(f"cuda:{self.device}").contiguous()

    def _release(self, i: int, slot):
        self.free_slots[i].append(slot)
        self.idle.append((i, slot))

    def _evict_one(self, keep: int) -> bool:
        """Close the least recently used idle slot of a machine other than `keep`."""
        for n, (j, slot) in enumerate(self.idle):
            if j != keep:
                del self.idle[n]
                self.free_slots[j].remove(slot)
                slot.close()
                self.footprint -= self.slot_bytes[j]
                return True
        return False

    def _estimate(self, i: int) -> int:
        """Device bytes of a slot of machine i: measured once one was made, else scaled
        from the slots made so far by DOF count (0 before the first slot of any machine)."""
        if i in self.slot_bytes:
            return self.slot_bytes[i]
        known = [(self.slot_bytes[j], self.machines[j].n_dof) for j in self.slot_bytes]
        if not known:
            return 0
        per_dof = max(b / max(n, 1) for b, n in known)
        return int(per_dof * self.machines[i].n_dof)

    def _slot(self, i: int):
        if self.free_slots[i]:
            slot = self.free_slots[i].pop()
            self.idle.remove((i, slot))
            return slot
        est = self._estimate(i)
        while self.footprint + est > self.budget and self._evict_one(i):
            pass
        if self.footprint + est > self.budget:
            return None
        from .binding import Solver

        s = Solver(self.device, own_stream=True)
        try:
            s.set_machine(self.machines[i], precision=self.precision)
            # slots overlap one another; a slot's own graph runs as one chain
            s.set_graph_branches(False)
            b = s.footprint()
        except Exception:
            s.close()
            raise
        self.slot_bytes[i] = b
        self.footprint += b
        # the estimate can be short: back under the budget if idle slots allow, else the new
        # slot is closed again and the request waits for active slots to finish
        while self.footprint > self.budget and self._evict_one(i):
            pass
        if self.footprint > self.budget:
            s.close()
            self.footprint -= b
            return None
        self.slots_made += 1
        self.peak_footprint = max(self.peak_footprint, self.footprint)
        if self.state[i] is None:
            self.set_state(i, np.full(s.n, self.machines[i].T0))
        return s

    def cancel(self, request: Request):
        """Ask the running loop to drop `request` (queued, or between its batches of steps)."""
        request.cancel_requested = True

    def close(self):
        for lst in self.free_slots.values():
            for s in lst:
                s.close()
            lst.clear()
        self.idle.clear()

    # ------------------------------------------------------------------ serving
    def run(self, requests: List[Request], clock=time.perf_counter) -> List[Request]:
        """Serve `requests` (arrival times relative to the start of the call); returns them
        with admission and completion times filled in."""
        for r in requests:
            r.n_steps = int(round(r.horizon_s / self.machines[r.machine_index].scheme.dt))
        pending = deque(sorted(requests, key=lambda r: r.arrival_s))
        waiting: List[Request] = []
        active = []  # [request, slot, steps not yet enqueued]
        t0 = clock()
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0].arrival_s <= now:
                waiting.append(pending.popleft())
            for r in [r for r in waiting if r.cancelled_by(now)]:
                waiting.remove(r)
                r.status, r.t_done = "cancelled", now
            i = 0
            while i < len(waiting) and len(active) < self.max_active:
                r = waiting[i]
                try:
                    slot = self._slot(r.machine_index)
                    if slot is None and not active:  # nothing running will free device memory
                        raise RuntimeError(f"machine {r.machine_index} does not fit the HBM budget "
                                           f"({self.budget} bytes) even with every other slot closed")
                except Exception as e:  # this request fails alone; the others go on
                    del waiting[i]
                    r.status, r.error, r.t_done = "failed", str(e), clock() - t0
                    continue
                if slot is None:
                    i += 1
                    continue
                del waiting[i]
                m = self.machines[r.machine_index]
                slot.set_temperature(self.state[r.machine_index], t0=m.t0)
                r.t_admit = clock() - t0
                active.append([r, slot, r.n_steps])
            progressed = False
            for a in list(active):
                r, slot, left = a
                if not slot.poll():
                    continue
                if r.cancelled_by(clock() - t0):  # between batches: none of its steps in flight
                    active.remove(a)
                    self._release(r.machine_index, slot)
                    r.status, r.t_done = "cancelled", clock() - t0
                    progressed = True
                    continue
                if left > 0:
                    k = min(self.chunk, left)
                    slot.step_async(k)
                    a[2] -= k
                else:
                    slot.synchronize()  # surfaces device errors of the request's steps
                    T = slot.temperature()
                    r.t_done = clock() - t0
                    r.status = "done"
                    if self.keep_results:
                        r.result = T
                    active.remove(a)
                    self._release(r.machine_index, slot)
                progressed = True
            if not progressed:
                if not active and not waiting and pending:
                    time.sleep(max(0.0, min(pending[0].arrival_s - (clock() - t0), 0.01)))
                else:
                    time.sleep(20e-6)
        return requests


def summarize(requests: List[Request], machines, n_dof) -> dict:
    """Latency percentiles, per-request look-ahead factors and aggregate throughput of the
    requests served to the end; cancelled and failed ones are counted apart."""
    counts = {"cancelled": sum(r.status == "cancelled" for r in requests),
              "failed": sum(r.status == "failed" for r in requests)}
    requests = [r for r in requests if r.status == "done"]
    if not requests:
        return {"requests": 0, **counts}
    lat = np.array([r.latency_s for r in requests])
    eta = np.array([r.eta for r in requests])
    span = max(r.t_done for r in requests) - min(r.arrival_s for r in requests)
    units = 0.0
    for r in requests:
        sc = machines[r.machine_index].scheme
        n_int = sc.M - 1 if sc.nodes == "lobatto" else sc.M
        units += n_dof[r.machine_index] * r.n_steps * n_int * sc.P
    return {
        "requests": len(requests),
        **counts,
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max())},
        "eta_per_request": {"p50": float(np.percentile(eta, 50)), "p1": float(np.percentile(eta, 1)),
                            "min": float(eta.min())},
        "makespan_s": float(span),
        "dof_substeps_per_s": units / span,
        "simulated_s_per_s": float(sum(r.horizon_s for r in requests) / span),
    }
