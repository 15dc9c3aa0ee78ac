"""Continuous-batching request loop over the batched C-ABI (lbm_batch_*).

Requests (cavity, duct or pulsatile solves of different sizes) arrive over
time.  The server admits them in arrival order while a slot and the memory
budget allow, keeps their populations resident on the device, advances every
admitted domain together in chunks of ``check_every`` steps (one batched
launch per chunk), and after each chunk runs the FP64 reductions of all
domains at once.  A domain retires when its residual (the all-component form
over the last chunk) reaches ``tol`` or it reaches its step cap; its slot and
memory go to the next waiting request.  With ``max_active_cells`` set, a new
request is admitted only while the admitted domains hold fewer cells than
that (enough to saturate the device), so large requests run nearly in
arrival order while small ones share the device.  Time-to-converged is measured from
arrival to retirement, so queueing is included.

Because every domain has its own step counter and checks fall at the same
multiples of ``check_every`` of its own counter however the batch is mixed,
a request's result does not depend on what else is running.

``SequentialBackend`` serves the same trace one domain at a time, the
baseline the batched server is compared with.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from . import inputs, lbm


class Busy(Exception):
    """No slot or memory for another domain right now."""


@dataclasses.dataclass
class Outcome:
    rid: int
    arrival: float
    admitted: float = -1.0
    done: float = -1.0
    steps: int = 0
    residual: Optional[float] = None
    cells: int = 0
    storage: str = ""
    fingerprint: tuple = ()
    u: Optional[np.ndarray] = None  # final velocity field (Server(keep_fields=True))

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def fingerprint(stats) -> tuple:
    return (stats.step, tuple(stats.sum_abs_u), tuple(stats.sum_u), stats.sum_P, stats.max_abs_u)


class BatchBackend:
    """All admitted domains in one lbm_batch."""

    def __init__(self, capacity: int, budget_bytes: int, stream, launch=(64, 2, 0)):
        self.capacity = capacity
        self.b = lbm.lbm_batch_create(capacity, budget_bytes, stream)
        lbm.lbm_batch_set_launch(self.b, *launch)

    def add(self, case: inputs.Case) -> int:
        try:
            slot = lbm.lbm_batch_add(self.b, case.Q, case.nx, case.ny, case.nz, case.storage,
                                     case.faces, case.u_wall, edge=case.edge, nu=case.nu,
                                     force=case.force,
                                     force_period=case.period, rounding=case.rounding)
        except lbm.LBMError as e:
            if e.code == lbm.LBM_EBUSY:
                raise Busy() from e
            raise
        lbm.lbm_batch_init_equilibrium(self.b, slot)
        return slot

    def remove(self, slot: int) -> None:
        lbm.lbm_batch_remove(self.b, slot)

    def step(self, nsteps: int, chunk: int) -> None:
        lbm.lbm_batch_step(self.b, nsteps, chunk)

    def reductions(self) -> Dict[int, object]:
        return lbm.lbm_batch_reductions_all(self.b, self.capacity)

    def residual(self, slot: int) -> float:
        """Eq. cavity_creterion of the slot's last reduction (library call)."""
        return lbm.lbm_batch_residual(self.b, slot, lbm.LBM_RESIDUAL_CAVITY)

    def read_u(self, slot: int, case: inputs.Case) -> np.ndarray:
        import torch
        out = torch.empty(3 * case.cells, dtype=torch.float64, device="cuda")
        lbm.lbm_batch_read_fields(self.b, slot, lbm.LBM_FIELD_U, out)
        return out.cpu().numpy().reshape(3, case.nz, case.ny, case.nx)

    def close(self) -> None:
        lbm.lbm_batch_destroy(self.b)


class SequentialBackend:
    """One domain at a time, one single-domain handle per request."""

    def __init__(self, stream, launch=(64, 2, 1)):
        self.stream = stream
        self.launch = launch
        self.h = None
        self.capacity = 1

    def add(self, case: inputs.Case) -> int:
        if self.h is not None:
            raise Busy()
        h = lbm.lbm_create(case.Q, case.nx, case.ny, case.nz, case.storage, self.stream)
        lbm.lbm_set_geometry(h, case.faces, case.u_wall, case.edge)
        lbm.lbm_set_params(h, nu=case.nu, force=case.force, force_period=case.period,
                           rounding=case.rounding)
        lbm.lbm_set_launch(h, *self.launch)
        lbm.lbm_init_equilibrium(h)
        self.h = h
        return 0

    def remove(self, slot: int) -> None:
        lbm.lbm_destroy(self.h)
        self.h = None

    def step(self, nsteps: int, chunk: int) -> None:
        if self.h is not None:
            lbm.lbm_step(self.h, nsteps)

    def reductions(self) -> Dict[int, object]:
        return {} if self.h is None else {0: lbm.lbm_reductions(self.h)}

    def residual(self, slot: int) -> float:
        return lbm.lbm_residual(self.h, lbm.LBM_RESIDUAL_CAVITY)

    def read_u(self, slot: int, case: inputs.Case) -> np.ndarray:
        return lbm.read_u(self.h, case.nx, case.ny, case.nz)

    def close(self) -> None:
        if self.h is not None:
            lbm.lbm_destroy(self.h)
            self.h = None


class Server:
    def __init__(self, backend, check_every: int = 100, tol: float = 1e-8, chunk: int = 50,
                 max_active_cells: int = 0,
                 case_of: Callable = inputs.request_case,
                 clock: Callable[[], float] = time.perf_counter,
                 sleep: Callable[[float], None] = time.sleep,
                 keep_fields: bool = False):
        self.backend = backend
        self.keep_fields = keep_fields
        self.check_every = check_every
        self.tol = tol
        self.max_active_cells = max_active_cells
        self.chunk = chunk
        self.case_of = case_of
        self.clock = clock
        self.sleep = sleep

    def run(self, trace: List[inputs.Request]) -> Dict[int, Outcome]:
        out = {r.rid: Outcome(r.rid, r.arrival) for r in trace}
        pending = collections.deque(sorted(trace, key=lambda r: r.arrival))
        waiting: collections.deque = collections.deque()
        active: Dict[int, tuple] = {}  # slot -> (request, case)
        t0 = self.clock()
        while pending or waiting or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            while waiting:  # admit in arrival order while resources allow
                r = waiting[0]
                case = self.case_of(r)
                if (self.max_active_cells and active and
                        sum(c.cells for _, c in active.values()) + case.cells
                        > self.max_active_cells):
                    break  # the device is already saturated
                try:
                    slot = self.backend.add(case)
                except Busy:
                    break
                waiting.popleft()
                active[slot] = (r, case)
                out[r.rid].admitted = self.clock() - t0
                out[r.rid].cells = case.cells
                out[r.rid].storage = case.storage
            if not active:
                if pending:
                    self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                continue
            self.backend.step(self.check_every, self.chunk)
            stats = self.backend.reductions()
            for slot, (r, case) in list(active.items()):
                o = out[r.rid]
                o.steps += self.check_every
                st = stats[slot]
                # Eq. cavity_creterion over the last interval; none before the
                # second check of a request (no earlier snapshot yet)
                res = self.backend.residual(slot) if st.prev_step >= 0 else None
                o.residual = res
                if st.nonfinite or (res is not None and res <= self.tol) or o.steps >= r.max_steps:
                    o.done = self.clock() - t0
                    o.fingerprint = fingerprint(st)
                    if self.keep_fields:
                        o.u = self.backend.read_u(slot, case)
                    self.backend.remove(slot)
                    del active[slot]
        return out


def summarize(outcomes: Dict[int, Outcome], wall: float) -> dict:
    lat = np.array([o.latency for o in outcomes.values()])
    updates = sum(o.cells * o.steps for o in outcomes.values())
    return {"requests": len(outcomes),
            "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()),
            "glups": updates / wall / 1e9,
            "lattice_updates": int(updates),
            "wall_s": wall,
            "converged": sum(1 for o in outcomes.values()
                             if o.residual is not None and o.residual <= 1e-8)}
