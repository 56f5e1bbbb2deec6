"""Continuous-batching server for expansion runs.

Requests (N, w, dt, softening, steps, initial positions) arrive over time.  The server
admits a request as soon as its device footprint fits the memory budget (first come,
first served, with optional backfill of later requests that fit while the head of the
queue waits), keeps every admitted bunch resident in one batch context, and advances all
of them together in step blocks of one persistent kernel launch per time step.  A
request leaves at the end of the block in which its step count is reached; its result
(final positions, velocities, accelerations and moments) is copied out and its memory
returns to the budget, so waiting requests join at the next block.

Latency of a request = completion time - arrival time (queueing included).
Throughput = pair interactions of all steps run / wall time of the run.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np

from . import capi


@dataclasses.dataclass
class ServeRequest:
    rid: int
    arrival: float                 # seconds after the start of the run
    n: int
    w: float
    dt: float
    softening: float
    steps: int
    positions: np.ndarray          # [n][3] m
    velocities: np.ndarray | None = None


@dataclasses.dataclass
class ServeResult:
    rid: int
    n: int
    steps: int
    arrival: float
    admitted: float
    completed: float
    positions: np.ndarray
    velocities: np.ndarray
    accelerations: np.ndarray
    diagnostics: dict

    @property
    def latency(self) -> float:
        return self.completed - self.arrival

    @property
    def queueing(self) -> float:
        return self.admitted - self.arrival


def percentile(values, q):
    """Nearest-rank percentile (q in [0, 100]) of a non-empty sequence."""
    v = sorted(values)
    k = max(0, min(len(v) - 1, math.ceil(q / 100.0 * len(v)) - 1))
    return v[k]


class Server:
    def __init__(self, budget_bytes: int, block_steps: int = 16, backfill: bool = True,
                 clock=time.perf_counter, sleep=time.sleep):
        self.batch = capi.Batch(budget_bytes, graph_block=block_steps if block_steps % 2 == 0 else 0)
        self.budget = int(budget_bytes)
        self.block_steps = int(block_steps)
        self.backfill = backfill
        self.clock = clock
        self.sleep = sleep
        self.pending: collections.deque[ServeRequest] = collections.deque()
        self.active: dict[int, dict] = {}
        self.results: list[ServeResult] = []
        self.rejected: list[int] = []
        self.cancelled: list[int] = []
        self._cancel: set[int] = set()
        self.pairs = 0.0
        self.blocks = 0

    def close(self):
        self.batch.close()

    def cancel(self, rid: int):
        """Cancel a request: dropped if it waits, removed (memory freed) at the next block
        boundary if it runs.  Unknown or finished ids are ignored."""
        self._cancel.add(rid)

    def _apply_cancellations(self):
        if not self._cancel:
            return
        kept = collections.deque()
        for r in self.pending:
            if r.rid in self._cancel:
                self.cancelled.append(r.rid)
                self._cancel.discard(r.rid)
            else:
                kept.append(r)
        self.pending = kept
        for slot in [s for s, a in self.active.items() if a["req"].rid in self._cancel]:
            a = self.active.pop(slot)
            self.batch.remove(slot)
            self.cancelled.append(a["req"].rid)
            self._cancel.discard(a["req"].rid)
        # ids not seen yet stay marked: they are dropped when they arrive

    def _free(self) -> int:
        return self.budget - self.batch.info()["bytes_used"]

    def _admit(self, now: float):
        """Admit waiting requests that fit, in arrival order (later ones may backfill)."""
        kept = collections.deque()
        blocked = False
        while self.pending:
            r = self.pending.popleft()
            need = capi.pp_batch_footprint(r.n)
            if need > self.budget:
                self.rejected.append(r.rid)          # can never fit
                continue
            if (blocked and not self.backfill) or need > self._free():
                blocked = True
                kept.append(r)
                continue
            slot = self.batch.add(r.positions, r.w, r.dt, r.softening, r.velocities)
            self.active[slot] = {"req": r, "left": r.steps, "admitted": now}
        self.pending = kept

    def _retire(self, now: float):
        for slot in [s for s, a in self.active.items() if a["left"] == 0]:
            a = self.active.pop(slot)
            r = a["req"]
            pos, vel, acc, step = self.batch.state(slot, r.n)
            diag = self.batch.diagnostics(slot)
            self.batch.remove(slot)
            self.results.append(ServeResult(r.rid, r.n, step, r.arrival, a["admitted"],
                                            self.clock() - self.t0, pos, vel, acc, diag))

    def run(self, requests: list[ServeRequest], on_block=None) -> dict:
        """Serve a trace to completion; returns the latency/throughput report.

        on_block(server), if given, is called after every step block (for example to
        cancel requests)."""
        arrivals = collections.deque(sorted(requests, key=lambda r: r.arrival))
        self.t0 = self.clock()
        while arrivals or self.pending or self.active:
            now = self.clock() - self.t0
            while arrivals and arrivals[0].arrival <= now:
                r = arrivals.popleft()
                if r.rid in self._cancel:
                    self.cancelled.append(r.rid)
                    self._cancel.discard(r.rid)
                    continue
                self.pending.append(r)
            self._apply_cancellations()
            self._admit(now)
            # requests that reached zero steps (steps = 0) finish at once
            self._retire(now)
            if not self.active:
                if arrivals:
                    self.sleep(max(0.0, arrivals[0].arrival - (self.clock() - self.t0)))
                elif self.pending:
                    break                               # nothing can ever be admitted
                continue
            block = min(self.block_steps, min(a["left"] for a in self.active.values()))
            self.batch.step(block)
            self.blocks += 1
            for a in self.active.values():
                a["left"] -= block
                self.pairs += float(a["req"].n) ** 2 * block
            self._retire(self.clock() - self.t0)
            if on_block is not None:
                on_block(self)
        wall = self.clock() - self.t0
        lat = [r.latency for r in self.results]
        rep = {"requests": len(requests), "completed": len(self.results),
               "rejected": len(self.rejected), "cancelled": len(self.cancelled),
               "wall_s": wall, "blocks": self.blocks,
               "pairs": self.pairs, "pairs_per_s": self.pairs / wall if wall > 0 else float("nan")}
        if lat:
            rep.update({"p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
                        "max_latency_s": max(lat),
                        "mean_queueing_s": float(np.mean([r.queueing for r in self.results]))})
        return rep


def requests_from_trace(trace, n_scale: float = 1.0, steps_scale: float = 1.0,
                        n_max: int | None = None) -> list[ServeRequest]:
    """Turn workloads.serve_trace() items into requests, optionally scaled down (N and
    step counts multiplied by the given factors, N capped at n_max) to bound run time."""
    out = []
    for req in trace:
        b = req.bunch
        n = max(2, int(round(b.n * n_scale)))
        if n_max is not None:
            n = min(n, n_max)
        steps = max(1, int(round(b.steps * steps_scale)))
        from .workloads import uniform_sphere
        pos = uniform_sphere(n, b.scale, b.seed)
        out.append(ServeRequest(req.rid, req.arrival, n, b.w, b.dt, b.eps, steps, pos))
    return out
