"""Serving many independent D2V16 problems on one GPU: continuous batching.

Requests (``workloads.RequestSpec``) arrive over time.  The server

* admits them in arrival order while the device memory they need (two state
  buffers and the scratch buffer, exactly as ``dbm_state_bytes`` and
  ``dbm_scratch_bytes`` report) fits in the HBM budget; a request that does
  not fit waits at the head of the queue, so admission is first come, first
  served;
* keeps every admitted state resident on the device until the request is
  done (its initial fields are built on the device, no host copy of a state
  is ever made);
* groups the running requests by species count, one CUDA stream per group:
  S <= 4 are stepped together as one ``Batch`` (one launch per step and chunk
  of instances), larger S one instance after the other on the group stream;
* advances a group in quanta: all members by q = min(quantum, smallest
  number of steps a member still needs), so every request gets exactly its
  own step count; between quanta finished members leave, newly admitted
  ones join, and the batch is rebuilt for the new membership;
* finishes a request by reading its conserved totals (and optionally its
  final state) into pinned host memory; the request's latency runs from its
  arrival to the moment that copy has completed;
* withdraws a request at its ``cancel_at`` time: a waiting one at once, a
  running one at its group's next quantum boundary, when none of its work
  is in flight, releasing its memory.

``run_sequential`` is the baseline: the same requests solved first come,
first served, one at a time, in FP64 or FP32.

Every batch of a group uses the same kernel configuration (tile shape,
launch form, L2 promotion), so a request's result does not depend on which
other requests it was served with.

The queueing decisions (``Admission``, ``quantum``) are plain Python and
need no GPU; ``Server.run`` drives the CUDA library through ``dbm``.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

from . import dbm as D
from . import workloads as W

# kernel configuration of the batched groups (tile shape, launch form, L2
# promotion): what the tuner picks for the 64-instance mix of sides 64 to
# 512, and the fastest shape measured on instances of 256^2 to 4096^2
DEFAULT_CONFIG = {"tile": (64, 4), "cells": 1, "persistent": 0, "promote": 1}


class Admission:
    """HBM-footprint admission: the bytes of the admitted requests never
    exceed the budget."""

    def __init__(self, budget: int):
        self.budget = int(budget)
        self.used = 0
        self.peak = 0

    def fits(self, nbytes: int) -> bool:
        return self.used + nbytes <= self.budget

    def admit(self, nbytes: int) -> None:
        assert self.fits(nbytes)
        self.used += nbytes
        self.peak = max(self.peak, self.used)

    def release(self, nbytes: int) -> None:
        self.used -= nbytes
        assert self.used >= 0


def quantum(remaining: List[int], qmax: int) -> int:
    """Steps of the next quantum of a group: no member is stepped past its
    own step count."""
    return max(1, min(min(remaining), qmax))


def footprint(problem, precision: str = "fp32") -> int:
    """Device bytes a request holds while it is served."""
    h = D.dbm_init(D.params_from_problem(problem, precision))
    try:
        return 2 * D.dbm_state_bytes(h) + D.dbm_scratch_bytes(h)
    finally:
        D.dbm_destroy(h)


@dataclass
class Result:
    rid: int
    ns: int
    cells: int
    nsteps: int
    arrival: float
    admitted: float
    finished: float
    status: int
    conservation: np.ndarray
    f: Optional[np.ndarray] = None
    cancelled: bool = False  # withdrawn before it finished (no result state)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def units(self) -> int:
        return self.cells * self.ns * self.nsteps


@dataclass
class _Active:
    spec: W.RequestSpec
    solver: "D.Solver"
    nbytes: int
    admitted: float
    remaining: int
    cancelled: bool = False


@dataclass
class _Done:
    active: _Active
    stream: object
    event: object
    cons: object  # pinned host tensor
    f: object = None


@dataclass
class _Group:
    ns: int
    stream: object
    members: List[_Active] = field(default_factory=list)
    incoming: List[_Active] = field(default_factory=list)
    batch: object = None
    event: object = None
    busy: bool = False
    quantum_steps: int = 0
    rebuilds: int = 0


class Server:
    """Continuous-batching server on one device (see the module docstring)."""

    def __init__(self, device="cuda", hbm_budget: Optional[int] = None, qmax: int = 128,
                 config: Optional[dict] = None, keep_f: bool = False, max_batch_ns: int = 4):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(0.8 * free)
        self.adm = Admission(hbm_budget)
        self.qmax = int(qmax)
        self.config = dict(DEFAULT_CONFIG if config is None else config)
        self.keep_f = keep_f
        self.max_batch_ns = max_batch_ns
        self.groups: Dict[int, _Group] = {}
        self.launch_quanta = 0

    # -- groups ---------------------------------------------------------

    def _group(self, ns: int) -> _Group:
        g = self.groups.get(ns)
        if g is None:
            g = _Group(ns=ns, stream=self.torch.cuda.Stream(device=self.device))
            self.groups[ns] = g
        return g

    def _start(self, spec: W.RequestSpec, nbytes: int, now: float) -> None:
        torch = self.torch
        g = self._group(spec.ns)
        pb = W.request_problem(spec)
        with torch.cuda.stream(g.stream):
            s = D.Solver(pb, "fp32", device=self.device)
            s.set_state(*W.request_fields(spec, self.device))
        g.incoming.append(_Active(spec=spec, solver=s, nbytes=nbytes, admitted=now, remaining=spec.nsteps))

    def _finish(self, g: _Group, a: _Active) -> _Done:
        torch = self.torch
        with torch.cuda.stream(g.stream):
            cons = a.solver.conservation()
            host = torch.empty(cons.shape, dtype=cons.dtype, pin_memory=True)
            host.copy_(cons, non_blocking=True)
            fh = None
            if self.keep_f:
                f = a.solver.get_f()
                fh = torch.empty(f.shape, dtype=f.dtype, pin_memory=True)
                fh.copy_(f, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(g.stream)
        return _Done(active=a, stream=g.stream, event=ev, cons=host, f=fh)

    def _advance(self, g: _Group, done: List[_Done], dropped: List[_Active]) -> None:
        """Between quanta (no work of the group in flight): retire finished
        and cancelled members, take in new ones, launch the next quantum."""
        torch = self.torch
        changed = bool(g.incoming)
        keep = []
        for a in g.members + g.incoming:
            if a.cancelled:
                dropped.append(a)
                changed = True
            elif a.remaining == 0:
                done.append(self._finish(g, a))
                changed = True
            else:
                keep.append(a)
        g.members = keep
        g.incoming = []
        if not g.members:
            if g.batch is not None:
                g.batch.close()
                g.batch = None
            return
        batched = g.ns <= self.max_batch_ns
        with torch.cuda.stream(g.stream):
            if batched and (changed or g.batch is None):
                if g.batch is not None:
                    g.batch.close()
                g.batch = D.Batch([a.solver for a in g.members], stream=g.stream, tune=False, config=self.config)
                g.rebuilds += 1
            q = quantum([a.remaining for a in g.members], self.qmax)
            if batched:
                g.batch.step(q)
            else:
                for a in g.members:
                    a.solver.step(q)
            g.event = torch.cuda.Event()
            g.event.record(g.stream)
        for a in g.members:
            a.remaining -= q
        g.busy = True
        g.quantum_steps += q
        self.launch_quanta += 1

    # -- the serving loop ----------------------------------------------

    def run(self, specs: List[W.RequestSpec], poll: float = 2e-4) -> List[Result]:
        """Serve ``specs`` (arrival times relative to the call) and return
        one result per request, in completion order."""
        pending = deque(sorted(specs, key=lambda s: s.arrival))
        sizes = {s.rid: footprint(W.request_problem(s)) for s in specs}
        for s in specs:
            if sizes[s.rid] > self.adm.budget:
                raise ValueError(f"request {s.rid} needs {sizes[s.rid]} bytes, more than the HBM budget")
        queue: deque = deque()
        done: List[_Done] = []
        results: List[Result] = []
        t0 = time.perf_counter()

        def withdrawn(spec, admitted, now):
            return Result(rid=spec.rid, ns=spec.ns, cells=spec.cells, nsteps=spec.nsteps, arrival=spec.arrival,
                          admitted=admitted, finished=now, status=0, conservation=np.zeros(0), cancelled=True)

        while pending or queue or done or any(g.members or g.incoming or g.busy for g in self.groups.values()):
            now = time.perf_counter() - t0
            progressed = False
            # cancellations: waiting requests leave at once, running ones at
            # their group's next quantum boundary (their memory is released then)
            due = lambda q: q.cancel_at is not None and q.cancel_at <= now
            for wait in (pending, queue):
                for spec in [q for q in wait if due(q)]:
                    wait.remove(spec)
                    results.append(withdrawn(spec, None, now))
                    progressed = True
            for g in self.groups.values():
                for a in g.members + g.incoming:
                    if due(a.spec):
                        a.cancelled = True
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            while queue and self.adm.fits(sizes[queue[0].rid]):
                spec = queue.popleft()
                self.adm.admit(sizes[spec.rid])
                self._start(spec, sizes[spec.rid], now)
                progressed = True
            for g in self.groups.values():
                if g.busy and g.event.query():
                    g.busy = False
                if not g.busy and (g.members or g.incoming):
                    dropped: List[_Active] = []
                    self._advance(g, done, dropped)
                    for a in dropped:
                        a.solver.close()
                        self.adm.release(a.nbytes)
                        results.append(withdrawn(a.spec, a.admitted, time.perf_counter() - t0))
                    progressed = True
            still = []
            for d in done:
                if d.event.query():
                    a = d.active
                    with self.torch.cuda.stream(d.stream):
                        status = a.solver.status()[0]
                    f = d.f.numpy().copy() if d.f is not None else None
                    results.append(Result(rid=a.spec.rid, ns=a.spec.ns, cells=a.spec.cells, nsteps=a.spec.nsteps,
                                          arrival=a.spec.arrival, admitted=a.admitted,
                                          finished=time.perf_counter() - t0, status=status,
                                          conservation=d.cons.numpy().copy(), f=f))
                    a.solver.close()
                    self.adm.release(a.nbytes)
                    progressed = True
                else:
                    still.append(d)
            done = still
            if not progressed:
                time.sleep(poll)
        for g in self.groups.values():
            if g.batch is not None:
                g.batch.close()
                g.batch = None
        return results


def run_sequential(specs: List[W.RequestSpec], precision: str = "fp64", device="cuda",
                   keep_f: bool = False) -> List[Result]:
    """The baseline of continuous batching: first come, first served, one
    request at a time, each a plain single-problem solve (``Solver``, one
    step launch per time step) in ``precision``.  Arrival times are
    honoured: a request that arrives while another runs waits for it.  Each
    request's latency runs from its arrival to the moment its conserved
    totals (and, with ``keep_f``, its final state) are in host memory."""
    import torch

    dev = torch.device(device)
    stream = torch.cuda.Stream(device=dev)
    results: List[Result] = []
    t0 = time.perf_counter()
    for spec in sorted(specs, key=lambda q: q.arrival):
        wait = spec.arrival - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        admitted = time.perf_counter() - t0
        with torch.cuda.stream(stream):
            s = D.Solver(W.request_problem(spec), precision, device=dev)
            s.set_state(*W.request_fields(spec, dev))
            s.step(spec.nsteps)
            cons = s.conservation().cpu().numpy()
            f = s.get_f().cpu().numpy() if keep_f else None
            status = s.status()[0]
        finished = time.perf_counter() - t0
        s.close()
        results.append(Result(rid=spec.rid, ns=spec.ns, cells=spec.cells, nsteps=spec.nsteps, arrival=spec.arrival,
                              admitted=admitted, finished=finished, status=status, conservation=cons, f=f))
    return results


def summarize(results: List[Result]) -> dict:
    """Latency percentiles and throughput (species-cell updates per second
    from the first arrival to the last completion) of the completed
    requests."""
    results = [r for r in results if not r.cancelled]
    lat = np.array([r.latency for r in results])
    t_first = min(r.arrival for r in results)
    t_last = max(r.finished for r in results)
    units = sum(r.units for r in results)
    return {"requests": len(results), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": t_last - t_first, "units": units,
            "throughput": units / (t_last - t_first)}


def simulate_sequential(specs: List[W.RequestSpec], rate_by_ns: Dict[int, float]) -> dict:
    """An extrapolation, not a run: first come, first served, one request at
    a time, each taking units / rate(S) seconds, for mixes too large to solve
    sequentially in the time at hand (``run_sequential`` solves them)."""
    t = 0.0
    lat = []
    units = 0
    first = min(s.arrival for s in specs)
    for s in sorted(specs, key=lambda q: q.arrival):
        t = max(t, s.arrival) + s.units / rate_by_ns[s.ns]
        lat.append(t - s.arrival)
        units += s.units
    lat = np.array(lat)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": t - first, "throughput": units / (t - first)}
