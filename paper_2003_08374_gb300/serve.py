"""Continuous-batching server for many independent micro-continuum simulations.

Requests (a case plus a step count) arrive over time.  Between rounds the
scheduler admits every arrived request that fits the free device memory (the
library's own device-byte estimate against cudaMemGetInfo, minus a reserve)
and the slot limit, keeps the admitted requests' fields resident on the device,
and advances all of them together as one batch (mdbs_batch: one kernel launch
per step phase, one CUDA graph per step), so that newly admitted work overlaps
with the work already on the GPU.  Requests join and leave the batch between
rounds (mdbs_batch_add / mdbs_batch_remove).  A round is never longer than the smallest
remaining step count, so every request runs exactly its own number of steps;
finished requests are read back and release their memory at once.  Because a
member's arithmetic does not depend on the other members, a request's result
is the same alone and in any mix.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import mdbs


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    case: object            # workloads.Case with its fields
    steps: int
    admitted: float = None
    finished: float = None
    rejected: bool = False
    error: str = None
    result: dict = field(default=None, repr=False)
    stats: dict = field(default=None, repr=False)


class Server:
    def __init__(self, max_active=256, round_steps=10, reserve_bytes=2 << 30, keep_fields=True,
                 stream_handle=None, free_bytes_fn=None):
        self.free_bytes_fn = free_bytes_fn
        self.max_active = max_active
        self.round_steps = round_steps
        self.reserve = reserve_bytes
        self.keep_fields = keep_fields
        self.stream_handle = stream_handle
        self.rounds = 0
        self.rebuilds = 0
        self.cell_steps = 0
        self.peak_active = 0
        self.not_converged_rounds = 0

    def _free_bytes(self):
        if self.free_bytes_fn is not None:
            return self.free_bytes_fn()
        import torch
        free, _ = torch.cuda.mem_get_info()
        return free

    def run(self, requests, clock=time.perf_counter):
        pending = sorted(requests, key=lambda r: r.arrival)
        active = []          # (request, simulation, remaining steps)
        batch = None
        t0 = clock()
        i = 0
        while i < len(pending) or active:
            now = clock() - t0
            # admission: arrived requests in order while slots and memory allow
            budget = self._free_bytes() - self.reserve
            while i < len(pending) and pending[i].arrival <= now and len(active) < self.max_active:
                req = pending[i]
                need = mdbs.bytes_required(req.case)
                if need > budget:
                    if active:
                        break  # wait for resident requests to finish and free memory
                    req.rejected = True  # does not fit even on an idle device
                    i += 1
                    continue
                sim = mdbs.Simulation(req.case)
                if self.stream_handle is not None:
                    sim.set_stream(self.stream_handle)
                if batch is not None:
                    batch.add(sim)  # joins before the next round (mdbs_batch_add)
                    self.rebuilds += 1
                req.admitted = clock() - t0
                active.append([req, sim, req.steps])
                budget -= need
                i += 1
            if not active:
                if i < len(pending):
                    time.sleep(max(0.0, min(pending[i].arrival - (clock() - t0), 0.05)))
                continue
            if batch is None:
                batch = mdbs.Batch([a[1] for a in active])
                if self.stream_handle is not None:
                    batch.set_stream(self.stream_handle)
                self.rebuilds += 1
            self.peak_active = max(self.peak_active, len(active))
            k = min(self.round_steps, min(a[2] for a in active))
            failed = []
            try:
                batch.step(k)
            except mdbs.MdbsError as e:
                if e.code == mdbs.ERR_NOT_CONVERGED:
                    # the round's steps were taken; a solve stopped at max_cg (counted)
                    self.not_converged_rounds += 1
                elif e.code != mdbs.ERR_DIVERGED:
                    raise
                else:
                    # retire the members whose fields went non-finite; the others are unaffected
                    for a in active:
                        st = a[1].stats()
                        if not (np.isfinite(st["mass"]) and np.isfinite(st["alpha_min"])):
                            failed.append(a)
            self.rounds += 1
            self.cell_steps += k * sum(a[0].case.cells for a in active if a not in failed)
            done = []
            for a in active:
                if a in failed:
                    a[0].error = "diverged"
                    done.append(a)
                    continue
                a[2] -= k
                if a[2] == 0:
                    done.append(a)
            if done:
                for a in done:
                    if len(batch.sims) > 1:
                        batch.remove(a[1])  # leaves before the next round (mdbs_batch_remove)
                        self.rebuilds += 1
                    else:
                        batch.close()
                        batch = None
                for a in done:
                    req, sim = a[0], a[1]
                    if req.error is None:
                        req.finished = clock() - t0
                        req.stats = sim.stats()
                        if self.keep_fields:
                            req.result = sim.fields()
                    sim.close()
                    active.remove(a)
        if batch is not None:
            batch.close()
        wall = clock() - t0
        return summarize(requests, wall, self)


def summarize(requests, wall, server):
    lat = np.array([r.finished - r.arrival for r in requests if r.finished is not None])
    wait = np.array([r.admitted - r.arrival for r in requests if r.admitted is not None])
    return {
        "requests": len(requests),
        "completed": int(lat.size),
        "rejected": int(sum(1 for r in requests if r.rejected)),
        "failed": int(sum(1 for r in requests if r.error)),
        "wall_s": wall,
        "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
        "mean_queue_wait_s": float(wait.mean()) if wait.size else None,
        "served_cell_steps_per_s": server.cell_steps / wall if wall > 0 else None,
        "rounds": server.rounds,
        "batch_rebuilds": server.rebuilds,
        "peak_active": server.peak_active,
        "rounds_with_unconverged_solves": server.not_converged_rounds,
    }


def fractured_request_case(side, ca, seed, precision=0, sigma=0.07, mu_w=1e-3, cfl=0.5, **kw):
    """A fractured porous cube (the 3-D fractured-block recipe) whose inlet velocity
    realises capillary number ca = mu_w u / sigma.  At high ca the flow funnels into
    the fracture, so the time step follows the CFL number (capped at 1e-6 s)."""
    from . import workloads as W
    frac = max(2, side // 16)
    return W.grf_3d(shape=(side, side, side), seed=seed, corr_len=max(2.0, side / 16.0), frac_w=frac,
                    inlet_u=ca * sigma / mu_w, precision=precision, cfl=cfl, dt=1e-6, dt_max=1e-6, **kw)
