"""Continuous-batching server for evaporation runs.

Requests (lattice parameters, seeded initial state, step count) arrive over
time. The server keeps their lattices resident in one batch arena, admits a
request as soon as its lattice fits in the free arena (admission by free device
memory, first come first served; optionally also capped in resident sites),
and advances all admitted lattices together
with the batched step (one persistent launch per time step over every member).
Each run records a time series of the paper's observables every `diag_every`
steps: interface position (film) or droplet radius, the last step's evaporated
mass (the flux through the sink) and the cumulative evaporated mass
(arXiv:1701.03637 Sec. III). A finished run leaves the batch at once, freeing
its range for the next request. Every member computes exactly what a lone run
computes, so a result does not depend on the mix it was served in. A run whose
diagnostics report a non-finite density or a negative sink complement is
evicted at that record and reported with the status; the others carry on.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

from ._native import ScError


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the stream starts
    params: dict
    init: dict
    steps: int


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    sites: int
    series: list = field(default_factory=list)  # (step, interface_z, radius, flux_last, evaporated_mass, mass_r)
    status: int = 0  # diagnostics status that ended the run early (SC_ENONFINITE, SC_ESINKNEG); 0 = completed

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _record(lat, res):
    """Append the run's diagnostics to its series; a non-zero status (a non-finite
    density or a negative sink complement) ends the run: it is stored in the result
    and returned, and the caller evicts the run."""
    d = lat.diagnostics()
    if d["status"] != 0:
        res.status = int(d["status"])
        return res.status
    res.series.append((d["step"], d["interface_z"], d["radius"], d["flux_last"], d["evaporated_mass"], d["mass_r"]))
    return 0


class Server:
    """Serve requests with continuous batching on the current CUDA device."""

    def __init__(self, arena_bytes: int, storage="f16", diag_every: int = 100, tile: int = 0, zchunk: int = 0,
                 batch=None, max_active_sites: int = 0):
        if batch is None:
            from . import Batch
            batch = Batch(arena_bytes, storage)
        self.batch = batch
        self.storage = storage
        self.diag_every = int(diag_every)
        # admission also stops at this many resident sites (0: the arena is the only
        # limit): enough work to fill the GPU, few enough runs that each one keeps a
        # large share of it, which keeps first-come-first-served latencies short
        self.max_active_sites = int(max_active_sites)
        if tile or zchunk:
            self.batch.configure(tile, zchunk)

    def close(self):
        self.batch.close()

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep):
        """Serve `requests` (sorted by arrival); returns the Results in request order
        (a run evicted for a bad diagnostics status has Result.status != 0)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        active = {}   # slot -> (request, lattice, result, steps done)
        done = {}
        t0 = clock()
        while pending or active:
            now = clock() - t0
            # admit every arrived request that fits, in arrival order
            while pending and pending[0].arrival <= now:
                r = pending[0]
                sites = r.params["nx"] * r.params["ny"] * r.params["nz"]
                if active and self.max_active_sites and \
                        sum(v[1].n for v in active.values()) + sites > self.max_active_sites:
                    break
                try:
                    slot, lat = self.batch.add(r.params)
                except ScError as e:
                    if e.code == -2:
                        if not active:
                            raise RuntimeError(f"request {r.rid} does not fit in an empty arena") from e
                        break  # wait for a member to finish
                    raise
                pending.pop(0)
                lat.init(r.init)
                self.batch.set_steps(slot, r.steps)
                res = Result(r.rid, r.arrival, clock() - t0, 0.0, r.steps, lat.n)
                if _record(lat, res):  # a state that is already bad: reported, never stepped
                    res.finished = clock() - t0
                    done[r.rid] = res
                    self.batch.remove(slot)
                    continue
                active[slot] = (r, lat, res, 0)
            if not active:
                if pending:
                    sleep(max(0.0, pending[0].arrival - (clock() - t0)))
                continue
            # advance every member to its next diagnostics point (none steps past its limit)
            k = min(min(self.diag_every - d % self.diag_every, r.steps - d) for r, _, _, d in active.values())
            self.batch.step(k)
            for slot in list(active):
                r, lat, res, d = active[slot]
                d += k
                failed = (d % self.diag_every == 0 or d == r.steps) and _record(lat, res) != 0
                if d == r.steps or failed:  # finished, or evicted with its status
                    res.finished = clock() - t0
                    done[r.rid] = res
                    self.batch.remove(slot)
                    del active[slot]
                else:
                    active[slot] = (r, lat, res, d)
        return [done[r.rid] for r in sorted(requests, key=lambda r: r.rid)]


def serve_one_at_a_time(requests, storage="f32", diag_every: int = 100, clock=time.perf_counter, sleep=time.sleep):
    """The same stream served one run at a time (first come first served) through the
    single-lattice path: the baseline the batched server is compared with."""
    from . import Lattice
    out = []
    t0 = clock()
    for r in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if r.arrival > now:
            sleep(r.arrival - now)
        lat = Lattice(dict(r.params, storage=storage))
        lat.init(r.init)
        res = Result(r.rid, r.arrival, clock() - t0, 0.0, r.steps, lat.n)
        done = r.steps if _record(lat, res) else 0
        while done < r.steps:
            k = min(diag_every - done % diag_every, r.steps - done)
            lat.step(k)
            done += k
            if _record(lat, res):
                break
        res.finished = clock() - t0
        lat.close()
        out.append(res)
    return sorted(out, key=lambda x: x.rid)


def dispatch(requests, rank: int, world: int):
    """Round-robin dispatch of a request stream over `world` GPUs in arrival order:
    rank r serves requests r, r + world, r + 2 world, ... of the stream (each request
    on exactly one rank, no data exchanged between ranks). Arrival times are kept,
    so every rank sees its share of the stream in real time."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    order = sorted(requests, key=lambda q: (q.arrival, q.rid))
    return [q for k, q in enumerate(order) if k % world == rank]


def percentile(values, q):
    v = sorted(values)
    if not v:
        return float("nan")
    pos = (len(v) - 1) * q / 100.0
    lo = int(pos)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (pos - lo)
