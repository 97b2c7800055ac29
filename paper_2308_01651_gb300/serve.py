"""Continuous-batching simulation server over the C ABI.

Requests (a problem record, a number of steps and an arrival time) are
admitted while device memory allows -- each one's footprint comes from
ep_footprint_bytes before anything is allocated -- and a free slot exists.
Admitted simulations stay resident on the GPU and advance together: the
server steps the whole resident set with ep_step_batch in chunks of a few
steps, so a request that arrives while others run joins the next chunk,
its work overlapping theirs on the device.  When a simulation has taken its
steps, its activation times and final potential are read back, the
instance is destroyed, its memory is free for the next admission, and its
time to result (arrival to read-back) is recorded.

The batch changes whenever a request joins or leaves; ep_step_batch then
builds the new batch's tables and graph (cached per instance list).  Every
instance's arithmetic is its own (block ranges per instance), so a result
does not depend on which other requests shared its chunks, up to the
rounding of the inner iterations (see the batched-stepping tests).
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import ep


@dataclass
class Request:
    rid: int
    prob: dict
    steps: int
    arrival: float  # seconds after the server starts
    precision: int = ep.EP_PREC_FP32_REFINED


@dataclass
class Result:
    rid: int
    nodes: int
    steps: int
    arrival: float
    admitted: float
    done: float
    activation_ms: np.ndarray = field(repr=False)
    potential_mV: np.ndarray = field(repr=False)

    @property
    def time_to_result(self):
        return self.done - self.arrival


def footprint(prob, precision=ep.EP_PREC_FP32_REFINED):
    return ep.ep_footprint_bytes(prob["mesh"], prob["model"], precision=precision, op32=ep.EP_OP_STENCIL)


class Server:
    """memory_budget: device bytes the resident simulations may use;
    max_slots: resident simulations at most; chunk: steps per batched call."""

    def __init__(self, memory_budget, max_slots=64, chunk=20, clock=time.perf_counter):
        self.budget = int(memory_budget)
        self.max_slots = max_slots
        self.chunk = chunk
        self.clock = clock
        self.used = 0
        self.active = []  # [request, instance, steps left, admitted time, footprint]
        self.results = []
        self.dof_steps = 0
        self.log = []

    def _admit(self, req, now):
        fp = footprint(req.prob, req.precision)
        inst = ep.Instance(req.prob, precision=req.precision, op32=ep.EP_OP_STENCIL)
        self.used += fp
        self.active.append([req, inst, req.steps, now, fp])

    def _retire(self, entry, now):
        req, inst, _, admitted, fp = entry
        at = inst.activation_times()
        u = inst.potential()
        n = inst.n
        inst.close()
        self.used -= fp
        self.results.append(Result(req.rid, n, req.steps, req.arrival, admitted, self.clock() - self.t0,
                                   at, u))

    def run(self, requests):
        """Serves the requests (sorted by arrival) to completion; returns the
        results in completion order."""
        pending = sorted(requests, key=lambda r: r.arrival)
        too_big = [r for r in pending if footprint(r.prob, r.precision) > self.budget]
        if too_big:
            raise ValueError(f"request {too_big[0].rid} does not fit the memory budget")
        self.t0 = self.clock()
        while pending or self.active:
            now = self.clock() - self.t0
            # admit, in arrival order, what has arrived and fits
            while pending and pending[0].arrival <= now and len(self.active) < self.max_slots and \
                    self.used + footprint(pending[0].prob, pending[0].precision) <= self.budget:
                self._admit(pending.pop(0), now)
            if not self.active:
                # idle until the next arrival
                wait = pending[0].arrival - now
                if wait > 0:
                    time.sleep(min(wait, 0.05))
                continue
            # one chunk for every resident simulation, never past its end
            k = min(self.chunk, min(e[2] for e in self.active))
            ep.ep_step_batch([e[1].h for e in self.active], k)
            for e in self.active:
                e[2] -= k
                self.dof_steps += e[1].n * k
            self.log.append((now, len(self.active), k, self.used))
            done = [e for e in self.active if e[2] == 0]
            self.active = [e for e in self.active if e[2] > 0]
            now = self.clock() - self.t0
            for e in done:
                self._retire(e, now)
        self.makespan = self.clock() - self.t0
        return self.results

    def summary(self):
        ttr = np.array([r.time_to_result for r in self.results])
        return {
            "requests": len(self.results),
            "makespan_s": self.makespan,
            "dof_steps_per_s": self.dof_steps / self.makespan if self.makespan > 0 else 0.0,
            "time_to_result_s": {"p50": float(np.percentile(ttr, 50)), "p99": float(np.percentile(ttr, 99)),
                                 "max": float(ttr.max())},
            "max_resident": max((e[1] for e in self.log), default=0),
            "max_resident_bytes": max((e[3] for e in self.log), default=0),
            "chunks": len(self.log),
        }


def poisson_arrivals(n, rate, g):
    """n arrival times (s) of a Poisson process of the given rate (1/s)."""
    return np.cumsum(g.exponential(1.0 / rate, size=n))


def request_mix(n, g, n_lo=1.0e4, n_hi=2.2e6, t_lo=200.0, t_hi=600.0, dt=0.05, shell_fraction=0.5):
    """Problem records of the serving workload: sizes log-uniform in
    [n_lo, n_hi] nodes, slab or truncated-ellipsoid shell (each with
    probability 1/2), Bueno-Orovio or TTP06 (1/2 each), durations uniform in
    [t_lo, t_hi] ms.  Shapes follow the slab and shell generators, scaled to
    the drawn size."""
    from . import inputs as I

    out = []
    for _ in range(n):
        N = math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))
        T = g.uniform(t_lo, t_hi)
        model = I.TTP06 if g.uniform() < 0.5 else I.BO
        if g.uniform() < shell_fraction:
            # shell nt x nphi x nlong with the 20 x 400 x 260 proportions
            s = (N / (21 * 400 * 261)) ** (1.0 / 3.0)
            nt = max(2, int(round(20 * s)))
            nphi = max(8, int(round(400 * s)))
            nlong = max(4, int(round(260 * s)))
            p = I.shell_ttp06(nt=nt, nphi=nphi, nlong=nlong, T=T, dt=dt)
            if model == I.BO:
                p = I.as_bo(p)
        else:
            p = I.batch_slabs(count=1, n_lo=N, n_hi=N * 1.0000001, T=T, dt=dt,
                              seed_offset=int(g.integers(1 << 30)))[0]
        out.append((p, int(round(T / dt))))
    return out
