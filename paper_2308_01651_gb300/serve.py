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

Admission does not stall the residents: an admitted request's instance is
created (upload, operator assembly, graph build: ep_create) on a worker
thread with its own CUDA stream while the main thread keeps stepping the
resident set; the new instance joins at the first chunk boundary after its
creation has finished.  Its footprint is reserved from the moment it is
admitted.  The per-chunk log records when each chunk started and ended and
how many creations were in flight meanwhile.

The batch changes whenever a request joins or leaves; ep_step_batch then
builds the new batch's tables and graph (cached per instance list).  Every
instance's arithmetic is its own (block ranges per instance), so a result
does not depend on which other requests shared its chunks, up to the
rounding of the inner iterations (see the batched-stepping tests).
"""
import concurrent.futures as cf
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
    max_slots: resident simulations at most; chunk: steps per batched call;
    background: create admitted instances on a worker thread (False: on the
    stepping thread, between chunks)."""

    def __init__(self, memory_budget, max_slots=64, chunk=20, clock=time.perf_counter, background=True):
        self.budget = int(memory_budget)
        self.max_slots = max_slots
        self.chunk = chunk
        self.clock = clock
        self.background = background
        self.used = 0
        self.active = []  # [request, instance, steps left, admitted time, footprint]
        self.creating = []  # [request, future, footprint, admission time]
        self.results = []
        self.dof_steps = 0
        # per chunk: (start s, resident, steps, reserved bytes, end s, creations in flight)
        self.log = []
        self.create_s = []

    def _create(self, req):
        t = self.clock()
        inst = ep.Instance(req.prob, precision=req.precision, op32=ep.EP_OP_STENCIL)
        return inst, self.clock() - t

    def _admit(self, req, now, pool):
        fp = footprint(req.prob, req.precision)
        self.used += fp
        if pool is None:
            inst, dt = self._create(req)
            self.create_s.append(dt)
            self.active.append([req, inst, req.steps, now, fp])
        else:
            self.creating.append([req, pool.submit(self._create, req), fp, now])

    def _join_created(self, block):
        """Moves finished creations into the resident set; with block, waits
        for the first one when nothing else could run."""
        if block and self.creating:
            cf.wait([c[1] for c in self.creating], return_when=cf.FIRST_COMPLETED)
        still = []
        for req, fut, fp, adm in self.creating:
            if fut.done():
                inst, dt = fut.result()  # re-raises a creation failure
                self.create_s.append(dt)
                self.active.append([req, inst, req.steps, self.clock() - self.t0, fp])
            else:
                still.append([req, fut, fp, adm])
        self.creating = still

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
        pool = cf.ThreadPoolExecutor(max_workers=1) if self.background else None
        try:
            self._serve(pending, pool)
        finally:
            if pool is not None:
                pool.shutdown(wait=True)
        return self.results

    def _serve(self, pending, pool):
        self.t0 = self.clock()
        while pending or self.active or self.creating:
            now = self.clock() - self.t0
            # admit, in arrival order, what has arrived and fits
            while pending and pending[0].arrival <= now and \
                    len(self.active) + len(self.creating) < self.max_slots and \
                    self.used + footprint(pending[0].prob, pending[0].precision) <= self.budget:
                self._admit(pending.pop(0), now, pool)
            self._join_created(block=not self.active)
            if not self.active:
                if not self.creating:
                    # idle until the next arrival
                    wait = pending[0].arrival - (self.clock() - self.t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                continue
            # one chunk for every resident simulation, never past its end
            k = min(self.chunk, min(e[2] for e in self.active))
            t_start = self.clock() - self.t0
            ep.ep_step_batch([e[1].h for e in self.active], k)
            for e in self.active:
                e[2] -= k
                self.dof_steps += e[1].n * k
            t_end = self.clock() - self.t0
            self.log.append((t_start, len(self.active), k, self.used, t_end, len(self.creating)))
            done = [e for e in self.active if e[2] == 0]
            self.active = [e for e in self.active if e[2] > 0]
            for e in done:
                self._retire(e, t_end)
        self.makespan = self.clock() - self.t0

    def summary(self):
        ttr = np.array([r.time_to_result for r in self.results])
        overlapped = [e for e in self.log if e[5] > 0]
        return {
            "requests": len(self.results),
            "makespan_s": self.makespan,
            "dof_steps_per_s": self.dof_steps / self.makespan if self.makespan > 0 else 0.0,
            "time_to_result_s": {"p50": float(np.percentile(ttr, 50)), "p99": float(np.percentile(ttr, 99)),
                                 "max": float(ttr.max())},
            "max_resident": max((e[1] for e in self.log), default=0),
            "max_resident_bytes": max((e[3] for e in self.log), default=0),
            "chunks": len(self.log),
            "chunks_during_creation": len(overlapped),
            "create_s": {"mean": float(np.mean(self.create_s)) if self.create_s else 0.0,
                         "max": float(np.max(self.create_s)) if self.create_s else 0.0},
        }


def ps_arrival_rate(capacity, mean_work, mean_fp_work, budget_bytes, rho_max=0.9):
    """Arrival rate (1/s) at which the expected resident footprint of a
    processor-sharing server equals budget_bytes.  capacity: measured
    DoF-steps/s of the batched device; mean_work: E[N steps] of a request;
    mean_fp_work: E[footprint x N steps].  With load rho = rate E[s] / X a
    request of work s stays s / (X (1 - rho)) (M/G/1 processor sharing), so
    by Little's law the resident bytes are rate E[fp s] / (X (1 - rho));
    setting them to the budget gives
        rate = budget X / (E[fp s] + budget E[s]),
    capped at rho_max X / E[s] (a load that close to 1 has no steady state
    within a finite run).  Returns (rate, load)."""
    rate = budget_bytes * capacity / (mean_fp_work + budget_bytes * mean_work)
    cap = rho_max * capacity / mean_work
    rate = min(rate, cap)
    return rate, rate * mean_work / capacity


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
