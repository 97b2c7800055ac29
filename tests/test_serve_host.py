"""Host logic of the continuous-batching server (admission by footprint,
slots, chunking, retirement) against a fake library: no GPU."""
import types

import numpy as np
import pytest

from paper_2308_01651_gb300 import serve


class FakeInstance:
    live = 0

    def __init__(self, prob, precision=None, op32=None):
        self.n = prob["n"]
        self.h = object()
        self.steps = 0
        FakeInstance.live += 1

    def activation_times(self):
        return np.full(self.n, float(self.steps))

    def potential(self):
        return np.zeros(self.n)

    def close(self):
        FakeInstance.live -= 1


def make_fake(monkeypatch, calls):
    insts = {}

    def Instance(prob, precision=None, op32=None):
        i = FakeInstance(prob, precision, op32)
        insts[id(i.h)] = i
        return i

    def ep_step_batch(handles, n):
        calls.append((len(handles), n))
        for h in handles:
            insts[id(h)].steps += n

    fake = types.SimpleNamespace(Instance=Instance, ep_step_batch=ep_step_batch,
                                 EP_PREC_FP32_REFINED=1, EP_OP_STENCIL=2)
    monkeypatch.setattr(serve, "ep", fake)
    monkeypatch.setattr(serve, "footprint", lambda prob, precision=1: prob["bytes"])


def _req(i, n, steps, arrival, nbytes):
    return serve.Request(rid=i, prob={"n": n, "bytes": nbytes}, steps=steps, arrival=arrival, precision=1)


def test_chunks_never_overrun_a_request(monkeypatch):
    calls = []
    make_fake(monkeypatch, calls)
    srv = serve.Server(memory_budget=100, max_slots=4, chunk=10, background=False)
    res = srv.run([_req(0, 5, 25, 0.0, 10), _req(1, 7, 12, 0.0, 10)])
    assert {r.rid: r.activation_ms[0] for r in res} == {0: 25.0, 1: 12.0}
    assert FakeInstance.live == 0
    # the second request retires after 12 steps: chunks 10, 2, then 10, 3 for the first
    assert calls == [(2, 10), (2, 2), (1, 10), (1, 3)]
    assert srv.dof_steps == 5 * 25 + 7 * 12


def test_admission_respects_budget_and_slots(monkeypatch):
    calls = []
    make_fake(monkeypatch, calls)
    srv = serve.Server(memory_budget=25, max_slots=2, chunk=100, background=False)
    reqs = [_req(i, 3, 5 + i, 0.0, 10) for i in range(5)]
    res = srv.run(reqs)
    assert len(res) == 5 and FakeInstance.live == 0
    assert max(e[1] for e in srv.log) <= 2
    assert max(e[3] for e in srv.log) <= 25
    assert all(c[0] <= 2 for c in calls)


def test_oversized_request_is_refused(monkeypatch):
    make_fake(monkeypatch, [])
    srv = serve.Server(memory_budget=5, max_slots=2)
    with pytest.raises(ValueError):
        srv.run([_req(0, 3, 5, 0.0, 10)])


def test_poisson_arrivals_seeded():
    g1, g2 = np.random.default_rng(7), np.random.default_rng(7)
    a, b = serve.poisson_arrivals(100, 50.0, g1), serve.poisson_arrivals(100, 50.0, g2)
    assert np.array_equal(a, b) and np.all(np.diff(a) > 0)
    assert 1.0 < a[-1] < 3.5  # 100 arrivals at 50/s


def test_background_creation_does_not_stall_residents(monkeypatch):
    """A slow creation (0.2 s) runs on the worker thread: the resident
    request keeps taking chunks meanwhile, the new one joins later, every
    result is complete and the footprint was reserved from admission on."""
    import threading
    import time as _t

    calls = []
    make_fake(monkeypatch, calls)
    fake_instance = serve.ep.Instance
    main = threading.get_ident()
    made_on = []

    def slow_instance(prob, precision=None, op32=None):
        made_on.append(threading.get_ident())
        if prob["n"] == 9:
            _t.sleep(0.2)
        return fake_instance(prob, precision, op32)

    monkeypatch.setattr(serve.ep, "Instance", slow_instance)
    step_batch = serve.ep.ep_step_batch

    def slow_step(handles, n):  # a chunk takes 0.5 ms
        _t.sleep(0.0005)
        step_batch(handles, n)

    monkeypatch.setattr(serve.ep, "ep_step_batch", slow_step)
    srv = serve.Server(memory_budget=100, max_slots=4, chunk=1)
    res = srv.run([_req(0, 5, 1000, 0.0, 10), _req(1, 9, 3, 0.01, 20)])
    assert sorted(r.rid for r in res) == [0, 1] and FakeInstance.live == 0
    assert all(t != main for t in made_on)
    s = srv.summary()
    assert s["chunks_during_creation"] >= 2  # stepping went on during the slow creation
    assert max(e[3] for e in srv.log) == 30


def test_ps_arrival_rate():
    # budget large against the resident work: the load cap applies
    rate, rho = serve.ps_arrival_rate(1e9, 1e8, 1e8 * 1e8, 1e12, rho_max=0.9)
    assert abs(rho - 0.9) < 1e-12 and abs(rate - 9.0) < 1e-9
    # small budget: Little's law with processor sharing gives the budget back
    X, Es, Efs, B = 1e9, 1e8, 3e16, 5e8
    rate, rho = serve.ps_arrival_rate(X, Es, Efs, B)
    resident = rate * Efs / (X * (1.0 - rho))
    assert rho < 0.9 and abs(resident - B) < 1e-6 * B
