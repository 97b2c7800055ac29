"""The continuous-batching server on the GPU: requests that arrive while
others run join the resident batch; each result equals the same simulation
run alone within the batched-stepping tolerance (potentials 1e-9 relative,
activation times within one step)."""
import numpy as np
import pytest

from paper_2308_01651_gb300 import ep, serve
from paper_2308_01651_gb300 import inputs as I

from .helpers import rel_err

pytestmark = pytest.mark.gpu


def _requests():
    h = 0.01
    probs = [I.slab_ttp06(nx=30, ny=8, nz=6, L=(30 * h, 8 * h, 6 * h), T=50.0),
             I.slab_bo_small(nx=14, ny=6, nz=5, L=(0.7, 0.3, 0.25), T=50.0),
             I.as_bo(I.shell_ttp06(nt=3, nphi=16, nlong=10, T=50.0)),
             I.slab_ttp06(nx=21, ny=9, nz=5, L=(21 * h, 9 * h, 5 * h), T=50.0)]
    # long enough that the later requests (created on the server's worker
    # thread while the first ones step) join them
    steps = [900, 700, 800, 500]
    arrivals = [0.0, 0.0, 0.002, 0.004]
    return [serve.Request(rid=i, prob=p, steps=k, arrival=a)
            for i, (p, k, a) in enumerate(zip(probs, steps, arrivals))]


def test_served_results_equal_alone():
    reqs = _requests()
    srv = serve.Server(memory_budget=2 << 30, max_slots=8, chunk=5)
    res = {r.rid: r for r in srv.run(reqs)}
    assert sorted(res) == [0, 1, 2, 3]
    assert max(e[1] for e in srv.log) >= 2, "requests shared chunks"
    for q in reqs:
        inst = ep.Instance(q.prob, precision=q.precision, op32=ep.EP_OP_STENCIL)
        inst.step(q.steps)
        u, at = inst.potential(), inst.activation_times()
        inst.close()
        r = res[q.rid]
        assert r.steps == q.steps and r.time_to_result >= 0.0
        assert rel_err(r.potential_mV, u) <= 1e-9
        assert np.array_equal(np.isnan(r.activation_ms), np.isnan(at))
        ok = ~np.isnan(at)
        if ok.any():
            assert np.abs(r.activation_ms[ok] - at[ok]).max() <= q.prob["dt"] + 1e-12
    s = srv.summary()
    assert s["requests"] == 4 and s["dof_steps_per_s"] > 0


def test_memory_budget_limits_residency():
    """A budget of the largest request's footprint: every request completes
    and the resident footprint never exceeds the budget."""
    reqs = _requests()[:3]
    big = max(serve.footprint(q.prob) for q in reqs)
    srv = serve.Server(memory_budget=big, max_slots=8, chunk=5)
    res = srv.run(reqs)
    assert len(res) == 3
    assert max(e[3] for e in srv.log) <= big
