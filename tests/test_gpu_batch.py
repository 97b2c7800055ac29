"""Batched stepping (ep_step_batch): instances of uneven sizes and different
ionic models advance together, one launch per phase, the step in one CUDA
graph per batch.

Every instance keeps its own block counts in the non-persistent kernels, and
the persistent inner solver gets a share of the GPU in proportion to its size,
so a batched instance differs from the same instance stepped alone only in
the rounding of its inner iterations; both are refined to ||r|| <= 1e-10 ||b||.
Tolerance: potentials within 1e-9 relative of the instance run alone,
activation times within one time step.  The oracle pins one batched
trajectory directly (refined tolerances of the parity tests).
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

from .helpers import gpu_state, rel_err

pytestmark = pytest.mark.gpu

REF, FP64 = ep.EP_PREC_FP32_REFINED, ep.EP_PREC_FP64
ST = ep.EP_OP_STENCIL


def _mix():
    h = 0.01
    return [
        I.slab_bo_small(nx=12, ny=7, nz=5, L=(0.6, 0.35, 0.25), T=3.0),
        I.slab_ttp06(nx=40, ny=9, nz=6, L=(40 * h, 9 * h, 6 * h), T=3.0),
        I.slab_ttp06(nx=23, ny=11, nz=7, L=(23 * h, 11 * h, 7 * h), T=3.0),  # ragged tiles
        I.slab_bo_small(nx=33, ny=5, nz=4, L=(0.66, 0.1, 0.08), T=3.0),
    ]


def _alone(prob, steps, precision=REF):
    inst = ep.Instance(prob, precision=precision, op32=ST)
    inst.step(steps)
    out = (inst.potential(), inst.activation_times(), inst.stats())
    inst.close()
    return out


def _check_same(inst, ref, dt):
    u, at, st = ref
    ub, atb = inst.potential(), inst.activation_times()
    assert rel_err(ub, u) <= 1e-9, rel_err(ub, u)
    assert np.array_equal(np.isnan(atb), np.isnan(at))
    ok = ~np.isnan(at)
    if ok.any():
        assert np.abs(atb[ok] - at[ok]).max() <= dt + 1e-12
    assert inst.stats()["step"] == st["step"]


def test_batch_matches_each_instance_alone():
    probs = _mix()
    K = 40
    alone = [_alone(p, K) for p in probs]
    insts = [ep.Instance(p, precision=REF, op32=ST) for p in probs]
    try:
        # two calls: the second reuses the batch's graph; the TTP06 instances
        # change BDF order (1 -> 2) inside the first call
        ep.ep_step_batch([i.h for i in insts], 25)
        ep.ep_step_batch([i.h for i in insts], K - 25)
        for inst, ref, p in zip(insts, alone, probs):
            _check_same(inst, ref, p["dt"])
            assert inst.stats()["relres"] <= 1e-10
    finally:
        for i in insts:
            i.close()


def test_batched_trajectory_against_oracle():
    probs = _mix()[:2]
    K = 30
    insts = [ep.Instance(p, precision=REF, op32=ST) for p in probs]
    try:
        ep.ep_step_batch([i.h for i in insts], K)
        for inst, p in zip(insts, probs):
            sim = O.sim_from_problem(p)
            sim.step(K)
            u_ref = sim.potential()
            assert rel_err(gpu_state(inst)["u_n"], u_ref) <= 1e-5
    finally:
        for i in insts:
            i.close()


def test_batch_with_unbatchable_member_steps_each_alone():
    """An FP64 instance in the list: the call steps every instance on its own
    graph, with results identical to stepping it alone."""
    probs = _mix()[:2]
    K = 12
    ref64 = _alone(probs[0], K, precision=FP64)
    ref32 = _alone(probs[1], K)
    a = ep.Instance(probs[0], precision=FP64)
    b = ep.Instance(probs[1], precision=REF, op32=ST)
    try:
        ep.ep_step_batch([a.h, b.h], K)
        assert np.array_equal(a.potential(), ref64[0])
        assert np.array_equal(b.potential(), ref32[0])
    finally:
        a.close()
        b.close()


def test_batch_membership_changes():
    """Plans follow the instance list: a destroyed member invalidates its
    batch; a new list builds a new plan; states stay per instance."""
    probs = _mix()
    a = ep.Instance(probs[0], precision=REF, op32=ST)
    b = ep.Instance(probs[1], precision=REF, op32=ST)
    c = None
    try:
        ep.ep_step_batch([a.h, b.h], 10)
        b.close()
        c = ep.Instance(probs[2], precision=REF, op32=ST)
        ep.ep_step_batch([a.h, c.h], 10)
        ep.ep_step_batch([c.h, a.h], 5)  # another order: another plan
        assert a.stats()["step"] == 25 and c.stats()["step"] == 15
        _check_same(a, _alone(probs[0], 25), probs[0]["dt"])
        _check_same(c, _alone(probs[2], 15), probs[2]["dt"])
    finally:
        a.close()
        if c is not None:
            c.close()


def test_batch_argument_errors():
    p = _mix()[0]
    a = ep.Instance(p, precision=REF, op32=ST)
    try:
        with pytest.raises(ep.EpError) as e:
            ep.ep_step_batch([a.h, a.h], 1)
        assert e.value.status == ep.EP_EINVAL
        with pytest.raises(ep.EpError) as e:
            ep.ep_step_batch([a.h], -1)
        assert e.value.status == ep.EP_EINVAL
        ep.ep_step_batch([], 3)  # empty batch: nothing to do
    finally:
        a.close()
