"""The allocation-free residual check (ep_residual_norm_noalloc).

Some host applications cannot let this library allocate device memory where
they check a solve: their GPU memory belongs to another allocator (a
framework's caching allocator, or a pool that reserves the device's memory at
start-up), so a cudaMalloc there would fail or break the owner's accounting.
ep_residual_norm_noalloc serves them: it recomputes the relative residual of
an instance's last solve with a fixed scratch array inside the library
instead of any allocation.  This file checks it against the residual the
solver itself reports through ep_get_stats, on two calls in a row, after
steps of an FP32-refined instance.  When the step's last residual came from
the solver's residual pass (the step took a refinement sweep), the check runs
the same nodes per thread in the same summation order and must agree to
1e-12 relative.  When the step's first residual already met the tolerance
(no sweep), the solver formed it from its A u history instead of an operator
apply; both are float-float evaluations accurate to about 1e-14 of ||b||, so
they must agree to 1e-13 in the relative residual.  Before the first step,
and after a state load (whose potential no solve produced), the call is
refused with EP_EINVAL.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _problem():
    return I.slab_ttp06(nx=40, ny=12, nz=8, L=(0.4, 0.12, 0.08), T=5.0)


def _check_against_solver(inst, steps):
    inst.step(steps)
    st = inst.stats()
    reported = st["relres"]
    before = inst.save()
    first = ep.ep_residual_norm_noalloc(inst.h)
    second = ep.ep_residual_norm_noalloc(inst.h)
    assert reported > 0.0 and reported <= 1e-10
    assert first == second
    if st["sweeps"] >= 1:
        # same nodes per thread and summation order as the solver's
        # residual pass
        assert abs(first - reported) <= 1e-12 * reported
    else:
        assert abs(first - reported) <= 1e-13
    # the check reads the instance and changes nothing in it
    assert np.array_equal(before, inst.save())
    return st["sweeps"] >= 1


def test_residual_norm_noalloc_matches_solver_residual():
    inst = ep.Instance(_problem(), precision=ep.EP_PREC_FP32_REFINED)
    strict = 0
    try:
        for steps in (1, 25, 7):
            strict += _check_against_solver(inst, steps)
    finally:
        inst.close()
    assert strict >= 1


def test_residual_norm_noalloc_needs_a_solve():
    inst = ep.Instance(_problem(), precision=ep.EP_PREC_FP32_REFINED)
    try:
        with pytest.raises(ep.EpError) as e:
            ep.ep_residual_norm_noalloc(inst.h)
        assert e.value.status == ep.EP_EINVAL
        inst.step(10)
        buf = inst.save()
        inst.step(3)
        inst.load(buf)
        with pytest.raises(ep.EpError) as e:
            ep.ep_residual_norm_noalloc(inst.h)
        assert e.value.status == ep.EP_EINVAL
        # the next step's solve makes it valid again
        _check_against_solver(inst, 1)
    finally:
        inst.close()
