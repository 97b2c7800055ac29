"""The allocation-free residual check (ep_residual_norm_noalloc).

Some callers must not allocate device memory at the point where they check a
solve -- while capturing a stream into a graph, in a host callback, or under
an allocator that owns all device memory.  ep_residual_norm_noalloc serves
them: it recomputes the relative FP64 residual of an instance's last solve
using a fixed scratch array inside the library instead of any allocation.
This file checks it against the residual the solver itself reports through
ep_get_stats, on two calls in a row, after steps of an FP32-refined instance.
When the step's last residual came from the solver's residual kernel (the
step took a refinement sweep), the check runs the same nodes per thread in
the same summation order and must agree to 1e-12 relative.  When the step's
first residual already met the tolerance (no sweep), the solver formed it
from its A u history instead of an operator apply; both are float-float
evaluations accurate to about 1e-14 of ||b||, so they must agree to 1e-13
in the relative residual.  It is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _problem():
    return I.slab_ttp06(nx=40, ny=12, nz=8, L=(0.4, 0.12, 0.08), T=5.0)


def test_residual_norm_noalloc_matches_solver_residual():
    inst = ep.Instance(_problem(), precision=ep.EP_PREC_FP32_REFINED)
    strict = 0
    try:
        for steps in (1, 25, 7):
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
                # residual kernel
                assert abs(first - reported) <= 1e-12 * reported
                strict += 1
            else:
                assert abs(first - reported) <= 1e-13
            # the check reads the instance and changes nothing in it
            assert np.array_equal(before, inst.save())
    finally:
        inst.close()
    assert strict >= 1
