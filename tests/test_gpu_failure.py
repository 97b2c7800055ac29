"""Failure detection on the GPU without a fault: the persistent solver's
grid barrier waits a bounded time for blocks that never arrive, records
EP_ETIMEOUT and returns; the CUDA context stays usable."""
import numpy as np
import pytest

from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_bounded_barrier_wait_times_out_and_context_survives():
    assert ep.ep_selftest_barrier_timeout() == ep.EP_ETIMEOUT
    assert ep.ep_selftest_barrier_timeout() == ep.EP_ETIMEOUT  # repeatable
    # the context still runs a refined solve normally
    prob = I.slab_ttp06(nx=16, ny=6, nz=4, L=(0.16, 0.06, 0.04), T=1.0)
    inst = ep.Instance(prob, precision=ep.EP_PREC_FP32_REFINED)
    try:
        inst.step(10)
        st = inst.stats()
        assert st["step"] == 10 and st["relres"] <= 1e-10
        assert np.isfinite(inst.potential()).all()
    finally:
        inst.close()
