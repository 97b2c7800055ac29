"""The oracle's parallel loops give the same bits on any number of threads.

The oracle splits nodes (ionic step) and matrix rows (products) among OpenMP
threads and sums dot products in fixed chunks of consecutive terms, then the
chunks in order, so the thread count changes neither the summation order nor
the result.  Checked on a TTP06 slab of more than one dot-product chunk
(11,193 nodes), 30 steps through the stimulus and the first upstrokes.
"""
import numpy as np

import oracle.oracle as O
from paper_2308_01651_gb300 import inputs as I


def _run(threads):
    prev = O.set_threads(0)
    try:
        O.set_threads(threads)
        prob = I.slab_ttp06(nx=40, ny=20, nz=12, L=(0.4, 0.2, 0.12), T=1.5)
        sim = O.sim_from_problem(prob)
        sim.step(prob["nsteps"])
        return sim.potential(), sim.activation()[0], sim.last_iters
    finally:
        O.set_threads(prev)


def test_thread_count_does_not_change_the_result():
    u1, at1, it1 = _run(1)
    u4, at4, it4 = _run(4)
    assert u1.shape[0] == 41 * 21 * 13
    assert np.array_equal(u1, u4)
    assert np.array_equal(at1, at4, equal_nan=True)
    assert it1 == it4
    assert np.isfinite(at1).any()
