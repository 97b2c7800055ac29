"""Single-cell pre-pacing on the GPU (ep_prepace) against the oracle's
(or_prepace), both FP64 with the same semi-implicit scheme: end states
within 1e-9 relative after a few thousand steps; tissue instances start
from a pre-paced table per cell type."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

from .helpers import gpu_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,amp,period,beats", [(ep.EP_MODEL_TTP06, 35.714, 400.0, 3),
                                                    (ep.EP_MODEL_BO, 1.0, 300.0, 3)])
def test_prepace_matches_oracle(model, amp, period, beats):
    cells = np.array([0, 1, 2], dtype=np.uint8)
    g = ep.ep_prepace(model, cells, period, beats, 0.05, amp, 2.0, bdf_order=2)
    for c in cells:
        ref = O.prepace(model, int(c), period, beats, 0.05, amp, 2.0, bdf=2)
        scale = np.maximum(np.abs(ref), 1e-3)
        assert np.max(np.abs(g[c] - ref) / scale) <= 1e-9, (c, np.max(np.abs(g[c] - ref) / scale))


def test_tissue_starts_from_prepaced_states():
    cells = np.array([0, 1, 2], dtype=np.uint8)
    table = ep.ep_prepace(ep.EP_MODEL_TTP06, cells, 400.0, 2, 0.05, 35.714, 2.0)
    m, geo = I.shell_mesh(3, 12, 6)
    f0, s0 = I.shell_helix_fibres(geo)
    i, j, k = I.node_ijk(m)
    cell = I.depth_celltype(i, 3)
    prob = I.problem(m, f0, s0, I.cond_sigma(1.4, 0.5, 0.25), I.TTP06, 0.05, 2, 5.0,
                     [dict(amp=35.714, t0=0.0, dur=2.0)], [(k <= 1).astype(np.uint8)], cell=cell)
    prob["initial"] = table
    inst = ep.Instance(prob, precision=ep.EP_PREC_FP64)
    st = gpu_state(inst)
    inst.close()
    assert np.array_equal(st["u_n"], table[cell, 0])
    assert np.array_equal(st["w_n"], table[cell, 1:].T)
    assert len(set(cell.tolist())) == 3
