"""Values the paper prints (tests/golden/, each fixture with its citation)
against what the oracle and the synthetic workloads use (CPU).

The paper prints the TTP06 epicardial initial conditions and the N-version
slab's conductivities and applied current (Sec. 3.2.1); both sides of the
parity tests start from them.  The activation times it reports there are
checked on the GPU (tests/test_gpu_nversion.py) against the same fixture.
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import inputs as I

from .helpers import golden


@pytest.mark.parametrize("cell", [O.EPI, O.ENDO, O.MID])
def test_oracle_ttp06_initial_state_is_the_papers(cell):
    """Every TTP06 cell type starts from the paper's epicardial initial
    conditions (the paper prints no others), state by state."""
    g = golden("ttp06_epi_initial_state.json")
    u0, w0 = O.initial(O.TTP06, cell)
    assert u0 == g["V_mV"]
    assert len(w0) == len(g["state_order"]) == 18
    for k, name in enumerate(g["state_order"]):
        assert w0[k] == g["states"][name], (name, w0[k], g["states"][name])


def test_nversion_workload_matches_the_paper():
    """The N-version workload's diffusivities are the printed conductivities
    (m^2/s) in cm^2/ms (x 10), its pulse the printed 35.714 V/s (= mV/ms) for
    2 ms, on the nodes of the 1.5 mm cube at one corner."""
    g = golden("nversion_slab.json")
    prob = I.nversion(dx=0.05, dt=0.005, T=1.0)
    c = prob["cond"]
    assert c["is_D"]
    sig = g["conductivity_m2_per_s"]
    want = (sig["longitudinal"] * 10.0, sig["transversal"] * 10.0, sig["normal"] * 10.0)
    assert np.allclose(c["sigma"], want, rtol=1e-14, atol=0.0)
    (p,) = prob["pulses"]
    st = g["stimulus"]
    assert p["amp"] == st["amplitude_V_per_s"]
    assert p["dur"] == pytest.approx(st["duration_s"] * 1e3, rel=1e-15)
    xyz = prob["mesh"]["xyz"]
    inside = prob["masks"][0].astype(bool)
    edge_cm = st["cube_edge_m"] * 1e2
    assert inside[np.argmin(np.linalg.norm(xyz, axis=1))]  # the corner node
    assert xyz[inside].max() <= edge_cm + 1e-9
    cube = np.all(xyz <= edge_cm + 1e-9, axis=1)
    assert np.array_equal(inside, cube)
