"""GPU parity of triquadratic (Q2, 27-node) slabs against the oracle's
assembled Q2 matrices (Sec. 1.2: hexahedral elements of any degree).

The GPU path applies the Q2 operators matrix-free (sum factorisation, FP32
inner CG, float-float refinement to ||r|| <= 1e-10 ||b||); the oracle
assembles M and K on 27-node elements in FP64 and solves with CG to 1e-12.
Tolerances are the refined parity tests': one step from the same state
within 1e-6 relative on u (states 1e-5), trajectories with activation times
within 0.5 ms.
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

from .helpers import gpu_state, oracle_to_gpu, rel_err, synthetic_front_state

pytestmark = pytest.mark.gpu

REF = ep.EP_PREC_FP32_REFINED


def q2_ttp06(nx, ny, nz, bdf=2, T=10.0):
    h = 0.02  # element size; nodes every 0.01 cm
    return I.slab_ttp06_q2(nx=nx, ny=ny, nz=nz, L=(nx * h, ny * h, nz * h), T=T, bdf=bdf)


def _one_step(prob, sim):
    inst = ep.Instance(prob, precision=REF)
    try:
        oracle_to_gpu(sim, inst, prob)
        inst.step(1)
        sim.step(1)
        g = gpu_state(inst)
        st = inst.stats()
    finally:
        inst.close()
    return g, st


@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 2, 2), (7, 5, 3), (12, 4, 3)])
def test_q2_single_step_synthetic_front(dims):
    """Seeded front on Q2 slabs of 1 to 144 elements (fewer elements than a
    block's nine, ragged against the blocks)."""
    prob = q2_ttp06(*dims)
    g = I.rng(800 + sum(dims))
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, g)
    sim = O.sim_from_problem(prob)
    sim.set_state(u_n, u_nm1, w_n, w_nm1, 7)
    gg, st = _one_step(prob, sim)
    u, _, w, _ = sim.get_state()
    assert st["relres"] <= 1e-10
    assert rel_err(gg["u_n"], u) <= 1e-6
    for s in range(w.shape[0]):
        assert rel_err(gg["w_n"][s], w[s]) <= 1e-5, s


@pytest.mark.parametrize("bdf", [1, 2, 3])
def test_q2_single_step_after_oracle_run(bdf):
    """The oracle runs into the upstroke on Q2 elements, its state goes into
    the GPU instance, both take one step (every BDF order)."""
    prob = q2_ttp06(8, 3, 2, bdf=bdf)
    sim = O.sim_from_problem(prob)
    sim.step(50)
    gg, _ = _one_step(prob, sim)
    u = sim.get_state()[0]
    assert gg["step"] == 51
    assert rel_err(gg["u_n"], u) <= 1e-6


def test_q2_trajectory_bo_and_ttp06():
    """Bueno-Orovio (40 ms) and TTP06 (15 ms) Q2 slabs from rest: activation
    times within 0.5 ms of the oracle's, the same set of activated nodes.
    (The TTP06 slab is stimulated in x <= 0.04 cm, as slab_ttp06_q2 does.)"""
    tt = q2_ttp06(16, 4, 3, T=15.0)
    for prob in (I.slab_bo_q2(nx=8, ny=4, nz=2, L=(0.8, 0.4, 0.2), T=40.0), tt):
        sim = O.sim_from_problem(prob)
        sim.step(prob["nsteps"])
        at_ref = sim.activation()[0]
        inst = ep.Instance(prob, precision=REF)
        try:
            inst.step(prob["nsteps"])
            at = inst.activation_times()
        finally:
            inst.close()
        assert np.array_equal(np.isnan(at), np.isnan(at_ref))
        assert np.nanmax(at_ref) > 5.0
        assert np.nanmax(np.abs(at - at_ref)) <= 0.5


def test_q2_deterministic_graph_host_and_checkpoint():
    """Q2 steps are bitwise reproducible, the same replayed from the CUDA
    graph and host-driven (per-kernel profiling), and a restart from a
    checkpoint continues bit for bit."""
    prob = q2_ttp06(10, 4, 3, T=5.0)
    a = ep.Instance(prob, precision=REF)
    b = ep.Instance(prob, precision=REF)
    c = ep.Instance(prob, precision=REF)
    try:
        a.step(30)
        b.step(10)
        ep.ep_profile_enable(b.h, True)
        b.step(10)
        prof = ep.ep_profile_read(b.h)
        ep.ep_profile_enable(b.h, False)
        b.step(10)
        assert np.array_equal(a.save(), b.save())
        assert prof["apply32_q2"][0] > 0 and prof["rhs"][0] == 10
        buf = a.save()
        a.step(15)
        c.load(buf)
        c.step(15)
        assert np.array_equal(a.save(), c.save())
    finally:
        for i in (a, b, c):
            i.close()


def test_q2_full_size_slab_step():
    """The 100 x 35 x 15-element Q2 slab (201 x 71 x 31 = 442,401 nodes, the
    node grid of the Q1 benchmark slab) from rest through the stimulus: every
    step refined to 1e-10; the stimulated face depolarises, the far face
    stays at rest (the stimulus covers x <= 0.04 cm)."""
    prob = I.slab_ttp06_q2(T=3.0)
    inst = ep.Instance(prob, precision=REF)
    try:
        for _ in range(prob["nsteps"]):
            inst.step(1)
            assert inst.stats()["relres"] <= 1e-10
        u = inst.potential()
    finally:
        inst.close()
    i, _, _ = I.node_ijk(prob["mesh"])
    assert u[i == 0].min() > -20.0
    assert np.abs(u[i == 200] - (-85.23)).max() < 1.0
