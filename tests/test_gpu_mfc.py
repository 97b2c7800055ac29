"""The matrix-free FP32 operator on curved (shell) meshes: element
coordinates and fibre frames staged by TMA, the Jacobian, the diffusion
tensor and the mass term formed per Gauss point (Sec. 1.2, Eq. (6) with D of
Eq. (3)).  Checked through the C ABI against the FP64 oracle (one step from a
seeded synthetic front on shells smaller than, equal to and ragged against
the kernel's 8 x 8 tiles, relative 1e-6 on u; a trajectory's activation
times within 0.5 ms), against the stored-stencil operator, and for bitwise
reproducibility (two runs, graph-driven against host-driven stepping, a
checkpoint restart)."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

from .helpers import gpu_state, rel_err, synthetic_front_state

pytestmark = pytest.mark.gpu

REF, MF, ST = ep.EP_PREC_FP32_REFINED, ep.EP_OP_MATRIX_FREE, ep.EP_OP_STENCIL


def shell_problem(nt, nphi, nlong, T=10.0, stim_rows=1):
    m, geo = I.shell_mesh(nt, nphi, nlong)
    f0, s0 = I.shell_helix_fibres(geo)
    i, j, k = I.node_ijk(m)
    return I.problem(m, f0, s0, I.cond_sigma(1.4, 0.5, 0.25), I.TTP06, 0.05, 2, T,
                     [dict(amp=35.714, t0=0.0, dur=2.0)], [(k <= stim_rows).astype(np.uint8)],
                     cell=I.depth_celltype(i, nt))


def step_from_state(prob, state, op32, precision=REF):
    u_n, u_nm1, w_n, w_nm1 = state
    N = len(u_n)
    inst = ep.Instance(prob, precision=precision, op32=op32)
    inst.load(ep.state_pack(prob["model"], prob["bdf"], prob["dt"], 7, u_n, u_nm1, w_n, w_nm1,
                            np.full(N, np.nan), np.full(N, -np.inf)))
    inst.step(1)
    st = inst.stats()
    u = gpu_state(inst)["u_n"]
    inst.close()
    return u, st


@pytest.mark.parametrize("dims", [(1, 3, 1), (3, 16, 8), (5, 17, 9), (7, 9, 3), (20, 24, 12), (31, 10, 7)])
def test_mfc_single_step_against_oracle(dims):
    prob = shell_problem(*dims)
    g = I.rng(700 + dims[0] + dims[1])
    state = synthetic_front_state(prob, g)
    sim = O.sim_from_problem(prob)
    sim.set_state(*state, 7)
    sim.step(1)
    u_ref = sim.get_state()[0]
    u, st = step_from_state(prob, state, MF)
    assert st["op32"] == MF
    assert st["relres"] <= 1e-10
    assert rel_err(u, u_ref) <= 1e-6


def test_mfc_agrees_with_stencil_operator():
    prob = shell_problem(6, 40, 20)
    state = synthetic_front_state(prob, I.rng(711))
    u_mf, st_mf = step_from_state(prob, state, MF)
    u_st, st_st = step_from_state(prob, state, ST)
    assert st_mf["op32"] == MF and st_st["op32"] == ST
    # both refine to 1e-10 of ||b||; the inner operators differ in float rounding
    assert rel_err(u_mf, u_st) <= 1e-8


def test_mfc_trajectory_against_oracle():
    prob = shell_problem(4, 24, 16, T=20.0, stim_rows=2)
    sim = O.sim_from_problem(prob)
    sim.step(prob["nsteps"])
    at_ref, _ = sim.activation()
    inst = ep.Instance(prob, precision=REF, op32=MF)
    inst.step(prob["nsteps"])
    at = inst.activation_times()
    inst.close()
    assert np.isfinite(at_ref).sum() > 0.2 * len(at_ref)
    assert np.array_equal(np.isnan(at), np.isnan(at_ref))
    assert np.nanmax(np.abs(at - at_ref)) <= 0.5


def test_mfc_reproducible_graph_host_checkpoint():
    prob = shell_problem(5, 20, 10, T=5.0, stim_rows=2)
    runs = []
    for _ in range(2):
        inst = ep.Instance(prob, precision=REF, op32=MF)
        inst.step(30)
        runs.append(inst.save())
        inst.close()
    assert np.array_equal(runs[0], runs[1])
    a = ep.Instance(prob, precision=REF, op32=MF)
    a.step(10)
    ep.ep_profile_enable(a.h, True)
    a.step(10)
    prof = ep.ep_profile_read(a.h)
    ep.ep_profile_enable(a.h, False)
    buf = a.save()
    a.step(10)
    assert np.array_equal(a.save(), runs[0])
    assert prof["apply32_mf"][0] == prof["update32"][0] > 0
    b = ep.Instance(prob, precision=REF, op32=MF)
    b.load(buf)
    b.step(10)
    assert np.array_equal(b.save(), runs[0])
    a.close()
    b.close()


def test_mfc_autotune_on_shells_reports_both():
    prob = shell_problem(4, 16, 8)
    inst = ep.Instance(prob, precision=REF, op32=ep.EP_OP_AUTO)
    st = inst.stats()
    inst.close()
    assert st["tune_us_mf"] > 0 and st["tune_us_stencil"] > 0
    assert st["op32"] in (MF, ST)
