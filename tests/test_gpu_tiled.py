"""The persistent solve's operator apply on tiles staged in shared memory by
bulk copies (options.solve_tiles = 2) against the node-parallel apply
(solve_tiles = 1) and the FP64 oracle.

The cases cover the tile geometry: tiles one row high with one plane each
(16 x 9 tiles of a 4 x 16 x 9-node periodic shell: every tile reads a seam
row or a plane outside the mesh), tiles ten rows high -- the last one four --
over ranges of one or two planes (a 9 x 64 x 41-node shell), and slabs,
whose rows and planes outside the mesh read zeros.

Tolerances: the two applies form the same rows (the same bits); the dot
products group their float partials by tile instead of by node stride, so
the CG scalars round differently and the two refinements stop at different
iterates within the 1e-10 residual target.  One step from the same state:
potentials within 1e-8 relative.  Over 200 steps through the stimulus and
the upstroke the ionic model carries those differences along (4.5e-8
relative measured on the small shell): potentials within the refined path's
one-step parity tolerance against the oracle, 1e-6 relative, activation
times within one step.  Against the oracle as the other refined
trajectories: activation times within 0.5 ms, u within 1 mV away from each
node's upstroke, one step within 1e-6 relative.
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

from .helpers import gpu_state, rel_err, synthetic_front_state

pytestmark = pytest.mark.gpu

REF = ep.EP_PREC_FP32_REFINED


def _shell(nt, nphi, nlong, T):
    m, geo = I.shell_mesh(nt, nphi, nlong)
    f0, s0 = I.shell_helix_fibres(geo)
    i, j, k = I.node_ijk(m)
    return I.problem(m, f0, s0, I.cond_sigma(1.4, 0.5, 0.25), I.TTP06, 0.05, 2, T,
                     [dict(amp=35.714, t0=0.0, dur=2.0)], [(k <= 1).astype(np.uint8)],
                     cell=I.depth_celltype(i, nt))


def _run(prob, steps, tiles):
    inst = ep.Instance(prob, precision=REF, op32=ep.EP_OP_STENCIL, solve_tiles=tiles)
    st0 = inst.stats()
    inst.step(steps)
    out = inst.potential(), inst.activation_times(), inst.stats()
    inst.close()
    assert st0["solve_tiles"] == (1 if tiles == 2 else 0)
    return out


def _close(a, b, dt):
    (u1, at1, s1), (u2, at2, s2) = a, b
    assert s1["relres"] <= 1e-10 and s2["relres"] <= 1e-10
    assert rel_err(u1, u2) <= 1e-6
    assert np.array_equal(np.isnan(at1), np.isnan(at2))
    ok = ~np.isnan(at1)
    if ok.any():
        assert np.abs(at1[ok] - at2[ok]).max() <= dt + 1e-12


@pytest.mark.parametrize("dims", [(3, 16, 8), (8, 64, 40)])
def test_shell_tiles_match_node_parallel(dims):
    """(3, 16, 8): 4 x 16 x 9 nodes, 16 x 9 tiles of one row and one plane;
    (8, 64, 40): 9 x 64 x 41 nodes, 7 x 21 tiles of ten rows (the last four)
    and one or two planes.  200 steps (10 ms): stimulus and upstroke."""
    prob = _shell(*dims, T=10.0)
    _close(_run(prob, 200, 2), _run(prob, 200, 1), prob["dt"])


def test_slab_tiles_match_node_parallel():
    h = 0.01
    prob = I.slab_ttp06(nx=24, ny=9, nz=6, L=(24 * h, 9 * h, 6 * h), T=10.0)
    _close(_run(prob, 200, 2), _run(prob, 200, 1), prob["dt"])


def test_tiled_trajectory_against_oracle():
    """TTP06 slab 0.4 x 0.1 x 0.06 cm over 25 ms (the wave crosses it), the
    tiled solve against the oracle."""
    h = 0.01
    prob = I.slab_ttp06(nx=40, ny=10, nz=6, L=(40 * h, 10 * h, 6 * h), T=25.0)
    sim = O.sim_from_problem(prob)
    inst = ep.Instance(prob, precision=REF, op32=ep.EP_OP_STENCIL, solve_tiles=2)
    assert inst.stats()["solve_tiles"] == 1
    snaps = []
    for s in range(prob["nsteps"]):
        sim.step(1)
        inst.step(1)
        if s % 10 == 9:
            snaps.append(((s + 1) * prob["dt"], sim.potential(), inst.potential()))
    at_ref, _ = sim.activation()
    at = inst.activation_times()
    inst.close()
    assert np.array_equal(np.isnan(at), np.isnan(at_ref))
    assert np.nanmax(np.abs(at - at_ref)) <= 0.5
    for t, u_ref, u in snaps:
        near = np.abs(np.nan_to_num(at_ref, nan=-1e9) - t) <= 2 * prob["dt"]
        assert np.abs(u - u_ref)[~near].max() <= 1.0


def test_tiled_and_node_parallel_one_step_agree():
    """One step from the same synthetic front: the two applies' solutions
    differ only within the refinement's tolerance."""
    prob = _shell(8, 64, 40, T=10.0)
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, I.rng(78), width=0.2)
    N = len(u_n)
    buf = ep.state_pack(prob["model"], prob["bdf"], prob["dt"], 7, u_n, u_nm1, w_n, w_nm1,
                        np.full(N, np.nan), np.full(N, -np.inf))
    out = []
    for tiles in (2, 1):
        inst = ep.Instance(prob, precision=REF, op32=ep.EP_OP_STENCIL, solve_tiles=tiles)
        inst.load(buf)
        inst.step(1)
        out.append(gpu_state(inst)["u_n"])
        inst.close()
    assert rel_err(out[0], out[1]) <= 1e-8


def test_tiled_shell_single_step_against_oracle():
    """One step from a seeded synthetic front on the (8, 64, 40) shell."""
    prob = _shell(8, 64, 40, T=10.0)
    g = I.rng(77)
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, g, width=0.2)
    sim = O.sim_from_problem(prob)
    sim.set_state(u_n, u_nm1, w_n, w_nm1, 7)
    sim.step(1)
    u_ref = sim.get_state()[0]
    N = len(u_n)
    inst = ep.Instance(prob, precision=REF, op32=ep.EP_OP_STENCIL, solve_tiles=2)
    inst.load(ep.state_pack(prob["model"], prob["bdf"], prob["dt"], 7, u_n, u_nm1, w_n, w_nm1,
                            np.full(N, np.nan), np.full(N, -np.inf)))
    inst.step(1)
    st = inst.stats()
    err = rel_err(gpu_state(inst)["u_n"], u_ref)
    inst.close()
    assert st["solve_tiles"] == 1 and st["relres"] <= 1e-10
    assert err <= 1e-6
