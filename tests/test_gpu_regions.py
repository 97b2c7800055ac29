"""Subdomains on the GPU (paper Sec. 1.1.2): per-region conductivities and a
non-conductive scar, against the oracle.  Tolerances as in the parity tests:
one step from an identical state 1e-10 (FP64) / 1e-6 (refined) relative;
trajectories: the same activated set, activation times within one step
(FP64) / 0.5 ms (refined)."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

from .helpers import gpu_state, oracle_to_gpu, rel_err, synthetic_front_state

pytestmark = pytest.mark.gpu

FP64, REF = ep.EP_PREC_FP64, ep.EP_PREC_FP32_REFINED


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (REF, 1e-6)])
@pytest.mark.parametrize("dims", [(40, 12, 6), (23, 9, 5)])
def test_single_step_with_scar_and_grey_zone(precision, tol, dims):
    nx, ny, nz = dims
    prob = I.slab_regions(nx=nx, ny=ny, nz=nz)
    g = I.rng(900 + nx)
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, g)
    sim = O.sim_from_problem(prob)
    off = sim.active() == 0
    assert off.any()
    # excluded nodes at a steady level (BDF with zero current keeps it)
    u_nm1[off] = u_n[off]
    w_nm1[:, off] = w_n[:, off]
    sim.set_state(u_n, u_nm1, w_n, w_nm1, 5)
    inst = ep.Instance(prob, precision=precision)
    oracle_to_gpu(sim, inst, prob)
    inst.step(1)
    sim.step(1)
    gs = gpu_state(inst)
    u, _, w, _ = sim.get_state()
    inst.close()
    assert rel_err(gs["u_n"], u) <= tol
    # excluded nodes hold their potential (through the linear solve) and
    # their states (copied) on both sides
    scale = np.abs(u_n).max()
    assert np.abs(u[off] - u_n[off]).max() <= 1e-12 * scale
    assert np.abs(gs["u_n"][off] - u_n[off]).max() <= tol * scale
    assert np.array_equal(w[:, off], w_n[:, off])
    ref_w = w_n[:, off].copy()
    if precision == REF:  # gates in float; concentrations as float-float pairs
        ng = 13
        ref_w[:ng] = ref_w[:ng].astype(np.float32).astype(np.float64)
    assert np.allclose(gs["w_n"][:, off], ref_w, rtol=1e-14, atol=0)


@pytest.mark.parametrize("precision,at_tol", [(FP64, 0.05 + 1e-9), (REF, 0.5)])
def test_scar_wall_blocks_the_wave_like_the_oracle(precision, at_tol):
    prob = I.slab_regions(nx=24, ny=4, nz=3, wall=True, T=20.0, model=I.BO)
    K = int(round(20.0 / prob["dt"]))
    sim = O.sim_from_problem(prob)
    sim.step(K)
    at_ref, _ = sim.activation()
    inst = ep.Instance(prob, precision=precision)
    inst.step(K)
    at = inst.activation_times()
    inst.close()
    assert np.array_equal(np.isnan(at), np.isnan(at_ref))
    x = prob["mesh"]["xyz"][:, 0] / prob["mesh"]["L"][0]
    assert np.isnan(at[x > 0.6]).all() and not np.isnan(at[x < 0.4]).any()
    ok = ~np.isnan(at_ref)
    assert np.abs(at[ok] - at_ref[ok]).max() <= at_tol


def test_regions_refuse_the_matrix_free_operator():
    prob = I.slab_regions(nx=10, ny=4, nz=3)
    with pytest.raises(ep.EpError) as e:
        ep.Instance(prob, precision=REF, op32=ep.EP_OP_MATRIX_FREE)
    assert e.value.status == ep.EP_EUNSUPPORTED
    inst = ep.Instance(prob, precision=REF)  # AUTO picks the stencil operator
    assert inst.stats()["op32"] == ep.EP_OP_STENCIL
    inst.close()


def test_regions_in_a_batch_match_alone():
    probs = [I.slab_regions(nx=20, ny=6, nz=4, T=5.0), I.slab_regions(nx=16, ny=5, nz=3, wall=True, T=5.0)]
    K = 30
    alone = []
    for p in probs:
        i = ep.Instance(p, precision=REF)
        i.step(K)
        alone.append(i.potential())
        i.close()
    insts = [ep.Instance(p, precision=REF) for p in probs]
    try:
        ep.ep_step_batch([i.h for i in insts], K)
        for i, u in zip(insts, alone):
            assert rel_err(i.potential(), u) <= 1e-9
    finally:
        for i in insts:
            i.close()
