"""Applied-current shapes on the GPU against the oracle: Gaussian impulse
profiles (per-node weights) and pulse trains.  Tolerances as in the parity
tests: one step 1e-10 (FP64) / 1e-6 (refined) relative; trajectories: the
same activated set, activation times within one step / 0.5 ms."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

from .helpers import gpu_state, oracle_to_gpu, rel_err, synthetic_front_state

pytestmark = pytest.mark.gpu

FP64, REF = ep.EP_PREC_FP64, ep.EP_PREC_FP32_REFINED


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (REF, 1e-6)])
def test_single_step_with_gaussian_impulses(precision, tol):
    prob = I.slab_gaussian_pacing(nx=30, ny=10, nz=5)
    g = I.rng(321)
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, g)
    sim = O.sim_from_problem(prob)
    sim.set_state(u_n, u_nm1, w_n, w_nm1, 5)  # step 6: both pulses on
    inst = ep.Instance(prob, precision=precision)
    oracle_to_gpu(sim, inst, prob)
    inst.step(1)
    sim.step(1)
    gs = gpu_state(inst)
    inst.close()
    assert rel_err(gs["u_n"], sim.get_state()[0]) <= tol


@pytest.mark.parametrize("precision,at_tol", [(FP64, 0.05 + 1e-9), (REF, 0.5)])
def test_gaussian_pulse_train_trajectory(precision, at_tol):
    prob = I.slab_gaussian_pacing(nx=24, ny=8, nz=3, T=24.0, model=I.BO, period=12.0, dur=1.0)
    K = int(round(24.0 / prob["dt"]))
    sim = O.sim_from_problem(prob)
    sim.step(K)
    at_ref, _ = sim.activation()
    inst = ep.Instance(prob, precision=precision)
    inst.step(K)
    at = inst.activation_times()
    inst.close()
    assert np.array_equal(np.isnan(at), np.isnan(at_ref))
    ok = ~np.isnan(at_ref)
    assert ok.sum() > 0.5 * ok.size
    assert np.abs(at[ok] - at_ref[ok]).max() <= at_tol


def test_weight_validation():
    prob = I.slab_gaussian_pacing(nx=6, ny=4, nz=2)
    prob["pulses"][0] = dict(prob["pulses"][0], weight=np.full(prob["mesh"]["xyz"].shape[0], np.nan))
    with pytest.raises(ep.EpError) as e:
        ep.Instance(prob, precision=REF)
    assert e.value.status == ep.EP_EINVAL


def _element_pulse_problem(kind):
    """A TTP06 problem whose stimulus is a region of elements (I_app
    integrated by the Gauss rule): a corner box of a slab, or the apical rows
    of a small shell."""
    if kind == "slab":
        h = 0.01
        prob = I.slab_ttp06(nx=24, ny=9, nz=6, L=(24 * h, 9 * h, 6 * h), T=12.0)
        elem = I.element_box_mask(prob["mesh"], (0.0, 0.0, 0.0), (0.05, 0.04, 0.03))
    else:
        m, geo = I.shell_mesh(3, 16, 8)
        f0, s0 = I.shell_helix_fibres(geo)
        i, j, k = I.node_ijk(m)
        prob = I.problem(m, f0, s0, I.cond_sigma(1.4, 0.5, 0.25), I.TTP06, 0.05, 2, 12.0,
                         [dict(amp=35.714, t0=0.0, dur=2.0)], [np.zeros(len(i), np.uint8)],
                         cell=I.depth_celltype(i, 3))
        elem = np.zeros(m["hex"].shape[0], np.uint8)
        elem[: 3 * 16 * 2] = 1  # the two apical element rows (k = 0, 1)
    assert 0 < elem.sum() < elem.size
    prob["pulses"] = [dict(prob["pulses"][0], elem=elem)]
    return prob


@pytest.mark.parametrize("kind", ["slab", "shell"])
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (REF, 1e-6)])
def test_element_region_pulse_single_step(kind, precision, tol):
    prob = _element_pulse_problem(kind)
    g = I.rng(333)
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, g)
    sim = O.sim_from_problem(prob)
    sim.set_state(u_n, u_nm1, w_n, w_nm1, 5)  # step 6: the pulse is on
    inst = ep.Instance(prob, precision=precision)
    oracle_to_gpu(sim, inst, prob)
    inst.step(1)
    sim.step(1)
    gs = gpu_state(inst)
    inst.close()
    assert rel_err(gs["u_n"], sim.get_state()[0]) <= tol


@pytest.mark.parametrize("kind", ["slab", "shell"])
@pytest.mark.parametrize("precision,at_tol", [(FP64, 0.05 + 1e-9), (REF, 0.5)])
def test_element_region_pulse_trajectory(kind, precision, at_tol):
    prob = _element_pulse_problem(kind)
    sim = O.sim_from_problem(prob)
    sim.step(prob["nsteps"])
    at_ref, _ = sim.activation()
    inst = ep.Instance(prob, precision=precision)
    inst.step(prob["nsteps"])
    at = inst.activation_times()
    inst.close()
    assert np.array_equal(np.isnan(at), np.isnan(at_ref))
    ok = ~np.isnan(at_ref)
    assert ok.sum() > 0.2 * ok.size
    assert np.abs(at[ok] - at_ref[ok]).max() <= at_tol


def test_element_region_pulse_refused_on_q2():
    prob = I.slab_ttp06_q2(nx=4, ny=3, nz=2, L=(0.08, 0.06, 0.04), T=1.0)
    prob["pulses"] = [dict(prob["pulses"][0], elem=np.ones(4 * 3 * 2, np.uint8))]
    with pytest.raises(ep.EpError) as e:
        ep.Instance(prob, precision=REF)
    assert e.value.status == ep.EP_EUNSUPPORTED
