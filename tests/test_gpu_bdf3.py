"""GPU parity of BDF order 3 (Sec. 1.2: BDF of order sigma in {1, 2, 3}).

A BDF3 instance keeps a third time level (n-2) of the potential and the
ionic states and, on the refined path, a third level of the float-float
potential and of the A u history.  The first steps ramp the order up
(BDF1, BDF2, then BDF3), each order with its own alpha/dt on the operator.

Tolerances are those of the BDF1/BDF2 parity tests: one step from the same
state within 1e-10 relative (FP64) and 1e-6 (refined); trajectories with
activation times within one time step (FP64) or 0.5 ms (refined).
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

from .helpers import gpu_state, oracle_to_gpu, rel_err, synthetic_front_state

pytestmark = pytest.mark.gpu

FP64, REF = ep.EP_PREC_FP64, ep.EP_PREC_FP32_REFINED
ST = ep.EP_OP_STENCIL


def ttp06(nx=24, ny=9, nz=6, T=20.0, dt=0.05):
    h = 0.01
    return I.slab_ttp06(nx=nx, ny=ny, nz=nz, L=(nx * h, ny * h, nz * h), T=T, bdf=3, dt=dt)


def bo(**kw):
    p = I.slab_bo_small(**kw)
    p["bdf"] = 3
    return p


def _compare(g, sim, precision, tol):
    u_n, u_nm1, w_n, _ = sim.get_state()
    u_nm2, w_nm2 = sim.get_level2()
    assert rel_err(g["u_n"], u_n) <= tol
    # the older levels are the previous steps' values, carried over exactly
    # in FP64 (and to a float-float rounding on the refined path)
    assert rel_err(g["u_nm1"], u_nm1) <= (1e-14 if precision == FP64 else 1e-7)
    assert rel_err(g["u_nm2"], u_nm2) <= (1e-14 if precision == FP64 else 1e-7)
    for s in range(w_n.shape[0]):
        assert rel_err(g["w_n"][s], w_n[s]) <= (1e-5 if precision == REF else tol), s


@pytest.mark.parametrize("kind", ["bo", "ttp06"])
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (REF, 1e-6)])
def test_bdf3_single_step_after_oracle_run(kind, precision, tol):
    """The oracle runs into the upstroke with BDF3, its three levels go into
    the GPU instance, both take one BDF3 step."""
    if kind == "bo":
        prob = bo(nx=12, ny=7, nz=5, L=(0.6, 0.35, 0.25))
        k = 30
    else:
        prob = ttp06()
        k = 60
    sim = O.sim_from_problem(prob)
    sim.step(k)
    inst = ep.Instance(prob, precision=precision)
    try:
        oracle_to_gpu(sim, inst, prob)
        inst.step(1)
        sim.step(1)
        g = gpu_state(inst)
        assert g["bdf_order"] == 3 and g["step"] == k + 1
        _compare(g, sim, precision, tol)
    finally:
        inst.close()


@pytest.mark.parametrize("dims", [(1, 1, 1), (37, 11, 7), (33, 9, 5)])
@pytest.mark.parametrize("precision", [FP64, REF])
def test_bdf3_single_step_synthetic_three_levels(dims, precision):
    """Seeded synthetic front with three distinct levels (the n-2 level is
    shifted further), on meshes smaller than and ragged against the tiles."""
    nx, ny, nz = dims
    prob = ttp06(nx=nx, ny=ny, nz=nz)
    g = I.rng(700 + nx)
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, g)
    u_nm2 = u_nm1 - 0.5 * (u_n - u_nm1) + g.normal(0.0, 1e-3, size=u_n.shape)
    w_nm2 = w_nm1 * (1.0 - 1e-3 * g.normal(size=w_nm1.shape))
    sim = O.sim_from_problem(prob)
    sim.set_state(u_n, u_nm1, w_n, w_nm1, 7)
    sim.set_level2(u_nm2, w_nm2)
    inst = ep.Instance(prob, precision=precision)
    try:
        oracle_to_gpu(sim, inst, prob)
        inst.step(1)
        sim.step(1)
        tol = 1e-10 if precision == FP64 else 1e-6
        _compare(gpu_state(inst), sim, precision, tol)
    finally:
        inst.close()


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (REF, 1e-6)])
def test_bdf3_order_ramp_first_steps(precision, tol):
    """From the initial state: step 1 is BDF1, step 2 BDF2, then BDF3; every
    step's state against the oracle's (each order change re-scales A)."""
    prob = ttp06(T=1.0)
    sim = O.sim_from_problem(prob)
    inst = ep.Instance(prob, precision=precision)
    try:
        for k in range(6):
            inst.step(1)
            sim.step(1)
            g = gpu_state(inst)
            assert g["step"] == k + 1
            assert rel_err(g["u_n"], sim.get_state()[0]) <= tol, k
    finally:
        inst.close()


def test_bdf3_trajectories():
    """BO slab (1386 nodes, 100 ms) in FP64 and refined, TTP06 slab refined
    (25 ms): activation times against the oracle's BDF3 run."""
    prob = bo()
    sim = O.sim_from_problem(prob)
    sim.step(prob["nsteps"])
    at_ref, _ = sim.activation()
    for precision, bound in ((FP64, prob["dt"] + 1e-9), (REF, 0.5)):
        inst = ep.Instance(prob, precision=precision)
        inst.step(prob["nsteps"])
        at = inst.activation_times()
        inst.close()
        assert np.array_equal(np.isnan(at), np.isnan(at_ref))
        assert np.nanmax(np.abs(at - at_ref)) <= bound
    prob = ttp06(nx=40, ny=10, nz=6, T=25.0)
    sim = O.sim_from_problem(prob)
    sim.step(prob["nsteps"])
    at_ref, _ = sim.activation()
    inst = ep.Instance(prob, precision=REF)
    inst.step(prob["nsteps"])
    at = inst.activation_times()
    inst.close()
    assert np.array_equal(np.isnan(at), np.isnan(at_ref))
    assert np.nanmax(np.abs(at - at_ref)) <= 0.5


def test_bdf3_checkpoint_bitwise_and_level_check():
    """A refined BDF3 restart continues bit for bit (three levels and the A u
    history in the exact extension); a BDF2 buffer does not load into a
    BDF3 instance."""
    prob = ttp06(nx=40, ny=12, nz=8, T=5.0)
    a = ep.Instance(prob, precision=REF)
    b = ep.Instance(prob, precision=REF)
    try:
        a.step(20)
        buf = a.save()
        a.step(20)
        b.load(buf)
        b.step(20)
        assert np.array_equal(a.save(), b.save())
        p2 = dict(prob, bdf=2)
        c = ep.Instance(p2, precision=REF)
        try:
            with pytest.raises(ep.EpError) as e:
                b.load(c.save())
            assert e.value.status == ep.EP_EINVAL
        finally:
            c.close()
    finally:
        a.close()
        b.close()


def test_bdf3_history_extrapolation_exact():
    """With a loose tolerance many steps stop at their first residual, whose
    A u_EXT = 3 y_n - 3 y_{n-1} + y_{n-2} comes from the A u history: the
    reported residual equals the one recomputed with the operator.

    Bound: each stored y = A u carries the float-float rounding of a 27-term
    row (~27 x 2^-48 of the row's absolute terms, a few times |y|); the
    extrapolation weighs three of them with |3| + |3| + |1| = 7 (BDF2: 3),
    so the two residual vectors differ by less than ~3e-12 of ||b||, as long
    as no extrapolated value enters a later window (the history restarts
    after such a step).  Both norms are then summed from float squares (per
    thread and block in float, totals in double), in different orders, which
    adds up to ~1e-6 of the norm itself: |reported - recomputed| <= 1e-6
    relres + 5e-12."""
    prob = ttp06(nx=30, ny=8, nz=6, T=30.0)
    inst = ep.Instance(prob, precision=REF, tol=1e-4)
    zero = 0
    try:
        for _ in range(prob["nsteps"]):
            inst.step(1)
            st = inst.stats()
            if st["sweeps"] == 0:
                zero += 1
                exact = ep.ep_residual_norm_noalloc(inst.h)
                assert abs(exact - st["relres"]) <= 1e-6 * exact + 5e-12, (exact, st["relres"])
    finally:
        inst.close()
    assert zero >= 5, zero


def test_bdf3_in_a_batch_matches_alone():
    """A BDF3 instance batched with a BDF2 and a BDF1 one: each as if alone."""
    h = 0.01
    probs = [ttp06(nx=40, ny=9, nz=6, T=3.0),
             I.slab_ttp06(nx=23, ny=11, nz=7, L=(23 * h, 11 * h, 7 * h), T=3.0),
             I.slab_bo_small(nx=12, ny=7, nz=5, L=(0.6, 0.35, 0.25), T=3.0)]
    K = 30
    alone = []
    for p in probs:
        inst = ep.Instance(p, precision=REF, op32=ST)
        inst.step(K)
        alone.append(inst.potential())
        inst.close()
    insts = [ep.Instance(p, precision=REF, op32=ST) for p in probs]
    try:
        ep.ep_step_batch([i.h for i in insts], 10)
        ep.ep_step_batch([i.h for i in insts], K - 10)
        for inst, u in zip(insts, alone):
            assert rel_err(inst.potential(), u) <= 1e-9
            assert inst.stats()["step"] == K
    finally:
        for i in insts:
            i.close()


@pytest.mark.parametrize("bdf", [2, 3])
def test_history_chain_stays_bounded(bdf):
    """With a tolerance so loose that almost every step ends at its first
    pass, extrapolated A u values would feed on each other (BDF3 weighs a
    past level's error by 3 per step); the history restarts after every
    step that ends on an extrapolated value, so the reported residual keeps
    matching the recomputed one over many consecutive steps (bound as in
    the test above)."""
    h = 0.01
    prob = I.slab_ttp06(nx=30, ny=8, nz=6, L=(30 * h, 8 * h, 6 * h), T=10.0, bdf=bdf, dt=0.05)
    inst = ep.Instance(prob, precision=REF, tol=3e-2)
    zero = 0
    try:
        for _ in range(100):
            inst.step(1)
            st = inst.stats()
            if st["sweeps"] == 0:
                zero += 1
                exact = ep.ep_residual_norm_noalloc(inst.h)
                assert abs(exact - st["relres"]) <= 1e-6 * exact + 5e-12, (exact, st["relres"])
    finally:
        inst.close()
    assert zero >= 50, zero
