"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances:
  * FP64 path, one step from an identical state: max |du| / max |u| <= 1e-10
    (both solve Eq. (6) to a relative residual of 1e-12; the gap is rounding
    order and the CG stopping point).
  * FP32_REFINED path, one step: the FP64 residual is driven to 1e-10 and the
    ionic update runs in float, so relative 1e-6 on u.
  * Trajectories: activation times within one time step (FP64) and 0.5 ms
    (refined); u within 1 mV outside +-2 steps of each node's upstroke.
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

from .helpers import gpu_state, oracle_to_gpu, rel_err, synthetic_front_state

pytestmark = pytest.mark.gpu

FP64, REF = ep.EP_PREC_FP64, ep.EP_PREC_FP32_REFINED


def small_ttp06(nx=24, ny=9, nz=6, bdf=2, T=20.0, dt=0.05):
    h = 0.01
    p = I.slab_ttp06(nx=nx, ny=ny, nz=nz, L=(nx * h, ny * h, nz * h), T=T, bdf=bdf, dt=dt)
    return p


def one_step_from(prob, sim, precision, **opts):
    inst = ep.Instance(prob, precision=precision, **opts)
    oracle_to_gpu(sim, inst, prob)
    inst.step(1)
    sim.step(1)
    g = gpu_state(inst)
    u_n, _, w_n, _ = sim.get_state()
    at_raw, best = sim.activation_raw()
    inst.close()
    return g, u_n, w_n, best


@pytest.mark.parametrize("kind", ["bo", "ttp06"])
@pytest.mark.parametrize("precision,tol", [(FP64, 1e-10), (REF, 1e-6)])
def test_single_step_after_oracle_run(kind, precision, tol):
    """Run the oracle into the upstroke, inject its state, take one step on
    both sides."""
    if kind == "bo":
        prob = I.slab_bo_small(nx=12, ny=7, nz=5, L=(0.6, 0.35, 0.25))
        k = 30
    else:
        prob = small_ttp06()
        k = 60
    sim = O.sim_from_problem(prob)
    sim.step(k)
    g, u, w, best = one_step_from(prob, sim, precision)
    assert g["step"] == k + 1
    assert rel_err(g["u_n"], u) <= tol
    # FP32 gates (fast float intrinsics) sit a few float ulps from the FP64
    # oracle; FP64 states within the FP64 bound
    for s in range(w.shape[0]):
        assert rel_err(g["w_n"][s], w[s]) <= (1e-5 if precision == REF else tol), s
    assert rel_err(g["best"], best) <= max(tol * 1e3, 1e-7)


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 3), (37, 11, 7), (33, 9, 5), (64, 16, 8)])
@pytest.mark.parametrize("precision", [FP64, REF])
def test_single_step_synthetic_ragged(dims, precision):
    """Seeded synthetic front on meshes that are smaller than, equal to and
    ragged against the kernel tiles."""
    nx, ny, nz = dims
    prob = small_ttp06(nx=nx, ny=ny, nz=nz)
    g = I.rng(500 + nx)
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, g)
    sim = O.sim_from_problem(prob)
    sim.set_state(u_n, u_nm1, w_n, w_nm1, 7)
    gg, u, w, best = one_step_from(prob, sim, precision)
    tol = 1e-10 if precision == FP64 else 1e-6
    assert rel_err(gg["u_n"], u) <= tol


@pytest.mark.parametrize("op32", [ep.EP_OP_MATRIX_FREE, ep.EP_OP_STENCIL])
def test_refined_operators_agree(op32):
    prob = small_ttp06(nx=40, ny=12, nz=8)
    g = I.rng(77)
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, g)
    sim = O.sim_from_problem(prob)
    sim.set_state(u_n, u_nm1, w_n, w_nm1, 3)
    gg, u, w, best = one_step_from(prob, sim, REF, op32=op32)
    assert rel_err(gg["u_n"], u) <= 1e-6


def test_shell_single_step():
    m, geo = I.shell_mesh(3, 16, 8)
    f0, s0 = I.shell_helix_fibres(geo)
    i, j, k = I.node_ijk(m)
    prob = I.problem(m, f0, s0, I.cond_sigma(1.4, 0.5, 0.25), I.TTP06, 0.05, 2, 10.0,
                     [dict(amp=35.714, t0=0.0, dur=2.0)], [(k <= 1).astype(np.uint8)],
                     cell=I.depth_celltype(i, 3))
    g = I.rng(33)
    sim = O.sim_from_problem(prob)
    sim.step(25)
    for precision, tol in ((FP64, 1e-10), (REF, 1e-6)):
        s2 = O.sim_from_problem(prob)
        u_n, u_nm1, w_n, w_nm1 = sim.get_state()
        s2.set_state(u_n, u_nm1, w_n, w_nm1, sim.stepindex)
        gg, u, w, best = one_step_from(prob, s2, precision)
        assert rel_err(gg["u_n"], u) <= tol


def test_trajectory_bo_fp64_and_refined():
    """The Bueno-Orovio slab (1386 nodes, BDF1, 100 ms): FP64 activation
    times equal the oracle's to one step; refined ones within 0.5 ms."""
    prob = I.slab_bo_small()
    sim = O.sim_from_problem(prob)
    sim.step(prob["nsteps"])
    at_ref, _ = sim.activation()
    u_ref = sim.potential()
    for precision in (FP64, REF):
        inst = ep.Instance(prob, precision=precision)
        inst.step(prob["nsteps"])
        at = inst.activation_times()
        u_mv = inst.potential()
        inst.close()
        assert np.array_equal(np.isnan(at), np.isnan(at_ref))
        err = np.nanmax(np.abs(at - at_ref))
        if precision == FP64:
            assert err <= prob["dt"] + 1e-9
            assert np.abs(u_mv - (85.7 * u_ref - 84.0)).max() <= 1e-6
        else:
            assert err <= 0.5
            assert np.abs(u_mv - (85.7 * u_ref - 84.0)).max() <= 1.0


def test_trajectory_ttp06_refined():
    """TTP06 slab 0.4 x 0.1 x 0.06 cm over 25 ms (the wave crosses it):
    activation times within 0.5 ms of the oracle's, u within 1 mV away from
    each node's upstroke, and the conduction velocity along x (plane means
    between 0.25 and 0.75 Lx, and every line of nodes along x) within 1 %."""
    import bench

    prob = small_ttp06(nx=40, ny=10, nz=6, T=25.0)
    sim = O.sim_from_problem(prob)
    inst = ep.Instance(prob, precision=REF)
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
    # u within 1 mV away from each node's upstroke (+-2 steps of its activation)
    for t, u_ref, u in snaps:
        near = np.abs(np.nan_to_num(at_ref, nan=-1e9) - t) <= 2 * prob["dt"]
        assert np.abs(u - u_ref)[~near].max() <= 1.0
    cv_ref = bench.conduction_velocity(prob["mesh"], at_ref)
    cv = bench.conduction_velocity(prob["mesh"], at)
    assert cv_ref is not None and cv is not None
    assert 0.04 < cv_ref[0] < 0.08  # cm/ms: the wave crossed the slab
    assert abs(cv[0] - cv_ref[0]) <= 0.01 * cv_ref[0]
    assert np.max(np.abs(cv[1] - cv_ref[1]) / cv_ref[1]) <= 0.01


def test_deterministic_and_checkpoint_roundtrip():
    prob = small_ttp06(nx=40, ny=12, nz=8, T=5.0)
    runs = []
    for _ in range(2):
        inst = ep.Instance(prob, precision=REF)
        inst.step(40)
        runs.append(inst.save())
        inst.close()
    assert np.array_equal(runs[0], runs[1])
    # restart from a checkpoint reproduces the uninterrupted run bitwise
    a = ep.Instance(prob, precision=REF)
    a.step(20)
    buf = a.save()
    a.step(20)
    b = ep.Instance(prob, precision=REF)
    b.load(buf)
    b.step(20)
    assert np.array_equal(a.save(), b.save())


def test_failure_status_nan_and_noconv():
    prob = small_ttp06(nx=8, ny=4, nz=3)
    inst = ep.Instance(prob, precision=FP64)
    st = ep.state_unpack(inst.save())
    st["u_n"][5] = np.nan  # host-side injection
    inst.load(ep.state_pack(prob["model"], prob["bdf"], prob["dt"], 0, st["u_n"], st["u_nm1"],
                            st["w_n"], st["w_nm1"], st["at"], st["best"]))
    with pytest.raises(ep.EpError) as e:
        inst.step(1)
    assert e.value.status == ep.EP_ENAN
    with pytest.raises(ep.EpError) as e:
        inst.step(1)  # sticky
    assert e.value.status == ep.EP_ENAN
    inst.close()
    inst = ep.Instance(prob, precision=FP64, max_iter=1, tol=1e-14)
    with pytest.raises(ep.EpError) as e:
        inst.step(3)
    assert e.value.status == ep.EP_ENOCONV
    inst.close()


def test_full_size_slab_single_step():
    """The full 200 x 70 x 30 TTP06 slab (442,401 nodes) in the launch
    configuration the benchmark uses: one step from a seeded synthetic front,
    both precisions against the oracle."""
    prob = I.slab_ttp06()
    g = I.rng(900)
    u_n, u_nm1, w_n, w_nm1 = synthetic_front_state(prob, g, width=0.02)
    sim = O.sim_from_problem(prob)
    sim.set_state(u_n, u_nm1, w_n, w_nm1, 5)
    sim.step(1)
    u_ref = sim.get_state()[0]
    for precision, tol in ((FP64, 1e-10), (REF, 1e-6)):
        inst = ep.Instance(prob, precision=precision)
        buf = ep.state_pack(prob["model"], prob["bdf"], prob["dt"], 5, u_n, u_nm1, w_n, w_nm1,
                            np.full(len(u_n), np.nan), np.full(len(u_n), -np.inf))
        inst.load(buf)
        inst.step(1)
        assert rel_err(gpu_state(inst)["u_n"], u_ref) <= tol
        inst.close()


def test_graph_and_host_driven_stepping_agree():
    """Steps replayed from the CUDA graph, steps with host-driven loops and
    per-kernel profiling, and a mix of both give bitwise the same state."""
    prob = small_ttp06(nx=40, ny=12, nz=8, T=5.0)
    a = ep.Instance(prob, precision=REF)
    a.step(30)
    b = ep.Instance(prob, precision=REF)
    b.step(10)
    ep.ep_profile_enable(b.h, True)
    b.step(10)
    prof = ep.ep_profile_read(b.h)
    ep.ep_profile_enable(b.h, False)
    b.step(10)
    assert np.array_equal(a.save(), b.save())
    # the refined step's per-node end runs inside the next ionic kernel
    assert prof["ionic"][0] == 10 and "finish" not in prof
    if "solve32" in prof:  # the whole solve (sweeps, corrections, residuals)
        # in one persistent launch per step
        assert prof["solve32"][0] == 10 and "resid" not in prof and "correct" not in prof
    else:
        apply = prof.get("apply32_mf", prof.get("apply32_stencil"))
        assert apply[0] == prof["update32"][0] > 0
    assert all(ms > 0 for _, ms in prof.values())
    for prec in (FP64,):
        c = ep.Instance(prob, precision=prec)
        c.step(5)
        ep.ep_profile_enable(c.h, True)
        c.step(5)
        ep.ep_profile_enable(c.h, False)
        c.step(5)
        d = ep.Instance(prob, precision=prec)
        d.step(15)
        assert np.array_equal(c.save(), d.save())


def test_steps_converging_at_first_residual_keep_history_exact():
    """With a loose tolerance many steps meet it at their first residual (no
    sweep), whose A u_EXT comes from the A u history; such a step must record
    A u_EXT as its own A u, or the next steps' history would be stale.  After
    every such step the relative residual the solver reports (from the
    history) must equal the one recomputed from scratch (b - A u_n with the
    operator, ep_residual_norm_noalloc): both residuals are float-float, but
    their norms are float sums taken over different thread grids, so they
    agree to ~1e-7 relative (a stale history would be off by O(1))."""
    prob = small_ttp06(nx=30, ny=8, nz=6, T=30.0)
    inst = ep.Instance(prob, precision=REF, tol=1e-5)
    zero_sweeps = 0
    try:
        for _ in range(prob["nsteps"]):
            inst.step(1)
            st = inst.stats()
            if st["sweeps"] == 0:
                zero_sweeps += 1
                exact = ep.ep_residual_norm_noalloc(inst.h)
                assert abs(exact - st["relres"]) <= 1e-6 * exact, (exact, st["relres"])
    finally:
        inst.close()
    assert zero_sweeps >= 5, zero_sweeps


def test_ionic_block_sizes_agree_bitwise():
    """The ionic kernel's block size (64, 128, 256 threads, or the
    create-time autotuner's choice) changes no result: one node per thread
    and no reductions, so the states after 30 steps are bitwise equal."""
    prob = small_ttp06(nx=40, ny=12, nz=8, T=5.0)
    saves, chosen = [], None
    for bt in (64, 128, 256, 0):
        inst = ep.Instance(prob, precision=REF, ionic_threads=bt)
        st = inst.stats()
        assert st["ionic_threads"] == (bt if bt else st["ionic_threads"])
        if bt == 0:
            chosen = st["ionic_threads"]
        inst.step(30)
        saves.append(inst.save())
        inst.close()
    assert chosen in (64, 128, 256)
    for sv in saves[1:]:
        assert np.array_equal(sv, saves[0])


def test_ionic_block_size_option_is_validated():
    prob = small_ttp06(nx=4, ny=3, nz=2)
    with pytest.raises(ep.EpError) as e:
        ep.Instance(prob, precision=REF, ionic_threads=96)
    assert e.value.status == ep.EP_EINVAL
