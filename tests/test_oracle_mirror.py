"""Mirror and rotation symmetry of the oracle's whole simulation (CPU).

A slab with fibres along x, a diffusion tensor diagonal in x, y, z, and a
stimulus box centred in the slab is invariant under each of the reflections
x -> Lx - x, y -> Ly - y, z -> Lz - z; so are the mass and stiffness matrices,
the ionic model and the stimulus, hence the potential and the activation map
at every step.  A wrong node or neighbour index in the assembly, an
off-by-one in the stimulus box or an asymmetric treatment of the boundary
nodes breaks it.  Differences left: the CG's rounding and stopping point
(relative residual 1e-12 per step).
"""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import inputs as I


def _centred_problem(bdf, model):
    nx, ny, nz = 16, 8, 4
    L = (0.8, 0.4, 0.2)
    m = I.slab_mesh(nx, ny, nz, L)
    n = m["xyz"].shape[0]
    f0, s0 = I.uniform_fibres(n)
    mask = I.box_mask(m["xyz"], (0.3, 0.1, 0.05), (0.5, 0.3, 0.15), 0.05)
    if model == I.BO:
        cond, pulse, T = I.cond_D(1.3e-3, 0.45e-3, 0.45e-3), dict(amp=2.0, t0=0.0, dur=1.0, period=0.0), 30.0
    else:
        cond, pulse, T = I.cond_sigma(1.4, 0.5, 0.25), dict(amp=35.714, t0=0.0, dur=2.0, period=0.0), 15.0
    return I.problem(m, f0, s0, cond, model, 0.05, bdf, T, [pulse], [mask], name="centred")


@pytest.mark.parametrize("model,bdf", [(I.BO, 1), (I.BO, 2), (I.TTP06, 2)])
def test_solution_is_mirror_symmetric(model, bdf):
    prob = _centred_problem(bdf, model)
    sim = O.sim_from_problem(prob)
    shape = (5, 9, 17)  # (NZ, NY, NX)
    for _ in range(prob["nsteps"] // 50):
        sim.step(50)
        u = sim.potential().reshape(shape)
        scale = np.abs(u).max()
        for axis in range(3):
            assert np.abs(u - np.flip(u, axis)).max() <= 1e-9 * scale, axis
    at = sim.activation()[0].reshape(shape)
    assert np.isfinite(at).sum() > at.size // 2  # the wave left the box
    for axis in range(3):
        a, b = at, np.flip(at, axis)
        assert np.array_equal(np.isnan(a), np.isnan(b))
        ok = ~np.isnan(a)
        assert np.abs(a[ok] - b[ok]).max() <= prob["dt"] + 1e-12


def test_shell_solution_is_rotation_invariant():
    """The truncated-ellipsoid shell is a surface of revolution meshed with
    the same element column at every azimuth (periodic in phi); the helix
    fibres, the cell types (by depth) and the apical stimulus (whole rings)
    do not depend on phi.  So a rotation by one element column maps the
    problem onto itself and the potential and activation times are the same
    in every column, to the rounding of the nodes' sines and cosines and the
    CG's stopping point (measured 4e-10).  A wrong neighbour across the
    periodic seam or an azimuth-dependent index breaks it."""
    p = I.shell_ttp06(nt=3, nphi=16, nlong=10, T=10.0)
    sim = O.sim_from_problem(p)
    sim.step(p["nsteps"])
    shape = (11, 16, 4)  # (longitudinal, azimuthal, transmural)
    u = sim.potential().reshape(shape)
    assert np.abs(u - u.mean(axis=1, keepdims=True)).max() <= 1e-8 * np.abs(u).max()
    at = sim.activation()[0].reshape(shape)
    assert np.isfinite(at).sum() > 100  # the wave left the stimulated rings
    assert np.array_equal(np.isnan(at), np.isnan(np.roll(at, 1, axis=1)))
    ok = ~np.isnan(at)
    assert np.abs(at - np.roll(at, 1, axis=1))[ok].max() <= p["dt"] + 1e-12


def test_q2_solution_is_mirror_symmetric():
    """The same mirror symmetry on triquadratic (27-node) elements: a BO slab
    of 8 x 4 x 2 Q2 elements (17 x 9 x 5 nodes) with the centred stimulus box
    (measured ~1e-14)."""
    nx, ny, nz = 8, 4, 2
    m = I.slab_mesh_q2(nx, ny, nz, (0.8, 0.4, 0.2))
    n = m["xyz"].shape[0]
    f0, s0 = I.uniform_fibres(n)
    mask = I.box_mask(m["xyz"], (0.3, 0.1, 0.05), (0.5, 0.3, 0.15), 0.05)
    prob = I.problem(m, f0, s0, I.cond_D(1.3e-3, 0.45e-3, 0.45e-3), I.BO, 0.05, 2, 30.0,
                     [dict(amp=2.0, t0=0.0, dur=1.0, period=0.0)], [mask], name="centred_q2")
    sim = O.sim_from_problem(prob)
    sim.step(prob["nsteps"])
    u = sim.potential().reshape(2 * nz + 1, 2 * ny + 1, 2 * nx + 1)
    assert np.isfinite(sim.activation()[0]).all()  # the wave crossed the slab
    for axis in range(3):
        assert np.abs(u - np.flip(u, axis)).max() <= 1e-9 * np.abs(u).max(), axis
