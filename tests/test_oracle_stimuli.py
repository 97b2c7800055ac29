"""Oracle pins for the applied-current shapes (Sec. 1.1.2, Sec. 3.2):
spatial profiles (Gaussian impulses), spherical masks and pulse trains."""
import numpy as np

import oracle.oracle as O
from paper_2308_01651_gb300 import inputs as I


def _passive(n=(4, 3, 2), L=(0.4, 0.3, 0.2), pulses=(), masks=None, dt=0.05, bdf=1):
    m = I.slab_mesh(*n, L)
    nn = m["xyz"].shape[0]
    f0, s0 = I.uniform_fibres(nn)
    if masks is None:
        masks = np.ones((max(len(pulses), 1), nn), dtype=np.uint8)
    return m, O.Sim(m["xyz"], m["hex"], f0, s0, (1e-3, 1e-3, 1e-3), O.PASSIVE, dt, bdf, g=0.0,
                    pulses=list(pulses), masks=masks, act_thr=1.0)


def test_unit_weights_reproduce_the_mask_bitwise():
    p = dict(amp=1.5, t0=0.0, dur=0.5)
    m, a = _passive(pulses=[p])
    nn = m["xyz"].shape[0]
    _, b = _passive(pulses=[dict(p, weight=np.ones(nn))])
    a.step(20)
    b.step(20)
    assert np.array_equal(a.potential(), b.potential())


def test_response_is_linear_in_the_weight():
    """With the passive (linear) membrane the potential is affine in I_app:
    doubling the profile doubles the change from the unstimulated run."""
    m, base = _passive(pulses=[dict(amp=1.0, t0=0.0, dur=0.5)], masks=np.zeros((1, 60), dtype=np.uint8))
    w = I.gaussian_weight(m["xyz"], (0.1, 0.1, 0.0), 0.1)
    runs = []
    for s in (1.0, 2.0):
        _, sim = _passive(pulses=[dict(amp=1.0, t0=0.0, dur=0.5, weight=s * w)])
        sim.step(15)
        runs.append(sim.potential())
    base.step(15)
    u0 = base.potential()
    d1, d2 = runs[0] - u0, runs[1] - u0
    assert np.abs(d2 - 2.0 * d1).max() <= 1e-12 * np.abs(d2).max()
    # the profile peaks where the site is: the largest response sits there
    assert np.argmax(d1) == np.argmin(np.linalg.norm(m["xyz"] - np.array([0.1, 0.1, 0.0]), axis=1))


def test_pulse_train_windows():
    """A train (period in whole steps) is on exactly on steps k0 < m <= k0 + kd
    modulo the period: with a uniform passive response every active step adds
    amp dt, so the final potential counts the active steps."""
    dt, t0, dur, period, steps = 0.05, 0.1, 0.15, 0.5, 37
    m, sim = _passive(pulses=[dict(amp=1.0, t0=t0, dur=dur, period=period)], dt=dt)
    sim.step(steps)
    k0, kd, kp = round(t0 / dt), round(dur / dt), round(period / dt)
    active = sum(1 for mm in range(1, steps + 1) if mm > k0 and (mm - k0 - 1) % kp < kd)
    assert np.allclose(sim.potential(), active * dt, rtol=1e-12, atol=0)


def test_sphere_mask_and_gaussian_profile():
    m = I.slab_mesh(10, 10, 2, (1.0, 1.0, 0.2))
    c = (0.5, 0.5, 0.0)
    mk = I.sphere_mask(m["xyz"], c, 0.2, h=0.1)
    d = np.linalg.norm(m["xyz"] - np.array(c), axis=1)
    assert np.array_equal(mk.astype(bool), d <= 0.2 + 1e-10)
    w = I.gaussian_weight(m["xyz"], c, 0.1)
    assert np.allclose(w, np.exp(-d ** 2 / 0.02))
    assert w.max() == 1.0 and abs(w[np.argmin(d)] - 1.0) == 0.0


# ---- applied current on a region of elements (Gauss-point integration) ----
# The vector arising from I_app (Sec. 1.2, Eq. (6)) for I_app = amp on a
# region of whole elements: f_j = amp * sum over the region's elements of
# int_e phi_j.  Pins: on a box element, int_e phi_j = |e| / 8 for each of its
# 8 nodes (trilinear basis, exact); f sums to amp times the region's volume;
# with every element in the region f is the mass matrix's row sums M 1.

def test_element_region_vector_on_a_slab_box():
    nx, ny, nz, L = 6, 4, 3, (0.6, 0.4, 0.3)
    m = I.slab_mesh(nx, ny, nz, L)
    ei, ej, ek = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    order = np.argsort((ei + nx * (ej + ny * ek)).ravel())
    ijk = np.stack([ei.ravel()[order], ej.ravel()[order], ek.ravel()[order]], axis=1)
    elem = ((ijk[:, 0] < 2) & (ijk[:, 1] < 2) & (ijk[:, 2] < 1)).astype(np.uint8)
    f = O.element_region_vector(m["xyz"], m["hex"], elem)
    vol_e = 0.1 ** 3
    assert abs(f.sum() - 4 * vol_e) <= 1e-15
    count = np.zeros(m["xyz"].shape[0])
    for e in np.nonzero(elem)[0]:
        count[m["hex"][e]] += 1
    assert np.abs(f - count * vol_e / 8.0).max() <= 1e-18
    # the corner node belongs to one region element, the centre node of the
    # 2 x 2 x 1 block to four
    assert np.isclose(f[0], vol_e / 8.0, rtol=1e-14, atol=0)


def test_element_region_vector_of_all_elements_is_mass_row_sums():
    for mesh in (I.slab_mesh(5, 3, 2, (0.5, 0.3, 0.2)), I.shell_mesh(3, 12, 5)[0]):
        nn = mesh["xyz"].shape[0]
        f0, s0 = I.uniform_fibres(nn)
        sim = O.Sim(mesh["xyz"], mesh["hex"], f0, s0, (1e-3, 1e-3, 1e-3), O.PASSIVE, 0.05, 1, g=0.0,
                    pulses=[], masks=None, act_thr=1.0)
        rowptr, col, mv, kv = sim.matrices()
        rows = np.add.reduceat(mv, rowptr[:-1])
        f = O.element_region_vector(mesh["xyz"], mesh["hex"], np.ones(mesh["hex"].shape[0], np.uint8))
        assert np.abs(f - rows).max() <= 1e-14 * rows.max()
        assert abs(f.sum() - mv.sum()) <= 1e-13 * mv.sum()


def test_element_region_pulse_equals_nodal_pulse_on_the_whole_domain():
    """I_app = amp everywhere: the Gauss-integrated vector is M 1, exactly the
    nodal reading's M (amp 1), so both runs agree to rounding."""
    p = dict(amp=1.5, t0=0.0, dur=0.5)
    m, a = _passive(pulses=[p])
    ne = m["hex"].shape[0]
    _, b = _passive(pulses=[dict(p, elem=np.ones(ne, np.uint8))], masks=np.zeros((1, 60), np.uint8))
    a.step(20)
    b.step(20)
    assert np.abs(a.potential() - b.potential()).max() <= 1e-13 * np.abs(a.potential()).max()
    assert np.abs(a.potential()).max() > 0.1


def test_element_region_pulse_is_local():
    """A region of one corner element drives the nodes of that element more
    than any other and leaves a passive slab mirror-symmetric about the
    element's diagonal plane x = y (equal spacing)."""
    m = I.slab_mesh(4, 4, 2, (0.4, 0.4, 0.2))
    nn = m["xyz"].shape[0]
    f0, s0 = I.uniform_fibres(nn, f=(0.0, 0.0, 1.0), s=(1.0, 0.0, 0.0))
    elem = np.zeros(m["hex"].shape[0], np.uint8)
    elem[0] = 1
    sim = O.Sim(m["xyz"], m["hex"], f0, s0, (1e-3, 1e-3, 1e-3), O.PASSIVE, 0.05, 1, g=0.0,
                pulses=[dict(amp=1.0, t0=0.0, dur=0.5, elem=elem)], masks=np.zeros((1, nn), np.uint8),
                act_thr=1.0)
    sim.step(10)
    u = sim.potential()
    x, y, z = m["xyz"].T
    assert np.argmax(u) == 0
    swap = np.array([np.argmin(np.abs(x - y[i]) + np.abs(y - x[i]) + np.abs(z - z[i])) for i in range(nn)])
    assert np.abs(u - u[swap]).max() <= 1e-14 * u.max()
