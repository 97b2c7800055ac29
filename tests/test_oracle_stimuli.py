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
