"""Pins of the oracle's monodomain time discretisation (paper Sec. 1.2,
Eqs. (5)-(6)), of the stimulus window and of the activation-time rule.

  * BDF order on a manufactured solution: a passive membrane I_ion = g u,
    u = e^{-t} cos(pi x/Lx) cos(pi y/Ly) cos(pi z/Lz) (homogeneous Neumann,
    Eq. (2)), isotropic D, forcing I_app = (g - 1 + D pi^2 sum 1/L^2) u at the
    nodes.  Errors against a dt/64 run on the same mesh fall with slope 1 for
    BDF1 and 2 for BDF2 (the IMEX extrapolation keeps the order).
  * A spatially uniform pulse with g = 0 leaves u uniform (K 1 = 0), so each
    active step adds dt * amp: the pulse is active for exactly round(dur/dt)
    steps starting at step round(t0/dt) + 1.
  * A second one-step pulse inside the first makes one step's slope the
    largest, which fixes the activation time.
"""
import math

import numpy as np
import pytest

import oracle.oracle as O
from paper_2308_01651_gb300 import inputs as I


def manufactured_run(bdf, dt, T=1.0, n=(6, 4, 3), L=(0.6, 0.4, 0.3), D=1e-2, g=0.5, start=None, t0=0.0):
    """start: None (the exact u at t = 0, the scheme's start-up ramp), or
    (u(t0), u(t0 - dt), u(t0 - 2 dt)) of the discrete problem, continued at
    full order from t0."""
    m = I.slab_mesh(*n, L)
    xyz = m["xyz"]
    f0, s0 = I.uniform_fibres(xyz.shape[0])
    S = O.Sim(xyz, m["hex"], f0, s0, (D, D, D), O.PASSIVE, dt, bdf, g=g, tol=1e-13)
    shape = np.cos(math.pi * xyz[:, 0] / L[0]) * np.cos(math.pi * xyz[:, 1] / L[1]) * np.cos(math.pi * xyz[:, 2] / L[2])
    lam = math.pi ** 2 * sum(1.0 / l ** 2 for l in L)
    z = np.zeros((0, xyz.shape[0]))
    if start is None:
        S.set_state(shape, shape * math.exp(dt), z, z, 0)
    else:
        S.set_state(start[0], start[1], z, z, 2)
        S.set_level2(start[2], z)
    for k in range(int(round((T - t0) / dt))):
        t1 = t0 + (k + 1) * dt
        S.set_iapp_extra((g - 1.0 + D * lam) * math.exp(-t1) * shape)
        S.step(1)
    return S.potential()


@pytest.mark.parametrize("bdf,lo,hi", [(1, 0.85, 1.15), (2, 1.85, 2.2)])
def test_bdf_order_manufactured(bdf, lo, hi):
    dts = [0.1, 0.05, 0.025]
    ref = manufactured_run(bdf, dts[-1] / 64)
    errs = [np.abs(manufactured_run(bdf, dt) - ref).max() for dt in dts]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(lo < s < hi for s in slopes), (errs, slopes)


def test_bdf3_order_manufactured():
    """BDF3 (alpha = 11/6, f_BDF = 3 f_n - 3/2 f_{n-1} + 1/3 f_{n-2}, f_EXT =
    3 f_n - 3 f_{n-1} + f_{n-2}) from an exact three-level history converges
    at order 3; with its start-up ramp (a BDF1 and a BDF2 step) the first
    steps' larger errors remain, so the slope drops towards 2 but the error
    stays below BDF2's."""
    T, t0 = 1.0, 0.2
    fine = 0.1 / 2048
    ref = manufactured_run(3, fine, T=T)
    errs = []
    for dt in (0.1, 0.05, 0.025):
        # the discrete solution at t0 - 2 dt, t0 - dt, t0 from a much finer run
        hist = [manufactured_run(3, fine, T=t0 - j * dt) for j in (0, 1, 2)]
        errs.append(np.abs(manufactured_run(3, dt, T=T, start=hist, t0=t0) - ref).max())
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(2.7 < s < 3.4 for s in slopes), (errs, slopes)
    ramp3 = np.abs(manufactured_run(3, 0.05) - manufactured_run(3, 0.05 / 64)).max()
    bdf2 = np.abs(manufactured_run(2, 0.05) - manufactured_run(2, 0.05 / 64)).max()
    assert ramp3 < bdf2


@pytest.mark.parametrize("t0,dur,dt", [(0.0, 1.0, 0.05), (0.3, 0.2, 0.1), (1.0, 2.0, 0.05)])
def test_stimulus_window_and_activation(t0, dur, dt):
    """Pulse 1 (amplitude 2) covers the window; pulse 2 (amplitude 1) adds one
    step inside it, so the slope peaks on exactly that step."""
    m = I.slab_mesh(3, 2, 2, (0.3, 0.2, 0.2))
    n = m["xyz"].shape[0]
    f0, s0 = I.uniform_fibres(n)
    k0, kd = round(t0 / dt), round(dur / dt)
    j = kd // 2
    S = O.Sim(m["xyz"], m["hex"], f0, s0, (1e-3, 1e-3, 1e-3), O.PASSIVE, dt, 1, g=0.0,
              pulses=[dict(amp=2.0, t0=t0, dur=dur), dict(amp=1.0, t0=t0 + j * dt, dur=dt)],
              masks=np.ones((2, n), dtype=np.uint8), act_thr=1.0)
    S.step(k0 + kd + 5)
    u = S.potential()
    assert np.allclose(u, (2.0 * kd + 1.0) * dt, rtol=1e-10, atol=0)
    at, best = S.activation()
    assert np.allclose(at, (k0 + j + 1) * dt, rtol=0, atol=1e-12)
    assert np.allclose(best, 3.0 * dt, rtol=1e-10)


def test_manufactured_solution_converges_in_space():
    """With a small time step the discrete solution approaches the exact
    e^{-T} cos cos cos at second order in h; a wrong sign or factor on the
    ionic, applied-current or history term of Eq. (6) would leave an O(1) gap."""
    T, L = 0.5, (0.6, 0.4, 0.3)
    errs = []
    for n in [(6, 4, 3), (12, 8, 6)]:
        u = manufactured_run(2, 0.005, T=T, n=n, L=L)
        m = I.slab_mesh(*n, L)
        xyz = m["xyz"]
        exact = math.exp(-T) * np.cos(math.pi * xyz[:, 0] / L[0]) * np.cos(math.pi * xyz[:, 1] / L[1]) \
            * np.cos(math.pi * xyz[:, 2] / L[2])
        errs.append(np.abs(u - exact).max() / np.abs(exact).max())
    assert errs[0] < 0.1
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def _eigen_recurrence(bdf, lam, g, dt, nsteps):
    """Amplitudes a_n of a discrete eigenmode (K v = lam M v) under the IMEX
    step: (alpha/dt + lam) a_{n+1} = a_BDF/dt - g a_EXT, the order ramping
    1 -> 2 -> 3 over the first steps."""
    a = [1.0]
    for n in range(nsteps):
        order = min(bdf, n + 1)
        x = a[-1]
        y = a[-2] if len(a) > 1 else 0.0
        z = a[-3] if len(a) > 2 else 0.0
        if order == 1:
            alpha, aB, aE = 1.0, x, x
        elif order == 2:
            alpha, aB, aE = 1.5, 2 * x - 0.5 * y, 2 * x - y
        else:
            alpha, aB, aE = 11.0 / 6.0, 3 * x - 1.5 * y + z / 3.0, 3 * x - 3 * y + z
        a.append((aB / dt - g * aE) / (alpha / dt + lam))
    return np.array(a)


@pytest.mark.parametrize("bdf", [1, 2, 3])
def test_discrete_eigenmode_closed_form(bdf):
    """On a box of Q1 elements the nodal vector v = cos(pi x/Lx) cos(pi y/Ly)
    cos(pi z/Lz) is an exact eigenvector of the Neumann problem, K v = lam M v
    with lam = sum_d D_d (6/h_d^2)(1 - cos t_d)/(2 + cos t_d), t_d = pi h_d/L_d
    (the 1-D consistent mass h/6 [1 4 1] and stiffness 1/h [-1 2 -1], and
    their halved boundary rows, act on cos(pi i h/L) by those factors).  With
    a passive membrane I_ion = g u, anisotropic diagonal D, no stimulus, the
    whole IMEX step on that mode is a scalar recurrence, written out above:
    every step of the oracle must reproduce it (M, K, alpha, u_BDF, the
    explicit u_EXT in the ionic term, the order ramp)."""
    n, L = (7, 5, 3), (0.7, 0.4, 0.45)
    D = (2e-2, 0.7e-2, 0.4e-2)
    g, dt, steps = 0.8, 0.05, 12
    m = I.slab_mesh(*n, L)
    xyz = m["xyz"]
    f0, s0 = I.uniform_fibres(xyz.shape[0])
    S = O.Sim(xyz, m["hex"], f0, s0, D, O.PASSIVE, dt, bdf, g=g, tol=1e-14)
    v = np.cos(math.pi * xyz[:, 0] / L[0]) * np.cos(math.pi * xyz[:, 1] / L[1]) * np.cos(math.pi * xyz[:, 2] / L[2])
    lam = 0.0
    for d in range(3):
        h = L[d] / n[d]
        t = math.pi * h / L[d]
        lam += D[d] * (6.0 / h ** 2) * (1.0 - math.cos(t)) / (2.0 + math.cos(t))
    z = np.zeros((0, xyz.shape[0]))
    S.set_state(v, v, z, z, 0)
    amp = _eigen_recurrence(bdf, lam, g, dt, steps)
    for k in range(1, steps + 1):
        S.step(1)
        assert np.abs(S.potential() - amp[k] * v).max() <= 1e-11 * np.abs(amp[k]), k
    # the mode decays, and not at the continuous rate (the discrete lam is
    # what the check above fixes)
    cont = sum(D[d] * (math.pi / L[d]) ** 2 for d in range(3))
    assert abs(lam - cont) > 1e-3 * cont
