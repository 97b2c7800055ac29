"""Pins of the oracle's ionic models and of the semi-implicit ionic step
(paper Sec. 1.1.1 Eq. (1), Sec. 1.2 Eq. (4)).

What fixes each check:
  * Bueno-Orovio at u = 0, v = w = 1 has J_fi = J_so = J_si = 0, so a
    resting cell and a resting tissue stay at u = 0 exactly (bitwise).
  * The TTP06 initial conditions the paper prints (Sec. 3.2.1) are a rest
    state: an unstimulated cell must stay within 1 mV of -85.23 mV.
  * Action-potential features of the models' source publications (not printed
    in the paper): TTP06 overshoot of roughly +20..+50 mV, epicardial APD90
    near 300 ms, M cells about 80 ms longer; Bueno-Orovio epicardial peak
    u of 1.2..1.7 (u_mV = 85.7 u - 84, Sec. 3.2.3) with APD90 of 200..350 ms.
  * The semi-implicit step converges to a classical RK4 solution of the same
    ODE (Eq. (1)), at order 1 for BDF1.
  * Bueno-Orovio excitability: released above theta_v = 0.3 a cell fires,
    at or below it relaxes to rest (a mistyped threshold or gate constant
    moves that boundary).
"""
import numpy as np
import pytest

import oracle.oracle as O


def run_cell(model, cell, dt, T, amp, dur, order=1, u0=None):
    u, w = O.initial(model, cell)
    if u0 is not None:
        u = u0
    un1, wn1 = u, w.copy()
    n = int(round(T / dt))
    tr = np.empty(n)
    for k in range(n):
        iapp = amp if (k + 1) * dt <= dur + 1e-12 else 0.0
        unew, wnew = O.cell_step(model, order, dt, u, w, un1, wn1, iapp, cell=cell)
        un1, wn1 = u, w
        u, w = unew, wnew
        tr[k] = u
    return tr


def apd90(tr, dt, rest):
    peak = tr.max()
    thr = peak - 0.9 * (peak - rest)
    above = np.where(tr > thr)[0]
    return (above[-1] - above[0]) * dt, peak


def test_bo_rest_is_exact_single_cell():
    u, w = O.initial(O.BO)
    assert (u, *w) == (0.0, 1.0, 1.0, 0.0)
    assert O.iion(O.BO, u, w) == 0.0
    tr = run_cell(O.BO, O.EPI, 0.05, 500.0, 0.0, 0.0)
    assert np.all(tr == 0.0)


def test_bo_rest_is_exact_tissue():
    from paper_2308_01651_gb300 import inputs as I
    p = I.slab_bo_small(nx=6, ny=4, nz=3, L=(0.3, 0.2, 0.15))
    p["pulses"] = []
    p["masks"] = np.zeros((0, p["mesh"]["xyz"].shape[0]), dtype=np.uint8)
    S = O.sim_from_problem(p)
    S.step(200)
    u_n, _, w_n, _ = S.get_state()
    assert np.all(u_n == 0.0)
    assert np.all(w_n[0] == 1.0) and np.all(w_n[1] == 1.0)
    at, _ = S.activation()
    assert np.all(np.isnan(at))


@pytest.mark.parametrize("cell", [O.EPI, O.ENDO, O.MID])
def test_ttp06_paper_initial_state_is_rest(cell):
    u0, w0 = O.initial(O.TTP06, cell)
    assert u0 == -85.23
    assert w0[16] == 8.604 and w0[17] == 136.89 and w0[12] == 0.9073
    tr = run_cell(O.TTP06, cell, 0.05, 1000.0, 0.0, 0.0)
    assert np.abs(tr - u0).max() < 1.0


def test_ttp06_action_potential_features():
    dt = 0.02
    epi, pk_epi = apd90(run_cell(O.TTP06, O.EPI, dt, 600.0, 52.0, 1.0), dt, -85.23)
    endo, pk_endo = apd90(run_cell(O.TTP06, O.ENDO, dt, 600.0, 52.0, 1.0), dt, -85.23)
    mid, pk_mid = apd90(run_cell(O.TTP06, O.MID, dt, 600.0, 52.0, 1.0), dt, -85.23)
    for pk in (pk_epi, pk_endo, pk_mid):
        assert 20.0 < pk < 50.0
    assert 260.0 < epi < 340.0
    assert 260.0 < endo < 340.0
    assert mid > epi + 50.0


def test_bo_action_potential_features():
    dt = 0.02
    tr = run_cell(O.BO, O.EPI, dt, 600.0, 1.0, 1.0)
    apd, peak = apd90(tr, dt, 0.0)
    assert 1.2 < peak < 1.7
    assert 200.0 < apd < 350.0
    assert tr[-1] < 0.05


def rk4_cell(model, cell, dt, T, u0):
    u, w = O.initial(model, cell)
    y = np.concatenate([[u0], w])

    def f(y):
        a, b = O.rates(model, y[0], y[1:], cell=cell)
        return np.concatenate([[-O.iion(model, y[0], y[1:], cell=cell)], a - b * y[1:]])

    n = int(round(T / dt))
    out = np.empty(n)
    for k in range(n):
        k1 = f(y)
        k2 = f(y + 0.5 * dt * k1)
        k3 = f(y + 0.5 * dt * k2)
        k4 = f(y + dt * k3)
        y = y + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        out[k] = y[0]
    return out


def test_semi_implicit_step_converges_to_rk4():
    """Supra-threshold initial potential, no stimulus: the upstroke and early
    plateau, compared at t = 10, 20, 30 ms."""
    T = 30.0
    dref = 0.002
    ref = rk4_cell(O.TTP06, O.EPI, dref, T, -40.0)
    times = (10.0, 20.0, 30.0)
    errs = {1: [], 2: []}
    for order in (1, 2):
        for dt in (0.02, 0.01, 0.005):
            tr = run_cell(O.TTP06, O.EPI, dt, T, 0.0, 0.0, order=order, u0=-40.0)
            e = max(abs(tr[int(round(t / dt)) - 1] - ref[int(round(t / dref)) - 1]) for t in times)
            errs[order].append(e)
    r1 = [errs[1][i] / errs[1][i + 1] for i in range(2)]
    assert all(1.8 < r < 2.2 for r in r1), r1
    # BDF2 (with a BDF1 start and the h/j gates' switch at -40 mV) is far more
    # accurate than BDF1 and converges faster than first order
    assert all(e2 < 0.2 * e1 for e1, e2 in zip(errs[1], errs[2]))
    r2 = [errs[2][i] / errs[2][i + 1] for i in range(2)]
    assert all(r > 2.2 for r in r2), r2


def test_bo_excitation_threshold():
    """The minimal model is excitable with a threshold: a cell released
    above theta_v = 0.3 fires a full upstroke (fast inward J_fi opens), one
    released at theta_v or below relaxes towards rest without firing (first
    with tau_o2 = 6 ms, below theta_o = 0.006 with tau_o1 = 400 ms; epicardial
    set of Bueno-Orovio et al. 2008)."""
    fired = run_cell(O.BO, O.EPI, 0.01, 100.0, 0.0, 0.0, u0=0.35)
    assert fired.max() > 1.2
    for u0 in (0.10, 0.30):
        quiet = run_cell(O.BO, O.EPI, 0.01, 100.0, 0.0, 0.0, u0=u0)
        assert quiet.max() <= u0 and 0.0 < quiet[-1] < 0.006


# The fast TTP06 gates of the paper's epicardial initial state (Sec. 3.2.1)
# are at their voltage steady states: with time constants of 0.001-9 ms at
# -85.23 mV they have relaxed long before any state is recorded.  So the
# oracle's steady-state value a/b of each of them at the printed potential
# must reproduce the printed value to its last digit (one unit of it).  h
# (tau 8 ms) and j (76 ms) are still recovering from the last beat and are
# left out, like the slow gates and the concentrations.
FAST_GATES_LAST_DIGIT = {"m": 1e-5, "xr2": 1e-4, "s": 1e-6, "r": 1e-10, "d": 1e-8}


def test_ttp06_fast_gates_of_the_papers_initial_state_are_steady():
    from .helpers import golden
    g = golden("ttp06_epi_initial_state.json")
    order = g["state_order"]
    w = np.array([g["states"][k] for k in order])
    a, b = O.rates(O.TTP06, g["V_mV"], w, cell=O.EPI)
    for name, unit in FAST_GATES_LAST_DIGIT.items():
        k = order.index(name)
        assert 1.0 / b[k] < 10.0, name  # a fast gate: time constant below 10 ms
        assert abs(a[k] / b[k] - g["states"][name]) <= unit, (name, a[k] / b[k], g["states"][name])
