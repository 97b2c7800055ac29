"""Oracle pins for single-cell pre-pacing (Sec. 3.2: ionic states from 0D
simulations of many beats at the pacing period)."""
import numpy as np

import oracle.oracle as O


def test_unpaced_bueno_orovio_cell_stays_at_rest():
    out = O.prepace(O.BO, 2, 100.0, 5, 0.05, 0.0, 1.0)
    u0, w0 = O.initial(O.BO)
    assert out[0] == u0 == 0.0
    assert out[1] == 1.0 and out[2] == 1.0  # v, w stay at their rest values


def test_paced_ttp06_cell_approaches_a_periodic_state():
    """End-of-beat states of consecutive beats come closer as the beats go on
    (the point of pre-pacing): the potential and the gates settle within a
    few beats, the ion concentrations drift slowly (intracellular sodium
    over hundreds of beats, why the paper paces 1000 beats), with a
    beat-to-beat change that still shrinks."""
    def states(beats):
        return O.prepace(O.TTP06, 2, 800.0, beats, 0.05, 35.714, 2.0)

    s3, s4, s29, s30 = states(3), states(4), states(29), states(30)
    assert np.abs(s30 - s29).max() < np.abs(s4 - s3).max()
    fast = slice(0, 14)  # u and the 13 gates
    assert np.abs(s30[fast] - s29[fast]).max() < np.abs(s4[fast] - s3[fast]).max()
    assert np.abs(s30[1:14] - s29[1:14]).max() < 1e-3
    # resting at the end of a beat, not stuck depolarised
    assert -90.0 < s30[0] < -80.0


def test_prepace_zero_beats_returns_the_initial_state():
    init = np.arange(19, dtype=float) * 0.01 - 85.0
    out = O.prepace(O.TTP06, 0, 800.0, 0, 0.05, 35.714, 2.0, init=init)
    assert np.array_equal(out, init)
