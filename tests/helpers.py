"""Shared test helpers: run a problem record on the oracle and on the CUDA
library, move states between them, compare."""
import numpy as np

import oracle.oracle as O
from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I


def gpu_state(inst):
    return ep.state_unpack(inst.save())


def oracle_to_gpu(sim, inst, prob):
    """Copies the oracle's full state (time levels, states, activation) into
    the GPU instance through ep_load_state."""
    u_n, u_nm1, w_n, w_nm1 = sim.get_state()
    at_raw, best = sim.activation_raw()
    extra = {}
    if prob["bdf"] == 3:
        u_nm2, w_nm2 = sim.get_level2()
        extra = dict(u_nm2=u_nm2, w_nm2=w_nm2)
    buf = ep.state_pack(prob["model"], prob["bdf"], prob["dt"], sim.stepindex, u_n, u_nm1, w_n,
                        w_nm1, at_raw, best, **extra)
    inst.load(buf)


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def synthetic_front_state(prob, g, width=0.05):
    """A seeded synthetic state for one-step parity: resting ionic states and a
    smooth potential front along x (model units), with a slightly different
    previous time level so that BDF2 combinations are exercised."""
    xyz = prob["mesh"]["xyz"]
    n = xyz.shape[0]
    u0, w0 = O.initial(prob["model"])  # resting values (paper's TTP06 ICs / BO rest)
    x = xyz[:, 0] / max(xyz[:, 0].max(), 1e-12)
    x0 = g.uniform(0.3, 0.7)
    if prob["model"] == I.TTP06:
        lo, hi = -85.23, 20.0
    else:
        lo, hi = 0.0, 1.3
    prof = lo + (hi - lo) * 0.5 * (1.0 - np.tanh((x - x0) / width))
    u_n = prof + g.normal(0.0, 1e-3 * (hi - lo), size=n)
    u_nm1 = lo + (hi - lo) * 0.5 * (1.0 - np.tanh((x - x0 + 0.02) / width))
    w = np.tile(w0[:, None], (1, n))
    w_n = w * (1.0 + 1e-3 * g.normal(size=w.shape))
    w_nm1 = w.copy()
    return u_n, u_nm1, w_n, w_nm1


def golden(name):
    """A fixture of values the paper prints (tests/golden/<name>, with its
    citation inside)."""
    import json
    import os

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        return json.load(f)
