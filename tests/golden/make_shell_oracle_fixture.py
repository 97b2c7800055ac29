"""Writes tests/golden/shell_ttp06_oracle_40ms.npz: the FP64 oracle's
activation times and potential on the LV-shell workload (2,192,400 nodes,
TTP06 endo/M/epi, BDF2, dt 0.05 ms, apical stimulus) from t = 0 to 40 ms,
on a sample of its nodes (every fifth circumferential column of nodes: all
20 + 1 transmural and 260 + 1 longitudinal positions of it).

Calls only the oracle (oracle/) and the seeded input generator.  Stored:
  nodes      int32, sampled node indices
  at_step    uint16, activation time in steps (t = at_step * dt), 65535 where
             the node had not activated by the end of the window
  u_centi_mV int16, potential at the end of the window in units of 0.01 mV
  dt, t_end_ms, steps
Run: python tests/golden/make_shell_oracle_fixture.py [threads]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle.oracle as O  # noqa: E402
from paper_2308_01651_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "shell_ttp06_oracle_40ms.npz")
T_END = 40.0
EVERY = 5


def sample_nodes(prob):
    m = prob["mesh"]
    NX, NY = m["nx"] + 1, m["ny"]
    n = np.arange(m["xyz"].shape[0])
    j = (n // NX) % NY
    return n[j % EVERY == 0].astype(np.int32)


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    O.set_threads(threads)
    prob = I.shell_ttp06(T=T_END)
    t0 = time.time()
    sim = O.sim_from_problem(prob)
    print(f"assembled in {time.time() - t0:.1f} s", flush=True)
    steps = prob["nsteps"]
    t0 = time.time()
    for k in range(0, steps, 50):
        sim.step(min(50, steps - k))
        print(f"step {k + 50}: {time.time() - t0:.1f} s, {sim.last_iters} CG iterations", flush=True)
    at = sim.activation()[0]
    u = sim.potential()
    nodes = sample_nodes(prob)
    a = at[nodes]
    at_step = np.where(np.isnan(a), 65535, np.rint(a / prob["dt"])).astype(np.uint16)
    u_c = np.rint(u[nodes] * 100.0).astype(np.int16)
    np.savez_compressed(OUT, nodes=nodes, at_step=at_step, u_centi_mV=u_c, dt=prob["dt"], t_end_ms=T_END,
                        steps=steps)
    print(OUT, os.path.getsize(OUT), "bytes;", int((at_step != 65535).sum()), "sampled nodes activated")


if __name__ == "__main__":
    main()
