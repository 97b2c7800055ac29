"""Host-side measurement helpers of bench.py (no GPU): the conduction
velocity read from an activation map, the per-kernel byte models, the
committed DRAM traffic and the clock record."""
import numpy as np
import pytest

import bench
from paper_2308_01651_gb300 import inputs as I


def test_cv_planar_wave_exact():
    """A planar front t = x / v + t0 gives v back, in the mean and in every
    column (Q1 and Q2 slabs)."""
    for mesh in (I.slab_mesh(20, 5, 4, (1.0, 0.25, 0.2)), I.slab_mesh_q2(10, 3, 2, (1.0, 0.3, 0.2))):
        x = mesh["xyz"][:, 0]
        at = x / 0.061 + 2.5
        mean, col = bench.conduction_velocity(mesh, at)
        assert abs(mean - 0.061) <= 1e-12
        assert np.abs(col - 0.061).max() <= 1e-12


def test_cv_columns_and_mean():
    """Columns with their own speeds: each column's least-squares slope
    recovers its speed; the mean is distance over mean travel time (the
    harmonic mean of the column speeds), not their arithmetic mean."""
    mesh = I.slab_mesh(40, 3, 2, (2.0, 0.3, 0.2))
    g = I.rng(77)
    NX = 41
    ncol = mesh["xyz"].shape[0] // NX
    v = g.uniform(0.03, 0.08, size=ncol)
    x = mesh["xyz"][:, 0].reshape(ncol, NX)
    at = (x / v[:, None] + g.uniform(0, 1, size=(ncol, 1))).ravel()
    mean, col = bench.conduction_velocity(mesh, at)
    assert np.allclose(col, v, rtol=1e-12)
    # planes at x = 0.5 and 1.5: distance 1 over the mean of 1 / v
    assert abs(mean - 1.0 / np.mean(1.0 / v)) <= 1e-12


def test_cv_curved_front_slope_is_least_squares():
    """A front that accelerates: the column speed is the reciprocal of the
    least-squares line's slope over the window, checked against numpy's
    polyfit on the same nodes."""
    mesh = I.slab_mesh(30, 2, 2, (1.5, 0.2, 0.2))
    x = mesh["xyz"][:, 0]
    at = 20.0 * np.sqrt(x + 0.1)
    _, col = bench.conduction_velocity(mesh, at)
    xs = x[:31]
    sel = slice(int(np.argmin(np.abs(xs - 0.375))), int(np.argmin(np.abs(xs - 1.125))) + 1)
    slope = np.polyfit(xs[sel], (20.0 * np.sqrt(xs + 0.1))[sel], 1)[0]
    assert np.allclose(col, 1.0 / slope, rtol=1e-10)


def test_cv_undefined_cases():
    """No velocity for the shell, or when a node of the window never
    activated (the front has not crossed)."""
    mesh = I.slab_mesh(20, 2, 2, (1.0, 0.2, 0.2))
    at = mesh["xyz"][:, 0] / 0.05
    at[(mesh["xyz"][:, 0] > 0.6)] = np.nan
    assert bench.conduction_velocity(mesh, at) is None
    shell = dict(mesh, kind=I.MESH_SHELL)
    assert bench.conduction_velocity(shell, mesh["xyz"][:, 0]) is None


def test_kernel_models_scale():
    """Algorithmic bytes grow linearly with the nodes and with the inner
    iterations of the persistent solve."""
    N, E = 442401, 420000
    a = bench.kernel_model("solve32", N, E, inner_iters=10.0, sweeps=2.0)[0]
    b = bench.kernel_model("solve32", 2 * N, 2 * E, inner_iters=10.0, sweeps=2.0)[0]
    c = bench.kernel_model("solve32", N, E, inner_iters=20.0, sweeps=2.0)[0]
    assert abs(b / a - 2.0) < 1e-3
    assert c > a
    for name in ("ionic", "rhs", "resid"):
        m1 = bench.kernel_model(name, N, E)[0]
        m2 = bench.kernel_model(name, 2 * N, 2 * E)[0]
        assert m1 > 0 and abs(m2 / m1 - 2.0) < 1e-3


def test_algorithmic_bytes_per_node():
    """The roofline's algorithmic bytes are the hot path's per-node minimum:
    an inner CG iteration 60 B (x 4, y 4, fibres 24, seven FP32 vector
    touches 28; the shell adds 12 B of coordinates), a float-float residual
    48 B (+12), the right-hand side 28 B, the refined TTP06 ionic step
    2 (13 x 4 + 5 x 8) + 16 + 4 = 204 B."""
    N, E = 1000, 900
    one_it = bench.kernel_model("solve32", N, E, inner_iters=1.0, sweeps=0.0)[0] / N
    one_sw = bench.kernel_model("solve32", N, E, inner_iters=0.0, sweeps=1.0)[0] / N
    assert (one_it, one_sw) == (60, 48)
    sh_it = bench.kernel_model("solve32", N, E, inner_iters=1.0, sweeps=0.0, shell=True)[0] / N
    sh_sw = bench.kernel_model("solve32", N, E, inner_iters=0.0, sweeps=1.0, shell=True)[0] / N
    assert (sh_it, sh_sw) == (72, 60)
    assert bench.kernel_model("rhs", N, E)[0] / N == 28
    assert bench.kernel_model("ionic", N, E)[0] / N == 2 * (13 * 4 + 5 * 8) + 16 + 4


def test_clock_summary_parses_samples_and_reasons():
    """The clocks record of the bench line: median SM clock under load, the
    maximum, and every throttle reason seen Active in any sample (a sample
    line that is not a full record is skipped)."""
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A]",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = ["0, 1500, 2070, 1000, 0x40, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["samples"] == 0


def test_committed_traffic_scaling_and_staleness(monkeypatch):
    """Traffic of the persistent solve is the captured launch's DRAM bytes
    scaled by the ratio of algorithmic bytes (this run's average launch over
    the captured one, whose iterations and sweeps the record holds); a kernel
    whose sources changed since the capture reports none."""
    import json
    import os

    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["c2"]["solve32"]
    N, E = 442401, 420000
    # sources as at the capture (the check below does not depend on the
    # current files)
    monkeypatch.setattr(bench, "source_hash", lambda files: rec["source_hash"])
    cap = bench.kernel_model("solve32", N, E, rec["inner_iters"], sweeps=rec["sweeps"])[0]
    alg = bench.kernel_model("solve32", N, E, 8.45, sweeps=1.36)[0]
    t = bench.committed_traffic("c2", "solve32", N, E, alg)
    assert t == pytest.approx(rec["dram_bytes_per_launch"] * alg / cap, rel=1e-12)
    assert bench.committed_traffic("c2", "solve32", N, E, cap) == pytest.approx(rec["dram_bytes_per_launch"])
    monkeypatch.setattr(bench, "source_hash", lambda files: "changed")
    assert bench.committed_traffic("c2", "solve32", N, E, alg) is None
    assert bench.committed_traffic("c2", "no_such_kernel") is None
    assert bench.committed_traffic("no_such_workload", "solve32", N, E, alg) is None
