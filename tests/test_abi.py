"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/ep.h declares, validates arguments before touching the
device, and reports footprints."""
import os
import re

import numpy as np
import pytest

from paper_2308_01651_gb300 import ep
from paper_2308_01651_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "ep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ep_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    L = ep.lib()
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(ep.EXPORTS) == names


def _args(prob, **kw):
    pulses = [dict(p, mask=prob["masks"][k]) for k, p in enumerate(prob["pulses"])]
    return (prob["mesh"], prob["f0"], prob["s0"], prob["cond"], prob["model"]), dict(
        cell_type=prob["cell"], pulses=pulses, dt=prob["dt"], bdf_order=prob["bdf"], **kw)


@pytest.mark.parametrize("bad", [
    dict(dt=0.0), dict(dt=-1.0), dict(bdf_order=4), dict(bdf_order=0), dict(precision=7), dict(op32=9),
    dict(max_iter=-1), dict(tol=-1.0), dict(ionic_threads=96), dict(ionic_threads=-128),
    dict(solve_tiles=3), dict(solve_tiles=-1),
])
def test_create_rejects_bad_options(bad):
    prob = I.slab_bo_small(nx=4, ny=3, nz=2, L=(0.2, 0.15, 0.1))
    a, kw = _args(prob)
    kw.update(bad)
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(*a, **kw)
    assert e.value.status == ep.EP_EINVAL


def test_create_rejects_bad_mesh_and_inputs():
    prob = I.slab_bo_small(nx=4, ny=3, nz=2, L=(0.2, 0.15, 0.1))
    a, kw = _args(prob)
    m = dict(prob["mesh"])
    m["n_nodes"] = 7
    m.pop("xyz")
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(m, *a[1:], **kw)
    assert e.value.status == ep.EP_EINVAL and "n_nodes" in str(e.value)
    cond = dict(prob["cond"], sigma=(1e-3, -1.0, 1e-3))
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(a[0], a[1], a[2], cond, a[4], **kw)
    assert e.value.status == ep.EP_EINVAL
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(a[0], a[1], a[2], a[3], 5, **kw)
    assert e.value.status == ep.EP_EINVAL
    bad_cell = np.full(prob["mesh"]["xyz"].shape[0], 9, dtype=np.uint8)
    kw2 = dict(kw, cell_type=bad_cell)
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(*a, **kw2)
    assert e.value.status == ep.EP_EINVAL
    kw3 = dict(kw, pulses=kw["pulses"] * 5)
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(*a, **kw3)
    assert e.value.status == ep.EP_EINVAL
    # the matrix-free operator takes shells at most 31 elements across the wall
    m, geo = I.shell_mesh(32, 8, 4)
    f0, s0 = I.shell_helix_fibres(geo)
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(m, f0, s0, prob["cond"], I.TTP06, precision=ep.EP_PREC_FP32_REFINED,
                     op32=ep.EP_OP_MATRIX_FREE)
    assert e.value.status == ep.EP_EUNSUPPORTED
    # the tiled solve takes refined Q1 instances with the stencil operator
    for bad in (dict(precision=ep.EP_PREC_FP64, solve_tiles=2),
                dict(precision=ep.EP_PREC_FP32_REFINED, op32=ep.EP_OP_MATRIX_FREE, solve_tiles=2)):
        with pytest.raises(ep.EpError) as e:
            ep.ep_create(*a, **dict(kw, **bad))
        assert e.value.status == ep.EP_EUNSUPPORTED, bad


def test_footprint_scales_with_nodes():
    small = I.slab_mesh(30, 30, 30, (0.3, 0.3, 0.3))
    big = I.slab_mesh(60, 60, 60, (0.6, 0.6, 0.6))
    for prec in (ep.EP_PREC_FP64, ep.EP_PREC_FP32_REFINED):
        a = ep.ep_footprint_bytes(small, I.TTP06, precision=prec)
        b = ep.ep_footprint_bytes(big, I.TTP06, precision=prec)
        assert a > 0 and 6.5 < b / a < 8.5
    assert ep.ep_footprint_bytes(small, 9) == 0
    # per-node budget: the FP64 path keeps the symmetric 14-slot stencils in
    # double; the refined path keeps the same symmetric stencils of A and M as
    # float-float (224 B/node) and its TTP06 gates in float.  Both stay under
    # 768 B/node, i.e. above 3.5e8 nodes in 280 GB of HBM.
    n = 61 ** 3
    for prec in (ep.EP_PREC_FP64, ep.EP_PREC_FP32_REFINED):
        assert ep.ep_footprint_bytes(big, I.TTP06, precision=prec) < 768 * n
    assert ep.ep_footprint_bytes(big, I.BO, precision=ep.EP_PREC_FP64) < \
        ep.ep_footprint_bytes(big, I.TTP06, precision=ep.EP_PREC_FP64)


def test_state_pack_roundtrip():
    n, ns = 11, 18
    g = I.rng(3)
    arrs = [g.normal(size=n), g.normal(size=n), g.normal(size=(ns, n)), g.normal(size=(ns, n)),
            g.normal(size=n), g.normal(size=n)]
    buf = ep.state_pack(1, 2, 0.05, 17, *arrs)
    assert buf.size == 64 + 8 * n * (4 + 2 * ns)
    st = ep.state_unpack(buf)
    assert st["step"] == 17 and st["model"] == 1 and st["dt"] == 0.05
    for k, name in enumerate(["u_n", "u_nm1", "w_n", "w_nm1", "at", "best"]):
        assert np.array_equal(st[name], arrs[k])


def test_state_pack_roundtrip_bdf3():
    """BDF3 buffers carry a third level: u_n, u_nm1, u_nm2, then w_n, w_nm1,
    w_nm2, then at and best."""
    n, ns = 9, 3
    g = I.rng(4)
    u = [g.normal(size=n) for _ in range(3)]
    w = [g.normal(size=(ns, n)) for _ in range(3)]
    at, best = g.normal(size=n), g.normal(size=n)
    buf = ep.state_pack(0, 3, 0.05, 5, u[0], u[1], w[0], w[1], at, best, u_nm2=u[2], w_nm2=w[2])
    assert buf.size == 64 + 8 * n * (3 + 3 * ns + 2)
    body = buf[64:].view(np.float64)
    assert np.array_equal(body[2 * n:3 * n], u[2])
    assert np.array_equal(body[3 * n + 2 * ns * n:3 * n + 3 * ns * n], w[2].ravel())
    st = ep.state_unpack(buf)
    assert st["bdf_order"] == 3
    for name, v in [("u_n", u[0]), ("u_nm1", u[1]), ("u_nm2", u[2]), ("w_nm2", w[2]), ("at", at),
                    ("best", best)]:
        assert np.array_equal(st[name], v)
    with pytest.raises(ValueError):
        ep.state_pack(0, 3, 0.05, 5, u[0], u[1], w[0], w[1], at, best)


def test_q2_slab_validation_and_footprint():
    """Q2 slabs need FP32_REFINED and one region; the footprint counts the
    quadrature-point flux matrices and element buffers instead of stencils."""
    prob = I.slab_ttp06_q2(nx=4, ny=3, nz=2, L=(0.4, 0.3, 0.2), T=1.0)
    a, kw = _args(prob)
    kw.update(precision=ep.EP_PREC_FP64)
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(*a, **kw)
    assert e.value.status == ep.EP_EUNSUPPORTED
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(*a, **dict(kw, precision=ep.EP_PREC_FP32_REFINED, solve_tiles=2))
    assert e.value.status == ep.EP_EUNSUPPORTED
    bad = dict(prob["mesh"], n_nodes=10)
    bad.pop("xyz")
    with pytest.raises(ep.EpError) as e:
        ep.ep_create(bad, *a[1:], **dict(kw, precision=ep.EP_PREC_FP32_REFINED))
    assert e.value.status == ep.EP_EINVAL
    big = I.slab_mesh_q2(100, 35, 15, (2.0, 0.7, 0.3))
    fp = ep.ep_footprint_bytes(big, I.TTP06, precision=ep.EP_PREC_FP32_REFINED)
    n = big["xyz"].shape[0]
    assert n == 201 * 71 * 31
    assert 300 * n < fp < 900 * n
