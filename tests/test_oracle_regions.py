"""Oracle pins for subdomains (paper Sec. 1.1.2): per-region conductivities,
continuity of flux across interfaces (the Galerkin form with piecewise D),
and non-conductive regions excluded from the simulation."""
import numpy as np
import scipy.sparse as sp

import oracle.oracle as O
from paper_2308_01651_gb300 import inputs as I


def _with(prob, label, sigma, excluded):
    q = dict(prob)
    q["regions"] = dict(label=np.asarray(label, dtype=np.uint8), sigma=sigma, excluded=excluded)
    return q


def _assembled(prob):
    M, K, active = O.assemble_regions(prob)
    return M.toarray(), K.toarray(), active


def test_regions_split_stiffness_into_per_region_parts():
    """K of a two-region slab is the sum of each region's elements assembled
    with that region's conductivities; M does not depend on them."""
    p = I.slab_ttp06(nx=6, ny=4, nz=3, L=(0.06, 0.04, 0.03), T=1.0)
    c = I.element_centroids(p["mesh"])
    lab = (c[:, 0] > 0.03).astype(np.uint8)
    s0, s1 = (1.4, 0.5, 0.25), (0.3, 0.2, 0.1)
    M, K, act = _assembled(_with(p, lab, [s0, s1], [0, 0]))
    _, K0, _ = _assembled(_with(p, lab, [s0, s1], [0, 1]))  # region 1 removed
    _, K1, _ = _assembled(_with(p, lab, [s0, s1], [1, 0]))  # region 0 removed
    assert act.all()
    assert np.allclose(K, K0 + K1, rtol=0, atol=1e-15 * np.abs(K).max())
    # K 1 = 0 in each part and in the sum (Neumann on every region boundary)
    for k in (K, K0, K1):
        assert np.abs(k.sum(axis=1)).max() <= 1e-13 * np.abs(k).max()
    Mh, _, _ = _assembled(_with(p, lab, [s0, s0], [0, 0]))
    assert np.array_equal(M, Mh)


def test_uniformly_scaled_region_scales_stiffness():
    """K is linear in D: one region covering the slab with conductivities x 2
    doubles the homogeneous K exactly."""
    p = I.slab_ttp06(nx=5, ny=3, nz=2, L=(0.05, 0.03, 0.02), T=1.0)
    ne = p["mesh"]["hex"].shape[0]
    s = (1.4, 0.5, 0.25)
    _, K1, _ = _assembled(_with(p, np.zeros(ne), [s], [0]))
    _, K2, _ = _assembled(_with(p, np.zeros(ne), [tuple(2 * x for x in s)], [0]))
    assert np.array_equal(K2, 2.0 * K1)


def test_excluded_region_leaves_inactive_nodes_decoupled():
    """Excluded elements contribute to neither M nor K; nodes with no element
    left are inactive: a lone M diagonal equal to the consistent-mass
    diagonal their excluded elements would give (h^3 (2/3)^3 for an interior
    node of a uniform slab), no couplings, a zero K row; M stays symmetric
    positive definite, and 1^T M 1 = remaining volume + those diagonals."""
    p = I.slab_regions(nx=10, ny=6, nz=3)
    M, K, act = _assembled(p)
    nn = M.shape[0]
    inact = np.flatnonzero(act == 0)
    assert 0 < inact.size < nn
    h = np.array(p["mesh"]["L"]) / np.array([p["mesh"]["nx"], p["mesh"]["ny"], p["mesh"]["nz"]])
    ii, jj, kk = I.node_ijk(p["mesh"])
    interior = (ii > 0) & (ii < p["mesh"]["nx"]) & (jj > 0) & (jj < p["mesh"]["ny"]) & (kk > 0) & (kk < p["mesh"]["nz"])
    for v in inact:
        assert np.count_nonzero(M[v]) == 1 and np.count_nonzero(M[:, v]) == 1 and M[v, v] > 0
        if interior[v]:
            assert abs(M[v, v] - np.prod(h) * 8.0 / 27.0) <= 1e-15 * M[v, v]
        assert not K[v].any() and not K[:, v].any()
    assert np.allclose(M, M.T, rtol=0, atol=1e-15 * np.abs(M).max())
    assert np.allclose(K, K.T, rtol=0, atol=1e-15 * np.abs(K).max())
    assert np.linalg.eigvalsh(M).min() > 0
    lab = p["regions"]["label"]
    vol = np.prod(h) * np.count_nonzero(lab != 2)
    diag = M[inact, inact].sum()
    assert abs(M.sum() - (vol + diag)) <= 1e-12 * (vol + diag)
    assert np.abs(K.sum(axis=1)).max() <= 1e-13 * np.abs(K).max()


def test_scar_wall_blocks_conduction_and_holds_inactive_nodes():
    """A non-conductive layer across the slab stops the wave: nodes before it
    activate, nodes beyond it never do; inactive nodes keep their potential
    and states bitwise."""
    p = I.slab_regions(nx=24, ny=4, nz=3, wall=True, T=30.0, model=I.BO)
    sim = O.sim_from_problem(p)
    act = sim.active()
    u0, _, w0, _ = sim.get_state()
    sim.step(int(round(30.0 / p["dt"])))
    at, _ = sim.activation()
    x = p["mesh"]["xyz"][:, 0] / p["mesh"]["L"][0]
    assert not np.isnan(at[x < 0.4]).any(), "the near side activates"
    assert np.isnan(at[x > 0.6]).all(), "the far side is blocked"
    u, _, w, _ = sim.get_state()
    off = act == 0
    assert off.any()
    assert np.array_equal(u[off], u0[off]) and np.array_equal(w[:, off], w0[:, off])
