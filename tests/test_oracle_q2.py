"""Pins of the oracle's triquadratic (Q2, 27-node) hexahedra (Sec. 1.2: the
FE space has polynomial degree p, arbitrary on hexahedra).

What fixes each part:
  * element matrices on a box with a constant (anisotropic) D equal the
    Kronecker forms of exact 1-D integrals of the quadratic Lagrange basis,
    computed here with exact polynomial integration (no quadrature);
  * curved and sheared elements: partition of unity (rows of K sum to 0,
    the mass sums to the volume of an affine element) and invariance under
    a rotation of coordinates and fibres;
  * assembled slab matrices: symmetry, K 1 = 0, 1^T M 1 = volume, positive
    definite mass, 125-point rows, interior rows of K x = 0 for linear x;
  * the spatial error of a manufactured problem decreases at third order.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as P

import oracle.oracle as O
from paper_2308_01651_gb300 import inputs as I

# quadratic Lagrange polynomials on [0,1], nodes 0, 1/2, 1 (coefficients, low first)
L1D = [np.array([1.0, -3.0, 2.0]), np.array([0.0, 4.0, -4.0]), np.array([0.0, -1.0, 2.0])]


def _int01(c):
    ci = P.polyint(c)
    return P.polyval(1.0, ci) - P.polyval(0.0, ci)


def _tables():
    d = [P.polyder(c) for c in L1D]
    m = np.array([[_int01(P.polymul(L1D[a], L1D[b])) for b in range(3)] for a in range(3)])
    kk = np.array([[_int01(P.polymul(d[a], d[b])) for b in range(3)] for a in range(3)])
    dm = np.array([[_int01(P.polymul(d[a], L1D[b])) for b in range(3)] for a in range(3)])
    return m, kk, dm


def _kron3(a0, a1, a2):
    # local index a = a0 + 3 a1 + 9 a2: the direction-2 factor is the outer one
    return np.kron(a2, np.kron(a1, a0))


def _box_nodes(h, origin=(0.0, 0.0, 0.0)):
    X = np.zeros((27, 3))
    for a in range(27):
        idx = (a % 3, (a // 3) % 3, a // 9)
        for d in range(3):
            X[a, d] = origin[d] + 0.5 * idx[d] * h[d]
    return X


def test_q2_exact_1d_tables():
    m, kk, dm = _tables()
    assert np.allclose(m * 30.0, [[4, 2, -1], [2, 16, 2], [-1, 2, 4]], atol=1e-13)
    assert np.allclose(kk * 3.0, [[7, -8, 1], [-8, 16, -8], [1, -8, 7]], atol=1e-13)
    assert np.allclose(dm.sum(axis=0), 0.0, atol=1e-13)  # sum of the derivatives is 0


def test_q2_element_box_closed_form_anisotropic():
    g = I.rng(901)
    h = g.uniform(0.05, 0.3, size=3)
    X = _box_nodes(h, origin=g.uniform(-1, 1, size=3))
    # a constant fibre frame at a random orientation: constant full D
    A = np.linalg.qr(g.normal(size=(3, 3)))[0]
    f, s = A[:, 0], A[:, 1]
    dl, dt_, dn = 1.3e-3, 0.4e-3, 0.2e-3
    D = dn * np.eye(3) + (dl - dn) * np.outer(f, f) + (dt_ - dn) * np.outer(s, s)
    Me, Ke = O.element_matrices_q2(X, np.tile(f, (27, 1)), np.tile(s, (27, 1)), dl, dt_, dn)
    m, kk, dm = _tables()
    vol = h.prod()
    assert np.allclose(Me, vol * _kron3(m, m, m), rtol=1e-12, atol=1e-16 * vol)
    Kx = np.zeros((27, 27))
    for i in range(3):
        for j in range(3):
            fac = []
            for d in range(3):
                if d == i and d == j:
                    fac.append(kk)
                elif d == i:
                    fac.append(dm)
                elif d == j:
                    fac.append(dm.T)
                else:
                    fac.append(m)
            Kx += D[i, j] / (h[i] * h[j]) * _kron3(*fac)
    Kx *= vol
    assert np.abs(Ke - Kx).max() <= 1e-12 * np.abs(Kx).max()
    assert np.allclose(Ke, Ke.T, atol=1e-15 * np.abs(Kx).max())


def _curved_element(g):
    X = _box_nodes((0.2, 0.15, 0.1))
    # move the non-vertex nodes off their straight positions
    for a in range(27):
        idx = (a % 3, (a // 3) % 3, a // 9)
        if any(i == 1 for i in idx):
            X[a] += g.uniform(-0.01, 0.01, size=3)
    return X


def test_q2_curved_element_partition_of_unity_and_rotation():
    g = I.rng(902)
    X = _curved_element(g)
    f = g.normal(size=(27, 3))
    s = g.normal(size=(27, 3))
    Me, Ke = O.element_matrices_q2(X, f, s, 1.1e-3, 0.5e-3, 0.3e-3)
    assert np.abs(Ke.sum(axis=1)).max() <= 1e-13 * np.abs(Ke).max()
    assert np.all(np.linalg.eigvalsh(Me) > 0)
    R = np.linalg.qr(g.normal(size=(3, 3)))[0]
    Me2, Ke2 = O.element_matrices_q2(X @ R.T + 0.3, f @ R.T, s @ R.T, 1.1e-3, 0.5e-3, 0.3e-3)
    assert np.allclose(Me2, Me, rtol=1e-11, atol=1e-15 * np.abs(Me).max())
    assert np.allclose(Ke2, Ke, rtol=1e-10, atol=1e-12 * np.abs(Ke).max())


def test_q2_affine_element_mass_sums_to_volume():
    g = I.rng(903)
    A = np.eye(3) + 0.2 * g.normal(size=(3, 3))
    X = _box_nodes((1.0, 1.0, 1.0)) @ A.T
    f = np.tile([1.0, 0.0, 0.0], (27, 1))
    s = np.tile([0.0, 1.0, 0.0], (27, 1))
    Me, Ke = O.element_matrices_q2(X, f, s, 1e-3, 1e-3, 1e-3)
    assert Me.sum() == pytest.approx(abs(np.linalg.det(A)), rel=1e-13)
    assert np.abs(Ke.sum(axis=0)).max() <= 1e-13 * np.abs(Ke).max()


def test_q2_assembled_slab_invariants():
    prob = I.slab_ttp06_q2(nx=4, ny=3, nz=2, L=(0.4, 0.3, 0.2), T=1.0)
    m = prob["mesh"]
    D = O.diffusivities(prob["cond"])
    M, K = O.assemble_q2(m["xyz"], m["hex"], prob["f0"], prob["s0"], D)
    n = m["xyz"].shape[0]
    assert n == 9 * 7 * 5
    one = np.ones(n)
    assert abs(one @ (M @ one) - 0.4 * 0.3 * 0.2) <= 1e-15
    assert np.abs(K @ one).max() <= 1e-14 * abs(K).max()
    assert abs(M - M.T).max() <= 1e-18 and abs(K - K.T).max() <= 1e-17
    assert np.diff(M.indptr).max() == 125
    assert np.linalg.eigvalsh(M.toarray()).min() > 0
    # uniform fibres: interior rows of K x vanish for a linear x (Q2 holds
    # linear fields exactly and D is constant)
    p2 = I.slab_bo_q2(nx=4, ny=3, nz=2, L=(0.4, 0.3, 0.2), T=1.0)
    M2, K2 = O.assemble_q2(p2["mesh"]["xyz"], p2["mesh"]["hex"], p2["f0"], p2["s0"],
                           O.diffusivities(p2["cond"]))
    xyz = p2["mesh"]["xyz"]
    lin = 0.3 * xyz[:, 0] - 1.2 * xyz[:, 1] + 0.7 * xyz[:, 2] + 0.1
    i, j, k = I.node_ijk(p2["mesh"])
    inner = (i > 0) & (i < 8) & (j > 0) & (j < 6) & (k > 0) & (k < 4)
    r = K2 @ lin
    assert np.abs(r[inner]).max() <= 1e-13 * np.abs(r).max()


def test_q2_manufactured_third_order_in_space():
    """(c M + K) U = M F with F the nodal values of f = (c + pi^2 (Dx/Lx^2 +
    Dy/Ly^2 + Dz/Lz^2)) u for u = cos(pi x/Lx) cos(pi y/Ly) cos(pi z/Lz)
    (zero flux on the box): the nodal error falls at third order or faster
    (Q1 on the same node grids: second)."""
    import scipy.sparse.linalg as spla

    Lb = (1.0, 0.8, 0.6)
    Dd = (1.0, 0.6, 0.4)
    c = 1.0
    errs = []
    for ne in (2, 4, 8):
        mesh = I.slab_mesh_q2(ne, ne, ne, Lb)
        n = mesh["xyz"].shape[0]
        f0, s0 = I.uniform_fibres(n)
        M, K = O.assemble_q2(mesh["xyz"], mesh["hex"], f0, s0, Dd)
        x, y, z = mesh["xyz"].T
        u = np.cos(np.pi * x / Lb[0]) * np.cos(np.pi * y / Lb[1]) * np.cos(np.pi * z / Lb[2])
        lam = c + np.pi ** 2 * (Dd[0] / Lb[0] ** 2 + Dd[1] / Lb[1] ** 2 + Dd[2] / Lb[2] ** 2)
        U = spla.spsolve((c * M + K).tocsc(), M @ (lam * u))
        errs.append(np.abs(U - u).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders >= 2.7), (errs, orders)


def test_q2_oracle_front_converges_to_q1_front():
    """The BO slab on Q2 elements at two resolutions against Q1 on the finer
    node grid: the activation maps approach each other under refinement
    (both discretise the same front; on equal node grids Q2's error is the
    larger one here, its elements being twice as wide)."""
    L = (0.6, 0.3, 0.2)
    ref_p = I.slab_bo_small(nx=24, ny=12, nz=8, L=L, T=25.0)
    sim = O.sim_from_problem(ref_p)
    sim.step(ref_p["nsteps"])
    ref = sim.activation()[0].reshape(9, 13, 25)
    errs = []
    for ne, step in ((6, 2), (12, 1)):
        p = I.slab_bo_q2(nx=ne, ny=ne // 2, nz=ne // 3, L=L, T=25.0)
        sim = O.sim_from_problem(p)
        sim.step(p["nsteps"])
        at = sim.activation()[0]
        r = ref[::step, ::step, ::step].ravel()
        assert np.array_equal(np.isnan(at), np.isnan(r))
        errs.append(np.nanmax(np.abs(at - r)))
    assert np.nanmax(ref) > 8.0  # the front crossed the slab
    assert errs[0] <= 0.2 * np.nanmax(ref), errs
    assert errs[1] <= 0.5 * errs[0], errs
