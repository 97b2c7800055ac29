"""Pins of the oracle's finite-element part against closed forms and
invariants (paper Sec. 1.2, Eqs. (3) and (6)).

None of these re-types the oracle's quadrature: element matrices are checked
against exact 1-D integrals combined by Kronecker products, against rotation
invariance, against an independent 4-point Gauss volume of curved elements,
and the assembled matrices against K*1 = 0, 1^T M 1 = volume, symmetry and
positive definiteness; the linear solve against scipy's direct solver.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle.oracle as O
from paper_2308_01651_gb300 import inputs as I

# exact 1-D integrals on [0, h] for the linear basis l0 = 1 - x/h, l1 = x/h
def m1(h):
    return h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])


def s1(h):
    return np.array([[1.0, -1.0], [-1.0, 1.0]]) / h


def c1():
    # c[a, b] = int l_a' l_b dx = sign(a) / 2
    return np.array([[-0.5, -0.5], [0.5, 0.5]])


def box_closed_form(h, D):
    """K_e = sum_{p,q} D_pq (x)_d B_d^{pq}, M_e = (x)_d m1(h_d); local index
    a = a0 + 2 a1 + 4 a2, so the Kronecker order is d = 2, 1, 0."""
    K = np.zeros((8, 8))
    for p in range(3):
        for q in range(3):
            Bs = []
            for d in range(3):
                if d == p and d == q:
                    Bs.append(s1(h[d]))
                elif d == p:
                    Bs.append(c1())
                elif d == q:
                    Bs.append(c1().T)
                else:
                    Bs.append(m1(h[d]))
            K += D[p, q] * np.kron(Bs[2], np.kron(Bs[1], Bs[0]))
    M = np.kron(m1(h[2]), np.kron(m1(h[1]), m1(h[0])))
    return M, K


def random_frame(g):
    Q, _ = np.linalg.qr(g.normal(size=(3, 3)))
    return Q[:, 0], Q[:, 1], Q[:, 2]


def box_vertices(h, origin=(0.0, 0.0, 0.0)):
    X = np.zeros((8, 3))
    for a in range(8):
        X[a] = [origin[0] + (a & 1) * h[0], origin[1] + ((a >> 1) & 1) * h[1], origin[2] + ((a >> 2) & 1) * h[2]]
    return X


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_element_matrices_box_closed_form(seed):
    g = I.rng(100 + seed)
    h = g.uniform(0.01, 0.2, size=3)
    f, s, n = random_frame(g)
    dl, dt_, dn = g.uniform(1e-4, 2e-3, size=3)
    X = box_vertices(h, origin=g.normal(size=3))
    Me, Ke = O.element_matrices(X, np.tile(f, 8), np.tile(s, 8), dl, dt_, dn)
    D = dl * np.outer(f, f) + dt_ * np.outer(s, s) + dn * np.outer(n, n)
    Mx, Kx = box_closed_form(h, D)
    assert np.abs(Me - Mx).max() <= 1e-14 * np.abs(Mx).max()
    assert np.abs(Ke - Kx).max() <= 1e-13 * np.abs(Kx).max()


def test_element_matrices_affine_closed_form():
    """Sheared element x = A xi + b on the unit cube: K_e equals the unit-cube
    closed form with D' = |det A| A^{-1} D A^{-T}; a transposed Jacobian
    anywhere breaks this (A is not symmetric)."""
    g = I.rng(7)
    A = np.eye(3) * 0.1 + 0.03 * g.normal(size=(3, 3))
    b = g.normal(size=3)
    U = box_vertices((1.0, 1.0, 1.0))
    X = U @ A.T + b
    f, s, n = random_frame(g)
    dl, dt_, dn = 1.3e-3, 0.45e-3, 0.2e-3
    Me, Ke = O.element_matrices(X, np.tile(f, 8), np.tile(s, 8), dl, dt_, dn)
    D = dl * np.outer(f, f) + dt_ * np.outer(s, s) + dn * np.outer(n, n)
    Ai = np.linalg.inv(A)
    det = abs(np.linalg.det(A))
    Mx, Kx = box_closed_form((1.0, 1.0, 1.0), det * Ai @ D @ Ai.T)
    assert np.abs(Me - det * Mx).max() <= 1e-14 * np.abs(Mx).max() * det
    assert np.abs(Ke - Kx).max() <= 1e-12 * np.abs(Kx).max()


def test_element_matrices_rotation_invariance_curved():
    """Rotating a curved element and its fibres together leaves M_e and K_e
    unchanged."""
    g = I.rng(8)
    X = box_vertices((0.1, 0.12, 0.08)) + 0.02 * g.normal(size=(8, 3))
    F = g.normal(size=(8, 3))
    S = g.normal(size=(8, 3))
    R, _ = np.linalg.qr(g.normal(size=(3, 3)))
    M1, K1 = O.element_matrices(X, F, S, 1e-3, 4e-4, 2e-4)
    M2, K2 = O.element_matrices(X @ R.T, F @ R.T, S @ R.T, 1e-3, 4e-4, 2e-4)
    assert np.abs(M1 - M2).max() <= 1e-14 * np.abs(M1).max()
    assert np.abs(K1 - K2).max() <= 1e-12 * np.abs(K1).max()


def trilinear_volume_4pt(X):
    """Volume of a trilinear hexahedron by 4-point Gauss (det J has degree 2 per
    direction, so this is exact too, by a different rule)."""
    xg, wg = np.polynomial.legendre.leggauss(4)
    xg = 0.5 * (xg + 1.0)
    wg = 0.5 * wg
    vol = 0.0
    for i, a in enumerate(xg):
        for j, b in enumerate(xg):
            for k, c in enumerate(xg):
                J = np.zeros((3, 3))
                for n in range(8):
                    ia, ib, ic = n & 1, (n >> 1) & 1, (n >> 2) & 1
                    la, lb, lc = (a if ia else 1 - a), (b if ib else 1 - b), (c if ic else 1 - c)
                    da, db, dc = (1 if ia else -1), (1 if ib else -1), (1 if ic else -1)
                    J[:, 0] += X[n] * da * lb * lc
                    J[:, 1] += X[n] * la * db * lc
                    J[:, 2] += X[n] * la * lb * dc
                vol += wg[i] * wg[j] * wg[k] * np.linalg.det(J)
    return vol


def test_curved_element_mass_sums_to_volume():
    g = I.rng(9)
    X = box_vertices((0.1, 0.1, 0.1)) + 0.015 * g.normal(size=(8, 3))
    Me, Ke = O.element_matrices(X, np.tile([1.0, 0, 0], 8), np.tile([0, 1.0, 0], 8), 1e-3, 1e-3, 1e-3)
    assert abs(Me.sum() - trilinear_volume_4pt(X)) <= 1e-14
    # constants are in the kernel of the stiffness matrix
    assert np.abs(Ke @ np.ones(8)).max() <= 1e-14 * np.abs(Ke).max()
    # symmetric positive semi-definite
    assert np.abs(Ke - Ke.T).max() <= 1e-16 * np.abs(Ke).max() * 100
    assert np.linalg.eigvalsh(Ke).min() >= -1e-14 * np.abs(Ke).max()


def _csr(sim):
    rp, col, mv, kv = sim.matrices()
    n = len(rp) - 1
    M = sp.csr_matrix((mv, col, rp), shape=(n, n))
    K = sp.csr_matrix((kv, col, rp), shape=(n, n))
    return M, K


def _slab_sim(nx, ny, nz, L, rotating=True):
    m = I.slab_mesh(nx, ny, nz, L)
    if rotating:
        f0, s0 = I.rotating_slab_fibres(m["xyz"], L[2])
    else:
        f0, s0 = I.uniform_fibres(m["xyz"].shape[0])
    return O.Sim(m["xyz"], m["hex"], f0, s0, (1e-3, 3.6e-4, 1.8e-4), O.BO, 0.05, 1), m


def test_assembled_slab_invariants():
    sim, m = _slab_sim(6, 5, 4, (0.6, 0.4, 0.3))
    M, K = _csr(sim)
    one = np.ones(M.shape[0])
    assert abs(one @ (M @ one) - 0.6 * 0.4 * 0.3) <= 1e-15 * 10
    assert np.abs(K @ one).max() <= 1e-15 * abs(K).max() * 10
    assert abs(M - M.T).max() <= 1e-15 * abs(M).max()
    assert abs(K - K.T).max() <= 1e-15 * abs(K).max()
    A = (1.5 / 0.05) * M + K
    np.linalg.cholesky(A.toarray())  # raises unless SPD
    # 27-point coupling of structured Q1: interior rows have 27 entries
    assert np.diff(M.indptr).max() == 27


def test_assembled_shell_invariants_and_volume_convergence():
    def shell_volume_exact(a_e=2.5, c_e=6.5, w=1.0, cap=0.1):
        th_cap = math.asin(cap / a_e)
        # |d x/d(t,phi,theta)| for the parametrisation in inputs.shell_mesh
        def jac(th, t):
            a, c = a_e + t * w, c_e + t * w
            # columns: dx/dt, dx/dphi, dx/dtheta at phi = 0 (axisymmetric)
            J = np.array([[w * math.sin(th), 0.0, a * math.cos(th)],
                          [0.0, a * math.sin(th), 0.0],
                          [w * math.cos(th), 0.0, -c * math.sin(th)]])
            return abs(np.linalg.det(J))
        v, _ = scipy.integrate.dblquad(lambda th, t: jac(th, t), 0.0, 1.0,
                                       0.5 * math.pi, math.pi - th_cap, epsabs=1e-12, epsrel=1e-12)
        return 2.0 * math.pi * v

    Vx = shell_volume_exact()
    errs = []
    for (nt, nphi, nl) in [(2, 16, 8), (4, 32, 16)]:
        m, geo = I.shell_mesh(nt, nphi, nl)
        f0, s0 = I.shell_helix_fibres(geo)
        sim = O.Sim(m["xyz"], m["hex"], f0, s0, (1e-3, 3.6e-4, 1.8e-4), O.TTP06, 0.05, 2)
        M, K = _csr(sim)
        one = np.ones(M.shape[0])
        errs.append(abs(one @ (M @ one) - Vx) / Vx)
        assert np.abs(K @ one).max() <= 1e-13 * abs(K).max()
        assert abs(M - M.T).max() <= 1e-15 * abs(M).max()
        assert abs(K - K.T).max() <= 1e-15 * abs(K).max()
        assert M.diagonal().min() > 0
    # second-order geometric convergence of the trilinear mesh volume
    assert errs[1] < errs[0] / 3.0


def test_shell_elements_positively_oriented():
    m, geo = I.shell_mesh(3, 24, 10)
    X = m["xyz"][m["hex"]]
    for e in range(0, X.shape[0], 7):
        Me, _ = O.element_matrices(X[e], np.tile([1.0, 0, 0], 8), np.tile([0, 1.0, 0], 8), 1e-3, 1e-3, 1e-3)
        assert Me.sum() > 0 and np.all(np.diag(Me) > 0)


def test_pcg_matches_direct_solve():
    sim, m = _slab_sim(8, 6, 5, (0.8, 0.6, 0.5))
    M, K = _csr(sim)
    g = I.rng(11)
    b = g.normal(size=M.shape[0])
    A = (1.0 / 0.05) * M + K
    x_direct = spla.spsolve(A.tocsc(), b)
    # run the oracle's CG through a simulation step with a passive membrane:
    # the step solves (1/dt M + K) u = M (u_n/dt - g u_n + iapp); choose iapp
    # so that the right-hand side equals b.
    ps = O.Sim(m["xyz"], m["hex"], *I.rotating_slab_fibres(m["xyz"], 0.5), (1e-3, 3.6e-4, 1.8e-4),
               O.PASSIVE, 0.05, 1, g=0.0, tol=1e-12)
    iapp = spla.spsolve(M.tocsc(), b)
    ps.set_iapp_extra(iapp)
    ps.step(1)
    u = ps.potential()
    assert np.abs(u - x_direct).max() <= 1e-9 * np.abs(x_direct).max()
    assert np.linalg.norm(b - A @ u) <= 1.01e-12 * np.linalg.norm(b)
