"""ctypes binding of the FP64 CPU oracle (oracle.h).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the CUDA product path.  The
functions mirror oracle.h one to one; arrays are numpy float64 / int32 /
uint8, C-contiguous.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, i64, i32, vp = C.c_double, C.c_int64, C.c_int, C.c_void_p
        L.or_set_threads.argtypes = [i32]
        L.or_set_threads.restype = i32
        L.or_model_nstates.argtypes = [i32]
        L.or_model_nstates.restype = i32
        L.or_model_initial.argtypes = [i32, i32, vp, vp]
        L.or_model_rates.argtypes = [i32, i32, d, d, vp, vp, vp]
        L.or_model_iion.argtypes = [i32, i32, d, d, vp]
        L.or_model_iion.restype = d
        L.or_cell_step.argtypes = [i32, i32, d, i32, d, d, vp, d, vp, d, vp]
        L.or_cell_step.restype = d
        L.or_element_matrices.argtypes = [vp, vp, vp, d, d, d, vp, vp]
        L.or_element_matrices_q2.argtypes = [vp, vp, vp, d, d, d, vp, vp]
        L.or_assemble_q2.argtypes = [i64, i64, vp, vp, vp, vp, d, d, d, vp]
        L.or_assemble_q2.restype = i32
        L.or_sim_create_q2.argtypes = [i64, i64, vp, vp, vp, vp, d, d, d, i32, vp, d, d,
                                       i32, d, i32, i32, vp, vp, d]
        L.or_sim_create_q2.restype = vp
        L.or_sim_create.argtypes = [i64, i64, vp, vp, vp, vp, d, d, d, i32, vp, d, d,
                                    i32, d, i32, i32, vp, vp, d]
        L.or_sim_create.restype = vp
        L.or_sim_create_regions.argtypes = [i64, i64, vp, vp, vp, vp, vp, i32, vp, vp, i32, vp, d, d,
                                            i32, d, i32, i32, vp, vp, d]
        L.or_sim_create_regions.restype = vp
        L.or_sim_get_active.argtypes = [vp, vp]
        L.or_sim_set_pulse_weights.argtypes = [vp, i32, vp]
        L.or_sim_set_pulse_region.argtypes = [vp, i32, vp]
        L.or_element_region_vector.argtypes = [i64, i64, vp, vp, vp, vp]
        L.or_prepace.argtypes = [i32, i32, i32, d, d, i32, d, d, vp, vp]
        L.or_sim_get_level2.argtypes = [vp, vp, vp]
        L.or_sim_set_level2.argtypes = [vp, vp, vp]
        L.or_assemble_regions.argtypes = [i64, i64, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp]
        L.or_assemble_regions.restype = i32
        L.or_csr_free.argtypes = [vp]
        L.or_sim_destroy.argtypes = [vp]
        L.or_sim_step.argtypes = [vp, i64]
        L.or_sim_step.restype = i32
        L.or_sim_set_iapp_extra.argtypes = [vp, vp]
        L.or_sim_nodes.argtypes = [vp]
        L.or_sim_nodes.restype = i64
        L.or_sim_nstates.argtypes = [vp]
        L.or_sim_nstates.restype = i32
        L.or_sim_stepindex.argtypes = [vp]
        L.or_sim_stepindex.restype = i64
        L.or_sim_last_iters.argtypes = [vp]
        L.or_sim_last_iters.restype = i32
        L.or_sim_last_relres.argtypes = [vp]
        L.or_sim_last_relres.restype = d
        L.or_sim_get_state.argtypes = [vp, vp, vp, vp, vp]
        L.or_sim_set_state.argtypes = [vp, vp, vp, vp, vp, i64]
        L.or_sim_get_activation.argtypes = [vp, vp, vp]
        L.or_sim_set_activation.argtypes = [vp, vp, vp]
        L.or_sim_get_activation_raw.argtypes = [vp, vp, vp]
        L.or_sim_get_iion.argtypes = [vp, vp]
        L.or_sim_matrix.argtypes = [vp]
        L.or_sim_matrix.restype = vp
        _lib = L
    return _lib


BO, TTP06, PASSIVE = 0, 1, 2
ENDO, MID, EPI = 0, 1, 2


def set_threads(n=0):
    """Threads of the oracle's parallel loops (n <= 0: query); returns the
    count in effect (1 when the library was built without OpenMP).  Results
    do not depend on it."""
    return int(lib().or_set_threads(int(n)))


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def nstates(model):
    return lib().or_model_nstates(model)


def initial(model, cell=EPI):
    ns = max(nstates(model), 1)
    u = np.zeros(1)
    w = np.zeros(ns)
    lib().or_model_initial(model, cell, _p(u), _p(w))
    return float(u[0]), w[: nstates(model)]


def rates(model, u, w, cell=EPI, g=0.0):
    ns = max(nstates(model), 1)
    w = _f64(w)
    a = np.zeros(ns)
    b = np.zeros(ns)
    lib().or_model_rates(model, cell, g, float(u), _p(w), _p(a), _p(b))
    return a[: nstates(model)], b[: nstates(model)]


def iion(model, u, w, cell=EPI, g=0.0):
    w = _f64(w) if len(w) else np.zeros(1)
    return lib().or_model_iion(model, cell, g, float(u), _p(w))


def cell_step(model, order, dt, u_n, w_n, u_nm1, w_nm1, iapp, cell=EPI, g=0.0):
    ns = max(nstates(model), 1)
    w_n = _f64(w_n) if len(w_n) else np.zeros(1)
    w_nm1 = _f64(w_nm1) if len(w_nm1) else np.zeros(1)
    out = np.zeros(ns)
    u = lib().or_cell_step(model, cell, g, order, dt, u_n, _p(w_n), u_nm1, _p(w_nm1), iapp, _p(out))
    return u, out[: nstates(model)]


def element_region_vector(xyz, hex8, elem):
    """int_e phi_j summed over the elements with elem[e] != 0, per node j
    (or_element_region_vector): the Gauss-integrated vector of a unit applied
    current on that region of elements."""
    xyz = _f64(xyz).reshape(-1, 3)
    hex8 = np.ascontiguousarray(hex8, dtype=np.int32)
    if hex8.shape[1] != 8:
        raise ValueError("element regions take Q1 hexahedra")
    el = np.ascontiguousarray(elem, dtype=np.uint8).reshape(-1)
    out = np.zeros(xyz.shape[0])
    lib().or_element_region_vector(xyz.shape[0], hex8.shape[0], _p(xyz), _p(hex8), _p(el), _p(out))
    return out


def element_matrices(X, f, s, dl, dt_, dn):
    X, f, s = _f64(X).reshape(8, 3), _f64(f).reshape(8, 3), _f64(s).reshape(8, 3)
    Me = np.zeros((8, 8))
    Ke = np.zeros((8, 8))
    lib().or_element_matrices(_p(X), _p(f), _p(s), dl, dt_, dn, _p(Me), _p(Ke))
    return Me, Ke


def element_matrices_q2(X, f, s, dl, dt_, dn):
    """27-node (Q2) element matrices; local node a = a0 + 3 a1 + 9 a2."""
    X, f, s = _f64(X).reshape(27, 3), _f64(f).reshape(27, 3), _f64(s).reshape(27, 3)
    Me = np.zeros((27, 27))
    Ke = np.zeros((27, 27))
    lib().or_element_matrices_q2(_p(X), _p(f), _p(s), dl, dt_, dn, _p(Me), _p(Ke))
    return Me, Ke


class _CSR(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.POINTER(C.c_int64)),
                ("col", C.POINTER(C.c_int64)), ("mval", C.POINTER(C.c_double)),
                ("kval", C.POINTER(C.c_double))]


def _csr_to_scipy(A, sp):
    n, nnz = A.n, A.nnz
    rowptr = np.ctypeslib.as_array(A.rowptr, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(A.col, shape=(nnz,)).copy()
    mv = np.ctypeslib.as_array(A.mval, shape=(nnz,)).copy()
    kv = np.ctypeslib.as_array(A.kval, shape=(nnz,)).copy()
    return sp.csr_matrix((mv, col, rowptr), shape=(n, n)), sp.csr_matrix((kv, col, rowptr), shape=(n, n))


class Sim:
    """Monodomain simulation (oracle.h, or_sim_*)."""

    def __init__(self, xyz, hex8, f0, s0, D, model, dt, bdf_order, cell=None, g=0.0,
                 tol=1e-12, maxit=1000, pulses=(), masks=None, act_thr=1.0, regions=None):
        """regions: None, or (label per element, [(dl, dt, dn) per region],
        [excluded flag per region]) with diffusivities in cm^2/ms."""
        self.xyz = _f64(xyz)
        self.hex = np.ascontiguousarray(hex8, dtype=np.int32)
        self.f0 = _f64(f0)
        self.s0 = _f64(s0)
        nn, ne = self.xyz.shape[0], self.hex.shape[0]
        self.cell = None if cell is None else np.ascontiguousarray(cell, dtype=np.uint8)
        pl = np.zeros((max(len(pulses), 1), 4))
        for k, p in enumerate(pulses):
            pl[k] = [p["amp"], p["t0"], p["dur"], p.get("period", 0.0)]
        if len(pulses):
            m = np.ascontiguousarray(masks, dtype=np.uint8).reshape(len(pulses), nn)
        else:
            m = np.zeros((1, nn), dtype=np.uint8)
        self._pl, self._m = pl, m
        self.dt = dt
        if self.hex.shape[1] == 27:
            if regions is not None:
                raise ValueError("Q2 meshes take one region")
            self.h = lib().or_sim_create_q2(nn, ne, _p(self.xyz), _p(self.hex), _p(self.f0), _p(self.s0),
                                            D[0], D[1], D[2], model, _p(self.cell), g, dt, bdf_order,
                                            tol, maxit, len(pulses), _p(pl), _p(m), act_thr)
        elif regions is None:
            self.h = lib().or_sim_create(nn, ne, _p(self.xyz), _p(self.hex), _p(self.f0), _p(self.s0),
                                         D[0], D[1], D[2], model, _p(self.cell), g, dt, bdf_order,
                                         tol, maxit, len(pulses), _p(pl), _p(m), act_thr)
        else:
            label, rdiff, excl = regions
            self._label = np.ascontiguousarray(label, dtype=np.uint8)
            self._rdiff = _f64(np.asarray(rdiff, dtype=np.float64).reshape(-1, 3))
            self._excl = np.ascontiguousarray(excl, dtype=np.uint8)
            self.h = lib().or_sim_create_regions(
                nn, ne, _p(self.xyz), _p(self.hex), _p(self.f0), _p(self.s0), _p(self._label),
                self._rdiff.shape[0], _p(self._rdiff), _p(self._excl), model, _p(self.cell), g, dt,
                bdf_order, tol, maxit, len(pulses), _p(pl), _p(m), act_thr)
        if not self.h:
            raise ValueError("or_sim_create failed")
        for k, p in enumerate(pulses):
            if p.get("elem") is not None:
                v = element_region_vector(self.xyz, self.hex, p["elem"])
                lib().or_sim_set_pulse_region(self.h, k, _p(v))
            elif p.get("weight") is not None:
                w = _f64(p["weight"])
                lib().or_sim_set_pulse_weights(self.h, k, _p(w))
        self.nn = nn
        self.ns = lib().or_sim_nstates(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_sim_destroy(self.h)
            self.h = None

    def step(self, n=1):
        rc = lib().or_sim_step(self.h, n)
        if rc != 0:
            raise RuntimeError(f"oracle step failed: {rc}")

    def set_iapp_extra(self, v):
        self._extra = None if v is None else _f64(v)
        lib().or_sim_set_iapp_extra(self.h, _p(self._extra))

    @property
    def stepindex(self):
        return lib().or_sim_stepindex(self.h)

    @property
    def last_iters(self):
        return lib().or_sim_last_iters(self.h)

    @property
    def last_relres(self):
        return lib().or_sim_last_relres(self.h)

    def get_state(self):
        ns = max(self.ns, 1)
        u_n, u_nm1 = np.zeros(self.nn), np.zeros(self.nn)
        w_n, w_nm1 = np.zeros((ns, self.nn)), np.zeros((ns, self.nn))
        lib().or_sim_get_state(self.h, _p(u_n), _p(u_nm1), _p(w_n), _p(w_nm1))
        return u_n, u_nm1, w_n[: self.ns], w_nm1[: self.ns]

    def set_state(self, u_n, u_nm1, w_n, w_nm1, step):
        u_n, u_nm1 = _f64(u_n), _f64(u_nm1)
        w_n = _f64(w_n) if self.ns else np.zeros((1, self.nn))
        w_nm1 = _f64(w_nm1) if self.ns else np.zeros((1, self.nn))
        lib().or_sim_set_state(self.h, _p(u_n), _p(u_nm1), _p(w_n), _p(w_nm1), step)

    def activation(self):
        at, best = np.zeros(self.nn), np.zeros(self.nn)
        lib().or_sim_get_activation(self.h, _p(at), _p(best))
        return at, best

    def activation_raw(self):
        at, best = np.zeros(self.nn), np.zeros(self.nn)
        lib().or_sim_get_activation_raw(self.h, _p(at), _p(best))
        return at, best

    def set_activation(self, at, best):
        at, best = _f64(at), _f64(best)
        lib().or_sim_set_activation(self.h, _p(at), _p(best))

    def potential(self):
        return self.get_state()[0]

    def iion(self):
        v = np.zeros(self.nn)
        lib().or_sim_get_iion(self.h, _p(v))
        return v

    def get_level2(self):
        u = np.zeros(self.nn)
        w = np.zeros((self.ns, self.nn))
        lib().or_sim_get_level2(self.h, _p(u), _p(w))
        return u, w

    def set_level2(self, u_nm2, w_nm2):
        u, w = _f64(u_nm2), _f64(np.asarray(w_nm2).reshape(self.ns, self.nn))
        lib().or_sim_set_level2(self.h, _p(u), _p(w))

    def active(self):
        a = np.zeros(self.nn, dtype=np.uint8)
        lib().or_sim_get_active(self.h, _p(a))
        return a

    def matrices(self):
        """(rowptr, col, M values, K values) of the assembled CSR matrices."""
        A = _CSR.from_address(lib().or_sim_matrix(self.h))
        n, nnz = A.n, A.nnz
        rowptr = np.ctypeslib.as_array(A.rowptr, shape=(n + 1,)).copy()
        col = np.ctypeslib.as_array(A.col, shape=(nnz,)).copy()
        mv = np.ctypeslib.as_array(A.mval, shape=(nnz,)).copy()
        kv = np.ctypeslib.as_array(A.kval, shape=(nnz,)).copy()
        return rowptr, col, mv, kv


def diffusivities(cond):
    """Sec. 1.1.2 rescaling D = sigma / (chi_m C_m), unless the conductivity
    record already holds diffusivities."""
    s = cond["sigma"]
    if cond["is_D"]:
        return tuple(float(x) for x in s)
    return tuple(float(x) / (cond["chi_m"] * cond["Cm"]) for x in s)


def region_diffusivities(prob):
    """(label, per-region diffusivities, excluded flags) of a problem record
    with subdomains, the region conductivities rescaled like the bulk ones."""
    r = prob.get("regions")
    if r is None:
        return None
    c = prob["cond"]
    rd = [diffusivities(dict(c, sigma=tuple(sig))) for sig in r["sigma"]]
    return (r["label"], rd, r["excluded"])


def assemble_regions(prob):
    """Assembled M, K (scipy CSR) and the active-node flags of a problem
    record with subdomains."""
    import scipy.sparse as sp

    m = prob["mesh"]
    label, rd, excl = region_diffusivities(prob)
    xyz, hx = _f64(m["xyz"]), np.ascontiguousarray(m["hex"], dtype=np.int32)
    f0, s0 = _f64(prob["f0"]), _f64(prob["s0"])
    lab = np.ascontiguousarray(label, dtype=np.uint8)
    rdv = _f64(np.asarray(rd, dtype=np.float64).reshape(-1, 3))
    ex = np.ascontiguousarray(excl, dtype=np.uint8)
    nn, ne = xyz.shape[0], hx.shape[0]
    A = _CSR()
    active = np.zeros(nn, dtype=np.uint8)
    rc = lib().or_assemble_regions(nn, ne, _p(xyz), _p(hx), _p(f0), _p(s0), _p(lab), rdv.shape[0], _p(rdv),
                                   _p(ex), C.byref(A), _p(active))
    if rc != 0:
        raise ValueError("or_assemble_regions failed")
    out = _csr_to_scipy(A, sp)
    lib().or_csr_free(C.byref(A))
    return out[0], out[1], active


def assemble_q2(xyz, hex27, f0, s0, D):
    """Assembled M, K (scipy CSR) on 27-node hexahedra."""
    import scipy.sparse as sp

    xyz, hx = _f64(xyz), np.ascontiguousarray(hex27, dtype=np.int32)
    f0, s0 = _f64(f0), _f64(s0)
    A = _CSR()
    rc = lib().or_assemble_q2(xyz.shape[0], hx.shape[0], _p(xyz), _p(hx), _p(f0), _p(s0), D[0], D[1], D[2],
                              C.byref(A))
    if rc != 0:
        raise ValueError("or_assemble_q2 failed")
    out = _csr_to_scipy(A, sp)
    lib().or_csr_free(C.byref(A))
    return out


def sim_from_problem(prob, tol=1e-12, maxit=1000, **kw):
    """Oracle simulation of a problem record built by the inputs module."""
    m = prob["mesh"]
    if prob.get("regions") is not None:
        kw = dict(kw, regions=region_diffusivities(prob))
    return Sim(m["xyz"], m["hex"], prob["f0"], prob["s0"], diffusivities(prob["cond"]),
               prob["model"], prob["dt"], prob["bdf"], cell=prob["cell"], tol=tol, maxit=maxit,
               pulses=prob["pulses"], masks=prob["masks"], act_thr=prob["act_thr"], **kw)


def prepace(model, cell, period, beats, dt, amp, dur, bdf=2, init=None):
    """Single-cell pre-pacing (or_prepace): u and the states at the end."""
    ns = lib().or_model_nstates(model)
    out = np.zeros(1 + ns)
    ini = None if init is None else _f64(init)
    lib().or_prepace(model, cell, bdf, dt, period, beats, amp, dur, _p(ini), _p(out))
    return out
