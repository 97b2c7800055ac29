"""Python binding of the C ABI in include/ep.h (argument marshalling only).

Every function carries the C name and calls straight into libep_gb300.so,
whose CUDA kernels do all the work; there is no Python or CPU fallback.  If the
library is missing or fails to load, importing this module's functions raises.

Arrays are numpy (float64, uint8), C-contiguous, host memory.  ``Instance``
wraps an ep_instance* with the same calls as methods.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libep_gb300.so")

EP_OK, EP_EINVAL, EP_ENOMEM, EP_ENOCONV, EP_ENAN, EP_ETIMEOUT, EP_ECUDA, EP_EUNSUPPORTED = range(8)
STATUS_NAMES = {0: "EP_OK", 1: "EP_EINVAL", 2: "EP_ENOMEM", 3: "EP_ENOCONV", 4: "EP_ENAN",
                5: "EP_ETIMEOUT", 6: "EP_ECUDA", 7: "EP_EUNSUPPORTED"}
EP_MESH_SLAB, EP_MESH_SHELL, EP_MESH_SLAB_Q2 = 0, 1, 2
EP_MODEL_BO, EP_MODEL_TTP06 = 0, 1
EP_CELL_ENDO, EP_CELL_MID, EP_CELL_EPI = 0, 1, 2
EP_PREC_FP64, EP_PREC_FP32_REFINED = 0, 1
EP_OP_AUTO, EP_OP_MATRIX_FREE, EP_OP_STENCIL = 0, 1, 2
EP_MAX_PULSES = 4

# every function the header declares (checked against include/ep.h by a test)
EXPORTS = ["ep_create", "ep_step", "ep_step_async", "ep_sync", "ep_step_batch", "ep_read_potential",
           "ep_activation_times", "ep_state_bytes", "ep_save_state", "ep_load_state",
           "ep_footprint_bytes", "ep_get_stats", "ep_potential_device", "ep_destroy", "ep_last_error",
           "ep_profile_enable", "ep_profile_read", "ep_residual_norm_noalloc", "ep_prepace",
           "ep_selftest_barrier_timeout"]


class EpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ep_mesh(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("L", C.c_double * 3), ("xyz", C.c_void_p), ("n_nodes", C.c_int64), ("region", C.c_void_p)]


class ep_fibers(C.Structure):
    _fields_ = [("f0", C.c_void_p), ("s0", C.c_void_p)]


EP_MAX_REGIONS = 8


class ep_conductivities(C.Structure):
    _fields_ = [("sigma_l", C.c_double), ("sigma_t", C.c_double), ("sigma_n", C.c_double),
                ("chi_m", C.c_double), ("Cm", C.c_double), ("is_D", C.c_int32), ("n_regions", C.c_int32),
                ("region_sigma", (C.c_double * 3) * EP_MAX_REGIONS),
                ("non_conductive", C.c_uint8 * EP_MAX_REGIONS)]


class ep_ionic_model(C.Structure):
    _fields_ = [("model", C.c_int32), ("cell_type", C.c_void_p), ("initial", C.c_void_p)]


class ep_pulse(C.Structure):
    _fields_ = [("amp", C.c_double), ("t0", C.c_double), ("dur", C.c_double), ("period", C.c_double),
                ("mask", C.c_void_p), ("weight", C.c_void_p), ("elem", C.c_void_p)]


class ep_stimulus(C.Structure):
    _fields_ = [("n_pulses", C.c_int32), ("pulses", C.POINTER(ep_pulse))]


class ep_options(C.Structure):
    _fields_ = [("dt", C.c_double), ("bdf_order", C.c_int32), ("precision", C.c_int32),
                ("tol", C.c_double), ("max_iter", C.c_int32), ("inner_tol", C.c_double),
                ("max_sweeps", C.c_int32), ("op32", C.c_int32), ("cuda_stream", C.c_void_p),
                ("ionic_threads", C.c_int32), ("solve_tiles", C.c_int32)]


class ep_stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("cg_iters", C.c_int32), ("sweeps", C.c_int32),
                ("relres", C.c_double), ("op32", C.c_int32), ("solve_threads", C.c_int32),
                ("device_bytes", C.c_size_t), ("tune_us_mf", C.c_double), ("tune_us_stencil", C.c_double),
                ("ionic_threads", C.c_int32), ("solve_tiles", C.c_int32)]


class ep_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("ms_total", C.c_double)]


_lib = None


def lib():
    """The loaded CUDA library; raises if it is not built or cannot load."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(python paper_2308_01651_gb300/build.py)")
        L = C.CDLL(LIB_PATH)
        P, vp, i64, i32, sz = C.POINTER, C.c_void_p, C.c_int64, C.c_int32, C.c_size_t
        st = C.c_int
        L.ep_create.argtypes = [P(ep_mesh), P(ep_fibers), P(ep_conductivities), P(ep_ionic_model),
                                P(ep_stimulus), P(ep_options), P(vp)]
        L.ep_create.restype = st
        for f in ("ep_step", "ep_step_async"):
            getattr(L, f).argtypes = [vp, i64]
            getattr(L, f).restype = st
        L.ep_sync.argtypes = [vp]
        L.ep_sync.restype = st
        L.ep_step_batch.argtypes = [P(vp), i32, i64]
        L.ep_step_batch.restype = st
        for f in ("ep_read_potential", "ep_activation_times"):
            getattr(L, f).argtypes = [vp, vp, i64]
            getattr(L, f).restype = st
        L.ep_state_bytes.argtypes = [vp]
        L.ep_state_bytes.restype = sz
        L.ep_save_state.argtypes = [vp, vp, sz]
        L.ep_save_state.restype = st
        L.ep_load_state.argtypes = [vp, vp, sz]
        L.ep_load_state.restype = st
        L.ep_footprint_bytes.argtypes = [P(ep_mesh), P(ep_ionic_model), P(ep_options)]
        L.ep_footprint_bytes.restype = sz
        L.ep_get_stats.argtypes = [vp, P(ep_stats)]
        L.ep_get_stats.restype = st
        L.ep_potential_device.argtypes = [vp, P(vp)]
        L.ep_potential_device.restype = st
        L.ep_profile_enable.argtypes = [vp, i32]
        L.ep_profile_enable.restype = st
        L.ep_profile_read.argtypes = [vp, P(ep_kernel_time), i32, P(i32), i32]
        L.ep_profile_read.restype = st
        L.ep_residual_norm_noalloc.argtypes = [vp, P(C.c_double)]
        L.ep_residual_norm_noalloc.restype = st
        L.ep_selftest_barrier_timeout.argtypes = [P(i32)]
        L.ep_selftest_barrier_timeout.restype = st
        d = C.c_double
        L.ep_prepace.argtypes = [i32, vp, i32, d, i32, d, d, d, i32, vp, vp]
        L.ep_prepace.restype = st
        L.ep_destroy.argtypes = [vp]
        L.ep_destroy.restype = st
        L.ep_last_error.argtypes = []
        L.ep_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def ep_last_error():
    return lib().ep_last_error().decode()


def _check(status):
    if status != EP_OK:
        raise EpError(status, ep_last_error())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Args:
    """ctypes structures for one ep_create / ep_footprint_bytes call, keeping
    the numpy buffers they point into alive."""

    def __init__(self, mesh, f0=None, s0=None, cond=None, model=EP_MODEL_TTP06, cell_type=None,
                 pulses=(), dt=0.05, bdf_order=2, precision=EP_PREC_FP64, tol=0.0, max_iter=0,
                 inner_tol=0.0, max_sweeps=0, op32=EP_OP_AUTO, cuda_stream=None, regions=None,
                 initial=None, ionic_threads=0, solve_tiles=0):
        """regions: None, or dict(label=per-element uint8, sigma=[(l, t, n)
        per region] in the units of cond, excluded=[flag per region])."""
        keep = []
        m = ep_mesh()
        m.kind, m.nx, m.ny, m.nz = mesh["kind"], mesh["nx"], mesh["ny"], mesh["nz"]
        for d in range(3):
            m.L[d] = mesh["L"][d]
        if mesh["kind"] == EP_MESH_SHELL:
            xyz = _f64(mesh["xyz"])
            keep.append(xyz)
            m.xyz = _ptr(xyz)
        else:
            m.xyz = None
        m.n_nodes = mesh["xyz"].shape[0] if "xyz" in mesh else mesh["n_nodes"]
        if regions is not None:
            lab = np.ascontiguousarray(regions["label"], dtype=np.uint8)
            keep.append(lab)
            m.region = _ptr(lab)
        self.mesh = m
        fb = ep_fibers()
        if f0 is not None:
            f0, s0 = _f64(f0), _f64(s0)
            keep += [f0, s0]
            fb.f0, fb.s0 = _ptr(f0), _ptr(s0)
        self.fibers = fb
        c = ep_conductivities()
        if cond is not None:
            c.sigma_l, c.sigma_t, c.sigma_n = cond["sigma"]
            c.chi_m, c.Cm, c.is_D = cond["chi_m"], cond["Cm"], 1 if cond["is_D"] else 0
        if regions is not None:
            c.n_regions = len(regions["sigma"])
            for r, sig in enumerate(regions["sigma"]):
                for k in range(3):
                    c.region_sigma[r][k] = sig[k]
                c.non_conductive[r] = 1 if regions["excluded"][r] else 0
        self.cond = c
        io = ep_ionic_model()
        io.model = model
        if cell_type is not None:
            ct = np.ascontiguousarray(cell_type, dtype=np.uint8)
            keep.append(ct)
            io.cell_type = _ptr(ct)
        if initial is not None:
            ini = _f64(initial)
            keep.append(ini)
            io.initial = _ptr(ini)
        self.ionic = io
        arr = (ep_pulse * max(len(pulses), 1))()
        for k, p in enumerate(pulses):
            mk = np.ascontiguousarray(p["mask"], dtype=np.uint8)
            keep.append(mk)
            arr[k].amp, arr[k].t0, arr[k].dur = p["amp"], p["t0"], p["dur"]
            arr[k].period = p.get("period", 0.0)
            arr[k].mask = _ptr(mk)
            if p.get("weight") is not None:
                wt = _f64(p["weight"])
                keep.append(wt)
                arr[k].weight = _ptr(wt)
            if p.get("elem") is not None:
                el = np.ascontiguousarray(p["elem"], dtype=np.uint8)
                keep.append(el)
                arr[k].elem = _ptr(el)
        keep.append(arr)
        s = ep_stimulus()
        s.n_pulses = len(pulses)
        s.pulses = C.cast(arr, C.POINTER(ep_pulse))
        self.stim = s
        o = ep_options()
        o.dt, o.bdf_order, o.precision = dt, bdf_order, precision
        o.tol, o.max_iter, o.inner_tol, o.max_sweeps, o.op32 = tol, max_iter, inner_tol, max_sweeps, op32
        o.cuda_stream = cuda_stream
        o.ionic_threads = ionic_threads
        o.solve_tiles = solve_tiles
        self.opts = o
        self._keep = keep


def ep_create(mesh, f0, s0, cond, model, cell_type=None, pulses=(), **opts):
    """Creates an instance; see ep.h for every argument.  Returns a handle."""
    a = _Args(mesh, f0, s0, cond, model, cell_type, pulses, **opts)
    h = C.c_void_p()
    _check(lib().ep_create(C.byref(a.mesh), C.byref(a.fibers), C.byref(a.cond), C.byref(a.ionic),
                           C.byref(a.stim), C.byref(a.opts), C.byref(h)))
    return h


def ep_footprint_bytes(mesh, model, **opts):
    a = _Args(mesh, model=model, **opts)
    return lib().ep_footprint_bytes(C.byref(a.mesh), C.byref(a.ionic), C.byref(a.opts))


def ep_step(h, n_steps=1):
    _check(lib().ep_step(h, n_steps))


def ep_step_async(h, n_steps=1):
    _check(lib().ep_step_async(h, n_steps))


def ep_sync(h):
    _check(lib().ep_sync(h))


def ep_step_batch(handles, n_steps=1):
    arr = (C.c_void_p * len(handles))(*[x.value if isinstance(x, C.c_void_p) else x for x in handles])
    _check(lib().ep_step_batch(arr, len(handles), n_steps))


def ep_read_potential(h, n):
    out = np.empty(n, dtype=np.float64)
    _check(lib().ep_read_potential(h, _ptr(out), n))
    return out


def ep_activation_times(h, n):
    out = np.empty(n, dtype=np.float64)
    _check(lib().ep_activation_times(h, _ptr(out), n))
    return out


def ep_state_bytes(h):
    return lib().ep_state_bytes(h)


def ep_save_state(h):
    nb = ep_state_bytes(h)
    buf = np.zeros(nb, dtype=np.uint8)
    _check(lib().ep_save_state(h, _ptr(buf), nb))
    return buf


def ep_load_state(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().ep_load_state(h, _ptr(buf), buf.size))


def ep_get_stats(h):
    s = ep_stats()
    _check(lib().ep_get_stats(h, C.byref(s)))
    return dict(step=s.step, cg_iters=s.cg_iters, sweeps=s.sweeps, relres=s.relres, op32=s.op32,
                solve_threads=s.solve_threads,
                device_bytes=s.device_bytes, tune_us_mf=s.tune_us_mf, tune_us_stencil=s.tune_us_stencil,
                ionic_threads=s.ionic_threads, solve_tiles=s.solve_tiles)


def ep_potential_device(h):
    p = C.c_void_p()
    _check(lib().ep_potential_device(h, C.byref(p)))
    return p.value


def ep_profile_enable(h, on=True):
    _check(lib().ep_profile_enable(h, 1 if on else 0))


def ep_profile_read(h, reset=False):
    """{kernel name: (launches, total ms)} since the last reset."""
    cap = 32
    arr = (ep_kernel_time * cap)()
    n = C.c_int32()
    _check(lib().ep_profile_read(h, arr, cap, C.byref(n), 1 if reset else 0))
    return {arr[k].name.decode(): (arr[k].launches, arr[k].ms_total) for k in range(min(n.value, cap))}


def ep_prepace(model, cell_types, period_ms, beats, dt, amp, dur_ms, bdf_order=2, initial=None):
    """Single-cell pre-pacing (ep.h): returns an (n_cells, 1 + S) array of u
    and the states at the end of the last beat."""
    ct = np.ascontiguousarray(cell_types, dtype=np.uint8)
    S1 = 1 + (3 if model == EP_MODEL_BO else 18)
    out = np.zeros((ct.size, S1))
    ini = None if initial is None else _f64(np.asarray(initial).reshape(ct.size, S1))
    _check(lib().ep_prepace(model, _ptr(ct), ct.size, period_ms, beats, dt, amp, dur_ms, bdf_order, _ptr(ini),
                            _ptr(out)))
    return out


def ep_residual_norm_noalloc(h):
    """Relative FP64 residual of the last solve, computed without allocating
    (see ep.h)."""
    out = C.c_double()
    _check(lib().ep_residual_norm_noalloc(h, C.byref(out)))
    return out.value


def ep_selftest_barrier_timeout():
    """The status a timed-out grid barrier records (EP_ETIMEOUT)."""
    out = C.c_int32()
    _check(lib().ep_selftest_barrier_timeout(C.byref(out)))
    return out.value


def ep_destroy(h):
    _check(lib().ep_destroy(h))


# ---- checkpoint buffer layout (ep.h) -------------------------------------

HEADER = np.dtype([("magic", "S8"), ("version", "<i4"), ("model", "<i4"), ("n_nodes", "<i8"),
                   ("n_states", "<i4"), ("bdf_order", "<i4"), ("step", "<i8"), ("dt", "<f8"),
                   ("reserved", "<i8", (2,))])


def state_pack(model, bdf_order, dt, step, u_n, u_nm1, w_n, w_nm1, at, best, u_nm2=None, w_nm2=None):
    """Builds an EPSTATE1 buffer (ep.h layout) from host arrays; BDF3 buffers
    carry the third level (u_nm2, w_nm2)."""
    n = len(u_n)
    ns = w_n.shape[0]
    hdr = np.zeros(1, dtype=HEADER)
    hdr["magic"], hdr["version"], hdr["model"], hdr["n_nodes"] = b"EPSTATE1", 1, model, n
    hdr["n_states"], hdr["bdf_order"], hdr["step"], hdr["dt"] = ns, bdf_order, step, dt
    us, ws = [u_n, u_nm1], [w_n, w_nm1]
    if bdf_order == 3:
        if u_nm2 is None or w_nm2 is None:
            raise ValueError("a BDF3 state needs u_nm2 and w_nm2")
        us.append(u_nm2)
        ws.append(w_nm2)
    body = np.concatenate([_f64(u) for u in us] + [_f64(w).ravel() for w in ws] + [_f64(at), _f64(best)])
    return np.concatenate([hdr.view(np.uint8), body.view(np.uint8)])


def state_unpack(buf):
    hdr = np.frombuffer(buf[:64].tobytes(), dtype=HEADER)[0]
    n, ns = int(hdr["n_nodes"]), int(hdr["n_states"])
    L = 3 if int(hdr["bdf_order"]) == 3 else 2
    # the portable part only (a refined instance's extension follows it)
    body = np.frombuffer(buf[64:64 + 8 * n * (L + L * ns + 2)].tobytes(), dtype=np.float64).copy()
    o = 0

    def take(k):
        nonlocal o
        v = body[o:o + k]
        o += k
        return v

    us = [take(n) for _ in range(L)]
    ws = [take(ns * n).reshape(ns, n) for _ in range(L)]
    at, best = take(n), take(n)
    out = dict(model=int(hdr["model"]), bdf_order=int(hdr["bdf_order"]), step=int(hdr["step"]),
               dt=float(hdr["dt"]), u_n=us[0], u_nm1=us[1], w_n=ws[0], w_nm1=ws[1], at=at, best=best)
    if L == 3:
        out.update(u_nm2=us[2], w_nm2=ws[2])
    return out


class Instance:
    """An ep_instance* with the ABI's calls as methods (created from a
    problem record of the inputs module)."""

    def __init__(self, prob, precision=EP_PREC_FP64, **opts):
        m = prob["mesh"]
        pulses = [dict(p, mask=prob["masks"][k]) for k, p in enumerate(prob["pulses"])]
        self.n = m["xyz"].shape[0]
        self.model = prob["model"]
        self.h = ep_create(m, prob["f0"], prob["s0"], prob["cond"], prob["model"],
                           cell_type=prob["cell"], pulses=pulses, dt=prob["dt"],
                           bdf_order=prob["bdf"], precision=precision, regions=prob.get("regions"),
                           initial=prob.get("initial"), **opts)

    def step(self, n=1):
        ep_step(self.h, n)

    def step_async(self, n=1):
        ep_step_async(self.h, n)

    def sync(self):
        ep_sync(self.h)

    def potential(self):
        return ep_read_potential(self.h, self.n)

    def activation_times(self):
        return ep_activation_times(self.h, self.n)

    def save(self):
        return ep_save_state(self.h)

    def load(self, buf):
        ep_load_state(self.h, buf)

    def stats(self):
        return ep_get_stats(self.h)

    def close(self):
        if self.h:
            ep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
