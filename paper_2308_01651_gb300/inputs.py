"""Seeded synthetic inputs: meshes, fibre fields, cell-type labels, stimulus
masks and whole problem descriptions.

This module holds no arithmetic of the method (no finite elements, no ionic
model, no time stepping).  It is the one piece both the CUDA path and the
oracle consume, so that they see identical inputs.  Shapes follow the paper's
workloads (Sec. 3.2): slabs of cardiac tissue (the N-version benchmark of
Sec. 3.2.1, the layered ventricular slab of Sec. 3.2.4) and an idealised
left-ventricular shell (Sec. 3.2.3), here a truncated prolate ellipsoid.  The
paper's own meshes and LDRBM fibres are not available; analytic fibres and
structured meshes stand in for them.

Units: cm, ms, mV (Bueno-Orovio: dimensionless u), conductivity-derived
diffusivities in cm^2/ms.

Mesh node numbering (both kinds): node (i, j, k) has index
i + (nx+1) * (j + NY * k), with NY = ny + 1 for slabs and NY = ny for the
shell (periodic in j).  Element (i, j, k) has local nodes
a = ia + 2 ib + 4 ic at (i+ia, j+ib, k+ic).

Fibre vectors are rounded to float32-representable doubles so a float32
copy on the device holds exactly the same values.
"""
import math

import numpy as np

MASTER_SEED = 20230803

# model / cell identifiers shared by the C ABI and the oracle
BO, TTP06 = 0, 1
ENDO, MID, EPI = 0, 1, 2
MESH_SLAB, MESH_SHELL, MESH_SLAB_Q2 = 0, 1, 2
# thickness of the slab stimuli's face layer (cm)
STIM_LAYER_CM = 0.04

# activation slope thresholds (model units per ms): 1 mV/ms, i.e. 1/85.7 per ms
# in Bueno-Orovio's dimensionless potential (u_mV = 85.7 u - 84)
ACT_THR = {BO: 1.0 / 85.7, TTP06: 1.0}


def rng(offset=0):
    return np.random.Generator(np.random.PCG64(MASTER_SEED + offset))


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


# ---------------------------------------------------------------- meshes ----

def slab_mesh(nx, ny, nz, L):
    """Structured box [0,Lx]x[0,Ly]x[0,Lz] with nx x ny x nz hexahedra."""
    Lx, Ly, Lz = L
    x = np.arange(nx + 1) * (Lx / nx)
    y = np.arange(ny + 1) * (Ly / ny)
    z = np.arange(nz + 1) * (Lz / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    hexes = _hex_connectivity(nx, ny, nz, periodic_y=False)
    return dict(kind=MESH_SLAB, nx=nx, ny=ny, nz=nz, L=(Lx, Ly, Lz), xyz=xyz, hex=hexes)


def slab_mesh_q2(nx, ny, nz, L):
    """The box [0,Lx]x[0,Ly]x[0,Lz] with nx x ny x nz triquadratic (27-node)
    hexahedra: nodes on the grid of half the element size,
    (2nx+1)(2ny+1)(2nz+1) of them, node (I, J, K) = I + NX (J + NY K); the
    element (i, j, k) holds the nodes 2i..2i+2 x 2j..2j+2 x 2k..2k+2, local
    node a = a0 + 3 a1 + 9 a2 at (2i+a0, 2j+a1, 2k+a2)."""
    Lx, Ly, Lz = L
    NX, NY, NZ = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    x = np.arange(NX) * (Lx / (2 * nx))
    y = np.arange(NY) * (Ly / (2 * ny))
    z = np.arange(NZ) * (Lz / (2 * nz))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    cols = []
    for a in range(27):
        a0, a1, a2 = a % 3, (a // 3) % 3, a // 9
        cols.append((2 * i + a0) + NX * ((2 * j + a1) + NY * (2 * k + a2)))
    hexes = np.stack(cols, axis=1).astype(np.int32)
    return dict(kind=MESH_SLAB_Q2, nx=nx, ny=ny, nz=nz, L=(Lx, Ly, Lz), xyz=xyz, hex=hexes)


def _hex_connectivity(nx, ny, nz, periodic_y):
    NX = nx + 1
    NY = ny if periodic_y else ny + 1
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    cols = []
    for a in range(8):
        ia, ib, ic = a & 1, (a >> 1) & 1, (a >> 2) & 1
        jj = (j + ib) % ny if periodic_y else j + ib
        cols.append((i + ia) + NX * (jj + NY * (k + ic)))
    return np.stack(cols, axis=1).astype(np.int32)


def shell_mesh(nt, nphi, nlong, a_endo=2.5, c_endo=6.5, wall=1.0, cap_radius=0.1):
    """Truncated prolate-ellipsoid shell.

    Point (t, phi, theta): x = (a_e + t w) sin(theta) cos(phi),
    y = (a_e + t w) sin(theta) sin(phi), z = (c_e + t w) cos(theta), with
    t in [0, 1] across the wall (index i), phi periodic (index j, nphi nodes),
    theta from pi - theta_cap at the apex (k = 0) to pi/2 at the base
    (k = nlong, z = 0).  The apical opening of radius cap_radius on the
    endocardium keeps every hexahedron non-degenerate.  Returns the mesh and
    the (t, phi, theta) of each node.
    """
    theta_cap = math.asin(cap_radius / a_endo)
    t = np.linspace(0.0, 1.0, nt + 1)
    phi = np.arange(nphi) * (2.0 * math.pi / nphi)
    theta = np.linspace(math.pi - theta_cap, 0.5 * math.pi, nlong + 1)
    TH, PH, T = np.meshgrid(theta, phi, t, indexing="ij")
    T, PH, TH = T.ravel(), PH.ravel(), TH.ravel()
    a = a_endo + T * wall
    c = c_endo + T * wall
    xyz = np.stack([a * np.sin(TH) * np.cos(PH), a * np.sin(TH) * np.sin(PH), c * np.cos(TH)], axis=1)
    hexes = _hex_connectivity(nt, nphi, nlong, periodic_y=True)
    m = dict(kind=MESH_SHELL, nx=nt, ny=nphi, nz=nlong, L=(0.0, 0.0, 0.0), xyz=xyz, hex=hexes)
    return m, dict(t=T, phi=PH, theta=TH, a_endo=a_endo, c_endo=c_endo, wall=wall)


# ---------------------------------------------------------------- fibres ----

def uniform_fibres(n, f=(1.0, 0.0, 0.0), s=(0.0, 1.0, 0.0)):
    f0 = np.tile(np.asarray(f, dtype=np.float64), (n, 1))
    s0 = np.tile(np.asarray(s, dtype=np.float64), (n, 1))
    return _f32(f0), _f32(s0)


def rotating_slab_fibres(xyz, Lz, deg_bottom=60.0, deg_top=-60.0):
    """Fibres in the x-y plane, angle varying linearly in z (Sec. 3.2.4)."""
    ang = np.deg2rad(deg_bottom + (deg_top - deg_bottom) * (xyz[:, 2] / Lz))
    f0 = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], axis=1)
    s0 = np.stack([-np.sin(ang), np.cos(ang), np.zeros_like(ang)], axis=1)
    return _f32(f0), _f32(s0)


def shell_helix_fibres(geo, deg_endo=60.0, deg_epi=-60.0):
    """Helix angle varying linearly from endocardium to epicardium; the sheet
    direction s0 is the transmural surface normal."""
    T, PH, TH = geo["t"], geo["phi"], geo["theta"]
    a = geo["a_endo"] + T * geo["wall"]
    c = geo["c_endo"] + T * geo["wall"]
    e_phi = np.stack([-np.sin(PH), np.cos(PH), np.zeros_like(PH)], axis=1)
    d_th = np.stack([a * np.cos(TH) * np.cos(PH), a * np.cos(TH) * np.sin(PH), -c * np.sin(TH)], axis=1)
    e_th = d_th / np.linalg.norm(d_th, axis=1, keepdims=True)
    nrm = np.cross(e_th, e_phi)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    alpha = np.deg2rad(deg_endo + (deg_epi - deg_endo) * T)
    f0 = np.cos(alpha)[:, None] * e_phi + np.sin(alpha)[:, None] * e_th
    return _f32(f0), _f32(nrm)


# -------------------------------------------------------- labels, masks -----

def depth_celltype(i_index, nt):
    """Endo / mid / epi by thirds of the wall thickness (node index i of nt)."""
    i = np.asarray(i_index)
    out = np.full(i.shape, EPI, dtype=np.uint8)
    out[3 * i < 2 * nt] = MID
    out[3 * i < nt] = ENDO
    return out


def box_mask(xyz, lo, hi, h):
    """Nodes inside the closed box [lo, hi] with tolerance 1e-9 h."""
    tol = 1e-9 * h
    lo = np.asarray(lo) - tol
    hi = np.asarray(hi) + tol
    return np.all((xyz >= lo) & (xyz <= hi), axis=1).astype(np.uint8)


def element_box_mask(mesh, lo, hi):
    """Elements whose centroid lies in the box [lo, hi] (one byte per element,
    in the connectivity's order): a region of whole elements; for a box whose
    faces are element faces these are exactly the elements inside it."""
    c = mesh["xyz"][mesh["hex"][:, :8]].mean(axis=1)
    return np.all((c >= np.asarray(lo)) & (c <= np.asarray(hi)), axis=1).astype(np.uint8)


def node_ijk(mesh):
    q2 = mesh["kind"] == MESH_SLAB_Q2
    NX = 2 * mesh["nx"] + 1 if q2 else mesh["nx"] + 1
    NY = mesh["ny"] if mesh["kind"] == MESH_SHELL else (2 * mesh["ny"] + 1 if q2 else mesh["ny"] + 1)
    idx = np.arange(mesh["xyz"].shape[0])
    return idx % NX, (idx // NX) % NY, idx // (NX * NY)


def face_layer_mask(mesh, face, thickness=STIM_LAYER_CM):
    """Nodes within `thickness` (cm) of a face of a slab (face 0..5 = x-, x+,
    y-, y+, z-, z+): a single node layer at the face carries the current of
    half an element (Q1) or a sixth (Q2) and does not start a propagating
    wave in these slabs (checked: with it alone the TTP06 slab activates
    seven node layers and the front dies)."""
    d = face // 2
    x = mesh["xyz"][:, d]
    L = mesh["L"][d]
    tol = 1e-9 * max(L, 1e-300)
    near = x <= thickness + tol if face % 2 == 0 else x >= L - thickness - tol
    return near.astype(np.uint8)


def face_mask(mesh, face):
    """Nodes on a face of a slab: face in 0..5 = x-, x+, y-, y+, z-, z+."""
    i, j, k = node_ijk(mesh)
    n = (mesh["nx"], mesh["ny"], mesh["nz"])[face // 2] * (2 if mesh["kind"] == MESH_SLAB_Q2 else 1)
    idx = (i, j, k)[face // 2]
    return (idx == (0 if face % 2 == 0 else n)).astype(np.uint8)


# -------------------------------------------------------------- problems ----

def cond_D(dl, dt_, dn):
    """Conductivity record holding diffusivities directly (cm^2/ms)."""
    return dict(sigma=(float(dl), float(dt_), float(dn)), chi_m=1.0, Cm=1.0, is_D=True)


def cond_sigma(sl, st, sn, chi_m=1400.0, Cm=1.0):
    """Conductivity record holding conductivities (mS/cm), the membrane
    surface-to-volume ratio chi_m (1/cm) and capacitance C_m (uF/cm^2); each
    consumer rescales them to diffusivities itself."""
    return dict(sigma=(float(sl), float(st), float(sn)), chi_m=float(chi_m), Cm=float(Cm), is_D=False)


def problem(mesh, f0, s0, cond, model, dt, bdf, T, pulses, masks, cell=None, name=""):
    n = mesh["xyz"].shape[0]
    if cell is None:
        cell = np.full(n, EPI, dtype=np.uint8)
    return dict(name=name, mesh=mesh, f0=f0, s0=s0, cond=cond, model=model, cell=cell,
                dt=dt, bdf=bdf, T=T, nsteps=int(round(T / dt)), pulses=list(pulses),
                masks=np.asarray(masks, dtype=np.uint8).reshape(len(pulses), n),
                act_thr=ACT_THR[model])


def slab_bo_small(nx=20, ny=10, nz=5, L=(1.0, 0.5, 0.25), T=100.0, amp=1.0):
    """Bueno-Orovio slab, 1386 nodes at the default size: f0 along x,
    D_l = 1.3e-3, D_t = D_n = 0.45e-3 cm^2/ms, BDF1, dt 0.05 ms, 1 ms pulse
    in a 0.1 cm corner cube."""
    m = slab_mesh(nx, ny, nz, L)
    n = m["xyz"].shape[0]
    f0, s0 = uniform_fibres(n)
    h = min(L[0] / nx, L[1] / ny, L[2] / nz)
    mask = box_mask(m["xyz"], (0, 0, 0), (0.1, 0.1, 0.1), h)
    return problem(m, f0, s0, cond_D(1.3e-3, 0.45e-3, 0.45e-3), BO, 0.05, 1, T,
                   [dict(amp=amp, t0=0.0, dur=1.0, period=0.0)], [mask], name="slab_bo")


def slab_ttp06(nx=200, ny=70, nz=30, L=(2.0, 0.7, 0.3), T=400.0, bdf=2, dt=0.05):
    """TTP06 epicardial slab, 442,401 nodes at the default size: fibre angle
    +60 -> -60 deg linear in z, sigma 1.4/0.5/0.25 mS/cm, chi_m 1400/cm,
    C_m 1 uF/cm^2, BDF2, dt 0.05 ms; stimulus in the layer x <= 0.04 cm at
    the x = 0 face, 35.714 mV/ms for 2 ms (the paper's N-version
    amplitude)."""
    m = slab_mesh(nx, ny, nz, L)
    f0, s0 = rotating_slab_fibres(m["xyz"], L[2])
    mask = face_layer_mask(m, 0)
    return problem(m, f0, s0, cond_sigma(1.4, 0.5, 0.25), TTP06, dt, bdf, T,
                   [dict(amp=35.714, t0=0.0, dur=2.0, period=0.0)], [mask], name="slab_ttp06")


def slab_ttp06_q2(nx=100, ny=35, nz=15, L=(2.0, 0.7, 0.3), T=400.0, bdf=2, dt=0.05):
    """The TTP06 slab of slab_ttp06 on triquadratic elements of twice the
    size: the same node grid (201 x 71 x 31 = 442,401 nodes at the default
    size), fibres, conductivities, time step and stimulus amplitude.  The
    stimulus covers x <= 0.04 cm (two element layers): on Q2 elements the
    x = 0 face alone carries a sixth of an element layer's current (the
    integral of the face's basis functions) and starts no wave."""
    m = slab_mesh_q2(nx, ny, nz, L)
    f0, s0 = rotating_slab_fibres(m["xyz"], L[2])
    mask = face_layer_mask(m, 0)
    return problem(m, f0, s0, cond_sigma(1.4, 0.5, 0.25), TTP06, dt, bdf, T,
                   [dict(amp=35.714, t0=0.0, dur=2.0, period=0.0)], [mask], name="slab_ttp06_q2")


def slab_bo_q2(nx=10, ny=5, nz=3, L=(1.0, 0.5, 0.3), T=60.0, amp=1.0, bdf=1):
    """Bueno-Orovio slab on triquadratic elements: f0 along x, D_l = 1.3e-3,
    D_t = D_n = 0.45e-3 cm^2/ms, dt 0.05 ms, 1 ms pulse in a 0.1 cm corner
    cube."""
    m = slab_mesh_q2(nx, ny, nz, L)
    n = m["xyz"].shape[0]
    f0, s0 = uniform_fibres(n)
    h = min(L[0] / nx, L[1] / ny, L[2] / nz) / 2
    mask = box_mask(m["xyz"], (0, 0, 0), (0.1, 0.1, 0.1), h)
    return problem(m, f0, s0, cond_D(1.3e-3, 0.45e-3, 0.45e-3), BO, 0.05, bdf, T,
                   [dict(amp=amp, t0=0.0, dur=1.0, period=0.0)], [mask], name="slab_bo_q2")


def nversion(dx=0.01, dt=0.005, T=50.0, stimulus="elements"):
    """N-version benchmark slab (Sec. 3.2.1): 20 x 7 x 3 mm, fibres along
    the long axis (x here), TTP06 epicardial, D_l = 0.95298e-3,
    D_t = D_n = 0.12576e-3 cm^2/ms (the paper's 0.95298e-4 / 0.12576e-4 m^2/s),
    35.714 mV/ms for 2 ms in a 1.5 mm corner cube, BDF2.  stimulus:
    "elements" -- the cube as a region of elements, its current integrated by
    the Gauss rule (the cubic impulse as a function of space); "nodes" -- the
    nodes of the closed cube, entering as M I_app(nodes)."""
    L = (2.0, 0.7, 0.3)
    nx, ny, nz = (int(round(l / dx)) for l in L)
    m = slab_mesh(nx, ny, nz, L)
    n = m["xyz"].shape[0]
    f0, s0 = uniform_fibres(n)
    mask = box_mask(m["xyz"], (0, 0, 0), (0.15, 0.15, 0.15), dx)
    pulse = dict(amp=35.714, t0=0.0, dur=2.0, period=0.0)
    if stimulus == "elements":
        pulse["elem"] = element_box_mask(m, (0, 0, 0), (0.15, 0.15, 0.15))
    elif stimulus != "nodes":
        raise ValueError(stimulus)
    return problem(m, f0, s0, cond_D(0.95298e-3, 0.12576e-3, 0.12576e-3), TTP06, dt, 2, T,
                   [pulse], [mask], name="nversion")


def shell_ttp06(nt=20, nphi=400, nlong=260, T=500.0, dt=0.05, bdf=2):
    """Truncated prolate-ellipsoid LV shell, endocardial semi-axes
    2.5/2.5/6.5 cm, wall 1 cm; helix fibres +60 -> -60 deg, s0 transmural;
    TTP06 endo/mid/epi by thirds of the wall; stimulus on the apical three
    element rows; 2,192,400 nodes at the default size."""
    m, geo = shell_mesh(nt, nphi, nlong)
    f0, s0 = shell_helix_fibres(geo)
    i, j, k = node_ijk(m)
    cell = depth_celltype(i, nt)
    mask = (k <= 3).astype(np.uint8)
    p = problem(m, f0, s0, cond_sigma(1.4, 0.5, 0.25), TTP06, dt, bdf, T,
                [dict(amp=35.714, t0=0.0, dur=2.0, period=0.0)], [mask], cell=cell, name="shell_ttp06")
    p["geo"] = geo
    return p


def as_bo(prob, amp=1.0, dur=2.0):
    """The same geometry, fibres, conductivities and stimulated nodes with the
    Bueno-Orovio model (amplitude in its units per ms)."""
    pulses = [dict(p, amp=amp, dur=dur) for p in prob["pulses"]]
    q = problem(prob["mesh"], prob["f0"], prob["s0"], prob["cond"], BO, prob["dt"], prob["bdf"], prob["T"],
                pulses, prob["masks"], name=prob["name"] + "_bo")
    for k in ("geo",):
        if k in prob:
            q[k] = prob[k]
    return q


def sphere_mask(xyz, centre, radius, h=1.0):
    """Nodes inside a ball (closed, with a tolerance of 1e-9 h): the
    paper's spherical impulse."""
    d = np.linalg.norm(np.asarray(xyz) - np.asarray(centre, dtype=np.float64), axis=1)
    return (d <= radius + 1e-9 * h).astype(np.uint8)


def gaussian_weight(xyz, centre, sd):
    """exp(-|x - c|^2 / (2 sd^2)) at every node: the paper's Gaussian
    impulse profile (site c, standard deviation sd)."""
    d2 = np.sum((np.asarray(xyz) - np.asarray(centre, dtype=np.float64)) ** 2, axis=1)
    return np.exp(-d2 / (2.0 * sd * sd))


def slab_gaussian_pacing(nx=30, ny=10, nz=5, h=0.01, T=20.0, dt=0.05, model=None, sites=None, sd=0.025,
                         amp=None, period=0.0, dur=2.0):
    """Slab paced by Gaussian impulses (Sec. 3.2, the idealised ventricle's
    protocol): one pulse per site, each with its own profile; TTP06 by
    default (amplitude 35.714 mV/ms), Bueno-Orovio with model=BO (1/ms)."""
    L = (nx * h, ny * h, nz * h)
    p = slab_ttp06(nx=nx, ny=ny, nz=nz, L=L, T=T, dt=dt)
    if model == BO:
        p = as_bo(p)
    if sites is None:
        sites = [(0.2 * L[0], 0.5 * L[1], 0.0), (0.8 * L[0], 0.2 * L[1], L[2])]
    a = amp if amp is not None else (35.714 if p["model"] == TTP06 else 1.0)
    xyz = p["mesh"]["xyz"]
    pulses, masks = [], []
    for c in sites:
        w = gaussian_weight(xyz, c, sd)
        pulses.append(dict(amp=a, t0=0.0, dur=dur, period=period, weight=w))
        masks.append((w > 1e-3).astype(np.uint8))
    q = problem(p["mesh"], p["f0"], p["s0"], p["cond"], p["model"], p["dt"], p["bdf"], T, pulses, masks,
                name=p["name"] + "_gauss")
    return q


def element_centroids(mesh):
    """Centroid of every element (element order of the connectivity)."""
    return mesh["xyz"][mesh["hex"]].mean(axis=1)


def slab_regions(nx=40, ny=12, nz=6, h=0.01, T=20.0, dt=0.05, bdf=2, model=None, wall=False):
    """TTP06 slab with subdomains (Sec. 1.1.2): region 0 healthy tissue, region
    1 a grey zone with the conductivities halved, region 2 a non-conductive
    scar.  wall=False: a scar block in the middle of the slab (x in
    [0.4, 0.6], y in [0.25, 0.75] of the lengths, through z) ringed by a grey
    zone 0.15 of the length wide; wall=True: a scar layer across the whole
    section at x in [0.45, 0.55] of the length (a complete conduction
    block).  Stimulus on the x = 0 face."""
    L = (nx * h, ny * h, nz * h)
    p = slab_ttp06(nx=nx, ny=ny, nz=nz, L=L, T=T, bdf=bdf, dt=dt)
    if model == BO:
        p = as_bo(p)
    c = element_centroids(p["mesh"]) / np.array(L)
    label = np.zeros(c.shape[0], dtype=np.uint8)
    if wall:
        label[(c[:, 0] >= 0.45) & (c[:, 0] <= 0.55)] = 2
    else:
        grey = (c[:, 0] >= 0.25) & (c[:, 0] <= 0.75) & (c[:, 1] >= 0.1) & (c[:, 1] <= 0.9)
        scar = (c[:, 0] >= 0.4) & (c[:, 0] <= 0.6) & (c[:, 1] >= 0.25) & (c[:, 1] <= 0.75)
        label[grey] = 1
        label[scar] = 2
    s0 = tuple(p["cond"]["sigma"])
    p["regions"] = dict(label=label, sigma=[s0, tuple(0.5 * x for x in s0), s0], excluded=[0, 0, 1])
    p["name"] = p["name"] + ("_wall" if wall else "_scar")
    return p


def batch_slabs(count=96, n_lo=2.0e4, n_hi=4.0e5, T=300.0, dt=0.05, seed_offset=2, h=0.01):
    """Uneven batch of slabs: node counts log-uniform in [n_lo, n_hi], aspect
    nx/ny uniform in [1, 4] with nz = ny, h = 0.01 cm, model Bernoulli(1/2)
    Bueno-Orovio / TTP06, each conductivity times lognormal(0, 0.3), stimulus
    in the 0.04 cm layer at a uniformly chosen face."""
    g = rng(seed_offset)
    out = []
    for b in range(count):
        N = math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))
        a = g.uniform(1.0, 4.0)
        ny = max(2, int(round((N / a) ** (1.0 / 3.0) - 1.0)))
        nx = max(2, int(round(a * (ny + 1) - 1)))
        nz = ny
        model = TTP06 if g.uniform() < 0.5 else BO
        sig = np.array([1.4, 0.5, 0.25]) * np.exp(g.normal(0.0, 0.3, size=3))
        face = int(g.integers(0, 6))
        m = slab_mesh(nx, ny, nz, (nx * h, ny * h, nz * h))
        n = m["xyz"].shape[0]
        f0, s0 = uniform_fibres(n)
        mask = face_layer_mask(m, face)
        amp, dur = (35.714, 2.0) if model == TTP06 else (1.0, 2.0)
        out.append(problem(m, f0, s0, cond_sigma(*sig), model, dt, 2, T,
                           [dict(amp=amp, t0=0.0, dur=dur, period=0.0)], [mask],
                           name=f"batch{b}"))
    return out
