"""Seeded synthetic inputs: T10 box / cylinder meshes, ANCF beam / shell meshes,
nodal fields, load schedules.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests. It holds none of the method's arithmetic: it only builds
geometry (node coordinates, element connectivity) and draws random numbers.
Everything the method computes (shape functions, quadrature, stresses,
assembly) lives on either side of the parity tests, never here.

Mesh convention (shared interface, not arithmetic):
  * T10 node order: corners 0..3, then midside nodes on edges
    4:(0,1) 5:(1,2) 6:(0,2) 7:(0,3) 8:(1,3) 9:(2,3).
    The paper leaves the ordering open (T10 has 10 shape functions, Sec. 4.3);
    this is the VTK quadratic-tetra order.
  * Corners are ordered so that det[x1-x0, x2-x0, x3-x0] > 0.
  * Midside nodes sit exactly at edge midpoints (straight-sided elements).
  * Box meshes: nx*ny*nz hexahedra, each cut into 6 tetrahedra by the Kuhn
    (Freudenthal) split along the (0,0,0)-(1,1,1) diagonal, which is conforming
    between neighbouring hexahedra.  The T10 nodes are then exactly the
    (2nx+1)(2ny+1)(2nz+1) points of the half-spacing grid; node id
    = (i*NY + j)*NZ + k with i along x (slowest).

The workloads mirror the paper's T10 cantilever scaling benchmark (Sec. 5.1):
a box clamped on its x = 0 face.  The paper's own meshes are not available, so
these seeded boxes stand in for them.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

T10_EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))


@dataclass
class Mesh:
    X: np.ndarray            # (nn, 3) float64 reference coordinates
    conn: np.ndarray         # (ne, 10) int32 connectivity
    fixed_nodes: np.ndarray  # (nfixed,) int32, sorted
    extent: tuple            # (Lx, Ly, Lz) bounding box lengths
    hex_size: tuple          # (hx, hy, hz) hexahedron edge per axis
    body_of_elem: np.ndarray | None = None   # (ne,) int32 for multi-body meshes
    body_of_node: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def nn(self):
        return self.X.shape[0]

    @property
    def ne(self):
        return self.conn.shape[0]


def _kuhn_corner_offsets():
    """The 6 Kuhn tetrahedra of the unit cube as corner offset lists."""
    tets = []
    for perm in itertools.permutations(range(3)):
        p = np.zeros(3, dtype=np.int64)
        path = [p.copy()]
        for ax in perm:
            p = p.copy()
            p[ax] += 1
            path.append(p)
        tets.append(np.stack(path))          # (4, 3) offsets in {0,1}
    return np.stack(tets)                     # (6, 4, 3)


def _orient_and_midsides(gcorner):
    """gcorner: (ne, 4, 3) integer grid coords (even) of corners.

    Returns (ne, 10, 3) integer grid coords with corners oriented positively
    and midside nodes at edge midpoints.
    """
    d1 = gcorner[:, 1] - gcorner[:, 0]
    d2 = gcorner[:, 2] - gcorner[:, 0]
    d3 = gcorner[:, 3] - gcorner[:, 0]
    vol6 = np.einsum("ei,ei->e", np.cross(d1, d2), d3)
    neg = vol6 < 0
    g = gcorner.copy()
    g[neg, 1], g[neg, 2] = gcorner[neg, 2], gcorner[neg, 1]
    mids = [(g[:, a] + g[:, b]) // 2 for a, b in T10_EDGES]
    return np.concatenate([g, np.stack(mids, axis=1)], axis=1)


def box_t10(nx, ny, nz, Lx, Ly, Lz, fixed_face_x0=True):
    """Structured T10 box mesh (see module docstring)."""
    NX, NY, NZ = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    xs = np.linspace(0.0, Lx, NX)
    ys = np.linspace(0.0, Ly, NY)
    zs = np.linspace(0.0, Lz, NZ)
    gx, gy, gz = np.meshgrid(xs, ys, zs, indexing="ij")
    X = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)

    hi, hj, hk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hexes = np.stack([hi.ravel(), hj.ravel(), hk.ravel()], axis=1)   # (nhex, 3)
    offs = _kuhn_corner_offsets()                                      # (6, 4, 3)
    gcorner = 2 * (hexes[:, None, None, :] + offs[None, :, :, :])      # (nhex, 6, 4, 3)
    gcorner = gcorner.reshape(-1, 4, 3)
    g = _orient_and_midsides(gcorner)                                  # (ne, 10, 3)
    conn = (g[..., 0] * NY + g[..., 1]) * NZ + g[..., 2]
    conn = conn.astype(np.int32)
    if fixed_face_x0:
        fixed = np.nonzero(X[:, 0] == 0.0)[0].astype(np.int32)
    else:
        fixed = np.zeros(0, dtype=np.int32)
    return Mesh(X=X, conn=conn, fixed_nodes=fixed, extent=(Lx, Ly, Lz),
                hex_size=(Lx / nx, Ly / ny, Lz / nz),
                meta=dict(kind="box", n=(nx, ny, nz)))


def cylinder_t10(nr, nz, R, Lz, fixed_face_z0=True):
    """T10 cylinder: a (2nr x 2nr x nz) hexahedral block whose square cross
    section is mapped onto the disk of radius R (square-to-disk map), then
    Kuhn-split.  Axis along z; the clamped face is z = 0."""
    m = box_t10(2 * nr, 2 * nr, nz, 2.0, 2.0, Lz, fixed_face_x0=False)
    a = m.X[:, 0] - 1.0
    b = m.X[:, 1] - 1.0
    # elliptical-grid square-to-disk map (Fong): smooth, keeps straight midsides
    # only approximately, so midside nodes are re-placed at edge midpoints below.
    u = a * np.sqrt(np.maximum(0.0, 1.0 - 0.5 * b * b))
    w = b * np.sqrt(np.maximum(0.0, 1.0 - 0.5 * a * a))
    X = np.stack([R * u, R * w, m.X[:, 2]], axis=1)
    # corners first, then midsides as the mean of their edge's corners
    conn = m.conn
    for mid, (p, q) in enumerate(T10_EDGES, start=4):
        X[conn[:, mid]] = 0.5 * (X[conn[:, p]] + X[conn[:, q]])
    fixed = (np.nonzero(m.X[:, 2] == 0.0)[0].astype(np.int32)
             if fixed_face_z0 else np.zeros(0, dtype=np.int32))
    return Mesh(X=X, conn=conn, fixed_nodes=fixed, extent=(2 * R, 2 * R, Lz),
                hex_size=(2 * R / (2 * nr), 2 * R / (2 * nr), Lz / nz),
                meta=dict(kind="cylinder", n=(nr, nz)))


# ---------------------------------------------------------------------------
# Nodal fields
# ---------------------------------------------------------------------------

def uniform_perturbation(mesh, frac, rng, local=False):
    """q = X + U(-frac*h_i, frac*h_i) per axis per node; clamped nodes stay at X.
    h_i is the hex edge of the structured grid, or with local=True the node's
    own spacing: half the smallest altitude of the elements at the node (the
    cylinder's square-to-disk map makes rim elements much flatter than the
    grid spacing)."""
    if local:
        c = mesh.conn[:, :4]
        P = mesh.X[c]
        vol6 = np.abs(np.einsum("ij,ij->i", P[:, 1] - P[:, 0],
                                np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0])))
        faces = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))
        area2 = np.stack([np.linalg.norm(np.cross(P[:, j] - P[:, i], P[:, k] - P[:, i]), axis=1)
                          for i, j, k in faces], axis=1)
        he = 0.5 * vol6 / area2.max(axis=1)          # half the smallest altitude
        hn = np.full(mesh.nn, np.inf)
        np.minimum.at(hn, mesh.conn.ravel(), np.repeat(he, 10))
        scale = (frac * hn)[:, None]
    else:
        scale = (frac * np.asarray(mesh.hex_size))[None, :]
    d = rng.uniform(-1.0, 1.0, size=mesh.X.shape) * scale
    d[mesh.fixed_nodes] = 0.0
    return mesh.X + d


def gaussian_velocity(mesh, sigma, rng):
    v = rng.normal(0.0, sigma, size=mesh.X.shape)
    v[mesh.fixed_nodes] = 0.0
    return v


def _min_corner_volume_ratio(mesh, x):
    """Smallest ratio of deformed to reference corner-tetrahedron volume: a
    geometric sanity check of a generated displacement field."""
    c = mesh.conn[:, :4]

    def vol(P):
        a, b, d, e = P[c[:, 0]], P[c[:, 1]], P[c[:, 2]], P[c[:, 3]]
        return np.einsum("ei,ei->e", np.cross(b - a, d - a), e - a)

    return float(np.min(vol(x) / vol(mesh.X)))


def sine_mode_field(mesh, amp_frac, rng, nmodes=8, min_ratio=0.2, max_halvings=8):
    """Smooth seeded displacement: u(X) = s(x) * sum_m a_m d_m sin(2*pi*k_m.X/L + phi_m).

    k_m = (n_x, n_y, n_z) with n_x in {1,2,3} and n_y, n_z in {0,1}; d_m random
    unit directions, phi_m ~ U(0, 2pi), a_m ~ U(0.5, 1).  The envelope
    s(x) = x / Lx keeps the clamped x = 0 face at rest.  The field is rescaled
    so that max |u| = amp_frac * Lx.  While the smallest corner-volume ratio is
    at or below `min_ratio`, the modes with a transverse wavenumber are halved
    (then the field is rescaled again); the number of halvings is returned.
    """
    L = np.asarray(mesh.extent, dtype=np.float64)
    nxs = rng.integers(1, 4, size=nmodes)
    nys = rng.integers(0, 2, size=nmodes)
    nzs = rng.integers(0, 2, size=nmodes)
    d = rng.normal(size=(nmodes, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=nmodes)
    amp = rng.uniform(0.5, 1.0, size=nmodes)
    k = np.stack([nxs, nys, nzs], axis=1).astype(np.float64)
    transverse = (nys + nzs) > 0
    X = mesh.X
    env = (X[:, 0] - X[:, 0].min()) / L[0]
    arg = 2.0 * np.pi * (X / L[None, :]) @ k.T + phi[None, :]      # (nn, nmodes)
    S = np.sin(arg)
    halvings = 0
    while True:
        u = env[:, None] * ((S * amp[None, :]) @ d)
        u *= (amp_frac * L[0]) / np.max(np.linalg.norm(u, axis=1))
        u[mesh.fixed_nodes] = 0.0
        ratio = _min_corner_volume_ratio(mesh, X + u)
        if ratio > min_ratio or halvings >= max_halvings or not transverse.any():
            break
        amp = np.where(transverse, 0.5 * amp, amp)
        halvings += 1
    return X + u, dict(halvings=halvings, min_corner_ratio=ratio,
                       modes=k.astype(int).tolist())


def tip_load_schedule(mesh, nsteps, period, max_force, rng):
    """Seeded tip load: every `period` steps a new total force of magnitude
    U(0, max_force) in a random unit direction, split uniformly over the nodes
    of the x = Lx face.  Returns a function step -> (nn*3,) external force."""
    xmax = mesh.X[:, 0].max()
    tip = np.nonzero(np.isclose(mesh.X[:, 0], xmax))[0]
    nseg = (nsteps + period - 1) // period
    mags = rng.uniform(0.0, max_force, size=nseg)
    dirs = rng.normal(size=(nseg, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)

    def f_ext(step):
        s = min(step // period, nseg - 1)
        f = np.zeros((mesh.nn, 3))
        f[tip] = (mags[s] * dirs[s]) / len(tip)
        return f.reshape(-1)

    return f_ext


def merge_meshes(meshes):
    """Concatenate independent meshes into one multi-body mesh (no shared nodes)."""
    Xs, conns, fixed, boe, bon = [], [], [], [], []
    off = 0
    for b, m in enumerate(meshes):
        Xs.append(m.X)
        conns.append(m.conn + off)
        fixed.append(m.fixed_nodes + off)
        boe.append(np.full(m.ne, b, dtype=np.int32))
        bon.append(np.full(m.nn, b, dtype=np.int32))
        off += m.nn
    X = np.concatenate(Xs)
    return Mesh(X=X, conn=np.concatenate(conns).astype(np.int32),
                fixed_nodes=np.concatenate(fixed).astype(np.int32),
                extent=tuple(X.max(0) - X.min(0)), hex_size=meshes[0].hex_size,
                body_of_elem=np.concatenate(boe), body_of_node=np.concatenate(bon),
                meta=dict(kind="multi", nbodies=len(meshes)))


# ---------------------------------------------------------------------------
# The configured workloads (seeds: numpy default_rng(1000 + k) for workload k)
# ---------------------------------------------------------------------------

GRAVITY = (0.0, 0.0, -9.81)

SVK_1E7 = dict(kind="svk", E=1e7, nu=0.3, rho0=1000.0)
MR_C2 = dict(kind="mr", C10=5e5, C01=1e5, kappa=1e8, rho0=1000.0)


def workload_small_svk():
    """Cantilever box 1.0 x 0.1 x 0.1 m, 10x2x2 hexes -> 240 T10, 525 nodes.
    SVK E=1e7, nu=0.3, rho=1000; q_n = X +- 1% hex size; v ~ N(0, 0.01)."""
    rng = np.random.default_rng(1000 + 1)
    m = box_t10(10, 2, 2, 1.0, 0.1, 0.1)
    q = uniform_perturbation(m, 0.01, rng)
    v = gaussian_velocity(m, 0.01, rng)
    mat = dict(SVK_1E7, eta_d=0.0, lambda_d=0.0)
    return dict(name="box 1.0x0.1x0.1 m, 10x2x2 hex x6 = 240 T10, SVK", mesh=m,
                q_n=q, v=v, material=mat, h=1e-3)


def workload_mid_mr_kv():
    """Box 4.0 x 0.8 x 0.8 m, 40x8x8 hexes -> 15,360 T10, 23,409 nodes.
    Compressible Mooney-Rivlin C10=5e5, C01=1e5, kappa=1e8 plus Kelvin-Voigt
    eta = lambda_d = 1e3; 8 sine modes at 5% of the length; v ~ N(0, 0.05)."""
    rng = np.random.default_rng(1000 + 2)
    m = box_t10(40, 8, 8, 4.0, 0.8, 0.8)
    q, info = sine_mode_field(m, 0.05, rng)
    v = gaussian_velocity(m, 0.05, rng)
    mat = dict(MR_C2, eta_d=1e3, lambda_d=1e3)
    return dict(name="box 4.0x0.8x0.8 m, 40x8x8 hex x6 = 15,360 T10, MR+KV", mesh=m,
                q_n=q, v=v, material=mat, h=1e-3, field_info=info)


def workload_large_svk_kv(scale=1):
    """Box 20 x 4 x 2 m, 200x40x20 hexes -> 960,000 T10, 1,331,721 nodes.
    SVK E=1e7, nu=0.3 plus Kelvin-Voigt 1e3; 8 sine modes at 2% of the length;
    v ~ N(0, 0.05).  `scale` < 1 shrinks the hex counts (same physical box)
    for quick runs."""
    rng = np.random.default_rng(1000 + 5)
    nx, ny, nz = (max(1, int(round(200 * scale))), max(1, int(round(40 * scale))),
                  max(1, int(round(20 * scale))))
    m = box_t10(nx, ny, nz, 20.0, 4.0, 2.0)
    q, info = sine_mode_field(m, 0.02, rng)
    v = gaussian_velocity(m, 0.05, rng)
    mat = dict(SVK_1E7, eta_d=1e3, lambda_d=1e3)
    return dict(name=f"box 20x4x2 m, {nx}x{ny}x{nz} hex x6 = {m.ne:,} T10, SVK+KV",
                mesh=m, q_n=q, v=v, material=mat, h=1e-3, field_info=info)


def workload_warm_start_svk():
    """Box 12 x 1.2 x 1.2 m, 120x12x12 hexes -> 103,680 T10, 150,625 nodes;
    SVK E=1e7, nu=0.3; gravity plus a seeded tip load U(0, 500) N in a random
    direction, redrawn every 100 steps."""
    rng = np.random.default_rng(1000 + 4)
    m = box_t10(120, 12, 12, 12.0, 1.2, 1.2)
    mat = dict(SVK_1E7, eta_d=0.0, lambda_d=0.0)
    f_ext = tip_load_schedule(m, 2000, 100, 500.0, rng)
    return dict(name="box 12x1.2x1.2 m, 120x12x12 hex x6 = 103,680 T10, SVK", mesh=m,
                q_n=m.X.copy(), v=np.zeros_like(m.X), material=mat, h=1e-3,
                f_ext=f_ext, rng=rng)


def workload_batched(nbodies=48, seed=1000 + 3, lo=1000, hi=60000):
    """48 independent bodies, element counts log-uniform in [lo, hi]; half
    boxes (aspect 1:1:1 .. 10:1:1), half cylinders; half SVK, half MR; +-2%
    nodal perturbation of each node's own spacing; one face clamped per body."""
    rng = np.random.default_rng(seed)
    meshes, mats, qs, vs = [], [], [], []
    for b in range(nbodies):
        target = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        if b % 2 == 0:
            aspect = rng.uniform(1.0, 10.0)
            n = max(1, int(round((target / (6.0 * aspect)) ** (1.0 / 3.0))))
            m = box_t10(max(1, int(round(aspect * n))), n, n,
                        0.1 * aspect * n, 0.1 * n, 0.1 * n)
        else:
            # cylinder: 6 * (2nr)^2 * nz elements with nz ~ 2*(2nr)
            nr = max(1, int(round((target / 48.0) ** (1.0 / 3.0))))
            nz = max(1, int(round(target / (24.0 * nr * nr))))
            m = cylinder_t10(nr, nz, 0.1 * nr, 0.1 * nz)
        q = uniform_perturbation(m, 0.02, rng, local=True)
        v = gaussian_velocity(m, 0.01, rng)
        meshes.append(m)
        qs.append(q)
        vs.append(v)
        mats.append(dict(SVK_1E7, eta_d=0.0, lambda_d=0.0) if b % 4 < 2
                    else dict(MR_C2, eta_d=0.0, lambda_d=0.0))
    mesh = merge_meshes(meshes)
    return dict(name=f"{nbodies} bodies, {mesh.ne:,} T10 total", mesh=mesh,
                q_n=np.concatenate(qs), v=np.concatenate(vs), materials=mats,
                mat_of_elem=mesh.body_of_elem.copy(), h=1e-3, meshes=meshes)


# ---------------------------------------------------------------------------
# ANCF meshes (the beam and shell scaling benchmarks, Sec. 5.2 and 5.3)
#
# Coefficient convention (shared interface, not arithmetic): physical node p
# owns the four coefficient vectors 4p + (0: position r, 1: r_x, 2: r_y,
# 3: r_z).  A beam element lists its two nodes' coefficients (8); a shell
# element its four corners' (16), corners in the order (-1,-1), (1,-1),
# (1,1), (-1,1) of its natural coordinates.  E0 holds the reference
# coefficients: node positions and the unit axis vectors as gradients.
# ---------------------------------------------------------------------------

ANCF_BEAM = "ancf3243"
ANCF_SHELL = "ancf3443"

# Material of the paper's element-type scaling benchmarks (SVK, E = 7e8 Pa,
# nu = 0.33, rho0 = 2700 kg/m^3).
SVK_7E8 = dict(kind="svk", E=7e8, nu=0.33, rho0=2700.0, eta_d=0.0, lambda_d=0.0)


@dataclass
class AncfMesh:
    kind: str                # ANCF_BEAM or ANCF_SHELL
    E0: np.ndarray           # (ncoef, 3) float64 reference coefficient vectors
    conn: np.ndarray         # (ne, nen) int32 coefficient indices
    dims: np.ndarray         # (ne, 3) element length, width, height
    fixed_nodes: np.ndarray  # (nfixed,) int32 clamped coefficients, sorted
    nphys: int               # physical nodes
    phys_x: np.ndarray       # (nphys, 3) physical node positions
    meta: dict = field(default_factory=dict)

    @property
    def nn(self):
        return self.E0.shape[0]

    @property
    def ne(self):
        return self.conn.shape[0]

    @property
    def X(self):
        return self.E0


def _ancf_coefficients(P):
    """Reference coefficients of physical nodes at P (np, 3): r = P, r_x, r_y,
    r_z = the global unit vectors."""
    E0 = np.zeros((4 * len(P), 3))
    E0[0::4] = P
    E0[1::4] = (1.0, 0.0, 0.0)
    E0[2::4] = (0.0, 1.0, 0.0)
    E0[3::4] = (0.0, 0.0, 1.0)
    return E0


def beam_ancf3243(ne, L=0.2, W=0.1, H=0.1):
    """A chain of ne beam elements along x (element e spans nodes e, e+1);
    node 0 clamped (its four coefficients)."""
    P = np.zeros((ne + 1, 3))
    P[:, 0] = L * np.arange(ne + 1)
    e = np.arange(ne)[:, None]
    conn = np.concatenate([4 * e + np.arange(4), 4 * (e + 1) + np.arange(4)], axis=1).astype(np.int32)
    dims = np.tile([L, W, H], (ne, 1)).astype(np.float64)
    return AncfMesh(ANCF_BEAM, _ancf_coefficients(P), conn, dims, np.arange(4, dtype=np.int32), ne + 1, P)


def shell_ancf3443(nx, ny, Lx=4.0, Ly=2.0, H=0.1):
    """An nx x ny grid of shell elements on [0, Lx] x [0, Ly] (node (i, j) has
    id i (ny + 1) + j); every node on the edge x = 0 clamped."""
    i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    P = np.stack([i.ravel() * (Lx / nx), j.ravel() * (Ly / ny), np.zeros(i.size)], axis=1)
    nid = lambda a, b: a * (ny + 1) + b
    ei, ej = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    ei, ej = ei.ravel(), ej.ravel()
    corners = np.stack([nid(ei, ej), nid(ei + 1, ej), nid(ei + 1, ej + 1), nid(ei, ej + 1)], axis=1)
    conn = (4 * corners[:, :, None] + np.arange(4)).reshape(-1, 16).astype(np.int32)
    dims = np.tile([Lx / nx, Ly / ny, H], (nx * ny, 1)).astype(np.float64)
    fixed = (4 * nid(0, np.arange(ny + 1))[:, None] + np.arange(4)).ravel().astype(np.int32)
    return AncfMesh(ANCF_SHELL, _ancf_coefficients(P), conn, dims, np.sort(fixed), P.shape[0], P)


def ancf_bend(mesh, kappa):
    """Coefficients of the reference body bent about the y axis with curvature
    kappa (x along the arc): r = (sin(kx)/k, y, (1 - cos(kx))/k), r_x and r_z
    rotated by the angle kx, r_y unchanged."""
    E = mesh.E0.copy()
    x = mesh.phys_x[:, 0]
    t = kappa * x
    E[0::4, 0] = np.sin(t) / kappa
    E[0::4, 2] = (1.0 - np.cos(t)) / kappa
    E[1::4] = np.stack([np.cos(t), np.zeros_like(t), np.sin(t)], axis=1)
    E[3::4] = np.stack([-np.sin(t), np.zeros_like(t), np.cos(t)], axis=1)
    return E


def ancf_perturbation(mesh, q, frac, rng):
    """q + U(-frac, frac) scaled per coefficient: positions by the element
    dimensions, gradients by 1 (dimensionless); clamped coefficients keep E0."""
    scale = np.ones_like(q)
    scale[0::4] = mesh.dims[0][None, :]
    d = rng.uniform(-1.0, 1.0, size=q.shape) * frac * scale
    out = q + d
    out[mesh.fixed_nodes] = mesh.E0[mesh.fixed_nodes]
    return out


def workload_ancf_beam(ne=10, seed=1000 + 6):
    """ANCF3243 beam (L = 0.2, W = H = 0.1 per element; SVK 7e8 / 0.33 / 2700),
    bent to a curvature of 0.5 / m and perturbed by 0.1%; v ~ N(0, 0.01)."""
    rng = np.random.default_rng(seed)
    m = beam_ancf3243(ne)
    q = ancf_perturbation(m, ancf_bend(m, 0.5), 0.001, rng)
    v = rng.normal(0.0, 0.01, size=q.shape)
    v[m.fixed_nodes] = 0.0
    return dict(name=f"ANCF3243 beam, {ne:,} elements", mesh=m, q_n=q, v=v, material=dict(SVK_7E8), h=1e-3)


def workload_ancf_shell(nx=4, ny=3, seed=1000 + 7):
    """ANCF3443 shell 4 x 2 x 0.1 m (SVK 7e8 / 0.33 / 2700) on an nx x ny grid,
    bent to a curvature of 0.25 / m about y and perturbed by 0.1%; v ~ N(0, 0.01)."""
    rng = np.random.default_rng(seed)
    m = shell_ancf3443(nx, ny)
    q = ancf_perturbation(m, ancf_bend(m, 0.25), 0.001, rng)
    v = rng.normal(0.0, 0.01, size=q.shape)
    v[m.fixed_nodes] = 0.0
    return dict(name=f"ANCF3443 shell, {nx}x{ny} = {nx * ny:,} elements", mesh=m, q_n=q, v=v,
                material=dict(SVK_7E8), h=5e-4)
