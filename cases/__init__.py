"""Seeded synthetic inputs for the GFM dynamic-pressure equation.

This module builds meshes, volume-fraction fields and predicted face fluxes
shaped like the paper's workloads (Sec. 4.1: 2D progressive-wave tank;
Sec. 4.2: 3D green-water box).  It holds none of the method's arithmetic:
no interface fraction, no face coefficient, no jump, no solver.  Both the CPU
oracle and the CUDA path read their inputs from here and from nowhere else.

Mesh convention (face addressing, Sec. 3, Fig. "polyhedral CV"): cells are
numbered 0..n-1; every internal face f has an owner o < neighbour nu, an area
vector S_f pointing from owner to neighbour, and a face centre.  Boundary
faces are walls and are not listed.  Geometry arrays are structure-of-arrays:
``Sf[k, f]`` is component k of S_f, ``C[k, i]`` component k of cell centre i.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Case",
    "structured_mesh",
    "graded_mesh",
    "quad_mesh",
    "wavy_mesh",
    "permute_mesh",
    "alpha_cut_2d",
    "alpha_subsampled_3d",
    "random_face_flux",
    "stokes2_eta",
    "make_case",
    "batch_shapes",
    "batch_cases",
    "column_case",
    "still_water_case",
    "box_case",
    "CONFIGS",
]

RHO_W = 1000.0
RHO_A = 1.0
G = (0.0, -9.81, 0.0)


@dataclass
class Case:
    """One GFM pressure problem: mesh + alpha + predicted flux + physics."""

    name: str
    n: int
    F: int
    owner: np.ndarray  # int32 [F]
    neighbour: np.ndarray  # int32 [F]
    Sf: np.ndarray  # float64 [3, F]
    C: np.ndarray  # float64 [3, n]
    V: np.ndarray  # float64 [n]
    xf: np.ndarray  # float64 [3, F] face centres
    alpha: np.ndarray  # float64 [n]
    phi: np.ndarray  # float64 [F] predicted face flux
    rho_w: float = RHO_W
    rho_a: float = RHO_A
    g: tuple = G
    ref_cell: int = 0
    ref_value: float = 0.0
    rtol: float = 1e-12
    mode: str = "fp64"
    dims: tuple = ()
    meta: dict = field(default_factory=dict)
    fv_ptr: np.ndarray | None = None  # int32 [F+1] face polygons: vertices of face f are
    fv_xyz: np.ndarray | None = None  # float64 [3, nv] columns fv_ptr[f]..fv_ptr[f+1]-1, in order round it

    @property
    def faces_per_cell(self) -> float:
        return self.F / self.n


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def structured_mesh(nx: int, ny: int, nz: int, lx: float, ly: float, lz: float,
                    origin=(0.0, 0.0, 0.0)) -> dict:
    """Uniform hex mesh in face-addressed form.

    Cell (i, j, k) has index i + nx*(j + ny*k).  Internal faces are sorted by
    (owner, neighbour), the upper-triangular order of a face-addressed mesh.
    With nz == 1 the mesh is 2D: front/back faces are empty and not listed.
    """
    dx, dy, dz = lx / nx, ly / ny, lz / nz
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    i = idx % nx
    j = (idx // nx) % ny
    k = idx // (nx * ny)
    C = np.empty((3, n))
    C[0] = origin[0] + (i + 0.5) * dx
    C[1] = origin[1] + (j + 0.5) * dy
    C[2] = origin[2] + (k + 0.5) * dz
    V = np.full(n, dx * dy * dz)

    own, nb, S, XF = [], [], [], []
    for axis, step, ok, area in (
        (0, 1, i < nx - 1, dy * dz),
        (1, nx, j < ny - 1, dx * dz),
        (2, nx * ny, k < nz - 1, dx * dy),
    ):
        o = idx[ok]
        if o.size == 0:
            continue
        own.append(o)
        nb.append(o + step)
        s = np.zeros((3, o.size))
        s[axis] = area
        S.append(s)
        xf = C[:, o].copy()
        xf[axis] += 0.5 * (dx, dy, dz)[axis]
        XF.append(xf)
    owner = np.concatenate(own)
    neighbour = np.concatenate(nb)
    Sf = np.concatenate(S, axis=1)
    xfc = np.concatenate(XF, axis=1)
    order = np.lexsort((neighbour, owner))
    return dict(
        n=n, F=owner.size,
        owner=owner[order].astype(np.int32), neighbour=neighbour[order].astype(np.int32),
        Sf=np.ascontiguousarray(Sf[:, order]), C=C, V=V, xf=np.ascontiguousarray(xfc[:, order]),
        dims=(nx, ny, nz), spacing=(dx, dy, dz), origin=tuple(origin),
    )


def graded_mesh(xn, yn, zn) -> dict:
    """Tensor-product hex mesh from node coordinates (cells of uneven size),
    in the same face-addressed form and cell numbering as structured_mesh.
    Face centres lie on the line between the two cell centres, but not
    half-way between them."""
    xn, yn, zn = (np.asarray(v, dtype=np.float64) for v in (xn, yn, zn))
    nx, ny, nz = xn.size - 1, yn.size - 1, zn.size - 1
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    i = idx % nx
    j = (idx // nx) % ny
    k = idx // (nx * ny)
    dxs, dys, dzs = np.diff(xn), np.diff(yn), np.diff(zn)
    C = np.empty((3, n))
    C[0] = 0.5 * (xn[i] + xn[i + 1])
    C[1] = 0.5 * (yn[j] + yn[j + 1])
    C[2] = 0.5 * (zn[k] + zn[k + 1])
    V = dxs[i] * dys[j] * dzs[k]
    own, nb, S, XF, PV = [], [], [], [], []
    for axis, step, ok in ((0, 1, i < nx - 1), (1, nx, j < ny - 1), (2, nx * ny, k < nz - 1)):
        o = idx[ok]
        if o.size == 0:
            continue
        io, jo, ko = i[ok], j[ok], k[ok]
        s = np.zeros((3, o.size))
        xf = C[:, o].copy()
        # the face's four corners, in order round it
        lo = np.stack([xn[io], yn[jo], zn[ko]])
        hi = np.stack([xn[io + 1], yn[jo + 1], zn[ko + 1]])
        a, b = [q for q in range(3) if q != axis]
        corners = []
        for ca, cb in ((0, 0), (1, 0), (1, 1), (0, 1)):
            v = np.empty((3, o.size))
            v[axis] = hi[axis]
            v[a] = hi[a] if ca else lo[a]
            v[b] = hi[b] if cb else lo[b]
            corners.append(v)
        PV.append(np.stack(corners, axis=1))  # [3, 4, m]
        if axis == 0:
            s[0] = dys[jo] * dzs[ko]
            xf[0] = xn[io + 1]
        elif axis == 1:
            s[1] = dxs[io] * dzs[ko]
            xf[1] = yn[jo + 1]
        else:
            s[2] = dxs[io] * dys[jo]
            xf[2] = zn[ko + 1]
        own.append(o)
        nb.append(o + step)
        S.append(s)
        XF.append(xf)
    owner = np.concatenate(own)
    neighbour = np.concatenate(nb)
    Sf = np.concatenate(S, axis=1)
    xfc = np.concatenate(XF, axis=1)
    pv = np.concatenate(PV, axis=2)
    order = np.lexsort((neighbour, owner))
    F = owner.size
    return dict(
        n=n, F=F,
        owner=owner[order].astype(np.int32), neighbour=neighbour[order].astype(np.int32),
        Sf=np.ascontiguousarray(Sf[:, order]), C=C, V=V, xf=np.ascontiguousarray(xfc[:, order]),
        dims=(nx, ny, nz), spacing=(float(dxs.min()), float(dys.min()), float(dzs.min())),
        origin=(float(xn[0]), float(yn[0]), float(zn[0])),
        fv_ptr=np.arange(0, 4 * F + 1, 4, dtype=np.int32),
        fv_xyz=np.ascontiguousarray(pv[:, :, order].transpose(0, 2, 1).reshape(3, 4 * F)),
    )


def quad_mesh(X, Y, dz: float) -> dict:
    """2D mesh of convex quadrilaterals from node coordinates X, Y of shape
    (ny + 1, nx + 1), extruded one cell deep (dz), in the face-addressed form
    and cell numbering of structured_mesh.  Cell centres are polygon
    centroids, face centres edge midpoints, area vectors the edge normals
    times dz pointing to the higher-numbered cell.  Cells need not be
    orthogonal: d_f and S_f are generally not parallel."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    ny, nx = X.shape[0] - 1, X.shape[1] - 1
    n = nx * ny
    # vertices counter-clockwise: (i,j), (i+1,j), (i+1,j+1), (i,j+1)
    vx = np.stack([X[:-1, :-1], X[:-1, 1:], X[1:, 1:], X[1:, :-1]], axis=-1).reshape(n, 4)
    vy = np.stack([Y[:-1, :-1], Y[:-1, 1:], Y[1:, 1:], Y[1:, :-1]], axis=-1).reshape(n, 4)
    x1, y1 = np.roll(vx, -1, axis=1), np.roll(vy, -1, axis=1)
    cr = vx * y1 - x1 * vy
    area = 0.5 * cr.sum(axis=1)
    cx = ((vx + x1) * cr).sum(axis=1) / (6.0 * area)
    cy = ((vy + y1) * cr).sum(axis=1) / (6.0 * area)
    if np.any(area <= 0):
        raise ValueError("quad_mesh: cells must be convex and counter-clockwise")
    C = np.stack([cx, cy, np.full(n, 0.5 * dz)])
    V = area * dz
    idx = np.arange(n).reshape(ny, nx)
    own, nb, S, XF, PV = [], [], [], [], []

    def edge_polygon(ax, ay, bx, by):  # the edge extruded over [0, dz]: 4 corners in order
        z0, z1 = np.zeros(ax.size), np.full(ax.size, dz)
        return np.stack([np.stack([ax, ay, z0]), np.stack([bx, by, z0]), np.stack([bx, by, z1]),
                         np.stack([ax, ay, z1])], axis=1)

    # faces between (i, j) and (i+1, j): edge from node (j, i+1) to (j+1, i+1)
    o = idx[:, :-1].reshape(-1)
    ax, ay = X[:-1, 1:-1].reshape(-1), Y[:-1, 1:-1].reshape(-1)
    bx, by = X[1:, 1:-1].reshape(-1), Y[1:, 1:-1].reshape(-1)
    own.append(o)
    nb.append(o + 1)
    S.append(np.stack([(by - ay) * dz, -(bx - ax) * dz, np.zeros(o.size)]))
    XF.append(np.stack([0.5 * (ax + bx), 0.5 * (ay + by), np.full(o.size, 0.5 * dz)]))
    PV.append(edge_polygon(ax, ay, bx, by))
    # faces between (i, j) and (i, j+1): edge from node (j+1, i) to (j+1, i+1)
    o = idx[:-1, :].reshape(-1)
    ax, ay = X[1:-1, :-1].reshape(-1), Y[1:-1, :-1].reshape(-1)
    bx, by = X[1:-1, 1:].reshape(-1), Y[1:-1, 1:].reshape(-1)
    own.append(o)
    nb.append(o + nx)
    S.append(np.stack([-(by - ay) * dz, (bx - ax) * dz, np.zeros(o.size)]))
    XF.append(np.stack([0.5 * (ax + bx), 0.5 * (ay + by), np.full(o.size, 0.5 * dz)]))
    PV.append(edge_polygon(ax, ay, bx, by))
    owner = np.concatenate(own)
    neighbour = np.concatenate(nb)
    Sf = np.concatenate(S, axis=1)
    xfc = np.concatenate(XF, axis=1)
    pv = np.concatenate(PV, axis=2)
    order = np.lexsort((neighbour, owner))
    F = owner.size
    return dict(
        n=n, F=F,
        owner=owner[order].astype(np.int32), neighbour=neighbour[order].astype(np.int32),
        Sf=np.ascontiguousarray(Sf[:, order]), C=C, V=V, xf=np.ascontiguousarray(xfc[:, order]),
        dims=(nx, ny, 1), spacing=(float(np.diff(X, axis=1).min()), float(np.diff(Y, axis=0).min()), dz),
        origin=(float(X.min()), float(Y.min()), 0.0),
        fv_ptr=np.arange(0, 4 * F + 1, 4, dtype=np.int32),
        fv_xyz=np.ascontiguousarray(pv[:, :, order].transpose(0, 2, 1).reshape(3, 4 * F)),
    )


def wavy_mesh(nx: int, ny: int, lx: float = 2.0, ly: float = 1.0, eps: float = 0.04) -> dict:
    """A smoothly distorted, non-orthogonal quad mesh of the rectangle
    [0, lx] x [0, ly] with straight walls: nodes displaced by
    eps lx sin(pi x/lx) sin(2 pi y/ly) in x and eps ly sin(2 pi x/lx) sin(pi y/ly)
    in y, an O(1) distortion that does not fade under refinement."""
    xs, ys = np.linspace(0.0, lx, nx + 1), np.linspace(0.0, ly, ny + 1)
    x, y = np.meshgrid(xs, ys)
    X = x + eps * lx * np.sin(math.pi * x / lx) * np.sin(2.0 * math.pi * y / ly)
    Y = y + eps * ly * np.sin(2.0 * math.pi * x / lx) * np.sin(math.pi * y / ly)
    return quad_mesh(X, Y, lx / nx)


def permute_mesh(mesh: dict, perm: np.ndarray, face_fields=()) -> dict:
    """Relabel cells by ``new = perm[old]`` and re-sort faces.

    A face whose relabelled owner exceeds its neighbour is flipped: owner and
    neighbour swap, and S_f (and every oriented face field given in
    ``face_fields``) changes sign.  Faces are then sorted by (owner, neighbour).
    Returns a new mesh dict plus the re-sorted face fields under ``"fields"``.
    """
    n = mesh["n"]
    perm = np.asarray(perm, dtype=np.int64)
    o = perm[mesh["owner"]]
    nu = perm[mesh["neighbour"]]
    flip = o > nu
    sign = np.where(flip, -1.0, 1.0)
    o2 = np.where(flip, nu, o)
    n2 = np.where(flip, o, nu)
    order = np.lexsort((n2, o2))
    C = np.empty_like(mesh["C"])
    C[:, perm] = mesh["C"]
    V = np.empty_like(mesh["V"])
    V[perm] = mesh["V"]
    out = dict(mesh)
    out.update(
        owner=o2[order].astype(np.int32), neighbour=n2[order].astype(np.int32),
        Sf=np.ascontiguousarray((mesh["Sf"] * sign)[:, order]), C=C, V=V,
        xf=np.ascontiguousarray(mesh["xf"][:, order]), perm=perm,
    )
    out["fields"] = [np.ascontiguousarray((np.asarray(ff) * sign)[order]) for ff in face_fields]
    if mesh.get("fv_xyz") is not None:  # equal-size polygons: reorder them with the faces
        ptr = np.asarray(mesh["fv_ptr"])
        nvf = np.diff(ptr)
        if np.all(nvf == nvf[0]):
            k = int(nvf[0])
            out["fv_xyz"] = np.ascontiguousarray(
                mesh["fv_xyz"].reshape(3, -1, k)[:, order, :].reshape(3, -1))
            out["fv_ptr"] = ptr
        else:
            out.pop("fv_xyz")
            out.pop("fv_ptr")
    return out


# ----------------------------------------------------------------------------
# volume fraction (Eq. 10: alpha = V+/V)
# ----------------------------------------------------------------------------

_GL_X, _GL_W = np.polynomial.legendre.leggauss(10)


def _crossings(eta, x0: float, x1: float, level: float, nsample: int = 33) -> list:
    """Points in (x0, x1) where eta(x) == level, by sampling + bisection."""
    xs = np.linspace(x0, x1, nsample)
    fs = eta(xs) - level
    out = []
    for a, b, fa, fb in zip(xs[:-1], xs[1:], fs[:-1], fs[1:]):
        if fa == 0.0:
            out.append(a)
            continue
        if fa * fb < 0.0:
            lo, hi, flo = a, b, fa
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                fm = eta(np.array([mid]))[0] - level
                if fm == 0.0:
                    lo = hi = mid
                    break
                if (fm < 0.0) == (flo < 0.0):
                    lo, flo = mid, fm
                else:
                    hi = mid
            out.append(0.5 * (lo + hi))
    return out


def alpha_cut_2d(mesh: dict, eta) -> np.ndarray:
    """Exact cut fraction of every 2D cell under the surface y = eta(x).

    alpha_ij = (1/(dx dy)) * integral over the cell's x-span of
    clamp(eta(x) - y_j, 0, dy) dx, evaluated piecewise between the points where
    eta crosses the cell's bottom and top edges with 10-point Gauss-Legendre
    (eta is smooth between those points, so this is accurate to rounding).
    """
    nx, ny, nz = mesh["dims"]
    assert nz == 1
    dx, dy, _ = mesh["spacing"]
    x0g, y0g, _ = mesh["origin"]
    alpha = np.zeros((ny, nx))
    for i in range(nx):
        xa, xb = x0g + i * dx, x0g + (i + 1) * dx
        xs = np.linspace(xa, xb, 65)
        es = eta(xs)
        lo, hi = es.min(), es.max()
        jlo = max(int(math.floor((lo - y0g) / dy)) - 1, 0)
        jhi = min(int(math.floor((hi - y0g) / dy)) + 1, ny - 1)
        alpha[:jlo, i] = 1.0
        for j in range(jlo, jhi + 1):
            yb = y0g + j * dy
            yt = yb + dy
            if lo >= yt:
                alpha[j, i] = 1.0
                continue
            if hi <= yb:
                alpha[j, i] = 0.0
                continue
            pts = sorted({xa, xb, *_crossings(eta, xa, xb, yb), *_crossings(eta, xa, xb, yt)})
            tot = 0.0
            for a, b in zip(pts[:-1], pts[1:]):
                if b <= a:
                    continue
                xq = 0.5 * (a + b) + 0.5 * (b - a) * _GL_X
                hq = np.clip(eta(xq) - yb, 0.0, dy)
                tot += 0.5 * (b - a) * float(np.dot(_GL_W, hq))
            alpha[j, i] = tot / (dx * dy)
        # rows above jhi stay 0
    return alpha.reshape(-1)


def alpha_subsampled_3d(mesh: dict, inside, m: int = 5, margin=None) -> np.ndarray:
    """alpha = fraction of the m^3 sub-sample points of each cell inside water.

    ``inside(x, y, z)`` returns a bool array.  ``margin(x, y, z)`` (optional)
    returns, at cell centres, True where the cell is certainly pure (all
    sub-samples agree with the centre); only the remaining cells are
    sub-sampled.
    """
    dx, dy, dz = mesh["spacing"]
    C = mesh["C"]
    n = mesh["n"]
    centre_in = inside(C[0], C[1], C[2])
    alpha = centre_in.astype(np.float64)
    if margin is None:
        todo = np.arange(n)
    else:
        todo = np.nonzero(~margin(C[0], C[1], C[2]))[0]
    off = (np.arange(m) + 0.5) / m - 0.5
    ox, oy, oz = np.meshgrid(off * dx, off * dy, off * dz, indexing="ij")
    ox, oy, oz = ox.reshape(-1), oy.reshape(-1), oz.reshape(-1)
    chunk = 65536
    for s in range(0, todo.size, chunk):
        t = todo[s:s + chunk]
        X = C[0, t][:, None] + ox[None, :]
        Y = C[1, t][:, None] + oy[None, :]
        Z = C[2, t][:, None] + oz[None, :]
        alpha[t] = inside(X, Y, Z).sum(axis=1) / float(m ** 3)
    return alpha


# ----------------------------------------------------------------------------
# predicted face flux
# ----------------------------------------------------------------------------

def random_face_flux(mesh: dict, rng: np.random.Generator, nmodes: int = 8,
                     amp: float = 0.1, two_d: bool | None = None) -> np.ndarray:
    """phi*_f = S_f . u(x_f), u a seeded sum of smooth trigonometric modes.

    u(x) = sum_m a_m trig_m(k_m . x + theta_m) with a_m ~ U(-amp, amp)^3,
    |k_m| <= 2*pi/(4*delta) (delta = smallest cell size), trig_m alternating
    sin/cos.  The field is generally not divergence free, so the pressure
    equation has a non-trivial source.
    """
    dx, dy, dz = mesh["spacing"]
    if two_d is None:
        two_d = mesh["dims"][2] == 1
    delta = min(dx, dy) if two_d else min(dx, dy, dz)
    kmax = 2.0 * math.pi / (4.0 * delta)
    xf = mesh["xf"]
    u = np.zeros_like(xf)
    for mi in range(nmodes):
        a = rng.uniform(-amp, amp, size=3)
        d = rng.normal(size=3)
        if two_d:
            a[2] = 0.0
            d[2] = 0.0
        d /= max(np.linalg.norm(d), 1e-300)
        kvec = d * rng.uniform(0.0, kmax)
        theta = rng.uniform(0.0, 2.0 * math.pi)
        arg = kvec[0] * xf[0] + kvec[1] * xf[1] + kvec[2] * xf[2] + theta
        t = np.sin(arg) if mi % 2 == 0 else np.cos(arg)
        u += a[:, None] * t[None, :]
    return np.einsum("kf,kf->f", mesh["Sf"], u)


# ----------------------------------------------------------------------------
# wave shapes (Sec. 4.1 progressive wave; Sec. 4.2 green water)
# ----------------------------------------------------------------------------

def stokes2_eta(depth: float, k: float, a: float, x0: float = 0.0):
    """Second-order Stokes surface elevation over finite depth."""
    kd = k * depth
    a2 = (k * a * a / 4.0) * math.cosh(kd) * (2.0 + math.cosh(2.0 * kd)) / math.sinh(kd) ** 3

    def eta(x):
        th = k * (np.asarray(x) - x0)
        return depth + a * np.cos(th) + a2 * np.cos(2.0 * th)

    return eta


def _case_from(mesh, alpha, phi, name, ref_ijk, **kw) -> Case:
    nx, ny, nz = mesh["dims"]
    i, j, k = ref_ijk
    ref = i + nx * (j + ny * k)
    if "perm" in mesh:
        ref = int(mesh["perm"][ref])
    return Case(name=name, n=mesh["n"], F=mesh["F"], owner=mesh["owner"], neighbour=mesh["neighbour"],
                Sf=mesh["Sf"], C=mesh["C"], V=mesh["V"], xf=mesh["xf"], alpha=np.ascontiguousarray(alpha),
                phi=np.ascontiguousarray(phi), ref_cell=int(ref), dims=mesh["dims"],
                fv_ptr=mesh.get("fv_ptr"), fv_xyz=mesh.get("fv_xyz"), **kw)


def _wave_tank(nx, ny, lx, ly, depth, ka, nwaves, seed, name, rtol, mode, thickness=None) -> Case:
    dz = lx / nx if thickness is None else thickness
    mesh = structured_mesh(nx, ny, 1, lx, ly, dz)
    k = 2.0 * math.pi * nwaves / lx
    eta = stokes2_eta(depth, k, ka / k)
    alpha = alpha_cut_2d(mesh, eta)
    rng = np.random.default_rng(seed)
    phi = random_face_flux(mesh, rng)
    return _case_from(mesh, alpha, phi, name, (0, ny - 1, 0), rtol=rtol, mode=mode,
                      meta=dict(ka=ka, nwaves=nwaves, depth=depth, seed=seed))


def make_case(config: int, seed: int | None = None) -> Case:
    """The five workload recipes (seed = 1000 + config unless given)."""
    if seed is None:
        seed = 1000 + config
    if config == 1:
        mesh = structured_mesh(64, 32, 1, 2.0, 1.0, 2.0 / 64)
        eta = lambda x: 0.5 + 0.02 * np.cos(2.0 * math.pi * np.asarray(x))  # noqa: E731
        alpha = alpha_cut_2d(mesh, eta)
        phi = random_face_flux(mesh, np.random.default_rng(seed))
        return _case_from(mesh, alpha, phi, "tank2d_64x32", (0, 31, 0), rtol=1e-12, mode="fp64",
                          meta=dict(seed=seed))
    if config in (2, 5):
        c = _wave_tank(1024, 512, 16.0, 4.0, 2.0, 0.1, 4, seed, "tank2d_1024x512", 1e-10, "mixed")
        if config == 5:
            c.name = "adjoint_tank2d_1024x512"
        return c
    if config == 3:
        return green_water_box(256, 128, 128, seed)
    if config == 4:
        raise ValueError("config 4 is a batch: use batch_cases()")
    raise ValueError(f"unknown config {config}")


def green_water_box(nx: int, ny: int, nz: int, seed: int, permute: bool = True) -> Case:
    """3D box (x, y up, z) of 4 x 2 x 2 m: a bumpy layer, a dam-break column
    and floating spheres give a folded, multiply connected interface."""
    lx, ly, lz = 4.0, 2.0, 2.0
    mesh = structured_mesh(nx, ny, nz, lx, ly, lz)
    rng = np.random.default_rng(seed)
    nb = 8
    A = rng.uniform(0.05, 0.3, nb)
    sig = rng.uniform(0.1, 0.4, nb)
    cx = rng.uniform(0.0, lx, nb)
    cz = rng.uniform(0.0, lz, nb)
    ns = 6
    sr = rng.uniform(0.05, 0.2, ns)
    sc = np.stack([rng.uniform(0.3, lx - 0.3, ns), rng.uniform(1.2, 1.75, ns), rng.uniform(0.3, lz - 0.3, ns)])

    def surface(x, z):
        s = 0.6
        for b in range(nb):
            s = s + A[b] * np.exp(-((x - cx[b]) ** 2 + (z - cz[b]) ** 2) / (2.0 * sig[b] ** 2))
        return s

    def inside(x, y, z):
        w = y < surface(x, z)
        w |= (x < 1.0) & (y < 1.4)
        for s in range(ns):
            w |= (x - sc[0, s]) ** 2 + (y - sc[1, s]) ** 2 + (z - sc[2, s]) ** 2 < sr[s] ** 2
        return w

    dx, dy, dz = mesh["spacing"]
    h = max(dx, dy, dz)
    # |grad surface| <= sum A/sigma * e^{-1/2}; margin covers the half-diagonal
    slope = float(np.sum(A / sig)) * math.exp(-0.5)
    m_layer = h * math.sqrt(3.0) * (1.0 + slope)

    def pure(x, y, z):
        ok = np.abs(y - surface(x, z)) > m_layer
        ok &= (np.abs(x - 1.0) > h) | (y > 1.4 + h)
        ok &= (np.abs(y - 1.4) > h) | (x > 1.0 + h)
        for s in range(ns):
            dist = np.sqrt((x - sc[0, s]) ** 2 + (y - sc[1, s]) ** 2 + (z - sc[2, s]) ** 2)
            ok &= np.abs(dist - sr[s]) > h * math.sqrt(3.0)
        return ok

    alpha = alpha_subsampled_3d(mesh, inside, 5, pure)
    phi = random_face_flux(mesh, rng, two_d=False)
    if permute:
        perm = rng.permutation(mesh["n"])
        pm = permute_mesh(mesh, perm, face_fields=(phi,))
        alpha_p = np.empty_like(alpha)
        alpha_p[perm] = alpha
        phi = pm.pop("fields")[0]
        mesh, alpha = pm, alpha_p
    return _case_from(mesh, alpha, phi, f"box3d_{nx}x{ny}x{nz}", (0, ny - 1, 0), rtol=1e-8, mode="mixed",
                      meta=dict(seed=seed, permuted=permute))


def batch_shapes(ntanks: int = 64, seed0: int = 4000, nx_range=(128, 1024), ny_range=(64, 256)) -> list:
    """(nx, ny, ka, wavelengths) of each tank of a batch (tank t uses seed
    seed0 + t), without building the tanks."""
    out = []
    for t in range(ntanks):
        rng = np.random.default_rng(seed0 + t)
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        ka = float(rng.uniform(0.02, 0.15))
        nw = int(rng.integers(1, 7))
        out.append((nx, ny, ka, nw))
    return out


def batch_cases(ntanks: int = 64, seed0: int = 4000, nx_range=(128, 1024), ny_range=(64, 256),
                only=None) -> list:
    """Batch of 2D wave tanks of uneven size (tank t uses seed seed0 + t).
    ``only`` (optional): the tank indices to build, in the order given."""
    shapes = batch_shapes(ntanks, seed0, nx_range, ny_range)
    out = []
    for t in (range(ntanks) if only is None else only):
        nx, ny, ka, nw = shapes[t]
        out.append(_wave_tank(nx, ny, 16.0, 4.0, 2.0, ka, nw, seed0 + 10_000 + t, f"tank{t}_{nx}x{ny}",
                              1e-8, "mixed"))
    return out


CONFIGS = {
    1: "tank2d_64x32: plain FP64, rtol 1e-12",
    2: "tank2d_1024x512: FP64 vs mixed, rtol 1e-10",
    3: "box3d_256x128x128 permuted: mixed, rtol 1e-8",
    4: "64 tanks 128..1024 x 64..256: batched mixed, rtol 1e-8",
    5: "adjoint on tank2d_1024x512",
}


# ----------------------------------------------------------------------------
# small cases for tests
# ----------------------------------------------------------------------------

def column_case(ny: int = 8, ly: float = 1.0, level: float = 0.43, seed: int = 7, flux: bool = True,
                width: float = 0.1) -> Case:
    """1 x ny x 1 water column, flat surface at y = level."""
    mesh = structured_mesh(1, ny, 1, width, ly, width)
    alpha = alpha_cut_2d(mesh, lambda x: np.full_like(np.asarray(x, dtype=float), level))
    rng = np.random.default_rng(seed)
    phi = rng.uniform(-1e-3, 1e-3, mesh["F"]) if flux else np.zeros(mesh["F"])
    return _case_from(mesh, alpha, phi, f"column_{ny}", (0, ny - 1, 0), rtol=1e-13)


def still_water_case(nx: int = 16, ny: int = 8, lx: float = 2.0, ly: float = 1.0, level: float = 0.4375 + 0.01,
                     nz: int = 1, lz: float | None = None) -> Case:
    """Flat free surface, no predicted flux: the balanced-force test case."""
    lz = lx / nx if lz is None else lz
    mesh = structured_mesh(nx, ny, nz, lx, ly, lz)
    if nz == 1:
        alpha = alpha_cut_2d(mesh, lambda x: np.full_like(np.asarray(x, dtype=float), level))
    else:
        dy = ly / ny
        alpha = np.clip((level - (mesh["C"][1] - 0.5 * dy)) / dy, 0.0, 1.0)
    return _case_from(mesh, alpha, np.zeros(mesh["F"]), f"still_{nx}x{ny}x{nz}", (0, ny - 1, 0), rtol=1e-13)


def box_case(nx: int, ny: int, nz: int = 1, seed: int = 11, ka: float = 0.1, nwaves: int = 1,
             lx: float = 2.0, ly: float = 1.0, permute: bool = False, alpha_noise: float = 0.0) -> Case:
    """Small wave tank (2D, or 3D extruded in z) with optional cell permutation."""
    lz = lx / nx if nz == 1 else lx * nz / nx
    mesh = structured_mesh(nx, ny, nz, lx, ly, lz)
    k = 2.0 * math.pi * nwaves / lx
    depth = 0.5 * ly
    eta = stokes2_eta(depth, k, ka / k)
    rng = np.random.default_rng(seed)
    if nz == 1:
        alpha = alpha_cut_2d(mesh, eta)
    else:
        base = structured_mesh(nx, ny, 1, lx, ly, lx / nx)
        a2 = alpha_cut_2d(base, eta).reshape(ny, nx)
        alpha = np.broadcast_to(a2[None], (nz, ny, nx)).reshape(-1).copy()
    if alpha_noise > 0.0:
        mix = (alpha > 0.0) & (alpha < 1.0)
        alpha[mix] = np.clip(alpha[mix] + rng.uniform(-alpha_noise, alpha_noise, mix.sum()), 0.0, 1.0)
    phi = random_face_flux(mesh, rng)
    if permute:
        perm = rng.permutation(mesh["n"])
        pm = permute_mesh(mesh, perm, face_fields=(phi,))
        alpha_p = np.empty_like(alpha)
        alpha_p[perm] = alpha
        phi = pm.pop("fields")[0]
        mesh, alpha = pm, alpha_p
    return _case_from(mesh, alpha, phi, f"box_{nx}x{ny}x{nz}", (0, ny - 1, 0), rtol=1e-13)
