"""Seeded synthetic inputs: hexahedral meshes, materials and boundary tags.

This module holds no arithmetic of the DPG method.  It produces the plain
arrays that both the CUDA path (through ``dpg_setup_mesh``) and the test
oracle consume, shaped like the paper's cases:

* rectangular waveguides with PEC walls, a TE_mn port at x3 = 0 and an
  impedance outlet at the far end (Sec. 4.1, Table of App. C.1);
* box cavities with PEC walls and a tangential Dirichlet excitation
  n x E = (sin(pi x2), 0, 0) on the top face (the Fichera excitation of
  Sec. 4.2), optionally with jittered interior vertices and per-element
  random permittivity.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014), a counter-based
generator: value k of stream s is splitmix64(seed + s * 2^32 + k), so every
draw can be recomputed independently.

Mesh conventions: vertex v = i + 2 j + 4 k of an element sits at reference
corner (i, j, k); every element's local axes point along the global +x1, +x2,
+x3 directions.  Face f = 2 d + s is the face xi_d = s.  Boundary tags:
face_bc 0 = none, 1 = Dirichlet (group in face_grp indexes ``dirichlet``),
2 = Robin (group indexes ``robin``).
"""
from dataclasses import dataclass, field

import numpy as np

BC_NONE, BC_DIRICHLET, BC_ROBIN = 0, 1, 2
DIRICHLET_ZERO, DIRICHLET_SIN_PI_X2, DIRICHLET_TE = 0, 1, 2
C0 = 299792458.0

_MASK = (1 << 64) - 1


def splitmix64(x):
    """splitmix64 finaliser applied to uint64 array x (wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over='ignore'):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, stream, count):
    """count doubles in [0,1) from the counter-based stream (seed, stream)."""
    ctr = np.uint64(seed) + np.uint64(stream) * np.uint64(1 << 32) + np.arange(count, dtype=np.uint64)
    return (splitmix64(ctr) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


@dataclass
class Mesh:
    vert: np.ndarray            # (nv, 3) float64
    elem: np.ndarray            # (ne, 8) int32
    p: np.ndarray               # (ne,) int8
    eps: np.ndarray             # (ne,) complex128, dimensionless, loss => Im > 0
    mu: np.ndarray              # (ne,) complex128
    face_bc: np.ndarray         # (ne, 6) int8
    face_grp: np.ndarray        # (ne, 6) int16
    omega: float                # dimensionless angular frequency 2 pi f L / c0, L = 1 m
    robin: list = field(default_factory=list)      # [{'zinv': complex, 'port': None | (a, b, m, n, eps, mu)}]
    dirichlet: list = field(default_factory=list)  # [{'kind': int, 'port': None | (a, b, m, n, eps, mu)}]
    name: str = ""
    grid: tuple = None          # (nx, ny, nz) for structured meshes

    @property
    def n_elem(self):
        return self.elem.shape[0]


def omega_from_hz(f_hz, L=1.0):
    return 2.0 * np.pi * f_hz * L / C0


def te_zinv(omega, a, b, m, n, eps=1.0, mu=1.0):
    """Impedance parameter k3 / (omega mu) of a TE_mn guide (the paper's port/outlet value)."""
    kc2 = (m * np.pi / a) ** 2 + (n * np.pi / b) ** 2
    k3 = np.sqrt(complex(omega * omega * eps * mu - kc2))
    return k3 / (omega * mu)


def structured_hex(lx, ly, lz, nx, ny, nz, origin=(0.0, 0.0, 0.0)):
    """Uniform hex grid: vertices (nv,3), elements (ne,8), element grid coords (ne,3)."""
    xs = origin[0] + np.linspace(0.0, lx, nx + 1)
    ys = origin[1] + np.linspace(0.0, ly, ny + 1)
    zs = origin[2] + np.linspace(0.0, lz, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing='ij')
    vert = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    vid = lambda i, j, k: (k * (ny + 1) + j) * (nx + 1) + i
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing='ij')
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    elem = np.zeros((i.size, 8), dtype=np.int32)
    for v in range(8):
        di, dj, dk = v & 1, (v >> 1) & 1, (v >> 2) & 1
        elem[:, v] = vid(i + di, j + dj, k + dk)
    return vert, elem, np.stack([i, j, k], axis=1)


def box_boundary_tags(ijk, nx, ny, nz, spec):
    """face_bc / face_grp from a per-side spec {'x0': (bc, grp), ...}; sides not given stay 0."""
    ne = ijk.shape[0]
    bc = np.zeros((ne, 6), dtype=np.int8)
    grp = np.zeros((ne, 6), dtype=np.int16)
    n = (nx, ny, nz)
    for d, axis in enumerate('xyz'):
        for s in (0, 1):
            key = f'{axis}{s}'
            if key not in spec:
                continue
            on = ijk[:, d] == (0 if s == 0 else n[d] - 1)
            bc[on, 2 * d + s] = spec[key][0]
            grp[on, 2 * d + s] = spec[key][1]
    return bc, grp


def waveguide(a, b, length, nx, ny, nz, f_hz, p, name="waveguide", m=1, n=0):
    """PEC-walled guide [0,a]x[0,b]x[0,length], TE_mn port at x3=0, impedance end at x3=length."""
    omega = omega_from_hz(f_hz)
    vert, elem, ijk = structured_hex(a, b, length, nx, ny, nz)
    zinv = te_zinv(omega, a, b, m, n)
    spec = {'x0': (BC_DIRICHLET, 0), 'x1': (BC_DIRICHLET, 0), 'y0': (BC_DIRICHLET, 0),
            'y1': (BC_DIRICHLET, 0), 'z0': (BC_ROBIN, 0), 'z1': (BC_ROBIN, 1)}
    bc, grp = box_boundary_tags(ijk, nx, ny, nz, spec)
    ne = elem.shape[0]
    return Mesh(vert=vert, elem=elem, p=np.full(ne, p, dtype=np.int8),
                eps=np.ones(ne, dtype=complex), mu=np.ones(ne, dtype=complex),
                face_bc=bc, face_grp=grp, omega=omega,
                robin=[{'zinv': zinv, 'port': (a, b, m, n, 1.0, 1.0)}, {'zinv': zinv, 'port': None}],
                dirichlet=[{'kind': DIRICHLET_ZERO, 'port': None}], name=name, grid=(nx, ny, nz))


def waveguide_2d_config(p=1, refine=1):
    """0.086 m x 0.043 m guide section in the x1-x3 plane, 8 x 4 cells at refine=1.

    The paper solves only in 3D and shows the x1-x3 plane of its guide; the
    two-dimensional case is one cell layer in x2 (thickness h = 0.086/8 m, PEC
    on both x2 faces, which the TE10 field satisfies exactly).
    """
    a, length = 0.086, 0.043
    nx, nz = 8 * refine, 4 * refine
    h = a / 8
    return waveguide(a, h, length, nx, 1, nz, 2.45e9, p, name=f"waveguide2d_8x4_r{refine}_p{p}")


def waveguide_3d_config(nx=32, ny=16, nz=64, p=2):
    """WR340-like guide 86.36 x 43.18 x 300 mm, TE10 at 2.45 GHz, uniform hex grid."""
    return waveguide(0.08636, 0.04318, 0.300, nx, ny, nz, 2.45e9, p,
                     name=f"waveguide3d_{nx}x{ny}x{nz}_p{p}")


def cavity(n, p, omega=5.0, jitter=0.0, seed=20260903, eps_mode=None, name="cavity", L=1.0):
    """Unit box cavity n^3, PEC walls, top face x3 = L driven by n x E = (sin(pi x2), 0, 0).

    jitter: interior vertices move by U[-jitter h, jitter h]^3; boundary
    vertices only tangentially, so faces stay planar.  eps_mode 'random':
    Re eps = exp(U[0, ln 80]), Im eps = U[0, 20] per element (streams 3, 4).
    """
    vert, elem, ijk = structured_hex(L, L, L, n, n, n)
    h = L / n
    if jitter > 0:
        nv = vert.shape[0]
        for d in range(3):
            u = uniform01(seed, d, nv)
            dv = (2.0 * u - 1.0) * jitter * h
            on_bnd = (np.abs(vert[:, d]) < 1e-12) | (np.abs(vert[:, d] - L) < 1e-12)
            dv[on_bnd] = 0.0
            vert[:, d] += dv
    spec = {'x0': (BC_DIRICHLET, 0), 'x1': (BC_DIRICHLET, 0), 'y0': (BC_DIRICHLET, 0),
            'y1': (BC_DIRICHLET, 0), 'z0': (BC_DIRICHLET, 0), 'z1': (BC_DIRICHLET, 1)}
    bc, grp = box_boundary_tags(ijk, n, n, n, spec)
    ne = elem.shape[0]
    eps = np.ones(ne, dtype=complex)
    if eps_mode == 'random':
        re = np.exp(uniform01(seed, 3, ne) * np.log(80.0))
        im = 20.0 * uniform01(seed, 4, ne)
        eps = re + 1j * im
    return Mesh(vert=vert, elem=elem, p=np.full(ne, p, dtype=np.int8), eps=eps,
                mu=np.ones(ne, dtype=complex), face_bc=bc, face_grp=grp, omega=omega,
                robin=[], dirichlet=[{'kind': DIRICHLET_ZERO, 'port': None},
                                     {'kind': DIRICHLET_SIN_PI_X2, 'port': None}],
                name=name, grid=(n, n, n))


def sphere_obstacle(mesh, center=(0.5, 0.5, 0.5), radius=0.2, eps=20.0 + 5.0j):
    """Set eps on the elements whose centroid lies inside the sphere; returns the mask."""
    cen = mesh.vert[mesh.elem].mean(axis=1)
    mask = np.linalg.norm(cen - np.asarray(center)[None, :], axis=1) < radius
    mesh.eps = mesh.eps.copy()
    mesh.eps[mask] = eps
    return mask


def _graded_unit(n, toward_hi, grade):
    """n + 1 nodes on [0, 1], denser toward 1 (toward_hi) or 0, spacing ratio set by grade >= 1."""
    t = np.arange(n + 1, dtype=np.float64) / n
    return 1.0 - (1.0 - t) ** grade if toward_hi else t ** grade


def order_mix(ne, fractions, seed, stream=5):
    """Trial degrees 1..len(fractions) in exact proportions (rounded), seeded permutation."""
    counts = [int(np.floor(f * ne)) for f in fractions]
    counts[0] += ne - sum(counts)
    p = np.concatenate([np.full(c, k + 1, dtype=np.int8) for k, c in enumerate(counts)])
    perm = np.argsort(uniform01(seed, stream, ne), kind='stable')
    out = np.empty(ne, dtype=np.int8)
    out[perm] = p
    return out


def fichera_cavity(n_unit, grade=1.0, omega=5.0, p=None, mix=(0.4, 0.3, 0.2, 0.1), seed=20260904,
                   name="fichera"):
    """Fichera-corner cavity ((0,2)^3 minus [0,1]^3, plus [1,2]^2 x [2,3]) on a graded tensor grid.

    Every unit interval of the axes is split into n_unit cells, graded toward
    the re-entrant corner (1, 1, 1) and the re-entrant edges at x3 = 2 (grade
    1 = uniform).  The grid is conforming: the local refinement of an adaptive
    mesh is imitated by the grading, not by hanging faces.  PEC walls, and on
    the top face x3 = 3 the excitation n x E = (sin(pi x2), 0, 0) (Sec. 4.2).
    Trial degrees: p for all elements if given, else drawn in the proportions
    ``mix`` for p = 1, 2, ... (seeded permutation, stream 5).
    """
    lo = _graded_unit(n_unit, True, grade)
    hi = 1.0 + _graded_unit(n_unit, False, grade)
    xs = np.concatenate([lo, hi[1:]])                       # [0, 2]
    zs = np.concatenate([lo, hi[1:], 2.0 + _graded_unit(n_unit, False, grade)[1:]])  # [0, 3]
    nx, nz = xs.size - 1, zs.size - 1
    Z, Y, X = np.meshgrid(zs, xs, xs, indexing='ij')
    allv = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    vid = lambda i, j, k: (k * (nx + 1) + j) * (nx + 1) + i
    k, j, i = np.meshgrid(np.arange(nz), np.arange(nx), np.arange(nx), indexing='ij')
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    c = np.stack([0.5 * (xs[i] + xs[i + 1]), 0.5 * (xs[j] + xs[j + 1]), 0.5 * (zs[k] + zs[k + 1])], axis=1)
    lower = (c[:, 2] < 2.0) & ~((c[:, 0] < 1.0) & (c[:, 1] < 1.0) & (c[:, 2] < 1.0))
    top = (c[:, 0] > 1.0) & (c[:, 1] > 1.0) & (c[:, 2] > 2.0)
    keep = lower | top
    i, j, k = i[keep], j[keep], k[keep]
    elem = np.zeros((i.size, 8), dtype=np.int64)
    for v in range(8):
        elem[:, v] = vid(i + (v & 1), j + ((v >> 1) & 1), k + ((v >> 2) & 1))
    used, inv = np.unique(elem.ravel(), return_inverse=True)
    vert = allv[used]
    elem = inv.reshape(elem.shape).astype(np.int32)
    ne = elem.shape[0]
    # boundary faces: faces that no other element shares
    bc = np.zeros((ne, 6), dtype=np.int8)
    grp = np.zeros((ne, 6), dtype=np.int16)
    keys = {}
    for d in range(3):
        for s in (0, 1):
            f = 2 * d + s
            cs = [v for v in range(8) if ((v >> d) & 1) == s]
            fk = np.sort(elem[:, cs], axis=1)
            for e in range(ne):
                t = tuple(fk[e])
                keys[t] = keys.get(t, 0) + 1
    for d in range(3):
        for s in (0, 1):
            f = 2 * d + s
            cs = [v for v in range(8) if ((v >> d) & 1) == s]
            fk = np.sort(elem[:, cs], axis=1)
            for e in range(ne):
                if keys[tuple(fk[e])] == 1:
                    bc[e, f] = BC_DIRICHLET
                    ztop = d == 2 and s == 1 and abs(vert[elem[e, cs[0]], 2] - 3.0) < 1e-12
                    grp[e, f] = 1 if ztop else 0
    pk = np.full(ne, p, dtype=np.int8) if p is not None else order_mix(ne, mix, seed)
    return Mesh(vert=vert, elem=elem, p=pk, eps=np.ones(ne, dtype=complex), mu=np.ones(ne, dtype=complex),
                face_bc=bc, face_grp=grp, omega=omega, robin=[],
                dirichlet=[{'kind': DIRICHLET_ZERO, 'port': None}, {'kind': DIRICHLET_SIN_PI_X2, 'port': None}],
                name=name)


def refined_box(n, refine, p=1, lengths=(1.0, 1.0, 1.0), omega=5.0, bc="cavity", name="refined_box"):
    """One level of 2:1 refinement of an n = (nx, ny, nz) box grid: hanging faces and edges.

    refine: coarse cells (i, j, k) split into 8 children.  Vertices live on the
    lattice of half cells, so children and their coarse neighbours share the
    corner and mid-edge / mid-face points; a coarse face next to a refined cell
    is matched by four child faces (a 2:1 hanging face).  Geometry is affine
    (axis-aligned box).  bc "cavity": PEC walls with n x E = (sin(pi x2), 0, 0)
    on the top face x3 = lz (the excitation of Sec. 4.2).  p: one degree for all
    elements, or a callable (element index, is_child) -> degree.
    """
    nx, ny, nz = n
    lx, ly, lz = lengths
    refine = set(tuple(c) for c in refine)
    L = (2 * nx + 1, 2 * ny + 1, 2 * nz + 1)
    lid = lambda i, j, k: (k * L[1] + j) * L[0] + i
    elems, child = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if (i, j, k) in refine:
                    for c in range(8):
                        a, b, cc = c & 1, (c >> 1) & 1, (c >> 2) & 1
                        elems.append([lid(2 * i + a + (v & 1), 2 * j + b + ((v >> 1) & 1), 2 * k + cc + ((v >> 2) & 1))
                                      for v in range(8)])
                        child.append(True)
                else:
                    elems.append([lid(2 * i + 2 * (v & 1), 2 * j + 2 * ((v >> 1) & 1), 2 * k + 2 * ((v >> 2) & 1))
                                  for v in range(8)])
                    child.append(False)
    elem = np.array(elems, dtype=np.int64)
    used, inv = np.unique(elem.ravel(), return_inverse=True)
    ii = used % L[0]
    jj = (used // L[0]) % L[1]
    kk = used // (L[0] * L[1])
    vert = np.stack([ii * lx / (2 * nx), jj * ly / (2 * ny), kk * lz / (2 * nz)], axis=1)
    elem = inv.reshape(elem.shape).astype(np.int32)
    ne = elem.shape[0]
    bc_arr = np.zeros((ne, 6), dtype=np.int8)
    grp = np.zeros((ne, 6), dtype=np.int16)
    ext = (lx, ly, lz)
    for e in range(ne):
        X = vert[elem[e]]
        for d in range(3):
            for s in (0, 1):
                cs = [v for v in range(8) if ((v >> d) & 1) == s]
                coord = X[cs, d]
                target = ext[d] if s else 0.0
                if np.all(np.abs(coord - target) < 1e-12):
                    bc_arr[e, 2 * d + s] = BC_DIRICHLET
                    grp[e, 2 * d + s] = 1 if (d == 2 and s == 1) else 0
    child = np.array(child)
    if callable(p):
        pk = np.array([p(e, bool(child[e])) for e in range(ne)], dtype=np.int8)
    else:
        pk = np.full(ne, p, dtype=np.int8)
    return Mesh(vert=vert, elem=elem, p=pk, eps=np.ones(ne, dtype=complex), mu=np.ones(ne, dtype=complex),
                face_bc=bc_arr, face_grp=grp, omega=omega, robin=[],
                dirichlet=[{'kind': DIRICHLET_ZERO, 'port': None}, {'kind': DIRICHLET_SIN_PI_X2, 'port': None}],
                name=name)


def amr_box(n, lengths, keep, refine, p=1, omega=5.0, mix=None, seed=20260904, name="amr"):
    """A masked box grid with one level of 2:1 refinement (hanging faces and edges).

    n = (nx, ny, nz) coarse cells over [0, lx] x [0, ly] x [0, lz]; keep(c) and
    refine(c) take a coarse cell centre c.  Kept cells not refined are single
    elements; refined ones are split into 8 children.  Faces without a kept
    neighbour cell are walls: PEC, and n x E = (sin(pi x2), 0, 0) on the top
    plane x3 = lz (Sec. 4.2).  Degrees: p for all, or the proportions `mix` for
    p = 1, 2, ... (seeded permutation, stream 5).
    """
    nx, ny, nz = n
    lx, ly, lz = lengths
    h = (lx / nx, ly / ny, lz / nz)
    cen = lambda i, j, k: np.array([(i + 0.5) * h[0], (j + 0.5) * h[1], (k + 0.5) * h[2]])
    kept = {(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx) if keep(cen(i, j, k))}
    ref = {c for c in kept if refine(cen(*c))}
    L = (2 * nx + 1, 2 * ny + 1, 2 * nz + 1)
    lid = lambda i, j, k: (k * L[1] + j) * L[0] + i
    elems, walls = [], []
    for (i, j, k) in sorted(kept, key=lambda c: (c[2], c[1], c[0])):
        cells = [(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)] if (i, j, k) in ref else [None]
        for ch in cells:
            if ch is None:
                base, span = (2 * i, 2 * j, 2 * k), 2
            else:
                base, span = (2 * i + ch[0], 2 * j + ch[1], 2 * k + ch[2]), 1
            elems.append([lid(base[0] + span * (v & 1), base[1] + span * ((v >> 1) & 1),
                              base[2] + span * ((v >> 2) & 1)) for v in range(8)])
            w = []
            for d in range(3):
                for s in (0, 1):
                    # a wall when the face lies on the cell's face and no kept cell is across
                    on_cell_face = ch is None or ch[d] == s
                    nb = [i, j, k]
                    nb[d] += 1 if s else -1
                    w.append(on_cell_face and tuple(nb) not in kept)
            walls.append(w)
    elem = np.array(elems, dtype=np.int64)
    used, inv = np.unique(elem.ravel(), return_inverse=True)
    ii = used % L[0]
    jj = (used // L[0]) % L[1]
    kk = used // (L[0] * L[1])
    vert = np.stack([ii * lx / (2 * nx), jj * ly / (2 * ny), kk * lz / (2 * nz)], axis=1)
    elem = inv.reshape(elem.shape).astype(np.int32)
    ne = elem.shape[0]
    bc = np.zeros((ne, 6), dtype=np.int8)
    grp = np.zeros((ne, 6), dtype=np.int16)
    for e in range(ne):
        for f in range(6):
            if walls[e][f]:
                bc[e, f] = BC_DIRICHLET
                top = f == 5 and abs(vert[elem[e, 4], 2] - lz) < 1e-12
                grp[e, f] = 1 if top else 0
    pk = np.full(ne, p, dtype=np.int8) if mix is None else order_mix(ne, mix, seed)
    return Mesh(vert=vert, elem=elem, p=pk, eps=np.ones(ne, dtype=complex), mu=np.ones(ne, dtype=complex),
                face_bc=bc, face_grp=grp, omega=omega, robin=[],
                dirichlet=[{'kind': DIRICHLET_ZERO, 'port': None}, {'kind': DIRICHLET_SIN_PI_X2, 'port': None}],
                name=name)


def fichera_amr(n_unit, radius=0.75, mix=(0.4, 0.3, 0.2, 0.1), p=None, seed=20260904):
    """Fichera-corner cavity, n_unit coarse cells per unit length, cells within `radius` of the
    re-entrant corner (1, 1, 1) refined once (2:1 hanging faces); degrees drawn in `mix`."""
    def keep(c):
        lower = c[2] < 2.0 and not (c[0] < 1.0 and c[1] < 1.0 and c[2] < 1.0)
        top = c[0] > 1.0 and c[1] > 1.0 and c[2] > 2.0
        return lower or top
    refine = lambda c: np.linalg.norm(c - np.array([1.0, 1.0, 1.0])) < radius
    n = (2 * n_unit, 2 * n_unit, 3 * n_unit)
    return amr_box(n, (2.0, 2.0, 3.0), keep, refine, p=p if p is not None else 1,
                   mix=None if p is not None else mix, seed=seed, name=f"fichera_amr_{n_unit}_r{radius}")


class OctreeHexMesh:
    """Axis-aligned hexahedra refined as an octree over kept coarse cells (geometry only).

    The coarse grid has n = (nx, ny, nz) cells over [0, lx] x [0, ly] x [0, lz];
    ``keep(centre)`` selects the coarse cells of the domain.  A leaf is
    (level, i, j, k) on the level's grid (2^level cells per coarse cell and
    direction).  The mesh stays 2:1 balanced across faces, edges and vertices:
    refining a leaf first refines every coarser leaf that touches it
    (recursively), and a family of eight children is merged back only when no
    leaf touching the parent is more than one level finer than the parent.
    Walls (faces without a domain cell across) are PEC, and the plane x3 = lz
    carries n x E = (sin(pi x2), 0, 0) (the excitation of Sec. 4.2).
    """

    _OFF = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy, dz) != (0, 0, 0)]

    def __init__(self, n, lengths, keep, p=2, omega=5.0, name="octree"):
        self.n = tuple(int(v) for v in n)
        self.lengths = tuple(float(v) for v in lengths)
        h = [lengths[d] / n[d] for d in range(3)]
        self.kept = {(i, j, k) for k in range(n[2]) for j in range(n[1]) for i in range(n[0])
                     if keep(np.array([(i + 0.5) * h[0], (j + 0.5) * h[1], (k + 0.5) * h[2]]))}
        self.leaves = {(0, i, j, k) for (i, j, k) in self.kept}
        self.p, self.omega, self.name = p, omega, name

    def in_domain(self, l, i, j, k):
        if min(i, j, k) < 0:
            return False
        c = (i >> l, j >> l, k >> l)
        return c[0] < self.n[0] and c[1] < self.n[1] and c[2] < self.n[2] and c in self.kept

    def leaf_at(self, l, i, j, k):
        """The leaf covering cell (l, i, j, k) at its level or coarser, or None (refined further, or outside)."""
        for lev in range(l, -1, -1):
            s = l - lev
            c = (lev, i >> s, j >> s, k >> s)
            if c in self.leaves:
                return c
        return None

    def refine(self, c):
        if c not in self.leaves:
            return
        l, i, j, k = c
        for dx, dy, dz in self._OFF:  # every touching leaf must be at least as fine as c first
            q = (l, i + dx, j + dy, k + dz)
            if self.in_domain(*q):
                L = self.leaf_at(*q)
                if L is not None and L[0] < l:
                    self.refine(L)
        self.leaves.discard(c)
        for ch in range(8):
            self.leaves.add((l + 1, 2 * i + (ch & 1), 2 * j + ((ch >> 1) & 1), 2 * k + ((ch >> 2) & 1)))

    def _children(self, c):
        l, i, j, k = c
        return [(l + 1, 2 * i + (ch & 1), 2 * j + ((ch >> 1) & 1), 2 * k + ((ch >> 2) & 1)) for ch in range(8)]

    def can_coarsen(self, parent):
        if parent[0] < 0 or any(ch not in self.leaves for ch in self._children(parent)):
            return False
        l, i, j, k = parent
        for dx, dy, dz in self._OFF:
            q = (l, i + dx, j + dy, k + dz)
            if not self.in_domain(*q) or self.leaf_at(*q) is not None:
                continue  # outside, or covered by a leaf of level <= l
            # q is refined: none of its children may be refined further
            if any(ch not in self.leaves for ch in self._children(q)):
                return False
        return True

    def adapt(self, leaves, marks):
        """Refine the leaves marked +1, then merge the families whose eight children are all marked -1."""
        for c, m in zip(leaves, marks):
            if m > 0:
                self.refine(c)
        parents = sorted({(c[0] - 1, c[1] >> 1, c[2] >> 1, c[3] >> 1) for c, m in zip(leaves, marks)
                          if m < 0 and c[0] > 0})
        want = {c for c, m in zip(leaves, marks) if m < 0}
        for P in parents:
            if all(ch in want for ch in self._children(P)) and self.can_coarsen(P):
                for ch in self._children(P):
                    self.leaves.discard(ch)
                self.leaves.add(P)

    def ordered_leaves(self):
        top = max(c[0] for c in self.leaves)
        key = lambda c: ((c[3] << (top - c[0])), (c[2] << (top - c[0])), (c[1] << (top - c[0])), c[0])
        return sorted(self.leaves, key=key)

    def mesh(self):
        """Mesh of the current leaves (and the leaf of each element, in element order)."""
        leaves = self.ordered_leaves()
        top = max(c[0] for c in leaves)
        scale = 1 << top
        ids, elems = {}, []
        for (l, i, j, k) in leaves:
            s = 1 << (top - l)
            row = []
            for v in range(8):
                key = ((i + (v & 1)) * s, (j + ((v >> 1) & 1)) * s, (k + ((v >> 2) & 1)) * s)
                row.append(ids.setdefault(key, len(ids)))
            elems.append(row)
        pts = np.zeros((len(ids), 3))
        for key, v in ids.items():
            pts[v] = [key[d] * self.lengths[d] / (self.n[d] * scale) for d in range(3)]
        elem = np.array(elems, dtype=np.int32)
        ne = elem.shape[0]
        bc = np.zeros((ne, 6), dtype=np.int8)
        grp = np.zeros((ne, 6), dtype=np.int16)
        for e, (l, i, j, k) in enumerate(leaves):
            for d in range(3):
                for s in (0, 1):
                    q = [i, j, k]
                    q[d] += 1 if s else -1
                    if not self.in_domain(l, *q):
                        bc[e, 2 * d + s] = BC_DIRICHLET
                        top_plane = d == 2 and s == 1 and (k + 1) == self.n[2] << l
                        grp[e, 2 * d + s] = 1 if top_plane else 0
        pk = np.full(ne, self.p, dtype=np.int8)
        m = Mesh(vert=pts, elem=elem, p=pk, eps=np.ones(ne, dtype=complex), mu=np.ones(ne, dtype=complex),
                 face_bc=bc, face_grp=grp, omega=self.omega, robin=[],
                 dirichlet=[{'kind': DIRICHLET_ZERO, 'port': None}, {'kind': DIRICHLET_SIN_PI_X2, 'port': None}],
                 name=f"{self.name}_{ne}")
        return m, leaves


def fichera_octree(p=2, omega=5.0):
    """The Fichera oven of Sec. 4.2 as an octree mesh: (0,2)^3 minus [0,1]^3, plus [1,2]^2 x [2,3], starting
    from its eight unit cells (the initial mesh of Sec. 4.2)."""
    def keep(c):
        lower = c[2] < 2.0 and not (c[0] < 1.0 and c[1] < 1.0 and c[2] < 1.0)
        top = c[0] > 1.0 and c[1] > 1.0 and c[2] > 2.0
        return lower or top
    return OctreeHexMesh((2, 2, 3), (2.0, 2.0, 3.0), keep, p=p, omega=omega, name=f"fichera_octree_p{p}")
