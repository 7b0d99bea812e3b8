"""Trace constraints of 2:1 hanging faces and edges for the oracle (test infrastructure only).

The paper's adaptive meshes refine in h (Sec. 4.2) and so have hanging faces,
but it does not state how their traces are constrained.  Reading taken here:
an edge or face that lies inside a larger edge or face of a neighbour (a slave)
carries no unknowns of its own; its trace is the larger entity's (the
master's) trace restricted to it, which keeps the trace single-valued and
inside every neighbour's trace space.  As for mixed degrees, each element
keeps its own nodal trace coefficients, u-hat_K = R_K u-hat:
* a coefficient on a master entity of K is the nodal value of that entity's
  global trace (1D Lagrange polynomials of the entity order at K's node, the
  edges of a face entering through the closed factor of the face order);
* a coefficient on a slave is the master's trace evaluated at the physical node
  (through the master owner's reference coordinates), times the ratio of the
  tangents J_K e_c and J_M e_c (1/2 for a 2:1 child).
Entity order: min over the elements that touch the entity's geometry of p + 1,
and an edge of a master face at most the face's order.
Geometry is assumed affine (containment and the inverse map use it).
Uniform meshes without refinement reproduce ``mixed.solve_mixed``.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis, element, system
from .mixed import _closed, _edge_key, _face_key, _lag, _open

_TOL = 1e-10


def _corner(mesh, e, pos):
    return int(mesh.elem[e, pos[0] + 2 * pos[1] + 4 * pos[2]])


def _element_entities(mesh, e):
    """[(key, kind, axis c (edges) or normal d (faces), geometry)] of element e's 12 edges and 6 faces."""
    out = []
    for c in range(3):
        tr = [q for q in range(3) if q != c]
        for s1 in (0, 1):
            for s2 in (0, 1):
                k = _edge_key(mesh, e, c, {tr[0]: s1, tr[1]: s2})
                out.append((k, 'E', c, mesh.vert[[k[1], k[2]]]))
    for d in range(3):
        for sd in (0, 1):
            k = _face_key(mesh, e, d, sd)
            out.append((k, 'F', d, mesh.vert[list(k[1])]))
    return out


def _in_segment(x, a, b):
    t = np.dot(x - a, b - a) / np.dot(b - a, b - a)
    return -_TOL <= t <= 1 + _TOL and np.linalg.norm(a + t * (b - a) - x) < _TOL * max(1.0, np.linalg.norm(b - a))


def _in_face(x, C, interior=False):
    # C: corners in order (0,0), (1,0), (0,1), (1,1) of the face's two axes (a parallelogram);
    # interior: strictly inside (not on the face's boundary)
    A = np.stack([C[1] - C[0], C[2] - C[0]], axis=1)
    st, *_ = np.linalg.lstsq(A, x - C[0], rcond=None)
    lo, hi = (1e-6, 1 - 1e-6) if interior else (-_TOL, 1 + _TOL)
    return (np.all(st >= lo) and np.all(st <= hi)
            and np.linalg.norm(A @ st + C[0] - x) < _TOL * max(1.0, np.linalg.norm(A)))


class Topology:
    """Masters, owners and orders of every edge and face of a (possibly 2:1 refined) hex mesh."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.ents = {}       # key -> (kind, axis, geometry)
        self.owner = {}      # key -> an element that has it as its own entity
        self.touch = {}      # key -> elements whose own entity is this one
        for e in range(mesh.elem.shape[0]):
            for k, kind, ax, geo in _element_entities(mesh, e):
                self.ents[k] = (kind, ax, geo)
                self.owner.setdefault(k, e)
                self.touch.setdefault(k, set()).add(e)
        keys = list(self.ents)
        self.master = {}
        for k in keys:
            kind, ax, geo = self.ents[k]
            self.master[k] = k
            # an edge inside a larger edge (same axis), else inside a face; a face inside a larger face
            for kind_m in (('E', 'F') if kind == 'E' else ('F',)):
                found = None
                for m in keys:
                    km, axm, geom = self.ents[m]
                    if m == k or km != kind_m:
                        continue
                    if kind == 'E' and km == 'E':
                        if axm != ax or np.linalg.norm(geom[1] - geom[0]) <= np.linalg.norm(geo[1] - geo[0]) + _TOL:
                            continue
                        if _in_segment(geo[0], *geom) and _in_segment(geo[1], *geom):
                            found = m
                    elif km == 'F':
                        if kind == 'E':
                            # an edge inside the face, not on its boundary (edges on the
                            # boundary belong to the face's edges)
                            if axm == ax:
                                continue
                            if all(_in_face(x, geom) for x in geo) and _in_face(0.5 * (geo[0] + geo[1]), geom, True):
                                found = m
                        else:
                            if axm != ax or _area(geom) <= _area(geo) + _TOL:
                                continue
                            if all(_in_face(x, geom) for x in geo):
                                found = m
                    if found is not None:
                        break
                if found is not None:
                    self.master[k] = found
                    break
        # follow chains (an edge inside a face that is itself a slave) to the top master
        for k in keys:
            m = self.master[k]
            while self.master[m] != m:
                m = self.master[m]
            self.master[k] = m
        # order of a master: min over the elements touching it or any of its slaves
        self.order = {}
        for k in keys:
            m = self.master[k]
            r = min(int(mesh.p[e]) + 1 for e in self.touch[k])
            self.order[m] = min(self.order.get(m, r), r)
        self.normal = {k: self.ents[k][1] for k in keys if self.ents[k][0] == 'F'}
        # an edge of a master face is capped by the face's order: the face's
        # trace (edge functions included) must lie in the trace space of every
        # element touching the face, including lower-degree children on it
        # (automatic on conforming meshes, where the face's elements contain its edges)
        for k in keys:
            if self.ents[k][0] != 'F' or not self.is_master(k):
                continue
            e = self.owner[k]
            d = self.normal[k]
            sd = int(round(np.mean([_inverse(mesh, e, x)[d] for x in self.ents[k][2]])))
            for c in range(3):
                if c == d:
                    continue
                eax = [q for q in range(3) if q != c and q != d][0]
                for send in (0, 1):
                    em = self.master[_edge_key(mesh, e, c, {d: sd, eax: send})]
                    self.order[em] = min(self.order[em], self.order[k])

    def is_master(self, k):
        return self.master[k] == k


def _area(C):
    return np.linalg.norm(np.cross(C[1] - C[0], C[2] - C[0]))


def _map(mesh, e, xi):
    return element.trilinear(mesh.vert[mesh.elem[e]], np.atleast_2d(xi))


def _inverse(mesh, e, x):
    """Reference point of physical x in element e (affine elements)."""
    X = mesh.vert[mesh.elem[e]]
    x0, J = element.trilinear(X, np.array([[0.0, 0.0, 0.0]]))
    return np.linalg.solve(J[0], x - x0[0])


def number(topo):
    """Global trace ids (one field) of the master entities: (key, local index) -> id."""
    gid = {}
    for key in sorted((k for k in topo.ents if topo.is_master(k)), key=lambda k: (k[0], k[1:])):
        r = topo.order[key]
        if key[0] == 'E':
            for i2 in range(r):
                gid[(key, ('e', i2))] = len(gid)
        else:
            for c in [q for q in range(3) if q != topo.normal[key]]:
                for a in range(r):
                    for b in range(1, r):
                        gid[(key, ('f', c, a, b))] = len(gid)
    return gid


def _add(acc, other, scale=1.0):
    for g, v in other.items():
        acc[g] = acc.get(g, 0.0) + scale * v


def edge_trace(topo, gid, key, e, xi):
    """Covariant coefficient along element e's tangent of edge `key` (an entity of e) at e's point xi."""
    mesh = topo.mesh
    c = topo.ents[key][1]
    m = topo.master[key]
    if m == key:
        r = topo.order[key]
        L = _lag(_open(r), xi[c])
        return {gid[(key, ('e', q))]: L[q] for q in range(r)}
    x, J = _map(mesh, e, xi)
    em = topo.owner[m]
    xim = _inverse(mesh, em, x[0])
    _, Jm = _map(mesh, em, xim)
    tK, tM = J[0][:, c], Jm[0][:, c]
    scale = np.dot(tK, tM) / np.dot(tM, tM)
    out = {}
    if m[0] == 'E':
        _add(out, edge_trace(topo, gid, m, em, xim), scale)
    else:
        _add(out, face_trace(topo, gid, m, em, c, xim), scale)
    return out


def face_trace(topo, gid, key, e, c, xi):
    """Covariant coefficient along e's axis c of face `key` (an entity of e) at e's point xi."""
    mesh = topo.mesh
    m = topo.master[key]
    if m != key:
        x, J = _map(mesh, e, xi)
        em = topo.owner[m]
        xim = _inverse(mesh, em, x[0])
        _, Jm = _map(mesh, em, xim)
        tK, tM = J[0][:, c], Jm[0][:, c]
        out = {}
        _add(out, face_trace(topo, gid, m, em, c, xim), np.dot(tK, tM) / np.dot(tM, tM))
        return out
    d = topo.normal[key]
    sd = int(round(xi[d]))
    eax = [q for q in range(3) if q != c and q != d][0]
    rF = topo.order[key]
    Lo, Lc = _lag(_open(rF), xi[c]), _lag(_closed(rF), xi[eax])
    out = {}
    for a in range(rF):
        for b in range(1, rF):
            g = gid[(key, ('f', c, a, b))]
            out[g] = out.get(g, 0.0) + Lo[a] * Lc[b]
    for send, endidx in ((0, 0), (1, rF)):
        ekey = _edge_key(mesh, e, c, {d: sd, eax: send})
        xe = np.array(xi, dtype=float)
        xe[eax] = float(send)
        _add(out, edge_trace(topo, gid, ekey, e, xe), Lc[endidx])
    return out


def element_R(topo, gid, e):
    """R_K (12 r_K^2 x local columns) and the global ids of its columns (one field)."""
    mesh = topo.mesh
    rK = int(mesh.p[e]) + 1
    idx = basis.nedelec_index(rK)
    oK, cK = _open(rK), _closed(rK)
    rows = []
    for k in basis.trace_functions(rK):
        c, ii = idx[k]
        ent = basis.trace_entity(rK, c, ii)
        xi = np.array([oK[ii[q]] if q == c else cK[ii[q]] for q in range(3)])
        if ent[0] == 'edge':
            _, _, (d1, s1), (d2, s2) = ent
            rows.append(edge_trace(topo, gid, _edge_key(mesh, e, c, {d1: s1, d2: s2}), e, xi))
        else:
            _, d, sd = ent
            rows.append(face_trace(topo, gid, _face_key(mesh, e, d, sd), e, c, xi))
    cols = sorted({g for row in rows for g, v in row.items() if abs(v) > 0})
    pos = {g: j for j, g in enumerate(cols)}
    R = np.zeros((len(rows), len(cols)))
    for i, row in enumerate(rows):
        for g, v in row.items():
            if g in pos:
                R[i, pos[g]] += v
    return R, np.array(cols, dtype=np.int64)


def dirichlet_values(topo, gid):
    """Fixed E-hat values of the master entities on Dirichlet faces (nodal interpolation at their own nodes)."""
    mesh = topo.mesh
    fixed, has_data = {}, {}
    for e in range(mesh.elem.shape[0]):
        for f in range(6):
            if mesh.face_bc[e, f] != system.BC_DIRICHLET:
                continue
            spec = dict(mesh.dirichlet[mesh.face_grp[e, f]])
            spec['omega'] = mesh.omega
            Et = system.dirichlet_Et(spec)
            d, sd = f // 2, f % 2
            tang = [q for q in range(3) if q != d]
            fkey = _face_key(mesh, e, d, sd)
            dofs = []
            if topo.is_master(fkey):
                rF = topo.order[fkey]
                for c in tang:
                    eax = [q for q in tang if q != c][0]
                    for a in range(rF):
                        for b in range(1, rF):
                            node = [0.0] * 3
                            node[d], node[c], node[eax] = float(sd), _open(rF)[a], _closed(rF)[b]
                            dofs.append((gid[(fkey, ('f', c, a, b))], node, c))
            for c in tang:
                eax = [q for q in tang if q != c][0]
                for send in (0, 1):
                    ekey = _edge_key(mesh, e, c, {d: sd, eax: send})
                    if not topo.is_master(ekey):
                        continue
                    re = topo.order[ekey]
                    for i2 in range(re):
                        node = [0.0] * 3
                        node[d], node[eax], node[c] = float(sd), float(send), _open(re)[i2]
                        dofs.append((gid[(ekey, ('e', i2))], node, c))
            for g, node, c in dofs:
                if Et is None:
                    fixed.setdefault(g, 0.0)
                    continue
                if has_data.get(g, False):
                    continue
                x, J = element.trilinear(mesh.vert[mesh.elem[e]], np.array([node]))
                nv = np.linalg.inv(J[0]).T @ system.face_normal_ref(f)
                nv /= np.linalg.norm(nv)
                fixed[g] = Et(x, nv[None, :])[0] @ J[0][:, c]
                has_data[g] = True
    return fixed


def solve(mesh, source=None):
    """Algorithm 1 with R_K from masters, slaves and entity orders (direct solve)."""
    topo = Topology(mesh)
    gid = number(topo)
    nE = len(gid)
    ne = mesh.elem.shape[0]
    els, conds, Rs = [], [], []
    for e in range(ne):
        X = mesh.vert[mesh.elem[e]]
        el = element.element_matrices(X, int(mesh.p[e]), mesh.omega, complex(mesh.eps[e]), complex(mesh.mu[e]),
                                      system.element_faces(mesh, e), source=source)
        els.append(el)
        conds.append(element.condense(el))
        R, gl = element_R(topo, gid, e)
        Rfull = np.block([[R, np.zeros_like(R)], [np.zeros_like(R), R]])
        Rs.append((Rfull, np.concatenate([gl, nE + gl])))
    fixed = dirichlet_values(topo, gid)
    colmax = np.zeros(2 * nE)
    scale = max(np.abs(el.Bh).max() for el in els)
    for el, (R, gl) in zip(els, Rs):
        np.maximum.at(colmax, gl, np.abs(el.Bh @ R).max(axis=0))
    free = np.full(2 * nE, -1, dtype=np.int64)
    cnt = 0
    for g in range(nE):
        if g not in fixed:
            free[g] = cnt
            cnt += 1
    for g in range(nE):
        if colmax[nE + g] > 1e-12 * scale:
            free[nE + g] = cnt
            cnt += 1
    n = cnt
    xfix = np.zeros(2 * nE, dtype=complex)
    for g, v in fixed.items():
        xfix[g] = v
    A = sp.lil_matrix((n, n), dtype=complex)
    b = np.zeros(n, dtype=complex)
    for e in range(ne):
        R, gl = Rs[e]
        S, s = conds[e]['S'], conds[e]['s']
        SR = R.conj().T @ S @ R
        sR = R.conj().T @ (s - S @ (R @ xfix[gl]))
        fr = free[gl]
        m = fr >= 0
        A[np.ix_(fr[m], fr[m])] = A[np.ix_(fr[m], fr[m])] + SR[np.ix_(m, m)]
        b[fr[m]] += sR[m]
    A = A.tocsr()
    x = np.linalg.solve(A.toarray(), b) if n <= 6000 else spla.splu(A.tocsc()).solve(b)
    xfull = xfix.copy()
    xfull[free >= 0] = x[free[free >= 0]]
    recs = [element.recover(els[e], conds[e], Rs[e][0] @ xfull[Rs[e][1]]) for e in range(ne)]
    return dict(elements=els, conds=conds, R=Rs, A=A, b=b, x=x, free=free, xfix=xfix, xfull=xfull, rec=recs, n=n,
                topo=topo, gid=gid, eta=np.array([rc['eta'] for rc in recs]))
