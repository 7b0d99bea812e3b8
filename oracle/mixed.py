"""Mixed-order DPG assembly for the oracle (test infrastructure only).

The paper refines in h only (Sec. 4.2); mixed trial orders are the batching
case of this build.  Reading taken here: every mesh entity (edge, face) carries
trace unknowns of order r_E = min over the elements that contain it of
(p_K + 1), so each trace lies in every neighbour's own trace space.  Element K
is still formed and condensed at its own order (Sec. 2.3); its local trace
coefficients are the values of the global trace at its own Nedelec nodes,
u-hat_K = R_K u-hat.  With the nodal basis of ``basis`` (open Gauss-Legendre
and closed Gauss-Lobatto Lagrange factors) the entries of R_K are products of
1D Lagrange polynomials of the entity order evaluated at the element's nodes.
On a face the global trace is the order-r_F Nedelec trace whose edge
coefficients are the edges' own (lower or equal order) edge polynomials.

For uniform p, R_K is the identity selection and ``solve_mixed`` reproduces
``system.solve`` (pinned in tests/test_oracle_mixed.py).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis, element, system


def _lag(nodes, x):
    return basis.lagrange_1d(nodes, np.atleast_1d(x))[0][0]


def _open(r):
    return basis.gauss_legendre(r)[0]


def _closed(r):
    return basis.gauss_lobatto_nodes(r + 1)


def _edge_key(mesh, e, c, s1pos):
    """Ordered vertex pair of element e's edge along axis c; s1pos = {axis: side} of the transverse axes."""
    def corner(pos):
        return int(mesh.elem[e, pos[0] + 2 * pos[1] + 4 * pos[2]])
    pos0 = [0, 0, 0]
    pos1 = [0, 0, 0]
    for d, sd in s1pos.items():
        pos0[d] = sd
        pos1[d] = sd
    pos1[c] = 1
    return ('E', corner(pos0), corner(pos1))


def _face_key(mesh, e, d, sd):
    a, b = [q for q in range(3) if q != d]
    cs = []
    for (ta, tb) in ((0, 0), (1, 0), (0, 1), (1, 1)):
        pos = [0, 0, 0]
        pos[d] = sd
        pos[a] = ta
        pos[b] = tb
        cs.append(int(mesh.elem[e, pos[0] + 2 * pos[1] + 4 * pos[2]]))
    return ('F', tuple(cs))


def entity_orders(mesh):
    """Trace order r_E of every edge and face (min over the elements containing it) and face normals."""
    order = {}
    normal = {}
    for e in range(mesh.elem.shape[0]):
        r = int(mesh.p[e]) + 1
        for c in range(3):
            tr = [q for q in range(3) if q != c]
            for s1 in (0, 1):
                for s2 in (0, 1):
                    k = _edge_key(mesh, e, c, {tr[0]: s1, tr[1]: s2})
                    order[k] = min(order.get(k, r), r)
        for d in range(3):
            for sd in (0, 1):
                k = _face_key(mesh, e, d, sd)
                order[k] = min(order.get(k, r), r)
                normal[k] = d
    return order, normal


def element_R(mesh, e, order, gid):
    """R_K (12 r_K^2 x n_local_global) and the global trace ids of its columns (one field)."""
    rK = int(mesh.p[e]) + 1
    idx = basis.nedelec_index(rK)
    oK, cK = _open(rK), _closed(rK)
    cols = {}
    entries = []
    tsel = basis.trace_functions(rK)
    for j, k in enumerate(tsel):
        c, ii = idx[k]
        ent = basis.trace_entity(rK, c, ii)
        xc = oK[ii[c]]
        if ent[0] == 'edge':
            _, _, (d1, s1), (d2, s2) = ent
            key = _edge_key(mesh, e, c, {d1: s1, d2: s2})
            re = order[key]
            oe = _open(re)
            for i2 in range(re):
                entries.append((j, gid[(key, ('e', i2))], _lag(oe, xc)[i2]))
        else:
            _, d, sd = ent
            eax = [q for q in range(3) if q != c and q != d][0]
            xe = cK[ii[eax]]
            key = _face_key(mesh, e, d, sd)
            rF = order[key]
            oF, cF = _open(rF), _closed(rF)
            Lo, Lc = _lag(oF, xc), _lag(cF, xe)
            for a in range(rF):
                for b in range(1, rF):
                    entries.append((j, gid[(key, ('f', c, a, b))], Lo[a] * Lc[b]))
            # the two edges of this face along c, at xi_eax = 0 and 1
            for send, endidx in ((0, 0), (1, rF)):
                ekey = _edge_key(mesh, e, c, {d: sd, eax: send})
                re = order[ekey]
                oe = _open(re)
                Le = _lag(oe, xc)
                for i2 in range(re):
                    entries.append((j, gid[(ekey, ('e', i2))], Lc[endidx] * Le[i2]))
    for (_, g, _) in entries:
        if g not in cols:
            cols[g] = len(cols)
    R = np.zeros((len(tsel), len(cols)))
    for (j, g, v) in entries:
        R[j, cols[g]] += v
    gl = np.zeros(len(cols), dtype=np.int64)
    for g, c in cols.items():
        gl[c] = g
    return R, gl


def number_mixed(mesh):
    """Global trace ids (one field) keyed by (entity, within-entity index)."""
    order, normal = entity_orders(mesh)
    gid = {}
    for key in sorted(order, key=lambda k: (k[0], k[1:])):
        r = order[key]
        if key[0] == 'E':
            for i2 in range(r):
                gid[(key, ('e', i2))] = len(gid)
        else:
            # tangential components of the face (element axes agree across it)
            for c in [q for q in range(3) if q != normal[key]]:
                for a in range(r):
                    for b in range(1, r):
                        gid[(key, ('f', c, a, b))] = len(gid)
    return order, gid


def dirichlet_values_mixed(mesh, order, gid):
    """Fixed E-hat values: nodal interpolation of the tangential datum at each entity's own nodes."""
    fixed, has_data = {}, {}
    for e in range(mesh.elem.shape[0]):
        X = mesh.vert[mesh.elem[e]]
        for f in range(6):
            if mesh.face_bc[e, f] != system.BC_DIRICHLET:
                continue
            spec = dict(mesh.dirichlet[mesh.face_grp[e, f]])
            spec['omega'] = mesh.omega
            Et = system.dirichlet_Et(spec)
            d, sd = f // 2, f % 2
            tang = [q for q in range(3) if q != d]
            dofs = []  # (global id, reference node, component)
            fkey = _face_key(mesh, e, d, sd)
            rF = order[fkey]
            for c in tang:
                eax = [q for q in tang if q != c][0]
                for a in range(rF):
                    for b in range(1, rF):
                        node = [0.0, 0.0, 0.0]
                        node[d] = float(sd)
                        node[c] = _open(rF)[a]
                        node[eax] = _closed(rF)[b]
                        dofs.append((gid[(fkey, ('f', c, a, b))], node, c))
                for send in (0, 1):
                    ekey = _edge_key(mesh, e, c, {d: sd, eax: send})
                    re = order[ekey]
                    for i2 in range(re):
                        node = [0.0, 0.0, 0.0]
                        node[d] = float(sd)
                        node[eax] = float(send)
                        node[c] = _open(re)[i2]
                        dofs.append((gid[(ekey, ('e', i2))], node, c))
            for g, node, c in dofs:
                if Et is None:
                    fixed.setdefault(g, 0.0)
                    continue
                if has_data.get(g, False):
                    continue
                x, J = element.trilinear(X, np.array([node]))
                # unit normal of the (planar) face at the node: J^{-T} N_ref (Nanson)
                nv = np.linalg.inv(J[0]).T @ system.face_normal_ref(f)
                nv /= np.linalg.norm(nv)
                fixed[g] = Et(x, nv[None, :])[0] @ J[0][:, c]
                has_data[g] = True
    return fixed


def solve_mixed(mesh, source=None):
    """Algorithm 1 with per-element orders: elements at their own order, traces at entity order."""
    ne = mesh.elem.shape[0]
    order, gid = number_mixed(mesh)
    nE = len(gid)
    els, conds, Rs = [], [], []
    for e in range(ne):
        X = mesh.vert[mesh.elem[e]]
        el = element.element_matrices(X, int(mesh.p[e]), mesh.omega, complex(mesh.eps[e]), complex(mesh.mu[e]),
                                      system.element_faces(mesh, e), source=source)
        els.append(el)
        conds.append(element.condense(el))
        R, gl = element_R(mesh, e, order, gid)
        # both fields share the entity structure: block-diagonal R for [E-hat, H-hat]
        Rfull = np.block([[R, np.zeros_like(R)], [np.zeros_like(R), R]])
        Rs.append((Rfull, np.concatenate([gl, nE + gl])))
    fixed = dirichlet_values_mixed(mesh, order, gid)
    # unpaired H-hat unknowns: global columns of B-hat_K R_K that vanish everywhere
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
    return dict(elements=els, conds=conds, R=Rs, A=A, b=b, x=x, free=free, xfix=xfix, xfull=xfull, rec=recs,
                n=n, order=order, gid=gid, eta=np.array([rc['eta'] for rc in recs]))
