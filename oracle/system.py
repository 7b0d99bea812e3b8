"""Global trace numbering, assembly, solve and recovery for the oracle (test infrastructure only).

Algorithm 1 / Algorithm 2 of the paper: per cell form (G, B, B-hat, l), condense
(Sec. 2.3, Eq. linear_system), distribute local to global, solve for the trace
unknowns, reconstruct u and Psi per cell and evaluate ||Psi||_V.

The oracle's own numbering: every trace function of every element is keyed by
its mesh entity (edge = ordered vertex pair along the local axis; face =
vertex ids at the four face corners in local axis order) plus its index inside
the entity; keys get global ids in first-seen order, separately for E-hat and
H-hat.  E-hat unknowns on Dirichlet faces are fixed by nodal interpolation of
the tangential datum (our reading; data faces win over zero faces on shared
edges).  H-hat unknowns whose B-hat column vanishes (below 1e-12 of the block's largest
entry) in every element (the unconstrained Robin DoFs noted at the end of
Sec. 2.3) are removed.

Mesh input: the plain arrays of ``paper_2609_03155_b300.inputs.Mesh`` passed
in as an object with attributes vert, elem, p, eps, mu, face_bc, face_grp,
omega, robin, dirichlet (this module does not import that package).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis, element, physics

BC_NONE, BC_DIRICHLET, BC_ROBIN = 0, 1, 2


def robin_g(spec, normal):
    """Callable g(x) for a Robin group: TE_mn port datum or zero."""
    if spec.get('port') is None:
        return None
    a, b, m, n, eps, mu = spec['port']
    return physics.te_port_g(normal, spec['omega'], a, b, m, n, eps, mu)


def dirichlet_Et(spec):
    """Tangential Dirichlet datum E_t(x, n) for a Dirichlet group, or None for zero (PEC)."""
    kind = spec.get('kind', 0)
    if kind == 0:
        return None
    if kind == 1:
        # n x E = (sin(pi x2), 0, 0)  =>  E_t = (n x E) x n
        def Et(x, n):
            v = np.zeros((len(x), 3), dtype=complex)
            v[:, 0] = np.sin(np.pi * x[:, 1])
            return np.cross(v, n)
        return Et
    if kind == 2:
        a, b, m, nn, eps, mu = spec['port']

        def Et(x, n):
            E, _ = physics.te_fields(x, spec['omega'], a, b, m, nn, eps, mu)
            return np.cross(n, np.cross(E, n))
        return Et
    if kind == 3:
        return spec['callable']
    raise ValueError("unknown Dirichlet kind")


def face_normal_ref(f):
    d, s = f // 2, f % 2
    N = np.zeros(3)
    N[d] = 2.0 * s - 1.0
    return N


def element_faces(mesh, e):
    """Face descriptors for element.element_matrices (Robin faces only)."""
    faces = []
    X = mesh.vert[mesh.elem[e]]
    for f in range(6):
        if mesh.face_bc[e, f] == BC_ROBIN:
            spec = dict(mesh.robin[mesh.face_grp[e, f]])
            spec['omega'] = mesh.omega
            # the paper's Robin faces are planar: outward normal from the face centre
            d, s = f // 2, f % 2
            c = np.full((1, 3), 0.5)
            c[0, d] = s
            _, J = element.trilinear(X, c)
            nv = np.linalg.inv(J[0]).T @ face_normal_ref(f)
            nv /= np.linalg.norm(nv)
            faces.append({'robin': (spec['zinv'], robin_g(spec, nv))})
        else:
            faces.append(None)
    return faces


def trace_keys(mesh, e, r):
    """Global keys of the 12 r^2 trace functions of element e (oracle numbering)."""
    corner = lambda i, j, k: int(mesh.elem[e, i + 2 * j + 4 * k])
    keys = []
    idx = basis.nedelec_index(r)
    for k in basis.trace_functions(r):
        c, ii = idx[k]
        ent = basis.trace_entity(r, c, ii)
        if ent[0] == 'edge':
            _, c_, (d1, s1), (d2, s2) = ent
            ends = []
            for t in (0, 1):
                pos = [0, 0, 0]
                pos[c] = t
                pos[d1] = s1
                pos[d2] = s2
                ends.append(corner(*pos))
            keys.append(('E', ends[0], ends[1], ii[c]))
        else:
            _, d, s = ent
            a, b = [q for q in range(3) if q != d]
            cs = []
            for (ta, tb) in ((0, 0), (1, 0), (0, 1), (1, 1)):
                pos = [0, 0, 0]
                pos[d] = s
                pos[a] = ta
                pos[b] = tb
                cs.append(corner(*pos))
            other = [q for q in range(3) if q != c and q != d][0]
            keys.append(('F', tuple(cs), c, ii[c], ii[other]))
    return keys


def trace_on_face(r, f):
    """Local trace positions (0..12r^2-1) whose entity lies on face f = 2d+s."""
    d0, s0 = f // 2, f % 2
    idx = basis.nedelec_index(r)
    out = []
    for pos, k in enumerate(basis.trace_functions(r)):
        c, ii = idx[k]
        ent = basis.trace_entity(r, c, ii)
        if ent[0] == 'edge':
            if ent[2] == (d0, s0) or ent[3] == (d0, s0):
                out.append(pos)
        elif ent[1] == d0 and ent[2] == s0:
            out.append(pos)
    return out


class Numbering:
    pass


def number_traces(mesh):
    """Oracle numbering of E-hat and H-hat unknowns; checks orientation consistency."""
    ne = mesh.elem.shape[0]
    p = int(mesh.p[0])
    if np.any(mesh.p != p):
        raise ValueError("the oracle supports uniform p only")
    r = p + 1
    gid = {}
    edges_seen = set()
    faces_seen = {}
    loc2glob = np.zeros((ne, 12 * r * r), dtype=np.int64)
    for e in range(ne):
        for k, key in enumerate(trace_keys(mesh, e, r)):
            if key[0] == 'E':
                if (key[2], key[1]) in edges_seen:
                    raise ValueError("edge orientation mismatch")
                edges_seen.add((key[1], key[2]))
            else:
                srt = tuple(sorted(key[1]))
                if faces_seen.setdefault(srt, key[1]) != key[1]:
                    raise ValueError("face orientation mismatch")
            if key not in gid:
                gid[key] = len(gid)
            loc2glob[e, k] = gid[key]
    num = Numbering()
    num.n_entity_dofs = len(gid)
    num.loc2glob = loc2glob
    num.r = r
    return num


def dirichlet_values(mesh, num):
    """Fixed E-hat values by nodal interpolation on Dirichlet faces: {global id: value}."""
    r = num.r
    nodes = basis.nedelec_nodes(r)
    idx = basis.nedelec_index(r)
    tsel = basis.trace_functions(r)
    fixed = {}
    has_data = {}
    for e in range(mesh.elem.shape[0]):
        X = mesh.vert[mesh.elem[e]]
        for f in range(6):
            if mesh.face_bc[e, f] != BC_DIRICHLET:
                continue
            spec = dict(mesh.dirichlet[mesh.face_grp[e, f]])
            spec['omega'] = mesh.omega
            Et = dirichlet_Et(spec)
            for pos in trace_on_face(r, f):
                g = num.loc2glob[e, pos]
                if Et is None:
                    if g not in fixed:
                        fixed[g] = 0.0
                    continue
                c = idx[tsel[pos]][0]
                xi = nodes[tsel[pos]][None, :]
                x, J = element.trilinear(X, xi)
                d, s = f // 2, f % 2
                nv = np.linalg.inv(J[0]).T @ face_normal_ref(f)
                nv /= np.linalg.norm(nv)
                val = Et(x, nv[None, :])[0] @ J[0][:, c]
                if not has_data.get(g, False):
                    fixed[g] = val
                    has_data[g] = True
    return fixed


def solve(mesh, source=None, direct=True, cg_rtol=1e-12, keep_elements=True):
    """Run the whole DPG pipeline of Algorithm 1 on ``mesh`` in complex FP64.

    Returns a dict with per-element data (element matrices, condensation,
    recovery), the global system and the trace solution.
    """
    ne = mesh.elem.shape[0]
    p = int(mesh.p[0])
    num = number_traces(mesh)
    nt = 12 * num.r * num.r
    els, conds = [], []
    for e in range(ne):
        X = mesh.vert[mesh.elem[e]]
        el = element.element_matrices(X, p, mesh.omega, complex(mesh.eps[e]), complex(mesh.mu[e]),
                                      element_faces(mesh, e), source=source)
        els.append(el)
        conds.append(element.condense(el))
    nE = num.n_entity_dofs
    # global ids: E-hat g in [0, nE), H-hat g in [nE, 2 nE)
    fixed = dirichlet_values(mesh, num)
    hcol_nonzero = np.zeros(nE, dtype=bool)
    for e in range(ne):
        # a column is structurally zero when it is below rounding of the block
        Bh_H = els[e].Bh[:, nt:]
        nz = np.max(np.abs(Bh_H), axis=0) > 1e-12 * np.max(np.abs(els[e].Bh))
        hcol_nonzero[num.loc2glob[e][nz]] = True
    free = np.full(2 * nE, -1, dtype=np.int64)
    cnt = 0
    for g in range(nE):
        if g not in fixed:
            free[g] = cnt
            cnt += 1
    for g in range(nE):
        if hcol_nonzero[g]:
            free[nE + g] = cnt
            cnt += 1
    n = cnt
    xfix = np.zeros(2 * nE, dtype=complex)
    for g, v in fixed.items():
        xfix[g] = v
    rows, cols, vals = [], [], []
    b = np.zeros(n, dtype=complex)
    l2g = []
    for e in range(ne):
        gl = np.concatenate([num.loc2glob[e], nE + num.loc2glob[e]])
        l2g.append(gl)
        S, s = conds[e]['S'], conds[e]['s']
        fr = free[gl]
        lift = S @ xfix[gl]
        for i in range(len(gl)):
            if fr[i] < 0:
                continue
            b[fr[i]] += s[i] - lift[i]
            m = fr >= 0
            rows.append(np.full(m.sum(), fr[i]))
            cols.append(fr[m])
            vals.append(S[i, m])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    if direct:
        if n <= 6000:
            x = np.linalg.solve(A.toarray(), b)
        else:
            x = spla.splu(A.tocsc()).solve(b)
        info = None
    else:
        x, info = cg(A, b, rtol=cg_rtol)
    # recovery per element
    xfull = xfix.copy()
    xfull[free >= 0] = x[free[free >= 0]]
    recs = []
    for e in range(ne):
        uh = xfull[l2g[e]]
        recs.append(element.recover(els[e], conds[e], uh))
    out = dict(num=num, elements=els if keep_elements else None, conds=conds, A=A, b=b, x=x,
               free=free, xfix=xfix, xfull=xfull, l2g=l2g, rec=recs, n=n, cg_info=info)
    out['eta'] = np.array([rc['eta'] for rc in recs])
    return out


def cg(A, b, rtol=1e-10, atol=0.0, max_iter=100000, x0=None):
    """Unpreconditioned conjugate gradients on a Hermitian positive definite A (Sec. 2.3).

    x0 = 0, stops when ||r||_2 <= max(rtol ||b||_2, atol).  Complex arithmetic,
    alpha = r^H r / p^H A p.  Returns (x, dict(iters, relres, converged)).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    p = r.copy()
    rr = np.vdot(r, r).real
    bn = np.linalg.norm(b)
    tol = max(rtol * bn, atol)
    it = 0
    while np.sqrt(rr) > tol and it < max_iter:
        Ap = A @ p
        alpha = rr / np.vdot(p, Ap).real
        x += alpha * p
        r -= alpha * Ap
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, dict(iters=it, relres=np.sqrt(rr) / bn if bn > 0 else 0.0, converged=np.sqrt(rr) <= tol)


def fields_at(mesh, e, u, xi):
    """Interior E and H of element e at reference points xi from its coefficients u."""
    p = int(mesh.p[e])
    L = basis.lagrange3_eval(p, xi)
    nL = L.shape[1]
    E = np.stack([L @ u[d * nL:(d + 1) * nL] for d in range(3)], axis=1)
    H = np.stack([L @ u[(3 + d) * nL:(4 + d) * nL] for d in range(3)], axis=1)
    return E, H


def l2_field_error(mesh, sol, exact, nq=None):
    """Relative L2(Omega) errors of E and H against a closed form exact(x) -> (E, H)."""
    p = int(mesh.p[0])
    nq = nq or p + 4
    xi, w = element.tensor_points(nq)
    errE = errH = nrmE = nrmH = 0.0
    for e in range(mesh.elem.shape[0]):
        X = mesh.vert[mesh.elem[e]]
        x, J = element.trilinear(X, xi)
        det = np.linalg.det(J)
        E, H = fields_at(mesh, e, sol['rec'][e]['u'], xi)
        Ex, Hx = exact(x)
        wd = w * det
        errE += np.sum(wd * np.sum(np.abs(E - Ex) ** 2, axis=1))
        errH += np.sum(wd * np.sum(np.abs(H - Hx) ** 2, axis=1))
        nrmE += np.sum(wd * np.sum(np.abs(Ex) ** 2, axis=1))
        nrmH += np.sum(wd * np.sum(np.abs(Hx) ** 2, axis=1))
    return np.sqrt(errE / nrmE), np.sqrt(errH / nrmH)
