"""Pins of the oracle's hanging-face constraints (2:1 refinement; slaves take their master's trace)."""
import numpy as np
import pytest

from oracle import basis, element, hanging, mixed, system
from paper_2609_03155_b300 import inputs


def test_without_refinement_it_is_the_mixed_order_solver():
    m = inputs.refined_box((2, 1, 1), [], p=lambda e, ch: 1 + (e % 2))
    a = hanging.solve(m)
    b = mixed.solve_mixed(m)
    assert a['n'] == b['n']
    for e in range(m.n_elem):
        assert np.allclose(a['rec'][e]['u'], b['rec'][e]['u'], rtol=0, atol=1e-12)


def test_slave_entities_of_one_refined_cell():
    m = inputs.refined_box((2, 1, 1), [(0, 0, 0)], p=1)
    topo = hanging.Topology(m)
    slaves = [k for k in topo.ents if not topo.is_master(k)]
    # one coarse face split in four: 4 child faces, 4 interior cross edges, 8 half edges
    assert sum(1 for k in slaves if k[0] == 'F') == 4
    assert sum(1 for k in slaves if k[0] == 'E') == 12
    assert sum(1 for k in slaves if k[0] == 'E' and topo.master[k][0] == 'F') == 4


def _tangential_trace_on(mesh, e, u_tr, f, pts_phys):
    """Tangential E-hat of element e's local trace coefficients at physical points of its face f."""
    r = int(mesh.p[e]) + 1
    X = mesh.vert[mesh.elem[e]]
    x0, J = element.trilinear(X, np.array([[0.0, 0.0, 0.0]]))
    xi = np.linalg.solve(J[0], (pts_phys - x0[0]).T).T
    val, _ = basis.nedelec_eval(r, xi)
    tsel = basis.trace_functions(r)
    E = np.einsum('nkc,k->nc', val[:, tsel, :], u_tr) @ np.linalg.inv(J[0])  # J^{-T} f  (row form)
    d = f // 2
    nrm = np.linalg.inv(J[0]).T @ system.face_normal_ref(f)
    nrm /= np.linalg.norm(nrm)
    return E - np.outer(E @ nrm, nrm)


@pytest.mark.parametrize("orders", ["uniform", "mixed"])
def test_trace_is_continuous_across_the_hanging_face(orders):
    """For a random global trace, fine and coarse sides give the same tangential trace on the shared face."""
    p = 2 if orders == "uniform" else (lambda e, ch: 2 if ch else 3)
    m = inputs.refined_box((2, 1, 1), [(0, 0, 0)], p=p)
    topo = hanging.Topology(m)
    gid = hanging.number(topo)
    rng = np.random.default_rng(7)
    g = rng.normal(size=len(gid))
    coarse = [e for e in range(m.n_elem) if np.ptp(m.vert[m.elem[e]][:, 0]) > 0.4][0]
    Rc, glc = hanging.element_R(topo, gid, coarse)
    uc = Rc @ g[glc]
    pts = []
    for a in np.linspace(0.05, 0.95, 5):
        for b in np.linspace(0.05, 0.95, 5):
            pts.append([0.5, a, b])  # the coarse cell's face x = 0.5
    pts = np.array(pts)
    Ec = _tangential_trace_on(m, coarse, uc, 0, pts)
    for e in range(m.n_elem):
        X = m.vert[m.elem[e]]
        if e == coarse or abs(X[:, 0].max() - 0.5) > 1e-12:
            continue
        Rk, glk = hanging.element_R(topo, gid, e)
        uk = Rk @ g[glk]
        lo, hi = X.min(axis=0), X.max(axis=0)
        inside = np.all((pts[:, 1:] >= lo[1:] - 1e-12) & (pts[:, 1:] <= hi[1:] + 1e-12), axis=1)
        Ek = _tangential_trace_on(m, e, uk, 1, pts[inside])
        assert np.allclose(Ek, Ec[inside], rtol=0, atol=1e-12 * np.abs(Ec).max())


def test_manufactured_solution_exact_with_hanging_faces(monkeypatch):
    """A polynomial Maxwell solution inside every element's spaces is reproduced exactly on a 2:1 mesh."""
    rng = np.random.default_rng(4)
    omega, eps, mu, zinv = 2.0, 1.5 + 0.2j, 1.2 + 0j, 0.6 + 0.1j
    Ex = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    E0 = rng.normal(size=3) + 1j * rng.normal(size=3)
    curlE = np.array([Ex[2, 1] - Ex[1, 2], Ex[0, 2] - Ex[2, 0], Ex[1, 0] - Ex[0, 1]])
    H0 = curlE / (1j * omega * mu)
    exact = lambda x: (E0[None, :] + x @ Ex.T, np.broadcast_to(H0, (len(x), 3)).copy())
    src = lambda x: 1j * omega * eps * exact(x)[0]
    m = inputs.refined_box((2, 1, 1), [(1, 0, 0)], p=lambda e, ch: 1 if ch else 2, lengths=(1.0, 0.8, 0.6))
    ne = m.n_elem
    m.eps, m.mu = np.full(ne, eps), np.full(ne, mu)
    m.omega = omega
    bc = m.face_bc.copy()
    grp = np.zeros_like(m.face_grp)
    for e in range(ne):
        for f in (1, 3, 4):  # x1, y1, z0 sides: Robin; the others Dirichlet
            if bc[e, f] == inputs.BC_DIRICHLET:
                bc[e, f] = inputs.BC_ROBIN
    m.face_bc, m.face_grp = bc, grp
    Et = lambda x, nn: np.cross(nn, np.cross(exact(x)[0], nn))
    m.robin = [{'zinv': zinv, 'port': 'manufactured'}]
    m.dirichlet = [{'kind': 3, 'callable': Et}]

    def rg(spec, normal):
        nn = np.asarray(normal)

        def g(x):
            E, H = exact(x)
            N = np.broadcast_to(nn, E.shape)
            return np.cross(N, H) + zinv * np.cross(N, np.cross(E, N))
        return g
    monkeypatch.setattr(system, "robin_g", rg)
    sol = hanging.solve(m, source=src)
    errE = errH = nE = nH = 0.0
    for e in range(ne):
        xi, w = element.tensor_points(int(m.p[e]) + 4)
        x, J = element.trilinear(m.vert[m.elem[e]], xi)
        wd = w * np.linalg.det(J)
        E, H = system.fields_at(m, e, sol['rec'][e]['u'], xi)
        Eex, Hex = exact(x)
        errE += np.sum(wd * np.sum(np.abs(E - Eex) ** 2, 1))
        errH += np.sum(wd * np.sum(np.abs(H - Hex) ** 2, 1))
        nE += np.sum(wd * np.sum(np.abs(Eex) ** 2, 1))
        nH += np.sum(wd * np.sum(np.abs(Hex) ** 2, 1))
    assert np.sqrt(errE / nE) < 1e-11 and np.sqrt(errH / nH) < 1e-11
    assert sol['eta'].max() < 1e-10
