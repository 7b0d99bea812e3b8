"""Pins of the oracle's mixed-order assembly (per-entity trace order = min of the neighbours)."""
import numpy as np
import pytest

from oracle import mixed, system
from paper_2609_03155_b300 import inputs


def test_uniform_order_reproduces_the_uniform_solver():
    m = inputs.waveguide(0.05, 0.03, 0.12, 1, 1, 3, 2.45e9, 1)
    a = system.solve(m)
    b = mixed.solve_mixed(m)
    assert a['n'] == b['n']
    for e in range(m.n_elem):
        assert np.allclose(b['R'][e][0] @ b['xfull'][b['R'][e][1]], a['xfull'][a['l2g'][e]], rtol=0, atol=1e-12)
    assert np.allclose(a['eta'], b['eta'], rtol=1e-9, atol=1e-15)


def test_uniform_order_reproduces_the_uniform_solver_on_jittered_lossy_mesh():
    """Non-affine elements, Dirichlet data, Robin port and lossy materials: same field as system.solve."""
    nx, ny, nz = 2, 2, 1
    vert, elem, ijk = inputs.structured_hex(0.3, 0.2, 0.1, nx, ny, nz)
    rng = np.random.default_rng(11)
    inner = (vert > 1e-12) & (vert < np.array([0.3, 0.2, 0.1]) - 1e-12)
    vert = vert + inner * rng.uniform(-0.012, 0.012, vert.shape)
    spec = {'x0': (inputs.BC_DIRICHLET, 0), 'x1': (inputs.BC_DIRICHLET, 1), 'y0': (inputs.BC_DIRICHLET, 0),
            'y1': (inputs.BC_DIRICHLET, 0), 'z0': (inputs.BC_ROBIN, 0), 'z1': (inputs.BC_ROBIN, 1)}
    bc, grp = inputs.box_boundary_tags(ijk, nx, ny, nz, spec)
    ne = elem.shape[0]
    omega = 9.0
    m = inputs.Mesh(vert=vert, elem=elem, p=np.full(ne, 1, np.int8),
                    eps=np.exp(rng.uniform(0, np.log(10), ne)) + 1j * rng.uniform(0, 3, ne),
                    mu=1.0 + 0.2 * rng.uniform(0, 1, ne) + 0.1j * rng.uniform(0, 1, ne), face_bc=bc, face_grp=grp,
                    omega=omega,
                    robin=[{'zinv': inputs.te_zinv(omega, 0.3, 0.2, 1, 0), 'port': (0.3, 0.2, 1, 0, 1.0, 1.0)},
                           {'zinv': 0.7 - 0.2j, 'port': None}],
                    dirichlet=[{'kind': inputs.DIRICHLET_ZERO, 'port': None},
                               {'kind': inputs.DIRICHLET_SIN_PI_X2, 'port': None}])
    a = system.solve(m)
    b = mixed.solve_mixed(m)
    assert a['n'] == b['n']
    for e in range(ne):
        assert np.allclose(b['rec'][e]['u'], a['rec'][e]['u'], rtol=0, atol=1e-10 * np.abs(a['rec'][e]['u']).max())
    assert np.allclose(a['eta'], b['eta'], rtol=1e-8, atol=1e-15)


@pytest.mark.parametrize("orders", [(1, 2), (2, 1, 3, 1)])
def test_manufactured_solution_exact_with_mixed_orders(orders, monkeypatch):
    """A polynomial solution inside every element's spaces is reproduced exactly across order jumps."""
    rng = np.random.default_rng(4)
    omega, eps, mu, zinv = 2.0, 1.5 + 0.2j, 1.2 + 0j, 0.6 + 0.1j
    Ex = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    E0 = rng.normal(size=3) + 1j * rng.normal(size=3)
    curlE = np.array([Ex[2, 1] - Ex[1, 2], Ex[0, 2] - Ex[2, 0], Ex[1, 0] - Ex[0, 1]])
    H0 = curlE / (1j * omega * mu)
    exact = lambda x: (E0[None, :] + x @ Ex.T, np.broadcast_to(H0, (len(x), 3)).copy())
    src = lambda x: 1j * omega * eps * exact(x)[0]
    n = len(orders)
    nx, ny, nz = (2, 1, 1) if n == 2 else (2, 2, 1)
    vert, elem, ijk = inputs.structured_hex(1.0, 0.8, 0.6, nx, ny, nz)
    spec = {'x0': (inputs.BC_DIRICHLET, 0), 'x1': (inputs.BC_ROBIN, 0), 'y0': (inputs.BC_DIRICHLET, 0),
            'y1': (inputs.BC_ROBIN, 0), 'z0': (inputs.BC_ROBIN, 0), 'z1': (inputs.BC_DIRICHLET, 0)}
    bc, grp = inputs.box_boundary_tags(ijk, nx, ny, nz, spec)
    ne = elem.shape[0]
    Et = lambda x, nn: np.cross(nn, np.cross(exact(x)[0], nn))
    m = inputs.Mesh(vert=vert, elem=elem, p=np.array(orders, np.int8), eps=np.full(ne, eps), mu=np.full(ne, mu),
                    face_bc=bc, face_grp=grp, omega=omega, robin=[{'zinv': zinv, 'port': 'manufactured'}],
                    dirichlet=[{'kind': 3, 'callable': Et}])

    def rg(spec, normal):
        nn = np.asarray(normal)

        def g(x):
            E, H = exact(x)
            N = np.broadcast_to(nn, E.shape)
            return np.cross(N, H) + zinv * np.cross(N, np.cross(E, N))
        return g
    monkeypatch.setattr(system, "robin_g", rg)
    sol = mixed.solve_mixed(m, source=src)
    eE, eH = system.l2_field_error(m, sol, exact) if len(set(orders)) == 1 else _l2_mixed(m, sol, exact)
    assert eE < 1e-11 and eH < 1e-11
    assert sol['eta'].max() < 1e-10


def _l2_mixed(mesh, sol, exact):
    from oracle import element
    errE = errH = nE = nH = 0.0
    for e in range(mesh.n_elem):
        p = int(mesh.p[e])
        xi, w = element.tensor_points(p + 4)
        X = mesh.vert[mesh.elem[e]]
        x, J = element.trilinear(X, xi)
        wd = w * np.linalg.det(J)
        E, H = system.fields_at(mesh, e, sol['rec'][e]['u'], xi)
        Ex, Hx = exact(x)
        errE += np.sum(wd * np.sum(np.abs(E - Ex) ** 2, 1))
        errH += np.sum(wd * np.sum(np.abs(H - Hx) ** 2, 1))
        nE += np.sum(wd * np.sum(np.abs(Ex) ** 2, 1))
        nH += np.sum(wd * np.sum(np.abs(Hx) ** 2, 1))
    return np.sqrt(errE / nE), np.sqrt(errH / nH)
