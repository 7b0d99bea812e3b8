"""Pins of the oracle's element matrices, condensation, recovery and estimator."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import basis, element, system
from paper_2609_03155_b300 import inputs


def _jittered_pair(seed=5):
    """Two hexes sharing the face x = 1, interior vertices jittered."""
    vert, elem, ijk = inputs.structured_hex(2.0, 1.0, 1.0, 2, 1, 1)
    rng = np.random.default_rng(seed)
    vert = vert + rng.uniform(-0.12, 0.12, size=vert.shape)
    return vert, elem


def _robin_faces(zinv, g):
    return [{'robin': (zinv, g)}] + [None] * 5


def test_hermitian_positive_definite_and_scaling():
    vert, elem = _jittered_pair()
    g = lambda x: np.stack([0 * x[:, 0], np.sin(x[:, 1]) + 0j, 1j * x[:, 2]], axis=1)
    el = element.element_matrices(vert[elem[0]], 2, 4.0, 2.0 + 0.3j, 1.0 + 0.1j, _robin_faces(0.7 + 0.2j, g))
    G = el.G
    assert np.linalg.norm(G - G.conj().T) / np.linalg.norm(G) < 1e-15
    assert np.linalg.eigvalsh(G).min() > 0
    c = element.condense(el)
    A = c['A_full']
    assert np.linalg.norm(A - A.conj().T) / np.linalg.norm(A) < 1e-14
    ev = np.linalg.eigvalsh((c['S'] + c['S'].conj().T) / 2)
    assert ev.min() > -1e-12 * ev.max()          # S_K is positive semi-definite locally
    assert np.linalg.eigvalsh(c['M1']).min() > 0  # B has full column rank


def test_piola_tangential_continuity_across_shared_face():
    """Trace functions keyed to the same global DoF agree tangentially on the shared face."""
    vert, elem = _jittered_pair()
    p, r = 1, 2
    mesh = inputs.Mesh(vert=vert, elem=elem, p=np.array([p, p], dtype=np.int8), eps=np.ones(2, complex),
                       mu=np.ones(2, complex), face_bc=np.zeros((2, 6), np.int8),
                       face_grp=np.zeros((2, 6), np.int16), omega=1.0)
    num = system.number_traces(mesh)
    tsel = basis.trace_functions(r)
    g = basis.gauss_legendre(4)[0]
    # element 0 face x=1 (f=1) meets element 1 face x=0 (f=0); same (y, z) parameters
    uv = np.array([[a, b] for a in g for b in g])
    pts0 = np.column_stack([np.ones(len(uv)), uv])
    pts1 = np.column_stack([np.zeros(len(uv)), uv])
    x0, J0 = element.trilinear(vert[elem[0]], pts0)
    x1, J1 = element.trilinear(vert[elem[1]], pts1)
    assert np.allclose(x0, x1, atol=1e-14)
    v0r, c0r = basis.nedelec_eval(r, pts0)
    v1r, c1r = basis.nedelec_eval(r, pts1)
    ph0, _, _ = element.piola(J0, v0r[:, tsel], c0r[:, tsel])
    ph1, _, _ = element.piola(J1, v1r[:, tsel], c1r[:, tsel])
    N = np.cross(J0[:, :, 1], J0[:, :, 2])
    n = N / np.linalg.norm(N, axis=1)[:, None]
    shared = 0
    for k0 in range(len(tsel)):
        gk = num.loc2glob[0, k0]
        k1s = np.where(num.loc2glob[1] == gk)[0]
        t0 = np.cross(n, ph0[:, k0])
        if not k1s.size:
            continue
        shared += 1
        t1 = np.cross(n, ph1[:, k1s[0]])
        assert np.abs(t0 - t1).max() < 1e-13
    assert shared == 4 * r + 2 * r * (r - 1)


def _manufactured(omega, eps, mu, seed=1):
    """Linear E, constant H = curl E / (i w mu) and source J = i w eps E solve Eq. (maxwell_dimensionless)."""
    rng = np.random.default_rng(seed)
    Ex = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    E0 = rng.normal(size=3) + 1j * rng.normal(size=3)
    curlE = np.array([Ex[2, 1] - Ex[1, 2], Ex[0, 2] - Ex[2, 0], Ex[1, 0] - Ex[0, 1]])
    H0 = curlE / (1j * omega * mu)

    def exact(x):
        E = E0[None, :] + x @ Ex.T
        return E, np.broadcast_to(H0, E.shape).copy()
    return exact, (lambda x: 1j * omega * eps * exact(x)[0])


@pytest.mark.parametrize("bcmode", ["robin", "dirichlet", "mixed"])
def test_manufactured_polynomial_solution_is_exact(bcmode, monkeypatch):
    """DPG is a minimum-residual method: a solution inside the discrete spaces is reproduced exactly."""
    omega, eps, mu, zinv = 3.0, 2.0 + 0.5j, 1.5 + 0j, 0.8 + 0.3j
    exact, src = _manufactured(omega, eps, mu)
    nx, ny, nz = (2, 1, 2) if bcmode == "mixed" else (2, 1, 1)
    vert, elem, ijk = inputs.structured_hex(1.0, 0.7, 0.5, nx, ny, nz)
    vert = vert + np.random.default_rng(9).uniform(-0.03, 0.03, vert.shape) * (
        (vert > 1e-9) & (vert < np.array([1.0, 0.7, 0.5]) - 1e-9))
    if bcmode == "robin":
        spec = {k: (inputs.BC_ROBIN, 0) for k in ('x0', 'x1', 'y0', 'y1', 'z0', 'z1')}
    elif bcmode == "dirichlet":
        spec = {k: (inputs.BC_DIRICHLET, 0) for k in ('x0', 'x1', 'y0', 'y1', 'z0', 'z1')}
    else:
        spec = {k: (inputs.BC_DIRICHLET, 0) for k in ('x0', 'x1', 'y0', 'y1')}
        spec.update({'z0': (inputs.BC_ROBIN, 0), 'z1': (inputs.BC_ROBIN, 0)})
    bc, grp = inputs.box_boundary_tags(ijk, nx, ny, nz, spec)
    ne = elem.shape[0]
    Et = lambda x, n: np.cross(n, np.cross(exact(x)[0], n))
    m = inputs.Mesh(vert=vert, elem=elem, p=np.full(ne, 1, np.int8), eps=np.full(ne, eps),
                    mu=np.full(ne, mu), face_bc=bc, face_grp=grp, omega=omega,
                    robin=[{'zinv': zinv, 'port': 'manufactured'}],
                    dirichlet=[{'kind': 3, 'callable': Et}])

    def rg(spec, normal):
        nn = np.asarray(normal)

        def g(x):
            E, H = exact(x)
            N = np.broadcast_to(nn, E.shape)
            return np.cross(N, H) + zinv * np.cross(N, np.cross(E, N))
        return g
    monkeypatch.setattr(system, "robin_g", rg)
    sol = system.solve(m, source=src)
    eE, eH = system.l2_field_error(m, sol, exact)
    assert eE < 1e-12 and eH < 1e-12
    assert sol['eta'].max() < 1e-11


def _tiny_mesh(ne_x=2):
    m = inputs.waveguide(0.05, 0.03, 0.04 * ne_x, 1, 1, ne_x, 2.45e9, 1)
    return m


def test_condensation_equals_brute_force_saddle_point():
    """Two-stage condensation (Eq. linear_system) = dense solve of the full block system of Sec. 2.3."""
    m = _tiny_mesh(2)
    sol = system.solve(m)
    ne = m.elem.shape[0]
    els = sol['elements']
    n_f, n_v, n_u, n_h = els[0].sizes
    free, xfix, l2g = sol['free'], sol['xfix'], sol['l2g']
    nfree = sol['n']
    N = ne * n_v + ne * n_u + nfree
    K = np.zeros((N, N), dtype=complex)
    rhs = np.zeros(N, dtype=complex)
    for e, el in enumerate(els):
        ps = slice(e * n_v, (e + 1) * n_v)
        us = slice(ne * n_v + e * n_u, ne * n_v + (e + 1) * n_u)
        K[ps, ps] = el.G
        K[ps, us] = el.B
        K[us, ps] = el.B.conj().T
        fr = free[l2g[e]]
        msk = fr >= 0
        cols = ne * n_v + ne * n_u + fr[msk]
        K[ps, cols] += el.Bh[:, msk]
        K[cols, ps] += el.Bh[:, msk].conj().T
        rhs[ps] = el.l - el.Bh @ xfix[l2g[e]]
    z = np.linalg.solve(K, rhs)
    xh = z[ne * n_v + ne * n_u:]
    assert np.linalg.norm(xh - sol['x']) / np.linalg.norm(sol['x']) < 1e-9
    for e in range(ne):
        Psi = z[e * n_v:(e + 1) * n_v]
        u = z[ne * n_v + e * n_u: ne * n_v + (e + 1) * n_u]
        assert np.linalg.norm(u - sol['rec'][e]['u']) / np.linalg.norm(u) < 1e-9
        assert np.linalg.norm(Psi - sol['rec'][e]['Psi']) / np.linalg.norm(Psi) < 1e-7


def test_estimator_routes_agree_and_optimality():
    """eta via Cholesky = eigen (dual norm) = sqrt(Psi^H G Psi); the trace solution minimises sum eta^2."""
    m = _tiny_mesh(3)
    sol = system.solve(m)
    for rc in sol['rec']:
        assert abs(rc['eta'] - rc['eta_eig']) <= 1e-10 * rc['eta']
        assert abs(rc['eta'] - rc['eta_psi']) <= 1e-9 * rc['eta']
    # J(uhat) = sum_K min_u ||l - B u - Bh uhat||^2_{G^{-1}} is quadratic with Hessian S
    def J(xfree):
        xf = sol['xfix'].copy()
        xf[sol['free'] >= 0] = xfree[sol['free'][sol['free'] >= 0]]
        tot = 0.0
        for e, el in enumerate(sol['elements']):
            rc = element.recover(el, sol['conds'][e], xf[sol['l2g'][e]])
            tot += rc['eta'] ** 2
        return tot
    x = sol['x']
    J0 = J(x)
    assert abs(J0 - np.sum(sol['eta'] ** 2)) < 1e-12 * max(J0, 1e-30) + 1e-24
    rng = np.random.default_rng(2)
    A = sol['A'].toarray()
    for _ in range(2):
        d = 1e-3 * (rng.normal(size=x.size) + 1j * rng.normal(size=x.size))
        inc = J(x + d) - J0
        quad = np.real(np.vdot(d, A @ d))
        assert inc > 0
        assert abs(inc - quad) < 1e-6 * quad


def test_complex_cg_equals_real_embedded_cg():
    """Complex Hermitian CG and CG on the real embedding [[Re, -Im], [Im, Re]] give the same iterates."""
    m = _tiny_mesh(2)
    sol = system.solve(m)
    A = sol['A'].toarray()
    b = sol['b']
    xc, infc = system.cg(A, b, rtol=1e-10)
    Ar = np.block([[A.real, -A.imag], [A.imag, A.real]])
    br = np.concatenate([b.real, b.imag])
    xr, infr = system.cg(Ar, br, rtol=1e-10)
    assert infc['iters'] == infr['iters']
    assert np.linalg.norm(xc - (xr[:b.size] + 1j * xr[b.size:])) <= 1e-10 * np.linalg.norm(xc)
    assert np.linalg.norm(xc - sol['x']) / np.linalg.norm(sol['x']) < 1e-7
