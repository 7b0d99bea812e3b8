"""Pins of the oracle's quadrature and bases against closed forms and exact integrals."""
import numpy as np
import pytest
import sympy as sym

from oracle import basis, element


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gauss_legendre_exactness(n):
    x, w = basis.gauss_legendre(n)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
    # degree 2n is not integrated exactly
    assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-8


def test_gauss_lobatto_closed_forms():
    assert np.allclose(basis.gauss_lobatto_nodes(2), [0, 1], atol=0)
    assert np.allclose(basis.gauss_lobatto_nodes(3), [0, 0.5, 1], atol=1e-15)
    # interior nodes of 4 points: roots of P3' -> +-1/sqrt(5)
    z = basis.gauss_lobatto_nodes(4)
    assert np.allclose(z, [0, 0.5 - 0.5 / np.sqrt(5), 0.5 + 0.5 / np.sqrt(5), 1], atol=1e-15)
    # 5 points: +-sqrt(3/7)
    z = basis.gauss_lobatto_nodes(5)
    assert np.allclose(z, [0, 0.5 - 0.5 * np.sqrt(3 / 7), 0.5, 0.5 + 0.5 * np.sqrt(3 / 7), 1], atol=1e-15)


def test_lagrange_cardinal_and_derivative():
    z = basis.gauss_lobatto_nodes(5)
    V, D = basis.lagrange_1d(z, z)
    assert np.allclose(V, np.eye(5), atol=1e-14)
    x = np.linspace(0.05, 0.95, 7)
    V, D = basis.lagrange_1d(z, x)
    assert np.allclose(V.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(D.sum(axis=1), 0.0, atol=1e-12)
    h = 1e-6
    Vp, _ = basis.lagrange_1d(z, x + h)
    Vm, _ = basis.lagrange_1d(z, x - h)
    assert np.allclose((Vp - Vm) / (2 * h), D, atol=1e-7)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_nedelec_curl_matches_finite_differences(r):
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.1, 0.9, size=(5, 3))
    val, curl = basis.nedelec_eval(r, pts)
    h = 1e-6
    grads = []
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        vp, _ = basis.nedelec_eval(r, pts + e)
        vm, _ = basis.nedelec_eval(r, pts - e)
        grads.append((vp - vm) / (2 * h))
    # curl_a = d_b v_c - d_c v_b
    fd = np.stack([grads[1][..., 2] - grads[2][..., 1],
                   grads[2][..., 0] - grads[0][..., 2],
                   grads[0][..., 1] - grads[1][..., 0]], axis=-1)
    assert np.allclose(fd, curl, atol=1e-6)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_space_dimensions(p):
    n_f, n_v, n_u, n_h = basis.dims(p)
    rt = p + 2
    assert len(basis.nedelec_index(rt)) == n_f == 3 * rt * (rt + 1) ** 2
    r = p + 1
    tr = basis.trace_functions(r)
    assert len(tr) == 12 * r * r == n_h // 2
    # edges: 12 r functions, faces: 6 * 2 r (r - 1)
    ents = [basis.trace_entity(r, *basis.nedelec_index(r)[k]) for k in tr]
    assert sum(1 for e in ents if e[0] == 'edge') == 12 * r
    assert sum(1 for e in ents if e[0] == 'face') == 12 * r * (r - 1)
    assert n_u == 6 * (p + 1) ** 3


def _exact_1d_tables(r):
    """1D integrals of Lagrange products on [0,1] to 40 digits.

    Nodes: roots of the shifted Legendre polynomial P_r(2t-1) (Gauss-Legendre)
    and 0, 1 plus the roots of P_r'(2t-1) (Gauss-Lobatto), found by sympy to 40
    digits; the Lagrange polynomials are multiplied and integrated exactly on
    their mpmath coefficients (no quadrature rule involved).
    """
    import functools
    import mpmath as mp
    mp.mp.dps = 40
    t = sym.symbols('t')
    opn = sorted(sym.Poly(sym.legendre(r, 2 * t - 1), t).nroots(n=40))
    dP = sym.Poly(sym.diff(sym.legendre(r, 2 * t - 1), t), t)
    closed = [sym.Integer(0)] + sorted(dP.nroots(n=40)) + [sym.Integer(1)]
    opn = [mp.mpf(str(sym.re(v))) for v in opn]
    closed = [mp.mpf(str(sym.re(v))) for v in closed]

    def polymul(a, b):
        out = [mp.mpf(0)] * (len(a) + len(b) - 1)
        for i, ai in enumerate(a):
            for j, bj in enumerate(b):
                out[i + j] += ai * bj
        return out

    def lag(nodes):
        out = []
        for j, zj in enumerate(nodes):
            f = [mp.mpf(1)]
            for m, zm in enumerate(nodes):
                if m != j:
                    f = polymul(f, [-zm / (zj - zm), 1 / (zj - zm)])
            out.append(f)
        return out
    deriv = lambda a: [k * a[k] for k in range(1, len(a))] or [mp.mpf(0)]
    integ01 = lambda a: sum(c / (k + 1) for k, c in enumerate(a))
    L = {0: lag(opn), 1: lag(closed)}
    tab = {}
    for ka in (0, 1):
        for kb in (0, 1):
            for da in (0, 1):
                for db in (0, 1):
                    A = np.zeros((len(L[ka]), len(L[kb])))
                    for i, fa in enumerate(L[ka]):
                        ga = deriv(fa) if da else fa
                        for j, fb in enumerate(L[kb]):
                            gb = deriv(fb) if db else fb
                            A[i, j] = float(integ01(polymul(ga, gb)))
                    tab[(ka, kb, da, db)] = A
    return tab


def _exact_reference_blocks(r):
    """Exact reference mass M, curl-curl C and curl-value X of Q^-_r Lambda^1 on [0,1]^3.

    Each basis function is f = prod_d l_{kind(d), i_d}(x_d) e_c, so every 3D
    integral is a product of exact 1D integrals.  curl(f e_c)_a = eps_{abc} d_b f.
    """
    tab = _exact_1d_tables(r)
    idx = basis.nedelec_index(r)
    n = len(idx)
    kind = lambda c, d: 0 if d == c else 1
    M = np.zeros((n, n))
    C = np.zeros((n, n))
    X = np.zeros((n, n))
    eps3 = np.zeros((3, 3, 3))
    for a, b, c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        eps3[a, b, c] = 1.0
        eps3[a, c, b] = -1.0

    def integral(ci, ii, di, cj, jj, dj):
        # prod over directions of 1D integrals; di/dj = direction differentiated (or -1)
        v = 1.0
        for d in range(3):
            v *= tab[(kind(ci, d), kind(cj, d), int(di == d), int(dj == d))][ii[d], jj[d]]
        return v
    for i, (ci, ii) in enumerate(idx):
        for j, (cj, jj) in enumerate(idx):
            if ci == cj:
                M[i, j] = integral(ci, ii, -1, cj, jj, -1)
            cc = 0.0
            xx = 0.0
            for a in range(3):
                for bi in range(3):
                    si = eps3[a, bi, ci]
                    if si == 0:
                        continue
                    for bj in range(3):
                        sj = eps3[a, bj, cj]
                        if sj != 0:
                            cc += si * sj * integral(ci, ii, bi, cj, jj, bj)
                    # X_ij = int curl(psi_i) . psi_j : component a of curl_i times psi_j (comp cj)
                    if a == cj:
                        xx += si * integral(ci, ii, bi, cj, jj, -1)
            C[i, j] = cc
            X[i, j] = xx
    return M, C, X


@pytest.mark.parametrize("h", [1.0, 0.5])
def test_gram_blocks_against_exact_integrals(h):
    """G of a cube (interior faces) = hand-derived blocks of the adjoint graph norm.

    From Eq. (test_inner_product) with real basis functions and conjugation on
    the first argument:  G_FF = C + (|w eps|^2 + a) M,  G_II = C + (|w mu|^2 + a) M,
    G_FI = i w conj(mu) X + i w eps X^T,  G_IF = G_FI^H, where on a cube of side
    h the covariant Piola map gives M = h M_ref, C = C_ref / h, X = X_ref.
    """
    p = 1
    r = p + 2
    Mr, Cr, Xr = _exact_reference_blocks(r)
    M, C, X = h * Mr, Cr / h, Xr
    omega, eps, mu, alpha = 2.3, 3.0 + 0.7j, 1.4 + 0.2j, 1.0
    Xv = np.array([[(v & 1) * h, ((v >> 1) & 1) * h, ((v >> 2) & 1) * h] for v in range(8)])
    el = element.element_matrices(Xv, p, omega, eps, mu, [None] * 6)
    nf = M.shape[0]
    G = el.G
    iw = 1j * omega
    GFF = C + (abs(omega * eps) ** 2 + alpha) * M
    GII = C + (abs(omega * mu) ** 2 + alpha) * M
    GFI = iw * np.conj(mu) * X + iw * eps * X.T
    scale = np.abs(G).max()
    assert np.abs(G[:nf, :nf] - GFF).max() / scale < 1e-13
    assert np.abs(G[nf:, nf:] - GII).max() / scale < 1e-13
    assert np.abs(G[:nf, nf:] - GFI).max() / scale < 1e-13
    assert np.abs(G[nf:, :nf] - GFI.conj().T).max() / scale < 1e-13
