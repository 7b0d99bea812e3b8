"""Absorbed power and its adjoint gradient w.r.t. per-element permittivity (test infrastructure only).

The paper has no adjoint; this is the reactor-optimisation use of the solver.
Absorbed power of an obstacle (the electric-loss term of Q_em in Sec. 3.2,
dimensionless): P = 1/2 omega sum_{K in obstacle} Im(eps_K) int_K |E|^2.

DPG (Sec. 2.1) is the minimiser of J(w) = sum_K ||l_K - B_K w_K||^2_{G_K^{-1}}
over w = (u, u-hat), with normal equations A w = f, A = sum B_K^H G_K^{-1} B_K,
f = sum B_K^H G_K^{-1} l_K (B_K = [B, B-hat]).  For a real parameter s of
element K (s = Re eps_K or Im eps_K), with g = dP/d(conj w) and A lambda = g:
    dP/ds = dP/ds|explicit + 2 Re( (B' lambda)^H psi - mu^H G' psi - mu^H B' w ),
    psi = G^{-1}(l - B_K w_K),  mu = G^{-1} B_K lambda_K,
where G' = dG_K/ds, B' = dB_K/ds follow from differentiating the test-norm
integrand of Eq. (test_inner_product) and the term (F, i w eps E) of Eq.
(bilinear_form).  G depends on |eps|^2 and conj(eps): it is not holomorphic,
so the two real derivatives are formed separately.  The adjoint system is
condensed exactly like the forward one (Eq. linear_system).
"""
import numpy as np
import scipy.linalg as sla

from . import basis, element, system


def e_mass(X, p):
    """L2 mass of one Cartesian component of the interior trial space on element X."""
    nq1 = p + 3
    xi, w = element.tensor_points(nq1)
    _, J = element.trilinear(X, xi)
    det = np.linalg.det(J)
    L = basis.lagrange3_eval(p, xi)
    return (L * (w * det)[:, None]).T @ L


def absorbed_power(mesh, sol, mask):
    """P = 1/2 omega sum_{K in mask} Im eps_K u_E^H M_E u_E  and per-element g_u = dP/d conj(u)."""
    p = int(mesh.p[0])
    nL = (p + 1) ** 3
    P = 0.0
    g = {}
    for e in np.where(mask)[0]:
        Me = e_mass(mesh.vert[mesh.elem[e]], p)
        uE = sol['rec'][e]['u'][:3 * nL]
        ME = np.kron(np.eye(3), Me)
        w2 = 0.5 * mesh.omega * mesh.eps[e].imag
        P += w2 * np.real(np.vdot(uE, ME @ uE))
        gu = np.zeros(6 * nL, dtype=complex)
        gu[:3 * nL] = w2 * (ME @ uE)
        g[e] = gu
    return P, g


def element_derivatives(X, p, omega, eps, mu, dp=1, alpha=1.0):
    """dG/dRe(eps), dG/dIm(eps), dB/dRe(eps), dB/dIm(eps) for one element (Robin terms do not depend on eps).

    The test-norm integrand of the F-type test functions contains
    curl I - i w conj(eps) F; d conj(eps)/d Re eps = 1, d conj(eps)/d Im eps = -i.
    The bilinear form contains (F, i w eps E).
    """
    rt = p + 1 + dp
    nq1 = p + dp + 2
    n_f, n_v, n_u, n_h = basis.dims(p, dp)
    nL = (p + 1) ** 3
    xi, w = element.tensor_points(nq1)
    _, J = element.trilinear(X, xi)
    vref, cref = basis.nedelec_eval(rt, xi)
    psi, cpsi, det = element.piola(J, vref, cref)
    wdet = w * det
    nq = len(w)
    iw = 1j * omega
    zero = np.zeros_like(psi)
    A1 = np.concatenate([cpsi, iw * np.conj(mu) * psi], axis=1)
    A2 = np.concatenate([-iw * np.conj(eps) * psi, cpsi], axis=1)
    A3 = np.concatenate([psi, zero], axis=1)
    A4 = np.concatenate([zero, psi], axis=1)
    T = np.concatenate([A1, A2, np.sqrt(alpha) * A3, np.sqrt(alpha) * A4], axis=2)
    Tw = (np.sqrt(wdet)[:, None, None] * T).transpose(0, 2, 1).reshape(nq * 12, n_v)
    L = basis.lagrange3_eval(p, xi)
    phiE = np.zeros((nq, 3 * nL, 3))
    for d in range(3):
        phiE[:, d * nL:(d + 1) * nL, d] = L
    Pm = np.einsum('q,qia,qja->ij', wdet, psi, phiE)
    out = {}
    for name, dconj_eps, deps in (('re', 1.0, 1.0), ('im', -1j, 1j)):
        dA2 = np.concatenate([-iw * dconj_eps * psi, zero], axis=1)
        dT = np.concatenate([np.zeros_like(A1), dA2, np.zeros_like(A3), np.zeros_like(A4)], axis=2)
        dTw = (np.sqrt(wdet)[:, None, None] * dT).transpose(0, 2, 1).reshape(nq * 12, n_v)
        dG = dTw.conj().T @ Tw + Tw.conj().T @ dTw
        dB = np.zeros((n_v, n_u + n_h), dtype=complex)
        dB[:n_f, :3 * nL] = iw * deps * Pm
        out['G_' + name] = dG
        out['B_' + name] = dB
    return out


def gradient(mesh, sol, mask):
    """P and (dP/dRe eps_K, dP/dIm eps_K) for every element, by the adjoint route."""
    p = int(mesh.p[0])
    nL = (p + 1) ** 3
    P, g = absorbed_power(mesh, sol, mask)
    ne = mesh.elem.shape[0]
    free, l2g = sol['free'], sol['l2g']
    n = sol['n']
    # condensed adjoint right-hand side: g_h - M2^H M1^{-1} g_u with g_h = 0
    rhs = np.zeros(n, dtype=complex)
    for e, gu in g.items():
        c = sol['conds'][e]
        gc = -c['M2'].conj().T @ np.linalg.solve(c['M1'], gu)
        fr = free[l2g[e]]
        m = fr >= 0
        np.add.at(rhs, fr[m], gc[m])
    A = sol['A']
    lam_free = np.linalg.solve(A.toarray(), rhs) if n <= 6000 else \
        __import__('scipy.sparse.linalg', fromlist=['spsolve']).spsolve(A.tocsc(), rhs)
    lam_full = np.zeros(free.shape[0], dtype=complex)
    lam_full[free >= 0] = lam_free[free[free >= 0]]
    dre = np.zeros(ne)
    dim = np.zeros(ne)
    for e in range(ne):
        el, c = sol['elements'][e], sol['conds'][e]
        lam_h = lam_full[l2g[e]]
        gu = g.get(e, np.zeros(6 * nL, dtype=complex))
        lam_u = np.linalg.solve(c['M1'], gu - c['M2'] @ lam_h)
        lam = np.concatenate([lam_u, lam_h])
        w = np.concatenate([sol['rec'][e]['u'], sol['xfull'][l2g[e]]])
        BK = np.concatenate([el.B, el.Bh], axis=1)
        psi = sla.cho_solve((c['L'], True), el.l - BK @ w)
        mu_ = sla.cho_solve((c['L'], True), BK @ lam)
        der = element_derivatives(mesh.vert[mesh.elem[e]], p, mesh.omega, complex(mesh.eps[e]),
                                  complex(mesh.mu[e]))
        for name, out in (('re', dre), ('im', dim)):
            dG, dB = der['G_' + name], der['B_' + name]
            val = 2.0 * np.real(np.vdot(dB @ lam, psi) - np.vdot(mu_, dG @ psi) - np.vdot(mu_, dB @ w))
            out[e] = val
        if mask[e]:
            Me = e_mass(mesh.vert[mesh.elem[e]], p)
            uE = sol['rec'][e]['u'][:3 * nL]
            dim[e] += 0.5 * mesh.omega * np.real(np.vdot(uE, np.kron(np.eye(3), Me) @ uE))
    return P, dre, dim


def power_of(mesh, mask):
    """P at the direct-solve DPG solution (for finite differences)."""
    sol = system.solve(mesh)
    return absorbed_power(mesh, sol, mask)[0]


def fd_gradient(mesh, mask, elems, h=1e-6):
    """Central finite differences of P w.r.t. Re eps and Im eps of the given elements."""
    out = []
    for e in elems:
        row = []
        for part in (1.0, 1j):
            eps0 = mesh.eps.copy()
            mesh.eps = eps0.copy()
            mesh.eps[e] += part * h
            Pp = power_of(mesh, mask)
            mesh.eps = eps0.copy()
            mesh.eps[e] -= part * h
            Pm = power_of(mesh, mask)
            mesh.eps = eps0
            row.append((Pp - Pm) / (2 * h))
        out.append(row)
    return np.array(out)
