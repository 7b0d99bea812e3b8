"""Element-local DPG matrices G_K, B_K, B-hat_K, l_K by quadrature (test infrastructure only).

Follows Sec. 2.2-2.3 of the paper literally, one term at a time:

* Eq. (test_inner_product): G_ij = (psi_i, psi_j)_V, the adjoint graph norm
  with alpha, including the Gamma_R boundary term.
* Eq. (bilinear_form): B_ij = b_h(psi_i, phi_j) on the interior trial space,
  and the Robin term -<F, Z^{-1} n x (E-hat x n)>_{Gamma_R} on the trace E-hat.
* Eq. (trace_pairing): B-hat_ij = <psi_i, phi-hat_j>_h.
* Eq. (linear_form): l_i = (F, J) - <F, g>_{Gamma_R}.

All forms are conjugate-linear in the first argument (Sec. 2.1); the basis
functions are real, the coefficients complex.  Test functions are ordered
[F-block (n_f), I-block (n_f)], interior trial [E (3 (p+1)^3), H (3 (p+1)^3)]
(component-major, tensor Lagrange inside), trace [E-hat (12 r^2), H-hat (12 r^2)]
in the order of ``basis.trace_functions``.

Geometry: trilinear hexahedron, vertex v = i + 2 j + 4 k at reference corner
(i, j, k).  Nedelec functions map by the covariant Piola transform
psi = J^{-T} psi_ref, curl psi = J curl_ref psi_ref / det J; faces use Nanson's
formula n dS = det J J^{-T} N_ref dS_ref.  Quadrature: Gauss-Legendre with
p + dp + 2 points per direction in the volume and on each face (our reading;
exact for affine elements).
"""
import numpy as np
import scipy.linalg as sla

from . import basis


def trilinear(X, xi):
    """Physical points x (N,3) and Jacobians J (N,3,3), J[a,b] = dx_a/dxi_b."""
    xi = np.asarray(xi, dtype=float)
    N = xi.shape[0]
    x = np.zeros((N, 3))
    J = np.zeros((N, 3, 3))
    for v in range(8):
        bits = [(v >> a) & 1 for a in range(3)]
        f = [xi[:, a] if bits[a] else 1.0 - xi[:, a] for a in range(3)]
        df = [np.ones(N) if bits[a] else -np.ones(N) for a in range(3)]
        shape = f[0] * f[1] * f[2]
        x += shape[:, None] * X[v][None, :]
        for b in range(3):
            g = df[b] * f[(b + 1) % 3] * f[(b + 2) % 3]
            J[:, :, b] += g[:, None] * X[v][None, :]
    return x, J


def tensor_points(n, dimsel=(0, 1, 2), fixed=None):
    """Tensor Gauss-Legendre points on the cube (fixed=None) or on a face.

    For a face, ``fixed`` = (d, s) puts xi_d = s and spans the other two axes.
    Returns (pts (N,3), weights (N,)).
    """
    g, w = basis.gauss_legendre(n)
    if fixed is None:
        pts, wts = [], []
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    pts.append([g[i], g[j], g[k]])
                    wts.append(w[i] * w[j] * w[k])
        return np.array(pts), np.array(wts)
    d, s = fixed
    a, b = [e for e in range(3) if e != d]
    pts, wts = [], []
    for j in range(n):
        for i in range(n):
            pt = [0.0, 0.0, 0.0]
            pt[d] = float(s)
            pt[a] = g[i]
            pt[b] = g[j]
            pts.append(pt)
            wts.append(w[i] * w[j])
    return np.array(pts), np.array(wts)


def piola(J, val_ref, curl_ref):
    """Covariant Piola map of reference values/curls at points with Jacobians J."""
    Jinv = np.linalg.inv(J)
    det = np.linalg.det(J)
    val = np.einsum('qba,qkb->qka', Jinv, val_ref)
    curl = np.einsum('qab,qkb->qka', J, curl_ref) / det[:, None, None]
    return val, curl, det


class ElementData:
    """Per-element matrices; attributes G, B, Bh, l and the sizes."""


def element_matrices(X, p, omega, eps, mu, faces, dp=1, alpha=1.0, source=None):
    """Compute G_K, B_K, B-hat_K, l_K for one hexahedron.

    X: (8,3) vertices.  faces: list of 6 entries (face f = 2 d + s, normal d,
    side s), each None or a dict {'robin': (zinv, g)} with zinv = Z_s^{-1}
    (complex) and g a callable x (N,3) -> (N,3) complex or None for g = 0.
    source: callable x -> J (N,3) complex or None.
    """
    X = np.asarray(X, dtype=float)
    r = p + 1
    rt = p + 1 + dp
    nq1 = p + dp + 2
    n_f, n_v, n_u, n_h = basis.dims(p, dp)
    nL = (p + 1) ** 3
    nt = n_h // 2
    iw = 1j * omega
    eb = np.conj(eps)
    mb = np.conj(mu)

    # ---- volume terms -----------------------------------------------------
    xi, w = tensor_points(nq1)
    xq, J = trilinear(X, xi)
    vref, cref = basis.nedelec_eval(rt, xi)
    psi, cpsi, det = piola(J, vref, cref)
    if np.any(det <= 0):
        raise ValueError("element with non-positive Jacobian")
    wdet = w * det
    nq = len(w)

    # test-norm integrand of Eq. (test_inner_product): for each test function the
    # four fields curl F + i w mu* I, curl I - i w eps* F, F, I  (conj-linear first slot)
    zero = np.zeros_like(psi)
    A1 = np.concatenate([cpsi, iw * mb * psi], axis=1)          # curl F + i w mu^* I
    A2 = np.concatenate([-iw * eb * psi, cpsi], axis=1)         # curl I - i w eps^* F
    A3 = np.concatenate([psi, zero], axis=1)                    # F
    A4 = np.concatenate([zero, psi], axis=1)                    # I
    T = np.concatenate([A1, A2, np.sqrt(alpha) * A3, np.sqrt(alpha) * A4], axis=2)
    Tw = (np.sqrt(wdet)[:, None, None] * T).transpose(0, 2, 1).reshape(nq * 12, n_v)
    G = Tw.conj().T @ Tw

    # interior trial functions: tensor Lagrange times a Cartesian unit vector
    L = basis.lagrange3_eval(p, xi)  # (nq, nL)
    phiE = np.zeros((nq, 3 * nL, 3))
    for d in range(3):
        phiE[:, d * nL:(d + 1) * nL, d] = L
    # Eq. (bilinear_form), interior part, written term by term
    F, cF = psi, cpsi
    I, cI = psi, cpsi
    B = np.zeros((n_v, n_u), dtype=complex)
    # rows F (0:n_f): (F, i w eps E) and (curl F, H)
    B[:n_f, :3 * nL] = np.einsum('q,qia,qja->ij', wdet, F.conj(), iw * eps * phiE)
    B[:n_f, 3 * nL:] = np.einsum('q,qia,qja->ij', wdet, cF.conj(), phiE)
    # rows I (n_f:): (curl I, E) and -(I, i w mu H)
    B[n_f:, :3 * nL] = np.einsum('q,qia,qja->ij', wdet, cI.conj(), phiE)
    B[n_f:, 3 * nL:] = -np.einsum('q,qia,qja->ij', wdet, I.conj(), iw * mu * phiE)

    l = np.zeros(n_v, dtype=complex)
    if source is not None:
        Jq = source(xq)
        l[:n_f] += np.einsum('q,qia,qa->i', wdet, F.conj(), Jq)

    # ---- face terms -------------------------------------------------------
    Bh = np.zeros((n_v, n_h), dtype=complex)
    tsel = basis.trace_functions(r)
    for f in range(6):
        d, s = f // 2, f % 2
        xi_f, wf = tensor_points(nq1, fixed=(d, s))
        xf, Jf = trilinear(X, xi_f)
        vr, cr = basis.nedelec_eval(rt, xi_f)
        psi_f, _, detf = piola(Jf, vr, cr)
        hr, hc = basis.nedelec_eval(r, xi_f)
        hr = hr[:, tsel, :]
        hc = hc[:, tsel, :]
        phih, _, _ = piola(Jf, hr, hc)
        Nref = np.zeros(3)
        Nref[d] = 2.0 * s - 1.0
        Jinv = np.linalg.inv(Jf)
        nvec = detf[:, None] * np.einsum('qba,b->qa', Jinv, Nref)   # det J J^{-T} N_ref
        dS = np.linalg.norm(nvec, axis=1)
        n = nvec / dS[:, None]
        wS = wf * dS
        n_x_phih = np.cross(n[:, None, :], phih)                       # n x E-hat
        robin = faces[f] is not None and 'robin' in faces[f]
        # Eq. (trace_pairing): <I, n x E-hat> on every face of dK
        Bh[n_f:, :nt] += np.einsum('q,qia,qja->ij', wS, psi_f.conj(), n_x_phih)
        if not robin:
            # <F, n x H-hat> on dK minus Gamma_R
            Bh[:n_f, nt:] += np.einsum('q,qia,qja->ij', wS, psi_f.conj(), n_x_phih)
        else:
            zinv, g = faces[f]['robin']
            # tangential part n x (E-hat x n)
            phih_t = np.cross(n[:, None, :], np.cross(phih, n[:, None, :]))
            # Eq. (bilinear_form): - <F, Z^{-1} n x (E-hat x n)>_{Gamma_R}
            Bh[:n_f, :nt] += -zinv * np.einsum('q,qia,qja->ij', wS, psi_f.conj(), phih_t)
            # Eq. (test_inner_product) boundary term: n x I + (Z^*)^{-1} n x (F x n)
            psi_t = np.cross(n[:, None, :], np.cross(psi_f, n[:, None, :]))
            n_x_psi = np.cross(n[:, None, :], psi_f)
            tau = np.concatenate([np.conj(zinv) * psi_t, n_x_psi], axis=1)   # (nq, n_v, 3)
            tw = (np.sqrt(wS)[:, None, None] * tau).transpose(0, 2, 1).reshape(-1, n_v)
            G += tw.conj().T @ tw
            # Eq. (linear_form): - <F, g>_{Gamma_R}
            if g is not None:
                gq = g(xf)
                l[:n_f] += -np.einsum('q,qia,qa->i', wS, psi_f.conj(), gq)
    out = ElementData()
    out.G, out.B, out.Bh, out.l = G, B, Bh, l
    out.sizes = (n_f, n_v, n_u, n_h)
    return out


def condense(el):
    """The two static condensations of Sec. 2.3, done literally.

    M1 = B^H G^{-1} B, M2 = B^H G^{-1} B-hat, M3 = B-hat^H G^{-1} B-hat,
    M4 = B^H G^{-1}, M5 = B-hat^H G^{-1};
    S = M3 - M2^H M1^{-1} M2,  s = (M5 - M2^H M1^{-1} M4) l   (Eq. linear_system).
    G^{-1} is applied through the Cholesky factor G = L L^H (G is Hermitian
    positive definite), as G^{-1} = L^{-H} L^{-1}: with W = L^{-1} [B, B-hat]
    the blocks are Gram products of W (forward-stable; the explicit inverse
    loses about a factor ten more digits for kappa(G) ~ 1e7).
    Returns M1..M5 (M4, M5 applied to l), S, s and A_full = [B B-hat]^H G^{-1} [B B-hat].
    """
    G, B, Bh, l = el.G, el.B, el.Bh, el.l
    L = np.linalg.cholesky(G)
    Wb = sla.solve_triangular(L, B, lower=True)
    Wh = sla.solve_triangular(L, Bh, lower=True)
    wl = sla.solve_triangular(L, l, lower=True)
    M1 = Wb.conj().T @ Wb
    M2 = Wb.conj().T @ Wh
    M3 = Wh.conj().T @ Wh
    M4l = Wb.conj().T @ wl
    M5l = Wh.conj().T @ wl
    M1inv_M2 = np.linalg.solve(M1, M2)
    M1inv_M4l = np.linalg.solve(M1, M4l)
    S = M3 - M2.conj().T @ M1inv_M2
    s = M5l - M2.conj().T @ M1inv_M4l
    A_full = np.block([[M1, M2], [M2.conj().T, M3]])
    return dict(M1=M1, M2=M2, M3=M3, M4l=M4l, M5l=M5l, S=S, s=s, A_full=A_full, L=L)


def recover(el, cond, uhat_K):
    """Local recovery and estimator of Sec. 2.3 for one element.

    u = M1^{-1}(M4 l - M2 u-hat);  Psi = G^{-1}(l - B u - B-hat u-hat)
    (sign of the block system); eta = sqrt(Psi^H G Psi) computed two ways:
    through the Cholesky factor (||L^{-1} r||) and through the eigen-
    decomposition of G (||G^{-1/2} r||, the dual-norm definition).
    """
    G, B, Bh, l = el.G, el.B, el.Bh, el.l
    u = np.linalg.solve(cond['M1'], cond['M4l'] - cond['M2'] @ uhat_K)
    res = l - B @ u - Bh @ uhat_K
    Psi = np.linalg.solve(G, res)
    eta_psi = np.sqrt(max(np.real(Psi.conj() @ G @ Psi), 0.0))
    y = sla.solve_triangular(cond['L'], res, lower=True)
    eta_chol = np.linalg.norm(y)
    lam, V = np.linalg.eigh(G)
    z = (V.conj().T @ res) / np.sqrt(lam)
    eta_eig = np.linalg.norm(z)
    return dict(u=u, Psi=Psi, res=res, eta=eta_chol, eta_psi=eta_psi, eta_eig=eta_eig)
