"""Electromagnetic power from a DPG solution (test infrastructure only).

Sec. 3.2: the dissipated power density is the negative divergence of the
time-averaged Poynting vector,
    Q_em = 1/2 omega eps_im |E|^2 + 1/2 omega mu_im |H|^2
in the dimensionless form of the solver (the conductivity is part of the
imaginary permittivity, Sec. 2.2), and the reference field E0 follows from a
prescribed input power through the port flux of the dimensionless solution,
    P_input = 1/2 E0^2 / Z0 * int_A Re(E x conj(H)) . n dA      (Eq. power_scaling).
Fields are the interior (L^2) fields u_K of each element, evaluated with the
Gauss-Legendre rule of the element pass (p + 3 points per direction); n is
the outward normal of the element face (Nanson: n dA = det J J^{-T} N_ref dxi).
"""
import numpy as np

from . import element, system

Z0 = 376.730313412  # impedance of free space, Ohm (mu0 c0)


def element_power(mesh, us, nq=None):
    """int_K Q_em dV for every element from its interior coefficients us[e]."""
    out = np.zeros(mesh.elem.shape[0])
    for e in range(mesh.elem.shape[0]):
        p = int(mesh.p[e])
        xi, w = element.tensor_points(nq or p + 3)
        X = mesh.vert[mesh.elem[e]]
        _, J = element.trilinear(X, xi)
        wd = w * np.linalg.det(J)
        E, H = system.fields_at(mesh, e, us[e], xi)
        eE = np.sum(wd * np.sum(np.abs(E) ** 2, axis=1))
        eH = np.sum(wd * np.sum(np.abs(H) ** 2, axis=1))
        out[e] = 0.5 * mesh.omega * (complex(mesh.eps[e]).imag * eE + complex(mesh.mu[e]).imag * eH)
    return out


def face_flux(mesh, us, faces, nq=None):
    """Sum over (element, face) pairs of int_f Re(E x conj(H)) . n_out dA (interior fields of the element)."""
    total = 0.0
    for e, f in faces:
        p = int(mesh.p[e])
        d, s = f // 2, f % 2
        xi, w = element.tensor_points(nq or p + 3, fixed=(d, s))
        X = mesh.vert[mesh.elem[e]]
        _, J = element.trilinear(X, xi)
        det = np.linalg.det(J)
        N = system.face_normal_ref(f)
        ndA = det[:, None] * np.einsum('qab,a->qb', np.linalg.inv(J), N)  # det J J^{-T} N (row q)
        E, H = system.fields_at(mesh, e, us[e], xi)
        S = np.real(np.cross(E, np.conj(H)))
        total += np.sum(w * np.sum(S * ndA, axis=1))
    return total


def e0_from_input_power(p_input, flux_in):
    """Reference electric field E0 (V/m) giving input power p_input (W) for a port inflow flux_in (Eq. power_scaling)."""
    return np.sqrt(2.0 * Z0 * p_input / flux_in)
