"""Pins of the oracle's power routines (Sec. 3.2: Q_em and the port flux of Eq. power_scaling)."""
import numpy as np

from oracle import basis, power
from paper_2609_03155_b300 import inputs


def _affine_mesh(A, x0, p, eps, mu, omega):
    """One parallelepiped element x = x0 + A xi."""
    corners = np.array([[(v >> a) & 1 for a in range(3)] for v in range(8)], float)
    vert = x0[None, :] + corners @ A.T
    return inputs.Mesh(vert=vert, elem=np.arange(8, dtype=np.int32)[None, :], p=np.array([p], np.int8),
                       eps=np.array([eps]), mu=np.array([mu]), face_bc=np.zeros((1, 6), np.int8),
                       face_grp=np.zeros((1, 6), np.int16), omega=omega)


def _interp(mesh, fieldE, fieldH):
    """Interior coefficients: nodal values at the Gauss-Legendre Lagrange nodes (x-index fastest)."""
    p = int(mesh.p[0])
    g = basis.gauss_legendre(p + 1)[0]
    nodes = np.array([[g[i], g[j], g[k]] for k in range(p + 1) for j in range(p + 1) for i in range(p + 1)])
    A = mesh.vert[1] - mesh.vert[0], mesh.vert[2] - mesh.vert[0], mesh.vert[4] - mesh.vert[0]
    x = mesh.vert[0][None, :] + nodes @ np.stack(A, axis=0)
    E, H = fieldE(x), fieldH(x)
    return np.concatenate([E[:, d] for d in range(3)] + [H[:, d] for d in range(3)]).astype(complex)


def test_element_power_closed_form_on_a_box():
    # box [0,2] x [0,1] x [0,3], E = (1, x, y), H = (0, 0, z):
    # int |E|^2 = 16, int |H|^2 = 18; Q = 1/2 w (Im eps 16 + Im mu 18)
    m = _affine_mesh(np.diag([2.0, 1.0, 3.0]), np.zeros(3), 1, 4.0 + 0.5j, 1.0 + 0.25j, 2.0)
    u = _interp(m, lambda x: np.stack([np.ones(len(x)), x[:, 0], x[:, 1]], 1),
                lambda x: np.stack([0 * x[:, 0], 0 * x[:, 0], x[:, 2]], 1))
    q = power.element_power(m, [u])
    assert abs(q[0] - 0.5 * 2.0 * (0.5 * 16.0 + 0.25 * 18.0)) < 1e-12


def test_face_flux_of_constant_fields_is_poynting_dot_vector_area():
    A = np.array([[1.0, 0.3, 0.2], [0.1, 0.8, -0.25], [0.05, 0.1, 1.2]])  # sheared, tilted faces
    m = _affine_mesh(A, np.array([0.2, -0.1, 0.3]), 2, 1.0, 1.0, 1.0)
    E0 = np.array([0.3 + 1j, 1.0, -0.5j])
    H0 = np.array([2.0, 0.5 - 0.5j, 0.25])
    u = _interp(m, lambda x: np.tile(E0, (len(x), 1)), lambda x: np.tile(H0, (len(x), 1)))
    S = np.real(np.cross(E0, np.conj(H0)))
    a1, a2, a3 = A[:, 0], A[:, 1], A[:, 2]
    # outward vector areas of the six faces xi_d = s
    areas = {0: -np.cross(a2, a3), 1: np.cross(a2, a3), 2: -np.cross(a3, a1), 3: np.cross(a3, a1),
             4: -np.cross(a1, a2), 5: np.cross(a1, a2)}
    for f, vec in areas.items():
        assert abs(power.face_flux(m, [u], [(0, f)]) - S @ vec) < 1e-12
    # closed surface, constant field: zero net flux
    assert abs(power.face_flux(m, [u], [(0, f) for f in range(6)])) < 1e-12


def test_free_space_impedance():
    mu0 = 4e-7 * np.pi  # within 1e-9 of the CODATA value
    assert abs(power.Z0 - mu0 * 299792458.0) < 1e-6 * power.Z0
    # P = 1/2 E0^2 / Z0 * flux inverted
    E0 = power.e0_from_input_power(1000.0, 0.02)
    assert abs(0.5 * E0 ** 2 / power.Z0 * 0.02 - 1000.0) < 1e-9
