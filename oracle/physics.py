"""Closed-form fields and constants for the oracle (test infrastructure only).

* Sec. 4.1: TE_mn mode of a rectangular waveguide [0,a] x [0,b] travelling
  along +x3, k1 = m pi / a, k2 = n pi / b, kc^2 = k1^2 + k2^2,
  k3 = sqrt(omega^2 eps mu - kc^2).
* Sec. 4.1 port / outlet conditions: Robin with Z_s^{-1} = k3 / (omega mu) and
  g = n x H_TE + Z_s^{-1} n x (E_TE x n) on the port, g = 0 on the outlet.
* App. A: omega = omega_dim L / c0 with L = 1 m (our reading, pinned by the
  Fichera frequency of App. C, which equals omega = 5).
"""
import numpy as np

C0 = 299792458.0


def omega_from_hz(f_hz, L=1.0):
    """Dimensionless angular frequency of App. A: 2 pi f L / c0."""
    return 2.0 * np.pi * f_hz * L / C0


def te_wavenumbers(omega, a, b, m, n, eps=1.0, mu=1.0):
    k1 = m * np.pi / a
    k2 = n * np.pi / b
    kc2 = k1 * k1 + k2 * k2
    k3 = np.sqrt(complex(omega * omega * eps * mu - kc2))
    return k1, k2, kc2, k3


def te_fields(x, omega, a, b, m, n, eps=1.0, mu=1.0):
    """E, H of the TE_mn mode at points x (N,3): the formula of Sec. 4.1."""
    k1, k2, kc2, k3 = te_wavenumbers(omega, a, b, m, n, eps, mu)
    x = np.asarray(x, dtype=float)
    c1, s1 = np.cos(k1 * x[:, 0]), np.sin(k1 * x[:, 0])
    c2, s2 = np.cos(k2 * x[:, 1]), np.sin(k2 * x[:, 1])
    ph = np.exp(1j * k3 * x[:, 2])
    E = np.zeros((len(x), 3), dtype=complex)
    H = np.zeros((len(x), 3), dtype=complex)
    pre = 1j * omega * mu / kc2
    E[:, 0] = pre * (-k2 * c1 * s2) * ph
    E[:, 1] = pre * (k1 * s1 * c2) * ph
    H[:, 0] = -1j * k3 * k1 / kc2 * s1 * c2 * ph
    H[:, 1] = -1j * k3 * k2 / kc2 * c1 * s2 * ph
    H[:, 2] = c1 * c2 * ph
    return E, H


def te_port_g(normal, omega, a, b, m, n, eps=1.0, mu=1.0):
    """Robin datum g(x) = n x H_TE + Z^{-1} n x (E_TE x n) with Z^{-1} = k3/(omega mu)."""
    nn = np.asarray(normal, dtype=float)
    zinv = te_wavenumbers(omega, a, b, m, n, eps, mu)[3] / (omega * mu)

    def g(x):
        E, H = te_fields(x, omega, a, b, m, n, eps, mu)
        N = np.broadcast_to(nn, E.shape)
        Et = np.cross(N, np.cross(E, N))
        return np.cross(N, H) + zinv * Et
    return g


def impedance_zinv(omega, a, b, m, n, eps=1.0, mu=1.0):
    """Z_s^{-1} = k_x3 / (omega mu_r) of the impedance condition in Sec. 4.1."""
    return te_wavenumbers(omega, a, b, m, n, eps, mu)[3] / (omega * mu)
