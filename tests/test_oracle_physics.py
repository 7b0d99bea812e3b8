"""Pins of the oracle against the paper's printed numbers and the closed-form TE mode."""
import os

import numpy as np
import pytest

from oracle import basis, physics, system
from paper_2609_03155_b300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden():
    out = {}
    for line in open(GOLD):
        if line.startswith('#') or not line.strip():
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


def _curl_fd(f, x, h=1e-6):
    g = []
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        g.append((f(x + e) - f(x - e)) / (2 * h))
    return np.stack([g[1][:, 2] - g[2][:, 1], g[2][:, 0] - g[0][:, 2], g[0][:, 1] - g[1][:, 0]], axis=1)


@pytest.mark.parametrize("mn", [(1, 0), (1, 1), (2, 1)])
def test_te_mode_solves_maxwell(mn):
    """The TE_mn formula of Sec. 4.1 satisfies Eq. (maxwell_dimensionless) with J = 0 and PEC walls."""
    m, n = mn
    a, b, omega, eps, mu = 0.25, 0.2, 51.3482, 1.0, 1.0
    x = np.random.default_rng(0).uniform(0, 1, size=(6, 3)) * np.array([a, b, 0.5])
    E = lambda y: physics.te_fields(y, omega, a, b, m, n, eps, mu)[0]
    H = lambda y: physics.te_fields(y, omega, a, b, m, n, eps, mu)[1]
    Ex, Hx = E(x), H(x)
    far = _curl_fd(E, x) - 1j * omega * mu * Hx
    amp = _curl_fd(H, x) + 1j * omega * eps * Ex
    assert np.abs(far).max() < 1e-5 * np.abs(omega * Hx).max()
    assert np.abs(amp).max() < 1e-5 * np.abs(omega * Ex).max()
    # PEC: tangential E vanishes on x1 = 0, a and x2 = 0, b
    for d, val in ((0, 0.0), (0, a), (1, 0.0), (1, b)):
        y = x.copy()
        y[:, d] = val
        nn = np.zeros(3)
        nn[d] = 1.0
        assert np.abs(np.cross(nn, E(y))).max() < 1e-12 * np.abs(Ex).max()


def test_outgoing_impedance_condition():
    """With Z^{-1} = k3/(omega mu) the TE10 wave satisfies n x H + Z^{-1} n x (E x n) = 0 at the outlet."""
    a, b, omega = 0.08636, 0.04318, inputs.omega_from_hz(2.45e9)
    zinv = physics.impedance_zinv(omega, a, b, 1, 0)
    x = np.random.default_rng(1).uniform(0, 1, size=(5, 3)) * np.array([a, b, 0])
    x[:, 2] = 0.3
    E, H = physics.te_fields(x, omega, a, b, 1, 0)
    nn = np.array([0, 0, 1.0])
    N = np.broadcast_to(nn, E.shape)
    res = np.cross(N, H) + zinv * np.cross(N, np.cross(E, N))
    assert np.abs(res).max() < 1e-13 * np.abs(H).max()
    # the port datum on the inlet (n = -x3) equals 2 i k3/k1 sin(k1 x1) e_2 at x3 = 0
    g = physics.te_port_g([0, 0, -1.0], omega, a, b, 1, 0)
    x[:, 2] = 0.0
    k1, _, _, k3 = physics.te_wavenumbers(omega, a, b, 1, 0)
    want = np.zeros((5, 3), complex)
    want[:, 1] = 2j * k3 / k1 * np.sin(k1 * x[:, 0])
    assert np.allclose(g(x), want, atol=1e-12)
    # the input generator's impedance parameter is the same number
    assert abs(inputs.te_zinv(omega, a, b, 1, 0) - zinv) < 1e-15


def test_paper_constants():
    gv = golden()
    # App. C.3: Z_s^{-1} of WR430 at 2.45 GHz (width 0.1092 m) = k3/(omega mu), L = 1 m, c0 exact
    omega = physics.omega_from_hz(2.45e9)
    zinv = physics.impedance_zinv(omega, gv['wr430_width_m'], 0.0546, 1, 0).real
    assert abs(zinv - gv['wr430_zinv']) < 1e-9
    # App. C.2 vs Sec. 4.2: f = 2.38567258e8 Hz is omega = 5 with L = 1 m
    assert abs(physics.omega_from_hz(gv['fichera_freq_hz']) - gv['fichera_omega']) < 1e-8


def _paper_guide_dofs(nx, ny, nz, p):
    """DoFs the paper counts: 4 (Re/Im x E-hat/H-hat) x full Nedelec space of FEEC order p+1."""
    m = inputs.waveguide(0.25, 0.25, 1.0, nx, ny, nz, 2.45e9, p)
    num = system.number_traces(m)
    r = p + 1
    interior = 3 * r * (r - 1) ** 2 * m.elem.shape[0]
    return 4 * (num.n_entity_dofs + interior)


def test_dof_counts_pin_the_space_indices():
    """Sec. 4.1: 720 DoFs on the coarsest 1x1x4 guide at p = 1, about 1.65 M on the finest (16x16x64)."""
    gv = golden()
    assert _paper_guide_dofs(1, 1, 4, 1) == gv['waveguide_dofs_coarsest']
    fine = _paper_guide_dofs(16, 16, 64, 1)
    assert abs(fine - gv['waveguide_dofs_finest_approx']) / gv['waveguide_dofs_finest_approx'] < 0.01
    assert fine == 1647360
    # p = 3 on the third level (4x4x16) has about 8x fewer DoFs than p = 1 on the fifth level
    ratio = fine / _paper_guide_dofs(4, 4, 16, 3)
    assert abs(ratio - gv['waveguide_dof_ratio_approx']) < 0.5


@pytest.mark.slow
def test_te10_convergence_rate_p1():
    """Sec. 4.1: L2 errors of E and H decrease at the optimal rate p + 1 (p = 1)."""
    gv = golden()
    errs = []
    for refine in (1, 2):
        m = inputs.waveguide_2d_config(p=1, refine=refine)
        sol = system.solve(m)
        ex = lambda x: physics.te_fields(x, m.omega, 0.086, m.vert[:, 1].max(), 1, 0)
        errs.append(system.l2_field_error(m, sol, ex))
    errs = np.array(errs)
    rates = np.log2(errs[0] / errs[1])
    assert np.all(rates > gv['waveguide_rate_p1'] - 0.25), rates
    assert errs[1].max() < 5e-3
