"""Power of a solution (Sec. 3.2: Q_em per element, port Poynting flux of Eq. power_scaling) against the oracle.

The GPU fields agree with the oracle's direct solve to 1e-10 relative (CG to
1e-13), so quadratic quantities of them agree to a few 1e-10: the bound is 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mixed, power
from oracle import system as osys
from paper_2609_03155_b300 import inputs
from test_gpu_parity import _lossy_jittered


@pytest.fixture(scope="module")
def dpg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_03155_b300 import dpg
    return dpg


def _gpu_power(dpg_mod, mesh):
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    x, rep = d.cg_solve(rtol=1e-13, max_iter=200000)
    assert rep['converged']
    q, flux = d.power(x)
    d.destroy()
    return q.cpu().numpy(), flux


def test_power_and_port_flux_match_oracle(dpg_mod):
    mesh = _lossy_jittered(1, n=(2, 2, 2))
    sol = osys.solve(mesh)
    us = [r['u'] for r in sol['rec']]
    q_or = power.element_power(mesh, us)
    q, flux = _gpu_power(dpg_mod, mesh)
    assert np.max(np.abs(q - q_or)) < 1e-9 * np.abs(q_or).max()
    for g in range(len(mesh.robin)):
        faces = [(e, f) for e in range(mesh.n_elem) for f in range(6)
                 if mesh.face_bc[e, f] == inputs.BC_ROBIN and mesh.face_grp[e, f] == g]
        f_or = power.face_flux(mesh, us, faces)
        assert abs(flux[g] - f_or) < 1e-9 * max(abs(f_or), 1e-300), (g, flux[g], f_or)


def test_power_on_mixed_degrees_matches_oracle(dpg_mod):
    mesh = inputs.fichera_cavity(1)
    mesh.eps = np.array([1.0, 3 + 1j, 1.0, 20 + 5j, 2 + 0.5j, 1.0, 20 + 5j, 4 + 2j])
    mesh.mu = np.array([1.0, 1.0, 1.0 + 0.2j, 1.0, 1.0, 1.0, 1.0, 1.0 + 0.1j])
    sol = mixed.solve_mixed(mesh)
    q_or = power.element_power(mesh, [r['u'] for r in sol['rec']])
    q, _ = _gpu_power(dpg_mod, mesh)
    assert np.max(np.abs(q - q_or)) < 1e-9 * np.abs(q_or).max()
