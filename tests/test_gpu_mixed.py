"""Mixed trial degrees on the CUDA path against the oracle's mixed-order solve.

Reading (the paper refines in h only): an edge or face carries trace unknowns
of order min over its elements of (p + 1); every element computes at its own
degree and sees the global trace through R_K (nodal evaluation).  The GPU and
the oracle number the unknowns differently, so the comparison is on what does
not depend on numbering: the number of unknowns, the interior field u_K of
every element and eta_K.  Tolerances as for one degree: u relative 1e-10 (CG to
1e-13 against the oracle's direct solve), eta_K relative 1e-9 per element.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mixed
from paper_2609_03155_b300 import inputs
from test_gpu_parity import _lossy_jittered, rel


@pytest.fixture(scope="module")
def dpg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_03155_b300 import dpg
    return dpg


def _case(name):
    if name == "fichera_n1":
        return inputs.fichera_cavity(1)  # degrees 1, 1, 1, 1, 2, 1, 2, 3; Dirichlet data on top
    if name == "fichera_n2_mix":
        return inputs.fichera_cavity(2, grade=1.5, mix=(0.4, 0.3, 0.3))  # 64 elements, degrees 1..3
    m = _lossy_jittered(1, n=(2, 2, 1))  # Robin port and impedance faces, lossy materials
    m.p = np.array([2, 1, 4, 3], np.int8)
    return m


@pytest.mark.parametrize("name", ["fichera_n1", "lossy_p1234", "fichera_n2_mix"])
def test_mixed_degrees_match_oracle(dpg_mod, name):
    mesh = _case(name)
    sol = mixed.solve_mixed(mesh)
    d = dpg_mod.DPG(mesh)
    assert d.n == sol['n']
    assert not d.uniform and list(d.p_elem) == list(mesh.p)
    d.element_batch()
    d.assemble()
    x, rep = d.cg_solve(rtol=1e-13, max_iter=200000)
    assert rep['converged']
    u, eta, etag = d.estimate(x)
    u = u.cpu().numpy()
    for e in range(mesh.n_elem):
        ue = u[d.u_off[e]:d.u_off[e + 1]]
        assert rel(ue, sol['rec'][e]['u']) < 1e-10, e
    eta_or = sol['eta']
    eta_g = eta.cpu().numpy()
    assert np.all(np.abs(eta_g - eta_or) <= 1e-9 * eta_or), np.max(np.abs(eta_g - eta_or) / eta_or)
    assert abs(etag - np.sqrt(np.sum(eta_or ** 2))) < 1e-9 * np.sqrt(np.sum(eta_or ** 2))
    d.destroy()


def test_mixed_degrees_trace_map_layout(dpg_mod):
    """Per-element offsets follow the degrees; unused slots appear only on elements with a lower-order entity."""
    mesh = inputs.fichera_cavity(1)
    d = dpg_mod.DPG(mesh)
    nh = np.array([24 * (int(p) + 1) ** 2 for p in mesh.p])
    nu = np.array([6 * (int(p) + 1) ** 3 for p in mesh.p])
    assert np.array_equal(np.diff(d.h_off), nh) and np.array_equal(np.diff(d.u_off), nu)
    m, fv = d.trace_map()
    assert m.shape == (d.h_off[-1],)
    unused = 0
    for e in range(mesh.n_elem):
        me = m[d.h_off[e]:d.h_off[e + 1]]
        if mesh.p[e] == 1:  # the lowest degree: every slot holds an unknown (no Robin faces here)
            assert np.all(me != -2)
        unused += np.sum(me == -2)
        used = me[me >= 0]
        assert len(np.unique(used)) == len(used)
    assert unused > 0
    d.destroy()


def test_mixed_degrees_adjoint_matches_gpu_finite_differences(dpg_mod):
    """Adjoint gradient through R_K: central differences of GPU solves on a mixed-degree cavity."""
    mesh = inputs.fichera_cavity(1)
    mesh.eps = np.array([1.0, 3 + 1j, 1.0, 20 + 5j, 2 + 0.5j, 1.0, 20 + 5j, 4 + 2j])
    mask = np.zeros(mesh.n_elem, bool)
    mask[[3, 6, 7]] = True
    d = dpg_mod.DPG(mesh, adjoint=True)
    mk = torch.tensor(mask.astype(np.uint8), device='cuda')
    eps0 = torch.tensor(mesh.eps, dtype=torch.complex128)
    Pfun = lambda e: dpg_mod.AbsorbedPower.apply(e, d, mk, 1e-13)
    eps = eps0.clone().requires_grad_(True)
    P = Pfun(eps)
    P.backward()
    g = eps.grad.numpy()
    h = 1e-6
    scale = np.abs(g).max()
    for e in range(mesh.n_elem):
        for part in (1.0, 1j):
            ep, em = eps0.clone(), eps0.clone()
            ep[e] += part * h
            em[e] -= part * h
            with torch.no_grad():
                fd = (Pfun(ep).item() - Pfun(em).item()) / (2 * h)
            an = g[e].real if part == 1.0 else g[e].imag
            assert abs(an - fd) < 1e-5 * scale + 1e-9 * abs(P.item()), (e, part, an, fd)
    d.destroy()
