"""The adaptive loop of Sec. 4.2 on the CUDA path against the oracle's loop, step by step.

Both loops start from the eight unit cells of the Fichera oven (p = 1 here,
to keep the oracle's dense solves small), estimate eta_K, mark by the fixed
fractions 0.30 / 0.05 of the paper's parameter table (dpg_mark_fraction on the
GPU side, oracle/adapt.py on the oracle side) and refine / coarsen the same
2:1 octree.  Per step: the same number of unknowns, u_K within 1e-10 and eta_K
within 1e-9 per element of the oracle's direct solve, identical marks, and a
decreasing global estimate.  Meshes beyond the first step have several
refinement levels, so hanging faces and edges of every kind occur.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adapt, hanging
from paper_2609_03155_b300 import inputs
from test_gpu_parity import rel


@pytest.fixture(scope="module")
def dpg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_03155_b300 import dpg
    return dpg


def test_adaptive_loop_matches_oracle(dpg_mod):
    t_gpu, t_or = inputs.fichera_octree(p=1), inputs.fichera_octree(p=1)
    E = []
    for step in range(3):
        m, leaves = t_gpu.mesh()
        mo, leaves_o = t_or.mesh()
        assert leaves == leaves_o
        sol = hanging.solve(mo)
        d = dpg_mod.DPG(m)
        assert d.n == sol['n']
        d.element_batch()
        d.assemble()
        x, rep = d.cg_solve(rtol=1e-13, max_iter=200000)
        assert rep['converged']
        u, eta, etag = d.estimate(x)
        u = u.cpu().numpy().reshape(-1)
        for e in range(m.n_elem):
            assert rel(u[d.u_off[e]:d.u_off[e + 1]], sol['rec'][e]['u']) < 1e-10, (step, e)
        eta_g = eta.cpu().numpy()
        assert np.all(np.abs(eta_g - sol['eta']) <= 1e-9 * sol['eta']), (step, np.max(np.abs(eta_g - sol['eta']) / sol['eta']))
        for power in (2, 1):
            marks = d.mark_fraction(eta, 0.30, 0.05, power=power)
            marks_or = adapt.mark_fraction(sol['eta'], 0.30, 0.05, power=power)
            assert np.array_equal(marks, marks_or), (step, power)
        E.append(etag)
        d.destroy()
        t_gpu.adapt(leaves, marks)
        t_or.adapt(leaves_o, marks_or)
    assert E[0] > E[1] > E[2], E
