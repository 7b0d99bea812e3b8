"""Failure detection on the device, without a fault, a trap or an endless wait.

* The CG kernel's grid barriers are bounded in time.  The test hook
  dpg_set_wait_limit(hold=1) makes no barrier release (a flag that nothing
  sets), so every wait runs out after a short limit; the solve must return
  DPG_ERR_TIMEOUT and the context must stay usable for the next solve.
* A failed element pass (a non-positive pivot) must not poison the next one:
  the pivot flags are cleared at the start of every pass, and assembly refuses
  to run on the factors of a failed pass.  The failure is made on the host: a
  NaN permittivity for one element (dpg_update_elements copies values
  asynchronously and does not validate them), which makes that element's
  pivots fail.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_03155_b300 import inputs


@pytest.fixture(scope="module")
def dpg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_03155_b300 import dpg
    return dpg


def test_cg_barrier_timeout_is_reported_and_context_survives(dpg_mod):
    mesh = inputs.waveguide_2d_config(p=1)
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    d.set_wait_limit(wait_ns=2_000_000, hold=True)  # 2 ms, no barrier releases
    for mode in (0, 5):  # plain FP64, and FP32-inner refinement with block Jacobi
        with pytest.raises(dpg_mod.DPGError) as err:
            d.cg_solve(mode=mode, rtol=1e-10)
        assert err.value.code == -6  # DPG_ERR_TIMEOUT
    torch.cuda.synchronize()
    d.set_wait_limit(hold=False)
    x, rep = d.cg_solve(rtol=1e-12)
    assert rep['converged'] and rep['rel_residual'] <= 1e-12
    d.destroy()


def test_failed_element_pass_does_not_poison_the_next(dpg_mod):
    mesh = inputs.waveguide_2d_config(p=1)
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    x_ref, rep = d.cg_solve(rtol=1e-12)
    assert rep['converged']
    eps_bad = torch.from_numpy(np.ascontiguousarray(mesh.eps, np.complex128).copy())
    eps_bad[5] = complex(float('nan'), 0.0)
    d.update_elements(eps=eps_bad)
    with pytest.raises(dpg_mod.DPGError) as err:
        d.element_batch()
    assert err.value.code == -4  # DPG_ERR_NOT_HPD
    with pytest.raises(dpg_mod.DPGError) as err:
        d.assemble()  # the failed pass's factors are not used
    assert err.value.code == -8  # DPG_ERR_STATE
    eps_ok = torch.from_numpy(np.ascontiguousarray(mesh.eps, np.complex128).copy())
    d.update_elements(eps=eps_ok)
    d.element_batch()
    d.assemble()
    x, rep = d.cg_solve(rtol=1e-12)
    assert rep['converged']
    assert float(torch.linalg.vector_norm(x - x_ref) / torch.linalg.vector_norm(x_ref)) < 1e-12
    d.destroy()
