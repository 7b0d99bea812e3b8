"""Streaming mode (DPG_FLAG_STREAM) against the stored mode on the same meshes.

With streaming the element pass keeps no per-element condensation data: each
chunk holds elements of one colour and is assembled into the CSR system as soon
as it is condensed, and recovery and the estimator condense every chunk again.
The arithmetic per element is the same; only the order of the assembly sums
changes.  Checked: the CSR values and right-hand side (relative 1e-13), the
trace solution and u_K (1e-10), eta_K per element (1e-9), the element dump,
and the unsupported combinations.  Cases: the guide section (real and complex
paths), a lossy jittered box, mixed degrees, 2:1 hanging faces.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2609_03155_b300 import inputs
from test_gpu_parity import _lossy_jittered, rel


@pytest.fixture(scope="module")
def dpg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_03155_b300 import dpg
    return dpg


def _case(name):
    if name == "waveguide2d":
        return inputs.waveguide_2d_config(p=1)
    if name == "lossy_p2":
        return _lossy_jittered(2, n=(2, 2, 2))
    if name == "fichera_mixed":
        return inputs.fichera_cavity(2, grade=1.5, mix=(0.4, 0.3, 0.3))
    return inputs.fichera_amr(1, radius=0.9, mix=(0.4, 0.3, 0.3))


def _run(dpg_mod, mesh, streaming, chunk=0):
    d = dpg_mod.DPG(mesh, streaming=streaming, chunk=chunk)
    d.element_batch()
    d.assemble()
    _, _, val, b = d.csr_copy()
    x, rep = d.cg_solve(rtol=1e-13, max_iter=200000)
    assert rep['converged']
    u, eta, etag = d.estimate(x)
    out = dict(val=val, b=b, x=x.cpu().numpy(), u=u.cpu().numpy().reshape(-1), eta=eta.cpu().numpy(), etag=etag,
               n=d.n)
    d.destroy()
    return out


@pytest.mark.parametrize("name", ["waveguide2d", "lossy_p2", "fichera_mixed", "fichera_amr"])
def test_stream_matches_stored(dpg_mod, name):
    mesh = _case(name)
    ref = _run(dpg_mod, mesh, False)
    st = _run(dpg_mod, mesh, True, chunk=5)  # small chunks: several per colour and degree
    assert st['n'] == ref['n']
    assert rel(st['val'], ref['val']) < 1e-13
    assert rel(st['b'], ref['b']) < 1e-13
    assert rel(st['x'], ref['x']) < 1e-10
    assert rel(st['u'], ref['u']) < 1e-10
    assert np.all(np.abs(st['eta'] - ref['eta']) <= 1e-9 * ref['eta'])


def test_stream_element_dump_and_unsupported(dpg_mod):
    mesh = _lossy_jittered(1)
    d = dpg_mod.DPG(mesh, streaming=True, chunk=2)
    ref = dpg_mod.DPG(mesh)
    ids = [0, 1, 2, 3]
    a, b = d.element_dump(ids), ref.element_dump(ids)
    assert rel(a['S'], b['S']) < 1e-13 and rel(a['G'], b['G']) == 0
    with pytest.raises(dpg_mod.DPGError) as err:
        d.autotune()
    assert err.value.code == -9
    d.destroy()
    ref.destroy()
