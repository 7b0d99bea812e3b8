"""The order-bucketed element pass against the per-order pass.

In bucketed mode a wave forms one chunk of every (order, arithmetic) list and
factors them all in persistent launches that take elements of every trial
order from a longest-first work list; each element still gets exactly the
arithmetic of the per-chunk kernel, and (stored mode) assembly keeps its
fixed colour order, so the trace solution and eta_K must be bitwise equal to
the per-order pass.  Checked on meshes that mix orders 1..4 with real and
complex elements, with one and with several waves, and in streaming mode
(where the chunking orders the assembly sums: equal to rounding), plus the
load-balance report of both modes.
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


def _mixed_guide():
    """6 x 3 x 6 guide (port: complex; the rest lossless: real) with orders 1..4 mixed."""
    m = inputs.waveguide_3d_config(6, 3, 6, 2)
    rng = np.random.default_rng(5)
    m.p = rng.choice(np.array([1, 2, 3, 4], np.int8), size=m.n_elem, p=[0.4, 0.3, 0.2, 0.1])
    return m


def _run(dpg_mod, mesh, bucketed, chunk=0, streaming=False):
    d = dpg_mod.DPG(mesh, chunk=chunk, streaming=streaming)
    if bucketed:
        d.set_bucketed(True)
    d.element_batch()
    bal = d.factor_balance()
    d.assemble()
    x, rep = d.cg_solve(rtol=1e-12, max_iter=200000)
    assert rep['converged']
    u, eta, _ = d.estimate(x)
    out = (x.clone(), eta.clone(), bal, d.n_elem)
    d.destroy()
    return out


@pytest.mark.parametrize("case", ["guide_p1234", "fichera_n2_mix"])
@pytest.mark.parametrize("chunk", [0, 7])
def test_bucketed_pass_is_bitwise_equal_to_per_order_pass(dpg_mod, case, chunk):
    mesh = _mixed_guide() if case == "guide_p1234" else inputs.fichera_cavity(2, grade=1.5, mix=(0.4, 0.3, 0.3))
    x0, e0, b0, ne = _run(dpg_mod, mesh, False, chunk)
    x1, e1, b1, _ = _run(dpg_mod, mesh, True, chunk)
    assert torch.equal(x0, x1)
    assert torch.equal(e0, e1)
    for b in (b0, b1):
        assert b['elements'] == ne
        assert 0.0 < b['sm_busy'] <= 1.0 and b['span_ms'] > 0.0


def test_bucketed_streaming_pass_matches(dpg_mod):
    """Streaming assembles chunk by chunk, so the chunking fixes the summation
    order of the CSR entries: against the stored pass the results agree to
    rounding (amplified by the CG's conditioning), not bitwise."""
    mesh = _mixed_guide()
    x0, e0, _, _ = _run(dpg_mod, mesh, False, 0, streaming=False)
    x1, e1, b1, ne = _run(dpg_mod, mesh, True, 5, streaming=True)
    assert float(torch.linalg.vector_norm(x1 - x0) / torch.linalg.vector_norm(x0)) < 1e-9
    assert float(torch.max(torch.abs(e1 - e0) / e0)) < 1e-8
    assert b1['elements'] == ne


def test_bucketed_mode_switch_and_fp64_factorisation(dpg_mod):
    mesh = _mixed_guide()
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    x_ref, _ = d.cg_solve(rtol=1e-12, max_iter=200000)
    d.set_bucketed(True)
    d.set_factor_arith(0)  # FP64-pipe factorisation: per-chunk launches inside each wave, no stamps
    d.element_batch()
    with pytest.raises(dpg_mod.DPGError):
        d.factor_balance()
    d.assemble()
    x64, _ = d.cg_solve(rtol=1e-12, max_iter=200000)
    assert float(torch.linalg.vector_norm(x64 - x_ref) / torch.linalg.vector_norm(x_ref)) < 1e-10
    d.set_factor_arith(1)
    with pytest.raises(dpg_mod.DPGError):
        d.autotune()  # per-order chunk sizes mean nothing to waves
    d.set_bucketed(False)
    d.element_batch()
    d.assemble()
    x, _ = d.cg_solve(rtol=1e-12, max_iter=200000)
    assert torch.equal(x, x_ref)
    d.destroy()
