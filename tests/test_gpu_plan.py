"""Launch plan of the element pass: CUDA graph replay, chunk sizes and the autotuner.

Per-element arithmetic does not depend on how elements are grouped into
launches, and the assembly sums in a fixed colour order, so the graph replay,
plain launches and any chunk size must give bit-identical systems and
solutions.
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


def _solve(d):
    d.element_batch()
    d.assemble()
    x, rep = d.cg_solve(rtol=1e-12, max_iter=100000)
    u, eta, _ = d.estimate(x)
    _, _, val, b = d.csr_copy()
    return x.cpu().numpy(), eta.cpu().numpy(), val, b


@pytest.mark.parametrize("name", ["waveguide", "fichera_mixed"])
def test_graph_replay_equals_plain_launches(dpg_mod, name):
    if name == "waveguide":
        mesh = inputs.waveguide_3d_config(4, 2, 6, p=2)
    else:
        mesh = inputs.fichera_cavity(2, grade=1.5)
    d = dpg_mod.DPG(mesh, chunk=7)  # several chunks per group, ragged last chunk
    d.set_graph(False)
    ref = _solve(d)
    d.set_graph(True)
    first = _solve(d)     # capture + replay
    second = _solve(d)    # replay of the captured graph
    for a, b in ((first, ref), (second, ref)):
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
    d.destroy()


def test_autotune_keeps_results_bitwise(dpg_mod):
    mesh = inputs.fichera_cavity(2, grade=1.5)
    d = dpg_mod.DPG(mesh, chunk=5)
    ref = _solve(d)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tuned = d.autotune(max_workspace_gb=8.0)
    groups = d.group_info()
    assert set(tuned) == {g[0] for g in groups}
    for p, n, cap in groups:
        assert cap == tuned[p][0]
        assert cap % sms == 0 or cap <= n
        assert tuned[p][1] > 0
    again = _solve(d)
    for u, v in zip(again, ref):
        assert np.array_equal(u, v)
    d.destroy()


def test_graph_replay_with_timing(dpg_mod):
    """Factorisation timing events inside the captured graph are recorded at every replay."""
    mesh = inputs.waveguide_3d_config(4, 2, 6, p=2)
    d = dpg_mod.DPG(mesh, chunk=10)
    d.element_batch()             # capture without timing
    d.timing_enable(True)
    d.element_batch()             # re-capture with external event nodes
    d.element_batch()             # replay
    t = d.timing_get()
    assert t["factor_elements"] == 2 * mesh.n_elem
    assert t["factor_launches"] > 0 and t["factor_ms"] > 0
    d.assemble()                  # no stale error left behind
    d.destroy()
