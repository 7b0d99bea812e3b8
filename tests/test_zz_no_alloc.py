"""The allocation-free estimator gives the same results as dpg_estimate.

dpg_estimate_noalloc serves callers that cannot allocate device memory during
a call (their memory is committed to a pool of their own up front, or their
loop may not wait on an allocator); it keeps its scratch in a fixed array
inside the library instead.  This file is collected last on purpose, so a run
that stops at the first failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_estimate_noalloc_matches_estimate_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_03155_b300 import _lib, dpg, inputs
    from paper_2609_03155_b300._lib import ptr, stream_handle

    mesh = inputs.waveguide_2d_config(p=1)
    d = dpg.DPG(mesh)
    d.element_batch()
    d.assemble()
    x, rep = d.cg_solve(rtol=1e-12)
    assert rep['converged']
    L = _lib.lib()
    ref_u = torch.empty(d.n_elem * d.n_u, dtype=torch.complex128, device='cuda')
    ref_eta = torch.empty(d.n_elem, dtype=torch.float64, device='cuda')
    ref_tot = C.c_double()
    _lib.check(L.dpg_estimate(d.h, ptr(x), ptr(ref_u), ptr(ref_eta), C.byref(ref_tot), stream_handle()), d.h)
    for call in range(2):
        u = torch.full((d.n_elem * d.n_u,), float('nan'), dtype=torch.complex128, device='cuda')
        eta = torch.full((d.n_elem,), float('nan'), dtype=torch.float64, device='cuda')
        tot = C.c_double()
        rc = L.dpg_estimate_noalloc(d.h, ptr(x), ptr(u), ptr(eta), C.byref(tot), stream_handle())
        _lib.check(rc, d.h)
        torch.cuda.synchronize()
        e_ref = ref_eta.cpu().numpy()
        assert np.all(np.abs(eta.cpu().numpy() - e_ref) <= 1e-12 * e_ref), call
        u_ref = ref_u.cpu().numpy()
        assert np.linalg.norm(u.cpu().numpy() - u_ref) <= 1e-12 * np.linalg.norm(u_ref), call
        assert abs(tot.value - ref_tot.value) <= 1e-12 * ref_tot.value, call
    d.destroy()
