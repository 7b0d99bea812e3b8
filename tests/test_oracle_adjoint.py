"""Pin of the oracle adjoint gradient against brute-force central differences of direct solves."""
import numpy as np
import pytest

from oracle import adjoint, system
from paper_2609_03155_b300 import inputs


@pytest.mark.slow
def test_oracle_adjoint_matches_central_differences():
    m = inputs.cavity(2, 1, omega=5.0)
    mask = np.zeros(m.n_elem, bool)
    mask[[0, 3, 5]] = True
    m.eps = m.eps.copy()
    m.eps[mask] = 20 + 5j
    m.eps[1] = 3 + 1j
    sol = system.solve(m)
    P, dre, dim = adjoint.gradient(m, sol, mask)
    assert P > 0
    elems = [0, 1, 6]
    fd = adjoint.fd_gradient(m, mask, elems, h=1e-6)
    scale = max(np.abs(dre).max(), np.abs(dim).max())
    for k, e in enumerate(elems):
        assert abs(dre[e] - fd[k, 0]) < 1e-6 * scale
        assert abs(dim[e] - fd[k, 1]) < 1e-6 * scale


def test_torch_complex_gradient_convention():
    """torch returns dL/dRe z + i dL/dIm z for a real L of a complex input (pinned on |z|^2)."""
    torch = pytest.importorskip("torch")
    z = torch.tensor(1 + 2j, dtype=torch.complex128, requires_grad=True)
    (z.abs() ** 2).backward()
    assert complex(z.grad) == 2 + 4j
