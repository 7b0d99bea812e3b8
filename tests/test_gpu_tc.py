"""Tensor-core (tcgen05, kind::tf32) quadrature contraction against exact and FP64 references.

* Small integers are exact in TF32 and their products and sums stay exact in
  FP32 below 2^24, so C = A^T B must match numpy bit for bit: this pins the
  operand layouts (no transposition or core-matrix mix-up survives it).
* On the element's real quadrature arrays the reduced modes perturb M, C, P, Q;
  their errors against FP64 are reported quantities with the bounds below
  (TF32: 10-bit mantissa, ~1e-3; 3xTF32: about FP32 accuracy, ~1e-6).
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


@pytest.mark.parametrize("shape", [(300, 300, 375), (300, 81, 375), (128, 128, 32), (37, 200, 45)])
@pytest.mark.parametrize("split", [1, 3])
def test_tc_gemm_exact_on_integers(dpg_mod, shape, split):
    Ma, Nb, Kd = shape
    rng = np.random.default_rng(Ma + 7 * Nb + Kd)
    A = rng.integers(-8, 9, size=(Kd, Ma)).astype(np.float64)
    B = rng.integers(-8, 9, size=(Kd, Nb)).astype(np.float64)
    C = dpg_mod.tc_gemm(A, B, split=split)
    assert np.array_equal(C, A.T @ B)


def test_tc_gemm_upper_only_leaves_lower_tiles(dpg_mod):
    rng = np.random.default_rng(3)
    A = rng.integers(-4, 5, size=(64, 300)).astype(np.float64)
    C0 = np.full((300, 300), 7.0)
    C = dpg_mod.tc_gemm(A, A, split=1, upper_only=True, C=C0)
    full = A.T @ A
    for bi in range(3):
        for bj in range(3):
            blk = (slice(128 * bi, 128 * bi + 128), slice(128 * bj, 128 * bj + 128))
            if bj < bi:
                assert np.all(C[blk] == 7.0)
            else:
                assert np.array_equal(C[blk], full[blk])


@pytest.mark.parametrize("split,bound", [(1, 2e-3), (3, 1e-5)])
def test_tc_gemm_rounding_error(dpg_mod, split, bound):
    rng = np.random.default_rng(5)
    A = rng.normal(size=(375, 300))
    B = rng.normal(size=(375, 81))
    C = dpg_mod.tc_gemm(A, B, split=split)
    ref = A.T @ B
    err = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    assert err < bound


@pytest.mark.parametrize("prec,bound", [(1, 5e-3), (2, 1e-5)])
def test_reduced_precision_element_matrices(dpg_mod, prec, bound):
    """G_K, B_K of jittered lossy elements in the reduced modes against the FP64 path (reported error)."""
    mesh = inputs.cavity(2, 2, jitter=0.1, eps_mode='random')
    ids = [0, 3, 5]
    ref = dpg_mod.DPG(mesh)
    r = ref.element_dump(ids)
    ref.destroy()
    d = dpg_mod.DPG(mesh, precision=prec)
    o = d.element_dump(ids)
    d.destroy()
    for key in ("G", "B"):
        err = np.linalg.norm(o[key] - r[key]) / np.linalg.norm(r[key])
        assert 0 < err < bound, (key, err)
