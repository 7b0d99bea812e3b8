"""Host-side work counts of the bench's roofline lines.

* The FP64-equivalent factorisation flops of one element (Cholesky of G,
  triangular solves, Gram product, second condensation; Sec. 2.3) against the
  same count taken term by term from the element sizes (1.237e9 at p = 2).
* The FP16 MMA flops the split-arithmetic factorisation issues per element,
  from its tile schedule, against ncu's count of FP16 tensor operations on one
  real p = 2 element (sm__ops_path_tensor_op_utchmma_src_fp16_dst_fp32:
  4.60e12 over 400 elements = 1.150e10); complex elements issue twice the
  MMA work per tile (the real part over the stacked real and imaginary
  columns, the imaginary part as two cross products) on tiles half as wide:
  four times the real count per element.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_factor_flops_p2():
    import bench
    assert bench.flops_factor_per_element(2) == pytest.approx(1.237460568e9, rel=1e-9)


def test_tc_mma_flops_match_the_measured_count():
    import bench
    real = bench.tc_mma_flops_per_element(2, False)
    assert real == pytest.approx(4.60e12 / 400, rel=2e-3)
    assert real == 11501830144
    # complex: twice the MMA work per tile, tiles half as wide -> 4x per element
    assert bench.tc_mma_flops_per_element(2, True) == 4 * real
    # more work at higher order, monotone
    assert [bench.tc_mma_flops_per_element(p, False) for p in (1, 2, 3, 4)] == sorted(
        bench.tc_mma_flops_per_element(p, False) for p in (1, 2, 3, 4))
