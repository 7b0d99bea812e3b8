"""The adaptive loop's pieces on the CPU: fixed-fraction marking (Sec. 4.2) and the 2:1 octree mesh.

Pins (not the oracle against itself):
* marking: the marked-for-refinement set is the minimal set of largest cells
  reaching the fraction of sum eta^power (checked against brute force over all
  prefix lengths), the coarsening set the maximal set of smallest cells within
  its fraction, and the two are disjoint;
* octree: every pair of touching leaves differs by at most one level (brute
  force over all pairs), the domain volume is kept, coarsening undoes a
  refinement that nothing else depends on;
* loop: on the Fichera oven of Sec. 4.2 at p = 1 the global estimate
  sqrt(sum eta_K^2) of the oracle decreases over three adaptation steps (the
  paper reports a monotonic decrease).
"""
import numpy as np
import pytest

from oracle import adapt, hanging
from paper_2609_03155_b300 import inputs


@pytest.mark.parametrize("power", [1, 2])
def test_marking_is_minimal_and_maximal_prefix(power):
    rng = np.random.default_rng(5)
    for trial in range(50):
        ne = int(rng.integers(1, 60))
        eta = rng.exponential(1.0, ne) ** 2
        m = adapt.mark_fraction(eta, 0.3, 0.05, power=power)
        e2 = eta ** power
        tot = e2.sum()
        order = np.argsort(-e2, kind="stable")
        k = int((m > 0).sum())
        assert set(np.where(m > 0)[0]) == set(order[:k])
        assert e2[order[:k]].sum() >= 0.3 * tot
        assert k == 0 or e2[order[:k - 1]].sum() < 0.3 * tot
        kc = int((m < 0).sum())
        asc = order[::-1]
        assert set(np.where(m < 0)[0]) == set(asc[:kc])
        assert e2[asc[:kc]].sum() <= 0.05 * tot
        if kc < ne and m[asc[kc]] != 1:
            assert e2[asc[:kc + 1]].sum() > 0.05 * tot
    assert np.all(adapt.mark_fraction(np.zeros(4)) == 0)


def _touching_levels_ok(leaves):
    top = max(c[0] for c in leaves)
    boxes = [(c[0], np.array(c[1:]) << (top - c[0]), (np.array(c[1:]) + 1) << (top - c[0])) for c in leaves]
    for a in range(len(boxes)):
        la, lo_a, hi_a = boxes[a]
        for b in range(a + 1, len(boxes)):
            lb, lo_b, hi_b = boxes[b]
            if np.all(lo_a <= hi_b) and np.all(lo_b <= hi_a) and abs(la - lb) > 1:
                return False
    return True


def test_octree_stays_balanced_and_keeps_volume():
    t = inputs.fichera_octree(p=1)
    for step in range(3):
        m, leaves = t.mesh()
        cen = np.array([m.vert[m.elem[e]].mean(0) for e in range(m.n_elem)])
        d = np.linalg.norm(cen - 1.0, axis=1)
        marks = np.zeros(m.n_elem, np.int8)
        marks[np.argsort(d)[:max(1, m.n_elem // 4)]] = 1
        t.adapt(leaves, marks)
        m, leaves = t.mesh()
        assert _touching_levels_ok(leaves)
        vol = sum(np.prod(m.vert[m.elem[e][7]] - m.vert[m.elem[e][0]]) for e in range(m.n_elem))
        assert abs(vol - 8.0) < 1e-12
    # coarsening everything that can be merged brings the mesh back towards the start
    n_before = len(t.leaves)
    m, leaves = t.mesh()
    t.adapt(leaves, -np.ones(len(leaves), np.int8))
    assert len(t.leaves) < n_before and _touching_levels_ok(t.ordered_leaves())


@pytest.mark.slow
def test_oracle_adaptive_loop_decreases_the_global_estimate():
    t = inputs.fichera_octree(p=1)
    E = []
    for step in range(3):
        m, leaves = t.mesh()
        sol = hanging.solve(m)
        E.append(float(np.sqrt(np.sum(sol['eta'] ** 2))))
        t.adapt(leaves, adapt.mark_fraction(sol['eta']))
    assert E[0] > E[1] > E[2], E
