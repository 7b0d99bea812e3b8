"""Fixed-fraction (Doerfler-type) marking for the adaptive loop of Sec. 4.2 (test infrastructure only).

Sec. 4.2 ranks the cells by their residual norm eta_K = ||Psi_K||_V and marks
the largest for refinement until their combined share reaches 30 % of the
total, and the smallest for coarsening until their combined share reaches
5 % (parameter table of App. C.2: refinement fraction 0.30, coarsening
fraction 0.05).  Reading taken here (the paper names the fractions but not
the measure): shares are of sum_K eta_K ("their combined residual", power 1,
the default) or of sum_K eta_K^2 (power 2, Doerfler's bulk criterion on the
squared global estimate of Sec. 4.2); refinement takes the smallest set of largest
cells whose sum reaches the fraction (the cell that crosses it included);
coarsening takes the largest set of smallest cells whose sum stays within
its fraction; a cell marked for refinement is never marked for coarsening;
ties are ordered by element index.
"""
import numpy as np


def mark_fraction(eta, refine=0.30, coarsen=0.05, power=1):
    """Marks per element: +1 refine, -1 coarsen, 0 keep."""
    e2 = np.abs(np.asarray(eta, dtype=np.float64)) ** power
    ne = e2.shape[0]
    total = float(np.sum(e2))
    marks = np.zeros(ne, dtype=np.int8)
    if ne == 0 or total <= 0.0:
        return marks
    idx = np.arange(ne)
    down = sorted(idx, key=lambda e: (-e2[e], e))  # largest first
    acc = 0.0
    for e in down:
        if acc >= refine * total:
            break
        marks[e] = 1
        acc += e2[e]
    acc = 0.0
    for e in reversed(down):  # smallest first
        if marks[e] == 1 or acc + e2[e] > coarsen * total:
            break
        marks[e] = -1
        acc += e2[e]
    return marks
