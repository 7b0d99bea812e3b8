"""Reference-cube bases and Gauss quadrature for the oracle (test infrastructure only).

Reference cube [0,1]^3.  Sec. 2.3 of the paper fixes the spaces:

* interior trial: each Cartesian component of E and H is a discontinuous
  tensor Lagrange polynomial of degree p in each direction;
* trace and test: Nedelec elements of the first kind (test enriched by dp).

Our index convention (the reading of Fig. 1 and the DoF counts of Sec. 4.1):
the Nedelec space of FEEC order r, Q^-_r Lambda^1, has for each component c
the scalar functions  l^open_{i_c}(x_c) * prod_{d != c} l^closed_{i_d}(x_d)
times the unit vector e_c, where ``open`` is the Lagrange basis on the r
Gauss-Legendre points (degree r-1) and ``closed`` the Lagrange basis on the
r+1 Gauss-Lobatto points (degree r).  Functions are ordered component-major
(c = 0, 1, 2) and, inside a component, lexicographically with i_0 fastest.
"""
import numpy as np


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0,1] (exact for degree 2n-1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_lobatto_nodes(n):
    """n >= 2 Gauss-Lobatto points on [0,1]: endpoints and the roots of P'_{n-1}."""
    if n < 2:
        raise ValueError("Gauss-Lobatto needs at least two points")
    inner = np.polynomial.legendre.Legendre.basis(n - 1).deriv().roots()
    x = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    return 0.5 * (x + 1.0)


def lagrange_1d(nodes, x):
    """Values and first derivatives of the Lagrange polynomials on ``nodes`` at ``x``.

    Returns (V, D), each of shape (len(x), len(nodes)), V[q, j] = l_j(x_q).
    Written directly as products (plain definition, no barycentric tricks).
    """
    nodes = np.asarray(nodes, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = len(nodes)
    V = np.ones((len(x), n))
    D = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                V[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
        for k in range(n):
            if k == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[k]))
            for m in range(n):
                if m != j and m != k:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            D[:, j] += term
    return V, D


def nedelec_index(r):
    """List of (c, (i0, i1, i2)) for Q^-_r Lambda^1 in the oracle's ordering."""
    out = []
    for c in range(3):
        n = [r + 1, r + 1, r + 1]
        n[c] = r
        for i2 in range(n[2]):
            for i1 in range(n[1]):
                for i0 in range(n[0]):
                    out.append((c, (i0, i1, i2)))
    return out


def nedelec_eval(r, pts):
    """Reference Nedelec basis of FEEC order r at points ``pts`` (N, 3).

    Returns (val, curl), each (N, nbasis, 3): the reference vector value f e_c
    and its reference curl grad(f) x e_c.
    """
    pts = np.asarray(pts, dtype=float)
    closed = gauss_lobatto_nodes(r + 1)
    opn = gauss_legendre(r)[0]
    tab = []  # tab[d][kind] = (V, D) with kind 0 = open, 1 = closed
    for d in range(3):
        tab.append((lagrange_1d(opn, pts[:, d]), lagrange_1d(closed, pts[:, d])))
    idx = nedelec_index(r)
    N = pts.shape[0]
    val = np.zeros((N, len(idx), 3))
    curl = np.zeros((N, len(idx), 3))
    for k, (c, ii) in enumerate(idx):
        f = np.ones(N)
        grad = np.ones((N, 3))
        for d in range(3):
            V, D = tab[d][0] if d == c else tab[d][1]
            f = f * V[:, ii[d]]
            for g in range(3):
                grad[:, g] *= D[:, ii[d]] if g == d else V[:, ii[d]]
        val[:, k, c] = f
        e = np.zeros(3)
        e[c] = 1.0
        curl[:, k, :] = np.cross(grad, e[None, :])
    return val, curl


def lagrange3_eval(p, pts):
    """Scalar tensor Lagrange basis of degree p on (p+1) Gauss-Legendre nodes.

    Returns (N, (p+1)^3) values, lexicographic with the x0 index fastest.
    """
    pts = np.asarray(pts, dtype=float)
    nodes = gauss_legendre(p + 1)[0]
    V = [lagrange_1d(nodes, pts[:, d])[0] for d in range(3)]
    n = p + 1
    out = np.zeros((pts.shape[0], n ** 3))
    for a2 in range(n):
        for a1 in range(n):
            for a0 in range(n):
                out[:, a0 + n * (a1 + n * a2)] = V[0][:, a0] * V[1][:, a1] * V[2][:, a2]
    return out


def nedelec_nodes(r):
    """Reference node of each Q^-_r Lambda^1 function (its Lagrange node), (nbasis, 3)."""
    closed = gauss_lobatto_nodes(r + 1)
    opn = gauss_legendre(r)[0]
    out = []
    for c, ii in nedelec_index(r):
        out.append([opn[ii[d]] if d == c else closed[ii[d]] for d in range(3)])
    return np.array(out)


def trace_entity(r, c, ii):
    """Entity of a Nedelec function on the reference cube, or None if interior.

    Returns ('edge', c, (d1, s1), (d2, s2)) for a function whose two transverse
    closed indices both sit on the boundary, ('face', d, s) for exactly one
    (normal direction d, side s in {0, 1}), else None (interior function, whose
    tangential trace vanishes on every face and is discarded, Sec. 2.3).
    """
    hits = []
    for d in range(3):
        if d == c:
            continue
        if ii[d] == 0:
            hits.append((d, 0))
        elif ii[d] == r:
            hits.append((d, 1))
    if len(hits) == 2:
        return ('edge', c, hits[0], hits[1])
    if len(hits) == 1:
        return ('face', hits[0][0], hits[0][1])
    return None


def trace_functions(r):
    """Indices (into nedelec_index(r)) of the 12 r^2 trace functions, in order."""
    return [k for k, (c, ii) in enumerate(nedelec_index(r)) if trace_entity(r, c, ii) is not None]


def dims(p, dp=1):
    """Per-element sizes (n_f, n_v, n_u, n_h) for trial degree p and enrichment dp."""
    rt = p + 1 + dp
    r = p + 1
    n_f = 3 * rt * (rt + 1) ** 2
    return n_f, 2 * n_f, 6 * (p + 1) ** 3, 2 * 12 * r * r
