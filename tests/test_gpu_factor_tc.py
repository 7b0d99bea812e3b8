"""Element factorisation with tensor-core trailing updates (DPG_FACTOR_TC_SPLIT) against exact and FP64 results.

The augmented element matrix of Sec. 2.3 is eliminated by a blocked partial
Cholesky; the trailing updates A -= P P^H run on FP16 tensor-core MMAs
through an error-free integer splitting of the panel rows.  Checks:
* exactness: with an identity diagonal block the panel is the given integer
  block, and one panel's update A - P P^H of integers below 2^20 is exactly
  representable, so the kernel must reproduce it bit for bit (every digit
  level and the recombination take part);
* FP64 accuracy: random Hermitian positive definite and augmented saddle
  matrices (ragged sizes, real and complex) against numpy's Cholesky and
  Schur complement, at the accuracy of the FP64 kernel;
* element level: S_K of lossy, jittered elements p = 1..3 against the oracle
  within 2 eps kappa(G_K), the per-element bound of the FP64 path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import element as oel
from oracle import system as osys
from paper_2609_03155_b300 import inputs


@pytest.fixture(scope="module")
def dpg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_03155_b300 import dpg
    return dpg


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("N", [70, 291])
def test_one_panel_update_is_exact_on_integers(dpg_mod, cplx, N):
    rng = np.random.default_rng(7 + N)
    A = np.zeros((N, N), complex if cplx else float)
    A[:32, :32] = np.eye(32)
    P = rng.integers(-2 ** 20, 2 ** 20, (N - 32, 32)).astype(float)
    if cplx:
        P = P + 1j * rng.integers(-2 ** 20, 2 ** 20, (N - 32, 32))
    P[5] = 0.0  # a zero row
    P[7, :] = np.where(np.arange(32) % 3 == 0, 1.0, 0.0)  # tiny entries next to large rows
    A[32:, :32] = P
    T = rng.integers(-2 ** 40, 2 ** 40, (N - 32, N - 32)).astype(float)
    if cplx:
        T = T + 1j * rng.integers(-2 ** 40, 2 ** 40, (N - 32, N - 32))
    A[32:, 32:] = np.tril(T)
    out, bad = dpg_mod.factor_check(A, nv=32, npiv=32)
    assert not bad
    want = np.tril(T - P @ P.conj().T)
    got = np.tril(out[32:, 32:])
    if cplx:  # the diagonal's imaginary part is not part of the result
        got = got - 1j * np.diag(np.diag(got).imag)
        want = want - 1j * np.diag(np.diag(want).imag)
    assert np.array_equal(got, want)
    assert np.array_equal(out[32:, :32], P)


def _hpd(rng, n, cplx, cond=1e6):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0))
    lam = np.geomspace(1.0, 1.0 / cond, n)
    D = np.exp(rng.uniform(-3, 3, n))  # uneven row scales, as in G_K
    return D[:, None] * (Q * lam) @ Q.conj().T * D[None, :]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("N", [100, 433])
def test_cholesky_matches_numpy_and_fp64_kernel(dpg_mod, cplx, N):
    rng = np.random.default_rng(N + 3 * cplx)
    G = _hpd(rng, N, cplx)
    L_ref = np.linalg.cholesky(G)
    L_tc, bad = dpg_mod.factor_check(G, nv=N, npiv=N)
    assert not bad
    L64, bad64 = dpg_mod.factor_check(G, nv=N, npiv=N, arith=0)
    assert not bad64
    L_tc, L64 = np.tril(L_tc), np.tril(L64)
    e_tc, e64 = rel(L_tc, L_ref), rel(L64, L_ref)
    # same accuracy class as the FP64 kernel (both are backward stable; the
    # forward error of a Cholesky factor grows with cond(G) ~ 1e6 here)
    assert e_tc < max(10 * e64, 1e-12), (e_tc, e64)
    # backward errors: the tensor-core factor's is of the FP64 kernel's size
    bw_tc = np.linalg.norm(L_tc @ L_tc.conj().T - G) / np.linalg.norm(G)
    bw64 = np.linalg.norm(L64 @ L64.conj().T - G) / np.linalg.norm(G)
    assert bw_tc < 10 * bw64 + 1e-15, (bw_tc, bw64)


@pytest.mark.parametrize("cplx", [False, True])
def test_augmented_condensation_matches_schur_complement(dpg_mod, cplx):
    """[[G, B], [B^H, 0]]: nv pivots, sign flip, nu pivots -> S = M3 - M2^H M1^-1 M2 with M = B^H G^-1 B."""
    rng = np.random.default_rng(11 + cplx)
    nv, nu, nh = 300, 81, 97
    m = nu + nh + 1
    N = nv + m
    G = _hpd(rng, nv, cplx, cond=1e7)
    B = rng.standard_normal((nv, m)) + (1j * rng.standard_normal((nv, m)) if cplx else 0)
    A = np.zeros((N, N), complex if cplx else float)
    A[:nv, :nv] = G
    A[nv:, :nv] = B.conj().T
    M = B.conj().T @ np.linalg.solve(G, B)
    S_ref = M[nu:, nu:] - M[nu:, :nu] @ np.linalg.solve(M[:nu, :nu], M[:nu, nu:])
    for arith in (1, 0):
        out, bad = dpg_mod.factor_check(A, nv=nv, npiv=nv + nu, arith=arith)
        assert not bad
        S = np.tril(out[nv + nu:, nv + nu:])
        S = S + np.tril(S, -1).conj().T
        err = rel(S, S_ref)
        if arith == 1:
            e_tc = err
        else:
            e64 = err
    assert e_tc < max(10 * e64, 1e-10), (e_tc, e64)


def _lossy_jittered(p, seed=11):
    nx, ny, nz = 2, 2, 1
    vert, elem, ijk = inputs.structured_hex(0.3, 0.2, 0.1, nx, ny, nz)
    rng = np.random.default_rng(seed)
    inner = (vert > 1e-12) & (vert < np.array([0.3, 0.2, 0.1]) - 1e-12)
    vert = vert + inner * rng.uniform(-0.012, 0.012, vert.shape)
    spec = {'x0': (inputs.BC_DIRICHLET, 0), 'x1': (inputs.BC_DIRICHLET, 1), 'y0': (inputs.BC_DIRICHLET, 0),
            'y1': (inputs.BC_DIRICHLET, 0), 'z0': (inputs.BC_ROBIN, 0), 'z1': (inputs.BC_ROBIN, 1)}
    bc, grp = inputs.box_boundary_tags(ijk, nx, ny, nz, spec)
    ne = elem.shape[0]
    eps = np.exp(rng.uniform(0, np.log(10), ne)) + 1j * rng.uniform(0, 3, ne)
    eps[1] = 4.0  # one lossless element without a Robin face: the real path
    mu = np.ones(ne, complex)
    omega = 9.0
    zinv = inputs.te_zinv(omega, 0.3, 0.2, 1, 0)
    return inputs.Mesh(vert=vert, elem=elem, p=np.full(ne, p, np.int8), eps=eps, mu=mu, face_bc=bc,
                       face_grp=grp, omega=omega,
                       robin=[{'zinv': zinv, 'port': (0.3, 0.2, 1, 0, 1.0, 1.0)}, {'zinv': 0.7 - 0.2j, 'port': None}],
                       dirichlet=[{'kind': inputs.DIRICHLET_ZERO, 'port': None},
                                  {'kind': inputs.DIRICHLET_SIN_PI_X2, 'port': None}],
                       name=f"lossy_jittered_p{p}")


@pytest.mark.parametrize("p", [1, 2, 3])
def test_condensed_element_matrices_match_oracle(dpg_mod, p):
    mesh = _lossy_jittered(p)
    ids = [0, 1, 2, 3]
    d = dpg_mod.DPG(mesh)
    d.set_factor_arith(1)
    out = d.element_dump(ids)
    d.set_factor_arith(0)
    out64 = d.element_dump(ids)
    d.destroy()
    for k, e in enumerate(ids):
        X = mesh.vert[mesh.elem[e]]
        el = oel.element_matrices(X, p, mesh.omega, complex(mesh.eps[e]), complex(mesh.mu[e]),
                                  osys.element_faces(mesh, e))
        cond = oel.condense(el)
        tol = 2 * 2.0 ** -53 * np.linalg.cond(el.G)  # 2 eps kappa(G_K), as for the FP64 kernel
        assert rel(out['S'][k], cond['S']) < tol, (e, rel(out['S'][k], cond['S']), rel(out64['S'][k], cond['S']), tol)
        if np.linalg.norm(cond['s']) > 0:
            assert rel(out['s'][k], cond['s']) < tol
