"""CUDA path (through the C ABI) against the CPU oracle, element by element and field by field.

Tolerances (each follows from the arithmetic of its step):
* G_K, B_K, B-hat_K, l_K (formation, well conditioned): relative Frobenius 1e-12.
* S_K, s_K (after G_K^{-1}): relative Frobenius 2 eps kappa(G_K) per element
  (eps = 2^-53), the forward-error scale of a backward-stable solve with G_K;
  two FP64 routes of the oracle itself (Cholesky, explicit inverse) differ by
  1/15 to 1/25 of eps kappa(G_K) on these elements.  On the full-size guide
  (kappa ~ 5e8) the bound is the tighter of that and ten times the measured
  two-route floor of the element.
* trace solution and interior field vs the oracle's direct solve: relative 1e-10
  (CG run to 1e-13 relative residual).
* eta_K (Sec. 2.3, ||Psi_K||_V = ||L^{-1} r_K||): per element, relative 1e-9,
  against the oracle's eta_K at the same trace solution (the GPU's), so that
  the comparison isolates the estimator.  Both sides form r_K = l - B u - B-hat uhat
  and apply L^{-1}; the oracle's own two routes (Cholesky and eigen) agree
  to ~1e-11 per element on these cases.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import element as oel
from oracle import system as osys
from paper_2609_03155_b300 import inputs


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def dpg_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_03155_b300 import dpg
    return dpg


def _lossy_jittered(p, n=(2, 2, 1), seed=11):
    """Small box with jittered interior vertices, lossy random materials, PEC + Robin port + Dirichlet data."""
    nx, ny, nz = n
    vert, elem, ijk = inputs.structured_hex(0.3, 0.2, 0.1 * nz, nx, ny, nz)
    rng = np.random.default_rng(seed)
    inner = (vert > 1e-12) & (vert < np.array([0.3, 0.2, 0.1 * nz]) - 1e-12)
    vert = vert + inner * rng.uniform(-0.012, 0.012, vert.shape)
    spec = {'x0': (inputs.BC_DIRICHLET, 0), 'x1': (inputs.BC_DIRICHLET, 1), 'y0': (inputs.BC_DIRICHLET, 0),
            'y1': (inputs.BC_DIRICHLET, 0), 'z0': (inputs.BC_ROBIN, 0), 'z1': (inputs.BC_ROBIN, 1)}
    bc, grp = inputs.box_boundary_tags(ijk, nx, ny, nz, spec)
    ne = elem.shape[0]
    eps = np.exp(rng.uniform(0, np.log(10), ne)) + 1j * rng.uniform(0, 3, ne)
    mu = 1.0 + 0.2 * rng.uniform(0, 1, ne) + 0.1j * rng.uniform(0, 1, ne)
    omega = 9.0
    zinv = inputs.te_zinv(omega, 0.3, 0.2, 1, 0)
    return inputs.Mesh(vert=vert, elem=elem, p=np.full(ne, p, np.int8), eps=eps, mu=mu, face_bc=bc,
                       face_grp=grp, omega=omega,
                       robin=[{'zinv': zinv, 'port': (0.3, 0.2, 1, 0, 1.0, 1.0)}, {'zinv': 0.7 - 0.2j, 'port': None}],
                       dirichlet=[{'kind': inputs.DIRICHLET_ZERO, 'port': None},
                                  {'kind': inputs.DIRICHLET_SIN_PI_X2, 'port': None}],
                       name=f"lossy_jittered_p{p}")


EPS64 = 2.0 ** -53


def s_bound(el):
    """Per-element bound on the relative error of S_K, s_K: 2 eps kappa(G_K)."""
    return 2 * EPS64 * np.linalg.cond(el.G)


def _oracle_element(mesh, e):
    X = mesh.vert[mesh.elem[e]]
    el = oel.element_matrices(X, int(mesh.p[e]), mesh.omega, complex(mesh.eps[e]), complex(mesh.mu[e]),
                              osys.element_faces(mesh, e))
    return el, oel.condense(el)


@pytest.mark.parametrize("case", ["waveguide2d_p1", "lossy_p1", "lossy_p2", "lossy_p3", "lossy_p4"])
def test_element_matrices_match_oracle(dpg_mod, case):
    if case == "waveguide2d_p1":
        mesh = inputs.waveguide_2d_config(p=1)
        ids = [0, 9, 20, 31]  # 0, 31: port / impedance faces (complex path); 9, 20: lossless (real path)
    else:
        p = int(case[-1])
        mesh = _lossy_jittered(p)
        ids = [0, 1, 2, 3] if p < 4 else [0, 1]  # the p = 4 oracle takes seconds per element
    d = dpg_mod.DPG(mesh)
    out = d.element_dump(ids)
    for k, e in enumerate(ids):
        el, cond = _oracle_element(mesh, e)
        assert rel(out['G'][k], el.G) < 1e-12
        assert rel(out['B'][k], el.B) < 1e-12
        assert rel(out['Bh'][k], el.Bh) < 1e-12
        if np.linalg.norm(el.l) > 0:
            assert rel(out['l'][k], el.l) < 1e-12
        else:
            assert np.linalg.norm(out['l'][k]) == 0
        tol = s_bound(el)
        assert rel(out['S'][k], cond['S']) < tol, (e, rel(out['S'][k], cond['S']), tol)
        if np.linalg.norm(cond['s']) > 0:
            assert rel(out['s'][k], cond['s']) < tol
    d.destroy()


def _gather(d, x):
    """Element-local trace vectors of a global GPU solution (through the library's own map)."""
    m, fv = d.trace_map()
    xn = x.cpu().numpy()
    loc = np.where(m >= 0, xn[np.clip(m, 0, None)], 0)
    loc = np.where(m == -1, fv, loc)
    return loc


@pytest.mark.parametrize("case", ["waveguide2d_p1", "lossy_p1", "lossy_p2"])
def test_solution_matches_oracle_direct_solve(dpg_mod, case):
    if case == "waveguide2d_p1":
        mesh = inputs.waveguide_2d_config(p=1)
    else:
        mesh = _lossy_jittered(int(case[-1]), n=(2, 2, 2))
    sol = osys.solve(mesh)
    d = dpg_mod.DPG(mesh)
    assert d.n == sol['n']
    d.element_batch()
    d.assemble()
    x, rep = d.cg_solve(rtol=1e-13, max_iter=200000)
    assert rep['converged']
    uh = _gather(d, x)
    uh_or = np.stack([sol['xfull'][g] for g in sol['l2g']])
    assert rel(uh, uh_or) < 1e-10
    u, eta, etag = d.estimate(x)
    u_or = np.stack([r['u'] for r in sol['rec']])
    assert rel(u.cpu().numpy(), u_or) < 1e-10
    # the oracle's estimator at the GPU's trace solution, element by element
    eta_or = np.array([oel.recover(sol['elements'][e], sol['conds'][e], uh[e])['eta'] for e in range(len(uh))])
    eta_g = eta.cpu().numpy()
    assert np.all(np.abs(eta_g - eta_or) <= 1e-9 * eta_or), np.max(np.abs(eta_g - eta_or) / eta_or)
    assert abs(etag - np.sqrt(np.sum(eta_or ** 2))) < 1e-9 * np.sqrt(np.sum(eta_or ** 2))
    assert d.estimate_clamped() == 0
    d.destroy()


def test_assembled_matrix_is_hermitian_and_matches_oracle_energy(dpg_mod):
    """CSR is Hermitian; x^H A x and x^H b agree with the oracle's assembled system for the same local vectors."""
    mesh = _lossy_jittered(1, n=(2, 1, 2))
    sol = osys.solve(mesh)
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    rp, col, val, b = d.csr_copy()
    import scipy.sparse as sp
    A = sp.csr_matrix((val, col, rp), shape=(d.n, d.n))
    assert abs(A - A.conj().T).max() <= 1e-12 * abs(A).max()
    # same physical trace field expressed in both numberings: use the oracle solution
    m, fv = d.trace_map()
    xg = np.zeros(d.n, complex)
    for e in range(mesh.n_elem):
        loc = sol['xfull'][sol['l2g'][e]]
        for t in range(d.n_h):
            if m[e, t] >= 0:
                xg[m[e, t]] = loc[t]
    Ao = sol['A']
    xo = sol['x']
    assert abs(np.vdot(xg, A @ xg) - np.vdot(xo, Ao @ xo)) < 1e-9 * abs(np.vdot(xo, Ao @ xo))
    assert abs(np.vdot(xg, b) - np.vdot(xo, sol['b'])) < 1e-9 * abs(np.vdot(xo, sol['b']))
    d.destroy()


def test_te10_waveguide_field_error(dpg_mod):
    """Config-1 guide: GPU field vs the closed-form TE10 mode (same error as the oracle's)."""
    mesh = inputs.waveguide_2d_config(p=1)
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    x, rep = d.cg_solve(rtol=1e-12)
    u, eta, etag = d.estimate(x)
    from oracle import physics
    res = {'rec': [{'u': ue} for ue in u.cpu().numpy()]}
    ex = lambda y: physics.te_fields(y, mesh.omega, 0.086, mesh.vert[:, 1].max(), 1, 0)
    eE, eH = osys.l2_field_error(mesh, res, ex)
    assert eE < 0.01 and eH < 0.01
    d.destroy()


@pytest.mark.parametrize("mode", [1, 2, 3, 4, 5, 1 | 16, 5 | 16, 5 | 32, 64, 64 | 4, 1 | 128, 5 | 128, 5 | 128 | 512,
                                  5 | 256, 5 | 128 | 256, 5 | 32 | 256])
def test_cg_modes_match_fp64(dpg_mod, mode):
    """IR (FP32 inner: full or Hermitian half storage or element by element, FP32 or FP64 inner vectors),
    Jacobi, entity-block Jacobi and the double-word (FP32 pair) solver reach the plain FP64 CG solution."""
    mesh = _lossy_jittered(1, n=(2, 2, 2))
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    x64, r64 = d.cg_solve(rtol=1e-12)
    xm, rm = d.cg_solve(mode=mode, rtol=1e-12, inner_rtol=1e-4)
    assert rm['converged'] and rm['rel_residual'] <= 1e-12
    if mode & 1:
        assert rm['outer'] >= 1
    if mode & 6:
        assert rm['iterations'] < r64['iterations']
    assert rel(xm.cpu().numpy(), x64.cpu().numpy()) < 1e-9
    d.destroy()


def test_deterministic_assembly_and_solve(dpg_mod):
    mesh = _lossy_jittered(1, n=(2, 2, 1))
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    _, _, v1, b1 = d.csr_copy()
    x1, _ = d.cg_solve(rtol=1e-12)
    d.element_batch()
    d.assemble()
    _, _, v2, b2 = d.csr_copy()
    x2, _ = d.cg_solve(rtol=1e-12)
    assert np.array_equal(v1, v2) and np.array_equal(b1, b2)
    assert torch.equal(x1, x2)
    # the element-by-element inner operator sums every row's slots in one fixed order
    x3, _ = d.cg_solve(mode=5 | 128, rtol=1e-12)
    x4, _ = d.cg_solve(mode=5 | 128, rtol=1e-12)
    assert torch.equal(x3, x4)
    d.destroy()


def test_element_by_element_operator_on_mixed_degrees_and_hanging_faces(dpg_mod):
    """Per-element slot counts differ (orders 1..4) and restricted elements
    map slots through the hanging-face constraints: the element-by-element
    inner solves must still reach the FP64 solution."""
    for mesh in (inputs.fichera_cavity(2, grade=1.5, mix=(0.4, 0.3, 0.3)), inputs.fichera_amr(2, radius=0.5)):
        d = dpg_mod.DPG(mesh)
        d.element_batch()
        d.assemble()
        x64, _ = d.cg_solve(rtol=1e-12, max_iter=200000)
        xe, re_ = d.cg_solve(mode=5 | 128, rtol=1e-12, max_iter=200000, inner_rtol=1e-4)
        assert re_['converged']
        assert rel(xe.cpu().numpy(), x64.cpu().numpy()) < 1e-9
        d.destroy()


def _obstacle_cavity(n=3, p=1):
    m = inputs.cavity(n, p, omega=5.0)
    mask = inputs.sphere_obstacle(m, radius=0.3, eps=20.0 + 5.0j)
    return m, mask


def test_adjoint_gradient_matches_oracle(dpg_mod):
    from oracle import adjoint as oadj
    m, mask = _obstacle_cavity(2, 1)
    mask[:] = False
    mask[[0, 3, 5]] = True
    m.eps = m.eps.copy()
    m.eps[mask] = 20 + 5j
    m.eps[1] = 3 + 1j
    sol = osys.solve(m)
    P_or, dre_or, dim_or = oadj.gradient(m, sol, mask)
    d = dpg_mod.DPG(m, adjoint=True)
    d.element_batch()
    d.assemble()
    x, rep = d.cg_solve(rtol=1e-13)
    mk = torch.tensor(mask.astype(np.uint8), device='cuda')
    P, dre, dim = d.grad_eps(x, mk, rtol=1e-13)
    assert abs(P - P_or) < 1e-10 * P_or
    scale = max(np.abs(dre_or).max(), np.abs(dim_or).max())
    assert np.abs(dre.cpu().numpy() - dre_or).max() < 1e-8 * scale
    assert np.abs(dim.cpu().numpy() - dim_or).max() < 1e-8 * scale
    d.destroy()


def test_adjoint_gradient_matches_gpu_finite_differences(dpg_mod):
    """Central differences (step 1e-6) of GPU solves on 20 seeded elements, 10 inside the obstacle."""
    m, mask = _obstacle_cavity(4, 1)
    d = dpg_mod.DPG(m, adjoint=True)
    mk = torch.tensor(mask.astype(np.uint8), device='cuda')
    eps0 = torch.tensor(m.eps, dtype=torch.complex128)
    Pfun = lambda e: dpg_mod.AbsorbedPower.apply(e, d, mk, 1e-13)
    eps = eps0.clone().requires_grad_(True)
    P = Pfun(eps)
    P.backward()
    g = eps.grad.numpy()
    rng = np.random.default_rng(20260903)
    inside, outside = np.where(mask)[0], np.where(~mask)[0]
    pick = list(rng.choice(inside, min(10, len(inside)), replace=False)) + \
        list(rng.choice(outside, 20 - min(10, len(inside)), replace=False))
    h = 1e-6
    scale = np.abs(g).max()
    for e in pick:
        for part in (1.0, 1j):
            ep, em = eps0.clone(), eps0.clone()
            ep[e] += part * h
            em[e] -= part * h
            with torch.no_grad():
                fd = (Pfun(ep).item() - Pfun(em).item()) / (2 * h)
            an = g[e].real if part == 1.0 else g[e].imag
            assert abs(an - fd) < 1e-5 * scale + 1e-9 * abs(P.item()), (e, part, an, fd)
    d.destroy()


def test_real_path_matches_complex_path(dpg_mod):
    """Lossless elements: the phase-scaled real factorisation gives the complex path's S_K, Z_K and field."""
    mesh = inputs.waveguide_3d_config(4, 2, 6, p=2)
    d = dpg_mod.DPG(mesh)
    inner = [e for e in range(mesh.n_elem) if not (mesh.face_bc[e] == 2).any()][:6]
    assert inner
    d.set_real_path(True)
    out_r = d.element_dump(inner)
    d.element_batch()
    d.assemble()
    x_r, _ = d.cg_solve(rtol=1e-13)
    u_r, eta_r, _ = d.estimate(x_r)
    d.set_real_path(False)
    out_c = d.element_dump(inner)
    d.element_batch()
    d.assemble()
    x_c, _ = d.cg_solve(rtol=1e-13)
    u_c, eta_c, _ = d.estimate(x_c)
    for k in range(len(inner)):
        assert rel(out_r['S'][k], out_c['S'][k]) < 1e-10
    assert rel(x_r.cpu().numpy(), x_c.cpu().numpy()) < 1e-10
    assert rel(u_r.cpu().numpy(), u_c.cpu().numpy()) < 1e-10
    er, ec = eta_r.cpu().numpy(), eta_c.cpu().numpy()
    assert np.all(np.abs(er - ec) <= 1e-9 * ec), np.max(np.abs(er - ec) / ec)
    d.destroy()


def test_cg_warm_start_resumes_a_stopped_solve(dpg_mod):
    """DPG_CG_X0: a solve stopped at 1e-5 and resumed reaches the cold solve's answer with fewer new iterations."""
    from paper_2609_03155_b300 import _lib
    mesh = inputs.waveguide_3d_config(4, 2, 6, p=2)
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    x_cold, rep_cold = d.cg_solve(rtol=1e-12, max_iter=100000)
    x, rep1 = d.cg_solve(rtol=1e-5, max_iter=100000)
    x, rep2 = d.cg_solve(x=x, mode=_lib.DPG_CG_FP64 | _lib.DPG_CG_X0, rtol=1e-12, max_iter=100000)
    assert rep2['converged'] and rep2['iterations'] < rep_cold['iterations']
    assert rel(x.cpu().numpy(), x_cold.cpu().numpy()) < 1e-9
    d.destroy()


def _condensation_floor(el, S):
    """Relative difference of S between two backward-stable FP64 routes (Cholesky, as the oracle does,
    and the explicit inverse of G): how closely any FP64 condensation of this element can agree."""
    BB = np.hstack([el.B, el.Bh])
    A = BB.conj().T @ np.linalg.inv(el.G) @ BB
    nu = el.B.shape[1]
    S_alt = A[nu:, nu:] - A[:nu, nu:].conj().T @ np.linalg.solve(A[:nu, :nu], A[:nu, nu:])
    return rel(S_alt, S)


def test_full_size_waveguide_sampled_elements(dpg_mod):
    """The 32x16x64 p=2 guide at full size (32,768 elements, the bench workload): element matrices of
    sampled elements (port corner, interior, wall, outlet) against the oracle, one by one.  These
    elements are small against the wavelength and G_K has kappa ~ 5e8, so the S_K bound is the tighter
    of 2 eps kappa(G_K) and ten times the disagreement of two FP64 routes on the same element."""
    mesh = inputs.waveguide_3d_config(32, 16, 64, 2)
    d = dpg_mod.DPG(mesh)
    ids = [0, 32 * 16 * 30 + 16 * 8 + 16, 32 * 16 * 40 + 31, mesh.n_elem - 1]
    out = d.element_dump(ids)
    d.destroy()
    for k, e in enumerate(ids):
        el, cond = _oracle_element(mesh, e)
        assert rel(out['G'][k], el.G) < 1e-12
        assert rel(out['B'][k], el.B) < 1e-12
        assert rel(out['Bh'][k], el.Bh) < 1e-12
        assert rel(out['S'][k], cond['S']) < min(s_bound(el), 10 * _condensation_floor(el, cond['S']))


def test_cg_reports_non_convergence(dpg_mod):
    from paper_2609_03155_b300 import _lib
    mesh = inputs.waveguide_3d_config(4, 2, 6, p=2)
    d = dpg_mod.DPG(mesh)
    d.element_batch()
    d.assemble()
    with pytest.raises(_lib.DPGError, match="NOT_CONVERGED"):
        d.cg_solve(rtol=1e-12, max_iter=5)
    x, rep = d.cg_solve(rtol=1e-12, max_iter=5, raise_on_nonconvergence=False)
    assert not rep['converged'] and rep['iterations'] <= 5
    d.destroy()
