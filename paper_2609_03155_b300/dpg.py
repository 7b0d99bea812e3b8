"""Python face of the C ABI: one class per handle, methods named after the ABI calls.

Marshalling only: numpy mesh arrays become the C descriptor, torch CUDA
tensors carry device buffers, torch streams carry the stream handle.  All
arithmetic of the method runs in libdpg.so.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import DPGError, check, ptr, stream_handle  # noqa: F401 (DPGError re-exported)


def _robin_groups(mesh):
    arr = (_lib.dpg_robin_group * max(1, len(mesh.robin)))()
    for k, g in enumerate(mesh.robin):
        z = complex(g['zinv'])
        arr[k].zinv_re, arr[k].zinv_im = z.real, z.imag
        port = g.get('port')
        if port is not None:
            a, b, m, n, eps, mu = port
            arr[k].port, arr[k].m, arr[k].n, arr[k].a, arr[k].b = 1, m, n, a, b
            arr[k].eps_re, arr[k].eps_im = complex(eps).real, complex(eps).imag
            arr[k].mu_re, arr[k].mu_im = complex(mu).real, complex(mu).imag
    return arr


def _dirichlet_groups(mesh):
    arr = (_lib.dpg_dirichlet_group * max(1, len(mesh.dirichlet)))()
    for k, g in enumerate(mesh.dirichlet):
        arr[k].kind = int(g['kind'])
        port = g.get('port')
        if port is not None:
            a, b, m, n, eps, mu = port
            arr[k].m, arr[k].n, arr[k].a, arr[k].b = m, n, a, b
            arr[k].eps_re, arr[k].eps_im = complex(eps).real, complex(eps).imag
            arr[k].mu_re, arr[k].mu_im = complex(mu).real, complex(mu).imag
    return arr


def element_sizes(p, dp=1):
    """(n_v, n_u, n_h) of one element of trial degree p."""
    r, rt = p + 1, p + 1 + dp
    return 6 * rt * (rt + 1) ** 2, 6 * (p + 1) ** 3, 24 * r * r


class DPG:
    """A DPG discretisation living on the current CUDA device (dpg_handle)."""

    def __init__(self, mesh, alpha=1.0, chunk=0, adjoint=False, precision=0, stream=None, streaming=False):
        L = _lib.lib()
        self.mesh = mesh
        self.factor_arith = _lib.DPG_FACTOR_TC_SPLIT  # the library's default
        self.bucketed = False
        keep = dict(
            vert=np.ascontiguousarray(mesh.vert, dtype=np.float64),
            elem=np.ascontiguousarray(mesh.elem, dtype=np.int32),
            p=np.ascontiguousarray(mesh.p, dtype=np.int8),
            eps=np.ascontiguousarray(mesh.eps, dtype=np.complex128),
            mu=np.ascontiguousarray(mesh.mu, dtype=np.complex128),
            bc=np.ascontiguousarray(mesh.face_bc, dtype=np.int8),
            grp=np.ascontiguousarray(mesh.face_grp, dtype=np.int16),
        )
        rob, dirg = _robin_groups(mesh), _dirichlet_groups(mesh)
        desc = _lib.dpg_mesh_desc(
            n_vert=keep['vert'].shape[0], vert=keep['vert'].ctypes.data, n_elem=keep['elem'].shape[0],
            elem=keep['elem'].ctypes.data, elem_p=keep['p'].ctypes.data, elem_eps=keep['eps'].ctypes.data,
            elem_mu=keep['mu'].ctypes.data, face_bc=keep['bc'].ctypes.data, face_grp=keep['grp'].ctypes.data,
            n_robin=len(mesh.robin), robin=C.cast(rob, C.POINTER(_lib.dpg_robin_group)),
            n_dirichlet=len(mesh.dirichlet), dirichlet=C.cast(dirg, C.POINTER(_lib.dpg_dirichlet_group)))
        prm = _lib.dpg_params(omega=float(mesh.omega), alpha=float(alpha), dp=1, precision=int(precision), chunk=int(chunk),
                              flags=(_lib.DPG_FLAG_ADJOINT if adjoint else 0) | (_lib.DPG_FLAG_STREAM if streaming else 0))
        h = C.c_void_p()
        check(L.dpg_setup_mesh(C.byref(h), C.byref(desc), C.byref(prm), stream_handle(stream)))
        self.h = h
        self.n, self.nnz, self.n_elem, self.n_v, self.n_u, self.n_h = self.sizes()
        self.p_elem, self.u_off, self.h_off = self.element_layout()
        self.uniform = bool(np.all(self.p_elem == self.p_elem[0]))

    # ---- ABI calls -----------------------------------------------------------
    def sizes(self):
        n, nnz = C.c_int64(), C.c_int64()
        ne, nv, nu, nh = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        check(_lib.lib().dpg_sizes(self.h, C.byref(n), C.byref(nnz), C.byref(ne), C.byref(nv), C.byref(nu),
                                   C.byref(nh)), self.h)
        return n.value, nnz.value, ne.value, nv.value, nu.value, nh.value

    def element_layout(self):
        """Per-element trial degree and the offsets of u and of the trace map (n_elem + 1 each)."""
        pe = np.empty(self.n_elem, np.int8)
        uo = np.empty(self.n_elem + 1, np.int64)
        ho = np.empty(self.n_elem + 1, np.int64)
        check(_lib.lib().dpg_element_layout(self.h, ptr(pe), ptr(uo), ptr(ho)), self.h)
        return pe, uo, ho

    def element_batch(self, stream=None):
        check(_lib.lib().dpg_element_batch(self.h, _lib.DPG_PASS_ASSEMBLE, stream_handle(stream)), self.h)

    def assemble(self, stream=None):
        check(_lib.lib().dpg_assemble(self.h, stream_handle(stream)), self.h)

    def cg_solve(self, x=None, b=None, mode=_lib.DPG_CG_FP64, rtol=1e-10, atol=0.0, max_iter=100000,
                 inner_rtol=5e-2, stream=None, raise_on_nonconvergence=True):
        if x is None:
            x = torch.zeros(self.n, dtype=torch.complex128, device='cuda')
        rep = _lib.dpg_cg_report()
        rc = _lib.lib().dpg_cg_solve(self.h, mode, rtol, atol, max_iter, inner_rtol, ptr(x), ptr(b),
                                     C.byref(rep), stream_handle(stream))
        if rc != 0 and (raise_on_nonconvergence or rc != -5):
            check(rc, self.h)
        return x, dict(iterations=rep.iterations, outer=rep.outer, rel_residual=rep.rel_residual, ms=rep.ms,
                       converged=bool(rep.converged))

    def estimate(self, xhat, want_u=True, stream=None):
        """u (n_elem x n_u for one degree, else flat at u_off), eta_K, sqrt(sum eta_K^2)."""
        u = torch.empty(int(self.u_off[-1]), dtype=torch.complex128, device='cuda') if want_u else None
        eta = torch.empty(self.n_elem, dtype=torch.float64, device='cuda')
        tot = C.c_double()
        check(_lib.lib().dpg_estimate(self.h, ptr(xhat), ptr(u), ptr(eta), C.byref(tot), stream_handle(stream)),
              self.h)
        if u is not None and self.uniform:
            u = u.view(self.n_elem, self.n_u)
        return u, eta, tot.value

    def mark_fraction(self, eta, refine=0.30, coarsen=0.05, power=1, stream=None):
        """Per-element marks (+1 refine, -1 coarsen, 0 keep) from eta (device tensor) by fixed fractions."""
        marks = np.zeros(self.n_elem, dtype=np.int8)
        check(_lib.lib().dpg_mark_fraction(self.h, ptr(eta), float(refine), float(coarsen), int(power),
                                           marks.ctypes.data, stream_handle(stream)), self.h)
        return marks

    def estimate_clamped(self):
        c = C.c_int32(0)
        check(_lib.lib().dpg_estimate_clamped(self.h, C.byref(c)), self.h)
        return c.value

    def update_elements(self, corners=None, eps=None, mu=None, stream=None):
        """Host -> device copy of per-element corners (n_elem x 8 x 3), eps, mu (use pinned tensors)."""
        check(_lib.lib().dpg_update_elements(self.h, ptr(corners), ptr(eps), ptr(mu), stream_handle(stream)), self.h)

    def cg_bytes_per_iteration(self, mode):
        b = C.c_int64()
        check(_lib.lib().dpg_cg_bytes_per_iteration(self.h, int(mode), C.byref(b)), self.h)
        return b.value

    def set_real_path(self, enable=True):
        check(_lib.lib().dpg_set_real_path(self.h, int(enable)), self.h)

    def set_graph(self, enable=True):
        check(_lib.lib().dpg_set_graph(self.h, int(enable)), self.h)

    def set_factor_arith(self, arith=_lib.DPG_FACTOR_TC_SPLIT):
        check(_lib.lib().dpg_set_factor_arith(self.h, int(arith)), self.h)
        self.factor_arith = int(arith)

    def set_estimator_store(self, enable=True):
        """Keep L^{-1}[B | B-hat | l] from each element pass; eta_K then needs no second element pass."""
        check(_lib.lib().dpg_set_estimator_store(self.h, int(enable)), self.h)

    def set_bucketed(self, enable=True):
        """Order-bucketed element pass: waves of every order's chunks, one persistent factorisation per wave."""
        check(_lib.lib().dpg_set_bucketed(self.h, int(enable)), self.h)
        self.bucketed = bool(enable)

    def factor_balance(self):
        """SM-busy fraction of the last pass's factorisation launches (1 - idle), their span and element count."""
        busy, span = C.c_double(), C.c_double()
        n = C.c_int64()
        check(_lib.lib().dpg_factor_balance(self.h, C.byref(busy), C.byref(span), C.byref(n)), self.h)
        return {"sm_busy": busy.value, "span_ms": span.value, "elements": n.value}

    def set_wait_limit(self, wait_ns=5_000_000_000, hold=False):
        check(_lib.lib().dpg_set_wait_limit(self.h, int(wait_ns), int(hold)), self.h)

    def group_info(self):
        """[(p, n_elem, chunk)] per order group."""
        ng = C.c_int32()
        p, n, cap = (np.zeros(4, np.int32) for _ in range(3))
        check(_lib.lib().dpg_group_info(self.h, C.byref(ng), ptr(p), ptr(n), ptr(cap)), self.h)
        return [(int(p[g]), int(n[g]), int(cap[g])) for g in range(ng.value)]

    def autotune(self, max_workspace_gb=40.0, stream=None):
        """Measured chunk size per order group: {p: (chunk, ms per element)}."""
        groups = self.group_info()
        caps = np.zeros(len(groups), np.int32)
        ms = np.zeros(len(groups), np.float32)
        check(_lib.lib().dpg_autotune(self.h, float(max_workspace_gb) * 2.0 ** 30, ptr(caps), ptr(ms),
                                      stream_handle(stream)), self.h)
        return {g[0]: (int(caps[k]), float(ms[k])) for k, g in enumerate(groups)}

    def timing_enable(self, enable=True):
        check(_lib.lib().dpg_timing_enable(self.h, int(enable)), self.h)

    def timing_get(self):
        t = _lib.dpg_timing()
        check(_lib.lib().dpg_timing_get(self.h, C.byref(t)), self.h)
        return {k: getattr(t, k) for k, _ in t._fields_}

    def grad_eps(self, xhat, mask, want_grad=True, cg_mode=_lib.DPG_CG_FP64, rtol=1e-12, max_iter=200000,
                 stream=None):
        """Absorbed power P of the obstacle (mask: cuda uint8, n_elem) and, if asked, dP/dRe eps, dP/dIm eps."""
        P = C.c_double()
        dre = torch.empty(self.n_elem, dtype=torch.float64, device='cuda') if want_grad else None
        dim = torch.empty(self.n_elem, dtype=torch.float64, device='cuda') if want_grad else None
        check(_lib.lib().dpg_grad_eps(self.h, ptr(xhat), ptr(mask), C.byref(P), ptr(dre), ptr(dim), cg_mode, rtol,
                                      max_iter, stream_handle(stream)), self.h)
        return P.value, dre, dim

    def power(self, xhat, want_flux=True, stream=None):
        """Per-element int_K Q_em dV (cuda float64, n_elem) and the outward Poynting flux per Robin group."""
        q = torch.empty(self.n_elem, dtype=torch.float64, device='cuda')
        flux = np.zeros(max(1, len(self.mesh.robin)), np.float64) if want_flux else None
        check(_lib.lib().dpg_power(self.h, ptr(xhat), ptr(q), ptr(flux) if want_flux else None,
                                   stream_handle(stream)), self.h)
        return q, (flux[:len(self.mesh.robin)] if want_flux else None)

    def trace_map(self):
        """Trace map and fixed values: n_elem x n_h for one degree, else flat at h_off."""
        m = np.empty(int(self.h_off[-1]), dtype=np.int32)
        fv = np.empty(int(self.h_off[-1]), dtype=np.complex128)
        check(_lib.lib().dpg_trace_map(self.h, ptr(m), ptr(fv)), self.h)
        if self.uniform:
            return m.reshape(self.n_elem, self.n_h), fv.reshape(self.n_elem, self.n_h)
        return m, fv

    def element_dump(self, ids, stream=None):
        """G, B, B-hat, l, S, s of elements that share one trial degree (S, s in the trace slots)."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        k = len(ids)
        nv, nu, nh = element_sizes(int(self.p_elem[ids[0]]))
        G = np.empty((k, nv, nv), np.complex128)
        B = np.empty((k, nv, nu), np.complex128)
        Bh = np.empty((k, nv, nh), np.complex128)
        l = np.empty((k, nv), np.complex128)
        S = np.empty((k, nh, nh), np.complex128)
        s = np.empty((k, nh), np.complex128)
        check(_lib.lib().dpg_element_dump(self.h, ptr(ids), k, ptr(G), ptr(B), ptr(Bh), ptr(l), ptr(S), ptr(s),
                                          stream_handle(stream)), self.h)
        return dict(G=G, B=B, Bh=Bh, l=l, S=S, s=s)

    def csr_copy(self, values=True, stream=None):
        rp = np.empty(self.n + 1, np.int64)
        col = np.empty(self.nnz, np.int32)
        val = np.empty(self.nnz, np.complex128) if values else None
        b = np.empty(self.n, np.complex128) if values else None
        check(_lib.lib().dpg_csr_copy(self.h, ptr(rp), ptr(col), ptr(val), ptr(b), stream_handle(stream)), self.h)
        return rp, col, val, b

    def destroy(self):
        if getattr(self, 'h', None):
            _lib.lib().dpg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tc_gemm(A, B, split=1, upper_only=False, C=None):
    """A^T B through the tensor-core contraction kernel (check hook; host float64 arrays)."""
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    Kd, Ma = A.shape
    Nb = B.shape[1]
    C = np.zeros((Ma, Nb)) if C is None else np.ascontiguousarray(C, np.float64).copy()
    check(_lib.lib().dpg_tc_gemm(split, Ma, Nb, Kd, ptr(A), ptr(B), ptr(C), int(upper_only)))
    return C


def factor_check(A, nv, npiv, nact=None, arith=_lib.DPG_FACTOR_TC_SPLIT):
    """Element factorisation kernel on one host matrix A (N x N, real or complex; lower triangle used).

    Returns (factored matrix, not_hpd flag) with the same layout (row-major
    numpy view of the column-major device layout is handled here).
    """
    A = np.asarray(A)
    N = A.shape[0]
    cplx = np.iscomplexobj(A)
    buf = np.ascontiguousarray(A.T, dtype=np.complex128 if cplx else np.float64)  # column-major
    out = np.empty_like(buf)
    bad = C.c_int32(0)
    check(_lib.lib().dpg_factor_check(int(arith), int(cplx), N, N if nact is None else int(nact), int(nv), int(npiv),
                                      buf.ctypes.data, out.ctypes.data, C.byref(bad)))
    return out.T.copy(), bool(bad.value)


def probe_peaks(stream=None):
    """(FP64, FP32) FMA throughput of the current device in FLOP/s."""
    a, b = C.c_double(), C.c_double()
    check(_lib.lib().dpg_probe_peaks(C.byref(a), C.byref(b), stream_handle(stream)))
    return a.value, b.value


class AbsorbedPower(torch.autograd.Function):
    """P(eps) = absorbed power of an obstacle, differentiable in the per-element permittivity.

    forward(eps, solver, mask): eps is a complex128 tensor (n_elem); the DPG
    forward solve runs on the solver's handle (built with adjoint=True).
    backward: the adjoint gradient, packed in torch's convention for a real
    function of a complex input, grad = dP/dRe(eps) + i dP/dIm(eps) (checked
    against torch on |z|^2 in the tests).  The handle's state belongs to the
    last forward: call backward before another forward on the same solver.
    """

    @staticmethod
    def forward(ctx, eps, solver, mask, cg_rtol=1e-12):
        e = eps.detach().to('cpu', torch.complex128).contiguous().pin_memory()
        solver.update_elements(eps=e)
        solver.element_batch()
        solver.assemble()
        x, rep = solver.cg_solve(rtol=cg_rtol)
        P, _, _ = solver.grad_eps(x, mask, want_grad=False)
        ctx.solver, ctx.mask, ctx.x, ctx.rtol = solver, mask, x, cg_rtol
        ctx.eps_device = eps.device
        torch.cuda.synchronize()
        return torch.tensor(P, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, grad_out):
        _, dre, dim = ctx.solver.grad_eps(ctx.x, ctx.mask, want_grad=True, rtol=ctx.rtol)
        g = torch.complex(dre, dim).to(ctx.eps_device)
        return grad_out.to(g.device) * g, None, None, None
