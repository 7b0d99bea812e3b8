"""Conjugate gradients on the trace system split over ranks (Sec. 2.3 end).

The rows of the Hermitian positive definite system are partitioned by
``partition.build_layouts``; each rank keeps its rows of A, of b and of the
iterates.  One iteration needs one halo exchange (the entries of the search
direction p that the rank's rows reference on other ranks, point to point
with the owners) and two scalar all-reduces (p^H A p, and r^H r for the step
and the stopping test).  The local product is the caller's: the rank's rows
of A applied to [p_owned, p_halo] in the layout's local numbering.

torch.distributed carries the exchange (gloo on CPU, NCCL on GPUs); complex
vectors travel as their real views.
"""
import torch
import torch.distributed as dist


def halo_exchange(layout, v, group=None):
    """Fill the halo part of v (length layout.n_local: owned, then halo) with
    the owners' entries; v's owned part is sent to the ranks that need it."""
    ops, recvs = [], []
    for q, idx in sorted(layout.send_to.items()):
        buf = torch.view_as_real(v[torch.as_tensor(idx, dtype=torch.long)].contiguous()) \
            if v.is_complex() else v[torch.as_tensor(idx, dtype=torch.long)].contiguous()
        ops.append(dist.P2POp(dist.isend, buf, q, group=group))
    for q, sl in sorted(layout.halo_from.items()):
        n = sl.stop - sl.start
        buf = torch.empty((n, 2) if v.is_complex() else (n,), dtype=torch.float64 if v.is_complex() else v.dtype,
                          device=v.device)
        ops.append(dist.P2POp(dist.irecv, buf, q, group=group))
        recvs.append((sl, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for sl, buf in recvs:
        v[sl] = torch.view_as_complex(buf) if v.is_complex() else buf


def _allreduce(value, device, group=None):
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def dist_cg(layout, matvec, b_owned, rtol=1e-10, max_iter=100000, group=None):
    """Unpreconditioned CG from x0 = 0 on the split system.

    layout: this rank's ``partition.RankLayout``; matvec(v_local) -> the
    rank's rows of A v (v_local: owned then halo entries); b_owned: the
    rank's rows of b.  Stops when ||r|| <= rtol ||b|| (global norms) or after
    max_iter iterations.  Returns (x_owned, iterations, relative residual),
    identical scalars on every rank.
    """
    no = layout.n_owned
    dev = b_owned.device
    x = torch.zeros_like(b_owned)
    r = b_owned.clone()
    p = torch.zeros(layout.n_local, dtype=b_owned.dtype, device=dev)
    p[:no] = r
    rr = _allreduce(torch.vdot(r, r).real.item(), dev, group)
    bb = rr
    tol2 = rtol * rtol * bb
    it = 0
    while rr > tol2 and it < max_iter:
        halo_exchange(layout, p, group)
        Ap = matvec(p)
        pAp = _allreduce(torch.vdot(p[:no], Ap).real.item(), dev, group)
        alpha = rr / pAp
        x += alpha * p[:no]
        r -= alpha * Ap
        rr_new = _allreduce(torch.vdot(r, r).real.item(), dev, group)
        beta = rr_new / rr
        rr = rr_new
        p[:no] = r + beta * p[:no]
        it += 1
    return x, it, (rr / bb) ** 0.5 if bb > 0 else 0.0
