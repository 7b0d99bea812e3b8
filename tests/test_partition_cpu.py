"""Row-partitioned CG of the trace system on CPU ranks (gloo).

The element passes shard with no exchange; the CG needs one halo exchange
and two scalar all-reduces per iteration.  Checked here without a GPU, on the
oracle's assembled system of a small 3D guide (2 x 1 x 6 hexahedra, p = 1,
TE10 port and absorbing end):

* layout invariants for slabs along x3 (every row owned once, halos hold only
  referenced off-rank columns, send lists mirror the halos; only adjacent
  slabs exchange);
* CG on 2 and 3 gloo ranks reaches the oracle's direct solution, with the
  iteration count of the single-process CG on the same system;
* the same on 2 ranks for the Fichera cavity with mixed orders 1..3 (the
  oracle's restricted, order-jumping trace system).
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import system as osys
from paper_2609_03155_b300 import inputs, partition


@pytest.fixture(scope="module")
def guide():
    mesh = inputs.waveguide_3d_config(2, 1, 6, 1)
    sol = osys.solve(mesh)
    A = sol['A'].tocsr()
    A.sort_indices()
    elem_rows = [sol['free'][g] for g in sol['l2g']]
    z = mesh.vert[mesh.elem].mean(axis=1)[:, 2]
    return dict(A=A, b=sol['b'], x=sol['x'], elem_rows=elem_rows, z=z, n=sol['n'])


@pytest.fixture(scope="module")
def fichera():
    """Mixed orders 1..3 with order jumps across faces (trace restriction)."""
    from oracle import mixed
    mesh = inputs.fichera_cavity(1)
    sol = mixed.solve_mixed(mesh)
    A = sol['A'].tocsr()
    A.sort_indices()
    elem_rows = [sol['free'][gl] for _, gl in sol['R']]
    z = mesh.vert[mesh.elem].mean(axis=1)[:, 2]
    return dict(A=A, b=sol['b'], x=sol['x'], elem_rows=elem_rows, z=z, n=sol['n'])


def _layouts(g, nranks):
    er = partition.slab_partition(g['z'], nranks)
    owner = partition.row_owner(g['elem_rows'], er, g['n'])
    return er, owner, partition.build_layouts(g['A'].indptr, g['A'].indices, owner, nranks)


def test_slab_partition_sizes_and_order():
    z = np.array([0.5, 0.1, 0.1, 0.9, 0.3, 0.7, 0.2])
    r = partition.slab_partition(z, 3)
    assert np.bincount(r).tolist() == [3, 2, 2]
    # slabs are contiguous in z: every element of rank k lies below every element of rank k + 1
    for k in range(2):
        assert z[r == k].max() <= z[r == k + 1].min()
    with pytest.raises(ValueError):
        partition.slab_partition(z, 8)


@pytest.mark.parametrize("nranks", [2, 3])
def test_layout_invariants(guide, nranks):
    er, owner, lays = _layouts(guide, nranks)
    partition.check_layouts(lays, guide['A'].indptr, guide['A'].indices, owner)
    # slabs along x3: only neighbouring slabs exchange, and every slab interface does
    for lay in lays:
        assert set(lay.halo_from) <= {lay.rank - 1, lay.rank + 1}
        assert set(lay.send_to) == set(lay.halo_from)
    for k in range(nranks - 1):
        assert k + 1 in lays[k].halo_from
    # the local rows reproduce the global product exactly
    A = guide['A']
    rng = np.random.default_rng(0)
    v = rng.standard_normal(guide['n']) + 1j * rng.standard_normal(guide['n'])
    for lay in lays:
        vals = A.data[lay.csr_pos]
        vl = np.concatenate([v[lay.owned], v[lay.halo]])
        y = np.array([vals[lay.rowptr[i]:lay.rowptr[i + 1]] @ vl[lay.cols[lay.rowptr[i]:lay.rowptr[i + 1]]]
                      for i in range(lay.n_owned)])
        np.testing.assert_allclose(y, (A @ v)[lay.owned], rtol=1e-13, atol=1e-13 * np.abs(A @ v).max())


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, g, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import scipy.sparse as sp

    from paper_2609_03155_b300 import dist_cg, partition as part
    dist.init_process_group("gloo", rank=rank, world_size=world)
    er = part.slab_partition(g['z'], world)
    owner = part.row_owner(g['elem_rows'], er, g['n'])
    lay = part.build_layouts(g['indptr'], g['indices'], owner, world)[rank]
    Aloc = sp.csr_matrix((g['data'][lay.csr_pos], lay.cols, lay.rowptr), shape=(lay.n_owned, lay.n_local))

    def matvec(v):
        return torch.from_numpy(Aloc @ v.numpy())

    b = torch.from_numpy(np.ascontiguousarray(g['b'][lay.owned]))
    x, it, rel = dist_cg.dist_cg(lay, matvec, b, rtol=1e-13, max_iter=20000)
    out[rank] = (lay.owned, x.numpy(), it, rel)
    dist.barrier()
    dist.destroy_process_group()


def _serial_cg_iterations(A, b, rtol):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    bb = rr
    it = 0
    while rr > rtol * rtol * bb:
        Ap = A @ p
        alpha = rr / np.vdot(p, Ap).real
        x += alpha * p
        r -= alpha * Ap
        rn = np.vdot(r, r).real
        p = r + (rn / rr) * p
        rr = rn
        it += 1
    return it


@pytest.mark.parametrize("world", [2, 3])
def test_dist_cg_gloo_matches_direct_solve(guide, world):
    _check_dist_cg(guide, world)


def test_dist_cg_gloo_mixed_orders(fichera):
    er, owner, lays = _layouts(fichera, 2)
    partition.check_layouts(lays, fichera['A'].indptr, fichera['A'].indices, owner)
    _check_dist_cg(fichera, 2)


def _check_dist_cg(guide, world):
    A = guide['A']
    g = dict(indptr=A.indptr, indices=A.indices, data=A.data, b=guide['b'], elem_rows=guide['elem_rows'],
             z=guide['z'], n=guide['n'])
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), g, out), nprocs=world, join=True)
    x = np.zeros(guide['n'], complex)
    its = set()
    for r in range(world):
        owned, xr, it, rel = out[r]
        x[owned] = xr
        its.add(it)
        assert rel <= 1e-13
    assert len(its) == 1  # identical scalars on every rank
    xd = guide['x']
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    # the split changes only the summation order of the dots: same iteration count within a few
    assert abs(its.pop() - _serial_cg_iterations(A, guide['b'], 1e-13)) <= 3
