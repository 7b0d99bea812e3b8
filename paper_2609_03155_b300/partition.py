"""Row partition of the condensed trace system for a CG split over ranks.

The element passes of the method (quadrature, factorisation, condensation,
recovery and eta_K; Sec. 2.3, Algorithm 2) are independent per element and
shard with no exchange.  The CG on the assembled trace system (Sec. 2.3 end)
needs one exchange per iteration: a rank's rows of A p reference entries of p
owned by the ranks across its slab interfaces.  This module is the host index
logic of that split, independent of the arithmetic:

* elements go to slabs of (nearly) equal element count along one axis
  (``slab_partition``);
* a trace unknown (a CSR row) belongs to the lowest rank among the elements
  that carry it, so every slab interface is owned by one side
  (``row_owner``);
* per rank, ``RankLayout`` numbers the owned rows first and the halo (the
  columns its rows reference on other ranks, grouped by owner, ascending
  global id within a group) after them, keeps its rows of the CSR with the
  columns in that local numbering, and lists for every other rank the owned
  rows that rank needs, in the order that rank's halo expects.

Only integer index work happens here; the CG that uses the layouts is
``dist_cg.py``.
"""
from dataclasses import dataclass, field

import numpy as np


def slab_partition(coord, nranks):
    """Rank of every element: contiguous slabs along ``coord`` (one value per
    element, e.g. the centroid's x3), each with n / nranks elements (the first
    n % nranks slabs one more); ties broken by element index."""
    coord = np.asarray(coord, dtype=float)
    n = coord.shape[0]
    if nranks < 1 or nranks > max(n, 1):
        raise ValueError("need 1 <= nranks <= number of elements")
    order = np.lexsort((np.arange(n), coord))
    sizes = np.full(nranks, n // nranks)
    sizes[: n % nranks] += 1
    owner = np.empty(n, dtype=np.int32)
    owner[order] = np.repeat(np.arange(nranks, dtype=np.int32), sizes)
    return owner


def row_owner(elem_rows, elem_rank, n):
    """Owner rank of each of the n rows: the lowest rank among the elements
    whose row list (global row ids, negative for fixed unknowns) holds it.
    Rows carried by no element raise."""
    own = np.full(n, np.iinfo(np.int32).max, dtype=np.int64)
    for rows, r in zip(elem_rows, elem_rank):
        rows = np.asarray(rows)
        rows = rows[rows >= 0]
        np.minimum.at(own, rows, int(r))
    if np.any(own == np.iinfo(np.int32).max):
        raise ValueError("a row is carried by no element")
    return own.astype(np.int32)


@dataclass
class RankLayout:
    rank: int
    owned: np.ndarray                 # global ids of the owned rows, ascending
    halo: np.ndarray                  # global ids of the halo columns (grouped by owner, ascending within)
    halo_from: dict = field(default_factory=dict)   # owner rank -> slice of the halo (local index range)
    send_to: dict = field(default_factory=dict)     # rank -> local indices of owned rows it needs, in its order
    rowptr: np.ndarray = None         # local CSR of the owned rows
    cols: np.ndarray = None           # column indices in the local numbering (owned, then halo)
    csr_pos: np.ndarray = None        # position in the global CSR of each local entry (to gather values)

    @property
    def n_owned(self):
        return self.owned.shape[0]

    @property
    def n_local(self):
        return self.owned.shape[0] + self.halo.shape[0]


def build_layouts(rowptr, cols, owner, nranks):
    """Per-rank layouts of a global CSR pattern (rowptr, cols) under the row
    ownership ``owner``.  Symmetric patterns (the trace system is Hermitian)
    make the send lists the mirror of the halos."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    owner = np.asarray(owner, dtype=np.int32)
    n = owner.shape[0]
    layouts = []
    for r in range(nranks):
        owned = np.nonzero(owner == r)[0].astype(np.int64)
        loc = np.full(n, -1, dtype=np.int64)
        loc[owned] = np.arange(owned.shape[0])
        # entries of the owned rows
        starts, ends = rowptr[owned], rowptr[owned + 1]
        counts = ends - starts
        pos = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)]) if owned.size else np.zeros(0, np.int64)
        gcols = cols[pos]
        ext = np.unique(gcols[owner[gcols] != r])
        # halo grouped by owner rank, ascending global id within a group
        ext = ext[np.lexsort((ext, owner[ext]))]
        lay = RankLayout(rank=r, owned=owned, halo=ext)
        base = owned.shape[0]
        for q in np.unique(owner[ext]):
            idx = np.nonzero(owner[ext] == q)[0]
            lay.halo_from[int(q)] = slice(base + int(idx[0]), base + int(idx[-1]) + 1)
        loc[ext] = base + np.arange(ext.shape[0])
        lay.rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        lay.cols = loc[gcols]
        lay.csr_pos = pos
        layouts.append(lay)
    # send lists: what rank q's halo holds from rank r, in q's order, as r's local indices
    for lay_q in layouts:
        for r, sl in lay_q.halo_from.items():
            need = lay_q.halo[sl.start - lay_q.n_owned: sl.stop - lay_q.n_owned]
            lay_r = layouts[r]
            lay_r.send_to[lay_q.rank] = np.searchsorted(lay_r.owned, need)
    return layouts


def check_layouts(layouts, rowptr, cols, owner):
    """Invariants of a partition (raises AssertionError): every row owned
    once; every column a rank's rows reference is owned or in its halo; the
    halo holds only referenced off-rank columns; r's send list to q is q's
    halo from r, entry by entry."""
    n = owner.shape[0]
    seen = np.zeros(n, dtype=np.int64)
    for lay in layouts:
        seen[lay.owned] += 1
        glob = np.concatenate([lay.owned, lay.halo])
        assert np.all(lay.cols >= 0) and np.all(lay.cols < lay.n_local)
        np.testing.assert_array_equal(glob[lay.cols], np.asarray(cols)[lay.csr_pos])
        assert np.all(owner[lay.halo] != lay.rank)
        assert np.unique(lay.cols[lay.cols >= lay.n_owned]).shape[0] == lay.halo.shape[0]
        for q, sl in lay.halo_from.items():
            sent = layouts[q].owned[layouts[q].send_to[lay.rank]]
            np.testing.assert_array_equal(sent, lay.halo[sl.start - lay.n_owned: sl.stop - lay.n_owned])
    assert np.all(seen == 1)
