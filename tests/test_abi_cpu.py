"""The C-ABI library loads and exports every symbol include/dpg.h declares (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2609_03155_b300 import _lib, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dpg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dpg_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    names = declared_functions()
    assert "dpg_setup_mesh" in names and "dpg_cg_solve" in names and len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def _desc(mesh):
    keep = dict(vert=np.ascontiguousarray(mesh.vert), elem=np.ascontiguousarray(mesh.elem, np.int32),
                p=np.ascontiguousarray(mesh.p, np.int8), eps=np.ascontiguousarray(mesh.eps, np.complex128),
                mu=np.ascontiguousarray(mesh.mu, np.complex128), bc=np.ascontiguousarray(mesh.face_bc, np.int8),
                grp=np.ascontiguousarray(mesh.face_grp, np.int16))
    rob = (_lib.dpg_robin_group * 2)()
    dirg = (_lib.dpg_dirichlet_group * 2)()
    d = _lib.dpg_mesh_desc(n_vert=keep['vert'].shape[0], vert=keep['vert'].ctypes.data, n_elem=keep['elem'].shape[0],
                           elem=keep['elem'].ctypes.data, elem_p=keep['p'].ctypes.data,
                           elem_eps=keep['eps'].ctypes.data, elem_mu=keep['mu'].ctypes.data,
                           face_bc=keep['bc'].ctypes.data, face_grp=keep['grp'].ctypes.data, n_robin=2,
                           robin=C.cast(rob, C.POINTER(_lib.dpg_robin_group)), n_dirichlet=1,
                           dirichlet=C.cast(dirg, C.POINTER(_lib.dpg_dirichlet_group)))
    return d, (keep, rob, dirg)


def _setup(mesh, **prm):
    d, keep = _desc(mesh)
    p = _lib.dpg_params(omega=prm.get('omega', 1.0), alpha=prm.get('alpha', 1.0), dp=prm.get('dp', 1),
                        precision=prm.get('precision', 0))
    h = C.c_void_p()
    rc = _lib.lib().dpg_setup_mesh(C.byref(h), C.byref(d), C.byref(p), None)
    return rc, h, _lib.lib().dpg_last_error(None).decode()


def test_setup_rejects_bad_arguments_before_touching_the_device():
    m = inputs.waveguide_2d_config(p=1)
    L = _lib.lib()
    h = C.c_void_p()
    assert L.dpg_setup_mesh(None, None, None, None) == -1
    assert L.dpg_setup_mesh(C.byref(h), None, None, None) == -1
    rc, _, msg = _setup(m, dp=2)
    assert rc == -9 and "dp" in msg
    rc, _, msg = _setup(m, alpha=0.0)
    assert rc == -1
    bad = inputs.waveguide_2d_config(p=1)
    bad.elem = bad.elem.copy()
    bad.elem[3, 2] = bad.vert.shape[0] + 5
    rc, _, msg = _setup(bad)
    assert rc == -2 and "range" in msg
    # a reflected element (x axis reversed) has a negative Jacobian
    bad = inputs.waveguide_2d_config(p=1)
    bad.elem = bad.elem.copy()
    bad.elem[0] = bad.elem[0][[1, 0, 3, 2, 5, 4, 7, 6]]
    rc, _, msg = _setup(bad)
    assert rc == -2 and "Jacobian" in msg
    # host-side fault injection: non-finite inputs are errors, not device faults
    bad = inputs.waveguide_2d_config(p=1)
    bad.eps = bad.eps.copy()
    bad.eps[5] = complex(np.nan, 0.0)
    rc, _, msg = _setup(bad)
    assert rc == -1 and "non-finite" in msg
    bad = inputs.waveguide_2d_config(p=1)
    bad.vert = bad.vert.copy()
    bad.vert[2, 1] = np.inf
    rc, _, msg = _setup(bad)
    assert rc == -2 and "non-finite" in msg
    # degrees outside 1..4 are rejected (mixed degrees within it are accepted)
    bad = inputs.waveguide_2d_config(p=1)
    bad.p = bad.p.copy()
    bad.p[0] = 5
    rc, _, msg = _setup(bad)
    assert rc == -2 and "degree" in msg
    # empty mesh
    d, keep = _desc(inputs.waveguide_2d_config(p=1))
    d.n_elem = 0
    prm = _lib.dpg_params(omega=1.0, alpha=1.0, dp=1, precision=0)
    assert L.dpg_setup_mesh(C.byref(h), C.byref(d), C.byref(prm), None) == -1
    assert "empty" in L.dpg_last_error(None).decode()
    # unknown precision mode
    rc, _, msg = _setup(inputs.waveguide_2d_config(p=1), precision=7)
    assert rc == -9 and "precision" in msg
    # null handles
    assert L.dpg_element_batch(None, 0, None) == -1
    assert L.dpg_assemble(None, None) == -1
    L.dpg_destroy(None)
