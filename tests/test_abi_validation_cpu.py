"""Host-side argument validation of the C ABI: malformed descriptors, physics
and null handles return DG_ERR_INVALID before any device work, so these calls
run without a GPU."""
import ctypes

import numpy as np
import pytest

from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build

DG_ERR_INVALID = 1   # dg_status (include/dg.h)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return B.load()


def _desc(**kw):
    d = B.MeshDesc()
    d.dim, d.p, d.nq1d, d.space = 3, 2, 0, B.SPACE_P
    for k in range(3):
        d.n[k], d.lo[k], d.hi[k] = 4, 0.0, 1.0
    for k, v in kw.items():
        if k in ("n", "lo", "hi"):
            for i, x in enumerate(v):
                getattr(d, k)[i] = x
        else:
            setattr(d, k, v)
    return d


def _phys(**kw):
    base = dict(gamma=1.4, Pr=0.72, mu=1e-3, Rgas=1.0, eta_br2=0.0, roe_delta=0.1)
    base.update(kw)
    return B.PhysicsDesc(*[base[k] for k, _ in B.PhysicsDesc._fields_])


@pytest.mark.parametrize("bad", [dict(dim=4), dict(dim=1), dict(p=-1), dict(p=9), dict(space=5),
                                 dict(nq1d=2), dict(nq1d=13), dict(n=(0, 4, 4)), dict(hi=(1.0, 0.0, 1.0))])
def test_structured_mesh_descriptor_rejected(lib, bad):
    h = B.P()
    assert lib.dg_mesh_create(ctypes.byref(_desc(**bad)), ctypes.byref(_phys()), None, ctypes.byref(h)) == \
        DG_ERR_INVALID
    assert not h.value


@pytest.mark.parametrize("bad", [dict(gamma=1.0), dict(Rgas=0.0), dict(mu=-1.0), dict(Pr=0.0),
                                 dict(roe_delta=-0.1), dict(eta_br2=-1.0)])
def test_physics_rejected(lib, bad):
    h = B.P()
    assert lib.dg_mesh_create(ctypes.byref(_desc()), ctypes.byref(_phys(**bad)), None, ctypes.byref(h)) == \
        DG_ERR_INVALID


def _tri_desc(keep, **kw):
    X = np.zeros((4, 2))
    tri = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    shift = np.zeros((2, 3, 2), dtype=np.int32)
    keep.extend([X, tri, shift])
    d = B.TriDesc()
    d.n_vert, d.n_tri, d.p, d.nq1d = 4, 2, 2, 0
    d.X = X.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.tri = tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    d.shift = shift.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    for k in range(2):
        d.lo[k], d.hi[k] = 0.0, 1.0
    for k, v in kw.items():
        if k in ("lo", "hi"):
            for i, x in enumerate(v):
                getattr(d, k)[i] = x
        elif k == "X":
            d.X = None
        else:
            setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad", [dict(n_vert=2), dict(n_tri=1), dict(p=-1), dict(p=9), dict(nq1d=13),
                                 dict(nq1d=2), dict(hi=(0.0, 1.0)), dict(X=None)])
def test_triangulation_descriptor_rejected(lib, bad):
    keep = []
    h = B.P()
    assert lib.dg_mesh_create_tri(ctypes.byref(_tri_desc(keep, **bad)), ctypes.byref(_phys()), None,
                                  ctypes.byref(h)) == DG_ERR_INVALID


def test_null_handles_rejected(lib):
    assert lib.dg_residual(None, None, None, None, None) == DG_ERR_INVALID
    assert lib.dg_jvp(None, None, None, 1.0, None, None, B.JVP_EXACT, None) == DG_ERR_INVALID
    o = B.pmg_opts((2, 1))
    h = B.P()
    assert lib.dg_pmg_setup(None, None, 1.0, ctypes.byref(o), None, ctypes.byref(h)) == DG_ERR_INVALID
    assert lib.dg_pmg_apply(None, None, None, None) == DG_ERR_INVALID
    assert lib.dg_pmg_destroy(None) == DG_ERR_INVALID
    assert lib.dg_mesh_destroy(None) == DG_ERR_INVALID
    n = ctypes.c_int()
    assert lib.dg_pmg_bilu_order(None, None, ctypes.byref(n), None) == DG_ERR_INVALID
