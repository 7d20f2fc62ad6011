"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function include/ep.h declares, and validates arguments
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2302_12519_gb300 as ep
from paper_2302_12519_gb300 import build as epbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    epbuild.build()
    return ep.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "ep.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(ep_[a-z_]+)\s*\(", txt))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert declared, "no declarations parsed"
    assert set(declared) == set(ep.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def _desc(nx=4, ny=4, nz=4, dx=0.5, model=ep.EP_BI, prec=ep.EP_FP32):
    d = ep.GridDesc()
    d.nx, d.ny, d.nz, d.dx_mm, d.model, d.precision = nx, ny, nz, dx, model, prec
    return d


def test_create_validates_descriptor(lib):
    h = ctypes.c_void_p()
    assert lib.ep_create(None, ctypes.byref(h)) == ep.EP_EINVAL
    for bad in (_desc(nx=0), _desc(dx=0.0), _desc(dx=float("nan")), _desc(model=3), _desc(prec=2)):
        assert lib.ep_create(ctypes.byref(bad), ctypes.byref(h)) == ep.EP_EINVAL
    d = _desc()
    assert lib.ep_create(ctypes.byref(d), ctypes.byref(h)) == ep.EP_OK
    lib.ep_destroy(h)


def test_setters_validate_before_any_device_work(lib):
    import workloads as W
    s = ep.Sim(3, 2, 2, 0.5, use_torch=False)
    n = s.n
    with pytest.raises(ep.EPError) as e:
        s.set_mask(np.ones(n - 1, np.uint8))
    assert e.value.status == ep.EP_EINVAL
    with pytest.raises(ep.EPError):
        s.set_fibres(np.full(3 * n, 2.0, np.float32))
    p = W.Params()
    p.sig_iT = -1.0
    with pytest.raises(ep.EPError) as e:
        s.set_params(p)
    assert e.value.status == ep.EP_EINVAL and "conductiv" in str(e.value)
    p = W.Params()
    p.jacobi_omega = 0
    p.check_every = 0
    with pytest.raises(ep.EPError):
        s.set_params(p)
    for _ in range(8):
        s.add_stimulus((0, 0, 0), (1, 1, 1), 0.0, 1.0, 0.5)
    with pytest.raises(ep.EPError):
        s.add_stimulus((0, 0, 0), (1, 1, 1), 0.0, 1.0, 0.5)
    # stepping without a mask is a state error, caught on the host
    with pytest.raises(ep.EPError) as e:
        s.step(1)
    assert e.value.status == ep.EP_ESTATE
    s.close()


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(ImportError):
        ep._lib_backup = ep._lib
        ep._lib = None
        try:
            ep.load(str(tmp_path / "missing.so"))
        finally:
            ep._lib = ep._lib_backup
