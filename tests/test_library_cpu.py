"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function include/*.h declares, and validates arguments
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
    txt = "".join(open(os.path.join(ROOT, "include", h)).read()
                  for h in sorted(os.listdir(os.path.join(ROOT, "include"))) if h.endswith(".h"))
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
        s.set_fibres(np.full(3 * n, 4.5, np.float32))
    with pytest.raises(ep.EPError):
        s.set_fibres(np.full(3 * n, np.nan, np.float32))
    s.set_fibres(np.full(3 * n, 1.5, np.float32))   # a fast-conducting fibre is longer than 1
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
    for solver, ok in ((0, True), (1, True), (2, True), (3, False), (-1, False)):   # the three elliptic solves
        p = W.Params()
        p.solver = solver
        if ok:
            s.set_params(p)
        else:
            with pytest.raises(ep.EPError) as e:
                s.set_params(p)
            assert e.value.status == ep.EP_EINVAL and "solver" in str(e.value)
    p = W.Params()
    p.solver, p.omega = 2, 2.0   # the SOR factor must stay below 2
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


def test_footprint_is_planned_on_the_host(lib):
    """ep_footprint needs no device: the layout plan is host work.  The peak
    adds the set-up staging (fp32 fibres, mask bytes, raw fp32 records: 29
    bytes a voxel) to the resident bytes, and an FP64 handle holds its eight
    state and solve fields at 8 instead of 4 bytes a voxel (an FP32 bidomain
    handle adds the correction form's third iterate, 4 bytes a voxel)."""
    import workloads as W
    c = W.random_case(3, 19, 13, 11)
    got = {}
    for prec in (ep.EP_FP32, ep.EP_FP64):
        s = ep.sim_from_case(c, use_torch=False, precision=prec)
        got[prec] = s.footprint()
        s.close()
    n = c.n
    (r32, p32), (r64, p64) = got[ep.EP_FP32], got[ep.EP_FP64]
    assert p32 - r32 == 29 * n and p64 - r64 == 29 * n
    assert r64 - r32 == 8 * 4 * n - 4 * n
    assert r32 >= 52 * n + 4 * c.n_tissue
    s = ep.Sim(5, 4, 3, 0.5, use_torch=False)
    with pytest.raises(ep.EPError) as e:
        s.footprint()
    assert e.value.status == ep.EP_ESTATE
    s.set_mask(np.zeros(s.n, np.uint8))
    with pytest.raises(ep.EPError) as e:
        s.footprint()
    assert e.value.status == ep.EP_EINVAL
    m = np.zeros(s.n, np.uint8)
    m[:7] = 1
    s.set_mask(m)   # a new mask is planned afresh
    r_a, _ = s.footprint()
    m[:30] = 1
    s.set_mask(m)
    r_b, _ = s.footprint()
    assert r_b > r_a
    s.close()


def test_footprint_counts_the_interval_estimate(lib):
    """A Chebyshev bidomain handle without a given interval estimates it at
    set-up: the peak adds the Lanczos scalars (82 doubles) and two partial sums
    per reduction chunk; with the interval given, or for damped Jacobi, nothing.
    FP32 damped-Jacobi and Chebyshev handles keep a third iterate (the
    correction form, 4 bytes a voxel); the eight-colour Gauss-Seidel handle,
    which works in place, does not, keeps eight residual partial sums per work
    item instead, and estimates nothing."""
    import workloads as W
    c = W.random_case(4, 17, 12, 10, model=W.BI)
    peaks = {}
    for key, solver, lmin, lmax in (("jac", 0, 0.0, 0.0), ("est", 1, 0.0, 0.0), ("given", 1, 0.01, 4.0),
                                    ("gs", 2, 0.0, 0.0)):
        c.params.solver, c.params.cheb_lmin, c.params.cheb_lmax = solver, lmin, lmax
        s = ep.sim_from_case(c, use_torch=False)
        peaks[key] = s.footprint()
        s.close()
    (rj, pj), (re_, pe), (rg, pg), (rs, ps) = peaks["jac"], peaks["est"], peaks["given"], peaks["gs"]
    assert re_ == rg == rj and pg - rg == pj - rj
    extra = (pe - re_) - (pj - rj)
    assert extra >= 8 * 82 + 16 and (extra - 8 * 82) % 16 == 0
    assert rs >= rj - 4 * c.n and ps - rs == pj - rj   # (this mask has more reduction chunks than 8 x items)
    # on one connected block the eight partial sums per item outgrow the reduction chunks
    blk = W.random_case(4, 40, 30, 20, model=W.BI, mask=np.ones((20, 30, 40), np.uint8))
    res = {}
    for solver in (0, 2):
        blk.params.solver = solver
        h = ep.sim_from_case(blk, use_torch=False)
        res[solver] = h.footprint()[0]
        h.close()
    assert res[2] - (res[0] - 4 * blk.n) > 0
    # damped Jacobi with estimated damping runs the same estimate
    c.params.solver, c.params.cheb_lmin, c.params.cheb_lmax, c.params.omega = 0, 0.0, 0.0, -1.0
    s = ep.sim_from_case(c, use_torch=False)
    assert s.footprint() == (rj, pj + extra)
    s.close()
    # FP64 handles run the plain iterations: no third iterate
    c.params.solver, c.params.omega = 1, 0.0
    s64 = ep.sim_from_case(c, use_torch=False, precision=ep.EP_FP64)
    c.params.solver = 0
    j64 = ep.sim_from_case(c, use_torch=False, precision=ep.EP_FP64)
    assert s64.footprint()[0] == j64.footprint()[0]
    s64.close()
    j64.close()


def test_torso_and_ecg_are_validated_and_planned_on_the_host(lib):
    """ep_set_torso / ep_set_ecg check their arguments without a device; a
    torso adds the domain's records (16 bytes a voxel) and work items to the
    resident bytes and its staging (1 byte a voxel) to the peak; an ECG adds its
    record (3 doubles a sample)."""
    import workloads as W
    c = W.with_torso(W.random_case(5, 12, 10, 9), sig_o=0.8, pad=1)
    plain = ep.sim_from_case(W.with_torso(W.random_case(5, 12, 10, 9), sig_o=0.8, pad=1), use_torch=False)
    plain.set_torso(np.zeros(c.n, np.uint8), 1.0)   # an all-zero torso is no torso
    plain.set_ecg(None, 0)
    s = ep.sim_from_case(c, use_torch=False, ecg_capacity=100)
    (r0, p0), (r1, p1) = plain.footprint(), s.footprint()
    assert p0 - r0 == 29 * c.n and p1 - r1 == 30 * c.n
    assert r1 - r0 >= 16 * c.n + 3 * 8 * 100
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(ep.EPError) as e:
            s.set_torso(c.torso, bad)
        assert e.value.status == ep.EP_EINVAL
    with pytest.raises(ep.EPError) as e:
        s.set_torso(np.zeros(7, np.uint8), 1.0)
    assert e.value.status == ep.EP_EINVAL
    for el in ([(0, 0, 0), (0, 0, 0), (c.nx, 0, 0)], [(-1, 0, 0), (0, 0, 0), (0, 0, 0)]):
        with pytest.raises(ep.EPError) as e:
            s.set_ecg(el, 10)
        assert e.value.status == ep.EP_EINVAL
    with pytest.raises(ep.EPError) as e:
        s.set_ecg([(0, 0, 0)] * 3, -1)
    assert e.value.status == ep.EP_EINVAL
    s.close()
    plain.close()


def test_sdf_encoder_validates_the_program_without_a_device(lib):
    """ep_sdf_encode checks programs, regions and the grid before it touches
    the device."""
    import workloads as W
    E = W.SdfNode(W.SDF_ELLIPSOID, 2.0, 2.0, 2.0)
    bad = [
        ([W.SdfNode(W.SDF_UNION)], [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)]),            # no operands
        ([E, E], [W.SdfRegion(0, 2, W.REGION_MYOCARDIUM)]),                                # two values left
        ([W.SdfNode(99)], [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)]),                      # unknown op
        ([W.SdfNode(W.SDF_ELLIPSOID, 0.0, 1.0, 1.0)], [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)]),   # zero size
        ([E], [W.SdfRegion(0, 2, W.REGION_MYOCARDIUM)]),                                   # range past the nodes
        ([E], [W.SdfRegion(0, 1, 7)]),                                                     # unknown kind
        ([E, E, W.SdfNode(W.SDF_SMOOTH_UNION, 0.0)], [W.SdfRegion(0, 3, W.REGION_MYOCARDIUM)]),   # zero width
    ]
    for nodes, regions in bad:
        with pytest.raises(ep.EPError) as e:
            ep.sdf_encode(nodes, regions, 4, 4, 4, 1.0, (0.0, 0.0, 0.0), 0.0)
        assert e.value.status == ep.EP_EINVAL
    deep = [E] * 33 + [W.SdfNode(W.SDF_UNION)] * 32
    with pytest.raises(ep.EPError) as e:
        ep.sdf_encode(deep, [W.SdfRegion(0, len(deep), W.REGION_MYOCARDIUM)], 4, 4, 4, 1.0, (0, 0, 0), 0.0)
    assert e.value.status == ep.EP_EINVAL
    with pytest.raises(ep.EPError) as e:
        ep.sdf_encode([E], [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)], 0, 4, 4, 1.0, (0, 0, 0), 0.0)
    assert e.value.status == ep.EP_EINVAL


def test_ecg_calls_validate_on_the_host(lib):
    """Without an ECG set up, ep_read_ecg is EP_EINVAL and reports no samples;
    capacity 0 switches a set-up ECG off again (no record in the footprint)."""
    import workloads as W
    c = W.random_case(6, 10, 9, 8)
    s = ep.sim_from_case(c, use_torch=False)
    n = ctypes.c_int(7)
    assert lib.ep_read_ecg(s._h, None, 0, ctypes.byref(n)) == ep.EP_EINVAL and n.value == 0
    r0 = s.footprint()
    s.set_ecg([(0, 0, 0), (1, 1, 1), (2, 2, 2)], 50)
    r1 = s.footprint()
    assert r1[0] == r0[0] + 3 * 8 * 50
    s.set_ecg(None, 0)
    assert s.footprint() == r0
    assert lib.ep_read_ecg(s._h, None, 0, ctypes.byref(n)) == ep.EP_EINVAL
    s.close()


def test_server_needs_a_device(lib):
    """Without a GPU the server cannot start and says so (no host fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    srv = ctypes.c_void_p()
    cfg = ep.ServerConfig()
    cfg.max_slots, cfg.chunk_steps = 2, 1
    assert lib.ep_server_create(ctypes.byref(cfg), ctypes.byref(srv)) == ep.EP_ECUDA
    cfg.max_slots = 0
    assert lib.ep_server_create(ctypes.byref(cfg), ctypes.byref(srv)) == ep.EP_EINVAL


def test_diffusion_scheme_is_validated(lib):
    import workloads as W
    s = ep.Sim(4, 4, 4, 0.5, use_torch=False)
    p = W.Params()
    p.diffusion = 2
    with pytest.raises(ep.EPError) as e:
        s.set_params(p)
    assert e.value.status == ep.EP_EINVAL and "diffusion" in str(e.value)
    p.diffusion = ep.EP_IMPLICIT
    s.set_params(p)
    # the implicit scheme's two extra fields show in the planned footprint
    s.set_mask(np.ones(s.n, np.uint8))
    r_ie, _ = s.footprint()
    p.diffusion = ep.EP_EXPLICIT
    s.set_params(p)
    r_ex, _ = s.footprint()
    assert r_ie - r_ex == 2 * 4 * s.n
    s.close()
