"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Element-wise at sizes the oracle finishes in seconds (several tiles and a
ragged tail in every axis), and at the full config sizes on quantities the
oracle computes in one pass (one operator application, one reaction +
diffusion step) or through properties that hold at any size (the elliptic
residual of the GPU solution under the oracle's operator)."""
import numpy as np
import pytest

import oracle
import paper_2302_12519_gb300 as ep
import workloads as W

pytestmark = pytest.mark.gpu

# FP32 stencil: terms are O(sigma/dx^2 |u|); 27-point sums in FP32 give relative
# errors of a few 1e-7 of the largest term.
FP32_OP_RTOL = 2e-5
# FP64 stencil on the very fibres the oracle uses (float32 values, the input type
# of ep_set_fibres): rounding of the sums only.
FP64_OP_RTOL = 1e-12
# FP64 stencil on a caller's FP64 fibres, which the library receives as float32:
# |f32(f) - f| <= 2^-24 |f| per component moves each tensor by at most
# 2^-23 (sig_L - sig_T), a few 1e-7 of the largest term.
FP64_CALLER_OP_RTOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_12519_gb300 import build
    build.build()
    ep.load()
    oracle.build()


def _sim(case, precision=None, model=None):
    return ep.sim_from_case(case, precision=precision, model=model)


def _op_case(kind, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "random":
        return W.random_case(seed, 37, 19, 23, fill=0.55)
    if kind == "ragged_small":
        return W.random_case(seed, 8, 7, 6)
    if kind == "wide":
        return W.random_case(seed, 95, 16, 9, fill=0.7)
    c = W.random_case(seed, 33, 15, 12)
    m = np.zeros_like(c.mask)
    if kind == "full":
        m[:] = 1
    elif kind == "isolated":
        m[::2, ::2, ::2] = 1          # isolated voxels: empty rows
        m[3:7, 3:9, 5:20] = 1
    elif kind == "sheet":
        m[5, :, :] = 1                # one-voxel-thick sheet
    elif kind == "column":
        m[:, 4:6, 7:9] = 1            # 2x2 column through every plane
    elif kind == "edges":
        m[0, :, :] = 1; m[-1, :, :] = 1; m[:, 0, :] = 1; m[:, :, -1] = 1
    elif kind == "single_in_tile":
        m[4, 3, 31] = 1               # lone voxel at a tile seam
        m[10, 14, 32] = 1
        m[2:5, 2:5, 2:5] = 1
    c.mask = m
    f = W.random_fibres(rng, m.shape)
    f[m == 0] = 0
    c.fib = f
    return c


@pytest.mark.parametrize("kind", ["random", "ragged_small", "wide", "full", "isolated", "sheet", "column", "edges",
                                  "single_in_tile"])
@pytest.mark.parametrize("precision", [ep.EP_FP32, ep.EP_FP64])
@pytest.mark.parametrize("fibres", ["caller", "float32"])
def test_operator_matches_oracle(kind, precision, fibres):
    """One operator application against the oracle's, element by element.
    "caller": the oracle takes the FP64 fibres as generated, the library their
    float32 values through ep_set_fibres; "float32": both take the float32 values."""
    c = _op_case(kind)
    if fibres == "float32":
        c = c.fibres_as_float32()
    g = oracle.Grid.from_case(c)
    s = _sim(c, precision=precision)
    rng = np.random.default_rng(1)
    t = c.mask.reshape(-1) > 0
    for sL, sT in ((0.2, 0.05), (0.4, 0.15)):
        u = rng.standard_normal(g.n)
        ref = g.apply_L(sL, sT, np.where(t, u, 0.0))
        got = s.apply_operator(sL, sT, u)
        scale = max(np.abs(ref).max(), 1e-30)
        tol = FP32_OP_RTOL if precision == ep.EP_FP32 else (FP64_OP_RTOL if fibres == "float32"
                                                              else FP64_CALLER_OP_RTOL)
        assert np.all(got[~t] == 0.0)
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol * scale)
    s.close()


def _pair(case, state_seed, precision):
    s = _sim(case, precision=precision)
    o = oracle.Sim(case)
    v, w, ve = W.random_state(state_seed, case)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    return s, o


@pytest.mark.parametrize("shape", [(8, 7, 6), (35, 10, 9)])
def test_one_step_monodomain_fp64(shape):
    c = W.random_case(2, *shape, model=W.MONO, dt=0.02).fibres_as_float32()
    s, o = _pair(c, 2, ep.EP_FP64)
    for _ in range(3):
        s.step(1)
        o.step()
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(s.read(ep.EP_W), st["w"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(s.read(ep.EP_TACT), st["tact"], rtol=0, atol=1e-9)


def test_one_step_bidomain_fp64_tight_solve():
    c = W.random_case(3, 13, 9, 8, model=W.BI, rel_tol=1e-11, check_every=5).fibres_as_float32()
    c.params.max_iter = 200000
    s, o = _pair(c, 3, ep.EP_FP64)
    for _ in range(2):
        stats = s.step(1)
        assert o.step() == 0
        assert stats.converged == 1
        assert stats.iters == o.last_iters   # the same iteration: exact diagonal, same stop rule
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(s.read(ep.EP_W), st["w"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7)


def _elliptic_relres(case, v, ve):
    """||b - (L_i + L_e) ve|| / ||b|| with b = -L_i v (zero mean per component),
    evaluated by the FP64 oracle."""
    g = oracle.Grid.from_case(case)
    p = case.params
    t = case.mask.reshape(-1) > 0
    b = -g.apply_L(p.sig_iL, p.sig_iT, np.where(t, v, 0.0))
    nc, comp = g.components()
    for cc in range(nc):
        sel = comp == cc
        b[sel] -= b[sel].mean()
    r = b - g.apply_L(p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT, np.where(t, ve, 0.0))
    return np.linalg.norm(r[t]) / np.linalg.norm(b[t])


def test_multistep_bidomain_fp32_small_shell():
    """FP32 GPU vs FP64 oracle over 100 steps of a small shell (unequal
    anisotropy): V_m within 0.5 mV, activation times within 1 %, and the GPU's
    extracellular potential solves the oracle's elliptic equation."""
    n = 20
    sc = n / 128
    c = W.shell_case(n, (40 * sc, 40 * sc, 55 * sc), 2.5, (0.2, 0.05, 0.2, 0.1), 0.05, 100, 4)
    s = _sim(c)
    o = oracle.Sim(c)
    for _ in range(c.steps):
        s.step(1, allow_noconv=True)
        o.step()
    st = o.state()
    vm_gpu, vm_ref = s.read(ep.EP_VM_MV), oracle.vm_mV(st["v"])
    assert np.abs(vm_gpu - vm_ref).max() <= 0.5
    ta_g, ta_r = s.read(ep.EP_TACT), st["tact"]
    act = ta_r > 0
    assert act.sum() > 20
    np.testing.assert_array_equal(ta_g > 0, act)
    assert np.all(np.abs(ta_g[act] - ta_r[act]) <= 0.01 * ta_r[act])
    rr = _elliptic_relres(c, s.read(ep.EP_V), s.read(ep.EP_VE))
    assert rr <= 2e-5, rr


@pytest.mark.parametrize("model", [W.MONO, W.BI])
def test_slab_fp32_matches_oracle(model):
    """The dense-slab construction of the roofline workload, at 24^3: FP32 GPU
    vs FP64 oracle over 60 steps, V_m within 0.5 mV, activation times within 1 %."""
    c = W.slab(24, model, unequal=model == W.BI)
    s = _sim(c)
    o = oracle.Sim(c)
    for _ in range(60):
        s.step(1, allow_noconv=True)
        o.step()
    st = o.state()
    assert np.abs(s.read(ep.EP_VM_MV) - oracle.vm_mV(st["v"])).max() <= 0.5
    ta_g, ta_r = s.read(ep.EP_TACT), st["tact"]
    act = ta_r > 0
    assert act.sum() > 50
    np.testing.assert_array_equal(ta_g > 0, act)
    assert np.all(np.abs(ta_g[act] - ta_r[act]) <= 0.01 * ta_r[act])


def test_config0_fp64_parity():
    """Config 0 (monodomain FP64 slab, 1000 steps): max |dV_m| <= 1e-3 mV and
    activation times within 1 %."""
    c = W.config0()
    s = _sim(c)
    o = oracle.Sim(c)
    s.step(c.steps)
    o.run(c.steps)
    st = o.state()
    dv = np.abs(s.read(ep.EP_VM_MV) - oracle.vm_mV(st["v"])).max()
    assert dv <= 1e-3, dv
    ta_g, ta_r = s.read(ep.EP_TACT), st["tact"]
    act = ta_r > 0
    assert act.sum() > 100
    np.testing.assert_array_equal(ta_g > 0, act)
    assert np.all(np.abs(ta_g[act] - ta_r[act]) <= 0.01 * ta_r[act])


def test_rest_state_is_fixed_point_bitwise():
    for model in (ep.EP_MONO, ep.EP_BI):
        c = W.random_case(5, 31, 12, 9, model=model)
        c.stimuli = []
        s = _sim(c)
        stats = s.step(5)
        assert stats.total_iters == 0
        assert np.all(s.read(ep.EP_V) == 0.0) and np.all(s.read(ep.EP_W) == 1.0)
        assert np.all(s.read(ep.EP_VE) == 0.0) and np.all(s.read(ep.EP_TACT) == -1.0)


def test_charge_conservation_fp64():
    c = W.random_case(6, 40, 11, 10, model=W.MONO)
    c.stimuli = []
    p = c.params
    p.tau_in = p.tau_out = p.tau_open = p.tau_close = 1e300
    s = _sim(c, precision=ep.EP_FP64)
    v, w, ve = W.random_state(6, c)
    s.set_state(v, w, ve)
    s.step(4)
    v1 = s.read(ep.EP_V)
    assert abs(v1.sum() - v.sum()) <= 1e-12 * np.abs(v).sum()


def test_equal_anisotropy_ve_is_minus_half_v():
    c = W.random_case(7, 14, 10, 9, model=W.BI, unequal=False, rel_tol=1e-11, check_every=5)
    c.params.max_iter = 300000
    s = _sim(c, precision=ep.EP_FP64)
    v, w, ve = W.random_state(7, c)
    s.set_state(v, w, ve)
    s.step(1)
    nc, comp = oracle.Grid.from_case(c).components()
    V, VE = s.read(ep.EP_V), s.read(ep.EP_VE)
    for cc in range(nc):
        sel = comp == cc
        np.testing.assert_allclose(VE[sel], -(V[sel] - V[sel].mean()) / 2, rtol=0, atol=1e-8)


def test_snapshot_resume_and_determinism():
    c = W.random_case(8, 29, 13, 11, model=W.BI)
    a = _sim(c)
    a.step(6)
    blob = a.read_state()
    a.step(5)
    ref = [a.read(f) for f in (ep.EP_V, ep.EP_W, ep.EP_VE, ep.EP_TACT)]
    b = _sim(c)
    b.write_state(blob)
    b.step(5)
    got = [b.read(f) for f in (ep.EP_V, ep.EP_W, ep.EP_VE, ep.EP_TACT)]
    for x, y in zip(ref, got):
        np.testing.assert_array_equal(x, y)


def test_noconvergence_is_reported_and_step_completes():
    c = W.random_case(9, 16, 12, 10, model=W.BI)
    c.params.max_iter = 7
    c.params.check_every = 3
    s = _sim(c)
    v, w, ve = W.random_state(9, c)
    s.set_state(v, w, ve)
    stats = s.step(1, allow_noconv=True)
    assert s.last_status == ep.EP_ENOCONV
    assert stats.iters == 7 and stats.step == 1


def _fullsize_checks(case, state_seed):
    """One full-size launch of each kernel family against the oracle."""
    g = oracle.Grid.from_case(case)
    s = _sim(case)
    t = case.mask.reshape(-1) > 0
    rng = np.random.default_rng(state_seed)
    u = rng.standard_normal(g.n)
    ref = g.apply_L(0.4, 0.15, np.where(t, u, 0.0))
    got = s.apply_operator(0.4, 0.15, u)
    np.testing.assert_allclose(got, ref, rtol=0, atol=FP32_OP_RTOL * np.abs(ref).max())
    # one bidomain step from a propagating state: v and w do not depend on the solve
    v, w, ve = W.random_state(state_seed, case)
    s.set_state(v, w, ve, 10)
    stats = s.step(1, allow_noconv=True)
    p1 = W.Params(**{**case.params.__dict__, "max_iter": 1})
    o = oracle.Sim(case, params=p1)
    o.set_state(v, w, ve, 10)
    o.step()
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=5e-6)
    np.testing.assert_allclose(s.read(ep.EP_W), st["w"], rtol=0, atol=1e-6)
    rr = _elliptic_relres(case, s.read(ep.EP_V), s.read(ep.EP_VE))
    return stats, rr


def test_config1_fullsize_kernels():
    c = W.config1(unequal=True)
    c.params.max_iter = 200000
    stats, rr = _fullsize_checks(c, 11)
    assert stats.iters > 0
    assert rr <= 2e-5, (rr, stats.iters, stats.rel_res)


def test_config2_fullsize_kernels():
    c = W.config2(unequal=True)
    c.params.max_iter = 4000   # a capped solve: the residual is checked against the reported one
    stats, rr = _fullsize_checks(c, 12)
    assert stats.iters > 0
    assert abs(rr - stats.rel_res) <= 0.05 * stats.rel_res + 1e-5, (rr, stats.rel_res)


@pytest.mark.parametrize("solver", [0, 1])
def test_fp32_correction_form_on_several_components_against_oracle(solver):
    """FP32 damped Jacobi and Chebyshev (correction form, R22) on a random mask
    with several face-connected components, each solve from v_e = 0 (a cold
    start: cycles restart along the way): every step converges, and V_m and
    V_e agree with the FP64 oracle (V_e to 0.05 mV: both solves stop at the
    same relative residual, 1e-6, not at the same iterate)."""
    import spectra
    c = W.random_case(57, 33, 21, 14, model=W.BI, fill=0.5)
    c.params.max_iter = 400000
    g = oracle.Grid.elliptic_from_case(c)
    assert g.components()[0] > 1
    if solver == 1:   # an interval from the oracle's operator: Lanczos top, a literal bottom below the spectrum's
        p = c.params
        hi = spectra.largest(g, p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT)
        c.params.solver, c.params.cheb_lmin, c.params.cheb_lmax = 1, 1e-4, 1.05 * hi
    s = ep.sim_from_case(c)
    o = oracle.Sim(c)
    v, w, _ = W.random_state(57, c)
    ve = np.zeros(c.n)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    for _ in range(3):
        assert s.step(1).converged == 1
        assert o.step() == 0
    st = o.state()
    assert np.abs(s.read(ep.EP_VM_MV) - oracle.vm_mV(st["v"])).max() <= 0.5
    assert np.abs(s.read(ep.EP_VE_MV) - 100.0 * st["ve"]).max() <= 0.05
    s.close()
    o.close()
