"""Implicit-Euler diffusion (Sec. "Implicit Euler", Eq. iejac1) on the CUDA
path against the FP64 oracle: the same Jacobi iteration with the same stop
rule, element by element, in FP64 and FP32, and its error handling."""
import numpy as np
import pytest

import oracle
import paper_2302_12519_gb300 as ep
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_12519_gb300 import build
    build.build()
    ep.load()
    oracle.build()


def _ie_case(seed, shape, model, **kw):
    c = W.random_case(seed, *shape, model=model, **kw)
    c.params.diffusion = 1
    return c


def _pair(case, state_seed, precision):
    s = ep.sim_from_case(case, precision=precision)
    o = oracle.Sim(case)
    v, w, ve = W.random_state(state_seed, case)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    return s, o


@pytest.mark.parametrize("shape", [(8, 7, 6), (35, 10, 9)])
def test_implicit_monodomain_fp64_matches_oracle(shape):
    """Three implicit steps: same sweeps to the same stop rule, so the states
    agree to rounding and the sweep counts are equal."""
    c = _ie_case(21, shape, W.MONO, dt=0.05, rel_tol=1e-10, check_every=3).fibres_as_float32()
    s, o = _pair(c, 21, ep.EP_FP64)
    total = 0
    for _ in range(3):
        stats = s.step(1)
        assert o.step() == 0
        total += stats.ie_total_iters
    st = o.state()
    assert total == o.ie_total_iters > 0
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(s.read(ep.EP_W), st["w"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(s.read(ep.EP_TACT), st["tact"], rtol=0, atol=1e-9)


def test_implicit_bidomain_fp64_matches_oracle():
    c = _ie_case(22, (13, 9, 8), W.BI, rel_tol=1e-11, check_every=5).fibres_as_float32()
    c.params.max_iter = 200000
    s, o = _pair(c, 22, ep.EP_FP64)
    for _ in range(2):
        stats = s.step(1)
        assert o.step() == 0
        assert stats.converged == 1
    st = o.state()
    assert s.read(ep.EP_V).shape == st["v"].shape
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(s.read(ep.EP_W), st["w"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7)


@pytest.mark.parametrize("model", [W.MONO, W.BI])
def test_implicit_fp32_small_shell_against_oracle(model):
    """FP32 GPU vs FP64 oracle over 100 implicit steps of a small shell:
    V_m within 0.5 mV, activation times within 1 %."""
    n = 20
    sc = n / 128
    c = W.shell_case(n, (40 * sc, 40 * sc, 55 * sc), 2.5, (0.2, 0.05, 0.2, 0.1), 0.05, 100, 4)
    c.model = model
    c.params.diffusion = 1
    s = ep.sim_from_case(c)
    o = oracle.Sim(c)
    for _ in range(c.steps):
        s.step(1, allow_noconv=True)
        o.step()
    st = o.state()
    assert np.abs(s.read(ep.EP_VM_MV) - oracle.vm_mV(st["v"])).max() <= 0.5
    ta_g, ta_r = s.read(ep.EP_TACT), st["tact"]
    act = ta_r > 0
    assert act.sum() > 20
    np.testing.assert_array_equal(ta_g > 0, act)
    assert np.all(np.abs(ta_g[act] - ta_r[act]) <= 0.01 * ta_r[act])


def test_implicit_solve_cap_is_reported():
    c = _ie_case(23, (16, 12, 10), W.MONO, rel_tol=1e-14, check_every=2).fibres_as_float32()
    c.params.max_iter = 3
    s, o = _pair(c, 23, ep.EP_FP64)
    stats = s.step(1, allow_noconv=True)
    assert s.last_status == ep.EP_ENOCONV and stats.ie_total_iters == 3 and stats.converged == 0
    assert o.step() == 1
    np.testing.assert_allclose(s.read(ep.EP_V), o.state()["v"], rtol=0, atol=1e-12)


def test_implicit_handles_are_not_batched():
    c = _ie_case(24, (12, 10, 8), W.BI)
    s = ep.sim_from_case(c)
    b = ep.Batch(2)
    with pytest.raises(ep.EPError) as e:
        b.add(s)
    assert e.value.status == ep.EP_EINVAL
    b.close()
