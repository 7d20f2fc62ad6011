"""Chebyshev-accelerated elliptic solve on the CUDA path: parity with the FP64
oracle's semi-iteration on the same interval (computed from the oracle's
operator, never from the library), the set-up estimate of the interval against
the oracle's spectrum, and the sweep savings."""
import numpy as np
import pytest

import oracle
import paper_2302_12519_gb300 as ep
import spectra
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_12519_gb300 import build
    build.build()
    ep.load()
    oracle.build()


def _dense_interval(case):
    """Smallest nonzero and largest eigenvalue of D^-1 A for the elliptic
    operator of the case, from the oracle's operator."""
    p = case.params
    return spectra.interval(oracle.Grid.elliptic_from_case(case), p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT)


def test_chebyshev_fp64_matches_oracle_on_the_same_interval():
    c = W.random_case(41, 13, 9, 8, model=W.BI, rel_tol=1e-11, check_every=5).fibres_as_float32()
    c.params.max_iter = 200000
    lo, hi = _dense_interval(c)
    c.params.solver, c.params.cheb_lmin, c.params.cheb_lmax = 1, 0.9 * lo, 1.1 * hi
    s = ep.sim_from_case(c, precision=ep.EP_FP64)
    o = oracle.Sim(c)
    v, w, ve = W.random_state(41, c)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    assert s.info().cheb_lmin == c.params.cheb_lmin
    for _ in range(2):
        stats = s.step(1)
        assert o.step() == 0 and stats.converged == 1 and stats.iters == o.last_iters
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7)


def test_estimated_interval_brackets_the_spectrum():
    """The set-up Lanczos estimate: lmax at or above the largest eigenvalue of
    D^-1 A (the library's fibres are the float32 values, within 1e-5), lmin
    between half and all of the smallest nonzero one."""
    c = W.random_case(42, 12, 10, 9, model=W.BI)
    c.params.solver = 1
    lo, hi = _dense_interval(c)
    s = ep.sim_from_case(c)
    info = s.info()
    assert hi * (1 - 1e-5) <= info.cheb_lmax <= hi * 1.1
    assert 0.5 * lo <= info.cheb_lmin <= 1.0 * lo


def test_chebyshev_fp32_shell_against_oracle_and_sweep_savings():
    """FP32 GPU vs FP64 oracle over 100 steps of a small shell, both on the
    interval of the oracle's spectrum (scaled as the set-up scales its
    estimate): V_m within 0.5 mV and activation times within 1 %, in a
    fraction of the damped-Jacobi sweeps."""
    n = 24
    sc = n / 128
    c = W.shell_case(n, (40 * sc, 40 * sc, 55 * sc), 3.0, (0.2, 0.05, 0.2, 0.1), 0.05, 100, 4)
    jac = ep.sim_from_case(c)
    jac_iters = sum(jac.step(1, allow_noconv=True).total_iters for _ in range(c.steps))
    c.params.solver = 1
    p = c.params
    c.params.cheb_lmin, c.params.cheb_lmax = spectra.chebyshev_params(
        oracle.Grid.elliptic_from_case(c), p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT)
    s = ep.sim_from_case(c)
    assert s.info().cheb_lmin == c.params.cheb_lmin
    o = oracle.Sim(c)
    cheb_iters = 0
    for _ in range(c.steps):
        st = s.step(1)   # the FP32 correction form reaches the tolerance at every step
        assert st.converged == 1
        cheb_iters += st.total_iters
        o.step()
    st = o.state()
    assert np.abs(s.read(ep.EP_VM_MV) - oracle.vm_mV(st["v"])).max() <= 0.5
    ta_g, ta_r = s.read(ep.EP_TACT), st["tact"]
    act = ta_r > 0
    assert act.sum() > 20
    np.testing.assert_array_equal(ta_g > 0, act)
    assert np.all(np.abs(ta_g[act] - ta_r[act]) <= 0.01 * ta_r[act])
    assert cheb_iters * 3 < jac_iters, (cheb_iters, jac_iters)


def test_chebyshev_interval_is_validated():
    c = W.random_case(43, 8, 8, 8, model=W.BI)
    c.params.solver, c.params.cheb_lmin, c.params.cheb_lmax = 1, 2.0, 1.0
    with pytest.raises(ep.EPError) as e:
        ep.sim_from_case(c)
    assert e.value.status == ep.EP_EINVAL


def test_estimated_jacobi_damping_is_stable_and_matches_oracle():
    """jacobi_omega < 0: damping from the set-up spectrum estimate,
    omega = min(1, 1.9 / lmax), lmax the largest Lanczos Ritz value scaled by
    1.05.  The library's omega keeps omega lambda_max(D^-1 A) below 2 on the
    oracle's spectrum and lies within 1 % of the rule applied to that spectrum;
    with the rule's omega from the oracle's spectrum given to both sides, the
    FP64 damped Jacobi solve equals the oracle's sweep for sweep."""
    c = W.random_case(44, 13, 9, 8, model=W.BI, rel_tol=1e-11, check_every=5).fibres_as_float32()
    c.params.max_iter = 400000
    c.params.omega = -1.0
    lo, hi = _dense_interval(c)
    s0 = ep.sim_from_case(c, precision=ep.EP_FP64)
    info = s0.info()
    s0.close()
    omega_ref = min(1.0, 1.9 / (1.05 * hi))
    assert info.omega * hi < 2.0
    assert info.omega == pytest.approx(omega_ref, rel=1e-2)
    c.params.omega = omega_ref
    s = ep.sim_from_case(c, precision=ep.EP_FP64)
    assert s.info().omega == omega_ref
    o = oracle.Sim(c)
    v, w, ve = W.random_state(44, c)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    for _ in range(2):
        stats = s.step(1)
        assert o.step() == 0 and stats.converged == 1 and stats.iters == o.last_iters
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7)
