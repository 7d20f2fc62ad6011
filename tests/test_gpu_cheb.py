"""Chebyshev-accelerated elliptic solve on the CUDA path: parity with the FP64
oracle's semi-iteration on the same interval, the set-up estimate of the
interval against a dense eigendecomposition, and the sweep savings."""
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


def _dense_interval(case):
    """Smallest nonzero and largest eigenvalue of D^-1 A for the elliptic
    operator of the case (dense, from the oracle's operator)."""
    g = oracle.Grid.from_case(case)
    p = case.params
    sL, sT = p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT
    t = np.nonzero(g.mask)[0]
    A = np.zeros((len(t), len(t)))
    for col, q in enumerate(t):
        e = np.zeros(g.n)
        e[q] = 1.0
        A[:, col] = g.apply_L(sL, sT, e)[t]
    d = np.diag(A)
    keep = d > 0
    A, d = A[np.ix_(keep, keep)], d[keep]
    lam = np.linalg.eigvalsh(A / np.sqrt(d)[:, None] / np.sqrt(d)[None, :])
    return lam[lam > 1e-9].min(), lam.max()


def test_chebyshev_fp64_matches_oracle_on_the_same_interval():
    c = W.random_case(41, 13, 9, 8, model=W.BI, rel_tol=1e-11, check_every=5)
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
        assert o.step() == 0 and stats.converged == 1
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7)


def test_estimated_interval_brackets_the_spectrum():
    """The set-up Lanczos estimate: lmax at or above the largest eigenvalue of
    D^-1 A (the library's diagonal is the fp16-rounded one, within 0.1 %),
    lmin between half and all of the smallest nonzero one."""
    c = W.random_case(42, 12, 10, 9, model=W.BI)
    c.params.solver = 1
    lo, hi = _dense_interval(c)
    s = ep.sim_from_case(c)
    info = s.info()
    assert hi * 0.999 <= info.cheb_lmax <= hi * 1.1
    assert 0.5 * lo <= info.cheb_lmin <= 1.0 * lo


def test_chebyshev_fp32_shell_against_oracle_and_sweep_savings():
    """FP32 GPU (estimated interval) vs FP64 oracle (the same interval) over 100
    steps of a small shell: V_m within 0.5 mV and activation times within 1 %,
    in a fraction of the damped-Jacobi sweeps."""
    n = 24
    sc = n / 128
    c = W.shell_case(n, (40 * sc, 40 * sc, 55 * sc), 3.0, (0.2, 0.05, 0.2, 0.1), 0.05, 100, 4)
    jac = ep.sim_from_case(c)
    jac_iters = sum(jac.step(1, allow_noconv=True).total_iters for _ in range(c.steps))
    c.params.solver = 1
    s = ep.sim_from_case(c)
    info = s.info()
    c.params.cheb_lmin, c.params.cheb_lmax = info.cheb_lmin, info.cheb_lmax
    o = oracle.Sim(c)
    cheb_iters = 0
    for _ in range(c.steps):
        cheb_iters += s.step(1, allow_noconv=True).total_iters
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
    omega = 1.9 / lmax.  It keeps omega lambda_max(D^-1 A) below 2 on the
    dense spectrum, and with that omega the FP64 damped Jacobi solve equals the
    oracle's."""
    c = W.random_case(44, 13, 9, 8, model=W.BI, rel_tol=1e-11, check_every=5)
    c.params.max_iter = 400000
    c.params.omega = -1.0
    lo, hi = _dense_interval(c)
    s = ep.sim_from_case(c, precision=ep.EP_FP64)
    info = s.info()
    assert info.omega == pytest.approx(min(1.0, 1.9 / info.cheb_lmax), rel=1e-15)
    assert info.omega * hi < 2.0
    c.params.omega = info.omega
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
