"""Torso and ECG on the CUDA path (Eq. bidomain1, lines 3-5; Sec.
"Electrocardiogram") against the FP64 oracle: the elliptic operator over
tissue + torso element by element, the bidomain step with a torso, the ECG
traces of a small heart in a box, and the error handling of the calls."""
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


def _torso_case(seed, shape, fill=0.85, sig_o=0.7, **kw):
    """Random tissue in a random torso; fibres rounded to float32, the values
    the library receives, so FP64 comparisons see rounding of the sums only."""
    base = W.random_case(seed, *shape, fill=0.45, **kw)
    return W.with_torso(base, sig_o=sig_o, fill=fill, seed=seed).fibres_as_float32()


def _oracle_interval(c):
    """The Chebyshev interval from the oracle's spectrum of D^-1 A over tissue +
    torso, scaled as the library scales its own estimate."""
    p = c.params
    return spectra.chebyshev_params(oracle.Grid.elliptic_from_case(c), p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT)


@pytest.mark.parametrize("shape", [(9, 7, 6), (70, 19, 37)])
@pytest.mark.parametrize("precision", [ep.EP_FP64, ep.EP_FP32])
def test_elliptic_operator_with_torso_matches_oracle(shape, precision):
    """The z-march kernel's elliptic operator (several work items in x, y and
    z, a ragged tail) against the oracle's on tissue + torso."""
    c = _torso_case(61, shape)
    p = c.params
    s = ep.sim_from_case(c, precision=precision)
    info = s.info()
    g = oracle.Grid.elliptic_from_case(c)
    dom = g.domain()
    assert info.n_domain == int(dom.sum()) and info.n_tissue == c.n_tissue
    rng = np.random.default_rng(61)
    u = rng.standard_normal(c.n) * dom
    got = s.apply_elliptic(u)
    ref = g.apply_L(p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT, u)
    scale = np.abs(ref).max()
    tol = 1e-12 if precision == ep.EP_FP64 else 2e-6
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol * scale)
    assert np.all(got[~dom] == 0.0)


def test_bidomain_step_with_torso_fp64_matches_oracle():
    """Three steps: the same sweeps to the same stop rule over tissue + torso,
    so v, w and v_e (on the torso too) agree to rounding."""
    c = _torso_case(62, (13, 10, 9), rel_tol=1e-11, check_every=5)
    c.params.max_iter = 400000
    s = ep.sim_from_case(c, precision=ep.EP_FP64)
    o = oracle.Sim(c)
    v, w, ve = W.random_state(62, c)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    for _ in range(3):
        stats = s.step(1)
        assert o.step() == 0 and stats.converged == 1
        assert stats.iters == o.last_iters
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(s.read(ep.EP_W), st["w"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7)
    off = c.mask.reshape(-1) == 0
    assert np.any(np.abs(st["ve"][off]) > 1e-4)   # the torso carries potential


def _heart_in_box(n=20, pad=2, steps=40, sig_o=1.0):
    """A small shell in a torso box, solved by the Chebyshev semi-iteration
    (damped Jacobi needs some 4e4 sweeps per step on this machine)."""
    sc = n / 128
    c = W.shell_case(n, (40 * sc, 40 * sc, 55 * sc), 3.0, (0.2, 0.05, 0.2, 0.1), 0.05, steps, 4)
    c = W.with_torso(c, sig_o=sig_o, pad=pad)
    c.params.solver = 1
    return c


def test_ecg_of_a_small_heart_in_a_torso_fp32_against_oracle():
    """FP32 GPU vs FP64 oracle (the same semi-iteration on the interval of the
    oracle's spectrum) over 40 steps of a small shell in a torso box: V_m
    within 0.5 mV, activation times within 1 %, and the electrode potentials
    and six leads within 2 % of the trace's range (both solves stop at the same
    relative residual, 1e-6, not at the same iterate)."""
    c = _heart_in_box()
    c.params.cheb_lmin, c.params.cheb_lmax = _oracle_interval(c)
    s = ep.sim_from_case(c, ecg_capacity=c.steps)
    o = oracle.Sim(c)
    phi_o = []
    for _ in range(c.steps):
        assert s.step(1).converged == 1   # the FP32 correction form reaches the tolerance at every step
        o.step()
        phi_o.append(oracle.electrode_potentials(c, o.state()["ve"]))
    t, phi, lead = s.read_ecg()
    phi_o = np.array(phi_o)
    assert phi.shape == (c.steps, 3)
    np.testing.assert_allclose(t, c.params.dt * np.arange(1, c.steps + 1), rtol=1e-12)
    span = np.ptp(phi_o)
    assert span > 0.05                                      # the heart beats into the torso
    np.testing.assert_allclose(phi, phi_o, rtol=0, atol=0.02 * span)
    lead_o = oracle.ecg_leads(phi_o)
    np.testing.assert_allclose(lead, lead_o, rtol=0, atol=0.04 * span)
    np.testing.assert_allclose(lead[:, 0] + lead[:, 2], lead[:, 1], atol=1e-9)   # Einthoven
    st = o.state()
    assert np.abs(s.read(ep.EP_VM_MV) - oracle.vm_mV(st["v"])).max() <= 0.5
    ta_g, ta_r = s.read(ep.EP_TACT), st["tact"]
    act = ta_r > 0
    assert act.sum() > 20
    np.testing.assert_array_equal(ta_g > 0, act)
    assert np.all(np.abs(ta_g[act] - ta_r[act]) <= 0.01 * ta_r[act])


def test_ecg_record_capacity_and_drain():
    c = _heart_in_box(n=16, pad=2, steps=10)
    s = ep.sim_from_case(c, ecg_capacity=4)
    s.step(3, allow_noconv=True)
    with pytest.raises(ep.EPError) as e:
        s.step(2)
    assert e.value.status == ep.EP_EBUSY
    t, phi, lead = s.read_ecg()
    assert len(t) == 3 and np.allclose(t, c.params.dt * np.arange(1, 4))
    s.step(4, allow_noconv=True)
    t2, _, _ = s.read_ecg()
    assert len(t2) == 4 and np.allclose(t2, c.params.dt * np.arange(4, 8))
    assert len(s.read_ecg()[0]) == 0


def test_torso_and_ecg_errors():
    c = _heart_in_box(n=16, pad=2, steps=10)
    mono = W.with_torso(W.random_case(63, 10, 9, 8, model=W.MONO), sig_o=1.0)
    with pytest.raises(ep.EPError) as e:
        ep.sim_from_case(mono).info()
    assert e.value.status == ep.EP_EINVAL
    s = ep.sim_from_case(c)
    s.info()
    with pytest.raises(ep.EPError) as e:
        s.set_torso(c.torso, 1.0)
    assert e.value.status == ep.EP_ESTATE
    bad = W.random_case(64, 10, 9, 8)
    bad.mask[0, 0, 0] = 0                   # an electrode off the tissue, and no torso
    s2 = ep.sim_from_case(bad)
    s2.set_ecg([(0, 0, 0), (9, 8, 7), (5, 4, 3)], 8)
    with pytest.raises(ep.EPError) as e:
        s2.info()
    assert e.value.status == ep.EP_EINVAL
    with pytest.raises(ep.EPError) as e:
        ep.sim_from_case(bad).set_ecg([(0, 0, 0), (10, 0, 0), (1, 1, 1)], 8)   # outside the grid
    assert e.value.status == ep.EP_EINVAL
    b = ep.Batch(2)
    with pytest.raises(ep.EPError) as e:
        b.add(ep.sim_from_case(c))
    assert e.value.status == ep.EP_EINVAL
    b.close()


def test_chebyshev_interval_with_torso_brackets_the_spectrum():
    """The device Lanczos over tissue + torso: lmax at or above the largest
    eigenvalue of D^-1 A of the torso operator, lmin between half and all of
    the smallest nonzero one."""
    c = _torso_case(65, (9, 8, 7), fill=0.9)
    c.params.solver = 1
    g = oracle.Grid.elliptic_from_case(c)
    p = c.params
    sL, sT = p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT
    t = np.nonzero(g.domain())[0]
    A = np.zeros((len(t), len(t)))
    for col, q in enumerate(t):
        e = np.zeros(g.n)
        e[q] = 1.0
        A[:, col] = g.apply_L(sL, sT, e)[t]
    d = np.diag(A)
    keep = d > 0
    A, d = A[np.ix_(keep, keep)], d[keep]
    lam = np.linalg.eigvalsh(A / np.sqrt(d)[:, None] / np.sqrt(d)[None, :])
    lo, hi = lam[lam > 1e-9].min(), lam.max()
    info = ep.sim_from_case(c).info()
    assert hi * (1 - 1e-5) <= info.cheb_lmax <= hi * 1.1
    assert 0.5 * lo <= info.cheb_lmin <= 1.0 * lo


def test_chebyshev_fp64_with_torso_matches_oracle():
    """FP64 Chebyshev semi-iteration over tissue + torso on an interval both
    sides share (from the oracle's spectrum): the same iterates to the same
    stop rule."""
    c = _torso_case(66, (11, 9, 8), fill=0.9, rel_tol=1e-11, check_every=5)
    c.params.max_iter = 200000
    c.params.solver = 1
    c.params.cheb_lmin, c.params.cheb_lmax = _oracle_interval(c)
    s = ep.sim_from_case(c, precision=ep.EP_FP64)
    o = oracle.Sim(c)
    v, w, ve = W.random_state(66, c)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    for _ in range(2):
        stats = s.step(1)
        assert o.step() == 0 and stats.converged == 1 and stats.iters == o.last_iters
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7)


def test_noalloc_step_with_torso_and_ecg_equals_step():
    """ep_step_noalloc on a torso handle (its own sweep items, the ECG record)
    gives the states and samples of ep_step."""
    c = _heart_in_box(n=16, pad=2, steps=6)
    a = ep.sim_from_case(c, ecg_capacity=8)
    b = ep.sim_from_case(c, ecg_capacity=8)
    a.info()
    b.info()
    for _ in range(3):
        a.step(2, allow_noconv=True)
        b.step_noalloc(2, allow_noconv=True)
    np.testing.assert_array_equal(a.read(ep.EP_V), b.read(ep.EP_V))
    np.testing.assert_array_equal(a.read(ep.EP_VE), b.read(ep.EP_VE))
    ta, pa, _ = a.read_ecg()
    tb, pb, _ = b.read_ecg()
    np.testing.assert_array_equal(ta, tb)
    np.testing.assert_array_equal(pa, pb)


def test_ecg_workload_fullsize_operator_and_capped_step():
    """The bench's ECG workload at full size (256^3, torso over the whole
    box): the two-term operator against the oracle's, and one step with a
    capped damped-Jacobi solve whose final residual, recomputed by the oracle
    in FP64 over tissue + torso, matches the one the GPU reported."""
    c = W.ecg_case()
    p = c.params
    p.max_iter = 4000
    sL, sT = p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT
    ge, gh = oracle.Grid.elliptic_from_case(c), oracle.Grid.from_case(c)
    dom = ge.domain()
    s = ep.sim_from_case(c)
    rng = np.random.default_rng(67)
    u = rng.standard_normal(c.n) * dom
    ref = ge.apply_L(sL, sT, u)
    np.testing.assert_allclose(s.apply_elliptic(u), ref, rtol=0, atol=2e-6 * np.abs(ref).max())
    v, w, ve = W.random_state(67, c)
    s.set_state(v, w, ve, 10)
    stats = s.step(1, allow_noconv=True)
    assert stats.iters > 0
    vg, xg = s.read(ep.EP_V), s.read(ep.EP_VE)
    b = -gh.apply_L(p.sig_iL, p.sig_iT, vg)
    b[c.mask.reshape(-1) == 0] = 0.0
    b[dom] -= b[dom].mean()          # one component: the whole box
    r = b - ge.apply_L(sL, sT, xg)
    rr = np.linalg.norm(r[dom]) / np.linalg.norm(b[dom])
    assert abs(rr - stats.rel_res) <= 0.05 * stats.rel_res + 1e-5, (rr, stats.rel_res)


def test_far_items_single_term_sweep_matches_oracle():
    """A small heart padded by a thick torso: the items whose stencil reach holds
    no tissue run the single-term kernel (sigma = sig_o I), the rest the two-term
    one.  The FP64 solve to 1e-11 (Chebyshev, both sides on the interval of the
    oracle's spectrum) equals the oracle's.  (Unconverged iterates are not
    compared: the library's Jacobi diagonal is 1/D rounded to float32, which
    changes the iterates but not the solution.)"""
    base = W.random_case(68, 8, 8, 8, fill=0.7, rel_tol=1e-11, check_every=5)
    c = W.with_torso(base, sig_o=0.9, pad=12).fibres_as_float32()
    c.params.max_iter = 400000
    c.params.solver = 1
    c.params.cheb_lmin, c.params.cheb_lmax = _oracle_interval(c)
    s = ep.sim_from_case(c, precision=ep.EP_FP64)
    info = s.info()
    assert 0 < info.n_segments_far < info.n_segments_elliptic
    o = oracle.Sim(c)
    v, w, ve = W.random_state(68, c)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    for _ in range(2):
        stats = s.step(1)
        assert o.step() == 0 and stats.converged == 1
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7)


def test_torso_fp32_jacobi_correction_form_against_oracle():
    """The FP32 damped Jacobi in correction form over tissue + torso (the
    single-term and two-term launches of one sweep both fold and restart):
    every step converges, and V_m and V_e agree with the FP64 oracle within the
    full-run gates (0.5 mV; both solves stop at rel_tol 1e-5)."""
    c = _heart_in_box(steps=2)
    c.params.solver, c.params.rel_tol, c.params.max_iter = 0, 1e-5, 400000
    s = ep.sim_from_case(c)
    o = oracle.Sim(c)
    for _ in range(c.steps):
        assert s.step(1).converged == 1
        assert o.step() == 0
    st = o.state()
    assert np.abs(s.read(ep.EP_VM_MV) - oracle.vm_mV(st["v"])).max() <= 0.5
    dve = np.abs(s.read(ep.EP_VE_MV) - 100.0 * st["ve"]).max()
    assert dve <= 0.5, dve
    s.close()
    o.close()
