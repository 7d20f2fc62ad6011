"""Eight-colour Gauss-Seidel / SOR elliptic solve on the CUDA path (the
deterministic form of the paper's in-place Jacobi): parity with the FP64
oracle's colour sweep on the same inputs, sweep for sweep, in FP64; FP32
against the FP64 oracle over a run; determinism of the in-place passes; the
refusals (torso, batch)."""
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


@pytest.mark.parametrize("seed,omega", [(51, 0.0), (52, 1.4)])
def test_gauss_seidel_fp64_matches_oracle_sweep_for_sweep(seed, omega):
    """Random masks (several components, ragged tiles), random state: the same
    sweep counts as the oracle and the same potentials, for Gauss-Seidel
    (omega <= 0 selects 1) and SOR."""
    c = W.random_case(seed, 37, 11, 9, model=W.BI, rel_tol=1e-10, check_every=3).fibres_as_float32()
    c.params.solver, c.params.omega, c.params.max_iter = 2, omega, 100000
    s = ep.sim_from_case(c, precision=ep.EP_FP64)
    assert s.info().omega == (omega if omega > 0 else 1.0)
    o = oracle.Sim(c)
    v, w, ve = W.random_state(seed, c)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    for _ in range(3):
        stats = s.step(1)
        assert o.step() == 0 and stats.converged == 1 and stats.iters == o.last_iters, (stats.iters, o.last_iters)
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7 * max(1.0, np.abs(st["ve"]).max()))
    s.close()
    o.close()


def test_gauss_seidel_one_capped_sweep_equals_oracle():
    """One sweep (max_iter = 1): eight in-place colour passes equal the oracle's
    colour sweep voxel for voxel.  The library divides by the diagonal stored
    as a float32 1/D (in FP64 handles too), so each correction carries a
    relative error up to 2^-24 and later colours see it through their
    neighbours: the bound is 5e-7 of the largest |v_e| (a colour visited out of
    order, or a stale neighbour, moves the iterate by O(1) of the correction)."""
    c = W.random_case(53, 45, 14, 10, model=W.BI, fill=0.8).fibres_as_float32()
    c.params.solver, c.params.max_iter, c.params.rel_tol = 2, 1, 0.0
    s = ep.sim_from_case(c, precision=ep.EP_FP64)
    o = oracle.Sim(c)
    v, w, ve = W.random_state(53, c)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    stats = s.step(1, allow_noconv=True)
    assert o.step() == 1 and stats.iters == 1 and o.last_iters == 1
    # the projection subtracts each component's mean of the final iterate on both sides
    ref = o.state()["ve"]
    got = s.read(ep.EP_VE)
    np.testing.assert_allclose(got, ref, rtol=0, atol=5e-7 * np.abs(ref).max())
    # the sweep did move the iterate: the bound above is far below the change
    assert np.abs(ref - np.where(c.mask.reshape(-1) > 0, ve, 0.0)).max() > 1e-3 * np.abs(ref).max()


def test_gauss_seidel_fp32_shell_against_oracle_and_deterministic():
    """FP32 GPU against the FP64 oracle over 60 steps of a small shell: V_m within
    0.5 mV and activation times within 1 %; two runs bitwise identical; fewer
    sweeps than the damped Jacobi iteration."""
    n = 24
    sc = n / 128
    c = W.shell_case(n, (40 * sc, 40 * sc, 55 * sc), 3.0, (0.2, 0.05, 0.2, 0.1), 0.05, 60, 4)
    jac = ep.sim_from_case(c)
    jac_iters = 0
    for _ in range(c.steps):
        jac_iters += jac.step(1).iters
    c.params.solver = 2
    runs = []
    gs_iters = 0
    for r in range(2):
        s = ep.sim_from_case(c)
        for _ in range(c.steps):
            st = s.step(1)
            assert st.converged == 1
            if r == 0:
                gs_iters += st.iters
        runs.append((s.read(ep.EP_VM_MV), s.read(ep.EP_VE_MV), s.read(ep.EP_TACT)))
        s.close()
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)
    o = oracle.Sim(c)
    for _ in range(c.steps):
        assert o.step() == 0
    st = o.state()
    vm, _, ta_g = runs[0]
    assert np.abs(vm - oracle.vm_mV(st["v"])).max() <= 0.5
    act = st["tact"] > 0
    assert act.sum() > 20
    np.testing.assert_array_equal(ta_g > 0, act)
    assert np.all(np.abs(ta_g[act] - st["tact"][act]) <= 0.01 * st["tact"][act])
    assert gs_iters < jac_iters, (gs_iters, jac_iters)
    print(f"24^3 shell, 60 steps: Gauss-Seidel {gs_iters} sweeps (x8 colour passes), damped Jacobi {jac_iters}")


def test_gauss_seidel_refused_with_torso_and_in_a_batch():
    c = W.random_case(54, 12, 10, 8, model=W.BI)
    c.params.solver = 2
    s = ep.sim_from_case(c)
    b = ep.Batch(2)
    with pytest.raises(ep.EPError):
        b.add(s)
    b.close()
    s.close()
    t = ep.sim_from_case(c, use_torch=True)
    torso = np.zeros(c.n, np.uint8)
    torso[(c.mask.reshape(-1) == 0)] = 1
    t.set_torso(torso, 1.0)
    with pytest.raises(ep.EPError):
        t.step(1)
    t.close()


def test_gauss_seidel_with_implicit_diffusion_fp64_matches_oracle():
    """The implicit-Euler parabolic step (Eq. iejac1) with the elliptic solve by
    Gauss-Seidel: sweep for sweep equal to the oracle's, in FP64."""
    c = W.random_case(55, 31, 12, 9, model=W.BI, rel_tol=1e-10, check_every=4).fibres_as_float32()
    c.params.solver, c.params.diffusion, c.params.max_iter = 2, 1, 100000
    s = ep.sim_from_case(c, precision=ep.EP_FP64)
    o = oracle.Sim(c)
    v, w, ve = W.random_state(55, c)
    s.set_state(v, w, ve, 0)
    o.set_state(v, w, ve, 0)
    for _ in range(2):
        stats = s.step(1)
        assert o.step() == 0 and stats.converged == 1 and stats.iters == o.last_iters, (stats.iters, o.last_iters)
    st = o.state()
    np.testing.assert_allclose(s.read(ep.EP_V), st["v"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(s.read(ep.EP_VE), st["ve"], rtol=0, atol=1e-7 * max(1.0, np.abs(st["ve"]).max()))
    s.close()
    o.close()
