"""Pins of the oracle's implicit-Euler diffusion (Sec. "Implicit Euler",
Eq. iejac1; Sec. "Diffusion"): the Jacobi step and its fixed point are checked
against an independent dense assembly of the operator, against conservation
of charge, and against the explicit step it must approach as dt -> 0."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_pins import _assemble_independent


def _quiet(case):
    """Reaction switched off: huge time constants, no stimulus."""
    case.stimuli = []
    p = case.params
    p.tau_in = p.tau_out = 1e300
    p.tau_open = p.tau_close = 1e300
    return case


@pytest.mark.parametrize("seed", [11, 12])
def test_ie_jacobi_step_and_solution_match_dense_algebra(seed):
    """With B = G'^T S G' assembled independently (scipy) and D = diag(B):
    one sweep from x0 is x1 = (I + aD)^-1 (f - a (B - D) x0) (Eq. iejac1 with
    A = -B), and the converged iterate solves (I + a B) x = f."""
    c = W.random_case(seed, 5, 4, 4, fill=0.7)
    g = oracle.Grid.from_case(c)
    sL, sT, a = 0.4, 0.15, 0.7
    B = _assemble_independent(c, sL, sT)
    t = np.nonzero(g.mask)[0]
    rng = np.random.default_rng(seed)
    f = np.zeros(g.n)
    f[t] = rng.standard_normal(len(t))
    x0 = np.zeros(g.n)
    x0[t] = rng.standard_normal(len(t))
    D = np.diag(B)
    x1_expect = (f[t] - a * (B @ x0[t] - D * x0[t])) / (1.0 + a * D)
    x1, it, _, _ = g.ie_jacobi(sL, sT, a, f, x0, tol=0.0, m=1, max_iter=1)
    assert it == 1
    np.testing.assert_allclose(x1[t], x1_expect, rtol=1e-13, atol=1e-13)
    x, it, rr, st = g.ie_jacobi(sL, sT, a, f, f, tol=1e-13, m=1, max_iter=100000)
    assert st == 0 and rr <= 1e-13 and it > 1
    xd = np.linalg.solve(np.eye(len(t)) + a * B, f[t])
    np.testing.assert_allclose(x[t], xd, rtol=0, atol=1e-11 * np.abs(xd).max())
    assert np.all(x[g.mask == 0] == 0.0)


def test_ie_jacobi_stop_rule_and_cap():
    """Checks every m sweeps: the reported residual is the last checked one,
    it is below the tolerance, and the sweep count is one past a check; a cap
    below convergence returns status 1 after exactly max_iter sweeps."""
    c = W.random_case(13, 9, 8, 7)
    g = oracle.Grid.from_case(c)
    rng = np.random.default_rng(13)
    f = rng.standard_normal(g.n) * (g.mask > 0)
    x, it, rr, st = g.ie_jacobi(0.2, 0.05, 2.0, f, f, tol=1e-9, m=4)
    assert st == 0 and rr <= 1e-9 and it % 4 == 1
    _, it2, _, st2 = g.ie_jacobi(0.2, 0.05, 2.0, f, f, tol=1e-9, m=4, max_iter=it - 1)
    assert st2 == 1 and it2 == it - 1


@pytest.mark.parametrize("model", [W.MONO, W.BI])
def test_ie_step_conserves_charge(model):
    """1^T (I + a L) = 1^T because L 1 = 0 with no-flux boundaries, so the
    implicit step keeps sum_T v to the solver tolerance (monodomain: exactly
    sum_T v*; bidomain: sum_T v* minus a 1^T L ve = sum_T v*)."""
    c = _quiet(W.random_case(14, 10, 8, 7, model=model, rel_tol=1e-13, check_every=1))
    c.params.diffusion = 1
    s = oracle.Sim(c)
    v, w, ve = W.random_state(14, c)
    s.set_state(v, w, ve)
    assert s.step() == 0
    v1 = s.state()["v"]
    assert not np.array_equal(v1, v)
    assert abs(v1.sum() - v.sum()) <= 1e-11 * np.abs(v).sum()
    assert s.ie_total_iters > 0


def test_ie_approaches_explicit_step_second_order_per_step():
    """Both schemes agree to first order: one step differs by a^2 L^2 v* + ...,
    so halving dt quarters the difference."""
    diffs = []
    for dt in (0.02, 0.01):
        out = []
        for scheme in (0, 1):
            c = _quiet(W.random_case(15, 10, 9, 8, model=W.MONO, dt=dt, rel_tol=1e-14, check_every=1))
            c.params.diffusion = scheme
            s = oracle.Sim(c)
            v, w, _ = W.random_state(15, c)
            s.set_state(v, w, None)
            s.step()
            out.append(s.state()["v"])
        diffs.append(np.abs(out[0] - out[1]).max())
    ratio = diffs[0] / diffs[1]
    assert diffs[1] > 0 and 3.6 < ratio < 4.4, diffs


def test_ie_rest_state_is_a_fixed_point_bitwise():
    for model in (W.MONO, W.BI):
        c = W.random_case(16, 9, 7, 6, model=model)
        c.stimuli = []
        c.params.diffusion = 1
        s = oracle.Sim(c)
        s.run(5)
        st = s.state()
        assert np.all(st["v"] == 0.0) and np.all(st["w"] == 1.0) and np.all(st["ve"] == 0.0)
        assert s.ie_total_iters == 0
