"""Pins of the oracle's Chebyshev-accelerated Jacobi solve (Golub and
Varga's semi-iterative method; the thesis lists faster solvers as future
work).  The recurrence is checked against the closed-form residual
polynomial on an independent eigendecomposition of D^-1 A, and the solve
against a dense solution."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_pins import _assemble_independent


def _cheb_poly(k, lam, lmin, lmax):
    """p_k(lam) = T_k((lmax + lmin - 2 lam) / (lmax - lmin)) / T_k((lmax + lmin) / (lmax - lmin))."""
    c = np.zeros(k + 1)
    c[k] = 1.0
    num = np.polynomial.chebyshev.chebval((lmax + lmin - 2.0 * lam) / (lmax - lmin), c)
    den = np.polynomial.chebyshev.chebval((lmax + lmin) / (lmax - lmin), c)
    return num / den


def _system(seed):
    c = W.random_case(seed, 5, 4, 4, fill=0.75)
    g = oracle.Grid.from_case(c)
    sL, sT = 0.4, 0.15
    B = _assemble_independent(c, sL, sT)
    t = np.nonzero(g.mask)[0]
    d = np.diag(B)
    ok = d > 0
    assert ok.all()
    Dh = np.sqrt(d)
    Msym = B / Dh[:, None] / Dh[None, :]          # D^-1/2 B D^-1/2: the spectrum of D^-1 B
    lam, V = np.linalg.eigh(Msym)
    return c, g, sL, sT, B, t, Dh, lam, V


@pytest.mark.parametrize("seed", [32, 35])   # masks without isolated voxels
def test_chebyshev_error_follows_the_residual_polynomial(seed):
    """After k steps from x0 the error is p_k(D^-1 A) e0 on every eigenvector
    whose eigenvalue lies in [lmin, lmax], and unchanged on the null space."""
    c, g, sL, sT, B, t, Dh, lam, V = _system(seed)
    nz = lam > 1e-10
    lmin, lmax = lam[nz].min(), lam.max()
    rng = np.random.default_rng(seed)
    xs = rng.standard_normal(len(t))
    b = np.zeros(g.n)
    b[t] = B @ xs
    x0 = np.zeros(g.n)
    x0[t] = rng.standard_normal(len(t))
    e0 = Dh * (xs - x0[t])                          # error in the symmetric coordinates
    c0 = V.T @ e0
    for k in (1, 2, 3, 7, 15):
        xk, it, _, _ = g.chebyshev(sL, sT, b, x0, lmin, lmax, tol=0.0, m=10 ** 6, max_iter=k)
        assert it == k
        ck = V.T @ (Dh * (xs - xk[t]))
        expect = c0 * np.where(nz, _cheb_poly(k, lam, lmin, lmax), 1.0)
        np.testing.assert_allclose(ck, expect, rtol=0, atol=1e-10 * np.abs(c0).max())


def test_chebyshev_solves_to_the_dense_solution():
    c, g, sL, sT, B, t, Dh, lam, V = _system(33)
    nz = lam > 1e-10
    rng = np.random.default_rng(33)
    b = np.zeros(g.n)
    b[t] = B @ rng.standard_normal(len(t))
    x, it, rr, st = g.chebyshev(sL, sT, b, np.zeros(g.n), lam[nz].min(), lam.max(), tol=1e-12, m=1)
    assert st == 0 and rr <= 1e-12
    xd = np.linalg.lstsq(B, b[t], rcond=None)[0]
    nc, comp = g.components()
    ct = comp[t]
    for cc in range(nc):
        sel = ct == cc
        xd[sel] -= xd[sel].mean()
        x[t[sel]] -= x[t[sel]].mean()
    np.testing.assert_allclose(x[t], xd, rtol=0, atol=1e-9 * max(1.0, np.abs(xd).max()))


def test_chebyshev_needs_far_fewer_sweeps_than_damped_jacobi():
    """On an elongated slab (slow modes dominate) the semi-iteration reaches
    the tolerance in a fraction of the damped-Jacobi sweeps."""
    c = W.random_case(34, 48, 6, 6, fill=1.0)
    g = oracle.Grid.from_case(c)
    sL, sT = 0.4, 0.15
    rng = np.random.default_rng(34)
    t = g.mask > 0
    u = rng.standard_normal(g.n) * t
    b = g.apply_L(sL, sT, u)
    omega = oracle.lib().og_default_omega(sL, sT)
    _, it_j, _, st_j = g.jacobi(sL, sT, b, np.zeros(g.n), omega=omega, tol=1e-8, m=1, max_iter=400000)
    # the interval: the Fourier bound above (the one the damping uses), an underestimate below
    lmax = 1.8 / omega
    _, it_c, _, st_c = g.chebyshev(sL, sT, b, np.zeros(g.n), 1e-4, lmax, tol=1e-8, m=1, max_iter=400000)
    assert st_j == 0 and st_c == 0
    assert it_c * 4 < it_j, (it_c, it_j)
