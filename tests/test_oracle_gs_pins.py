"""Pins of the oracle's eight-colour Gauss-Seidel / SOR solve (the
deterministic form of the thesis' in-place Jacobi, Sec. "Jacobi method").
One sweep is checked against the matrix-splitting form of SOR, solved by a
triangular solve on an independently assembled matrix in colour order; the
residual the stop rule sums against the update it produced; the converged
solve against a dense least-squares solution."""
import numpy as np
import pytest
from scipy.linalg import solve_triangular

import oracle
import workloads as W
from test_oracle_pins import _assemble_independent

SL, ST = 0.4, 0.15


def _colour(g, t):
    i, j, k = t % g.nx, (t // g.nx) % g.ny, t // (g.nx * g.ny)
    return (i & 1) + 2 * (j & 1) + 4 * (k & 1)


def _system(seed, shape=(7, 6, 5), fill=0.8):
    c = W.random_case(seed, *shape, fill=fill)
    g = oracle.Grid.from_case(c)
    A = _assemble_independent(c, SL, ST)
    t = np.nonzero(g.mask)[0]
    return c, g, A, t


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_same_colour_voxels_are_uncoupled(seed):
    """The 27-point operator couples no two distinct voxels of one colour, so a
    colour's updates are independent of their order."""
    c, g, A, t = _system(seed)
    col = _colour(g, t)
    same = col[:, None] == col[None, :]
    off = same & ~np.eye(len(t), dtype=bool)
    assert np.abs(A[off]).max() == 0.0
    # and two colours do not suffice: diagonal neighbours have equal i + j + k parity
    par = (t % g.nx + (t // g.nx) % g.ny + t // (g.nx * g.ny)) & 1
    two = (par[:, None] == par[None, :]) & ~np.eye(len(t), dtype=bool)
    assert np.abs(A[two]).max() > 0.0


@pytest.mark.parametrize("seed,omega", [(4, 1.0), (5, 1.0), (6, 1.5), (7, 0.7)])
def test_one_sweep_is_the_sor_splitting(seed, omega):
    """One sweep equals (D + omega L) x1 = omega b - (omega U + (omega - 1) D) x0
    with L, U the strict lower and upper parts of A in colour order (index
    order within a colour); the summed residual of the sweep equals the sum
    of (D (x1 - x0) / omega)^2."""
    c, g, A, t = _system(seed)
    d = np.diag(A)
    live = d > 0     # rows of isolated voxels are empty and stay as they are
    rng = np.random.default_rng(seed)
    b = np.zeros(g.n)
    b[t] = rng.standard_normal(len(t))
    x0 = np.zeros(g.n)
    x0[t] = rng.standard_normal(len(t))
    x1, iters, rr, st = g.gauss_seidel(SL, ST, b, x0, omega=omega, tol=0.0, m=1, max_iter=1)
    assert iters == 1 and st == 1
    perm = np.lexsort((t, _colour(g, t)))          # colour order, index order inside
    perm = perm[live[perm]]
    Ap = A[np.ix_(perm, perm)]
    Dp = np.diag(np.diag(Ap))
    Lp, Up = np.tril(Ap, -1), np.triu(Ap, 1)
    # isolated voxels (no row) keep their value and do not enter live rows
    xin = x0[t][perm]
    rhs = omega * b[t][perm] - (omega * Up + (omega - 1.0) * Dp) @ xin
    xs = solve_triangular(Dp + omega * Lp, rhs, lower=True)
    scale = max(1.0, np.abs(xs).max())
    np.testing.assert_allclose(x1[t][perm], xs, rtol=0, atol=1e-12 * scale)
    assert np.array_equal(x1[t][~live], x0[t][~live])
    # the stop rule's residual: r_q at its colour's update = D_q (x1 - x0)_q / omega
    r = np.diag(Ap) * (xs - xin) / omega
    r_iso = b[t][~live]     # isolated voxels: r = b (their row of A is 0), no update
    want = np.sqrt(np.sum(r ** 2) + np.sum(r_iso ** 2)) / np.linalg.norm(b[t])
    assert abs(rr - want) <= 1e-12 * want


@pytest.mark.parametrize("seed", [8, 9])
def test_converges_to_the_dense_solution(seed):
    """A compatible right-hand side (two components at fill 0.45), solved to
    1e-11: equal to the least-squares solution, both projected to zero mean
    per face-connected component; Gauss-Seidel needs fewer sweeps than the
    damped Jacobi iteration, and SOR at omega = 1.5 fewer still."""
    c, g, A, t = _system(seed, shape=(8, 7, 6), fill=0.55)
    rng = np.random.default_rng(seed)
    bt = A @ rng.standard_normal(len(t))
    b = np.zeros(g.n)
    b[t] = bt
    x, it_gs, rr, st = g.gauss_seidel(SL, ST, b, np.zeros(g.n), omega=1.0, tol=1e-11, m=1, max_iter=200000)
    assert st == 0 and rr <= 1e-11
    nc, comp = g.components()
    xd = np.linalg.lstsq(A, bt, rcond=None)[0]
    ct = comp[t]
    xg = x[t].copy()
    for cc in range(nc):
        sel = ct == cc
        xd[sel] -= xd[sel].mean()
        xg[sel] -= xg[sel].mean()
    np.testing.assert_allclose(xg, xd, rtol=0, atol=1e-8 * max(1.0, np.abs(xd).max()))
    _, it_j, _, st_j = g.jacobi(SL, ST, b, np.zeros(g.n), tol=1e-11, m=1, max_iter=400000)
    _, it_sor, _, st_s = g.gauss_seidel(SL, ST, b, np.zeros(g.n), omega=1.5, tol=1e-11, m=1, max_iter=200000)
    assert st_j == 0 and st_s == 0
    assert it_gs < it_j and it_sor < it_gs, (it_j, it_gs, it_sor)


def test_zero_rhs_and_default_omega():
    """||b|| = 0 returns after 0 sweeps with x unchanged; omega <= 0 is
    Gauss-Seidel (omega = 1)."""
    c, g, A, t = _system(10)
    x0 = np.zeros(g.n)
    x0[t] = 1.0
    x, it, rr, st = g.gauss_seidel(SL, ST, np.zeros(g.n), x0, omega=1.0)
    assert st == 0 and it == 0 and np.array_equal(x, x0)
    rng = np.random.default_rng(10)
    b = np.zeros(g.n)
    b[t] = rng.standard_normal(len(t))
    xa, *_ = g.gauss_seidel(SL, ST, b, x0, omega=0.0, tol=0.0, m=1, max_iter=3)
    xb, *_ = g.gauss_seidel(SL, ST, b, x0, omega=1.0, tol=0.0, m=1, max_iter=3)
    assert np.array_equal(xa, xb)


def test_step_with_gauss_seidel_matches_jacobi_step():
    """The bidomain step with the elliptic solve by Gauss-Seidel and by damped
    Jacobi, both to 1e-9: the same v_e to the tolerance, the same v."""
    n = 12
    sc = n / 128.0
    c = W.shell_case(n, (40 * sc, 40 * sc, 55 * sc), 2.5, (0.2, 0.05, 0.2, 0.1), 0.05, 3, 4)
    c.params.rel_tol = 1e-9
    c.params.max_iter = 400000
    outs = []
    for solver in (0, 2):
        c.params.solver = solver
        o = oracle.Sim(c)
        for _ in range(2):
            assert o.step() == 0
        outs.append(o.state())
        o.close()
    scale = max(1e-12, np.abs(outs[0]["ve"]).max())
    assert np.abs(outs[0]["ve"] - outs[1]["ve"]).max() <= 1e-6 * scale
    assert np.abs(outs[0]["v"] - outs[1]["v"]).max() <= 1e-8
