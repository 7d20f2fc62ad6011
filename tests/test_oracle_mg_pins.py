"""Pins of the multigrid-preconditioned CG study in oracle/mg.py (the
faster-solver future work of the thesis' chapter "Review & Outlook"; no
product path uses it): the probing assembly against the independent sparse
assembly, the Galerkin coarse operators (symmetric, constants in their null
space), the symmetry of the V-cycle preconditioner, and the solve against a
dense least-squares solution."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import mg
from test_oracle_pins import _assemble_independent

SL, ST = 0.4, 0.15


def _case(seed, shape=(16, 14, 12), fill=0.7):
    c = W.random_case(seed, *shape, fill=fill)
    return c, oracle.Grid.from_case(c)


@pytest.mark.parametrize("seed", [61, 62])
def test_probing_assembly_equals_independent_assembly(seed):
    c, g = _case(seed, (9, 8, 7))
    A, dom = mg.assemble(g, SL, ST)
    B = _assemble_independent(c, SL, ST)
    np.testing.assert_array_equal(dom, np.nonzero(c.mask.reshape(-1))[0])
    np.testing.assert_allclose(A.toarray(), B, rtol=0, atol=1e-13 * np.abs(B).max())


def test_galerkin_levels_are_symmetric_with_constants_in_the_null_space():
    c, g = _case(63, (20, 18, 17))
    levels = mg.hierarchy(g, SL, ST)
    assert len(levels) >= 2
    for lv in levels:
        A = lv.A.toarray()
        scale = np.abs(A).max()
        np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-13 * scale)
        assert np.abs(A @ np.ones(A.shape[0])).max() <= 1e-12 * scale
        assert lv.omega > 0.0 and np.all(lv.diag >= 0.0)
    for fine, coarse in zip(levels[:-1], levels[1:]):
        P = fine.P.toarray()
        # every fine voxel has exactly one parent, and the Galerkin product is exact
        assert np.array_equal(P.sum(axis=1), np.ones(P.shape[0]))
        np.testing.assert_allclose(coarse.A.toarray(), P.T @ fine.A.toarray() @ P, rtol=0,
                                   atol=1e-12 * np.abs(fine.A.toarray()).max())


def test_vcycle_is_a_symmetric_operator():
    """Pre- and post-smoothing are the same Jacobi sweeps, so M is symmetric:
    r1 . M(r2) = r2 . M(r1)."""
    c, g = _case(64, (20, 18, 17))
    levels = mg.hierarchy(g, SL, ST)
    m = levels[0].A.shape[0]
    rng = np.random.default_rng(64)
    r1, r2 = rng.standard_normal(m), rng.standard_normal(m)
    a, b = r1 @ mg.vcycle(levels, r2), r2 @ mg.vcycle(levels, r1)
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))


def test_pcg_solves_to_the_dense_solution():
    c, g = _case(65, (16, 14, 12), fill=0.55)
    A, dom = mg.assemble(g, SL, ST)
    rng = np.random.default_rng(65)
    bt = A @ rng.standard_normal(len(dom))
    b = np.zeros(g.n)
    b[dom] = bt
    x, iters, rel, ok, levels = mg.solve(g, SL, ST, b, np.zeros(g.n), 1e-11, 500)
    assert ok and rel <= 1e-11 and iters > 0
    xd = np.linalg.lstsq(A.toarray(), bt, rcond=None)[0]
    labels = mg.component_labels(g, dom)
    xs = x[dom]
    for cc in np.unique(labels):
        sel = labels == cc
        xd[sel] -= xd[sel].mean()
        xs[sel] -= xs[sel].mean()
    np.testing.assert_allclose(xs, xd, rtol=0, atol=1e-8 * max(1.0, np.abs(xd).max()))
    # the preconditioner pays: fewer iterations than the damped Jacobi sweeps to the same tolerance
    _, it6, _, ok6, _ = mg.solve(g, SL, ST, b, np.zeros(g.n), 1e-6, 500, levels=levels)
    _, it_j, _, st_j = g.jacobi(SL, ST, b, np.zeros(g.n), tol=1e-6, m=1, max_iter=400000)
    assert ok6 and st_j == 0 and it6 < it_j
