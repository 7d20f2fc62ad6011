"""Pins of the oracle's torso (Eq. bidomain1, lines 3-5: the extracellular
potential continues into a passive conductor around the heart) and of the
ECG lead formulas (Sec. "Electrocardiogram").

The torso operator is checked against an independent dense assembly of its
two terms, against the plain operator it reduces to without tissue, against
the domination of the intracellular operator that keeps the explicit split
stable, and against the layered closed form (an insulated torso layer takes
the potential of the tissue surface it touches); the step against charge
conservation, the rest state and boundedness."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_pins import _assemble_independent


def _dense_domain(g, sL, sT):
    t = np.nonzero(g.domain())[0]
    A = np.zeros((len(t), len(t)))
    for col, q in enumerate(t):
        e = np.zeros(g.n)
        e[q] = 1.0
        A[:, col] = g.apply_L(sL, sT, e)[t]
    return A, t


def _dense_domain_part(g, sL, sT, idx):
    A = np.zeros((len(idx), len(idx)))
    for col, q in enumerate(idx):
        e = np.zeros(g.n)
        e[q] = 1.0
        A[:, col] = g.apply_L(sL, sT, e)[idx]
    return A


@pytest.mark.parametrize("seed", [51, 52])
def test_torso_operator_matches_independent_assembly(seed):
    """Applying the oracle to unit vectors on tissue + torso gives the sum of
    the independently assembled tissue term (tissue pairs, fibre tensors) and
    torso term (domain pairs, sig_o I per torso voxel); the matrix is
    symmetric PSD with zero row sums, and its diagonal is the oracle's Jacobi
    diagonal."""
    c = W.with_torso(W.random_case(seed, 5, 4, 4, fill=0.5), sig_o=0.7, fill=0.8, seed=seed)
    g = oracle.Grid.elliptic_from_case(c)
    sL, sT = 0.4, 0.15
    A, t = _dense_domain(g, sL, sT)
    assert len(t) > c.n_tissue   # the torso joined the domain
    B = _assemble_independent(c, sL, sT, torso=c.torso, sig_o=0.7, part="tissue") + \
        _assemble_independent(c, sL, sT, torso=c.torso, sig_o=0.7, part="torso")
    np.testing.assert_allclose(A, B, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(A.sum(axis=1), 0.0, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > -1e-12
    np.testing.assert_allclose(g.diag_L(sL, sT)[t], np.diag(A), rtol=1e-13, atol=1e-13)


def test_torso_without_tissue_is_the_plain_isotropic_operator():
    """With no tissue voxel the torso term alone remains: the plain operator
    of the torso voxels with sigma_L = sigma_T = sig_o and zero fibres, bit for
    bit (the same sums in the same order)."""
    base = W.random_case(53, 9, 8, 7, fill=0.5)
    c = W.with_torso(base, sig_o=0.35, fill=0.7, seed=53)
    empty = np.zeros(c.n, np.uint8)
    g = oracle.Grid(c.nx, c.ny, c.nz, c.dx, empty, np.zeros(3 * c.n), c.torso, 0.35)
    plain = oracle.Grid(c.nx, c.ny, c.nz, c.dx, c.torso, np.zeros(3 * c.n))
    rng = np.random.default_rng(53)
    u = rng.standard_normal(c.n)
    np.testing.assert_array_equal(g.apply_L(0.4, 0.15, u), plain.apply_L(0.35, 0.35, u))
    np.testing.assert_array_equal(g.diag_L(0.4, 0.15), plain.diag_L(0.35, 0.35))
    nc, comp = g.components()
    nc2, comp2 = plain.components()
    assert nc == nc2 and np.array_equal(comp, comp2)


@pytest.mark.parametrize("seed", [54, 55])
def test_torso_operator_dominates_the_intracellular_one(seed):
    """A - L_i >= 0 on tissue + torso (L_i extended by zero), hence the
    operator of the explicit split, L_i - L_i A^+ L_i, is PSD and bounded by
    L_i: the bidomain step with a torso is as stable as the plain one."""
    c = W.with_torso(W.random_case(seed, 7, 6, 6, fill=0.5), sig_o=1.0, fill=0.9, seed=seed)
    p = c.params
    ge, gh = oracle.Grid.elliptic_from_case(c), oracle.Grid.from_case(c)
    idx = np.nonzero(ge.domain())[0]
    A = _dense_domain_part(ge, p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT, idx)
    Li = _dense_domain_part(gh, p.sig_iL, p.sig_iT, idx)
    assert np.linalg.eigvalsh(A - Li).min() > -1e-12
    M = Li - Li @ np.linalg.pinv(A, rcond=1e-12) @ Li
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev.min() > -1e-9 and ev.max() <= np.linalg.eigvalsh(Li).max() * (1 + 1e-9)


def _layered(sig_o):
    """Tissue slab i < 6 of a 10 x 3 x 3 box, fibres along x, torso i >= 6."""
    nx, ny, nz = 10, 3, 3
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, :, :6] = 1
    fib = np.zeros((nz, ny, nx, 3), np.float32)
    fib[..., 0] = mask
    p = W.Params(sig_iL=0.2, sig_iT=0.05, sig_eL=0.2, sig_eT=0.1, sig_o=sig_o)
    c = W.Case("layered", nx, ny, nz, 0.5, mask, fib, p, [])
    return W.with_torso(c, sig_o=sig_o)


@pytest.mark.parametrize("sig_o", [0.3, 2.0])
def test_layered_torso_closed_form(sig_o):
    """A potential varying along x only makes the problem one-dimensional.
    The torso layer then carries no current (its far face is insulated), so
    every torso voxel takes the potential of the tissue voxel at the surface,
    and the tissue potential is the torso-free one up to a constant."""
    c = _layered(sig_o)
    p = c.params
    sL, sT = p.sig_iL + p.sig_eL, p.sig_iT + p.sig_eT
    ge = oracle.Grid.elliptic_from_case(c)
    gh = oracle.Grid.from_case(c)
    v = np.zeros((c.nz, c.ny, c.nx))
    v[:, :, :6] = np.array([0.9, 0.7, 0.2, 0.05, 0.6, 0.3])
    b = -gh.apply_L(p.sig_iL, p.sig_iT, v.reshape(-1))
    b[c.mask.reshape(-1) == 0] = 0.0
    xe, _, _, st = ge.jacobi(sL, sT, b, np.zeros(c.n), tol=1e-13, m=1, max_iter=400000)
    xh, _, _, st2 = gh.jacobi(sL, sT, b, np.zeros(c.n), tol=1e-13, m=1, max_iter=400000)
    assert st == 0 and st2 == 0
    xe, xh = xe.reshape(c.nz, c.ny, c.nx), xh.reshape(c.nz, c.ny, c.nx)
    surface = xe[:, :, 5]
    np.testing.assert_allclose(xe[:, :, 6:], surface.mean(), rtol=0, atol=1e-9)
    np.testing.assert_allclose(xe[:, :, :6] - xe[0, 0, 0], xh[:, :, :6] - xh[0, 0, 0], rtol=0, atol=1e-9)


def test_torso_step_conserves_charge_and_keeps_rest():
    """The membrane state stays on the tissue (torso v, w untouched), the
    elliptic right-hand side sums to zero over the domain, and the rest state
    is a fixed point bit for bit."""
    c = W.with_torso(W.random_case(54, 9, 8, 7, fill=0.5, rel_tol=1e-12, check_every=1), sig_o=0.8,
                     fill=0.9, seed=54)
    c.stimuli = []
    s = oracle.Sim(c)
    s.run(3)
    st = s.state()
    assert np.all(st["v"] == 0.0) and np.all(st["w"] == 1.0) and np.all(st["ve"] == 0.0)
    c2 = W.with_torso(W.random_case(55, 9, 8, 7, fill=0.5, rel_tol=1e-12, check_every=1), sig_o=0.8,
                      fill=0.9, seed=55)
    s2 = oracle.Sim(c2)
    v, w, ve = W.random_state(55, c2)
    s2.set_state(v, w, ve)
    assert s2.step() == 0
    st2 = s2.state()
    off = c2.mask.reshape(-1) == 0
    assert np.all(st2["v"][off] == 0.0) and np.all(st2["w"][off] == 1.0)
    dom = oracle.Grid.elliptic_from_case(c2).domain()
    assert np.any(st2["ve"][dom & off] != 0.0)           # the potential reaches the torso
    nc, comp = oracle.Grid.elliptic_from_case(c2).components()
    for cc in range(nc):                                 # zero mean per domain component
        assert abs(st2["ve"][comp == cc].sum()) <= 1e-12 * max(1.0, np.abs(st2["ve"]).sum())


def test_ecg_lead_formulas():
    """The six limb leads of electrode potentials (RA, LA, LL) = (1, 2, 4) mV by
    hand, and the identities every lead set obeys: Einthoven's I + III = II and
    aVR + aVL + aVF = 0."""
    np.testing.assert_allclose(oracle.ecg_leads([1.0, 2.0, 4.0]), [1.0, 3.0, 2.0, -2.0, -0.5, 2.5], atol=0)
    rng = np.random.default_rng(56)
    L = oracle.ecg_leads(rng.standard_normal((50, 3)))
    np.testing.assert_allclose(L[:, 0] + L[:, 2], L[:, 1], atol=1e-14)
    np.testing.assert_allclose(L[:, 3] + L[:, 4] + L[:, 5], 0.0, atol=1e-14)
