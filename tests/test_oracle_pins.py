"""Pins for the FP64 CPU oracle: closed forms, invariants, special cases and
brute force on tiny grids.  None of these compares the oracle with itself or
with the CUDA path.  Each test names the passage of the thesis it pins."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _full_box(nx, ny, nz, dx, f=(1.0, 0.0, 0.0)):
    mask = np.ones((nz, ny, nx), np.uint8)
    fib = np.zeros((nz, ny, nx, 3))
    fib[...] = np.asarray(f, float) / max(np.linalg.norm(f), 1e-300)
    return oracle.Grid(nx, ny, nz, dx, mask, fib)


def _coords(nx, ny, nz, dx):
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * dx, (np.arange(ny) + 0.5) * dx,
                          (np.arange(nx) + 0.5) * dx, indexing="ij")
    return x, y, z


# ---------------------------------------------------------------------------
# operator: Sec. Operators (Eqs. refgrad2, refdiv3, Laplacian), Eq. sigma1
# ---------------------------------------------------------------------------

def test_quadratic_exact_in_interior_full_tensor():
    """For constant Sigma and quadratic u = x^T H x / 2 + c^T x the dual-grid
    gradient (Eq. refgrad2) and face divergence (Eq. refdiv3) are exact, so
    L u = -tr(Sigma H) at every interior voxel.  Catches a transposed tensor,
    a dropped off-diagonal term, a wrong sign or scale."""
    n, dx = 9, 0.3
    f = np.array([0.6, 0.48, 0.64])
    f /= np.linalg.norm(f)
    g = _full_box(n, n, n, dx, f)
    x, y, z = _coords(n, n, n, dx)
    H = np.array([[1.0, 0.3, -0.2], [0.3, -0.5, 0.7], [-0.2, 0.7, 2.0]])
    X = np.stack([x, y, z], -1)
    u = 0.5 * np.einsum("...i,ij,...j->...", X, H, X) + X @ np.array([0.1, -0.2, 0.3])
    sL, sT = 0.2, 0.05
    Sig = sT * np.eye(3) + (sL - sT) * np.outer(f, f)
    Lu = g.apply_L(sL, sT, u).reshape(n, n, n)
    np.testing.assert_allclose(Lu[1:-1, 1:-1, 1:-1], -np.trace(Sig @ H), rtol=0, atol=1e-11)


def test_manufactured_cosine_second_order():
    """u = cos(pi x/Lx) cos(pi y/Ly) cos(pi z/Lz) meets the no-flux condition
    on a full box with diagonal Sigma; L u -> -div(Sigma grad u) at O(dx^2) in
    the max norm over all voxels (the quadratic convergence reported in the
    operator convergence study of the experiments chapter)."""
    Lx, Ly, Lz = 2.0, 1.5, 1.0
    sL, sT = 0.2, 0.05
    errs = []
    for n in (16, 32):
        nx, ny, nz = n, int(n * Ly / Lx), int(n * Lz / Lx)
        dx = Lx / nx
        g = _full_box(nx, ny, nz, dx)
        x, y, z = _coords(nx, ny, nz, dx)
        u = np.cos(np.pi * x / Lx) * np.cos(np.pi * y / Ly) * np.cos(np.pi * z / Lz)
        ex = np.pi ** 2 * (sL / Lx ** 2 + sT / Ly ** 2 + sT / Lz ** 2) * u
        errs.append(np.abs(g.apply_L(sL, sT, u).reshape(nz, ny, nx) - ex).max())
    rate = math.log2(errs[0] / errs[1])
    assert 1.85 < rate < 2.15, (errs, rate)
    assert errs[1] < 0.015


def test_tangential_exact_on_flat_no_flux_faces():
    """Reading of the no-flux rule at the mask: a slab bounded in y and z with
    fibres along x and u = x^2 has L u = -2 sigma_L on every voxel away from the
    x ends, including the boundary layers (the face flux is not over-weighted
    next to the mask)."""
    nx, ny, nz, dx = 12, 5, 4, 0.25
    g = _full_box(nx, ny, nz, dx, (1.0, 0.0, 0.0))
    x, _, _ = _coords(nx, ny, nz, dx)
    Lu = g.apply_L(0.2, 0.05, x ** 2).reshape(nz, ny, nx)
    np.testing.assert_allclose(Lu[:, :, 1:-1], -2 * 0.2, rtol=0, atol=1e-12)


def test_plane_wave_reduces_to_1d_three_point():
    """On a one-voxel-thick cable the stencil is exactly sigma/dx^2 times the
    1-D three-point Laplacian (with no-flux ends)."""
    nx, dx = 20, 0.1
    g = _full_box(nx, 1, 1, dx, (1.0, 0.0, 0.0))
    rng = np.random.default_rng(0)
    u = rng.standard_normal(nx)
    Lu = g.apply_L(0.2, 0.05, u)
    ref = np.zeros(nx)
    ref[1:] += (u[1:] - u[:-1])
    ref[:-1] -= (u[1:] - u[:-1])
    np.testing.assert_allclose(Lu, 0.2 / dx ** 2 * ref, rtol=1e-12, atol=1e-12)


def test_one_voxel_sheet_is_2d_operator():
    """A one-voxel-thick sheet (nz = 1) with in-plane fibres: u = x y gives
    L u = -2 Sigma_xy exactly in the sheet interior (no z coupling)."""
    n, dx = 8, 0.2
    f = np.array([0.8, 0.6, 0.0])
    g = _full_box(n, n, 1, dx, f)
    x, y, _ = _coords(n, n, 1, dx)
    sL, sT = 0.2, 0.05
    Lu = g.apply_L(sL, sT, x * y).reshape(1, n, n)
    Sxy = (sL - sT) * f[0] * f[1]
    np.testing.assert_allclose(Lu[0, 1:-1, 1:-1], -2 * Sxy, rtol=0, atol=1e-12)


def _random_grid(seed, nx=8, ny=7, nz=6, fill=0.6):
    c = W.random_case(seed, nx, ny, nz, fill=fill)
    return c, oracle.Grid.from_case(c)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_symmetry_psd_conservation(seed):
    """L = G'^T S G' is symmetric positive semi-definite and L 1 = 0 on every
    component: charge is conserved under the no-flux condition (Eq. bidomain1,
    last line)."""
    c, g = _random_grid(seed)
    rng = np.random.default_rng(seed)
    t = c.mask.reshape(-1) > 0
    for sL, sT in ((0.2, 0.05), (0.4, 0.15)):
        u = rng.standard_normal(g.n) * t
        w = rng.standard_normal(g.n) * t
        Lu, Lw = g.apply_L(sL, sT, u), g.apply_L(sL, sT, w)
        scale = np.abs(u).sum() * np.abs(Lw).max()
        assert abs(u @ Lw - Lu @ w) <= 1e-13 * scale
        assert u @ Lu >= -1e-13 * scale
        assert abs(Lu.sum()) <= 1e-13 * np.abs(Lu).sum()
        assert np.all(Lu[~t] == 0.0)
        assert np.abs(g.apply_L(sL, sT, t.astype(float))).max() < 1e-13


def _dense(g, sL, sT):
    t = np.nonzero(g.mask)[0]
    A = np.zeros((len(t), len(t)))
    for col, q in enumerate(t):
        e = np.zeros(g.n)
        e[q] = 1.0
        A[:, col] = g.apply_L(sL, sT, e)[t]
    return A, t


def _assemble_independent(c, sL, sT, torso=None, sig_o=0.0, part="tissue"):
    """Independent sparse assembly of G'^T S G' (scipy), enumerating vertex
    blocks and their valid voxel pairs directly.  With a torso the matrix
    spans tissue + torso voxels, and part selects the term: "tissue" (pairs
    of tissue voxels, tensor from the tissue voxels of the block) or "torso"
    (pairs of any two domain voxels, tensor sig_o I per torso voxel of the
    block)."""
    import scipy.sparse as sp
    nx, ny, nz, dx = c.nx, c.ny, c.nz, c.dx
    heart = c.mask.astype(bool)
    m = heart if torso is None else heart | (np.asarray(torso).reshape(heart.shape) > 0)
    member = heart if part == "tissue" else m
    f = c.fib.astype(np.float64)
    t_idx = -np.ones(m.shape, int)
    t_idx[m] = np.arange(m.sum())
    rows, cols, vals, blocks = [], [], [], []
    r = 0
    for K in range(nz + 1):
        for J in range(ny + 1):
            for I in range(nx + 1):
                blk = [(k, j, i) for k in (K - 1, K) for j in (J - 1, J) for i in (I - 1, I)
                       if 0 <= i < nx and 0 <= j < ny and 0 <= k < nz and member[k, j, i]]
                S = np.zeros((3, 3))
                for (k, j, i) in blk:
                    if part == "tissue":
                        S += sT * np.eye(3) + (sL - sT) * np.outer(f[k, j, i], f[k, j, i])
                    elif not heart[k, j, i]:
                        S += sig_o * np.eye(3)
                S /= 8.0
                for a in range(3):
                    pairs = []
                    for (k, j, i) in blk:
                        hi = [i, j, k]
                        hi[a] += 1
                        hi_in_block = (hi[0] == I and a == 0) or (hi[1] == J and a == 1) or (hi[2] == K and a == 2)
                        if hi_in_block and hi[0] < nx and hi[1] < ny and hi[2] < nz and member[hi[2], hi[1], hi[0]]:
                            pairs.append((t_idx[k, j, i], t_idx[hi[2], hi[1], hi[0]]))
                    for lo_q, hi_q in pairs:
                        rows += [r + a, r + a]
                        cols += [hi_q, lo_q]
                        vals += [1.0 / (len(pairs) * dx), -1.0 / (len(pairs) * dx)]
                blocks.append(S)
                r += 3
    G = sp.csr_matrix((vals, (rows, cols)), shape=(r, int(m.sum())))
    Sb = sp.block_diag([sp.csr_matrix(b) for b in blocks], format="csr")
    return (G.T @ Sb @ G).toarray()


@pytest.mark.parametrize("seed", [5, 6])
def test_brute_force_dense_assembly_and_solve(seed):
    """Tiny grids: the matrix obtained by applying the oracle to unit vectors
    equals an independent sparse assembly of G'^T S G'; its diagonal equals
    the oracle's Jacobi diagonal; the damped Jacobi solve (Eq. dampjac1) agrees
    with a dense least-squares solve projected to zero mean per component."""
    c = W.random_case(seed, 5, 4, 4, fill=0.7)
    g = oracle.Grid.from_case(c)
    sL, sT = 0.4, 0.15
    A, t = _dense(g, sL, sT)
    B = _assemble_independent(c, sL, sT)
    np.testing.assert_allclose(A, B, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g.diag_L(sL, sT)[t], np.diag(A), rtol=1e-13, atol=1e-13)
    # a compatible right-hand side, solved to a tight tolerance
    rng = np.random.default_rng(seed)
    bt = A @ rng.standard_normal(len(t))
    b = np.zeros(g.n)
    b[t] = bt
    x, iters, rr, st = g.jacobi(sL, sT, b, np.zeros(g.n), tol=1e-12, m=1, max_iter=200000)
    assert st == 0 and rr <= 1e-12 and iters > 0
    nc, comp = g.components()
    xd = np.linalg.lstsq(A, bt, rcond=None)[0]
    ct = comp[t]
    for cc in range(nc):
        sel = ct == cc
        xd[sel] -= xd[sel].mean()
        x[t[sel]] -= x[t[sel]].mean()
    np.testing.assert_allclose(x[t], xd, rtol=0, atol=1e-8 * max(1.0, np.abs(xd).max()))


def test_components_match_library_labelling():
    """Face-connected components equal scipy.ndimage.label with the 6-neighbour
    structure (the pure-Neumann null space is one constant per component)."""
    from scipy import ndimage
    for seed in range(4):
        c = W.random_case(seed, 9, 8, 7, fill=0.35)
        g = oracle.Grid.from_case(c)
        nc, comp = g.components()
        lab, n2 = ndimage.label(c.mask, structure=ndimage.generate_binary_structure(3, 1))
        assert nc == n2
        lab = lab.reshape(-1) - 1
        # same partition up to renumbering
        pairs = set(zip(comp[lab >= 0].tolist(), lab[lab >= 0].tolist()))
        assert len(pairs) == nc
        assert np.all(comp[lab < 0] == -1)


def test_isolated_voxel_has_empty_row():
    """A tissue voxel with no tissue face-neighbour takes part in no valid pair:
    its row and diagonal are zero and the solver leaves it alone."""
    mask = np.zeros((3, 3, 3), np.uint8)
    mask[1, 1, 1] = 1
    fib = np.zeros((3, 3, 3, 3))
    fib[..., 0] = 1
    g = oracle.Grid(3, 3, 3, 0.5, mask, fib)
    u = np.arange(27, dtype=float)
    assert np.all(g.apply_L(0.2, 0.05, u) == 0.0)
    assert np.all(g.diag_L(0.2, 0.05) == 0.0)


# ---------------------------------------------------------------------------
# Jacobi damping: Eq. dampjac1 and the damping requirement of the Jacobi study
# ---------------------------------------------------------------------------

def test_undamped_jacobi_diverges_damped_converges():
    """The Laplacian solve needs damping: on an isotropic full box
    rho(D^-1 L) = 8/3 so omega = 1 diverges; the default damping converges."""
    n = 6
    g = _full_box(n, n, n, 0.5)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(g.n)
    b = g.apply_L(0.1, 0.1, u)
    _, it, rr, st = g.jacobi(0.1, 0.1, b, np.zeros(g.n), omega=1.0, tol=1e-8, m=1, max_iter=300)
    assert st == 1 and rr > 1.0
    _, it, rr, st = g.jacobi(0.1, 0.1, b, np.zeros(g.n), omega=0.0, tol=1e-8, m=1, max_iter=100000)
    assert st == 0 and rr <= 1e-8


def test_default_damping_bound_holds_on_masks():
    """The default omega is 1.8 / (8 sL / (sL + 2 sT)); the measured spectral
    radius of D^-1 L on random masks stays below that Fourier bound, so
    omega * rho < 2."""
    for seed in range(3):
        c, g = _random_grid(seed + 10, 7, 6, 5)
        for sL, sT in ((0.2, 0.05), (0.4, 0.15)):
            A, t = _dense(g, sL, sT)
            d = np.diag(A)
            keep = d > 0
            A = A[np.ix_(keep, keep)]
            rho = np.linalg.eigvals(A / d[keep][:, None]).real.max()
            omega = oracle.lib().og_default_omega(sL, sT)
            assert omega * rho < 1.9


# ---------------------------------------------------------------------------
# Mitchell-Schaeffer reaction: Eqs. ms1, ms2 with explicit Euler
# ---------------------------------------------------------------------------

def _cell(v0, w0=1.0, dt=0.01):
    mask = np.ones((1, 1, 1), np.uint8)
    fib = np.zeros((1, 1, 1, 3), np.float32)
    c = W.Case("cell", 1, 1, 1, 0.5, mask, fib, W.Params(dt=dt), [], model=W.MONO, precision=W.FP64)
    s = oracle.Sim(c)
    s.set_state(v=[v0], w=[w0], ve=[0.0])
    return s


def _trace(s, nsteps):
    vs, ws = [], []
    for _ in range(nsteps):
        st = s.state()
        vs.append(st["v"][0])
        ws.append(st["w"][0])
        s.step()
    return np.array(vs), np.array(ws)


def test_rest_state_is_a_fixed_point_bitwise():
    """v = 0, w = 1 without stimulus is an exact fixed point of Eqs. ms1/ms2 and
    of the diffusion and elliptic steps (L 0 = 0), in both models."""
    for model in (W.MONO, W.BI):
        c = W.random_case(3, 8, 6, 5, model=model)
        c.stimuli = []
        s = oracle.Sim(c)
        s.run(7)
        st = s.state()
        assert np.all(st["v"] == 0.0) and np.all(st["w"] == 1.0) and np.all(st["ve"] == 0.0)
        assert np.all(st["tact"] == -1.0)
        assert s.total_iters == 0


def test_excitation_threshold():
    """With w = 1 the cubic of Eq. ms1 has an unstable root a ~ 0.0528: kicks
    below a decay to rest, kicks above a fire an action potential."""
    a = GOLD["ms_threshold_a"]["value"]
    b = GOLD["ms_upper_state_b"]["value"]
    v, _ = _trace(_cell(a - 0.008), 3000)
    assert v.max() <= a and v[-1] < 0.1 * (a - 0.008) and np.all(np.diff(v) <= 0)
    v, _ = _trace(_cell(a + 0.008), 3000)
    assert v.max() > 0.9 and v.max() < b


def test_gate_closing_and_opening_branches():
    """Eq. ms2 with explicit Euler: while v >= v_gate the gate decays exactly as
    w_n = (1 - dt/tau_close)^n (closing branch read as -w/tau_close); the
    plateau lasts at least until w falls below 4 tau_in / tau_out; afterwards
    1 - w decays as (1 - dt/tau_open)^n."""
    dt = 0.01
    v, w = _trace(_cell(0.2, 1.0, dt), 60000)
    up = np.nonzero(v >= 0.13)[0]
    start, end = up[0], up[-1]
    assert np.all(np.diff(up) == 1)  # one contiguous action potential
    n = np.arange(end - start)
    np.testing.assert_allclose(w[start + 1:end + 1], w[start] * (1 - dt / 150.0) ** (n + 1), rtol=1e-9)
    apd = (end - start) * dt
    assert apd >= GOLD["apd_lower_bound_ms"]["value"]
    assert apd <= 1.25 * GOLD["apd_lower_bound_ms"]["value"]
    assert w[end] <= GOLD["plateau_gate_floor"]["value"] * 1.05
    rec = 1.0 - w[end + 1:end + 2001]
    m = np.arange(1, len(rec))
    np.testing.assert_allclose(rec[1:], rec[0] * (1 - dt / 120.0) ** m, rtol=1e-9)


# ---------------------------------------------------------------------------
# tissue dynamics: monodomain (Eq. monodomain1) and bidomain (Eq. bidomain1)
# ---------------------------------------------------------------------------

def test_plane_wave_conduction_velocity():
    """A planar front along the fibres travels at the bistable closed-form
    speed c = sqrt(D/(2 tau_in)) (b - 2a) with D = lambda/(1+lambda) sigma_L/K
    (Eq. monodomain1 with Eq. ms1); the oracle is within 2 % on a 0.04 mm
    cable.  A missing lambda/(1+lambda) or a wrong dx scaling would be off by
    >= 40 %."""
    dx, dt = 0.04, 0.002
    nx = int(round(6.0 / dx))
    mask = np.ones((1, 1, nx), np.uint8)
    fib = np.zeros((1, 1, nx, 3), np.float32)
    fib[..., 0] = 1.0
    st = W.Stimulus((0, 0, 0), (int(round(0.3 / dx)), 1, 1), 0.0, 1.0, 0.5)
    c = W.Case("cable", nx, 1, 1, dx, mask, fib, W.Params(dt=dt), [st], model=W.MONO,
               precision=W.FP64)
    s = oracle.Sim(c)
    s.run(int(round(25.0 / dt)))
    ta = s.state()["tact"]
    x = (np.arange(nx) + 0.5) * dx
    ia, ib = np.argmin(abs(x - 2.0)), np.argmin(abs(x - 5.0))
    cv = (x[ib] - x[ia]) / (ta[ib] - ta[ia])
    c_ex = GOLD["plane_wave_cv_mm_per_ms"]["value"]
    assert abs(cv / c_ex - 1.0) < 0.02, (cv, c_ex)


def test_charge_conservation_of_diffusion_step():
    """With the reaction switched off (huge time constants) the diffusion step
    conserves sum_T v exactly up to rounding (no-flux boundaries), in both
    models, and the elliptic right-hand side has zero sum."""
    for model in (W.MONO, W.BI):
        c = W.random_case(4, 9, 7, 6, model=model)
        c.stimuli = []
        p = c.params
        p.tau_in = p.tau_out = 1e300
        p.tau_open = p.tau_close = 1e300
        s = oracle.Sim(c)
        v, w, ve = W.random_state(4, c)
        s.set_state(v, w, ve)
        s0 = v.sum()
        s.step()
        v1 = s.state()["v"]
        assert abs(v1.sum() - s0) <= 1e-12 * np.abs(v).sum()
        assert not np.array_equal(v1, v)


def test_equal_anisotropy_elliptic_solution():
    """With Sigma_e = lambda Sigma_i the elliptic equation (Eq. bidomain1,
    line 2) is solved by ve = -v/(1+lambda) + const per component."""
    c = W.random_case(8, 8, 7, 6, model=W.BI, unequal=False, rel_tol=1e-12, check_every=1)
    c.params.max_iter = 400000
    s = oracle.Sim(c)
    v, w, ve = W.random_state(8, c)
    s.set_state(v, w, ve)
    assert s.step() == 0
    st = s.state()
    nc, comp = s.grid.components()
    t = comp >= 0
    for cc in range(nc):
        sel = comp == cc
        exp = -(st["v"][sel] - st["v"][sel].mean()) / 2.0
        np.testing.assert_allclose(st["ve"][sel], exp, rtol=0, atol=1e-8)
    assert np.all(st["ve"][~t] == 0.0)


def test_bidomain_approaches_monodomain_first_order_in_dt():
    """With Sigma_e = lambda Sigma_i the bidomain step (parabolic with the
    previous ve, Lie splitting) differs from the monodomain step only by the
    O(dt) splitting lag: halving dt halves the difference."""
    diffs = []
    for dt in (0.02, 0.01):
        out = []
        for model in (W.MONO, W.BI):
            c = W.random_case(9, 8, 8, 6, model=model, unequal=False, dt=dt, rel_tol=1e-11,
                              check_every=5)
            c.params.max_iter = 400000
            s = oracle.Sim(c)
            v, w, _ = W.random_state(9, c)
            # consistent start: ve = -v / (1 + lambda)
            ve = np.where(c.mask.reshape(-1) > 0, -v / 2.0, 0.0)
            s.set_state(v, w, ve)
            s.run(int(round(1.0 / dt)))
            out.append(s.state()["v"])
        diffs.append(np.abs(out[0] - out[1]).max())
    ratio = diffs[0] / diffs[1]
    assert diffs[0] > 0 and 1.7 < ratio < 2.3, diffs


def test_activation_time_is_first_crossing():
    """t_act is recorded once, at the first upward crossing of v = 0.5, inside
    the step interval where it happens."""
    s = _cell(0.2, 1.0, 0.01)
    prev = s.state()["v"][0]
    for n in range(2000):
        s.step()
        st = s.state()
        cur = st["v"][0]
        if prev < 0.5 <= cur:
            assert n * 0.01 <= st["tact"][0] <= (n + 1) * 0.01
            first = st["tact"][0]
            break
        prev = cur
    s.run(40000)
    assert s.state()["tact"][0] == first
