"""Seeded synthetic inputs for the voxel electrophysiology step.

This module is shared by the CPU oracle tests and the CUDA path's tests and
benchmark.  It builds *inputs only*: tissue masks, fibre fields, stimulus
boxes and parameter sets.  It contains none of the time-step arithmetic
(no ionic model, no diffusion operator, no solver).

Conventions
-----------
* Grid ``nx x ny x nz``; arrays have numpy shape ``(nz, ny, nx)`` so the flat
  C-order index is ``i + nx*(j + ny*k)`` (x fastest).
* Voxel ``(i, j, k)`` has centre ``((i+1/2) dx, (j+1/2) dx, (k+1/2) dx)``.
* ``mask`` is uint8 (1 = myocardium).  ``fib`` is float64 ``(nz, ny, nx, 3)``,
  unit or zero, as generated (no rounding to any storage precision): the FP64
  oracle takes it as it is and the library takes its float32 values (the type
  of ``ep_set_fibres``), so parity measures what the library does with a
  caller's fibres.  :meth:`Case.fibres_as_float32` gives the variant whose
  values both sides see exactly, for tests that pin FP64 arithmetic.
* Units: mm, ms, mS/mm; ``v`` dimensionless (0 rest, 1 peak).

Workload recipes (sizes and structure follow the thesis' experiments: the
Niederer-style slab of the EP benchmark section, the ellipsoidal ventricle
geometry and the rule-based helical fibres of the whole-heart chapter):

* ``config0``: monodomain FP64 slab 32^3, all tissue, dx 0.25, fibre angle
  -60..+60 deg linear in z, sigma 0.20/0.05, corner stimulus 4^3, dt 0.01,
  1000 steps.
* ``config1``: bidomain FP32, 128^3, ellipsoidal shell (55, 40, 40) voxels,
  wall 10 (9.5 % fill), transmural helical fibres, apex stimulus, dt 0.05,
  5000 steps.
* ``config2``: bidomain FP32, 256^3, two truncated ellipsoidal shells
  (biventricular, 20.3 % fill), fibres with seeded +-5 deg noise, 20000 steps.
* ``config3_instances`` / ``config4_requests``: many shell instances with
  sampled sizes, conductivities and stimulus sites.
* ``random_case``: small random masks/fibres for element-wise parity.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

MONO = 0
BI = 1
FP32 = 0
FP64 = 1


@dataclasses.dataclass
class Stimulus:
    lo: Tuple[int, int, int]  # inclusive voxel index (i, j, k)
    hi: Tuple[int, int, int]  # exclusive voxel index
    t_start: float = 0.0      # ms
    dur: float = 1.0          # ms
    amp: float = 0.5          # 1/ms, added to dv/dt


@dataclasses.dataclass
class Params:
    # Mitchell-Schaeffer constants (ms, dimensionless threshold)
    tau_in: float = 0.3
    tau_out: float = 6.0
    tau_open: float = 120.0
    tau_close: float = 150.0
    v_gate: float = 0.13
    # conductivities (mS/mm), intra- and extracellular
    sig_iL: float = 0.20
    sig_iT: float = 0.05
    sig_eL: float = 0.20
    sig_eT: float = 0.05
    lam: float = 1.0          # monodomain ratio lambda
    K: float = 1.0            # chi_m * C_m
    dt: float = 0.01          # ms
    omega: float = 0.0        # Jacobi damping; <= 0 selects 1.8 / (8 sL / (sL + 2 sT))
    rel_tol: float = 1e-6     # elliptic stop: ||b - A x|| <= rel_tol ||b||
    check_every: int = 10     # residual check interval (sweeps)
    max_iter: int = 100000    # sweep cap per solve
    diffusion: int = 0        # 0 explicit Euler, 1 implicit Euler (Eq. iejac1)
    solver: int = 0           # elliptic solve: 0 damped Jacobi (Eq. dampjac1), 1 Chebyshev-accelerated Jacobi,
                              # 2 eight-colour Gauss-Seidel / SOR (omega > 0 the SOR factor, else 1)
    cheb_lmin: float = 0.0    # spectral interval of D^-1 A for the Chebyshev solver (<= 0: estimated)
    cheb_lmax: float = 0.0
    sig_o: float = 0.0        # isotropic torso conductivity (mS/mm), used when the case has a torso


@dataclasses.dataclass
class Case:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    mask: np.ndarray          # uint8 (nz, ny, nx)
    fib: np.ndarray           # float64 (nz, ny, nx, 3), unit or zero
    params: Params
    stimuli: List[Stimulus]
    model: int = BI
    precision: int = FP32
    steps: int = 100
    torso: Optional[np.ndarray] = None      # uint8 (nz, ny, nx): conducting torso voxels outside the tissue
    electrodes: Optional[List[Tuple[int, int, int]]] = None   # (i, j, k) of RA, LA, LL

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_tissue(self) -> int:
        return int(self.mask.sum())

    def fib_flat(self) -> np.ndarray:
        """Fibres as a contiguous float32 array of length 3n, (fx, fy, fz) per
        voxel: the input type of ``ep_set_fibres``."""
        return np.ascontiguousarray(self.fib.reshape(-1, 3), dtype=np.float32).reshape(-1)

    def fibres_as_float32(self) -> "Case":
        """A copy whose fibres are rounded to float32 (kept as float64), so the
        oracle and the library see exactly the same values."""
        c = dataclasses.replace(self)
        c.fib = self.fib.astype(np.float32).astype(np.float64)
        return c

    def mask_flat(self) -> np.ndarray:
        return np.ascontiguousarray(self.mask.reshape(-1), dtype=np.uint8)


def _centres(n: Tuple[int, int, int], centre: Tuple[float, float, float]):
    """Voxel-centre coordinates (in voxel units) relative to ``centre`` = (cx, cy, cz)."""
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz) + 0.5 - centre[2],
                          np.arange(ny) + 0.5 - centre[1],
                          np.arange(nx) + 0.5 - centre[0], indexing="ij")
    return x, y, z


def _ellipsoid_level(x, y, z, ax, ay, az):
    return np.sqrt((x / ax) ** 2 + (y / ay) ** 2 + (z / az) ** 2)


def _helical_fibres(x, y, z, depth, helix_endo_deg=60.0, helix_epi_deg=-60.0):
    """Rule-based fibres: horizontal unit vector orthogonal to the position
    vector (circumferential direction), rotated about the position vector by a
    helix angle that varies linearly from endo (depth 0) to epi (depth 1)."""
    r = np.stack([x, y, z], axis=-1)
    rn = np.linalg.norm(r, axis=-1, keepdims=True)
    rhat = r / np.maximum(rn, 1e-12)
    circ = np.stack([-y, x, np.zeros_like(x)], axis=-1)  # z_hat x r
    cn = np.linalg.norm(circ, axis=-1, keepdims=True)
    fallback = np.zeros_like(circ)
    fallback[..., 0] = 1.0
    circ = np.where(cn > 1e-9, circ / np.maximum(cn, 1e-12), fallback)
    alpha = np.deg2rad(helix_endo_deg + (helix_epi_deg - helix_endo_deg) * depth)[..., None]
    f = np.cos(alpha) * circ + np.sin(alpha) * np.cross(rhat, circ)
    f /= np.maximum(np.linalg.norm(f, axis=-1, keepdims=True), 1e-12)
    return f


def _shell(x, y, z, semi, wall):
    """Mask and transmural depth of an ellipsoidal shell.

    ``semi`` = (ax, ay, az) outer semi-axes, inner semi-axes are semi - wall.
    Depth is the fraction along the ray from the centre between the inner
    (0) and outer (1) surfaces."""
    ax, ay, az = semi
    so = _ellipsoid_level(x, y, z, ax, ay, az)
    si = _ellipsoid_level(x, y, z, ax - wall, ay - wall, az - wall)
    m = (so <= 1.0) & (si > 1.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        depth = (1.0 - 1.0 / si) / (1.0 / so - 1.0 / si)
    depth = np.clip(np.nan_to_num(depth, nan=0.0), 0.0, 1.0)
    return m, depth


def _apex_block(mask: np.ndarray, ci: float, cj: float, size: int) -> Stimulus:
    """Stimulus block of side ``size`` at the lowest tissue voxel nearest to the
    vertical line through (ci, cj)."""
    nz, ny, nx = mask.shape
    i0 = int(math.floor(ci)) - size // 2
    j0 = int(math.floor(cj)) - size // 2
    col = mask[:, max(j0, 0):j0 + size, max(i0, 0):i0 + size]
    ks = np.nonzero(col.reshape(nz, -1).any(axis=1))[0]
    k0 = int(ks[0]) if len(ks) else 0
    return Stimulus(lo=(max(i0, 0), max(j0, 0), k0),
                    hi=(min(i0 + size, nx), min(j0 + size, ny), min(k0 + size, nz)),
                    t_start=0.0, dur=1.0, amp=0.5)


# --------------------------------------------------------------------------
# configs
# --------------------------------------------------------------------------

def config0() -> Case:
    n = 32
    k = np.arange(n)
    theta = np.deg2rad(-60.0 + 120.0 * k / (n - 1))
    f = np.zeros((n, n, n, 3), np.float64)
    f[..., 0] = np.cos(theta)[:, None, None]
    f[..., 1] = np.sin(theta)[:, None, None]
    p = Params(dt=0.01, sig_iL=0.20, sig_iT=0.05, sig_eL=0.20, sig_eT=0.05, lam=1.0, K=1.0)
    return Case("config0_mono_fp64_slab32", n, n, n, 0.25,
                np.ones((n, n, n), np.uint8), f, p,
                [Stimulus((0, 0, 0), (4, 4, 4), 0.0, 1.0, 0.5)],
                model=MONO, precision=FP64, steps=1000)


def slab(n: int = 512, model: int = MONO, unequal: bool = False) -> Case:
    """Dense all-tissue n^3 slab, the roofline workload whose working set is far
    above L2: fibres in the x-y plane rotating from -60 to +60 degrees through
    z (the config 0 rule), dx 0.5 mm, dt 0.05 ms, corner stimulus 8^3, FP32.
    ``unequal`` sets sigma_eT = 0.10 so that the bidomain solve is not the
    trivial equal-anisotropy one."""
    k = np.arange(n, dtype=np.float64)
    theta = np.deg2rad(-60.0 + 120.0 * k / max(n - 1, 1))
    fz = np.stack([np.cos(theta), np.sin(theta), np.zeros(n)], axis=-1)   # (n, 3), per z plane
    fib = np.broadcast_to(fz[:, None, None, :], (n, n, n, 3))
    p = Params(dt=0.05, sig_iL=0.20, sig_iT=0.05, sig_eL=0.20, sig_eT=0.10 if unequal else 0.05)
    return Case(f"slab{n}_{'bi' if model == BI else 'mono'}", n, n, n, 0.5, np.ones((n, n, n), np.uint8), fib, p,
                [Stimulus((0, 0, 0), (8, 8, 8), 0.0, 1.0, 0.5)], model=model, precision=FP32, steps=100)


def shell_case(n: int = 128, semi=(40.0, 40.0, 55.0), wall: float = 10.0,
               sig=(0.20, 0.05, 0.20, 0.05), dt: float = 0.05, steps: int = 5000,
               stim_size: int = 4, name: Optional[str] = None) -> Case:
    """Closed ellipsoidal shell centred in an n^3 grid (semi-axes in voxels,
    given as (ax, ay, az)); apex stimulus at the lowest tissue voxel."""
    c = n / 2.0
    x, y, z = _centres((n, n, n), (c, c, c))
    m, depth = _shell(x, y, z, semi, wall)
    f = _helical_fibres(x, y, z, depth)
    f[~m] = 0.0
    p = Params(dt=dt, sig_iL=sig[0], sig_iT=sig[1], sig_eL=sig[2], sig_eT=sig[3])
    mask = m.astype(np.uint8)
    stim = _apex_block(mask, c, c, stim_size)
    return Case(name or f"shell{n}", n, n, n, 0.5, mask, f, p, [stim],
                model=BI, precision=FP32, steps=steps)


def config1(unequal: bool = False) -> Case:
    sig = (0.20, 0.05, 0.20, 0.10) if unequal else (0.20, 0.05, 0.20, 0.05)
    return shell_case(128, (40.0, 40.0, 55.0), 10.0, sig, 0.05, 5000, 4,
                      name="config1_bi_shell128" + ("_unequal" if unequal else ""))


def config2(seed: int = 0, unequal: bool = False, n: int = 256) -> Case:
    """Biventricular mask from two truncated ellipsoidal shells in an n^3 grid
    (sizes given for n = 256 and scaled by n/256 otherwise)."""
    s = n / 256.0
    c = n / 2.0
    x, y, z = _centres((n, n, n), (c, c, c))
    lv_c = (0.0, -20.0 * s, 0.0)
    rv_c = (0.0, 30.0 * s, 0.0)
    lv_m, lv_d = _shell(x - lv_c[0], y - lv_c[1], z - lv_c[2], (85 * s, 85 * s, 125 * s), 32 * s)
    rv_m, rv_d = _shell(x - rv_c[0], y - rv_c[1], z - rv_c[2], (100 * s, 75 * s, 115 * s), 18 * s)
    lv_outer = _ellipsoid_level(x - lv_c[0], y - lv_c[1], z - lv_c[2], 85 * s, 85 * s, 125 * s) <= 1.0
    keep = z <= 85.0 * s
    lv = lv_m & keep
    rv = rv_m & ~lv_outer & keep
    m = lv | rv
    f_lv = _helical_fibres(x - lv_c[0], y - lv_c[1], z - lv_c[2], lv_d)
    f_rv = _helical_fibres(x - rv_c[0], y - rv_c[1], z - rv_c[2], rv_d)
    f = np.where(lv[..., None], f_lv, f_rv)
    # seeded +-5 deg rotation about a random axis orthogonal to f
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(f.shape)
    a -= (a * f).sum(-1, keepdims=True) * f
    a /= np.maximum(np.linalg.norm(a, axis=-1, keepdims=True), 1e-12)
    ang = np.deg2rad(rng.uniform(-5.0, 5.0, size=f.shape[:-1]))[..., None]
    # Rodrigues rotation of f about unit axis a (a orthogonal to f)
    f = f * np.cos(ang) + np.cross(a, f) * np.sin(ang)
    f /= np.maximum(np.linalg.norm(f, axis=-1, keepdims=True), 1e-12)
    f[~m] = 0.0
    sig = (0.20, 0.05, 0.20, 0.10) if unequal else (0.20, 0.05, 0.20, 0.05)
    p = Params(dt=0.05, sig_iL=sig[0], sig_iT=sig[1], sig_eL=sig[2], sig_eT=sig[3])
    mask = m.astype(np.uint8)
    stim = _apex_block(mask * lv.astype(np.uint8), c + lv_c[0], c + lv_c[1], max(2, int(round(6 * s))))
    return Case(f"config2_bi_biv{n}" + ("_unequal" if unequal else ""), n, n, n, 0.5, mask,
                f, p, [stim], model=BI, precision=FP32, steps=20000)


def ecg_case(n: int = 256, sig_o: float = 1.0, seed: int = 0) -> Case:
    """The config 2 heart in its n^3 box, every other voxel of the box a
    conducting torso of conductivity sig_o (mS/mm), electrodes RA, LA, LL at
    corners of the box (the ECG set-up of Sec. "Electrocardiogram")."""
    c = with_torso(config2(seed=seed, n=n), sig_o=sig_o)
    c.name = f"ecg_biv{n}_sigo{sig_o:g}"
    return c


def sampled_shell(rng: np.random.Generator, n: int, steps: int, name: str) -> Case:
    """One instance of the batched / served workloads: shell scaled by n/128
    from config 1, sampled conductivities, stimulus at a random tissue voxel."""
    s = n / 128.0
    siL = rng.uniform(0.15, 0.25)
    siT = siL / rng.uniform(3.0, 5.0)
    seL = rng.uniform(0.15, 0.25)
    seT = seL / rng.uniform(3.0, 5.0)
    case = shell_case(n, (40.0 * s, 40.0 * s, 55.0 * s), max(2.0, 10.0 * s),
                      (siL, siT, seL, seT), 0.05, steps, 4, name=name)
    idx = np.argwhere(case.mask > 0)
    k, j, i = idx[rng.integers(len(idx))]
    lo = (max(int(i) - 2, 0), max(int(j) - 2, 0), max(int(k) - 2, 0))
    hi = (min(int(i) + 2, n), min(int(j) + 2, n), min(int(k) + 2, n))
    case.stimuli = [Stimulus(lo, hi, 0.0, 1.0, 0.5)]
    return case


def config3_sizes(seed: int = 0, count: int = 64, lo: int = 48, hi: int = 160) -> List[int]:
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(lo, hi + 1, size=count)]


def config3_instances(seed: int = 0, count: int = 64, lo: int = 48, hi: int = 160,
                      steps: int = 1000) -> List[Case]:
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=count)
    return [sampled_shell(rng, int(n), steps, f"inst{q}_n{int(n)}") for q, n in enumerate(sizes)]


def config4_requests(seed: int = 0, count: int = 32, rate_per_s: float = 10.0,
                     lo: int = 64, hi: int = 256, steps: int = 1000):
    """Poisson arrival times (s) and request cases for the serving loop."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = rng.integers(lo, hi + 1, size=count)
    cases = [sampled_shell(rng, int(n), steps, f"req{q}_n{int(n)}") for q, n in enumerate(sizes)]
    return arrivals, cases


# --------------------------------------------------------------------------
# small random cases for element-wise parity
# --------------------------------------------------------------------------

def random_mask(rng: np.random.Generator, nx: int, ny: int, nz: int, fill: float = 0.6,
                blobs: int = 4) -> np.ndarray:
    """Union of random ellipsoidal blobs, plus salt noise, as uint8 (nz, ny, nx)."""
    x, y, z = _centres((nx, ny, nz), (0.0, 0.0, 0.0))
    m = np.zeros((nz, ny, nx), bool)
    for _ in range(blobs):
        c = rng.uniform(0, 1, 3) * np.array([nx, ny, nz])
        r = rng.uniform(0.3, 0.7, 3) * np.array([nx, ny, nz])
        m |= ((x - c[0]) / r[0]) ** 2 + ((y - c[1]) / r[1]) ** 2 + ((z - c[2]) / r[2]) ** 2 <= 1.0
    flip = rng.uniform(size=m.shape) < (1.0 - fill) * 0.2
    m ^= flip
    return m.astype(np.uint8)


def random_fibres(rng: np.random.Generator, shape, zero_frac: float = 0.05) -> np.ndarray:
    f = rng.standard_normal(tuple(shape) + (3,))
    f /= np.maximum(np.linalg.norm(f, axis=-1, keepdims=True), 1e-12)
    f[rng.uniform(size=shape) < zero_frac] = 0.0
    return f


def random_case(seed: int, nx: int, ny: int, nz: int, model: int = BI, precision: int = FP32,
                dx: float = 0.5, dt: float = 0.05, steps: int = 20, fill: float = 0.6,
                mask: Optional[np.ndarray] = None, unequal: bool = True,
                check_every: int = 10, rel_tol: float = 1e-6) -> Case:
    """Random mask and fibres, random initial state supplied separately via
    :func:`random_state`; a stimulus box near the grid origin."""
    rng = np.random.default_rng(seed)
    if mask is None:
        mask = random_mask(rng, nx, ny, nz, fill)
    fib = random_fibres(rng, (nz, ny, nx))
    fib[mask == 0] = 0.0
    p = Params(dt=dt, sig_iL=0.20, sig_iT=0.05, sig_eL=0.20, sig_eT=0.10 if unequal else 0.05,
               check_every=check_every, rel_tol=rel_tol)
    st = Stimulus((0, 0, 0), (min(4, nx), min(4, ny), min(4, nz)), 0.0, 1.0, 0.5)
    return Case(f"rand{seed}_{nx}x{ny}x{nz}", nx, ny, nz, dx, mask.astype(np.uint8), fib, p, [st],
                model=model, precision=precision, steps=steps)


def random_state(seed: int, case: Case):
    """A random excitable state (v, w, ve) in float64, zero on non-tissue voxels.

    v has a smooth front plus noise so that every stencil term is exercised."""
    rng = np.random.default_rng(seed + 7919)
    nz, ny, nx = case.mask.shape
    x, y, z = _centres((nx, ny, nz), (0.0, 0.0, 0.0))
    front = 0.5 * (1.0 - np.tanh((x + 0.7 * y + 0.4 * z - 0.5 * nx) / 2.0))
    v = np.clip(front + 0.05 * rng.standard_normal(front.shape), 0.0, 1.0)
    w = rng.uniform(0.2, 1.0, size=v.shape)
    ve = 0.1 * rng.standard_normal(v.shape)
    t = case.mask > 0
    d = t if case.torso is None else t | (case.torso > 0)   # v_e lives on tissue + torso
    return (np.where(t, v, 0.0).reshape(-1), np.where(t, w, 1.0).reshape(-1),
            np.where(d, ve, 0.0).reshape(-1))


def front_state(case: Case, rise_vox: float = 10.0, width_vox: float = 1.5):
    """A propagating start (v, w, ve) in float64: excited tissue below a
    horizontal front ``rise_vox`` voxels above the case's lowest tissue voxel
    (the apex of the shells), v = 1/2 (1 - tanh(d / width)) with d the height
    above the front, w = 1 (recovered gates), ve = 0.  Closed form, no seed:
    the full-run parity windows start here so that the front crosses many
    voxels within a few oracle steps."""
    nz, ny, nx = case.mask.shape
    ks = np.nonzero(case.mask.reshape(nz, -1).any(axis=1))[0]
    z0 = (float(ks[0]) if len(ks) else 0.0) + rise_vox
    z = np.broadcast_to(np.arange(nz, dtype=np.float64)[:, None, None] + 0.5, (nz, ny, nx))
    v = 0.5 * (1.0 - np.tanh((z - z0) / width_vox))
    t = case.mask > 0
    return (np.where(t, v, 0.0).reshape(-1), np.where(t, 1.0, 1.0).reshape(-1), np.zeros(case.n))


def corner_electrodes(nx: int, ny: int, nz: int) -> List[Tuple[int, int, int]]:
    """RA, LA, LL at corners of the box: the arms at the top (high z) on either
    side in y, the leg at the bottom corner diametrically opposite RA."""
    return [(0, ny - 1, nz - 1), (0, 0, nz - 1), (nx - 1, 0, 0)]


def with_torso(case: Case, sig_o: float = 1.0, pad: int = 0, fill: Optional[float] = None,
               seed: int = 0) -> Case:
    """The case's tissue inside a conducting torso of isotropic conductivity
    sig_o (mS/mm): the grid grows by `pad` voxels on every side and every
    non-tissue voxel of the box is torso (or, with `fill`, a random fraction of
    them, for tests).  Electrodes RA, LA, LL at corners of the box."""
    nx, ny, nz = case.nx + 2 * pad, case.ny + 2 * pad, case.nz + 2 * pad
    mask = np.zeros((nz, ny, nx), np.uint8)
    fib = np.zeros((nz, ny, nx, 3), np.float64)
    sl = (slice(pad, pad + case.nz), slice(pad, pad + case.ny), slice(pad, pad + case.nx))
    mask[sl] = case.mask
    fib[sl] = case.fib
    torso = (mask == 0).astype(np.uint8)
    electrodes = corner_electrodes(nx, ny, nz)
    if fill is not None:
        rng = np.random.default_rng(seed + 104729)
        torso &= (rng.random(torso.shape) < fill).astype(np.uint8)
        for (i, j, k) in electrodes:   # the electrodes stay on the domain
            torso[k, j, i] = 0 if mask[k, j, i] else 1
    p = dataclasses.replace(case.params, sig_o=sig_o)
    stims = [Stimulus(tuple(a + pad for a in st.lo), tuple(a + pad for a in st.hi), st.t_start, st.dur, st.amp)
             for st in case.stimuli]
    return Case(case.name + f"_torso{pad}", nx, ny, nz, case.dx, mask, fib, p, stims, model=case.model,
                precision=case.precision, steps=case.steps, torso=torso, electrodes=electrodes)


# ---------------------------------------------------------------------------
# Signed-distance scenes (inputs of the geometry encoder; the SDF arithmetic
# itself lives in the encoder and in the oracle, not here)
# ---------------------------------------------------------------------------
SDF_CUBOID, SDF_ELLIPSOID, SDF_CYLINDER, SDF_CONE = 0, 1, 2, 3
SDF_UNION, SDF_INTERSECT, SDF_SUBTRACT, SDF_HOLLOW, SDF_SMOOTH_UNION = 10, 11, 12, 13, 14
REGION_MYOCARDIUM, REGION_FAST, REGION_INSULATOR = 1, 2, 3
IDENTITY9 = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)


@dataclasses.dataclass
class SdfNode:
    op: int
    a: float = 0.0
    b: float = 0.0
    c: float = 0.0
    centre: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    rot: Tuple[float, ...] = IDENTITY9


@dataclasses.dataclass
class SdfRegion:
    first: int
    count: int
    kind: int
    axis: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    scale: float = 1.0


@dataclasses.dataclass
class SdfScene:
    nodes: List[SdfNode]
    regions: List[SdfRegion]
    nx: int
    ny: int
    nz: int
    dx: float
    origin: Tuple[float, float, float]
    helix_rad: float = 0.4 * math.pi


def rotation(axis: Tuple[float, float, float], angle: float) -> Tuple[float, ...]:
    """Row-major matrix of the rotation by -angle about axis (it maps scene
    coordinates into a frame turned by +angle)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    R = np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K
    return tuple(float(v) for v in R.T.reshape(-1))


class _Prog:
    """Builds postfix programs region by region."""

    def __init__(self):
        self.nodes: List[SdfNode] = []
        self.regions: List[SdfRegion] = []
        self._start = 0

    def push(self, op, a=0.0, b=0.0, c=0.0, centre=(0.0, 0.0, 0.0), rot=IDENTITY9):
        self.nodes.append(SdfNode(op, a, b, c, tuple(centre), tuple(rot)))
        return self

    def region(self, kind, axis=(0.0, 0.0, 1.0), scale=1.0):
        self.regions.append(SdfRegion(self._start, len(self.nodes) - self._start, kind, tuple(axis), scale))
        self._start = len(self.nodes)
        return self


def schematic_heart(n: int = 128, size_mm: float = 128.0, wall: float = 0.12, fast_gain: float = 2.0,
                    sig_L: float = 0.20, sig_T: float = 0.05) -> SdfScene:
    """The thesis' schematic whole heart (Sec. "Myocardium", "Fibre
    Directions"), sizes read off its figures (the text gives none), in mm
    with the origin at the centre of an n^3 box of side size_mm:
    - myocardium: the hollow union of two half-spheres above the origin
      (atria) and two half-ellipsoids below it (ventricles), plus the
      intra-ventricular septum, a vertical elliptic disc; the shells are
      `wall` thick in the primitives' normalised units;
    - the horizontal septum, an elliptic disc at the origin, is an insulator
      (zero conductivity), so is each hollow elliptic cone of the mitral and
      tricuspid valves that pierce it, and each hollow vertical vessel on top;
    - a vertical fast fibre (Purkinje) through the centre with `fast_gain`
      times the longitudinal conductivity, the only path from atria to
      ventricles."""
    P = _Prog()
    lv, rv = (14.0, 0.0, 0.0), (-16.0, 4.0, 0.0)
    up = (0.0, 0.0, 40.0)       # half-space z > 0: a cuboid above the origin
    down = (0.0, 0.0, -60.0)
    # myocardium: ((LA u RA) n up) u ((LV u RV) n down), hollowed, plus the septum disc
    P.push(SDF_ELLIPSOID, 26.0, 26.0, 26.0, (lv[0], lv[1], 0.0)).push(SDF_ELLIPSOID, 22.0, 22.0, 22.0, (rv[0], rv[1], 0.0))
    P.push(SDF_UNION).push(SDF_CUBOID, 60.0, 60.0, 40.0, up).push(SDF_INTERSECT)
    P.push(SDF_ELLIPSOID, 26.0, 26.0, 52.0, (lv[0], lv[1], 0.0)).push(SDF_ELLIPSOID, 22.0, 24.0, 46.0, (rv[0], rv[1], 0.0))
    P.push(SDF_UNION).push(SDF_CUBOID, 60.0, 60.0, 60.0, down).push(SDF_INTERSECT)
    P.push(SDF_UNION).push(SDF_HOLLOW, wall)
    P.push(SDF_ELLIPSOID, 3.0, 20.0, 40.0, (-1.0, 2.0, -20.0)).push(SDF_UNION)
    P.region(REGION_MYOCARDIUM)
    # horizontal septum: a thin elliptic disc across the whole heart
    P.push(SDF_ELLIPSOID, 48.0, 36.0, 2.0, (0.0, 2.0, 0.0)).region(REGION_INSULATOR)
    # valves: hollow elliptic cones through the septum; vessels: hollow cylinders above
    P.push(SDF_CONE, 7.0, 6.0, -0.3, (lv[0], lv[1] + 6.0, 0.0)).push(SDF_HOLLOW, 1.0)
    P.push(SDF_CONE, 6.0, 6.0, -0.3, (rv[0], rv[1] + 6.0, 0.0)).push(SDF_HOLLOW, 1.0).push(SDF_UNION)
    P.region(REGION_INSULATOR)
    P.push(SDF_CYLINDER, 6.0, 12.0, 0.0, (lv[0] - 6.0, 0.0, 40.0)).push(SDF_HOLLOW, 1.5)
    P.push(SDF_CYLINDER, 5.0, 12.0, 0.0, (rv[0] + 4.0, rv[1], 38.0)).push(SDF_HOLLOW, 1.5).push(SDF_UNION)
    P.region(REGION_INSULATOR)
    # fast fibre: vertical cylinder from the atria to the apex region
    scale = math.sqrt((fast_gain * sig_L - sig_T) / (sig_L - sig_T))
    P.push(SDF_CYLINDER, 1.6, 30.0, 0.0, (0.0, 2.0, -6.0)).region(REGION_FAST, (0.0, 0.0, 1.0), scale)
    dx = size_mm / n
    return SdfScene(P.nodes, P.regions, n, n, n, dx, (-size_mm / 2, -size_mm / 2, -size_mm / 2))


def random_scene(seed: int, n: int = 24, size_mm: float = 24.0) -> SdfScene:
    """A random scene for tests: every primitive and operator, rotations,
    three regions of each kind in turn."""
    rng = np.random.default_rng(seed)
    P = _Prog()

    def prim():
        op = int(rng.integers(0, 4))
        c = tuple(float(v) for v in rng.uniform(-size_mm / 4, size_mm / 4, 3))
        rot = rotation(tuple(rng.standard_normal(3)), float(rng.uniform(0, math.pi)))
        if op in (SDF_CUBOID, SDF_ELLIPSOID):
            a, b, cc = (float(v) for v in rng.uniform(2.0, size_mm / 3, 3))
        elif op == SDF_CYLINDER:
            a, b, cc = float(rng.uniform(1.5, size_mm / 4)), float(rng.uniform(2.0, size_mm / 3)), 0.0
        else:
            a, b, cc = float(rng.uniform(1.5, size_mm / 4)), float(rng.uniform(2.0, size_mm / 3)), float(rng.uniform(-0.5, 0.5))
        P.push(op, a, b, cc, c, rot)

    for kind in (REGION_MYOCARDIUM, REGION_INSULATOR, REGION_FAST):
        prim()
        for _ in range(int(rng.integers(1, 4))):
            prim()
            op = int(rng.choice([SDF_UNION, SDF_INTERSECT, SDF_SUBTRACT, SDF_SMOOTH_UNION]))
            P.push(op, float(rng.uniform(0.5, 3.0)) if op == SDF_SMOOTH_UNION else 0.0)
        if rng.random() < 0.5:
            P.push(SDF_HOLLOW, float(rng.uniform(0.1, 2.0)))
        ax = rng.standard_normal(3)
        P.region(kind, tuple(float(v) for v in ax / np.linalg.norm(ax)), float(rng.uniform(1.0, 1.6)))
    dx = size_mm / n
    return SdfScene(P.nodes, P.regions, n, n + 3, n - 2, dx, (-size_mm / 2, -size_mm / 2 - 1.0, -size_mm / 2 + 1.0))
