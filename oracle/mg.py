"""Multigrid-preconditioned conjugate gradients for the elliptic equation of
the bidomain step -- FP64 CPU oracle (TEST INFRASTRUCTURE ONLY: imported by
tests/, by __graft_entry__.smoke and by bench.py's CPU legs, never by the
product).

The thesis solves the elliptic equation (Eq. bidomain1, second line) by
Jacobi iteration (Eq. dampjac1) and names multigrid as future work for the
solver (chapter "Review & Outlook").  This is a study of that future work,
written out plainly; no CUDA path implements it (the operator's near-null
hourglass modes defeat constant aggregates).  Pinned by
tests/test_oracle_mg_pins.py: the probing assembly against an independent
assembly, the Galerkin levels, the symmetry of the V-cycle, the solve against
a dense least-squares solution.

* A = the elliptic operator L_{i+e} of the oracle (og_apply_L) on its domain
  (tissue, plus the torso if the grid has one), assembled exactly into a
  sparse matrix (its 27-point stencil probed with 27 colour classes).
* Levels l = 0 .. L-1.  Level l+1 is the grid halved (rounded up) in every
  axis; coarse voxel C = (I, J, K) owns the fine voxels (2I+a, 2J+b, 2K+c),
  a, b, c in {0, 1}.  The prolongation P_l copies a coarse value to the
  children of C that are in the level-l domain; the level-(l+1) domain is the
  set of coarse voxels with a child in it.  A_{l+1} = P_l^T A_l P_l (Galerkin):
  symmetric, positive semi-definite, and A_{l+1} 1 = 0 on every component, as
  on the fine level.  Coarsening stops at a grid of at most COARSEST voxels a
  side.
* Smoother: damped Jacobi, x <- x + omega_l D_l^-1 (r - A_l x), with D_l the
  diagonal of A_l (rows with D_l = 0 are left alone) and
  omega_l = OMEGA_SCALE / lambda_max(D_l^-1 A_l), the largest eigenvalue by
  POWER_STEPS power steps from a fixed start vector (all ones plus the
  index-based ramp below), times 1.05.
* V-cycle M(r) on level l: from x = 0, NU pre-smoothing sweeps, the residual
  restricted (P_l^T), the coarse correction M(P^T r) prolonged and added,
  NU post-smoothing sweeps; on the coarsest level COARSE_SWEEPS sweeps.
  Pre- and post-smoothing are the same, so M is symmetric.
* PCG (Hestenes-Stiefel) on A x = b from the warm start x0, with the
  preconditioned residual z = M r projected to zero mean on every
  face-connected component of the domain (the null space of A).  Stop when
  ||r_k||_2 <= tol ||b||_2 (r_k the recurred residual), checked for k = 0
  and after every iteration; at most max_iter iterations.
"""
from __future__ import annotations

from typing import List, Optional, Tuple

import numpy as np
import scipy.sparse as sp

NU = 2               # damped-Jacobi sweeps before and after the coarse correction
COARSE_SWEEPS = 64   # damped-Jacobi sweeps on the coarsest level
COARSEST = 8         # coarsen while the grid has more than this many voxels on a side
OMEGA_SCALE = 1.5    # omega_l = OMEGA_SCALE / (1.05 lambda_max(D_l^-1 A_l))
POWER_STEPS = 30


def assemble(grid, sL: float, sT: float) -> Tuple[sp.csr_matrix, np.ndarray]:
    """The elliptic operator of the oracle grid restricted to its domain, as a
    sparse matrix, and the domain's grid indices.  The stencil reaches one
    voxel in each axis, so the 27 classes (i mod 3, j mod 3, k mod 3) meet
    every voxel's 3x3x3 neighbourhood once each: applying the operator to the
    indicator of a class gives, at every voxel, its coefficient with the one
    class member next to it."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    n = nx * ny * nz
    dom = np.nonzero(grid.domain())[0]
    m = len(dom)
    pos = -np.ones(n, np.int64)
    pos[dom] = np.arange(m)
    q = np.arange(n)
    ii, jj, kk = q % nx, (q // nx) % ny, q // (nx * ny)
    qi, qj, qk = ii[dom], jj[dom], kk[dom]
    rows, cols, vals = [], [], []
    for cz in range(3):
        for cy in range(3):
            for cx in range(3):
                u = ((ii % 3 == cx) & (jj % 3 == cy) & (kk % 3 == cz)).astype(np.float64)
                Lu = grid.apply_L(sL, sT, u)[dom]
                pi = qi + (cx - qi + 1) % 3 - 1
                pj = qj + (cy - qj + 1) % 3 - 1
                pk = qk + (cz - qk + 1) % 3 - 1
                inside = (pi >= 0) & (pi < nx) & (pj >= 0) & (pj < ny) & (pk >= 0) & (pk < nz)
                col = np.full(m, -1, np.int64)
                col[inside] = pos[pi[inside] + nx * (pj[inside] + ny * pk[inside])]
                sel = (col >= 0) & (Lu != 0.0)
                rows.append(np.nonzero(sel)[0])
                cols.append(col[sel])
                vals.append(Lu[sel])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m, m))
    return A, dom


class Level:
    """One level: its grid size, domain (grid indices), operator, diagonal and
    damping, and (below the coarsest) the prolongation to it from the next."""

    def __init__(self, dims, dom, A):
        self.dims, self.dom, self.A = dims, dom, A
        self.diag = A.diagonal().copy()
        self.inv_diag = np.where(self.diag > 0, 1.0 / np.where(self.diag > 0, self.diag, 1.0), 0.0)
        self.omega = OMEGA_SCALE / (1.05 * lambda_max(A, self.inv_diag))
        self.P: Optional[sp.csr_matrix] = None   # to this level from the next coarser one


def lambda_max(A: sp.csr_matrix, inv_diag: np.ndarray) -> float:
    """Largest eigenvalue of D^-1 A by power steps from a fixed start vector."""
    m = A.shape[0]
    x = 1.0 + np.arange(m, dtype=np.float64) / max(m, 1)
    lam = 0.0
    for _ in range(POWER_STEPS):
        y = inv_diag * (A @ x)
        lam = float(np.linalg.norm(y) / max(np.linalg.norm(x), 1e-300))
        x = y / max(np.linalg.norm(y), 1e-300)
    return lam


def coarsen(level: Level) -> Tuple[Level, sp.csr_matrix]:
    """The next coarser level and the prolongation to `level` from it."""
    nx, ny, nz = level.dims
    cx, cy, cz = (nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2
    f = level.dom
    fi, fj, fk = f % nx, (f // nx) % ny, f // (nx * ny)
    parent = (fi // 2) + cx * ((fj // 2) + cy * (fk // 2))
    cdom = np.unique(parent)
    cpos = np.searchsorted(cdom, parent)
    P = sp.csr_matrix((np.ones(len(f)), (np.arange(len(f)), cpos)), shape=(len(f), len(cdom)))
    Ac = (P.T @ level.A @ P).tocsr()
    return Level((cx, cy, cz), cdom, Ac), P


def hierarchy(grid, sL: float, sT: float) -> List[Level]:
    A, dom = assemble(grid, sL, sT)
    levels = [Level((grid.nx, grid.ny, grid.nz), dom, A)]
    while max(levels[-1].dims) > COARSEST:
        c, P = coarsen(levels[-1])
        levels[-1].P = P
        levels.append(c)
    return levels


def smooth(level: Level, x: np.ndarray, b: np.ndarray, sweeps: int) -> np.ndarray:
    for _ in range(sweeps):
        x = x + level.omega * level.inv_diag * (b - level.A @ x)
    return x


def vcycle(levels: List[Level], b: np.ndarray, l: int = 0) -> np.ndarray:
    lv = levels[l]
    x = np.zeros_like(b)
    if l == len(levels) - 1:
        return smooth(lv, x, b, COARSE_SWEEPS)
    x = smooth(lv, x, b, NU)
    r = b - lv.A @ x
    x = x + lv.P @ vcycle(levels, lv.P.T @ r, l + 1)
    return smooth(lv, x, b, NU)


def component_labels(grid, dom: np.ndarray) -> np.ndarray:
    nc, comp = grid.components()
    return comp[dom]


def project(z: np.ndarray, labels: np.ndarray) -> np.ndarray:
    """z minus its mean on every component."""
    s = np.bincount(labels, weights=z)
    c = np.bincount(labels)
    return z - (s / np.maximum(c, 1))[labels]


def pcg(levels: List[Level], labels: np.ndarray, b: np.ndarray, x0: np.ndarray, tol: float, max_iter: int):
    """MG-preconditioned CG on the domain vectors: (x, iterations, relative
    residual, converged)."""
    A = levels[0].A
    x = x0.copy()
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return x, 0, 0.0, True
    r = b - A @ x
    rr = float(np.linalg.norm(r))
    if rr <= tol * nb:
        return x, 0, rr / nb, True
    z = project(vcycle(levels, r), labels)
    p = z.copy()
    rz = float(r @ z)
    for k in range(1, max_iter + 1):
        q = A @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rr = float(np.linalg.norm(r))
        if rr <= tol * nb:
            return x, k, rr / nb, True
        z = project(vcycle(levels, r), labels)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter, rr / nb, False


def solve(grid, sL: float, sT: float, b_grid: np.ndarray, x0_grid: np.ndarray, tol: float, max_iter: int,
          levels: Optional[List[Level]] = None):
    """Solve on grid vectors (domain entries used; the rest returned as 0):
    (x, iterations, relative residual, converged, levels)."""
    if levels is None:
        levels = hierarchy(grid, sL, sT)
    dom = levels[0].dom
    labels = component_labels(grid, dom)
    xd, k, rel, ok = pcg(levels, labels, np.asarray(b_grid, np.float64)[dom], np.asarray(x0_grid, np.float64)[dom],
                         tol, max_iter)
    x = np.zeros(grid.n)
    x[dom] = xd
    return x, k, rel, ok, levels
