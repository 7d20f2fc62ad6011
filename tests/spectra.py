"""Spectral interval of the Jacobi-preconditioned elliptic operator D^-1 A,
computed from the FP64 oracle's operator alone (never from the CUDA path), so
that parity tests of the Chebyshev semi-iteration and of the estimated
damping give both sides an interval fixed independently.

D^-1 A is similar to the symmetric D^-1/2 A D^-1/2, whose eigenvalues are
computed here: densely (numpy eigvalsh of the unit-vector assembly) on small
domains, else by the Lanczos method of scipy's eigsh on the operator itself.
The null space of A (the constants of each face-connected component of the
domain, Sec. "Jacobi Method" and the zero-mean reference potential) is
left out: the interval is [smallest nonzero, largest] eigenvalue.
"""
from __future__ import annotations

import numpy as np

DENSE_MAX = 2500   # domain voxels up to which the operator is assembled densely


def _restricted(g, sL, sT):
    """Coupled domain voxels (nonzero diagonal), their diagonal, and the
    component label of each."""
    dom = np.nonzero(g.domain())[0]
    d = g.diag_L(sL, sT)[dom]
    keep = d > 0
    idx = dom[keep]
    nc, comp = g.components()
    return idx, d[keep], comp[idx]


def interval(g, sL, sT):
    """(smallest nonzero, largest) eigenvalue of D^-1 A for the oracle grid g
    (oracle.Grid; its torso, if any, is part of the domain) with the elliptic
    conductivities sL, sT."""
    idx, d, comp = _restricted(g, sL, sT)
    m = len(idx)
    s = 1.0 / np.sqrt(d)

    def apply_b(y):
        u = np.zeros(g.n)
        u[idx] = s * y
        return s * g.apply_L(sL, sT, u)[idx]

    # null space of B = D^-1/2 A D^-1/2: D^1/2 times the constants of each component
    labels = np.unique(comp)
    Z = np.zeros((m, len(labels)))
    for j, c in enumerate(labels):
        sel = comp == c
        z = np.sqrt(d) * sel
        Z[:, j] = z / np.linalg.norm(z)
    if m <= DENSE_MAX:
        B = np.zeros((m, m))
        for col in range(m):
            e = np.zeros(m)
            e[col] = 1.0
            B[:, col] = apply_b(e)
        lam = np.linalg.eigvalsh(0.5 * (B + B.T))
        tol = 1e-9 * lam.max()
        nz = lam[lam > tol]
        # the component constants give exactly one zero each
        assert len(lam) - len(nz) == len(labels), (len(lam) - len(nz), len(labels))
        return float(nz.min()), float(lam.max())
    # larger domains: the operator assembled sparsely by probing (the stencil
    # reaches one voxel in each axis, so the 27 classes (i mod 3, j mod 3,
    # k mod 3) each meet every voxel's 3x3x3 neighbourhood once), then the
    # largest eigenvalue by Lanczos and the smallest nonzero one by
    # shift-invert just below 0: the component constants (one zero each) come
    # first, the next is the smallest nonzero eigenvalue
    import scipy.sparse as sp
    from scipy.sparse.linalg import eigsh

    nx, ny, nz = g.nx, g.ny, g.nz
    q = idx
    qi, qj, qk = q % nx, (q // nx) % ny, q // (nx * ny)
    pos = -np.ones(g.n, np.int64)
    pos[idx] = np.arange(m)
    ii = np.arange(g.n) % nx
    jj = (np.arange(g.n) // nx) % ny
    kk = np.arange(g.n) // (nx * ny)
    rows, cols, vals = [], [], []
    for cz in range(3):
        for cy in range(3):
            for cx in range(3):
                u = np.ascontiguousarray(((ii % 3 == cx) & (jj % 3 == cy) & (kk % 3 == cz)).astype(np.float64))
                Lu = g.apply_L(sL, sT, u)[idx]
                # the probed voxel of this class within one voxel of each row voxel
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
    Ds = sp.diags(s)
    B = (Ds @ A @ Ds).tocsc()
    B = (0.5 * (B + B.T)).tocsc()
    hi = float(eigsh(B, k=1, which="LA", tol=1e-10, return_eigenvectors=False)[0])
    nc = len(labels)
    lam = np.sort(eigsh(B, k=nc + 1, sigma=-1e-6 * hi, which="LM", tol=1e-12, return_eigenvectors=False))
    assert np.all(np.abs(lam[:nc]) < 1e-8 * hi), lam
    return float(lam[nc]), hi


def largest(g, sL, sT):
    """Largest eigenvalue of D^-1 A by the Lanczos method (scipy eigsh) on the
    oracle's operator, for domains too large to assemble."""
    from scipy.sparse.linalg import LinearOperator, eigsh

    idx, d, _ = _restricted(g, sL, sT)
    s = 1.0 / np.sqrt(d)

    def apply_b(y):
        u = np.zeros(g.n)
        u[idx] = s * y
        return s * g.apply_L(sL, sT, u)[idx]

    m = len(idx)
    return float(eigsh(LinearOperator((m, m), matvec=apply_b, dtype=np.float64), k=1, which="LA", tol=1e-8,
                       return_eigenvectors=False)[0])


def chebyshev_params(g, sL, sT):
    """The interval the library's set-up would target, scaled as it scales its
    own estimate (smallest by 0.8, largest by 1.05), from the oracle's spectrum."""
    lo, hi = interval(g, sL, sT)
    return 0.8 * lo, 1.05 * hi
