"""Pins of the oracle's geometry encoder (Sec. "Geometry": "Signed Distance
Function", "Primitives", "Encoding"; Sec. "Fibre Directions"): primitive
values at points where the definitions give exact numbers, the set algebra
as voxel-count identities, volumes against the analytic ones, the vertex
classes of shapes whose counts are known in closed form, and the fibre rule's
geometry."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _val(op, a, b, c, x, centre=(0.0, 0.0, 0.0), rot=W.IDENTITY9):
    return oracle.sdf_eval([W.SdfNode(op, a, b, c, centre, rot)], x)


def test_primitive_values_at_exact_points():
    # ellipsoid |p/r| - 1: centre -1, twice a semi-axis out +1, on the surface 0
    assert _val(W.SDF_ELLIPSOID, 2.0, 4.0, 8.0, (1.0, 2.0, 3.0), centre=(1.0, 2.0, 3.0)) == -1.0
    assert _val(W.SDF_ELLIPSOID, 2.0, 4.0, 8.0, (0.0, 8.0, 0.0)) == 1.0
    assert _val(W.SDF_ELLIPSOID, 2.0, 4.0, 8.0, (0.0, 0.0, -8.0)) == 0.0
    # cuboid max_i |p_i / r_i| - 1
    assert _val(W.SDF_CUBOID, 2.0, 4.0, 8.0, (4.0, -12.0, 0.0)) == 2.0
    assert _val(W.SDF_CUBOID, 2.0, 4.0, 8.0, (1.0, 2.0, 4.0)) == -0.5
    # cylinder max(|p_xy| - r, |p_z| - h)
    assert _val(W.SDF_CYLINDER, 3.0, 5.0, 0.0, (3.0, 4.0, 0.0)) == 2.0
    assert _val(W.SDF_CYLINDER, 3.0, 5.0, 0.0, (0.0, 0.0, -7.0)) == 2.0
    # cone max(|p_xy| - slope z - r, |p_z| - h): radius r + slope z at height z
    assert _val(W.SDF_CONE, 2.0, 10.0, 0.5, (6.0, 0.0, 8.0)) == 0.0
    assert _val(W.SDF_CONE, 2.0, 10.0, 0.5, (0.0, 0.0, 12.0)) == 2.0
    # a rotation by 90 degrees about z swaps the x and y half-extents
    R = (0.0, 1.0, 0.0, -1.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    assert _val(W.SDF_CUBOID, 1.0, 4.0, 1.0, (0.0, 3.0, 0.0), rot=R) == 2.0
    assert _val(W.SDF_CUBOID, 1.0, 4.0, 1.0, (3.0, 0.0, 0.0), rot=R) == -0.25


def test_operators_closed_forms():
    A = W.SdfNode(W.SDF_ELLIPSOID, 4.0, 4.0, 4.0)            # value at (8,0,0): 1
    B = W.SdfNode(W.SDF_CUBOID, 2.0, 2.0, 2.0)               # value at (8,0,0): 3
    x = (8.0, 0.0, 0.0)
    assert oracle.sdf_eval([A, B, W.SdfNode(W.SDF_UNION)], x) == 1.0
    assert oracle.sdf_eval([A, B, W.SdfNode(W.SDF_INTERSECT)], x) == 3.0
    assert oracle.sdf_eval([A, B, W.SdfNode(W.SDF_SUBTRACT)], x) == 1.0     # max(1, -3)
    assert oracle.sdf_eval([B, A, W.SdfNode(W.SDF_SUBTRACT)], x) == 3.0     # max(3, -1)
    assert oracle.sdf_eval([A, W.SdfNode(W.SDF_HOLLOW, 0.25)], x) == 0.75
    assert oracle.sdf_eval([A, W.SdfNode(W.SDF_HOLLOW, 0.25)], (0.0, 0.0, 0.0)) == 0.75   # |-1| - 0.25
    # smoothed minimum: plain min when the operands differ by at least k, min - k/4 when equal
    assert oracle.sdf_eval([A, B, W.SdfNode(W.SDF_SMOOTH_UNION, 2.0)], x) == 1.0
    C = W.SdfNode(W.SDF_ELLIPSOID, 4.0, 4.0, 4.0, (16.0, 0.0, 0.0))       # value at (8,0,0): 1
    assert oracle.sdf_eval([A, C, W.SdfNode(W.SDF_SMOOTH_UNION, 2.0)], x) == 0.5


def _encode(nodes, regions, n, dx=1.0, origin=None, helix=0.4 * math.pi):
    origin = origin if origin is not None else (-n * dx / 2,) * 3
    return oracle.sdf_encode(nodes, regions, n, n, n, dx, origin, helix)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_set_algebra_as_voxel_counts(seed):
    """Inclusion-exclusion holds exactly for the encoded sets:
    |A u B| + |A n B| = |A| + |B| and |A minus B| = |A| - |A n B|."""
    sc = W.random_scene(seed, n=20, size_mm=20.0)
    a, b = sc.nodes[0], sc.nodes[1]
    def count(prog):
        r = _encode(prog, [W.SdfRegion(0, len(prog), W.REGION_MYOCARDIUM)], 20)
        return r["n_tissue"]
    nA, nB = count([a]), count([b])
    nU = count([a, b, W.SdfNode(W.SDF_UNION)])
    nI = count([a, b, W.SdfNode(W.SDF_INTERSECT)])
    nD = count([a, b, W.SdfNode(W.SDF_SUBTRACT)])
    assert nU + nI == nA + nB and nD == nA - nI
    assert nA > 0 and nB > 0


def test_volumes_converge_to_the_analytic_ones():
    """An ellipsoid's voxel volume approaches 4/3 pi abc; the error is bounded
    by a surface layer of one voxel diagonal (rounded up to the area bound of
    the circumscribed box); a grid-aligned cuboid is exact."""
    a, b, c = 9.3, 6.1, 7.7
    V = 4.0 / 3.0 * math.pi * a * b * c
    errs = []
    for n, dx in ((24, 1.0), (48, 0.5), (96, 0.25)):
        r = _encode([W.SdfNode(W.SDF_ELLIPSOID, a, b, c)], [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)], n, dx)
        err = abs(r["n_tissue"] * dx ** 3 - V)
        errs.append(err)
        assert err <= 2 * (a * b + b * c + a * c) * 4 * math.sqrt(3) * dx
    assert errs[2] < errs[0]
    r = _encode([W.SdfNode(W.SDF_CUBOID, 5.25, 3.75, 2.25)], [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)], 16)
    assert r["n_tissue"] == 10 * 8 * 4   # centres at +-0.5 .. +-4.5 (x), +-3.5 (y), +-1.5 (z)


def test_vertex_classes_closed_forms():
    """Sec. "Encoding": a k^3 block of tissue inside the grid has (k-1)^3
    solid vertices and (k+1)^3 - (k-1)^3 surface vertices; one voxel has 8
    surface vertices; an all-tissue grid has only solid vertices (only voxels
    inside the grid count)."""
    n = 12
    for k in (1, 3, 5):
        h = k / 2.0 - 0.25   # half-extent that holds k voxel centres
        r = _encode([W.SdfNode(W.SDF_CUBOID, h, h, h, (0.5 if k % 2 else 0.0,) * 3)],
                    [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)], n)
        assert r["n_tissue"] == k ** 3
        cls = np.bincount(r["vertices"], minlength=3)
        assert cls[1] == (k - 1) ** 3 and cls[2] == (k + 1) ** 3 - (k - 1) ** 3
        assert cls[0] == (n + 1) ** 3 - (k + 1) ** 3
    r = _encode([W.SdfNode(W.SDF_CUBOID, 50.0, 50.0, 50.0)], [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)], 6)
    assert np.all(r["vertices"] == 1) and r["n_tissue"] == 216


def test_fibre_rule_geometry():
    """Sec. "Fibre Directions": unit fibres orthogonal to the position vector;
    elevation above the horizontal = helix * |p_xy| / |p| in sine form, i.e.
    the helix angle itself on the equator; helix 0 gives the horizontal
    circumferential direction; fast-fibre voxels carry scale * axis, and the
    scale of a gain g makes the longitudinal conductivity g sigma_L (Eq. sigma1)."""
    n, helix = 16, 0.4 * math.pi
    node = [W.SdfNode(W.SDF_ELLIPSOID, 7.0, 7.0, 7.0)]
    r = _encode(node, [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)], n, 1.0, helix=helix)
    f = r["fibres"].reshape(-1, 3)
    idx = np.nonzero(r["mask"])[0]
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)
    p = np.stack([i + 0.5 - n / 2, j + 0.5 - n / 2, k + 0.5 - n / 2], 1)
    fi = f[idx]
    np.testing.assert_allclose(np.linalg.norm(fi, axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose((fi * p).sum(1), 0.0, atol=1e-12)
    sin_el = math.sin(helix) * np.linalg.norm(p[:, :2], axis=1) / np.linalg.norm(p, axis=1)
    np.testing.assert_allclose(fi[:, 2], sin_el, atol=1e-12)
    r0 = _encode(node, [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM)], n, 1.0, helix=0.0)
    f0 = r0["fibres"].reshape(-1, 3)[idx]
    h = np.stack([-p[:, 1], p[:, 0], np.zeros(len(p))], 1) / np.linalg.norm(p[:, :2], axis=1)[:, None]
    np.testing.assert_allclose(f0, h, atol=1e-12)
    # fast fibre
    sL, sT, g = 0.2, 0.05, 2.0
    scale = math.sqrt((g * sL - sT) / (sL - sT))
    rf = _encode(node, [W.SdfRegion(0, 1, W.REGION_FAST, (0.0, 0.6, 0.8), scale)], n, 1.0)
    ff = rf["fibres"].reshape(-1, 3)[np.nonzero(rf["mask"])[0]]
    np.testing.assert_allclose(ff, np.broadcast_to(np.array([0.0, 0.6, 0.8]) * scale, ff.shape), atol=1e-6)
    S = sT * np.eye(3) + (sL - sT) * np.outer(ff[0], ff[0])
    assert abs(np.linalg.eigvalsh(S).max() - g * sL) < 1e-5


def test_regions_apply_in_order_and_insulators_are_not_tissue():
    """The last region containing a voxel decides; an insulator after the
    myocardium removes tissue, a fast fibre after it restores tissue."""
    big = W.SdfNode(W.SDF_CUBOID, 5.25, 5.25, 5.25)
    slab = W.SdfNode(W.SDF_CUBOID, 10.0, 10.0, 0.75)
    rod = W.SdfNode(W.SDF_CYLINDER, 1.2, 10.0)
    regs = [W.SdfRegion(0, 1, W.REGION_MYOCARDIUM), W.SdfRegion(1, 1, W.REGION_INSULATOR),
            W.SdfRegion(2, 1, W.REGION_FAST, (0.0, 0.0, 1.0), 1.5)]
    r = _encode([big, slab, rod], regs, 16)
    lab = r["label"].reshape(16, 16, 16)
    assert np.all(lab[7:9, 4:12, 4:12][:, [0, -1], :] == W.REGION_INSULATOR)   # the slab cuts the block
    assert np.all(lab[7:9, 7:9, 7:9] == W.REGION_FAST)                         # the rod pierces the slab
    # block minus the slab's two layers, plus the rod's 2 x 2 columns through the slab and outside the block
    assert r["n_tissue"] == 10 ** 3 - 2 * 10 * 10 + 2 * 4 + (16 - 10) * 4
