"""Geometry encoder on the GPU (Sec. "Geometry": "Primitives", "Encoding";
Sec. "Fibre Directions") against the oracle: voxel kinds, tissue mask and
vertex classes bit for bit (both take every inside/outside decision with the
same FP32 operations), fibres to FP32 rounding; then a bidomain-free
monodomain run on the encoded schematic heart, fast fibre included, against
the oracle's step."""
import math

import numpy as np
import pytest

import oracle
import paper_2302_12519_gb300 as ep
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_12519_gb300 import build
    build.build()
    ep.load()
    oracle.build()


def _both(sc):
    g = ep.sdf_encode(sc.nodes, sc.regions, sc.nx, sc.ny, sc.nz, sc.dx, sc.origin, sc.helix_rad)
    o = oracle.sdf_encode(sc.nodes, sc.regions, sc.nx, sc.ny, sc.nz, sc.dx, sc.origin, sc.helix_rad)
    return g, o


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_random_scenes_match_oracle_bit_for_bit(seed):
    sc = W.random_scene(seed, n=26, size_mm=24.0)
    g, o = _both(sc)
    np.testing.assert_array_equal(g["label"], o["label"])
    np.testing.assert_array_equal(g["mask"], o["mask"])
    np.testing.assert_array_equal(g["vertices"], o["vertices"])
    assert g["n_tissue"] == o["n_tissue"] == int(o["mask"].sum())
    np.testing.assert_allclose(g["fibres"], o["fibres"], rtol=0, atol=2e-6)


def test_schematic_heart_matches_oracle():
    sc = W.schematic_heart(96)
    g, o = _both(sc)
    for k in ("label", "mask", "vertices"):
        np.testing.assert_array_equal(g[k], o[k])
    assert g["n_tissue"] == o["n_tissue"] > 1000
    kinds = np.bincount(g["label"], minlength=4)
    assert kinds[W.REGION_MYOCARDIUM] > 0 and kinds[W.REGION_FAST] > 0 and kinds[W.REGION_INSULATOR] > 0
    np.testing.assert_allclose(g["fibres"], o["fibres"], rtol=0, atol=2e-6)


def test_monodomain_on_the_encoded_heart_matches_oracle():
    """The GPU-encoded heart (fast fibre longer than 1 included) drives a
    monodomain run; the oracle steps the same geometry (the encoder's FP64
    fibres; the library takes their float32 values): V_m within 0.5 mV after
    60 steps."""
    sc = W.schematic_heart(48)
    g = ep.sdf_encode(sc.nodes, sc.regions, sc.nx, sc.ny, sc.nz, sc.dx, sc.origin, sc.helix_rad)
    n = sc.nx
    mask = g["mask"].reshape(n, n, n)
    fib = g["fibres"].reshape(n, n, n, 3)
    p = W.Params(dt=0.02, sig_iL=0.2, sig_iT=0.05, sig_eL=0.2, sig_eT=0.05)
    idx = np.argwhere(mask)                      # stimulate the topmost tissue (the atria)
    top = idx[idx[:, 0] >= idx[:, 0].max() - 2]
    k0, j0, i0 = top[0]
    st = W.Stimulus((int(i0) - 2, int(j0) - 2, int(k0) - 2), (int(i0) + 3, int(j0) + 3, int(k0) + 3), 0.0, 1.0, 0.5)
    c = W.Case("heart48", n, n, n, sc.dx, mask.astype(np.uint8), fib, p, [st], model=W.MONO, steps=60)
    s = ep.sim_from_case(c)
    o = oracle.Sim(c)
    s.step(c.steps)
    o.run(c.steps)
    st_o = o.state()
    assert np.abs(s.read(ep.EP_VM_MV) - oracle.vm_mV(st_o["v"])).max() <= 0.5
    assert (st_o["v"] > 0.5).sum() > 10


def test_schematic_heart_fullsize_bit_for_bit():
    """The schematic heart at 256^3 (the bench encodes 512^3 with the same
    kernels and launch shape): every voxel's kind and every vertex class equal
    the oracle's."""
    sc = W.schematic_heart(256)
    g, o = _both(sc)
    for k in ("label", "mask", "vertices"):
        np.testing.assert_array_equal(g[k], o[k])
    assert g["n_tissue"] == o["n_tissue"]
