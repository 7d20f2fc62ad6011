"""Batched form: uneven instances advanced together in one persistent launch
per kernel, whole steps in one CUDA graph with device-side loops.  Every
instance's result must be the same alone and in the mix."""
import numpy as np
import pytest

import paper_2302_12519_gb300 as ep
import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = (ep.EP_V, ep.EP_W, ep.EP_VE, ep.EP_TACT)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_12519_gb300 import build
    build.build()
    ep.load()


def _cases(model=W.BI):
    rng = np.random.default_rng(5)
    cases = [W.sampled_shell(rng, n, 10, f"s{n}") for n in (24, 31, 40)]
    cases += [W.random_case(40 + i, 33 + 7 * i, 17 + 3 * i, 12 + i, model=model) for i in range(3)]
    for c in cases:
        c.model = model
    return cases


def _handles(cases, seed0=100):
    out = []
    for i, c in enumerate(cases):
        s = ep.sim_from_case(c)
        v, w, ve = W.random_state(seed0 + i, c)
        s.set_state(v, w, ve, 3)
        out.append(s)
    return out


@pytest.mark.parametrize("model", [W.BI, W.MONO])
def test_each_instance_same_alone_and_in_the_mix(model):
    cases = _cases(model)
    alone = _handles(cases)
    for s in alone:
        s.step(4, allow_noconv=True)
    mixed = _handles(cases)
    b = ep.Batch(len(cases) + 2)
    slots = [b.add(s) for s in mixed]
    b.step(2, allow_noconv=True)
    b.step(2, allow_noconv=True)   # two graph launches: the chunk boundary is seamless
    for s_alone, s_mix, slot in zip(alone, mixed, slots):
        st = b.slot_stats(slot)
        assert st.step == 7
        for f in FIELDS:
            np.testing.assert_array_equal(s_mix.read(f), s_alone.read(f))
    b.close()


def test_packed_and_solo_members_same_alone_and_in_the_mix():
    """Ten members: above eight, small members sweep through the packed kernel
    while the two large ones sweep in their own launches; all match their
    standalone runs bit for bit."""
    rng = np.random.default_rng(9)
    cases = [W.random_case(80 + i, 17 + 3 * i, 13 + i, 9 + (i % 4), model=W.BI) for i in range(8)]
    cases += [W.sampled_shell(rng, n, 10, f"big{n}") for n in (176, 184)]
    for c in cases:
        c.model = W.BI
    alone = _handles(cases, seed0=300)
    for s in alone:
        s.step(3, allow_noconv=True)
    mixed = _handles(cases, seed0=300)
    b = ep.Batch(len(cases))
    slots = [b.add(s) for s in mixed]
    info = b.info()
    assert 1 <= info.solo_members < len(cases)
    b.step(3, allow_noconv=True)
    for s_alone, s_mix, slot in zip(alone, mixed, slots):
        assert b.slot_stats(slot).step == 6
        for f in FIELDS:
            np.testing.assert_array_equal(s_mix.read(f), s_alone.read(f))
    b.close()


def test_admission_budget_and_capacity():
    cases = _cases()[:3]
    hs = _handles(cases)
    for h in hs:
        h.info()   # set-up, so the device footprint is known
    need = sum(h.info().device_bytes for h in hs[:2])
    b = ep.Batch(2, hbm_budget_bytes=need + 1)
    b.add(hs[0])
    b.add(hs[1])
    with pytest.raises(ep.EPError) as e:
        b.add(hs[2])
    assert e.value.status in (ep.EP_EBUSY, ep.EP_EREJECTED)
    b.close()
    b = ep.Batch(8, hbm_budget_bytes=hs[0].info().device_bytes + 16)
    b.add(hs[0])
    with pytest.raises(ep.EPError) as e:
        b.add(hs[1])
    assert e.value.status == ep.EP_EREJECTED
    b.remove(0)
    b.add(hs[0])   # room again after removal
    b.close()


def test_autotune_keeps_results_within_tolerance():
    cases = _cases()[:4]
    alone = _handles(cases, 300)
    for s in alone:
        s.step(3, allow_noconv=True)
    mixed = _handles(cases, 300)
    b = ep.Batch(4)
    for s in mixed:
        b.add(s)
    b.autotune(5)
    info = b.info()
    assert info.zseg in (8, 16, 32) and 8 <= info.sweeps_per_check <= 64
    b.step(3, allow_noconv=True)
    for s_alone, s_mix in zip(alone, mixed):
        # a different segment length changes only the order of the FP32 residual partial sums
        np.testing.assert_allclose(s_mix.read(ep.EP_VM_MV), s_alone.read(ep.EP_VM_MV), rtol=0, atol=0.5)
        np.testing.assert_allclose(s_mix.read(ep.EP_W), s_alone.read(ep.EP_W), rtol=0, atol=1e-4)
    b.close()


def test_mixed_solvers_same_alone_and_in_the_mix():
    """Damped-Jacobi and Chebyshev members in one batch: the table keeps each
    group to one solver (its own sweep kernel instance), interleaved slots
    included, and every member matches its standalone run bit for bit."""
    cases = _cases(W.BI)
    for i, c in enumerate(cases):
        c.params.solver = 1 if i % 2 else 0
    alone = _handles(cases, seed0=500)
    for s in alone:
        s.step(3, allow_noconv=True)
    mixed = _handles(cases, seed0=500)
    b = ep.Batch(len(cases))
    slots = [b.add(s) for s in mixed]
    assert b.info().groups >= 2
    b.step(3, allow_noconv=True)
    for s_alone, s_mix, slot in zip(alone, mixed, slots):
        assert b.slot_stats(slot).step == 6
        for f in FIELDS:
            np.testing.assert_array_equal(s_mix.read(f), s_alone.read(f))
    b.close()


@pytest.mark.parametrize("solver", [0, 1])
def test_capped_solves_same_alone_and_in_the_mix(solver):
    """Every solve hits its sweep cap (max_iter 7, rel_tol 0): the cap is met
    at the start of a launch, while other work items of the same member may be
    starting, so the finished flag must be read once per CTA (packed members
    copy their descriptor with the whole CTA).  Ten members (eight packed, two
    solo), twelve steps in one graph launch: every member equals its
    standalone run bit for bit, and every step reports the cap."""
    rng = np.random.default_rng(11)
    cases = [W.random_case(90 + i, 17 + 3 * i, 13 + i, 9 + (i % 4), model=W.BI) for i in range(8)]
    cases += [W.sampled_shell(rng, n, 10, f"cap{n}") for n in (176, 184)]
    for c in cases:
        c.model = W.BI
        c.params.solver, c.params.max_iter, c.params.rel_tol, c.params.check_every = solver, 7, 0.0, 3
    alone = _handles(cases, seed0=700)
    for s in alone:
        st = s.step(12, allow_noconv=True)
        assert st.converged == 0 and st.iters == 7
    mixed = _handles(cases, seed0=700)
    b = ep.Batch(len(cases))
    slots = [b.add(s) for s in mixed]
    assert 1 <= b.info().solo_members < len(cases)
    with pytest.raises(ep.EPError) as e:   # the cap reached: EP_ENOCONV unless allowed
        b.step(1)
    assert e.value.status == ep.EP_ENOCONV
    b.step(11, allow_noconv=True)
    for s_alone, s_mix, slot in zip(alone, mixed, slots):
        st = b.slot_stats(slot)
        assert st.step == 15 and st.iters == 7 and st.converged == 0
        for f in FIELDS:
            np.testing.assert_array_equal(s_mix.read(f), s_alone.read(f))
    b.close()
