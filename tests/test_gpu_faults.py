"""Failure detection on the CUDA path, with every failure made on the host:
a non-finite value written into the state, an unstable time step, a device
allocator that refuses memory, and a non-finite member of the batched and
served forms.  None of these faults, traps or hangs the GPU: the library's
kernels raise a device flag that the host reads after the step, and the
allocator hook returns NULL as a failing cudaMalloc would."""
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


def _nan_state(case, seed):
    v, w, ve = W.random_state(seed, case)
    q = int(np.nonzero(case.mask.reshape(-1))[0][len(v) // 7 % int(case.mask.sum())])
    v = v.copy()
    v[q] = np.nan
    return v, w, ve


@pytest.mark.parametrize("model", [W.MONO, W.BI])
def test_nan_in_the_state_is_reported_and_the_handle_recovers(model):
    c = W.random_case(81, 23, 14, 11, model=model)
    s = ep.sim_from_case(c)
    v, w, ve = _nan_state(c, 81)
    s.set_state(v, w, ve, 0)
    with pytest.raises(ep.EPError) as e:
        s.step(1)
    assert e.value.status == ep.EP_ENONFINITE
    # a clean state makes the handle usable again
    v, w, ve = W.random_state(81, c)
    s.set_state(v, w, ve, 0)
    stats = s.step(2, allow_noconv=True)
    assert s.last_status in (ep.EP_OK, ep.EP_ENOCONV) and stats.step == 2
    assert np.all(np.isfinite(s.read(ep.EP_V)))
    s.close()


def test_unstable_time_step_is_reported():
    """Explicit diffusion far above its stability bound (dt < 2 K dx^2 / (4 f sig_L),
    1.25 ms here; dt = 6 ms): the state overflows and the step says so."""
    c = W.random_case(82, 20, 12, 10, model=W.MONO, dt=6.0)
    s = ep.sim_from_case(c)
    v, w, ve = W.random_state(82, c)
    s.set_state(v, w, ve, 0)
    status = ep.EP_OK
    for _ in range(400):
        try:
            s.step(1)
        except ep.EPError as e:
            status = e.status
            break
    assert status == ep.EP_ENONFINITE
    s.close()


class FailingAllocator:
    """torch's caching allocator behind the dev_alloc / dev_free hooks that
    returns NULL from the fail_at-th request on (0: never), counting calls and
    the blocks it handed out."""

    def __init__(self, fail_at=0):
        self.alloc, self.free = ep.torch_allocator()
        self.fail_at = fail_at
        self.calls = 0
        self.live = set()

    def pair(self):
        def alloc(nbytes):
            self.calls += 1
            if self.fail_at and self.calls >= self.fail_at:
                return 0
            p = self.alloc(nbytes)
            self.live.add(p)
            return p

        def free(ptr):
            self.live.discard(ptr)
            self.free(ptr)

        return alloc, free


def test_failing_allocator_gives_enomem_without_a_leak():
    """The set-up's allocations fail at the first, a middle and the last
    request: the call returns EP_ENOMEM, every block already taken is given
    back, and a new handle with a working allocator runs."""
    import torch
    c = W.random_case(83, 21, 13, 12, model=W.BI)
    ok = FailingAllocator()
    s = ep.sim_from_case(c, allocator=ok.pair())
    s.info()   # set-up
    n_setup = ok.calls
    s.close()
    assert n_setup >= 10 and not ok.live
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    for k in sorted({1, n_setup // 2, n_setup}):
        bad = FailingAllocator(fail_at=k)
        s = ep.sim_from_case(c, allocator=bad.pair())
        with pytest.raises(ep.EPError) as e:
            s.step(1)
        assert e.value.status == ep.EP_ENOMEM, (k, e.value)
        assert not bad.live, f"failing at request {k}: {len(bad.live)} blocks not given back"
        s.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    s = ep.sim_from_case(c, allocator=FailingAllocator().pair())
    assert s.step(1, allow_noconv=True).step == 1
    s.close()


def test_batch_reports_a_nonfinite_member_and_the_others_are_unaffected():
    good = W.random_case(84, 26, 15, 12, model=W.BI)
    bad = W.random_case(85, 22, 17, 10, model=W.BI)
    alone = ep.sim_from_case(good)
    v, w, ve = W.random_state(84, good)
    alone.set_state(v, w, ve, 0)
    alone.step(3, allow_noconv=True)
    ref = {f: alone.read(f) for f in FIELDS}
    g = ep.sim_from_case(good)
    g.set_state(v, w, ve, 0)
    b_ = ep.sim_from_case(bad)
    b_.set_state(*_nan_state(bad, 85), 0)
    batch = ep.Batch(2)
    sg, sb = batch.add(g), batch.add(b_)
    with pytest.raises(ep.EPError) as e:
        batch.step(3)
    assert e.value.status == ep.EP_ENONFINITE
    for f in FIELDS:
        np.testing.assert_array_equal(g.read(f), ref[f])
    assert batch.slot_stats(sg).step == 3
    batch.close()


def test_server_retires_a_nonfinite_request_and_finishes_the_others():
    good = W.random_case(86, 24, 16, 12, model=W.BI)
    bad = W.random_case(87, 20, 18, 11, model=W.BI)
    v, w, ve = W.random_state(86, good)
    alone = ep.sim_from_case(good, use_torch=False)
    alone.set_state(v, w, ve, 0)
    alone.step(6, allow_noconv=True)
    ref = {f: alone.read(f) for f in FIELDS}
    alone.close()
    srv = ep.Server(max_slots=2, chunk_steps=2)
    sg = ep.sim_from_case(good, use_torch=False)
    sg.set_state(v, w, ve, 0)
    sb = ep.sim_from_case(bad, use_torch=False)
    sb.set_state(*_nan_state(bad, 87), 0)
    ig = srv.submit(sg, 6)
    ib = srv.submit(sb, 6)
    srv.drain(timeout_s=120)
    res = {r.id: (r, sim) for r, sim in srv.collect(max_results=4)}
    rb, _ = res[ib]
    assert rb.status == ep.EP_ENONFINITE and rb.steps_done < 6
    rg, simg = res[ig]
    assert rg.status in (ep.EP_OK, ep.EP_ENOCONV) and rg.steps_done == 6
    for f in FIELDS:
        np.testing.assert_array_equal(simg.read(f), ref[f])
    for _, sim in res.values():
        sim.close()
    srv.close()
