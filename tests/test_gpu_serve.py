"""Served form: requests released over time join a running batch (continuous
batching) under a device-memory budget.  Every request's result must be the
same as its handle stepped alone, whatever else shared the device with it."""
import ctypes
import time

import numpy as np
import pytest

import paper_2302_12519_gb300 as ep
import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = (ep.EP_V, ep.EP_W, ep.EP_VE, ep.EP_TACT)
STEPS = [5, 3, 7, 4, 6, 2, 5]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_12519_gb300 import build
    build.build()
    ep.load()


def _cases():
    rng = np.random.default_rng(11)
    cases = [W.sampled_shell(rng, n, 10, f"s{n}") for n in (24, 28, 36)]
    cases += [W.random_case(60 + i, 29 + 5 * i, 19 + 2 * i, 11 + i, model=W.BI) for i in range(3)]
    cases.append(W.random_case(70, 26, 21, 13, model=W.MONO))   # served beside the bidomain ones
    return cases


def _prepare(case, i):
    s = ep.sim_from_case(case, use_torch=False)
    if i % 2:   # odd requests arrive mid-run with a state; even ones start at rest, set up by the server
        v, w, ve = W.random_state(200 + i, case)
        s.set_state(v, w, ve, 2)
    return s


def test_each_request_same_alone_and_served():
    cases = _cases()
    alone = []
    for i, c in enumerate(cases):
        s = _prepare(c, i)
        s.step(STEPS[i], allow_noconv=True)
        alone.append({f: s.read(f) for f in FIELDS})
        s.close()
    srv = ep.Server(max_slots=3, chunk_steps=2)
    ids = [srv.submit(_prepare(c, i), STEPS[i], release_s=0.03 * i) for i, c in enumerate(cases)]
    srv.drain(timeout_s=300)
    got = srv.collect(max_results=32)   # no budget: nothing waits on results
    assert sorted(r.id for r, _ in got) == sorted(ids)
    for r, sim in got:
        i = ids.index(r.id)
        assert r.status in (ep.EP_OK, ep.EP_ENOCONV), r.status
        assert r.steps_done == STEPS[i]
        assert r.t_release_s <= r.t_admit_s <= r.t_done_s
        assert r.n_tissue == int(cases[i].mask.sum())
        for f in FIELDS:
            np.testing.assert_array_equal(sim.read(f), alone[i][f], err_msg=f"request {i} field {f}")
        sim.close()
    st = srv.stats()
    assert st.completed == len(cases) and st.queued == 0 and st.active == 0 and st.finished == 0
    assert st.hbm_in_use == 0
    assert st.voxel_steps == sum(STEPS[i] * int(c.mask.sum()) for i, c in enumerate(cases))
    srv.close()


def test_budget_admission_and_rejection():
    cases = _cases()[:4]
    sims = [_prepare(c, 2 * i) for i, c in enumerate(cases)]   # all fresh: set up by the server
    peaks = [s.footprint()[1] for s in sims]
    budget = int(max(peaks) * 1.2)   # about one request at a time
    big = ep.sim_from_case(W.random_case(90, 72, 70, 66, model=W.BI), use_torch=False)
    assert big.footprint()[1] > budget
    srv = ep.Server(max_slots=4, chunk_steps=3, hbm_budget_bytes=budget)
    ids = [srv.submit(s, 4) for s in sims]
    big_id = srv.submit(big, 2)
    # results hold their memory until collected: drain reports the wait instead of hanging
    with pytest.raises(ep.EPError) as e:
        srv.drain(timeout_s=300)
    assert e.value.status == ep.EP_EBUSY and "uncollected" in str(e.value)
    got = {r.id: (r, s) for r, s in srv.collect_n(len(ids) + 1, timeout_s=300)}
    assert got[big_id][0].status == ep.EP_EREJECTED and got[big_id][0].t_admit_s < 0
    for i in ids:
        r, s = got[i]
        assert r.status in (ep.EP_OK, ep.EP_ENOCONV) and r.steps_done == 4
        res, peak = s.footprint()
        assert r.device_bytes == res == s.info().device_bytes
    st = srv.stats()
    assert 0 < st.hbm_peak <= budget
    assert st.rejected == 1 and st.completed == len(ids)
    for r, s in got.values():
        s.close()
    srv.close()


def test_cancel_queued_and_running():
    c = _cases()[0]
    srv = ep.Server(max_slots=2, chunk_steps=1)
    late = srv.submit(_prepare(c, 0), 3, release_s=srv.now() + 1000.0)
    srv.cancel(late)
    long_id = srv.submit(_prepare(c, 1), 100000)
    t0 = time.time()
    while srv.stats().admitted < 1 and time.time() - t0 < 60:
        time.sleep(0.01)
    time.sleep(0.2)
    srv.cancel(long_id)
    srv.drain(timeout_s=120)
    got = {r.id: r for r, s in srv.collect(max_results=8)}
    assert got[late].status == ep.EP_ECANCELLED and got[late].steps_done == 0 and got[late].t_admit_s < 0
    assert got[long_id].status == ep.EP_ECANCELLED and 0 < got[long_id].steps_done < 100000
    with pytest.raises(ep.EPError) as e:
        srv.cancel(long_id)   # already finished
    assert e.value.status == ep.EP_EINVAL
    assert srv.stats().cancelled == 2
    srv.close()


def test_submit_validation():
    c = _cases()[0]
    srv = ep.Server(max_slots=2)
    s64 = ep.sim_from_case(c, use_torch=False, precision=W.FP64)
    with pytest.raises(ep.EPError) as e:
        srv.submit(s64, 2)
    assert e.value.status == ep.EP_EINVAL
    s = _prepare(c, 0)
    rid = srv.submit(s, 1, release_s=srv.now() + 1000.0)
    again = ctypes.c_longlong()
    st = srv._L.ep_server_submit(srv._h, srv._held[rid][1], 1, 0.0, ctypes.byref(again))
    assert st == ep.EP_EINVAL and "already held" in srv._L.ep_server_last_error(srv._h).decode()
    with pytest.raises(ValueError):
        srv.submit(ep.sim_from_case(c, use_torch=True), 1)
    srv.close()   # destroys the handle it still holds
    s64.close()
