"""ep_step_noalloc: the step variant for callers that cannot allocate device
memory while they run (memory planned up front, real-time loops, fixed
budgets).  Its scratch lives in one static device array inside the library.

This file is named to be collected last, so a run that stops at the first
failure has run every other test before it.  It must pass both on its own in
a fresh process and after the other tests (the static array then holds an
earlier call's contents, which the entry point clears)."""
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


def _pair(case, seed):
    v, w, ve = W.random_state(seed, case)
    a = ep.sim_from_case(case)
    b = ep.sim_from_case(case)
    for s in (a, b):
        s.set_state(v, w, ve, 0)   # set-up (the allocating part) happens here
    return a, b


@pytest.mark.parametrize("model", [ep.EP_BI, ep.EP_MONO])
def test_noalloc_step_matches_step_on_two_calls(model):
    """Two consecutive calls of the no-allocation step give the same state as
    two calls of ep_step, within the FP32 parity tolerance of the other tests
    (the kernels and their order are the same, so they agree to the bit)."""
    case = W.random_case(21, 37, 19, 15, model=model)   # random mask: several components
    a, b = _pair(case, 21)
    for _ in range(2):
        sa = a.step(1, allow_noconv=True)
        sb = b.step_noalloc(1, allow_noconv=True)
        assert sa.iters == sb.iters and sa.step == sb.step
        for f in FIELDS:
            np.testing.assert_allclose(b.read(f), a.read(f), rtol=0, atol=5e-6)
    a.close()
    b.close()


def test_noalloc_step_checks_setup_and_limits():
    """Without set-up the call refuses (set-up allocates); a mask with more
    tissue components than the static array holds is rejected."""
    case = W.random_case(22, 12, 10, 8, model=W.BI)
    s = ep.sim_from_case(case)
    with pytest.raises(ep.EPError) as e:
        s.step_noalloc(1)
    assert e.value.status == ep.EP_ESTATE
    s.close()
    n = 40
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    case = W.random_case(23, n, n, n, model=W.BI, mask=((i + j + k) % 2 == 0).astype(np.uint8))
    s = ep.sim_from_case(case)
    assert s.info().n_components > 4096
    with pytest.raises(ep.EPError) as e:
        s.step_noalloc(1)
    assert e.value.status == ep.EP_EINVAL and "4096" in str(e.value)
    s.close()
