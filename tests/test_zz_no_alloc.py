"""ep_step_noalloc: the step for callers that cannot allocate device memory
while they advance the model -- code that plans all its device memory up
front (a framework that forbids library allocations after initialisation), a
real-time loop that must not block in an allocator, a service with a fixed
memory budget.  Its scratch lives in one static device array inside the
library.

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


class CountingAllocator:
    """torch's caching allocator behind the library's dev_alloc / dev_free
    hooks, counting the calls."""

    def __init__(self):
        self.alloc, self.free = ep.torch_allocator()
        self.n_alloc = self.n_free = 0

    def pair(self):
        def alloc(nbytes):
            self.n_alloc += 1
            return self.alloc(nbytes)

        def free(ptr):
            self.n_free += 1
            self.free(ptr)

        return alloc, free


@pytest.mark.parametrize("model,solver", [(ep.EP_BI, 0), (ep.EP_MONO, 0), (ep.EP_BI, 1), (ep.EP_BI, 2)])
def test_noalloc_step_matches_step_on_two_calls(model, solver):
    """Two consecutive calls of the no-allocation step give the state that two
    calls of ep_step give, bit for bit (the same kernels in the same order;
    ep_step only queues its sweeps through a CUDA graph), while the handle's
    allocator hook is not called and the device's free memory does not move;
    for the damped-Jacobi, Chebyshev (FP32 correction form, interval estimated
    at set-up) and eight-colour Gauss-Seidel solves."""
    import torch
    case = W.random_case(21, 37, 19, 15, model=model)   # random mask: several components
    case.params.solver = solver
    v, w, ve = W.random_state(21, case)
    counter = CountingAllocator()
    a = ep.sim_from_case(case, allocator=counter.pair())
    b = ep.sim_from_case(case, allocator=counter.pair())
    for s in (a, b):
        s.set_state(v, w, ve, 0)   # set-up (the allocating part) happens here
    for _ in range(2):
        sa = a.step(1, allow_noconv=True)
        torch.cuda.synchronize()
        calls, free0 = counter.n_alloc, torch.cuda.mem_get_info()[0]
        sb = b.step_noalloc(1, allow_noconv=True)
        torch.cuda.synchronize()
        assert counter.n_alloc == calls, "the no-allocation step called the device allocator"
        assert torch.cuda.mem_get_info()[0] == free0, "device free memory changed during the call"
        assert sa.iters == sb.iters and sa.step == sb.step and sa.total_iters == sb.total_iters
        for f in FIELDS:
            np.testing.assert_array_equal(b.read(f), a.read(f))
    a.close()
    b.close()
    assert counter.n_free == counter.n_alloc   # every block the handles took came back


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
