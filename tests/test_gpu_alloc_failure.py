"""Allocation failures injected through the context's allocator hook
(kpm_options.alloc_fn): every device buffer of a context comes from the
hook, so a hook that returns NULL is how a full device looks to the
library.  kpm_create must return KPM_ENOMEM and free what it had taken;
a moment call whose work buffers cannot be had must return KPM_ENOMEM and
leave the context usable, giving the same moments once memory is back."""
import ctypes

import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1410_5242_gb300 import build
    build.build()
    from paper_1410_5242_gb300 import kpm as k
    return k


class FailingAllocator:
    """torch's caching allocator behind the hook, refusing every request
    from the `fail_from`-th on (counting from 0) while armed; keeps the
    pointers it handed out so that leaks show."""

    def __init__(self, kpm, fail_from=None):
        import torch
        self.fail_from = fail_from
        self.calls = 0
        self.live = set()

        def alloc(nbytes, user):
            k = self.calls
            self.calls += 1
            if self.fail_from is not None and k >= self.fail_from:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), device=0)
            self.live.add(p)
            return p

        def free(ptr, user):
            if ptr:
                self.live.discard(ptr)
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc = kpm.ALLOC_FN(alloc)
        self.free = kpm.FREE_FN(free)


@pytest.mark.parametrize("prec", [0, 1])
def test_create_fails_cleanly_at_every_allocation(kpm, prec):
    h = ham.ti_hamiltonian(4, 4, 4, gamma=0.5, seed=1)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    probe = FailingAllocator(kpm)
    with kpm.create(h, a, b, precision=prec, allocator=probe):
        pass
    n_allocs = probe.calls
    assert n_allocs >= 5 and not probe.live
    for k in range(n_allocs):
        al = FailingAllocator(kpm, fail_from=k)
        with pytest.raises(kpm.KPMError) as e:
            kpm.create(h, a, b, precision=prec, allocator=al)
        assert e.value.status == kpm.KPM_ENOMEM, k
        assert not al.live, k  # everything taken before the failure was given back


@pytest.mark.parametrize("prec", [0, 1])
def test_moments_fail_cleanly_and_the_context_recovers(kpm, prec):
    h = ham.ti_hamiltonian(4, 4, 5, gamma=0.7, seed=2)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    M, R = 32, 8
    with kpm.create(h, a, b, precision=prec) as ref_ctx:
        want = ref_ctx.moments(M, R, 3)
    al = FailingAllocator(kpm)
    with kpm.create(h, a, b, precision=prec, allocator=al) as ctx:
        al.fail_from = al.calls  # no more device memory from now on
        with pytest.raises(kpm.KPMError) as e:
            ctx.moments(M, R, 3)
        assert e.value.status == kpm.KPM_ENOMEM
        al.fail_from = None
        got = ctx.moments(M, R, 3)
    assert np.array_equal(got, want)
    assert not al.live
