"""The allocation-free sweep kpm_aug_spmmv_static against kpm_aug_spmmv.

kpm_aug_spmmv_static exists for callers that may not allocate device
memory when they call into the library: code whose device memory belongs to
another allocator or pool, and latency-critical loops in which cudaMalloc
would implicitly synchronise the device.  It takes its per-block scratch
from a fixed device array inside the library instead of allocating one.

Each case runs two calls in a row on each path from identical inputs (the
second call continues the recurrence with V and W swapped, so leftover
scratch from the first call would show) and compares W and eta within the
tolerances of the parity tests.  This file sorts last so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham
from kpm_inputs import vectors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1410_5242_gb300 import build
    build.build()
    from paper_1410_5242_gb300 import kpm as k
    return k


def _blocks(ctx, R, V0, W0):
    V, W = ctx.new_block(R), ctx.new_block(R)
    ctx.block_upload(R, V0, V)
    ctx.block_upload(R, W0, W)
    return V, W


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("R", [3, 32, 100, 256])
def test_static_sweep_matches_allocating_sweep_twice(kpm, prec, R):
    import torch
    h = ham.ti_hamiltonian(6, 5, 4, gamma=0.8, seed=2)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    n = h["n"]
    V0 = vectors.random_phase_block(5, n, range(R))
    g = np.random.default_rng(R)
    W0 = g.standard_normal((n, R)) + 1j * g.standard_normal((n, R))
    with kpm.create(h, a, b, precision=prec) as ctx:
        Va, Wa = _blocks(ctx, R, V0, W0)
        Vs, Ws = _blocks(ctx, R, V0, W0)
        eta_a = torch.full((3 * R,), np.nan, dtype=torch.float64, device="cuda")
        eta_s = torch.full((3 * R,), np.nan, dtype=torch.float64, device="cuda")
        for call in range(2):
            ctx.aug_spmmv(R, Va, Wa, eta_a)
            ctx.aug_spmmv_static(R, Vs, Ws, eta_s)
            torch.cuda.synchronize()
            wa, ws = ctx.block_download(R, Wa), ctx.block_download(R, Ws)
            ea, es = eta_a.cpu().numpy(), eta_s.cpu().numpy()
            tol_w, tol_e = (1e-13, 1e-12) if prec == 0 else (2e-6, 2e-6)
            np.testing.assert_allclose(ws, wa, rtol=0, atol=tol_w * np.abs(wa).max())
            np.testing.assert_allclose(es, ea, rtol=0, atol=tol_e * np.abs(ea[:R]).max())
            Va, Wa = Wa, Va   # next step of the recurrence: the new W becomes V
            Vs, Ws = Ws, Vs


@pytest.mark.parametrize("prec", [0, 1])
def test_static_sweep_allocates_nothing_on_a_fresh_context(kpm, prec):
    """On a context that has never run a sweep, two calls of the static
    sweep ask the context's allocator hook for nothing and leave PyTorch's
    allocation count unchanged, and give the allocating sweep's results
    (computed afterwards on a second context)."""
    import torch
    h = ham.ti_hamiltonian(6, 5, 4, gamma=0.8, seed=2)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    n, R = h["n"], 32
    V0 = vectors.random_phase_block(5, n, range(R))
    g = np.random.default_rng(7)
    W0 = g.standard_normal((n, R)) + 1j * g.standard_normal((n, R))
    with kpm.create(h, a, b, precision=prec) as ctx:
        V, W = _blocks(ctx, R, V0, W0)
        eta = torch.zeros(3 * R, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        hook0 = ctx._alloc.calls
        torch0 = torch.cuda.memory_stats()["allocation.all.allocated"]
        ctx.aug_spmmv_static(R, V, W, eta)
        ctx.aug_spmmv_static(R, W, V, eta)
        torch.cuda.synchronize()
        assert ctx._alloc.calls == hook0
        assert torch.cuda.memory_stats()["allocation.all.allocated"] == torch0
        ws, es = ctx.block_download(R, V), eta.cpu().numpy()
    with kpm.create(h, a, b, precision=prec) as ctx:
        V, W = _blocks(ctx, R, V0, W0)
        eta = torch.zeros(3 * R, dtype=torch.float64, device="cuda")
        ctx.aug_spmmv(R, V, W, eta)
        ctx.aug_spmmv(R, W, V, eta)
        torch.cuda.synchronize()
        wa, ea = ctx.block_download(R, V), eta.cpu().numpy()
    tol_w, tol_e = (1e-13, 1e-12) if prec == 0 else (2e-6, 2e-6)
    np.testing.assert_allclose(ws, wa, rtol=0, atol=tol_w * np.abs(wa).max())
    np.testing.assert_allclose(es, ea, rtol=0, atol=tol_e * np.abs(ea[:R]).max())


def test_static_sweep_rejects_too_many_columns(kpm):
    import torch
    h = ham.ti_hamiltonian(3, 3, 3, gamma=0.1, seed=1)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    R = 4096
    with kpm.create(h, a, b) as ctx:
        V, W = ctx.new_block(R), ctx.new_block(R)
        eta = torch.zeros(3 * R, dtype=torch.float64, device="cuda")
        with pytest.raises(kpm.KPMError) as e:
            ctx.aug_spmmv_static(R, V, W, eta)
        assert e.value.status == kpm.KPM_EINVAL
        assert float(eta.abs().sum()) == 0.0
