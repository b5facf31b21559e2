"""GPU tests of the autotuner: whatever launch shape, column-block width or
SELL layout it picks, the moments still agree with the FP64 oracle."""
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


def check(kpm, orc, h, a, b, eta, M, R, seed, prec):
    ref, _ = orc.moments(h, a, b, M, seed, range(R))
    if prec == 0:
        assert np.all(np.abs(eta - ref) <= 1e-10 * ref[:, :1])
    else:
        assert np.abs(kpm.eta_to_mu(eta) - orc.eta_to_mu(ref)).max() <= 1e-5


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("R", [8, 64, 100])
def test_autotune_then_moments(kpm, orc, prec, R):
    h = ham.ti_hamiltonian(8, 6, 5, gamma=1.0, seed=3)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    with kpm.create(h, a, b, precision=prec) as ctx:
        best = ctx.autotune(R, sweeps=3)
        assert best["max_block_width"] in (16, 32, 64)
        assert best["lanes_per_row"] * best["cols_per_lane"] == min(R, best["max_block_width"])
        eta = ctx.moments(48, R, 5)
    check(kpm, orc, h, a, b, eta, 48, R, 5, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_on_first_use(kpm, orc, prec):
    h = ham.random_hermitian(300, 6, seed=9, empty_rows=0.05)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    with kpm.create(h, a, b, precision=prec, autotune=True, chunk_height=16, sigma=64) as ctx:
        eta = ctx.moments(64, 16, 2)
        again = ctx.moments(64, 16, 2)
    assert np.array_equal(eta, again)
    check(kpm, orc, h, a, b, eta, 64, 16, 2, prec)


def test_layout_autotuner(kpm, orc):
    h = ham.random_hermitian(500, 5, seed=4, empty_rows=0.1)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    best = kpm.autotune_layout(h, a, b, 32, precision=kpm.PREC_FP32, sweeps=2)
    assert best["chunk_height"] in (8, 16, 32, 64, 128)  # kpm_autotune_layout's candidates
    assert best["sigma"] in (1, 256, 4096) and best["ms_per_sweep"] > 0
    with kpm.create(h, a, b, precision=kpm.PREC_FP32, chunk_height=best["chunk_height"],
                    sigma=best["sigma"], autotune=True) as ctx:
        eta = ctx.moments(32, 32, 1)
    check(kpm, orc, h, a, b, eta, 32, 32, 1, 1)
