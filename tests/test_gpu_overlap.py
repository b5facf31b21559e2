"""GPU test of programmatic dependent launches (include/kpm.h,
kpm_set_sweep_overlap, KPM_OVERLAP_PDL, the default): a staged sweep's
blocks may start while the previous kernel in the stream finishes, but wait
for it before touching the vector blocks or the eta partials, so every
result must equal that of plain launches bit for bit -- for the moment
calls (sweeps and eta reductions back to back) and for single sweeps issued
one after another."""
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


def scaled(h, k):
    return k.scale_from_bounds(*k.gershgorin(h), 0.01)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_programmatic_launches_match_plain_launches(kpm, prec):
    import torch
    from kpm_inputs import vectors
    h = ham.ti_hamiltonian(16, 16, 24, gamma=1.0, seed=4)
    a, b = scaled(h, kpm)
    M, R = 40, 32
    fp64 = prec == "fp64"
    with kpm.create(h, a, b, precision=kpm.PREC_FP64 if fp64 else kpm.PREC_FP32) as ctx:
        assert ctx.get_launch(R)["stages"] >= 1
        out = {}
        for mode in (kpm.OVERLAP_NONE, kpm.OVERLAP_PDL):
            ctx.set_sweep_overlap(mode)
            eta = ctx.moments(M, R, 3)
            # ten single sweeps in a row on the same stream, eta summed on
            # the device after each; before every other sweep a PyTorch
            # kernel scales V by 1/2 (the sweep must wait for it)
            V, W = ctx.new_block(R), ctx.new_block(R)
            ctx.block_upload(R, vectors.random_phase_block(5, h["n"], range(R)), V)
            e = torch.zeros((10, 3 * R), dtype=torch.float64, device="cuda")
            real = torch.float64 if fp64 else torch.float32
            for m in range(10):
                if m % 2:
                    V.view(real).mul_(0.5)
                ctx.aug_spmmv(R, V, W, e[m], init=(m == 0))
                V, W = W, V
            torch.cuda.synchronize()
            ctx.check_device_error()
            out[mode] = (eta, e.cpu().numpy(), ctx.block_download(R, V))
    for x, y in zip(out[kpm.OVERLAP_NONE], out[kpm.OVERLAP_PDL]):
        np.testing.assert_array_equal(x, y)


def test_sweep_overlap_rejects_unknown_modes(kpm):
    h = ham.ti_hamiltonian(4, 4, 4, gamma=0.5, seed=0)
    a, b = scaled(h, kpm)
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        for mode in (-1, 2):
            with pytest.raises(kpm.KPMError) as e:
                ctx.set_sweep_overlap(mode)
            assert e.value.status == kpm.KPM_EINVAL
        ctx.set_sweep_overlap(kpm.OVERLAP_NONE)
        ctx.set_sweep_overlap(kpm.OVERLAP_PDL)
