"""The row-partitioned run on the GPU (Sec. "Symmetric Heterogeneous
Execution"): every part in its own context with halo slots, all parts in
one process on one GPU (paper_1410_5242_gb300.partition.in_process_moments:
the halo rows packed and unpacked on the device, one part after the other,
so no kernel waits on another), against the oracle's moments of the whole
matrix and against the unpartitioned context's."""
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


@pytest.fixture(scope="module")
def partition(kpm):
    from paper_1410_5242_gb300 import partition as p
    return p


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("parts,R", [(2, 8), (3, 8), (2, 3)])
def test_partitioned_run_on_the_gpu(kpm, orc, partition, prec, parts, R):
    h = ham.ti_hamiltonian(8, 8, 12, gamma=0.9, seed=3)  # 12 planes of 256 rows
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M, seed = 64, 5
    rs = partition.slab_row_start(h["n"], parts, plane_rows=256)
    steps = [partition.GpuPartStep(p, a, b, precision=prec) for p in partition.build_parts(h, rs)]
    try:
        if R >= 8:
            assert all(s.ctx.get_launch(R)["stages"] >= 1 for s in steps)
        eta, eti = partition.in_process_moments(steps, M, R, seed)
    finally:
        for s in steps:
            s.close()
    ref, _ = orc.moments(h, a, b, M, seed, range(R))
    with kpm.create(h, a, b, precision=prec) as ctx:
        whole = ctx.moments(M, R, seed)
    eta0 = ref[:, :1]
    if prec == 0:
        assert np.all(np.abs(eta - ref) <= 1e-10 * eta0)
        assert np.all(np.abs(eta - whole) <= 1e-12 * eta0)
        assert np.all(np.abs(eti) <= 1e-12 * eta0)
    else:
        dmu = np.abs(kpm.eta_to_mu(eta) - orc.eta_to_mu(ref)).max()
        assert dmu <= 1e-5, dmu


def test_part_context_serves_sweeps_only_and_checks_pack_rows(kpm, partition):
    import torch
    h = ham.ti_hamiltonian(4, 4, 6, gamma=0.5, seed=1)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    rs = partition.slab_row_start(h["n"], 2, plane_rows=64)
    step = partition.GpuPartStep(partition.build_parts(h, rs)[0], a, b)
    try:
        with pytest.raises(kpm.KPMError) as e:
            step.ctx.moments(8, 4, 1)
        assert e.value.status == kpm.KPM_EUNSUPPORTED
        step.start(4, 2, 1)
        bad = torch.tensor([0, 1, 10_000], dtype=torch.int32, device="cuda")  # row outside
        buf = torch.zeros(3 * step.row_bytes, dtype=torch.uint8, device="cuda")
        step.ctx.halo_pack(4, step.V, bad, buf)
        torch.cuda.synchronize()
        with pytest.raises(kpm.KPMError) as e:
            step.ctx.check_device_error()
        assert e.value.status == kpm.KPM_EINVAL
        step.ctx.check_device_error()  # read and cleared
    finally:
        step.close()
