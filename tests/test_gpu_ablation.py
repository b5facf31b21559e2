"""GPU tests of the ablation paths (the paper's optimisation stages): the
naive library-call KPM-DOS of Fig. 3, the sweep variants without dot
products, and the per-sweep eta reduction, each against the oracle or the
fused path."""
import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham
from kpm_inputs import vectors, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1410_5242_gb300 import build
    build.build()
    from paper_1410_5242_gb300 import kpm as k
    return k


def test_naive_library_path_matches_oracle(kpm, orc):
    cfg = workloads.TI_SMALL
    h = ham.ti_hamiltonian(*cfg["dims"], gamma=cfg["gamma"], seed=cfg["seed"])
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    M, R, seed = cfg["M"], cfg["R"], cfg["seed"]
    with kpm.Naive(h, a, b) as nv:
        eta = nv.moments(M, R, seed)
    ref, _ = orc.moments(h, a, b, M, seed, range(R))
    assert np.all(np.abs(eta - ref) <= 1e-10 * ref[:, :1])


@pytest.mark.parametrize("prec", [0, 1])
def test_sweep_variants(kpm, prec):
    import torch
    h = ham.ti_hamiltonian(5, 6, 4, gamma=0.9, seed=7)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    R = 32
    g = np.random.default_rng(1)
    V0 = vectors.random_phase_block(3, h["n"], range(R))
    W0 = g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))
    with kpm.create(h, a, b, precision=prec) as ctx:
        def run(fn):
            V, W = ctx.new_block(R), ctx.new_block(R)
            ctx.block_upload(R, V0, V)
            ctx.block_upload(R, W0, W)
            fn(V, W)
            torch.cuda.synchronize()
            return ctx.block_download(R, W)
        full = run(lambda V, W: ctx.aug_spmmv(R, V, W, None))
        init = run(lambda V, W: ctx.aug_spmmv(R, V, W, None, init=True))
        nodot = run(lambda V, W: ctx.sweep_variant(R, V, W, 1))
        plain = run(lambda V, W: ctx.sweep_variant(R, V, W, 2))
        v0 = run(lambda V, W: ctx.sweep_variant(R, V, W, 0))
    assert np.array_equal(nodot, full) and np.array_equal(v0, full)
    assert np.array_equal(plain, init)
    with pytest.raises(kpm.KPMError):
        with kpm.create(h, a, b, precision=prec) as ctx:
            V, W = ctx.new_block(R), ctx.new_block(R)
            ctx.sweep_variant(R, V, W, 3)


@pytest.mark.parametrize("prec", [0, 1])
def test_per_sweep_reduction_gives_identical_moments(kpm, prec):
    h = ham.ti_hamiltonian(6, 6, 6, gamma=1.0, seed=4)
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    with kpm.create(h, a, b, precision=prec) as ctx:
        batched = ctx.moments(200, 16, 5)
        ctx.set_reduce_interval(1)
        per_sweep = ctx.moments(200, 16, 5)
        ctx.set_reduce_interval(7)
        seven = ctx.moments(200, 16, 5)
    assert np.array_equal(batched, per_sweep) and np.array_equal(batched, seven)
