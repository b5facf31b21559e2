"""Parity at the large lattice: 240 x 240 x 120 sites (N = 27,648,000 rows,
359,424,000 non-zeros, complex double; 7.2 GB matrix and 28 GB of vector
blocks at R = 32).  The oracle computes sampled outputs: the first 128
moments of vectors 0, 1, 16 and 31 (one oracle run, one host thread per
vector, shared by both forms); the full M = 1024 run is checked against
the short run (same kernels, so its first moments must be identical) and
against invariants that hold at any size."""
import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham
from kpm_inputs import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1410_5242_gb300 import build
    build.build()
    from paper_1410_5242_gb300 import kpm as k
    return k


COLS = [0, 1, 16, 31]
M_SHORT = 128


@pytest.fixture(scope="module")
def large():
    cfg = workloads.TI_LARGE
    return cfg, ham.ti_hamiltonian(*cfg["dims"], gamma=cfg["gamma"], seed=cfg["seed"])


@pytest.fixture(scope="module")
def large_ref(orc, large):
    """The oracle's first M_SHORT moments of the sampled vectors."""
    cfg, h = large
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    ref, _ = orc.moments(h, a, b, M_SHORT, cfg["seed"], COLS, threads=len(COLS))
    return ref


def test_large_lattice_fp64(kpm, large, large_ref):
    cfg, h = large
    n, R, M, seed = h["n"], cfg["R"], cfg["M"], cfg["seed"]
    assert n == 27_648_000 and len(h["col"]) == 13 * n
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    with kpm.create(h, a, b) as ctx:
        short = ctx.moments(M_SHORT, R, seed)
        full = ctx.moments(M, R, seed)
    ref = large_ref
    got = short[COLS]
    assert np.all(np.abs(got - ref) <= 1e-10 * ref[:, :1])
    big = np.abs(ref) >= 1e-3 * ref[:, :1]
    assert np.all(np.abs(got - ref)[big] <= 1e-10 * np.abs(ref[big]))
    assert np.array_equal(full[:, :M_SHORT], short)
    # invariants of the whole run: unit-modulus start vectors, norms, bounds
    np.testing.assert_allclose(full[:, 0], n, rtol=1e-13)
    assert np.all(full[:, 0::2] >= 0)
    c = 2 * full - full[:, [0, 1] * (M // 2)]
    c[:, :2] = full[:, :2]
    assert np.max(np.abs(c)) <= n * (1 + 1e-10)
    mu = kpm.eta_to_mu(full)
    assert mu[0] == pytest.approx(1.0, abs=1e-15)
    _, rho = kpm.dos(mu, 4096, a, b)
    assert rho.min() > -1e-6 * rho.max()


def test_large_lattice_fp32_staged(kpm, orc, large, large_ref):
    """The same lattice in complex float on the staged kernel (864,000
    chunks, half-complex form): the first 128 moments of vectors 0, 1, 16,
    31 against the oracle within the float form's tolerance, and the
    invariants of a 256-moment run."""
    cfg, h = large
    n, R, seed = h["n"], cfg["R"], cfg["seed"]
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        assert ctx.get_launch(R)["stages"] >= 1
        assert ctx.info()["half_complex"] == 1
        short = ctx.moments(M_SHORT, R, seed)
        full = ctx.moments(256, R, seed)
    ref = large_ref
    got = short[COLS]
    assert np.abs(kpm.eta_to_mu(got) - orc.eta_to_mu(ref)).max() <= 1e-5
    np.testing.assert_allclose(got[:, 0], ref[:, 0], rtol=1e-6)
    np.testing.assert_allclose(full[:, :M_SHORT], short, rtol=0, atol=1e-9 * n)
    np.testing.assert_allclose(full[:, 0], n, rtol=1e-6)
    assert np.all(full[:, 0::2] >= 0)
    mu = kpm.eta_to_mu(full)
    assert np.max(np.abs(mu)) <= 1 + 1e-5
