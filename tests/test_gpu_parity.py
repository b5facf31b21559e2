"""GPU parity: libkpm's CUDA path against the FP64 CPU oracle, element by
element on the same seeded inputs, through the C interface.

Tolerances.  FP64 form: eta within 1e-10 * eta_0 per moment (eta_0 = <nu_0|
nu_0>, so this is 1e-10 on the per-vector normalised moment, which stays
well defined for the near-zero odd moments of this particle-hole symmetric
model) and within 1e-10 relative wherever |eta_k| >= 1e-3 eta_0; single
sweeps within 1e-13 of max|W|.  FP32-storage form: Chebyshev moments mu_n
within 1e-5 (absolute, mu_0 = 1) of the oracle run on the double matrix.
"""
import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham
from kpm_inputs import vectors
from kpm_inputs import workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_MU_TOL = 1e-5


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


def check_eta_fp64(eta, ref):
    eta0 = ref[:, :1]
    err = np.abs(eta - ref)
    assert np.all(err <= FP64_TOL * eta0), "max |d eta|/eta_0 = %g" % (err / eta0).max()
    big = np.abs(ref) >= 1e-3 * eta0
    assert np.all(err[big] <= FP64_TOL * np.abs(ref[big]))


def random_block(n, R, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((n, R)) + 1j * g.standard_normal((n, R))


# ------------------------------------------------------------ single sweep
MATRICES = {
    "ti_4x4x5": lambda: ham.ti_hamiltonian(4, 4, 5, gamma=0.7, seed=3),
    "ragged_203": lambda: ham.random_hermitian(203, 7, seed=8, empty_rows=0.1),
    "ti_open_z": lambda: ham.ti_hamiltonian(3, 4, 6, gamma=1.0, seed=5, periodic=(True, True, False)),
}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("R", [1, 2, 3, 4, 8, 16, 24, 32, 64, 100])
@pytest.mark.parametrize("mat", sorted(MATRICES))
def test_single_sweep_matches_oracle(kpm, orc, mat, R, prec):
    import torch
    h = MATRICES[mat]()
    a, b = scaled(h, kpm)
    n = h["n"]
    V = random_block(n, R, 1)
    W = random_block(n, R, 2)
    with kpm.create(h, a, b, precision=prec, chunk_height=8 if mat == "ragged_203" else 32) as ctx:
        dV, dW = ctx.new_block(R), ctx.new_block(R)
        eta = torch.zeros(3 * R, dtype=torch.float64, device="cuda")
        for init in (False, True):
            ctx.block_upload(R, V, dV)
            ctx.block_upload(R, W, dW)
            if prec == 1:  # the FP32 form works on the rounded inputs
                Vin = ctx.block_download(R, dV)
                Win = ctx.block_download(R, dW)
            else:
                Vin, Win = V, W
            ctx.aug_spmmv(R, dV, dW, eta, init=init)
            Wg = ctx.block_download(R, dW)
            eg = eta.cpu().numpy().reshape(3, R)
            for r in range(R):
                w_ref, e_ref = orc.aug_spmv(h, a, b, Vin[:, r], np.zeros(n) if init else Win[:, r])
                if init:
                    w_ref = w_ref / 2
                    e_ref = np.array([e_ref[0], e_ref[1] / 2, e_ref[2] / 2])
                scale = np.abs(w_ref).max()
                if prec == 0:
                    np.testing.assert_allclose(Wg[:, r], w_ref, rtol=0, atol=1e-13 * scale)
                    np.testing.assert_allclose(eg[:, r], e_ref, rtol=0, atol=1e-12 * e_ref[0])
                else:
                    np.testing.assert_allclose(Wg[:, r], w_ref, rtol=0, atol=2e-6 * scale)
                    np.testing.assert_allclose(eg[:, r], e_ref, rtol=0, atol=2e-6 * e_ref[0])


# --------------------------------------------------------------- moments
def test_small_ti_fp64_moments_match_oracle(kpm, orc):
    cfg = workloads.TI_SMALL
    h = ham.ti_hamiltonian(*cfg["dims"], gamma=cfg["gamma"], seed=cfg["seed"])
    a, b = scaled(h, kpm)
    M, R, seed = cfg["M"], cfg["R"], cfg["seed"]
    ref, ref_im = orc.moments(h, a, b, M, seed, range(R))
    with kpm.create(h, a, b) as ctx:
        eta, eta_im = ctx.moments(M, R, seed, imag=True)
    check_eta_fp64(eta, ref)
    assert np.max(np.abs(eta_im)) <= 1e-12 * h["n"]
    assert np.max(np.abs(kpm.eta_to_mu(eta) - orc.eta_to_mu(ref))) <= FP64_TOL


def test_small_ti_fp32_moments_within_tolerance(kpm, orc):
    cfg = workloads.TI_SMALL
    h = ham.ti_hamiltonian(*cfg["dims"], gamma=cfg["gamma"], seed=cfg["seed"])
    a, b = scaled(h, kpm)
    M, R, seed = cfg["M"], cfg["R"], cfg["seed"]
    ref, _ = orc.moments(h, a, b, M, seed, range(R))
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        eta = ctx.moments(M, R, seed)
    dmu = np.abs(kpm.eta_to_mu(eta) - orc.eta_to_mu(ref))
    assert dmu.max() <= FP32_MU_TOL, dmu.max()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("M,R", [(2, 1), (4, 3), (64, 5), (130, 64), (40, 70)])
def test_ragged_matrix_moments(kpm, orc, prec, M, R):
    h = ham.random_hermitian(203, 7, seed=11, empty_rows=0.1)
    a, b = scaled(h, kpm)
    ref, _ = orc.moments(h, a, b, M, 4, range(R))
    with kpm.create(h, a, b, precision=prec, chunk_height=8, sigma=16) as ctx:
        eta = ctx.moments(M, R, 4)
    if prec == 0:
        # rows with no entries give zero-length chunks and padding rows
        check_eta_fp64(eta, ref)
    else:
        assert np.max(np.abs(kpm.eta_to_mu(eta) - orc.eta_to_mu(ref))) <= FP32_MU_TOL


def test_exact_trace_bloch_closed_form_on_gpu(kpm):
    from test_oracle_pins import bloch_spectrum, cheb
    dims = (4, 4, 4)
    h = ham.ti_hamiltonian(*dims, gamma=0.0)
    n = h["n"]
    a, b = scaled(h, kpm)
    M = 96
    with kpm.create(h, a, b) as ctx:
        eta = ctx.moments_v0(M, vectors.basis_block(n, 0, n))
    mu = kpm.eta_to_mu(eta)
    E = bloch_spectrum(*dims)
    want = np.array([np.mean(cheb(k, a * (E - b))) for k in range(M)])
    np.testing.assert_allclose(mu, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6)])
def test_diagonal_matrix_scalar_chebyshev_on_gpu(kpm, prec, tol):
    from test_oracle_pins import cheb
    g = np.random.default_rng(5)
    lam = g.uniform(-3.0, 5.0, 1000)
    h = ham.diagonal_matrix(lam)
    a, b = scaled(h, kpm)
    M = 256
    with kpm.create(h, a, b, precision=prec) as ctx:
        mu = kpm.eta_to_mu(ctx.moments(M, 8, 2))
    want = np.array([np.mean(cheb(k, a * (lam - b))) for k in range(M)])
    np.testing.assert_allclose(mu, want, rtol=0, atol=tol)


@pytest.mark.parametrize("prec", [0, 1])
def test_moments_are_bitwise_reproducible(kpm, prec):
    import torch
    h = ham.ti_hamiltonian(8, 8, 8, gamma=0.5, seed=0)
    a, b = scaled(h, kpm)
    with kpm.create(h, a, b, precision=prec) as ctx:
        e1 = ctx.moments(128, 16, 3)
        e2 = ctx.moments(128, 16, 3)
        dev = torch.empty((16, 128), dtype=torch.float64, device="cuda")
        ctx.moments_device(128, 16, 3, dev)
        torch.cuda.synchronize()
        e3 = dev.cpu().numpy()
    assert np.array_equal(e1, e2) and np.array_equal(e1, e3)


@pytest.mark.parametrize("prec", [0, 1])
def test_every_launch_shape_agrees(kpm, orc, prec):
    h = ham.ti_hamiltonian(5, 6, 4, gamma=0.9, seed=7)
    a, b = scaled(h, kpm)
    M = 32
    for R in (1, 2, 4, 8, 16, 32, 64):
        ref, _ = orc.moments(h, a, b, M, 9, range(R))
        with kpm.create(h, a, b, precision=prec) as ctx:
            for E in (1, 2, 4):
                T = R // E
                if T < 1 or T > 32 or R % E:
                    continue
                for threads in (128, 256):
                    try:
                        ctx.set_launch(R, T, E, threads)
                    except kpm.KPMError as e:
                        assert e.status == kpm.KPM_EUNSUPPORTED
                        continue
                    eta = ctx.moments(M, R, 9)
                    if prec == 0:
                        check_eta_fp64(eta, ref)
                    else:
                        dmu = np.abs(kpm.eta_to_mu(eta) - orc.eta_to_mu(ref)).max()
                        assert dmu <= FP32_MU_TOL


def test_gpu_entry_points_reject_bad_arguments(kpm):
    import ctypes
    import torch
    h = ham.ti_hamiltonian(3, 3, 3)
    a, b = scaled(h, kpm)
    with kpm.create(h, a, b) as ctx:
        out = np.empty(64)
        for M, R in ((3, 1), (0, 1), (1, 1), (4, 0), (4, -2)):
            rc = kpm.lib.kpm_moments(ctx.handle, M, R, 0,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, None)
            assert rc == kpm.KPM_EINVAL
        V = ctx.new_block(4)
        eta = torch.zeros(12, dtype=torch.float64, device="cuda")
        with pytest.raises(kpm.KPMError) as e:
            ctx.aug_spmmv(4, V, V, eta)
        assert e.value.status == kpm.KPM_EINVAL


def test_cudamalloc_and_torch_allocator_agree(kpm):
    h = ham.ti_hamiltonian(4, 4, 4, gamma=0.3, seed=1)
    a, b = scaled(h, kpm)
    with kpm.create(h, a, b, torch_allocator=False) as c1, kpm.create(h, a, b) as c2:
        assert np.array_equal(c1.moments(64, 8, 1), c2.moments(64, 8, 1))


# --------------------------------------- full-size lattice, sampled outputs
@pytest.fixture(scope="module")
def ti64():
    cfg = workloads.TI_64
    return cfg, ham.ti_hamiltonian(*cfg["dims"], gamma=cfg["gamma"], seed=cfg["seed"])


def test_full_size_single_sweep_fp64_sampled(kpm, orc, ti64):
    """64^3 lattice (N = 1,048,576), R = 32, bench launch shape: every eta of
    one sweep, and the updated W on sampled columns, against the oracle."""
    import torch
    cfg, h = ti64
    a, b = scaled(h, kpm)
    n, R = h["n"], cfg["R"]
    V = vectors.random_phase_block(cfg["seed"], n, range(R))
    W = random_block(n, R, 4)
    with kpm.create(h, a, b, chunk_height=cfg["chunk_height"], sigma=cfg["sigma"]) as ctx:
        dV, dW = ctx.new_block(R), ctx.new_block(R)
        ctx.block_upload(R, V, dV)
        ctx.block_upload(R, W, dW)
        eta = torch.zeros(3 * R, dtype=torch.float64, device="cuda")
        ctx.aug_spmmv(R, dV, dW, eta)
        Wg = ctx.block_download(R, dW)
        eg = eta.cpu().numpy().reshape(3, R)
    for r in (0, 1, 16, 31):
        w_ref, e_ref = orc.aug_spmv(h, a, b, V[:, r], W[:, r])
        np.testing.assert_allclose(Wg[:, r], w_ref, rtol=0, atol=1e-13 * np.abs(w_ref).max())
        np.testing.assert_allclose(eg[:, r], e_ref, rtol=0, atol=1e-12 * e_ref[0])


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_moments_sampled_columns(kpm, orc, ti64, prec):
    """64^3 lattice, R = 32 in one launch; columns 0 and 31 against the
    oracle over the first 200 moments (column r does not depend on R)."""
    cfg, h = ti64
    a, b = scaled(h, kpm)
    M, R = 200, cfg["R"]
    with kpm.create(h, a, b, precision=prec, chunk_height=cfg["chunk_height"],
                    sigma=cfg["sigma"]) as ctx:
        eta = ctx.moments(M, R, cfg["seed"])
    ref, _ = orc.moments(h, a, b, M, cfg["seed"], [0, 31])
    got = eta[[0, 31]]
    if prec == 0:
        check_eta_fp64(got, ref)
    else:
        dmu = np.abs(kpm.eta_to_mu(got) - orc.eta_to_mu(ref)).max()
        assert dmu <= FP32_MU_TOL, dmu


def test_config2_full_moment_count_sampled_columns(kpm, orc, ti64):
    """The bench workload in full: 64^3 lattice, complex double, M = 2000,
    R = 32, seed 1, the bench's layout and launch.  Columns 0 and 31 over all
    2000 moments against the oracle (R11 of the readings: 1e-10 eta_0, and
    1e-10 relative where |eta| >= 1e-3 eta_0).  At this grid the eta
    partials of about 570 sweeps fit one reduction batch, so the 1000 sweeps
    cross a batch boundary; batches of 300 sweeps must give the same
    moments bit for bit (each sweep's partials are summed in block order,
    whatever the batch)."""
    cfg, h = ti64
    a, b = scaled(h, kpm)
    M, R, seed = cfg["M"], cfg["R"], cfg["seed"]
    assert M == 2000
    with kpm.create(h, a, b, chunk_height=cfg["chunk_height"], sigma=cfg["sigma"]) as ctx:
        eta = ctx.moments(M, R, seed)
        ctx.set_reduce_interval(300)
        eta300 = ctx.moments(M, R, seed)
    assert np.array_equal(eta, eta300)
    ref, _ = orc.moments(h, a, b, M, seed, [0, 31], threads=2)
    check_eta_fp64(eta[[0, 31]], ref)


def test_config4_recipe_against_the_oracle(kpm, orc):
    """The precision form's own recipe: 64^3 lattice (gamma 1, seed 2),
    complex float storage, M = 1024, R = 32; vectors 0 and 1 against the
    FP64 oracle: max |d mu_n| <= 1e-5 and the Jackson DOS on K = 4096
    Chebyshev nodes within 1e-4 in relative L1 (a 1e-5 error in every
    moment could move it by up to (1 + 4(M-1)/pi) * 1e-5 = 1.3e-2; the
    errors measured are far smaller and of no fixed sign)."""
    cfg = workloads.TI_64_FP32
    h = ham.ti_hamiltonian(*cfg["dims"], gamma=cfg["gamma"], seed=cfg["seed"])
    a, b = scaled(h, kpm)
    M, R, seed = cfg["M"], cfg["R"], cfg["seed"]
    with kpm.create(h, a, b, precision=kpm.PREC_FP32, chunk_height=32, sigma=256) as ctx:
        eta = ctx.moments(M, R, seed)
    cols = [0, 1]
    ref, _ = orc.moments(h, a, b, M, seed, cols, threads=2)
    mu_g, mu_o = kpm.eta_to_mu(eta[cols]), orc.eta_to_mu(ref)
    dmu = np.abs(mu_g - mu_o).max()
    assert dmu <= FP32_MU_TOL, dmu
    _, rg = kpm.dos(mu_g, 4096, a, b)
    _, ro = orc.dos(mu_o, 4096, a, b)
    l1 = np.abs(rg - ro).sum() / np.abs(ro).sum()
    assert l1 <= 1e-4, l1
