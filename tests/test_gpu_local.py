"""GPU tests of the local and momentum-resolved moments (include/kpm.h,
kpm_moments_local and kpm_moments_plane_wave; the local DOS and A(k, E) of
Sec. "Application Scenario", Fig. 2): start vectors built on the device,
then the same sweeps as kpm_moments.  Parity with the FP64 oracle run on
start blocks the test builds itself (kpm_inputs.vectors): eta within 1e-10
of eta_0 per moment (and 1e-10 relative where |eta| >= 1e-3 eta_0) in complex
double, mu within 1e-5 in the complex float form; on the clean lattice the
closed forms (every site's LDOS is the Bloch DOS; a Bloch wave's moments
are the diagonal of T_n of the 4x4 Bloch matrix)."""
import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham
from kpm_inputs import vectors

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


def cheb(m, x):
    return np.cos(m * np.arccos(np.clip(x, -1.0, 1.0)))


def bloch_cheb_diag(q, v, a, b, M):
    """[T_n(a (H(k) - b))]_{alpha alpha} of the clean lattice's 4x4 Bloch
    matrix at k = 2 pi q (on-site v + 2 Gamma^1, hoppings times e^{i k.d})."""
    hk = v * np.eye(4) + 2.0 * ham.dirac_matrices()[1]
    for d, blk in ham.ti_blocks().items():
        hk = hk + blk * np.exp(2j * np.pi * np.dot(q, d))
    lam, U = np.linalg.eigh(hk)
    w = np.abs(U) ** 2
    return np.array([w @ cheb(n, a * (lam - b)) for n in range(M)])


# wave vectors: on the 6 x 5 x 4 lattice's Bloch grid, off it, and far
# outside [0, 1)
QS = np.array([[0, 0, 0], [1 / 6, 2 / 5, 1 / 4], [0.1234, 0.5, -0.3], [3.7, -2.25, 11.5],
               [5 / 6, 3 / 5, 3 / 4]])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_plane_wave_moments_match_oracle(kpm, orc, prec):
    dims = (6, 5, 4)
    h = ham.ti_hamiltonian(*dims, gamma=1.5, seed=3)
    a, b = scaled(h, kpm)
    M = 64
    q = np.repeat(QS, 4, axis=0)
    orb = np.tile(np.arange(4), len(QS))
    ref, _ = orc.moments_v0(h, a, b, M, vectors.plane_wave_block(dims, 4, q, orb))
    p = kpm.PREC_FP64 if prec == "fp64" else kpm.PREC_FP32
    with kpm.create(h, a, b, precision=p) as ctx:
        eta, eti = ctx.moments_plane_wave(M, dims, 4, q, orb, imag=True)
    if prec == "fp64":
        check_eta_fp64(eta, ref)
        assert np.abs(eti).max() <= 1e-12
    else:
        for r in range(len(q)):
            dmu = np.abs(kpm.eta_to_mu(eta[r:r + 1]) - orc.eta_to_mu(ref[r:r + 1])).max()
            assert dmu <= FP32_MU_TOL, (r, dmu)


def test_plane_wave_clean_lattice_closed_form(kpm):
    # wave vectors on the lattice's Bloch grid (multiples of 1/L per axis,
    # some outside [0, 1)): only there is a Bloch wave periodic, so that H
    # maps the four waves of one k into their span
    dims, v = (6, 5, 4), 0.25
    h = ham.ti_hamiltonian(*dims, potential=np.full(int(np.prod(dims)), v))
    a, b = scaled(h, kpm)
    M = 96
    grid = np.array([[0, 0, 0], [1 / 6, 2 / 5, 1 / 4], [5 / 6, 3 / 5, 3 / 4], [7 / 6, -2 / 5, 9 / 4],
                     [1 / 2, 0, 1 / 2]])
    q = np.repeat(grid, 4, axis=0)
    orb = np.tile(np.arange(4), len(grid))
    with kpm.create(h, a, b) as ctx:
        eta = ctx.moments_plane_wave(M, dims, 4, q, orb)
    for r in range(len(q)):
        want = bloch_cheb_diag(q[r], v, a, b, M)[:, orb[r]]
        np.testing.assert_allclose(kpm.eta_to_mu(eta[r:r + 1]), want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_local_moments_match_oracle(kpm, orc, prec):
    h = ham.ti_hamiltonian(7, 4, 5, gamma=2.0, seed=8)
    a, b = scaled(h, kpm)
    M = 64
    rows = np.array([0, 1, 2, 3, 57, 57, 300, h["n"] - 1] + list(range(400, 440)))  # R = 48
    ref, _ = orc.moments_v0(h, a, b, M, vectors.rows_block(h["n"], rows))
    p = kpm.PREC_FP64 if prec == "fp64" else kpm.PREC_FP32
    with kpm.create(h, a, b, precision=p) as ctx:
        eta = ctx.moments_local(M, rows)
    if prec == "fp64":
        check_eta_fp64(eta, ref)
    else:
        for r in range(len(rows)):
            dmu = np.abs(kpm.eta_to_mu(eta[r:r + 1]) - orc.eta_to_mu(ref[r:r + 1])).max()
            assert dmu <= FP32_MU_TOL, (r, dmu)


def test_ldos_clean_lattice_is_bloch_dos(kpm):
    dims, v = (8, 6, 5), -0.3
    h = ham.ti_hamiltonian(*dims, potential=np.full(int(np.prod(dims)), v))
    a, b = scaled(h, kpm)
    M = 80
    sites = [0, 13, 239]
    rows = np.array([4 * s + al for s in sites for al in range(4)])
    with kpm.create(h, a, b) as ctx:
        eta = ctx.moments_local(M, rows)
    # Bloch bands of the clean lattice: E = v +- sqrt(mass^2 + sum sin^2 k), twofold
    k = [2 * np.pi * np.arange(L) / L for L in dims]
    KX, KY, KZ = np.meshgrid(*k, indexing="ij")
    e = np.sqrt((2.0 - np.cos(KX) - np.cos(KY) - np.cos(KZ)) ** 2
                + np.sin(KX) ** 2 + np.sin(KY) ** 2 + np.sin(KZ) ** 2).ravel()
    E = np.concatenate([v + e, v - e])
    want = np.array([np.mean(cheb(n, a * (E - b))) for n in range(M)])
    for i in range(len(sites)):
        mu = kpm.eta_to_mu(eta[4 * i:4 * i + 4])
        np.testing.assert_allclose(mu, want, rtol=0, atol=1e-12)


def test_local_and_plane_wave_reject_bad_arguments(kpm):
    dims = (4, 4, 4)
    h = ham.ti_hamiltonian(*dims, gamma=0.5, seed=1)
    a, b = scaled(h, kpm)
    with kpm.create(h, a, b) as ctx:
        for rows in ([-1], [h["n"]]):
            with pytest.raises(kpm.KPMError) as e:
                ctx.moments_local(8, rows)
            assert e.value.status == kpm.KPM_EINVAL
        bad = [((4, 4, 5), 4, [0]), (dims, 2, [0]), (dims, 4, [4]), (dims, 4, [-1])]
        for d, norb, orb in bad:
            with pytest.raises(kpm.KPMError) as e:
                ctx.moments_plane_wave(8, d, norb, [[0.1, 0.2, 0.3]], orb)
            assert e.value.status == kpm.KPM_EINVAL
        with pytest.raises(kpm.KPMError) as e:
            ctx.moments_plane_wave(8, dims, 4, [[np.nan, 0, 0]], [0])
        assert e.value.status == kpm.KPM_EINVAL
        with pytest.raises(kpm.KPMError) as e:
            ctx.moments_plane_wave(7, dims, 4, [[0.1, 0, 0]], [0])  # odd M
        assert e.value.status == kpm.KPM_EINVAL
