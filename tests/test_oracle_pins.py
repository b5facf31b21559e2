"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself.  The expected values come from
dense eigendecompositions (numpy.linalg.eigh), closed forms (scalar
Chebyshev polynomials for a diagonal matrix, the 4x4 Bloch bands of the
clean lattice of Eq. 1), a library DCT, and invariants of Eq. 3 and the
stochastic trace.  A last group plants typical mistakes (a transposed
operand, a flipped sign) in the oracle's inputs and checks that the pins
reject them.
"""
import math
import os

import numpy as np
import pytest
import scipy.fft

from kpm_inputs import hamiltonians as ham
from kpm_inputs import rng, vectors

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cheb(m, x):
    """T_m(x) for |x| <= 1 via the trigonometric definition cos(m arccos x)."""
    return np.cos(m * np.arccos(np.clip(x, -1.0, 1.0)))


def eig_moments(dense, a, b, r, M):
    """eta_0..eta_{M-1} of start vector r from the eigendecomposition of H."""
    lam, U = np.linalg.eigh(dense)
    w = np.abs(U.conj().T @ r) ** 2
    x = a * (lam - b)
    eta = np.empty(M)
    for m in range(M // 2):
        eta[2 * m] = np.sum(w * cheb(m, x) ** 2)
        eta[2 * m + 1] = np.sum(w * cheb(m + 1, x) * cheb(m, x))
    return eta


def bloch_spectrum(nx, ny, nz, v=0.0, t=1.0):
    """Eigenvalues of the clean periodic lattice of Eq. 1: for each Bloch
    vector k, E = v +- sqrt((2 - t sum cos k_j)^2 + t^2 sum sin^2 k_j), each
    twofold (derived from the hopping blocks with anticommuting Gammas)."""
    kx = 2 * np.pi * np.arange(nx) / nx
    ky = 2 * np.pi * np.arange(ny) / ny
    kz = 2 * np.pi * np.arange(nz) / nz
    KX, KY, KZ = np.meshgrid(kx, ky, kz, indexing="ij")
    mass = 2.0 - t * (np.cos(KX) + np.cos(KY) + np.cos(KZ))
    kin = t * t * (np.sin(KX) ** 2 + np.sin(KY) ** 2 + np.sin(KZ) ** 2)
    e = np.sqrt(mass ** 2 + kin).ravel()
    return np.concatenate([v + e, v + e, v - e, v - e])


# --------------------------------------------------------------------- RNG
def test_splitmix64_reference_outputs():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    got = []
    s = 0
    for _ in range(3):
        s = (s + rng.GOLDEN) & rng.MASK64
        got.append(rng.mix_int(s))
    assert got == want


def test_oracle_uniform_matches_published_stream_definition(orc):
    # oracle (C) and input module (numpy) implement the same published generator
    idx = np.array([0, 1, 2, 1000, 2**40 + 3], dtype=np.uint64)
    for seed, stream in [(0, 0), (1, 1), (12345, 1), (2**63 + 7, 2)]:
        want = rng.uniform(seed, stream, idx)
        got = [orc.uniform(seed, stream, int(i)) for i in idx]
        assert np.array_equal(np.array(got), want)


def test_random_phase_vector_unit_modulus_and_columns(orc):
    n = 50
    blk = vectors.random_phase_block(7, n, [0, 3])
    for k, r in enumerate([0, 3]):
        v = orc.random_phase_vector(7, n, r)
        np.testing.assert_allclose(np.abs(v), 1.0, rtol=0, atol=1e-15)
        np.testing.assert_allclose(v, blk[:, k], rtol=0, atol=4e-16)


# -------------------------------------------------------------- Gershgorin
def test_gershgorin_closed_form_ti(orc):
    # t = 1: diagonal V_n +- 2, off-diagonal row sum 12 * 1/2 = 6
    h = ham.ti_hamiltonian(4, 3, 5, gamma=0.8, seed=3)
    lo, hi = orc.gershgorin(h)
    assert lo == pytest.approx(h["potential"].min() - 8.0, abs=1e-13)
    assert hi == pytest.approx(h["potential"].max() + 8.0, abs=1e-13)
    lam = np.linalg.eigvalsh(ham.to_dense(h))
    assert lo <= lam.min() and lam.max() <= hi


def test_gershgorin_small_by_hand(orc):
    # [[1, 2i], [-2i, -3]]: discs [1-2, 1+2] and [-3-2, -3+2]
    csr = {"n": 2, "row_ptr": np.array([0, 2, 4]), "col": np.array([0, 1, 0, 1]),
           "val": np.array([1, 2j, -2j, -3])}
    assert orc.gershgorin(csr) == (-5.0, 3.0)


def test_scale_from_bounds_maps_interval(orc):
    a, b = orc.scale_from_bounds(-3.0, 5.0, 0.01)
    assert b == 1.0
    assert a * (5.0 - b) == pytest.approx(0.99, abs=1e-15)
    assert a * (-3.0 - b) == pytest.approx(-0.99, abs=1e-15)
    with pytest.raises(ValueError):
        orc.scale_from_bounds(1.0, 1.0, 0.01)


# ------------------------------------------------------- single fused step
def test_aug_spmv_on_eigenvectors(orc):
    h = ham.ti_hamiltonian(3, 3, 4, gamma=0.5, seed=1)
    lam, U = np.linalg.eigh(ham.to_dense(h))
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    for k, j in [(0, 5), (17, 17), (100, 3)]:
        v, w = U[:, k], U[:, j]
        w_new, eta = orc.aug_spmv(h, a, b, v, w)
        s = 2 * a * (lam[k] - b)
        np.testing.assert_allclose(w_new, s * v - w, atol=1e-13)
        assert eta[0] == pytest.approx(1.0, abs=1e-14)
        assert eta[1] == pytest.approx(s - (1.0 if j == k else 0.0), abs=1e-13)
        assert abs(eta[2]) < 1e-13


def test_aug_spmv_matches_dense_product(orc):
    h = ham.random_hermitian(60, 5, seed=2, empty_rows=0.1)
    d = ham.to_dense(h)
    g = np.random.default_rng(0)
    v = g.standard_normal(60) + 1j * g.standard_normal(60)
    w = g.standard_normal(60) + 1j * g.standard_normal(60)
    a, b = 0.3, -0.2
    w_new, eta = orc.aug_spmv(h, a, b, v, w)
    ref = 2 * a * (d @ v - b * v) - w
    np.testing.assert_allclose(w_new, ref, atol=1e-12)
    assert eta[0] == pytest.approx(np.vdot(v, v).real, rel=1e-14)
    assert eta[1] + 1j * eta[2] == pytest.approx(np.vdot(ref, v), rel=1e-13)


# -------------------------------------------------------- full recurrence
def test_moments_match_dense_eigendecomposition(orc):
    h = ham.ti_hamiltonian(3, 3, 3, gamma=0.5, seed=4)
    d = ham.to_dense(h)
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M = 64
    er, ei = orc.moments(h, a, b, M, seed=11, cols=[0, 1, 2])
    blk = vectors.random_phase_block(11, h["n"], [0, 1, 2])
    for r in range(3):
        want = eig_moments(d, a, b, blk[:, r], M)
        assert np.max(np.abs(er[r] - want)) <= 1e-12 * want[0]
        assert np.max(np.abs(ei[r])) <= 1e-12 * want[0]


def test_diagonal_matrix_scalar_chebyshev(orc):
    g = np.random.default_rng(5)
    lam = g.uniform(-3.0, 5.0, 300)
    h = ham.diagonal_matrix(lam)
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M = 128
    er, _ = orc.moments(h, a, b, M, seed=2, cols=range(3))
    mu = orc.eta_to_mu(er)
    want = np.array([np.mean(cheb(k, a * (lam - b))) for k in range(M)])
    np.testing.assert_allclose(mu, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dims,v", [((4, 4, 4), 0.0), ((3, 4, 5), 0.3)])
def test_exact_trace_clean_lattice_bloch(orc, dims, v):
    h = ham.ti_hamiltonian(*dims, potential=np.full(int(np.prod(dims)), v))
    n = h["n"]
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M = 64
    er, ei = orc.moments_v0(h, a, b, M, vectors.basis_block(n, 0, n))
    mu = orc.eta_to_mu(er)
    E = bloch_spectrum(*dims, v=v)
    want = np.array([np.mean(cheb(k, a * (E - b))) for k in range(M)])
    np.testing.assert_allclose(mu, want, rtol=0, atol=1e-12)


def test_random_phase_trace_statistics(orc):
    dims = (4, 4, 4)
    h = ham.ti_hamiltonian(*dims, gamma=0.0)
    n = h["n"]
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M, R = 48, 16
    er, _ = orc.moments(h, a, b, M, seed=9, cols=range(R))
    mu = orc.eta_to_mu(er)
    E = bloch_spectrum(*dims)
    exact = np.array([np.mean(cheb(k, a * (E - b))) for k in range(M)])
    sigma = 1.0 / math.sqrt(R * n)   # Var <r|A|r> <= ||A||_F^2 for random phases
    assert np.max(np.abs(mu - exact)) < 5 * sigma
    assert mu[0] == pytest.approx(1.0, abs=1e-14)


def test_invariants_small_disordered_lattice(orc):
    h = ham.ti_hamiltonian(8, 8, 8, gamma=0.5, seed=0)
    n = h["n"]
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M, R = 256, 4
    er, ei = orc.moments(h, a, b, M, seed=0, cols=range(R))
    assert np.allclose(er[:, 0], n, rtol=1e-14)                # unit-modulus entries
    assert np.max(np.abs(ei)) <= 1e-12 * n                     # Hermitian H: real moments
    assert np.all(er[:, 0::2] >= 0)                            # eta_2m = <nu_m|nu_m>
    c = 2 * er - er[:, [0, 1] * (M // 2)]
    c[:, :2] = er[:, :2]
    assert np.max(np.abs(c)) <= n * (1 + 1e-12)                # ||T_n(H~)|| <= 1
    mu = orc.eta_to_mu(er)
    assert mu[0] == pytest.approx(1.0, abs=1e-15)
    for r in range(R):                                         # each vector: positive measure
        _, rho = orc.dos(orc.eta_to_mu(er[r:r + 1]), 1024, a, b)
        assert rho.min() > -1e-9 * rho.max()


# ------------------------------------------------------ reconstruction/DOS
def test_jackson_closed_forms(orc):
    for M in (2, 7, 64, 1000):
        g = orc.jackson(M)
        assert g[0] == pytest.approx(1.0, abs=1e-15)
        assert g[1] == pytest.approx(math.cos(math.pi / (M + 1)), abs=1e-14)
        assert np.all(np.diff(g) < 0) and g[-1] > 0


def test_jackson_kernel_is_positive(orc):
    M = 40
    g = orc.jackson(M)
    x = np.cos(np.linspace(0, np.pi, 301))
    for x0 in (-0.95, -0.3, 0.0, 0.6):
        k = g[0] + 2 * sum(g[n] * cheb(n, x) * cheb(n, x0) for n in range(1, M))
        assert k.min() > 0


def test_dos_quadrature_and_dct_roundtrip(orc):
    M, K = 64, 256
    g = np.random.default_rng(1)
    mu = np.concatenate([[1.0], g.uniform(-0.3, 0.3, M - 1)])
    a, b = 0.25, 1.5
    e, rho = orc.dos(mu, K, a, b)
    theta = np.pi * (np.arange(K) + 0.5) / K
    x = np.cos(theta)
    np.testing.assert_allclose(e, x / a + b, rtol=0, atol=1e-14)
    rt = rho / a
    # node quadrature: (pi/K) sum rho~(x_k) sqrt(1 - x_k^2) = g_0 mu_0
    assert (np.pi / K) * np.sum(rt * np.sin(theta)) == pytest.approx(1.0, abs=1e-13)
    # the DCT-II of the node values returns the damped coefficients
    f = rt * np.pi * np.sin(theta)
    y = scipy.fft.dct(f, type=2) / K
    coeff = np.concatenate([[y[0] / 2], y[1:M] / 2])
    np.testing.assert_allclose(coeff, orc.jackson(M) * mu, rtol=0, atol=1e-13)
    np.testing.assert_allclose(y[M:], 0.0, atol=1e-12)


def test_eta_to_mu_rejects_bad_shapes(orc):
    with pytest.raises(ValueError):
        orc.eta_to_mu(np.ones((2, 3)))
    with pytest.raises(ValueError):
        orc.eta_to_mu(np.zeros((1, 4)))


def test_oracle_rejects_bad_csr_and_odd_m(orc):
    h = ham.ti_hamiltonian(3, 3, 3)
    a, b = 0.1, 0.0
    with pytest.raises(ValueError):
        orc.kpm_vector(h, a, b, 5, np.ones(h["n"]))
    bad = dict(h, col=h["col"].copy())
    bad["col"][3] = h["n"]
    with pytest.raises(ValueError):
        orc.kpm_vector(bad, a, b, 4, np.ones(h["n"]))


# ---------------------------------------- planted mistakes fail the pins
def _transpose(csr):
    d = ham.to_dense(csr).T
    rows, cols = np.nonzero(d)
    return {"n": csr["n"], "row_ptr": np.searchsorted(rows, np.arange(csr["n"] + 1)).astype(np.int64),
            "col": cols.astype(np.int32), "val": d[rows, cols]}


def test_pins_reject_transposed_operand_and_sign_flip(orc):
    h = ham.ti_hamiltonian(3, 3, 3, gamma=0.5, seed=4)
    d = ham.to_dense(h)
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    b += 0.05  # keep a visible shift so that a sign flip matters
    M = 32
    r = vectors.random_phase_block(11, h["n"], [0])[:, 0]
    want = eig_moments(d, a, b, r, M)
    good, _ = orc.kpm_vector(h, a, b, M, r)
    assert np.max(np.abs(good - want)) <= 1e-12 * want[0]
    transposed, _ = orc.kpm_vector(_transpose(h), a, b, M, r)
    assert np.max(np.abs(transposed - want)) > 1e-6 * want[0]
    flipped, _ = orc.kpm_vector(h, a, -b, M, r)
    assert np.max(np.abs(flipped - want)) > 1e-6 * want[0]


# ------------------------------------------ local and momentum-resolved
def bloch_matrix(q, v=0.0, t=1.0):
    """4x4 Bloch Hamiltonian H(k) of the clean lattice of Eq. 1 at k = 2 pi q:
    the on-site block v + 2 Gamma^1 plus every hopping block times
    exp(i k . d) (a Bloch wave on orbital b is mapped into the span of the
    four Bloch waves of the same k)."""
    g1 = ham.dirac_matrices()[1]
    hk = v * np.eye(4) + 2.0 * g1
    for d, blk in ham.ti_blocks(t).items():
        hk = hk + blk * np.exp(2j * np.pi * np.dot(q, d))
    return hk


def matrix_cheb_diag(hk, a, b, M):
    """[T_n(a (H(k) - b))]_{alpha alpha}, n < M, from the 4x4 eigendecomposition."""
    lam, U = np.linalg.eigh(hk)
    x = a * (lam - b)
    w = np.abs(U) ** 2  # w[alpha, band]
    return np.array([w @ cheb(n, x) for n in range(M)])  # [M][4]


def test_plane_wave_moments_bloch_closed_form(orc):
    # a Bloch wave of the clean lattice on orbital alpha: its moments are the
    # diagonal entries of T_n of the 4x4 Bloch matrix (the A(k, E) of Fig. 2
    # restricted to one orbital)
    dims, v = (4, 5, 3), 0.2
    h = ham.ti_hamiltonian(*dims, potential=np.full(int(np.prod(dims)), v))
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M = 48
    qs = np.array([[0, 0, 0], [1 / 4, 2 / 5, 1 / 3], [3 / 4, 1 / 5, 2 / 3], [1 / 2, 3 / 5, 0]])
    for q in qs:
        er, _ = orc.moments_v0(h, a, b, M, vectors.plane_wave_block(dims, 4, [q] * 4, range(4)))
        want = matrix_cheb_diag(bloch_matrix(q, v), a, b, M)
        for alpha in range(4):
            mu = orc.eta_to_mu(er[alpha:alpha + 1])
            np.testing.assert_allclose(mu, want[:, alpha], rtol=0, atol=1e-12)


def test_ldos_clean_lattice_equals_bloch_dos(orc):
    # translation invariance: every site's local DOS (its four orbitals) is
    # the DOS of the clean lattice
    dims, v = (4, 3, 5), -0.4
    h = ham.ti_hamiltonian(*dims, potential=np.full(int(np.prod(dims)), v))
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M = 40
    E = bloch_spectrum(*dims, v=v)
    want = np.array([np.mean(cheb(k, a * (E - b))) for k in range(M)])
    for site in (0, 7, 59):
        er, _ = orc.moments_v0(h, a, b, M, vectors.rows_block(h["n"], range(4 * site, 4 * site + 4)))
        np.testing.assert_allclose(orc.eta_to_mu(er), want, rtol=0, atol=1e-12)


def test_ldos_diagonal_matrix_is_scalar_chebyshev(orc):
    lam = np.linspace(-2.5, 3.0, 23)
    h = ham.diagonal_matrix(lam)
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M = 32
    rows = [0, 5, 22]
    er, _ = orc.moments_v0(h, a, b, M, vectors.rows_block(h["n"], rows))
    for k, i in enumerate(rows):
        np.testing.assert_allclose(orc.eta_to_mu(er[k:k + 1]),
                                   [cheb(n, a * (lam[i] - b)) for n in range(M)], rtol=0, atol=1e-13)
