"""GPU tests of the ways consecutive sweeps overlap (include/kpm.h,
kpm_set_sweep_overlap).

Programmatic dependent launches (KPM_OVERLAP_PDL, the default) change only
when a sweep's blocks start: every result must equal that of plain launches
bit for bit, for the moment calls and for chains of single sweeps.

Sweep chains (KPM_OVERLAP_CHAIN): the sweeps between two eta reductions as one
cooperative launch of the staged kernel, each block starting a chunk of
sweep m once the chunks it depends on are done in sweep m - 1
(kpm_sweep_chain_deps; per-wave completion counters).  Every row is computed as in per-sweep launches, but the odd
sweeps visit the chunks in a half-rotated order, so each block's eta
partial sums cover other chunks: eta must agree with the per-sweep launches
to the rounding of those sums (1e-12 of eta_0 in complex double, 2e-6 in
complex float), and the moments with the oracle within the parity
tolerances.  Cases: both precisions and both entry forms, local (lattice)
and global (random matrix) dependencies, chunk counts that are not
multiples of the grid, every column-block width, reduction batches that
start on odd sweeps, and a batch of one sweep (no chain)."""
import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham
from paper_1410_5242_gb300 import kpm as kpm_mod

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


def peierls(h, t=0.3):
    """General complex entries with the lattice's sparsity (Hermitian)."""
    v = np.asarray(h["val"], dtype=np.complex128)
    rows = np.repeat(np.arange(h["n"]), np.diff(h["row_ptr"]))
    ph = np.where(h["col"] > rows, np.exp(1j * t), np.where(h["col"] < rows, np.exp(-1j * t), 1))
    return {"n": h["n"], "row_ptr": h["row_ptr"], "col": h["col"], "val": v * ph}


def run(ctx, M, R, seed, chain):
    """Moments with chains (or per-sweep launches), and the kernels the call
    launched."""
    ctx.set_sweep_overlap(kpm_mod.OVERLAP_CHAIN if chain else kpm_mod.OVERLAP_PDL)
    before = ctx.info()["kernel_launches"]
    eta = ctx.moments(M, R, seed)
    ctx.check_device_error()
    return eta, ctx.info()["kernel_launches"] - before


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
            # the device after each
            V, W = ctx.new_block(R), ctx.new_block(R)
            ctx.block_upload(R, vectors.random_phase_block(5, h["n"], range(R)), V)
            e = torch.zeros((10, 3 * R), dtype=torch.float64, device="cuda")
            for m in range(10):
                ctx.aug_spmmv(R, V, W, e[m], init=(m == 0))
                V, W = W, V
            torch.cuda.synchronize()
            ctx.check_device_error()
            out[mode] = (eta, e.cpu().numpy(), ctx.block_download(R, V))
    for x, y in zip(out[kpm.OVERLAP_NONE], out[kpm.OVERLAP_PDL]):
        np.testing.assert_array_equal(x, y)


def check_chain(eta_c, eta_s, fp64):
    eta0 = eta_s[:, :1]
    tol = 1e-12 if fp64 else 2e-6
    err = np.abs(eta_c - eta_s) / eta0
    assert err.max() <= tol, "max |d eta|/eta_0 = %g" % err.max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("form", ["half", "general"])
def test_chain_matches_per_sweep_launches_and_oracle(kpm, orc, prec, form):
    h = ham.ti_hamiltonian(16, 16, 24, gamma=1.0, seed=4)  # 768 chunks of 32 rows
    if form == "general":
        h = peierls(h)
    a, b = scaled(h, kpm)
    M, R, seed = 96, 32, 7
    cols = [0, 13, 31]
    fp64 = prec == "fp64"
    with kpm.create(h, a, b, precision=kpm.PREC_FP64 if fp64 else kpm.PREC_FP32) as ctx:
        assert ctx.info()["half_complex"] == (1 if form == "half" else 0)
        assert ctx.get_launch(R)["stages"] >= 1
        eta_c, n_c = run(ctx, M, R, seed, True)
        eta_s, n_s = run(ctx, M, R, seed, False)
    # one launch for the 48 sweeps instead of 48
    assert n_s - n_c == M // 2 - 1, (n_c, n_s)
    check_chain(eta_c, eta_s, fp64)
    ref, _ = orc.moments(h, a, b, M, seed, cols)
    if fp64:
        err = np.abs(eta_c[cols] - ref)
        assert np.all(err <= FP64_TOL * ref[:, :1])
    else:
        assert np.abs(kpm.eta_to_mu(eta_c[cols]) - orc.eta_to_mu(ref)).max() <= FP32_MU_TOL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_chain_with_global_dependencies(kpm, orc, prec):
    # a random sparse matrix: every chunk reads rows spread over the whole
    # matrix, so each chained sweep waits for nearly all of the previous one
    g = ham.random_hermitian(96000, 4, seed=11, empty_rows=0.02)  # 3,000 chunks
    a, b = scaled(g, kpm)
    M, R, seed = 40, 16, 3
    fp64 = prec == "fp64"
    with kpm.create(g, a, b, precision=kpm.PREC_FP64 if fp64 else kpm.PREC_FP32) as ctx:
        if ctx.get_launch(R)["stages"] < 1:
            pytest.skip("this matrix's gather lists leave the staged kernel out")
        eta_c, n_c = run(ctx, M, R, seed, True)
        eta_s, n_s = run(ctx, M, R, seed, False)
    assert n_c < n_s
    check_chain(eta_c, eta_s, fp64)
    cols = [0, 15]
    ref, _ = orc.moments(g, a, b, M, seed, cols)
    if fp64:
        assert np.all(np.abs(eta_c[cols] - ref) <= FP64_TOL * ref[:, :1])
    else:
        assert np.abs(kpm.eta_to_mu(eta_c[cols]) - orc.eta_to_mu(ref)).max() <= FP32_MU_TOL


@pytest.mark.parametrize("R", [8, 16, 24, 64, 100])
def test_chain_every_block_width(kpm, R):
    # 3,072 chunks (not a multiple of any grid here); R = 24 and 100 split
    # into column blocks of different widths, each its own chain
    h = ham.ti_hamiltonian(32, 32, 24, gamma=0.8, seed=2)
    a, b = scaled(h, kpm)
    M, seed = 24, 5
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        eta_c, n_c = run(ctx, M, R, seed, True)
        eta_s, n_s = run(ctx, M, R, seed, False)
    assert n_c < n_s
    check_chain(eta_c, eta_s, False)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_chain_reduction_batches_from_odd_sweeps(kpm, prec):
    # batches of 3 sweeps (m0 = 0, 3, 6, 9: two start on odd sweeps, whose V
    # is the second block) and a last batch of one sweep, launched alone
    h = ham.ti_hamiltonian(16, 16, 24, gamma=1.3, seed=8)
    a, b = scaled(h, kpm)
    M, R, seed = 20, 32, 9
    fp64 = prec == "fp64"
    with kpm.create(h, a, b, precision=kpm.PREC_FP64 if fp64 else kpm.PREC_FP32) as ctx:
        ctx.set_reduce_interval(3)
        eta_c, n_c = run(ctx, M, R, seed, True)
        eta_s, n_s = run(ctx, M, R, seed, False)
        ctx.set_reduce_interval(0)
        eta_1, _ = run(ctx, M, R, seed, True)  # one batch of 10 sweeps
    # 4 batches: 3 chains of 3 sweeps and one single sweep
    assert n_s - n_c == 3 * 2, (n_c, n_s)
    check_chain(eta_c, eta_s, fp64)
    check_chain(eta_1, eta_s, fp64)


def test_chain_off_below_two_chunks_per_block(kpm):
    # 6^3 sites: fewer chunks than two per block of the launch, so the
    # moments run per-sweep launches whatever the switch says
    h = ham.ti_hamiltonian(6, 6, 6, gamma=0.5, seed=1)
    a, b = scaled(h, kpm)
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        eta_c, n_c = run(ctx, 16, 32, 1, True)
        eta_s, n_s = run(ctx, 16, 32, 1, False)
    assert n_c == n_s
    np.testing.assert_array_equal(eta_c, eta_s)
