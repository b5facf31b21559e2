"""GPU tests of the staged sweep kernel (complex float storage; the V rows
each SELL chunk gathers are copied once into shared memory by bulk copies,
see include/kpm.h, kpm_launch.stages): the updated W must agree with the
register-path kernel's to single-precision rounding (the staged kernel sums
the real- and imaginary-part products of a row in two paired accumulators,
the register path in one chain) and be identical across stage counts, eta
must agree with it to the same rounding, and the moments must match the
FP64 oracle within the FP32-form tolerance, for every stage count, block
width, column-block split and row ordering."""
import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham
from kpm_inputs import vectors

pytestmark = pytest.mark.gpu

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


def random_block(n, R, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((n, R)) + 1j * g.standard_normal((n, R))


def sweep(ctx, R, V, W, init):
    import torch
    dV, dW = ctx.new_block(R), ctx.new_block(R)
    ctx.block_upload(R, V, dV)
    ctx.block_upload(R, W, dW)
    eta = torch.zeros(3 * R, dtype=torch.float64, device="cuda")
    ctx.aug_spmmv(R, dV, dW, eta, init=init)
    torch.cuda.synchronize()
    ctx.check_device_error()
    return ctx.block_download(R, dW), eta.cpu().numpy().reshape(3, R)


def test_staged_is_the_complex_float_default(kpm):
    h = ham.ti_hamiltonian(8, 8, 8, gamma=0.5, seed=0)
    a, b = scaled(h, kpm)
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        for R in (8, 16, 32, 64):
            l = ctx.get_launch(R)
            assert l["stages"] >= 2 and l["cols_per_lane"] == 4, (R, l)
            assert l["block_threads"] == 32 + 32 * (R // 4)
        for R in (2, 4):  # the whole row in one lane
            l = ctx.get_launch(R)
            assert l["stages"] >= 2 and l["lanes_per_row"] == 1 and l["cols_per_lane"] == R, l
            assert l["block_threads"] == 32 + 32
        assert ctx.get_launch(1)["stages"] == 0  # width 1: register path
    with kpm.create(h, a, b, chunk_height=4) as ctx:
        assert ctx.get_launch(32)["stages"] == 0  # no gather lists: register path


@pytest.mark.parametrize("R", [2, 4, 7, 8, 16, 24, 32, 64, 100])
@pytest.mark.parametrize("order", ["lattice", "cube"])
def test_staged_sweep_matches_register_path(kpm, R, order):
    dims = (8, 6, 5)
    h = ham.ti_hamiltonian(*dims, gamma=0.8, seed=2)
    a, b = scaled(h, kpm)
    row_order = ham.cube_row_order(dims, block=(2, 2, 2)) if order == "cube" else None
    g = np.random.default_rng(R)
    V = g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))
    W = g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))
    with kpm.create(h, a, b, precision=kpm.PREC_FP32, row_order=row_order) as ctx:
        widths = [w for w in (64, 32, 16, 8, 4, 2, 1) if R & w]
        for init in (False, True):
            ref = first = None
            for stages in (0, 2, 3, 4):
                try:
                    for w in widths:
                        if w >= 8:
                            ctx.set_launch(w, w // 4, 4, 128, stages=stages)
                        elif w >= 2:  # the whole row in one lane
                            ctx.set_launch(w, 1, w, 128, stages=stages)
                        else:  # width 1 always runs the register path
                            ctx.set_launch(w, 1, w, 128)
                except kpm.KPMError as e:
                    # more stages of 64-wide rows than shared memory holds
                    assert e.status == kpm.KPM_EUNSUPPORTED and stages > 2
                    continue
                Wg, eg = sweep(ctx, R, V, W, init)
                if ref is None:
                    ref = (Wg, eg)  # the register path
                    continue
                if first is None:
                    first = Wg
                assert np.array_equal(Wg, first), (stages, init)
                # a few float roundings of a row's 13 products and the old W
                wscale = np.abs(ref[0]).max()
                np.testing.assert_allclose(Wg, ref[0], rtol=0, atol=4e-6 * wscale)
                np.testing.assert_allclose(eg, ref[1], rtol=0, atol=1e-5 * ref[1][0].max())


@pytest.mark.parametrize("stages", [2, 3, 4])
@pytest.mark.parametrize("R", [2, 4, 8, 32, 64])
def test_staged_moments_match_oracle(kpm, orc, stages, R):
    h = ham.ti_hamiltonian(6, 7, 5, gamma=1.5, seed=4)
    a, b = scaled(h, kpm)
    M = 64
    cols = [0, R - 1]
    ref, _ = orc.moments(h, a, b, M, 9, cols)
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        try:
            if R >= 8:
                ctx.set_launch(R, R // 4, 4, 128, stages=stages)
            else:
                ctx.set_launch(R, 1, R, 128, stages=stages)
        except kpm.KPMError as e:
            assert e.status == kpm.KPM_EUNSUPPORTED and stages > 2
            pytest.skip("%d stages of %d-wide rows do not fit in shared memory" % (stages, R))
        eta = ctx.moments(M, R, 9)
    dmu = np.abs(kpm.eta_to_mu(eta[cols]) - orc.eta_to_mu(ref)).max()
    assert dmu <= FP32_MU_TOL, dmu


def test_staged_ragged_matrix(kpm, orc):
    # rows of different lengths, empty rows, padding rows, C = 8, 16 and 64
    # (gather lists past the inline runs at C = 64)
    h = ham.random_hermitian(517, 9, seed=13, empty_rows=0.08)
    a, b = scaled(h, kpm)
    M, R = 40, 16
    ref, _ = orc.moments(h, a, b, M, 5, range(R))
    for C in (8, 16, 64):  # C = 8: one consumer warp per block
        for sigma in (1, 64):
            with kpm.create(h, a, b, precision=kpm.PREC_FP32, chunk_height=C, sigma=sigma) as ctx:
                assert ctx.get_launch(R)["stages"] >= 2
                eta = ctx.moments(M, R, 5)
            dmu = np.abs(kpm.eta_to_mu(eta) - orc.eta_to_mu(ref)).max()
            assert dmu <= FP32_MU_TOL, (C, sigma, dmu)


def test_staged_full_size_sweep_matches_register_path(kpm):
    """64^3 lattice (N = 1,048,576), R = 32 in the bench's launch: W and eta
    of one sweep against the register path, to float rounding."""
    import torch
    h = ham.ti_hamiltonian(64, 64, 64, gamma=1.0, seed=2)
    a, b = scaled(h, kpm)
    R = 32
    V = vectors.random_phase_block(2, h["n"], range(R))
    g = np.random.default_rng(1)
    W = (g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))).astype(np.complex64)
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        assert ctx.get_launch(R)["stages"] >= 2
        Ws, es = sweep(ctx, R, V, W, False)
        ctx.set_launch(R, 8, 4, 128, stages=0)
        Wr, er = sweep(ctx, R, V, W, False)
    np.testing.assert_allclose(Ws, Wr, rtol=0, atol=4e-6 * np.abs(Wr).max())
    np.testing.assert_allclose(es, er, rtol=0, atol=1e-5 * er[0].max())
    torch.cuda.synchronize()


def test_staged_bounded_wait_expires_and_context_recovers(kpm):
    """The staged kernel's waits are bounded: with the producer stopped after
    one chunk per block (test hook), the consumers' wait for the second stage
    expires after about two seconds, the launch records KPM_ETIMEOUT in the
    context's error word, and the context computes correctly afterwards."""
    import time

    import torch
    h = ham.ti_hamiltonian(16, 16, 16, gamma=0.5, seed=1)  # 512 chunks: > 1 per block
    a, b = scaled(h, kpm)
    R = 32
    g = np.random.default_rng(3)
    V = g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))
    W = g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        assert ctx.get_launch(R)["stages"] >= 1
        want, want_eta = sweep(ctx, R, V, W, False)
        ctx.test_stall_staged(1)
        dV, dW = ctx.new_block(R), ctx.new_block(R)
        ctx.block_upload(R, V, dV)
        ctx.block_upload(R, W, dW)
        eta = torch.zeros(3 * R, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        ctx.aug_spmmv(R, dV, dW, eta)
        torch.cuda.synchronize()
        waited = time.perf_counter() - t0
        with pytest.raises(kpm.KPMError) as e:
            ctx.check_device_error()
        assert e.value.status == kpm.KPM_ETIMEOUT
        assert 0.5 < waited < 30.0
        ctx.check_device_error()  # read and cleared
        ctx.test_stall_staged(-1)
        got, got_eta = sweep(ctx, R, V, W, False)
    assert np.array_equal(got, want)
    assert np.array_equal(got_eta, want_eta)


def test_staged_bounded_wait_in_a_two_problem_ensemble(kpm):
    """The bounded waits of a staged launch over a table of two problems (one
    ensemble class).  With two lattices of 256 chunks each and between 256
    and 512 blocks, each block's second chunk belongs to the second problem,
    so in the stalled launch the consumer warps cross a problem boundary --
    and the eta flush there, the only barrier among them -- at the stage
    that never arrives.  The launches must end with KPM_ETIMEOUT (every wait
    gives up, no barrier is left short), and a batch built afterwards on the
    same contexts gives the moments of one built before, bit for bit."""
    import time

    import torch
    R, M = 32, 4
    ctxs = []
    for seed in (1, 2):
        h = ham.ti_hamiltonian(16, 16, 8, gamma=0.5, seed=seed)  # 256 chunks of 32 rows
        a, b = scaled(h, kpm)
        ctxs.append(kpm.create(h, a, b, precision=kpm.PREC_FP32))
    launch = ctxs[0].get_launch(R)
    assert launch["stages"] >= 1
    grid = launch["blocks_per_sm"] * torch.cuda.get_device_properties(0).multi_processor_count
    assert 256 < grid < 512, grid
    try:
        with kpm.Batch(ctxs, [M, M], [R, R], [5, 6]) as batch:
            batch.launch()
            want = [batch.eta(0), batch.eta(1)]
        ctxs[0].test_stall_staged(1)  # captured by batches built from now on
        with kpm.Batch(ctxs, [M, M], [R, R], [5, 6]) as batch:
            t0 = time.perf_counter()
            batch.launch()
            with pytest.raises(kpm.KPMError) as e:
                batch.eta(0)
            waited = time.perf_counter() - t0
        assert e.value.status == kpm.KPM_ETIMEOUT
        assert 0.5 < waited < 60.0
        ctxs[0].test_stall_staged(-1)
        with kpm.Batch(ctxs, [M, M], [R, R], [5, 6]) as batch:
            batch.launch()
            got = [batch.eta(0), batch.eta(1)]
    finally:
        for c in ctxs:
            c.close()
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def gamma_k(k):
    """gamma_k = k u / (1 - k u), u = 2^-24: the bound on the relative error
    of a sum of k rounded operations in single precision (Higham, Accuracy
    and Stability of Numerical Algorithms, Sec. 3.1)."""
    u = 2.0 ** -24
    return k * u / (1 - k * u)


@pytest.mark.parametrize("R", [32, 64])
def test_staged_float_eta_error_bound_on_a_wide_dynamic_range(kpm, orc, R):
    """The complex float form's eta accumulation against its error bound.
    Each lane sums the products of at most 8 rows per column in one FMA chain
    (16 rounded FMAs), the lanes of a warp's rows are added by an xor
    butterfly (log2(32/T) roundings: 2 at R = 32, 1 at R = 64), and
    everything after that is exact to O(u^2) (float-float pairs, then
    double).  So |eta_gpu - eta| <= gamma_18 * sum_i |terms_i|.  Rows of V
    and W are scaled by 10^U(-4, 4), where a single-precision running sum
    over the 1M rows fails that bound (checked below): <V|V> against the
    oracle on the same single-precision V, <W|V> against its definition in
    double on the W the kernel wrote."""
    import torch
    h = ham.ti_hamiltonian(64, 64, 64, gamma=1.0, seed=5)
    a, b = scaled(h, kpm)
    n = h["n"]
    g = np.random.default_rng(21)
    scale = 10.0 ** g.uniform(-4, 4, size=(n, 1))
    V = (scale * vectors.random_phase_block(5, n, range(R))).astype(np.complex64)
    W = (10.0 ** g.uniform(-4, 4, size=(n, 1)) * random_block(n, R, 6)).astype(np.complex64)
    V, W = V.astype(np.complex128), W.astype(np.complex128)
    with kpm.create(h, a, b, precision=kpm.PREC_FP32) as ctx:
        assert ctx.get_launch(R)["stages"] >= 1
        Wg, eg = sweep(ctx, R, V, W, False)
    bound = gamma_k(18)
    cols = [0, 7, R // 2, R - 1]
    for r in cols:
        _, e_ref = orc.aug_spmv(h, a, b, V[:, r], W[:, r])
        vv = e_ref[0]
        assert abs(eg[0, r] - vv) <= bound * vv, (r, abs(eg[0, r] - vv) / vv)
        # a single-precision running sum of the same terms misses the bound
        t = (V[:, r].real ** 2 + V[:, r].imag ** 2).astype(np.float32)
        naive = float(np.cumsum(t, dtype=np.float32)[-1])
        assert abs(naive - vv) > bound * vv
    w, v = Wg, V
    re_terms = np.abs(w.real * v.real) + np.abs(w.imag * v.imag)
    im_terms = np.abs(w.real * v.imag) + np.abs(w.imag * v.real)
    wv = np.sum(w.real * v.real + w.imag * v.imag, axis=0)
    wvi = np.sum(w.real * v.imag - w.imag * v.real, axis=0)
    assert np.all(np.abs(eg[1] - wv) <= bound * re_terms.sum(axis=0))
    assert np.all(np.abs(eg[2] - wvi) <= bound * im_terms.sum(axis=0))
