"""GPU tests of the staged sweep kernel in complex double (include/kpm.h,
kpm_launch.stages): the default for every width up to 32 wherever the context
has gather lists (two columns per lane, one at width 1), with R split into
blocks of at most 32 columns.  Two forms: the
general one (four FMAs per entry and column) and the half-complex one for
matrices whose every stored entry is purely real or purely imaginary, such
as the topological insulator of Sec. "Application Scenario" (two FMAs: the
skipped products are exact zeros).  Both must agree with the register-path
kernel to FP64 rounding (1e-13 of max|W| per sweep, the bound the register
path's own sweep tests use), be identical across stage counts, and give
moments within the FP64 parity tolerance of the oracle (1e-10 of eta_0 per
moment, and 1e-10 relative where |eta| >= 1e-3 eta_0)."""
import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


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


def half_complex(h):
    """The same sparsity with every entry made purely real or purely
    imaginary (by a rule symmetric in (i, j), so the matrix stays
    Hermitian; diagonal entries stay real)."""
    n = h["n"]
    rows = np.repeat(np.arange(n), np.diff(h["row_ptr"]))
    cols = h["col"].astype(np.int64)
    v = np.asarray(h["val"], dtype=np.complex128)
    imag = ((rows + cols) % 2 == 1) & (rows != cols)
    val = np.where(imag, 1j * v.imag, v.real + 0j)
    return {"n": n, "row_ptr": h["row_ptr"], "col": h["col"], "val": val}


def peierls(h, t=0.3):
    """The TI matrix with a phase e^{i t} on every hopping above the diagonal
    (e^{-i t} below: still Hermitian), so its entries are general complex."""
    v = np.asarray(h["val"], dtype=np.complex128)
    rows = np.repeat(np.arange(h["n"]), np.diff(h["row_ptr"]))
    phase = np.where(h["col"] > rows, np.exp(1j * t), np.where(h["col"] < rows, np.exp(-1j * t), 1))
    return {"n": h["n"], "row_ptr": h["row_ptr"], "col": h["col"], "val": v * phase}



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


def test_staged_is_the_complex_double_default(kpm):
    h = ham.ti_hamiltonian(8, 8, 8, gamma=0.5, seed=0)
    a, b = scaled(h, kpm)
    with kpm.create(h, a, b) as ctx:
        info = ctx.info()
        assert info["gather_lists"] == 1 and info["half_complex"] == 1
        for R in (8, 16, 32):
            l = ctx.get_launch(R)
            assert l["stages"] == 2 and l["cols_per_lane"] == 2, (R, l)
            assert l["block_threads"] == 32 + 32 * (R // 2)
        assert ctx.max_block_width() == 32
        for R, T, E in ((1, 1, 1), (2, 1, 2), (4, 2, 2)):  # narrow blocks
            l = ctx.get_launch(R)
            assert (l["stages"], l["lanes_per_row"], l["cols_per_lane"]) == (2, T, E), (R, l)
    g = ham.random_hermitian(300, 7, seed=3)
    a, b = scaled(g, kpm)
    with kpm.create(g, a, b) as ctx:
        info = ctx.info()
        assert info["gather_lists"] == 1 and info["half_complex"] == 0
        assert ctx.get_launch(8)["stages"] == 2
    with kpm.create(h, a, b, chunk_height=4) as ctx:  # no gather lists below C = 8
        assert ctx.info()["gather_lists"] == 0 and ctx.info()["half_complex"] == 0
        assert ctx.get_launch(32)["stages"] == 0


@pytest.mark.parametrize("R", [1, 2, 4, 7, 8, 16, 24, 32, 64, 100])
@pytest.mark.parametrize("form", ["half", "general"])
def test_staged_fp64_sweep_matches_register_path(kpm, R, form):
    if form == "half":
        h = ham.ti_hamiltonian(8, 6, 5, gamma=0.8, seed=2)
    else:
        h = ham.random_hermitian(611, 4, seed=R, empty_rows=0.05)
    a, b = scaled(h, kpm)
    g = np.random.default_rng(R)
    V = g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))
    W = g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))
    with kpm.create(h, a, b) as ctx:
        assert ctx.info()["half_complex"] == (1 if form == "half" else 0)
        widths = [w for w in (32, 16, 8, 4, 2, 1) if w <= R]
        rest, plan = R, []
        for w in widths:  # the context's column blocks (at most 32 wide)
            while rest >= w:
                plan.append(w)
                rest -= w
        for init in (False, True):
            ref = first = None
            for stages in (0, 1, 2):
                try:
                    for w in set(plan):
                        e = min(w, 2)
                        if stages:
                            ctx.set_launch(w, w // e, e, 128, stages=stages)
                        else:
                            ctx.set_launch(w, w, 1, 256)  # register path
                except kpm.KPMError as e:
                    # two stages of the random matrix's 32-wide gather lists
                    # (over 200 rows) do not fit in shared memory
                    assert e.status == kpm.KPM_EUNSUPPORTED and stages == 2 and form == "general"
                    continue
                Wg, eg = sweep(ctx, R, V, W, init)
                if ref is None:
                    ref = (Wg, eg)  # the register path
                    continue
                if first is None:
                    first = (Wg, eg)
                assert np.array_equal(Wg, first[0]), (stages, init)
                assert np.array_equal(eg, first[1]), (stages, init)
                scale = np.abs(ref[0]).max()
                np.testing.assert_allclose(Wg, ref[0], rtol=0, atol=1e-13 * scale)
                np.testing.assert_allclose(eg, ref[1], rtol=0, atol=1e-12 * ref[1][0].max())
            assert first is not None


@pytest.mark.parametrize("R", [1, 4, 8, 32, 64])
@pytest.mark.parametrize("form", ["half", "general"])
def test_staged_fp64_moments_match_oracle(kpm, orc, R, form):
    h = ham.ti_hamiltonian(6, 7, 5, gamma=1.5, seed=4)
    if form == "general":
        h = peierls(h)
    a, b = scaled(h, kpm)
    M = 64
    cols = sorted({0, R // 2, R - 1})
    ref, _ = orc.moments(h, a, b, M, 9, cols)
    with kpm.create(h, a, b) as ctx:
        assert ctx.info()["half_complex"] == (1 if form == "half" else 0)
        assert ctx.get_launch(min(R, 32))["stages"] == 2
        eta = ctx.moments(M, R, 9)
    check_eta_fp64(eta[cols], ref)


def test_staged_fp64_ragged_half_and_general(kpm, orc):
    # rows of different lengths, empty rows, padding rows; C = 8, 16 and 64
    # (gather lists past the inline runs at C = 64, where one stage of
    # 16-wide rows fits), both forms
    g = ham.random_hermitian(517, 9, seed=13, empty_rows=0.08)
    M, R = 40, 16
    for h, half in ((g, 0), (half_complex(g), 1)):
        a, b = scaled(h, kpm)
        ref, _ = orc.moments(h, a, b, M, 5, range(R))
        for C in (8, 16, 64):
            for sigma in (1, 64):
                with kpm.create(h, a, b, chunk_height=C, sigma=sigma) as ctx:
                    assert ctx.info()["half_complex"] == half
                    if C == 64:
                        ctx.set_launch(R, R // 2, 2, 128, stages=1)
                    assert ctx.get_launch(R)["stages"] >= 1
                    eta = ctx.moments(M, R, 5)
                check_eta_fp64(eta, ref)


@pytest.mark.parametrize("form", ["half", "general"])
def test_staged_fp64_many_chunks_per_block(kpm, orc, form):
    """16^3 lattice: 512 chunks of 32 rows over at most 456 blocks, so blocks
    take several chunks and the old W of a block's next chunk is read while
    it works on the current one."""
    h = ham.ti_hamiltonian(16, 16, 16, gamma=1.0, seed=6)
    if form == "general":
        h = peierls(h)
    a, b = scaled(h, kpm)
    for R in (8, 32):
        g = np.random.default_rng(R)
        V = g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))
        W = g.standard_normal((h["n"], R)) + 1j * g.standard_normal((h["n"], R))
        with kpm.create(h, a, b) as ctx:
            assert ctx.info()["half_complex"] == (1 if form == "half" else 0)
            l = ctx.get_launch(R)
            assert l["stages"] == 2
            assert ctx.info()["n_chunks"] > l["blocks_per_sm"] * 152  # blocks take 2 or more
            Ws, es = sweep(ctx, R, V, W, False)
            ctx.set_launch(R, R, 1, 256)  # register path
            Wr, er = sweep(ctx, R, V, W, False)
        np.testing.assert_allclose(Ws, Wr, rtol=0, atol=1e-13 * np.abs(Wr).max())
        np.testing.assert_allclose(es, er, rtol=0, atol=1e-12 * er[0].max())
    M, R = 48, 32
    cols = [0, 17, 31]
    ref, _ = orc.moments(h, a, b, M, 3, cols)
    with kpm.create(h, a, b) as ctx:
        eta = ctx.moments(M, R, 3)
    check_eta_fp64(eta[cols], ref)
