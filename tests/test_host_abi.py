"""CPU tests of libkpm's C interface: the library loads and exports every
function include/kpm.h declares, the host-only calls agree with the oracle,
the SELL-C-sigma converter reproduces H' = 2a(H - b 1) exactly, and bad
input is rejected with the documented status codes.  No GPU is touched."""
import ctypes
import os
import re

import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham
from paper_1410_5242_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kpm():
    pkg_build.build()
    from paper_1410_5242_gb300 import kpm as k
    return k


def header_functions():
    text = open(os.path.join(ROOT, "include", "kpm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kpm_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function(kpm):
    names = header_functions()
    assert len(names) >= 20
    so = ctypes.CDLL(kpm.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_checked_build_compiles_and_exports_every_declared_function(kpm):
    # the KPM_CHECK build (bounds checks in the staged sweep) is a second
    # library; without a GPU only its exports and its self-report are checked
    from paper_1410_5242_gb300 import build
    path = build.build(check=True)
    assert path.endswith("libkpm_check.so") and path != kpm.LIB_PATH
    so = ctypes.CDLL(path)
    missing = [n for n in header_functions() if not hasattr(so, n)]
    assert not missing, missing
    so.kpm_checked_build.restype = ctypes.c_int
    assert so.kpm_checked_build() == 1 and kpm.lib.kpm_checked_build() == 0
    so.kpm_test_corrupt_record.restype = ctypes.c_int
    so.kpm_test_corrupt_record.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32]
    assert so.kpm_test_corrupt_record(None, 0, 0, 0, 0) == kpm.KPM_EINVAL
    assert kpm.lib.kpm_test_corrupt_record(None, 0, 0, 0, 0) == kpm.KPM_EUNSUPPORTED


def test_gershgorin_and_scale_match_oracle(kpm, orc):
    for h in (ham.ti_hamiltonian(5, 4, 3, gamma=1.3, seed=2),
              ham.random_hermitian(90, 6, seed=1, empty_rows=0.1)):
        assert kpm.gershgorin(h) == orc.gershgorin(h)
        lo, hi = kpm.gershgorin(h)
        assert kpm.scale_from_bounds(lo, hi, 0.01) == orc.scale_from_bounds(lo, hi, 0.01)


def test_eta_to_mu_matches_oracle(kpm, orc):
    g = np.random.default_rng(3)
    eta = g.uniform(-1, 1, (5, 40)) * 100
    eta[:, 0] = g.uniform(50, 100, 5)
    np.testing.assert_allclose(kpm.eta_to_mu(eta), orc.eta_to_mu(eta), rtol=0, atol=1e-14)


@pytest.mark.parametrize("M,K", [(16, 64), (512, 1024), (4096, 4096)])
def test_dos_matches_oracle(kpm, orc, M, K):
    g = np.random.default_rng(M)
    mu = np.concatenate([[1.0], g.uniform(-0.2, 0.2, M - 1) / np.sqrt(1 + np.arange(1, M))])
    e1, r1 = kpm.dos(mu, K, 0.2, -0.4)
    e2, r2 = orc.dos(mu, K, 0.2, -0.4)
    np.testing.assert_array_equal(e1, e2)
    np.testing.assert_allclose(r1, r2, rtol=0, atol=1e-11 * np.abs(r2).max())


def _fold_reference(h, a, b):
    """2a(H - b 1) by the definition, with a stored diagonal everywhere."""
    n = h["n"]
    d = ham.to_dense(h)
    two_a = 2.0 * a
    out = np.zeros_like(d)
    nz = d != 0
    out[nz] = d[nz] * two_a
    diag = np.diag(d)
    out[np.arange(n), np.arange(n)] = (diag.real - b) * two_a + 1j * (diag.imag * two_a)
    return out


def _row_lengths(h, b):
    """Stored length of each row of H': the CSR row plus an inserted
    diagonal where H has none and b != 0."""
    n, rp, col = h["n"], h["row_ptr"], h["col"]
    has_diag = np.array([(col[rp[i]:rp[i + 1]] == i).any() for i in range(n)])
    return np.diff(rp) + ((~has_diag) & (b != 0)).astype(np.int64)


def _unpack(sell, rowlen):
    """Dense matrix in the original numbering, checking the layout on the way:
    perm is a permutation, entries beyond a row's length are padding (value
    0, the row's own index), chunk offsets are C * chunk length."""
    n, C = sell["n"], sell["C"]
    perm = sell["perm"]
    assert sorted(perm[:n]) == list(range(n))
    assert np.array_equal(perm[n:], np.arange(n, sell["n_pad"]))
    dense = np.zeros((n, n), dtype=np.complex128)
    for c in range(sell["n_chunks"]):
        base, clen = sell["chunk_ptr"][c], sell["chunk_len"][c]
        assert sell["chunk_ptr"][c + 1] - base == clen * C
        for r in range(C):
            p = c * C + r
            length = rowlen[perm[p]] if p < n else 0
            assert length <= clen
            for j in range(clen):
                e = base + j * C + r
                col, v = sell["col"][e], sell["val"][e]
                if j >= length:
                    assert v == 0 and col == p
                else:
                    dense[perm[p], perm[col]] += v
    return dense


@pytest.mark.parametrize("C,sigma", [(1, 1), (4, 1), (4, 8), (32, 256), (32, 1)])
def test_sell_roundtrip_ragged(kpm, C, sigma):
    h = ham.random_hermitian(203, 7, seed=C + sigma, empty_rows=0.15)
    a, b = 0.37, 0.61
    sell = kpm.sell_build(h, a, b, C=C, sigma=sigma)
    assert sell["n_pad"] % C == 0 and sell["n_pad"] >= h["n"]
    rowlen = _row_lengths(h, b)
    dense = _unpack(sell, rowlen)
    np.testing.assert_array_equal(dense, _fold_reference(h, a, b))
    # sigma-window sort: rows inside each window by non-increasing length
    for w in range(0, h["n"], sigma):
        seg = rowlen[sell["perm"][w:min(h["n"], w + sigma)]]
        assert np.all(np.diff(seg) <= 0) or sigma == 1
    # chunk length = longest row of the chunk
    for c in range(sell["n_chunks"]):
        rows = sell["perm"][c * C:(c + 1) * C]
        rows = rows[rows < h["n"]]
        assert sell["chunk_len"][c] == (rowlen[rows].max() if rows.size else 0)


def test_sell_ti_lattice_is_unpadded_identity(kpm):
    h = ham.ti_hamiltonian(8, 8, 8, gamma=0.5, seed=0)
    a, b = 0.12, 0.03
    sell = kpm.sell_build(h, a, b, C=32, sigma=256)
    assert np.array_equal(sell["perm"], np.arange(h["n"]))   # equal row lengths: stable
    assert sell["n_stored"] == sell["nnz"] == 13 * h["n"]
    assert np.all(sell["chunk_len"] == 13)
    dense = _unpack(sell, _row_lengths(h, b))
    np.testing.assert_array_equal(dense, _fold_reference(h, a, b))


def test_sell_missing_diagonal_is_inserted_only_when_b_nonzero(kpm):
    h = ham.random_hermitian(50, 4, seed=5)
    # drop every diagonal entry
    keep = np.repeat(np.arange(50), np.diff(h["row_ptr"])) != h["col"]
    rows = np.repeat(np.arange(50), np.diff(h["row_ptr"]))[keep]
    h2 = {"n": 50, "col": h["col"][keep], "val": h["val"][keep],
          "row_ptr": np.searchsorted(rows, np.arange(51)).astype(np.int64)}
    s0 = kpm.sell_build(h2, 0.5, 0.0, C=8, sigma=1)
    assert s0["nnz"] == h2["col"].size
    s1 = kpm.sell_build(h2, 0.5, 0.25, C=8, sigma=1)
    assert s1["nnz"] == h2["col"].size + 50
    dense = _unpack(s1, _row_lengths(h2, 0.25))
    np.testing.assert_array_equal(dense, _fold_reference(h2, 0.5, 0.25))


def _bad(h, **kw):
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in h.items()}
    out.update(kw)
    return out


def test_invalid_input_is_rejected(kpm):
    h = ham.ti_hamiltonian(3, 3, 3)
    col = h["col"].copy()
    col[[1, 2]] = col[[2, 1]]                     # unsorted row
    rp = h["row_ptr"].copy()
    rp[5] = rp[4] - 1                             # decreasing row pointer
    val = h["val"].copy()
    val[7] = np.nan
    oob = h["col"].copy()
    oob[0] = h["n"]
    for bad in (_bad(h, col=col), _bad(h, row_ptr=rp), _bad(h, val=val), _bad(h, col=oob)):
        with pytest.raises(kpm.KPMError) as e:
            kpm.gershgorin(bad)
        assert e.value.status == kpm.KPM_EINVAL
        with pytest.raises(kpm.KPMError) as e:
            kpm.sell_build(bad, 0.1, 0.0)
        assert e.value.status == kpm.KPM_EINVAL
    for C in (0, 3, 2048):
        with pytest.raises(kpm.KPMError):
            kpm.sell_build(h, 0.1, 0.0, C=C)
    with pytest.raises(kpm.KPMError):
        kpm.sell_build(h, -0.1, 0.0)
    with pytest.raises(kpm.KPMError):
        kpm.eta_to_mu(np.ones((2, 5)))
    with pytest.raises(kpm.KPMError):
        kpm.dos(np.ones(4), 8, 0.0, 0.0)
    with pytest.raises(kpm.KPMError):
        kpm.scale_from_bounds(2.0, 1.0)


def test_binding_without_the_library_fails_loudly(tmp_path):
    """The package's Python files without their built library: importing the
    binding raises (no fallback path), in both the normal and the checked
    build's selection."""
    import shutil
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = tmp_path / "paper_1410_5242_gb300"
    pkg.mkdir()
    for f in ("__init__.py", "kpm.py", "build.py", "model.py", "partition.py"):
        shutil.copy(os.path.join(root, "paper_1410_5242_gb300", f), pkg / f)
    for check in ("0", "1"):
        env = dict(os.environ, PYTHONPATH=str(tmp_path), KPM_CHECK=check)
        r = subprocess.run([sys.executable, "-c", "import paper_1410_5242_gb300.kpm"],
                           cwd=str(tmp_path), env=env, capture_output=True, text=True,
                           timeout=300)
        assert r.returncode != 0
        assert "ImportError" in r.stderr and "is not built" in r.stderr, r.stderr[-500:]


def test_empty_matrix_and_too_few_planes_are_rejected(kpm):
    """n = 0 has no spectrum to expand (every call takes n >= 1), and a
    partition needs at least one plane of align rows per part."""
    empty = {"n": 0, "row_ptr": np.zeros(1, dtype=np.int64), "col": np.zeros(0, dtype=np.int32),
             "val": np.zeros(0, dtype=np.complex128)}
    for call in (lambda: kpm.gershgorin(empty), lambda: kpm.lanczos_bounds(empty),
                 lambda: kpm.sell_build(empty, 0.1, 0.0), lambda: kpm.gather_build(empty, 0.1, 0.0),
                 lambda: kpm.staged_build(empty, 0.1, 0.0, "half32"),
                 lambda: kpm.Context(empty, 0.1, 0.0, torch_allocator=False)):
        with pytest.raises(kpm.KPMError) as e:
            call()
        assert e.value.status == kpm.KPM_EINVAL
    for n, parts, align in ((0, 1, 1), (1, 2, 1), (12, 4, 4), (10, 2, 4)):
        with pytest.raises(kpm.KPMError) as e:
            kpm.partition_rows(n, parts, align=align)
        assert e.value.status == kpm.KPM_EINVAL
    assert list(kpm.partition_rows(12, 3, align=4)) == [0, 4, 8, 12]


def test_create_rejects_bad_arguments_before_touching_a_device(kpm):
    h = ham.ti_hamiltonian(3, 3, 3)
    col = h["col"].copy()
    col[0] = -1
    for args in ((_bad(h, col=col), 0.1, 0.0), (h, 0.0, 0.0), (h, float("nan"), 0.0)):
        with pytest.raises(kpm.KPMError) as e:
            kpm.Context(*args, torch_allocator=False)
        assert e.value.status == kpm.KPM_EINVAL
    asym = _bad(h)
    asym["val"][3] += 0.5
    with pytest.raises(kpm.KPMError) as e:
        kpm.Context(asym, 0.1, 0.0, check_hermitian=True, torch_allocator=False)
    assert e.value.status == kpm.KPM_ENOTHERMITIAN


def test_create_without_gpu_reports_cuda_error(kpm):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ham.ti_hamiltonian(3, 3, 3)
    with pytest.raises(kpm.KPMError) as e:
        kpm.Context(h, 0.1, 0.0, torch_allocator=False)
    assert e.value.status == kpm.KPM_ECUDA


def test_status_strings(kpm):
    for code in range(0, -7, -1):
        assert kpm.status_string(code).startswith("KPM_")


def test_model_reproduces_paper_numbers():
    from paper_1410_5242_gb300 import model
    gold = {}
    path = os.path.join(ROOT, "tests", "golden", "code_balance.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            key, val, tol = line.split()[:3]
            gold[key] = (float(val), float(tol))
    assert model.sweep_flops(1, 13, 1) == gold["flops_per_row_vector"][0]
    assert model.sweep_bytes(1, 13, 1, 16) == gold["balance_numerator_R1"][0]
    v, t = gold["B_min_R1"]
    assert abs(model.code_balance(13, 1) - v) <= t
    v, t = gold["B_min_Rinf"]
    assert abs(model.code_balance(13, 10 ** 9) - v) <= t
    # Eq. 4 chain: aug_spmmv moves less than aug_spmv, which moves less than naive
    args = (2000, 10 ** 6, 13 * 10 ** 6, 32, 16)
    assert (model.kpm_traffic(*args, variant="aug_spmmv") < model.kpm_traffic(*args, variant="aug_spmv")
            < model.kpm_traffic(*args, variant="naive"))


@pytest.mark.parametrize("which", ["ti", "ragged", "diag"])
def test_lanczos_bounds_contain_spectrum_and_beat_gershgorin(kpm, which):
    h = {"ti": lambda: ham.ti_hamiltonian(5, 6, 6, gamma=1.0, seed=1),
         "ragged": lambda: ham.random_hermitian(300, 6, seed=3, empty_rows=0.05),
         "diag": lambda: ham.diagonal_matrix(np.linspace(-2.0, 5.0, 400))}[which]()
    lam = np.linalg.eigvalsh(ham.to_dense(h))
    glo, ghi = kpm.gershgorin(h)
    lo, hi = kpm.lanczos_bounds(h, steps=40, seed=2)
    assert lo <= lam.min() + 1e-9 * abs(lam.min()) and hi >= lam.max() - 1e-9 * abs(lam.max())
    assert glo <= lo and hi <= ghi
    if which != "diag":   # Gershgorin is exact for a diagonal matrix
        assert (hi - lo) < 0.8 * (ghi - glo)
    # more steps close in on the extreme eigenvalues while still containing them
    lo, hi = kpm.lanczos_bounds(h, steps=120, seed=2)
    assert lo <= lam.min() + 1e-9 * abs(lam.min()) and hi >= lam.max() - 1e-9 * abs(lam.max())
    assert abs(lo - lam.min()) < 1e-3 and abs(hi - lam.max()) < 1e-3


def test_lanczos_bounds_keep_the_recurrence_bounded(kpm, orc):
    h = ham.ti_hamiltonian(6, 6, 6, gamma=1.5, seed=5)
    a, b = kpm.scale_from_bounds(*kpm.lanczos_bounds(h, steps=40, seed=1), 0.01)
    ag, bg = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    assert a > 1.4 * ag                          # finer energy resolution per moment
    er, _ = orc.moments(h, a, b, 512, 3, range(4))
    n = h["n"]
    c = 2 * er - er[:, [0, 1] * 256]
    c[:, :2] = er[:, :2]
    assert np.max(np.abs(c)) <= n * (1 + 1e-9)  # spectrum of a(H - b) inside [-1, 1]


def test_lanczos_bounds_reject_bad_arguments(kpm):
    h = ham.ti_hamiltonian(3, 3, 3)
    with pytest.raises(kpm.KPMError):
        kpm.lanczos_bounds(h, steps=1)


def _expand_runs(gat, c):
    """The gather list of chunk c as row numbers, position by position."""
    rows = []
    for start, count in gat["runs"][gat["run_ptr"][c]:gat["run_ptr"][c + 1]]:
        rows.extend(range(start, start + count))
    return np.array(rows, dtype=np.int64)


@pytest.mark.parametrize("C,order", [(32, None), (8, None), (32, "cube"), (64, None)])
def test_gather_lists_reproduce_the_column_indices(kpm, C, order):
    # every stored entry reads, through its chunk's list, exactly the V row
    # its SELL column index names; each list holds the chunk's own rows
    # first and every other row once, in increasing order
    h = ham.ti_hamiltonian(6, 5, 4, gamma=0.7, seed=3)
    row_order = ham.cube_row_order((6, 5, 4), block=(2, 2, 2)) if order else None
    for m in (h, ham.random_hermitian(203, 5, seed=4, empty_rows=0.05)):
        ro = row_order if m is h else None
        sell, gat = kpm.gather_build(m, 0.1, 0.3, C=C, sigma=1, row_order=ro)
        assert gat["l_max"] == sell["chunk_len"].max()
        u_max = 0
        for c in range(sell["n_chunks"]):
            rows = _expand_runs(gat, c)
            r0 = c * C
            np.testing.assert_array_equal(rows[:C], np.arange(r0, r0 + C))
            rest = rows[C:]
            assert np.all(np.diff(rest) > 0)
            assert not np.any((rest >= r0) & (rest < r0 + C))
            e0, e1 = sell["chunk_ptr"][c], sell["chunk_ptr"][c + 1]
            cols = sell["col"][e0:e1]
            np.testing.assert_array_equal(rows[gat["lidx"][e0:e1]], cols)
            # nothing listed that no entry reads (own rows excepted)
            assert set(rest.tolist()) == set(cols.tolist()) - set(range(r0, r0 + C))
            # adjacent runs are merged
            runs = gat["runs"][gat["run_ptr"][c]:gat["run_ptr"][c + 1]]
            assert np.all(runs[:-1, 0] + runs[:-1, 1] != runs[1:, 0])
            u_max = max(u_max, rows.size)
        assert gat["u_max"] == u_max


def test_gather_lists_of_the_lattice_are_few_runs(kpm):
    # in lattice order a chunk of 8 sites along x reads its own 8 sites, the
    # two x neighbours and 8 sites in each of +-y, +-z: 42 sites in at most
    # 7 runs (fewer where an x neighbour continues the own rows)
    h = ham.ti_hamiltonian(16, 8, 8, gamma=0.5, seed=1)
    sell, gat = kpm.gather_build(h, 0.1, 0.0, C=32, sigma=1)
    nruns = np.diff(gat["run_ptr"])
    assert gat["u_max"] == 42 * 4
    assert np.all(np.diff(gat["run_ptr"]) <= 7)
    assert nruns.min() >= 5


def test_gather_build_rejects_small_chunks(kpm):
    h = ham.ti_hamiltonian(3, 3, 3)
    with pytest.raises(kpm.KPMError) as e:
        kpm.gather_build(h, 0.1, 0.0, C=4, sigma=1)
    assert e.value.status == kpm.KPM_EINVAL


def test_local_and_plane_wave_calls_reject_missing_arguments(kpm):
    # argument checks that need no context run before any device call
    import ctypes
    import numpy as np
    eta = np.empty(16)
    rows = np.zeros(2, dtype=np.int64)
    q = np.zeros(6)
    orb = np.zeros(2, dtype=np.int32)
    pd = eta.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    lib = kpm.lib
    assert lib.kpm_moments_local(None, 8, 2, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 pd, None, None) == kpm.KPM_EINVAL
    assert lib.kpm_moments_plane_wave(None, 8, 2, 2, 2, 2, 4,
                                      q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      orb.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), pd, None,
                                      None) == kpm.KPM_EINVAL


def test_sweep_overlap_and_reduce_interval_reject_bad_arguments(kpm):
    lib = kpm.lib
    for mode in (kpm.OVERLAP_NONE, kpm.OVERLAP_PDL, -1, 2):
        assert lib.kpm_set_sweep_overlap(None, mode) == kpm.KPM_EINVAL
    assert (kpm.OVERLAP_NONE, kpm.OVERLAP_PDL) == (0, 1)
    assert lib.kpm_set_reduce_interval(None, 1) == kpm.KPM_EINVAL


@pytest.mark.parametrize("C,sigma", [(32, 256), (8, 64)])
def test_conversions_do_not_depend_on_the_host_thread_count(kpm, monkeypatch, C, sigma):
    """kpm_sell_build and kpm_gather_build split rows, sorting windows and
    chunks among host threads (KPM_HOST_THREADS caps them): the layout and
    the gather lists must be identical for 1, 3 and 16 threads, on a lattice
    large enough for several parts and with ragged rows (open boundaries)."""
    h = ham.ti_hamiltonian(36, 30, 24, gamma=0.7, seed=5, periodic=(False, True, False))
    a, b = 0.11, 0.07
    got = []
    for t in ("1", "3", "16"):
        monkeypatch.setenv("KPM_HOST_THREADS", t)
        got.append(kpm.gather_build(h, a, b, C=C, sigma=sigma))
    (s0, g0) = got[0]
    assert not np.array_equal(s0["perm"][:s0["n"]], np.arange(s0["n"]))  # the sort moved rows
    for s1, g1 in got[1:]:
        for k in ("chunk_ptr", "chunk_len", "col", "val", "perm"):
            np.testing.assert_array_equal(s1[k], s0[k], err_msg=k)
        assert (s1["nnz"], s1["n_stored"]) == (s0["nnz"], s0["n_stored"])
        for k in ("lidx", "run_ptr", "runs"):
            np.testing.assert_array_equal(g1[k], g0[k], err_msg=k)
        assert (g1["u_max"], g1["l_max"]) == (g0["u_max"], g0["l_max"])


def test_invalid_input_is_rejected_in_any_part(kpm, monkeypatch):
    # errors placed near the end of large inputs, where a later thread's part
    # finds them
    monkeypatch.setenv("KPM_HOST_THREADS", "8")
    h = ham.ti_hamiltonian(32, 32, 32)
    n = h["n"]
    col = h["col"].copy()
    k = h["row_ptr"][n - 2]
    col[[k, k + 1]] = col[[k + 1, k]]
    val = h["val"].copy()
    val[-3] = np.inf
    rp = h["row_ptr"].copy()
    rp[n - 1] = rp[n - 2] - 1
    for bad in (_bad(h, col=col), _bad(h, val=val), _bad(h, row_ptr=rp)):
        with pytest.raises(kpm.KPMError) as e:
            kpm.sell_build(bad, 0.1, 0.0)
        assert e.value.status == kpm.KPM_EINVAL


def test_gershgorin_does_not_depend_on_the_host_thread_count(kpm, monkeypatch):
    h = ham.ti_hamiltonian(40, 30, 20, gamma=1.3, seed=9)
    got = []
    for t in ("1", "5", "16"):
        monkeypatch.setenv("KPM_HOST_THREADS", t)
        got.append(kpm.gershgorin(h))
    assert got[1] == got[0] and got[2] == got[0]


def _region_offsets(C, n, r):
    """Offsets of row r's entries 0..n-1 in a region of n entries per row
    laid out as documented: groups of 8, then of 4, 2, 1 (binary digits of
    n mod 8), a group of g entries starting at j holding row r's entries at
    C*j + g*r."""
    out, j = [], 0
    while j + 8 <= n:
        out += [C * j + 8 * r + e for e in range(8)]
        j += 8
    for g in (4, 2, 1):
        if n - j >= g:
            out += [C * j + g * r + e for e in range(g)]
            j += g
    return out


def _staged_offsets(C, L, r):
    """Index and value offsets (within a chunk of staged length L) of row r's
    entries j = 0..L-1 as the staged layout is documented: the first L - 1
    indices in groups of 8, then of 4, 2, 1 (binary digits of (L-1) mod 8),
    the last (own) entry's index at C*(L-1) + r; complex float values in
    pairs below (L-1) rounded down to even, others at C*j + r."""
    nm = L - 1
    idx, j = [], 0
    while j + 8 <= nm:
        idx += [C * j + 8 * r + e for e in range(8)]
        j += 8
    for g in (4, 2, 1):
        if nm - j >= g:
            idx += [C * j + g * r + e for e in range(g)]
            j += g
    idx.append(C * nm + r)
    np2 = nm & ~1
    valf = [C * (j & ~1) + 2 * r + (j & 1) if j < np2 else C * j + r for j in range(L)]
    vald = [C * j + r for j in range(L)]
    return np.array(idx), np.array(valf), np.array(vald)


@pytest.mark.parametrize("form", [0, 1, 2])
@pytest.mark.parametrize("C", [8, 32])
def test_staged_arrays_hold_each_row_with_its_own_entry_last(kpm, form, C):
    """kpm_staged_build: decoded through the documented layout and the gather
    lists, every row's staged entries are its SELL entries (values rounded to
    float for complex float, operand pairs for the half-complex form) plus
    zero fillers, the last one reading the row's own V row, and the offsets
    of a chunk cover it exactly once."""
    mats = [(ham.ti_hamiltonian(5, 4, 3, gamma=0.7, seed=3), 0.1, 0.3),
            # b = 0 and rows without a diagonal: chunks get one more entry
            (ham.random_hermitian(203, 5, seed=4, empty_rows=0.05, diag=False), 0.1, 0.0)]
    if form == 2:  # the half-complex form needs real or imaginary entries
        mats = mats[:1] + [(ham.ti_hamiltonian(4, 4, 3, gamma=0.0, seed=1), 0.1, 0.0)]
    for m, a, b in mats:
        sell, gat, stg = kpm.staged_build(m, a, b, form, C=C, sigma=1)
        for c in range(sell["n_chunks"]):
            rows = _expand_runs(gat, c)
            L0, L = sell["chunk_len"][c], stg["chunk_len"][c]
            e0, s0 = sell["chunk_ptr"][c], stg["chunk_ptr"][c]
            assert stg["chunk_ptr"][c + 1] - s0 == C * L
            own_missing = False
            covered_i, covered_v = [], []
            for r in range(C):
                p = c * C + r
                sel = [e0 + j * C + r for j in range(L0)]
                has_own = any(sell["col"][e] == p for e in sel)
                own_missing |= not has_own
                oi, ovf, ovd = _staged_offsets(C, L, r)
                covered_i += list(oi)
                covered_v += list(ovf if form == 1 else ovd)
                li = stg["lidx"][s0 + oi].astype(np.int64)
                vals = stg["val"][s0 + (ovf if form == 1 else ovd)]
                if form == 2:
                    imag = (li & 0x8000) != 0
                    li = li & 0x7FFF
                    # operand pairs back to the complex values
                    assert np.all(vals[~imag].real == vals[~imag].imag)
                    assert np.all(vals[imag].real == -vals[imag].imag)
                    vals = np.where(imag, 1j * vals.imag, vals.real + 0j)
                cols = rows[li]
                assert cols[-1] == p  # the own entry comes last
                want = sell["val"][sel]
                if form == 1:
                    want = want.astype(np.complex64).astype(np.complex128)
                got_nz = sorted((int(x), complex(v)) for x, v in zip(cols, vals) if v != 0)
                want_nz = sorted((int(x), complex(v)) for x, v in
                                 zip(sell["col"][sel], want) if v != 0)
                assert got_nz == want_nz
                # zero entries read the row's own V row only where SELL had
                # padding or a filler was added
                zero_cols = [x for x, v in zip(cols, vals) if v == 0]
                assert all(x == p for x in zero_cols) or any(
                    v == 0 for v in sell["val"][sel])
            assert L == L0 + (1 if own_missing else 0)
            assert sorted(covered_i) == list(range(C * L))
            assert sorted(covered_v) == list(range(C * L))
        assert stg["l_max"] == stg["chunk_len"].max()


def test_staged_build_rejects_full_complex_entries_in_the_half_form(kpm):
    h = ham.random_hermitian(64, 4, seed=2)  # general complex off-diagonals
    with pytest.raises(kpm.KPMError) as e:
        kpm.staged_build(h, 0.1, 0.0, kpm.STAGED_HALF, C=8, sigma=1)
    assert e.value.status == kpm.KPM_EINVAL


def test_half_float_staged_arrays_split_real_and_imaginary_entries(kpm):
    """kpm_staged_build, form 3 (half-complex float): decoded through the
    documented two-region layout, every row holds its real SELL entries in
    the real region, its imaginary ones in the imaginary region (one float
    each), zero fillers on its own index, and its own entry last; the
    offsets of a chunk cover it exactly once."""
    C = 32
    for m, a, b in ((ham.ti_hamiltonian(5, 4, 3, gamma=0.7, seed=3), 0.1, 0.3),
                    (ham.ti_hamiltonian(3, 4, 5, gamma=0.0, seed=1,
                                        periodic=(True, True, False)), 0.2, 0.0)):
        sell, gat, stg = kpm.staged_build(m, a, b, kpm.STAGED_HALF32, C=C, sigma=1)
        for c in range(sell["n_chunks"]):
            rows = _expand_runs(gat, c)
            L0, L, nA = sell["chunk_len"][c], stg["chunk_len"][c], stg["chunk_nre"][c]
            nB = L - 1 - nA
            e0, s0 = sell["chunk_ptr"][c], stg["chunk_ptr"][c]
            assert stg["chunk_ptr"][c + 1] - s0 == C * L
            covered = []
            for r in range(C):
                p = c * C + r
                offA = _region_offsets(C, nA, r)
                offB = [C * nA + o for o in _region_offsets(C, nB, r)]
                own = C * (L - 1) + r
                covered += offA + offB + [own]
                colA = rows[stg["lidx"][s0 + np.array(offA, dtype=np.int64)]] if nA else []
                colB = rows[stg["lidx"][s0 + np.array(offB, dtype=np.int64)]] if nB else []
                assert rows[stg["lidx"][s0 + own]] == p
                got = [(int(x), complex(v, 0)) for x, v in zip(colA, stg["val"][s0 + np.array(offA, dtype=np.int64)]) if v != 0] if nA else []
                got += [(int(x), complex(0, v)) for x, v in zip(colB, stg["val"][s0 + np.array(offB, dtype=np.int64)]) if v != 0] if nB else []
                if stg["val"][s0 + own] != 0:
                    got.append((p, complex(stg["val"][s0 + own], 0)))
                sel = [e0 + j * C + r for j in range(L0)]
                want = sell["val"][sel].astype(np.complex64).astype(np.complex128)
                want_nz = [(int(x), complex(v)) for x, v in zip(sell["col"][sel], want) if v != 0]
                assert sorted(got) == sorted(want_nz)
                # fillers read the row's own V row
                for cols, offs in ((colA, offA), (colB, offB)):
                    for x, o in zip(cols, offs):
                        if stg["val"][s0 + o] == 0:
                            assert x == p or any(v == 0 for v in sell["val"][sel])
            assert sorted(covered) == list(range(C * L))


def test_half_float_staged_build_rejects_full_complex_entries(kpm):
    h = ham.random_hermitian(64, 4, seed=2)
    with pytest.raises(kpm.KPMError) as e:
        kpm.staged_build(h, 0.1, 0.0, kpm.STAGED_HALF32, C=8, sigma=1)
    assert e.value.status == kpm.KPM_EINVAL
