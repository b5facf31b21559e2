"""The row partition of Sec. "Symmetric Heterogeneous Execution" on the CPU:
the library's part layout and exchange lists (kpm_partition_rows,
kpm_partition_build) and a whole row-partitioned KPM-DOS run, parts in one
process with the CPU local step of part_cpu_step, against the oracle's
moments of the unpartitioned matrix."""
import os
import sys

import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from part_cpu_step import CpuPartStep  # noqa: E402


@pytest.fixture(scope="module")
def kpm():
    from paper_1410_5242_gb300 import build
    build.build()
    from paper_1410_5242_gb300 import kpm as k
    return k


@pytest.fixture(scope="module")
def partition(kpm):
    from paper_1410_5242_gb300 import partition as p
    return p


def test_partition_rows_on_planes_with_weights(kpm):
    rs = kpm.partition_rows(4 * 4 * 4 * 10, 3, align=64)
    assert list(rs) == [0, 192, 448, 640]  # planes 3 + 4 + 3 of 10, all whole planes
    rs = kpm.partition_rows(640, 2, align=64, weights=[3.0, 1.0])
    assert list(rs) == [0, 512, 640]  # 3:1 share, rounded to planes
    rs = kpm.partition_rows(640, 10, align=64, weights=[100.0] + [1.0] * 9)
    assert np.all(np.diff(rs) >= 64)  # at least one plane each
    for args in ((640, 11, 64), (650, 2, 64), (640, 0, 64)):
        with pytest.raises(kpm.KPMError):
            kpm.partition_rows(*args)
    with pytest.raises(kpm.KPMError):
        kpm.partition_rows(640, 2, align=64, weights=[1.0, -1.0])


@pytest.mark.parametrize("which", ["lattice", "ragged"])
@pytest.mark.parametrize("parts", [2, 3])
def test_parts_hold_the_rows_and_matching_exchange_lists(kpm, which, parts):
    """Every part's local CSR maps back to its rows of the matrix; the halo
    rows are exactly the other parts' rows its entries read; part k sends to
    part q exactly q's halo slots owned by k, in q's order."""
    if which == "lattice":
        h = ham.ti_hamiltonian(3, 4, 6, gamma=0.7, seed=2)
        rs = kpm.partition_rows(h["n"], parts, align=3 * 4 * 4)
    else:
        h = ham.random_hermitian(301, 6, seed=5, empty_rows=0.05)
        rs = kpm.partition_rows(h["n"], parts)
    P = [kpm.partition_build(h, rs, k) for k in range(parts)]
    for k, p in enumerate(P):
        r0, nl = p["row0"], p["n_local"]
        assert r0 == rs[k] and nl == rs[k + 1] - rs[k]
        c = p["csr"]
        halo = p["halo_rows"]
        assert np.all(np.diff(halo) > 0) and not np.any((halo >= r0) & (halo < r0 + nl))
        read = set()
        for i in range(nl):
            lo, hi = c["row_ptr"][i], c["row_ptr"][i + 1]
            lc = c["col"][lo:hi]
            g = np.where(lc < nl, lc + r0, halo[np.maximum(lc - nl, 0)])
            glo, ghi = h["row_ptr"][r0 + i], h["row_ptr"][r0 + i + 1]
            order = np.argsort(g)
            np.testing.assert_array_equal(g[order], h["col"][glo:ghi])
            np.testing.assert_array_equal(c["val"][lo:hi][order], h["val"][glo:ghi])
            read |= set(int(x) for x in g if x < r0 or x >= r0 + nl)
        assert read == set(int(x) for x in halo)
        for i, q in enumerate(p["peer"]):
            rp = p["recv_ptr"]
            owned = halo[rp[i]:rp[i + 1]]
            assert np.all((owned >= rs[q]) & (owned < rs[q + 1]))
            pq = P[q]
            j = list(pq["peer"]).index(k)
            sent = pq["send_rows"][pq["send_ptr"][j]:pq["send_ptr"][j + 1]] + pq["row0"]
            np.testing.assert_array_equal(sent, owned)


@pytest.mark.parametrize("parts", [2, 3])
def test_partitioned_run_matches_the_oracle(kpm, orc, partition, parts):
    """All parts in one process with the CPU local step: the moments of the
    whole problem to 1e-10 eta_0 (the readings' FP64 tolerance)."""
    h = ham.ti_hamiltonian(4, 3, 6, gamma=0.8, seed=4)
    a, b = orc.scale_from_bounds(*orc.gershgorin(h), 0.01)
    M, R, seed = 40, 3, 7
    rs = partition.slab_row_start(h["n"], parts, plane_rows=4 * 3 * 4)
    steps = [CpuPartStep(p, a, b) for p in partition.build_parts(h, rs)]
    eta, eti = partition.in_process_moments(steps, M, R, seed)
    ref, ref_im = orc.moments(h, a, b, M, seed, range(R))
    eta0 = ref[:, :1]
    assert np.all(np.abs(eta - ref) <= 1e-10 * eta0)
    assert np.all(np.abs(eti) <= 1e-12 * eta0)
