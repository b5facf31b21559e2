"""Seeded synthetic sparse Hermitian matrices in CSR form.

The main generator builds the topological-insulator Hamiltonian of the
paper's application section (Eq. 1): nearest-neighbour hopping on an
Nx x Ny x Nz cubic lattice with four orbitals per site, the hopping block
across bond j being (Gamma^1 - i Gamma^{j+1})/2 plus its Hermitian conjugate,
and an on-site term V_n Gamma^0 + 2 Gamma^1.

The paper names the matrices only as "4x4 Dirac matrices" and describes V_n
as an external potential, so this module fixes one representation:
Gamma^0 = identity, Gamma^1 = tau_z (x) sigma_0 and Gamma^{2,3,4} =
tau_x (x) sigma_{x,y,z}, with orbital index alpha = 2*tau + sigma.  These are
Hermitian, square to one and anticommute pairwise, and with t = 1 every row
of the periodic lattice has exactly 13 non-zeros, as the paper states
(N_nz ~ 13 N).  The disorder is V_n = gamma*(u_n - 1/2) with u_n drawn from
SplitMix64 stream 0 at index n (uniform in [-gamma/2, gamma/2]).

Row index: i = 4*(x + Nx*(y + Ny*z)) + alpha (orbital fastest).

All functions return a dict with keys n, row_ptr (int64[n+1]), col (int32,
sorted ascending within each row) and val (complex128), plus generator
specific extras.  Nothing here computes anything of the KPM method itself.
"""
import numpy as np

from . import rng

_S0 = np.array([[1, 0], [0, 1]], dtype=np.complex128)
_SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def dirac_matrices():
    """Gamma^0..Gamma^4 in the representation described in the module docstring."""
    g0 = np.eye(4, dtype=np.complex128)
    g1 = np.kron(_SZ, _S0)
    g2 = np.kron(_SX, _SX)
    g3 = np.kron(_SX, _SY)
    g4 = np.kron(_SX, _SZ)
    return g0, g1, g2, g3, g4


def ti_blocks(t=1.0):
    """Hopping blocks of Eq. 1 keyed by site offset (dx, dy, dz).

    Entry H[(n, a), (n + d, b)] = block[d][a, b].  Hopping from site n to
    n + e_j carries -t * A_j with A_j = (Gamma^1 - i Gamma^{j+1})/2 on the
    element H[(n + e_j), (n)], so the row site n sees -t * A_j at offset -e_j
    and the Hermitian conjugate -t * A_j^dagger at offset +e_j.
    """
    g0, g1, g2, g3, g4 = dirac_matrices()
    blocks = {}
    for j, gj in enumerate((g2, g3, g4)):
        a_j = (g1 - 1j * gj) / 2.0
        e = [0, 0, 0]
        e[j] = 1
        blocks[tuple(-v for v in e)] = -t * a_j
        blocks[tuple(e)] = -t * a_j.conj().T
    return blocks


def disorder_potential(nx, ny, nz, gamma, seed):
    sites = nx * ny * nz
    u = rng.uniform(seed, rng.STREAM_DISORDER, np.arange(sites, dtype=np.uint64))
    return gamma * (u - 0.5)


def ti_hamiltonian(nx, ny, nz, gamma=0.0, seed=0, t=1.0, periodic=(True, True, True),
                   potential=None, chunk_sites=1 << 20):
    """Topological-insulator Hamiltonian of Eq. 1 as CSR.

    ``periodic`` gives the boundary condition per axis; a periodic axis needs
    at least 3 sites so that the +e_j and -e_j neighbours are distinct.
    ``potential`` (float64[sites]) overrides the seeded disorder.  Sites are
    processed in chunks of ``chunk_sites`` to bound temporary memory.
    """
    dims = (nx, ny, nz)
    for L, p in zip(dims, periodic):
        if L < 1 or (p and L < 3):
            raise ValueError("each periodic axis needs at least 3 sites")
    sites = nx * ny * nz
    n = 4 * sites
    if potential is None:
        potential = disorder_potential(nx, ny, nz, gamma, seed)
    potential = np.asarray(potential, dtype=np.float64)
    g1 = dirac_matrices()[1]
    blocks = ti_blocks(t)
    max_per_row = 1 + sum(int(np.count_nonzero(np.abs(b[0]) > 0)) for b in blocks.values())

    counts = np.empty(n, dtype=np.int64)
    col_parts, val_parts = [], []
    for s0 in range(0, sites, chunk_sites):
        s = np.arange(s0, min(sites, s0 + chunk_sites), dtype=np.int64)
        ns = s.size
        coords = (s % nx, (s // nx) % ny, s // (nx * ny))
        cols = np.full((ns, 4, max_per_row), -1, dtype=np.int64)
        vals = np.zeros((ns, 4, max_per_row), dtype=np.complex128)
        slot = np.zeros(4, dtype=np.int64)
        # on-site diagonal (Gamma^1 is diagonal in this representation)
        for a in range(4):
            cols[:, a, 0] = 4 * s + a
            vals[:, a, 0] = potential[s] + 2.0 * g1[a, a].real
            slot[a] = 1
        for d, blk in blocks.items():
            nb = []
            valid = np.ones(ns, dtype=bool)
            for axis in range(3):
                c = coords[axis] + d[axis]
                L = dims[axis]
                if periodic[axis]:
                    c = c % L
                else:
                    valid &= (c >= 0) & (c < L)
                    c = np.clip(c, 0, L - 1)
                nb.append(c)
            nsite = nb[0] + nx * (nb[1] + ny * nb[2])
            for a in range(4):
                for b in range(4):
                    h = blk[a, b]
                    if h == 0:
                        continue
                    k = slot[a]
                    cols[:, a, k] = np.where(valid, 4 * nsite + b, -1)
                    vals[:, a, k] = np.where(valid, h, 0.0)
                    slot[a] += 1
        cols = cols.reshape(4 * ns, max_per_row)
        vals = vals.reshape(4 * ns, max_per_row)
        key = np.where(cols < 0, np.iinfo(np.int64).max, cols)
        order = np.argsort(key, axis=1, kind="stable")
        cols = np.take_along_axis(cols, order, axis=1)
        vals = np.take_along_axis(vals, order, axis=1)
        keep = cols >= 0
        counts[4 * s0:4 * s0 + 4 * ns] = keep.sum(axis=1)
        col_parts.append(cols[keep].astype(np.int32))
        val_parts.append(vals[keep])
        del cols, vals, key, order, keep
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = col_parts[0] if len(col_parts) == 1 else np.concatenate(col_parts)
    del col_parts
    val = val_parts[0] if len(val_parts) == 1 else np.concatenate(val_parts)
    del val_parts
    return {
        "n": n,
        "row_ptr": row_ptr,
        "col": col,
        "val": val,
        "potential": potential,
        "dims": dims,
        "periodic": tuple(bool(p) for p in periodic),
    }


def cube_row_order(dims, block=(4, 4, 4)):
    """A row ordering (new position -> row) that lists the lattice sites
    block by block (bx x by x bz sites, blocks in x, then y, then z order;
    sites inside a block x-fastest) with the four orbitals of a site kept
    together, so that rows sharing neighbours sit next to each other."""
    nx, ny, nz = dims
    bx, by, bz = block
    s = np.arange(nx * ny * nz, dtype=np.int64)
    x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
    bxn, byn = -(-nx // bx), -(-ny // by)
    blk = (x // bx) + bxn * ((y // by) + byn * (z // bz))
    inner = (x % bx) + bx * ((y % by) + by * (z % bz))
    sites = np.lexsort((inner, blk))
    rows = (4 * sites[:, None] + np.arange(4)[None, :]).ravel()
    return rows.astype(np.int32)


def diagonal_matrix(diag):
    """CSR of a diagonal matrix with the given real diagonal."""
    diag = np.asarray(diag, dtype=np.float64)
    n = diag.size
    return {
        "n": n,
        "row_ptr": np.arange(n + 1, dtype=np.int64),
        "col": np.arange(n, dtype=np.int32),
        "val": diag.astype(np.complex128),
    }


def random_hermitian(n, avg_offdiag, seed, empty_rows=0.0, scale=1.0, diag=True):
    """Random sparse Hermitian matrix with ragged rows.

    Off-diagonal pairs (i, j), i < j, are drawn with probability
    avg_offdiag / n; values are complex, diagonal real.  A fraction
    ``empty_rows`` of rows (and their columns) is left without any entry,
    which exercises zero-length rows and chunks in the sparse converter.
    ``diag=False`` stores no diagonal at all (rows whose own entry the
    converter must supply).  Uses the numpy Generator seeded with ``seed``
    (inputs only).
    """
    g = np.random.default_rng(seed)
    p = min(1.0, avg_offdiag / max(n, 1))
    iu, ju = np.triu_indices(n, k=1)
    pick = g.random(iu.size) < p
    iu, ju = iu[pick], ju[pick]
    vo = (g.standard_normal(iu.size) + 1j * g.standard_normal(iu.size)) * scale / 2
    dv = g.standard_normal(n) * scale
    empty = g.random(n) < empty_rows
    keep = ~(empty[iu] | empty[ju])
    iu, ju, vo = iu[keep], ju[keep], vo[keep]
    di = np.nonzero(~empty)[0] if diag else np.zeros(0, dtype=np.int64)
    rows = np.concatenate([iu, ju, di])
    cols = np.concatenate([ju, iu, di])
    vals = np.concatenate([vo, vo.conj(), dv[di].astype(np.complex128)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    np.cumsum(row_ptr, out=row_ptr)
    return {"n": n, "row_ptr": row_ptr, "col": cols.astype(np.int32), "val": vals}


def to_dense(csr):
    n = csr["n"]
    a = np.zeros((n, n), dtype=np.complex128)
    rp = csr["row_ptr"]
    rows = np.repeat(np.arange(n), np.diff(rp))
    a[rows, csr["col"]] = csr["val"]
    return a


def val_ri(csr):
    """Values as interleaved (re, im) float64, the layout the C interfaces take."""
    return np.ascontiguousarray(csr["val"], dtype=np.complex128).view(np.float64)
