"""Row-partitioned KPM-DOS (Sec. "Symmetric Heterogeneous Execution"): the
rows of H are split into contiguous parts, one per process (z-slabs of the
lattice of Eq. 1 when the boundaries sit on whole planes); before every
sweep each part receives the rows of the vector block its rows read from
other parts -- the halo -- and the scalar products are summed over the parts
once, at the end, like the single global reduction of Table III.

The layout and the exchange lists come from the library
(kpm_partition_rows, kpm_partition_build).  A part's sweeps run in a
context holding only its rows, with the halo slots after them in every
vector block (kpm_options.n_halo); the halo rows are packed and unpacked on
the device (kpm_halo_pack, kpm_halo_unpack) and the start vectors are drawn
by global row (kpm_block_phases), so the parts together reproduce the
unpartitioned run's moments.

What moves between parts goes through a communicator object with two
methods, ``exchange(sends, recv_counts)`` and ``allreduce_sum(array)``:
TorchComm uses torch.distributed (NCCL between GPUs, gloo on CPU); a run of
all parts inside one process passes the buffers directly (in_process_moments).
"""
import numpy as np

from . import kpm


def slab_row_start(n, parts, plane_rows, weights=None):
    """Boundaries of `parts` contiguous row ranges on whole planes of
    plane_rows rows (kpm_partition_rows)."""
    return kpm.partition_rows(n, parts, align=plane_rows, weights=weights)


def build_parts(csr, row_start):
    """kpm_partition_build for every part."""
    return [kpm.partition_build(csr, row_start, k) for k in range(len(row_start) - 1)]


class GpuPartStep:
    """One part's sweeps on the GPU through libkpm: its local matrix in a
    context with halo slots, its two vector blocks, device-side packing and
    unpacking of the halo, and the per-sweep scalar products in a device
    array [sweeps][3][R]."""

    def __init__(self, part, a, b, precision=kpm.PREC_FP64, device=0, stream=None,
                 chunk_height=32, sigma=256):
        import torch
        self.torch = torch
        self.part = part
        self.stream = stream
        self.ctx = kpm.create(part["csr"], a, b, precision=precision, device=device,
                              chunk_height=chunk_height, sigma=sigma, n_halo=part["n_halo"],
                              global_n=part["n"], row0=part["row0"])
        self.device = device
        npr = len(part["peer"])
        sp = part["send_ptr"]
        self.send_rows = [torch.as_tensor(part["send_rows"][sp[q]:sp[q + 1]], device="cuda")
                          for q in range(npr)]
        self.R = None

    def start(self, R, sweeps, seed):
        torch = self.torch
        self.R = R
        self.V, self.W = self.ctx.new_block(R), self.ctx.new_block(R)
        self.row_bytes = self.ctx.block_bytes(R) // (self.ctx.info()["n_pad"] + self.part["n_halo"])
        self.ctx.block_phases(R, seed, self.V, stream=self.stream)
        self.eta = torch.zeros((sweeps, 3, R), dtype=torch.float64, device="cuda")
        self.m = 0

    def pack(self, q):
        """The rows peer q needs, as a device byte tensor."""
        rows = self.send_rows[q]
        buf = self.torch.empty(rows.numel() * self.row_bytes, dtype=self.torch.uint8, device="cuda")
        self.ctx.halo_pack(self.R, self.V, rows, buf, stream=self.stream)
        return buf

    def recv_bytes(self, q):
        rp = self.part["recv_ptr"]
        return int(rp[q + 1] - rp[q]) * self.row_bytes

    def unpack(self, q, buf):
        rp = self.part["recv_ptr"]
        self.ctx.halo_unpack(self.R, self.V, buf, int(rp[q]), int(rp[q + 1] - rp[q]),
                             stream=self.stream)

    def sweep(self):
        self.ctx.aug_spmmv(self.R, self.V, self.W, self.eta[self.m], init=(self.m == 0),
                           with_imag=True, stream=self.stream)
        self.V, self.W = self.W, self.V
        self.m += 1

    def partial_eta(self):
        """This part's scalar products of every sweep, host [sweeps][3][R]."""
        self.torch.cuda.synchronize()
        self.ctx.check_device_error()
        return self.eta.cpu().numpy()

    def close(self):
        self.ctx.close()


def eta_from_sweeps(e):
    """[sweeps][3][R] per-sweep sums (<V|V>, Re<W|V>, Im<W|V>) to eta [R][M]
    and Im eta [R][M]: sweep m gives eta_{2m} and eta_{2m+1} (Fig. 5)."""
    sweeps, _, R = e.shape
    eta = np.empty((R, 2 * sweeps))
    eti = np.zeros((R, 2 * sweeps))
    eta[:, 0::2] = e[:, 0, :].T
    eta[:, 1::2] = e[:, 1, :].T
    eti[:, 1::2] = e[:, 2, :].T
    return eta, eti


class TorchComm:
    """The exchange through torch.distributed: point-to-point sends and
    receives between peers (isend/irecv, waited for together, so the order
    of peers cannot deadlock), and one all-reduce of the scalar products.
    Device buffers go through the host for the gloo backend."""

    def __init__(self):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.host = dist.get_backend() == "gloo"

    def exchange(self, sends, recv_counts):
        """sends: {peer rank: byte tensor}; recv_counts: {peer rank: bytes}.
        Returns {peer rank: byte tensor} on the senders' device."""
        torch, dist = self.torch, self.dist
        dev = next(iter(sends.values())).device if sends else torch.device("cpu")
        where = "cpu" if self.host else dev
        out = {q: torch.empty(c, dtype=torch.uint8, device=where) for q, c in recv_counts.items()}
        reqs = []
        for q, buf in out.items():
            if buf.numel():
                reqs.append(dist.irecv(buf, src=q))
        for q, buf in sends.items():
            if buf.numel():
                reqs.append(dist.isend(buf.to(where), dst=q))
        for r in reqs:
            r.wait()
        return {q: b.to(dev) for q, b in out.items()}

    def allreduce_sum(self, arr):
        t = self.torch.as_tensor(np.ascontiguousarray(arr))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t.numpy()


def part_moments(step, comm, M, R, seed):
    """This process's part of a row-partitioned KPM-DOS run: eta [R][M] (and
    Im eta) of the whole problem, the same on every process.  Before every
    sweep (the initial one included) the halo of V is exchanged with the
    peers; the per-sweep scalar products are summed over the parts once, at
    the end."""
    if M < 2 or M % 2:
        raise ValueError("M must be even and >= 2")
    part = step.part
    peers = [int(q) for q in part["peer"]]
    step.start(R, M // 2, seed)
    for _ in range(M // 2):
        sends = {q: step.pack(i) for i, q in enumerate(peers)}
        counts = {q: step.recv_bytes(i) for i, q in enumerate(peers)}
        got = comm.exchange(sends, counts)
        for i, q in enumerate(peers):
            step.unpack(i, got[q])
        step.sweep()
    return eta_from_sweeps(comm.allreduce_sum(step.partial_eta()))


def in_process_moments(steps, M, R, seed):
    """All parts of a row-partitioned run in one process (for instance on one
    GPU): the same schedule as part_moments, with each part's halo filled
    from the other parts' packed rows directly.  Returns eta, Im eta."""
    if M < 2 or M % 2:
        raise ValueError("M must be even and >= 2")
    for st in steps:
        st.start(R, M // 2, seed)
    index = {int(st.part["part"]): st for st in steps}
    for _ in range(M // 2):
        packed = {}
        for st in steps:
            k = int(st.part["part"])
            for i, q in enumerate(st.part["peer"]):
                packed[(k, int(q))] = st.pack(i)  # rows part k sends to part q
        for st in steps:
            k = int(st.part["part"])
            for i, q in enumerate(st.part["peer"]):
                st.unpack(i, packed[(int(q), k)])
        for st in steps:
            st.sweep()
    total = sum(st.partial_eta() for st in index.values())
    return eta_from_sweeps(total)
