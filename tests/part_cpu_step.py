"""A part's local sweeps on the CPU for the tests of the row-partitioned run
(paper_1410_5242_gb300.partition): the same interface as GpuPartStep, with
the local fused step written out in numpy/scipy in double precision from its
definition (Fig. 5 on the part's rows: W <- 2a(H V - b V) - W over the local
rows, V extended by the halo rows; the initial step a(H V - b V); <V|V> and
<W|V> over the local rows).  Test infrastructure only: the library's path
is GpuPartStep."""
import numpy as np
import scipy.sparse as sp

from kpm_inputs import vectors


class CpuPartStep:
    def __init__(self, part, a, b):
        c = part["csr"]
        nl, nh = part["n_local"], part["n_halo"]
        self.H = sp.csr_matrix((c["val"], c["col"], c["row_ptr"]), shape=(nl, nl + nh))
        self.a, self.b = a, b
        self.part = part

    def start(self, R, sweeps, seed):
        p = self.part
        nl, nh, r0 = p["n_local"], p["n_halo"], p["row0"]
        full = vectors.random_phase_block(seed, p["n"], range(R))  # by global row
        self.V = np.zeros((nl + nh, R), dtype=np.complex128)
        self.V[:nl] = full[r0:r0 + nl]
        self.W = np.zeros_like(self.V)
        self.eta = np.zeros((sweeps, 3, R))
        self.m = 0
        self.R = R

    def pack(self, q):
        import torch
        sp_ = self.part["send_ptr"]
        rows = self.part["send_rows"][sp_[q]:sp_[q + 1]]
        return torch.from_numpy(np.ascontiguousarray(self.V[rows]).view(np.uint8).reshape(-1).copy())

    def recv_bytes(self, q):
        rp = self.part["recv_ptr"]
        return int(rp[q + 1] - rp[q]) * self.R * 16

    def unpack(self, q, buf):
        rp = self.part["recv_ptr"]
        nl = self.part["n_local"]
        rows = np.ascontiguousarray(buf.numpy()).view(np.complex128).reshape(-1, self.R)
        self.V[nl + rp[q]:nl + rp[q + 1]] = rows

    def sweep(self):
        nl = self.part["n_local"]
        a, b = self.a, self.b
        Vl = self.V[:nl]
        u = self.H @ self.V
        if self.m == 0:
            Wl = a * (u - b * Vl)
        else:
            Wl = 2 * a * (u - b * Vl) - self.W[:nl]
        self.W[:nl] = Wl
        wv = np.sum(np.conj(Wl) * Vl, axis=0)
        self.eta[self.m] = [np.sum(np.abs(Vl) ** 2, axis=0), wv.real, wv.imag]
        self.V, self.W = self.W, self.V
        self.m += 1

    def partial_eta(self):
        return self.eta
