"""Thin ctypes binding of libkpm (include/kpm.h): same names, argument
marshalling only.  Every step of the KPM hot path runs inside the library;
nothing here computes moments.  PyTorch supplies device memory (its
caching allocator is passed to the library as the allocator hook) and
streams.

The shared library is built in-tree by ``paper_1410_5242_gb300.build``;
importing this module fails loudly if it is missing.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# KPM_CHECK=1 in the environment: the checked build (bounds checks in the
# staged sweep, include/kpm.h), built by build.build(check=True)
CHECKED = os.environ.get("KPM_CHECK") == "1"
LIB_PATH = os.path.join(_PKG, "_build_check", "libkpm_check.so") if CHECKED else \
    os.path.join(_PKG, "_build", "libkpm.so")

KPM_OK = 0
KPM_EINVAL = -1
KPM_ENOTHERMITIAN = -2
KPM_ENOMEM = -3
KPM_ECUDA = -4
KPM_ETIMEOUT = -5
KPM_EUNSUPPORTED = -6

PREC_FP64 = 0
PREC_FP32 = 1
OVERLAP_NONE = 0   # kpm_set_sweep_overlap modes
OVERLAP_PDL = 1

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("chunk_height", ctypes.c_int32),
                ("sigma", ctypes.c_int32), ("check_hermitian", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("device", ctypes.c_int32),
                ("alloc_fn", ALLOC_FN), ("free_fn", FREE_FN), ("alloc_user", ctypes.c_void_p),
                ("row_order", ctypes.POINTER(ctypes.c_int32)), ("n_halo", ctypes.c_int64),
                ("global_n", ctypes.c_int64), ("row0", ctypes.c_int64)]


class Part(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("row0", ctypes.c_int64), ("n_local", ctypes.c_int64),
                ("n_halo", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_peers", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("row_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("col", ctypes.POINTER(ctypes.c_int32)), ("val_ri", ctypes.POINTER(ctypes.c_double)),
                ("halo_rows", ctypes.POINTER(ctypes.c_int64)),
                ("peer", ctypes.POINTER(ctypes.c_int32)),
                ("recv_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("send_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("send_rows", ctypes.POINTER(ctypes.c_int32))]


class Sell(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_pad", ctypes.c_int64), ("C", ctypes.c_int32),
                ("sigma", ctypes.c_int32), ("n_chunks", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_stored", ctypes.c_int64), ("chunk_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("chunk_len", ctypes.POINTER(ctypes.c_int32)),
                ("col", ctypes.POINTER(ctypes.c_int32)), ("val_ri", ctypes.POINTER(ctypes.c_double)),
                ("perm", ctypes.POINTER(ctypes.c_int32))]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_pad", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_stored", ctypes.c_int64), ("n_chunks", ctypes.c_int64), ("C", ctypes.c_int32),
                ("sigma", ctypes.c_int32), ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("matrix_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("gather_lists", ctypes.c_int32),
                ("half_complex", ctypes.c_int32), ("upload_bytes", ctypes.c_int64)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("steps", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("classes", ctypes.c_int16), ("staged_classes", ctypes.c_int16),
                ("kernel_launches", ctypes.c_int64),
                ("sweeps", ctypes.c_int64), ("algorithmic_bytes", ctypes.c_double)]


class Launch(ctypes.Structure):
    _fields_ = [("lanes_per_row", ctypes.c_int32), ("cols_per_lane", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("tile_groups", ctypes.c_int32), ("stages", ctypes.c_int32)]


class Staged(ctypes.Structure):
    _fields_ = [("n_chunks", ctypes.c_int64), ("n_stored", ctypes.c_int64),
                ("l_max", ctypes.c_int32), ("form", ctypes.c_int32),
                ("chunk_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("chunk_len", ctypes.POINTER(ctypes.c_int32)),
                ("chunk_nre", ctypes.POINTER(ctypes.c_int32)),
                ("lidx", ctypes.POINTER(ctypes.c_uint16)), ("val", ctypes.POINTER(ctypes.c_double)),
                ("valf", ctypes.POINTER(ctypes.c_float))]


class Gather(ctypes.Structure):
    _fields_ = [("n_chunks", ctypes.c_int64), ("n_runs", ctypes.c_int64),
                ("u_max", ctypes.c_int32), ("l_max", ctypes.c_int32),
                ("lidx", ctypes.POINTER(ctypes.c_uint16)), ("run_ptr", ctypes.POINTER(ctypes.c_int64)),
                ("runs", ctypes.POINTER(ctypes.c_int32))]


_i32, _i64, _u64, _d = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
_vp, _pd = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_pi32, _pi64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
_int = ctypes.c_int

_SIGS = {
    "kpm_default_options": (None, [ctypes.POINTER(Options)]),
    "kpm_status_string": (ctypes.c_char_p, [_int]),
    "kpm_gershgorin": (_int, [_i64, _pi64, _pi32, _pd, _pd, _pd]),
    "kpm_scale_from_bounds": (_int, [_d, _d, _d, _pd, _pd]),
    "kpm_lanczos_bounds": (_int, [_i64, _pi64, _pi32, _pd, _i32, _u64, _pd, _pd]),
    "kpm_eta_to_mu": (_int, [_pd, _i32, _i32, _pd]),
    "kpm_dos": (_int, [_pd, _i32, _i32, _d, _d, _pd, _pd]),
    "kpm_sell_build": (_int, [_i64, _pi64, _pi32, _pd, _d, _d, _i32, _i32, _pi32,
                              ctypes.POINTER(Sell)]),
    "kpm_sell_release": (None, [ctypes.POINTER(Sell)]),
    "kpm_gather_build": (_int, [ctypes.POINTER(Sell), ctypes.POINTER(Gather)]),
    "kpm_gather_release": (None, [ctypes.POINTER(Gather)]),
    "kpm_staged_build": (_int, [ctypes.POINTER(Sell), ctypes.POINTER(Gather), _i32,
                                ctypes.POINTER(Staged)]),
    "kpm_staged_release": (None, [ctypes.POINTER(Staged)]),
    "kpm_check_device_error": (_int, [_vp]),
    "kpm_partition_rows": (_int, [_i64, _i32, _pd, _i64, _pi64]),
    "kpm_partition_build": (_int, [_i64, _pi64, _pi32, _pd, _i32, _pi64, _i32,
                                   ctypes.POINTER(Part)]),
    "kpm_partition_release": (None, [ctypes.POINTER(Part)]),
    "kpm_halo_pack": (_int, [_vp, _i32, _vp, _vp, _i32, _vp, _vp]),
    "kpm_halo_unpack": (_int, [_vp, _i32, _vp, _vp, _i64, _i32, _vp]),
    "kpm_block_phases": (_int, [_vp, _i32, _u64, _vp, _vp]),
    "kpm_test_stall_staged": (_int, [_vp, _i64]),
    "kpm_create": (_int, [_i64, _pi64, _pi32, _pd, _d, _d, ctypes.POINTER(Options),
                          ctypes.POINTER(_vp)]),
    "kpm_destroy": (None, [_vp]),
    "kpm_moments": (_int, [_vp, _i32, _i32, _u64, _pd, _pd, _vp]),
    "kpm_moments_v0": (_int, [_vp, _i32, _i32, _pd, _pd, _pd, _vp]),
    "kpm_moments_local": (_int, [_vp, _i32, _i32, _pi64, _pd, _pd, _vp]),
    "kpm_moments_plane_wave": (_int, [_vp, _i32, _i32, _i32, _i32, _i32, _i32, _pd, _pi32, _pd,
                                      _pd, _vp]),
    "kpm_moments_batch": (_int, [ctypes.POINTER(_vp), _i32, _pi32, _pi32,
                                 ctypes.POINTER(_u64), ctypes.POINTER(_pd), _vp]),
    "kpm_get_info": (_int, [_vp, ctypes.POINTER(Info)]),
    "kpm_block_bytes": (_i64, [_vp, _i32]),
    "kpm_block_upload": (_int, [_vp, _i32, _pd, _vp, _vp]),
    "kpm_block_download": (_int, [_vp, _i32, _vp, _pd, _vp]),
    "kpm_aug_spmmv": (_int, [_vp, _i32, _vp, _vp, _vp, _i32, _i32, _vp]),
    "kpm_moments_device": (_int, [_vp, _i32, _i32, _u64, _vp, _vp, _vp]),
    "kpm_aug_spmmv_static": (_int, [_vp, _i32, _vp, _vp, _vp, _i32, _i32, _vp]),
    "kpm_batch_create": (_int, [ctypes.POINTER(_vp), _i32, _pi32, _pi32, ctypes.POINTER(_u64),
                                ctypes.POINTER(_vp)]),
    "kpm_batch_launch": (_int, [_vp, _vp]),
    "kpm_batch_eta": (_int, [_vp, _i32, _pd, _vp]),
    "kpm_batch_get_info": (_int, [_vp, ctypes.POINTER(BatchInfo)]),
    "kpm_batch_destroy": (None, [_vp]),
    "kpm_autotune": (_int, [_vp, _i32, _i32, _vp, ctypes.POINTER(Launch)]),
    "kpm_get_max_block_width": (_int, [_vp]),
    "kpm_autotune_layout": (_int, [_i64, _pi64, _pi32, _pd, _d, _d, ctypes.POINTER(Options), _i32,
                                   _i32, ctypes.POINTER(Options), _pd]),
    "kpm_sweep_variant": (_int, [_vp, _i32, _vp, _vp, _i32, _vp]),
    "kpm_set_reduce_interval": (_int, [_vp, _i32]),
    "kpm_set_sweep_overlap": (_int, [_vp, _i32]),
    "kpm_checked_build": (_int, []),
    "kpm_test_corrupt_record": (_int, [_vp, _i64, _i32, _i32, _i32]),
    "kpm_naive_create": (_int, [_i64, _pi64, _pi32, _pd, _d, _d, _i32, ctypes.POINTER(_vp)]),
    "kpm_naive_moments": (_int, [_vp, _i32, _i32, _u64, _vp, _vp]),
    "kpm_naive_destroy": (None, [_vp]),
    "kpm_get_launch": (_int, [_vp, _i32, ctypes.POINTER(Launch)]),
    "kpm_set_launch": (_int, [_vp, _i32, ctypes.POINTER(Launch)]),
}

if not os.path.exists(LIB_PATH):
    raise ImportError("%s is not built; run paper_1410_5242_gb300.build.build(%s) "
                      "or __graft_entry__.build() first"
                      % (LIB_PATH, "check=True" if CHECKED else ""))
lib = ctypes.CDLL(LIB_PATH)
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class KPMError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s" % (what, lib.kpm_status_string(status).decode()))


def _check(rc, what):
    if rc != KPM_OK:
        raise KPMError(rc, what)


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _csr(csr, n_cols=None):
    # n_cols: a part's local matrix has halo columns past its n rows (checked
    # by the library)
    rp = np.ascontiguousarray(csr["row_ptr"], dtype=np.int64)
    col = np.ascontiguousarray(csr["col"], dtype=np.int32)
    val = np.ascontiguousarray(csr["val"], dtype=np.complex128).view(np.float64)
    return int(csr["n"]), rp, col, val


def status_string(status):
    return lib.kpm_status_string(status).decode()


def default_options():
    o = Options()
    lib.kpm_default_options(ctypes.byref(o))
    return o


# --------------------------------------------------------------- host-only
def gershgorin(csr):
    n, rp, col, val = _csr(csr)
    lo, hi = _d(), _d()
    _check(lib.kpm_gershgorin(n, _p(rp, _i64), _p(col, _i32), _p(val, _d), ctypes.byref(lo),
                              ctypes.byref(hi)), "kpm_gershgorin")
    return lo.value, hi.value


def lanczos_bounds(csr, steps=30, seed=0):
    n, rp, col, val = _csr(csr)
    lo, hi = _d(), _d()
    _check(lib.kpm_lanczos_bounds(n, _p(rp, _i64), _p(col, _i32), _p(val, _d), steps, seed,
                                  ctypes.byref(lo), ctypes.byref(hi)), "kpm_lanczos_bounds")
    return lo.value, hi.value


def scale_from_bounds(emin, emax, eps=0.01):
    a, b = _d(), _d()
    _check(lib.kpm_scale_from_bounds(emin, emax, eps, ctypes.byref(a), ctypes.byref(b)),
           "kpm_scale_from_bounds")
    return a.value, b.value


def eta_to_mu(eta):
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    R, M = eta.shape
    mu = np.empty(M)
    _check(lib.kpm_eta_to_mu(_p(eta, _d), M, R, _p(mu, _d)), "kpm_eta_to_mu")
    return mu


def dos(mu, K, a, b):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    e, rho = np.empty(K), np.empty(K)
    _check(lib.kpm_dos(_p(mu, _d), mu.size, K, a, b, _p(e, _d), _p(rho, _d)), "kpm_dos")
    return e, rho


def sell_build(csr, a, b, C=32, sigma=256, row_order=None):
    """The SELL-C-sigma layout kpm_create would upload, as numpy arrays."""
    n, rp, col, val = _csr(csr)
    s = Sell()
    order = None if row_order is None else np.ascontiguousarray(row_order, dtype=np.int32)
    _check(lib.kpm_sell_build(n, _p(rp, _i64), _p(col, _i32), _p(val, _d), a, b, C, sigma,
                              _p(order, _i32) if order is not None else None, ctypes.byref(s)),
           "kpm_sell_build")
    try:
        out = _sell_dict(s)
    finally:
        lib.kpm_sell_release(ctypes.byref(s))
    return out


def gather_build(csr, a, b, C=32, sigma=256, row_order=None):
    """The SELL layout (as sell_build) and the staged kernel's gather lists of
    kpm_gather_build: (sell dict, {"u_max", "l_max", "lidx", "run_ptr", "runs"})."""
    n, rp, col, val = _csr(csr)
    s = Sell()
    order = None if row_order is None else np.ascontiguousarray(row_order, dtype=np.int32)
    _check(lib.kpm_sell_build(n, _p(rp, _i64), _p(col, _i32), _p(val, _d), a, b, C, sigma,
                              _p(order, _i32) if order is not None else None, ctypes.byref(s)),
           "kpm_sell_build")
    g = Gather()
    try:
        sell = _sell_dict(s)
        _check(lib.kpm_gather_build(ctypes.byref(s), ctypes.byref(g)), "kpm_gather_build")
        try:
            gat = {
                "u_max": g.u_max, "l_max": g.l_max,
                "lidx": np.ctypeslib.as_array(g.lidx, (max(s.n_stored, 1),))[:s.n_stored].copy(),
                "run_ptr": np.ctypeslib.as_array(g.run_ptr, (g.n_chunks + 1,)).copy(),
                "runs": np.ctypeslib.as_array(g.runs, (max(2 * g.n_runs, 1),))[:2 * g.n_runs]
                .copy().reshape(-1, 2),
            }
        finally:
            lib.kpm_gather_release(ctypes.byref(g))
    finally:
        lib.kpm_sell_release(ctypes.byref(s))
    return sell, gat


STAGED_FP64, STAGED_FP32, STAGED_HALF, STAGED_HALF32 = 0, 1, 2, 3


def staged_build(csr, a, b, form, C=32, sigma=256, row_order=None):
    """The SELL layout (as sell_build), the gather lists (as gather_build) and
    the staged kernel's entry arrays of kpm_staged_build for `form` (0 complex
    double, 1 complex float, 2 half-complex double, 3 half-complex float):
    (sell, gather, staged) with staged = {"chunk_ptr", "chunk_len",
    "chunk_nre" (form 3, else None), "l_max", "lidx", "val"} -- val a
    complex numpy array for forms 0-2 (float values widened), the real
    float64 array of the stored floats for form 3."""
    n, rp, col, val = _csr(csr)
    s = Sell()
    order = None if row_order is None else np.ascontiguousarray(row_order, dtype=np.int32)
    _check(lib.kpm_sell_build(n, _p(rp, _i64), _p(col, _i32), _p(val, _d), a, b, C, sigma,
                              _p(order, _i32) if order is not None else None, ctypes.byref(s)),
           "kpm_sell_build")
    g = Gather()
    st = Staged()
    try:
        sell = _sell_dict(s)
        _check(lib.kpm_gather_build(ctypes.byref(s), ctypes.byref(g)), "kpm_gather_build")
        try:
            gat = {
                "u_max": g.u_max, "l_max": g.l_max,
                "lidx": np.ctypeslib.as_array(g.lidx, (max(s.n_stored, 1),))[:s.n_stored].copy(),
                "run_ptr": np.ctypeslib.as_array(g.run_ptr, (g.n_chunks + 1,)).copy(),
                "runs": np.ctypeslib.as_array(g.runs, (max(2 * g.n_runs, 1),))[:2 * g.n_runs]
                .copy().reshape(-1, 2),
            }
            _check(lib.kpm_staged_build(ctypes.byref(s), ctypes.byref(g), form, ctypes.byref(st)),
                   "kpm_staged_build")
            try:
                ns = st.n_stored
                if form == STAGED_HALF32:
                    v = np.ctypeslib.as_array(st.valf, (max(ns, 1),))[:ns].astype(np.float64)
                elif form == STAGED_FP32:
                    v = np.ctypeslib.as_array(st.valf, (max(2 * ns, 2),))[:2 * ns].copy()
                    v = v.astype(np.float64).view(np.complex128)
                else:
                    v = np.ctypeslib.as_array(st.val, (max(2 * ns, 2),))[:2 * ns].copy()
                    v = v.view(np.complex128)
                stg = {
                    "n_stored": ns, "l_max": st.l_max,
                    "chunk_ptr": np.ctypeslib.as_array(st.chunk_ptr, (st.n_chunks + 1,)).copy(),
                    "chunk_len": np.ctypeslib.as_array(st.chunk_len, (max(st.n_chunks, 1),))
                    [:st.n_chunks].copy(),
                    "chunk_nre": (np.ctypeslib.as_array(st.chunk_nre, (max(st.n_chunks, 1),))
                                  [:st.n_chunks].copy() if form == STAGED_HALF32 else None),
                    "lidx": np.ctypeslib.as_array(st.lidx, (max(ns, 1),))[:ns].copy(),
                    "val": v,
                }
            finally:
                lib.kpm_staged_release(ctypes.byref(st))
        finally:
            lib.kpm_gather_release(ctypes.byref(g))
    finally:
        lib.kpm_sell_release(ctypes.byref(s))
    return sell, gat, stg


def partition_rows(n, parts, align=1, weights=None):
    """kpm_partition_rows: int64[parts + 1] row boundaries."""
    out = np.empty(parts + 1, dtype=np.int64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    _check(lib.kpm_partition_rows(int(n), int(parts), _p(w, _d) if w is not None else None,
                                  int(align), _p(out, _i64)), "kpm_partition_rows")
    return out


def partition_build(csr, row_start, part):
    """kpm_partition_build: one part's local CSR (columns: local rows, then
    n_local + halo slot), its halo rows and its exchange lists, as numpy."""
    n, rp, col, val = _csr(csr)
    rs = np.ascontiguousarray(row_start, dtype=np.int64)
    P = Part()
    _check(lib.kpm_partition_build(n, _p(rp, _i64), _p(col, _i32), _p(val, _d), rs.size - 1,
                                   _p(rs, _i64), int(part), ctypes.byref(P)), "kpm_partition_build")
    try:
        nl, nh, nnz, npr = P.n_local, P.n_halo, P.nnz, P.n_peers

        def arr(ptr, count, dtype):
            return np.ctypeslib.as_array(ptr, (max(count, 1),))[:count].astype(dtype, copy=True)
        send_ptr = arr(P.send_ptr, npr + 1, np.int64)
        out = {
            "n": P.n, "row0": P.row0, "n_local": nl, "n_halo": nh, "part": int(part),
            "csr": {"n": nl, "row_ptr": arr(P.row_ptr, nl + 1, np.int64),
                    "col": arr(P.col, nnz, np.int32),
                    "val": arr(P.val_ri, 2 * nnz, np.float64).view(np.complex128)},
            "halo_rows": arr(P.halo_rows, nh, np.int64),
            "peer": arr(P.peer, npr, np.int32),
            "recv_ptr": arr(P.recv_ptr, npr + 1, np.int64),
            "send_ptr": send_ptr,
            "send_rows": arr(P.send_rows, int(send_ptr[-1]), np.int32),
        }
    finally:
        lib.kpm_partition_release(ctypes.byref(P))
    return out


def _sell_dict(s):
    return {
            "n": s.n, "n_pad": s.n_pad, "C": s.C, "sigma": s.sigma, "n_chunks": s.n_chunks,
            "nnz": s.nnz, "n_stored": s.n_stored,
            "chunk_ptr": np.ctypeslib.as_array(s.chunk_ptr, (s.n_chunks + 1,)).copy(),
            "chunk_len": np.ctypeslib.as_array(s.chunk_len, (max(s.n_chunks, 1),))[:s.n_chunks].copy(),
            "col": np.ctypeslib.as_array(s.col, (max(s.n_stored, 1),))[:s.n_stored].copy(),
            "val": np.ctypeslib.as_array(s.val_ri, (max(2 * s.n_stored, 2),))[:2 * s.n_stored]
            .copy().view(np.complex128),
            "perm": np.ctypeslib.as_array(s.perm, (s.n_pad,)).copy(),
    }


# ------------------------------------------------------------------- GPU
def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    if stream is None:
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class _TorchAllocator:
    """Device allocator hook backed by PyTorch's caching allocator."""

    def __init__(self, device):
        torch = _torch()
        self.device = device
        self.calls = 0  # allocations the library asked for

        def alloc(nbytes, user):
            self.calls += 1
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device)
            except Exception:  # noqa: BLE001 - reported to the library as NULL
                return None

        def free(ptr, user):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


class Context:
    """kpm_create / kpm_destroy around a Hermitian CSR matrix and (a, b)."""

    def __init__(self, csr, a, b, precision=PREC_FP64, chunk_height=32, sigma=256,
                 check_hermitian=False, device=0, torch_allocator=True, autotune=False,
                 row_order=None, n_halo=0, global_n=0, row0=0, allocator=None):
        """allocator: None, or an object with ctypes callbacks `alloc`
        (ALLOC_FN) and `free` (FREE_FN) for every device buffer of the
        context (kpm_options.alloc_fn / free_fn), used instead of torch's
        caching allocator; it must stay alive as long as the context."""
        n, rp, col, val = _csr(csr, n_cols=csr["n"] + n_halo)
        opt = default_options()
        opt.n_halo = n_halo
        opt.global_n = global_n
        opt.row0 = row0
        opt.precision = precision
        opt.chunk_height = chunk_height
        opt.sigma = sigma
        opt.check_hermitian = 1 if check_hermitian else 0
        opt.device = device
        opt.autotune = 1 if autotune else 0
        if row_order is not None:
            self._row_order = np.ascontiguousarray(row_order, dtype=np.int32)
            opt.row_order = _p(self._row_order, _i32)
        self._alloc = None
        if allocator is not None:
            self._alloc = allocator
        elif torch_allocator:
            self._alloc = _TorchAllocator(device)
        if self._alloc is not None:
            opt.alloc_fn = self._alloc.alloc
            opt.free_fn = self._alloc.free
        h = ctypes.c_void_p()
        _check(lib.kpm_create(n, _p(rp, _i64), _p(col, _i32), _p(val, _d), a, b, ctypes.byref(opt),
                              ctypes.byref(h)), "kpm_create")
        self.handle = h
        self.n = n
        self.a, self.b = a, b
        self.precision = precision

    def close(self):
        if getattr(self, "handle", None):
            lib.kpm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- queries
    def info(self):
        i = Info()
        _check(lib.kpm_get_info(self.handle, ctypes.byref(i)), "kpm_get_info")
        return {f: getattr(i, f) for f, _ in Info._fields_}

    def block_bytes(self, R):
        return int(lib.kpm_block_bytes(self.handle, R))

    def get_launch(self, R):
        l = Launch()
        _check(lib.kpm_get_launch(self.handle, R, ctypes.byref(l)), "kpm_get_launch")
        return {f: getattr(l, f) for f, _ in Launch._fields_}

    def set_launch(self, R, lanes_per_row, cols_per_lane, block_threads=256, blocks_per_sm=0,
                   tile_groups=0, stages=0):
        l = Launch(lanes_per_row, cols_per_lane, block_threads, blocks_per_sm, tile_groups, stages)
        _check(lib.kpm_set_launch(self.handle, R, ctypes.byref(l)), "kpm_set_launch")

    def max_block_width(self):
        """kpm_get_max_block_width: widest column block this context uses."""
        return lib.kpm_get_max_block_width(self.handle)

    def check_device_error(self):
        _check(lib.kpm_check_device_error(self.handle), "kpm_check_device_error")

    def test_stall_staged(self, chunks_per_block):
        _check(lib.kpm_test_stall_staged(self.handle, chunks_per_block), "kpm_test_stall_staged")

    def autotune(self, R, sweeps=5, stream=None):
        """kpm_autotune: returns the launch shape chosen for the widest block."""
        l = Launch()
        _check(lib.kpm_autotune(self.handle, R, sweeps, _stream_ptr(stream), ctypes.byref(l)),
               "kpm_autotune")
        out = {f: getattr(l, f) for f, _ in Launch._fields_}
        out["max_block_width"] = lib.kpm_get_max_block_width(self.handle)
        return out

    # -- host-buffer calls
    def moments(self, M, R, seed, imag=False, stream=None):
        eta = np.empty((R, M))
        eti = np.empty((R, M)) if imag else None
        _check(lib.kpm_moments(self.handle, M, R, seed, _p(eta, _d),
                               _p(eti, _d) if imag else None, _stream_ptr(stream)), "kpm_moments")
        return (eta, eti) if imag else eta

    def moments_v0(self, M, v0, imag=False, stream=None):
        v0 = np.ascontiguousarray(v0, dtype=np.complex128)
        R = v0.shape[1]
        eta = np.empty((R, M))
        eti = np.empty((R, M)) if imag else None
        _check(lib.kpm_moments_v0(self.handle, M, R, _p(v0.view(np.float64), _d), _p(eta, _d),
                                  _p(eti, _d) if imag else None, _stream_ptr(stream)),
               "kpm_moments_v0")
        return (eta, eti) if imag else eta

    def moments_local(self, M, rows, imag=False, stream=None):
        """kpm_moments_local: eta[R][M] of the unit vectors of `rows`."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        R = rows.size
        eta = np.empty((R, M))
        eti = np.empty((R, M)) if imag else None
        _check(lib.kpm_moments_local(self.handle, M, R, _p(rows, _i64), _p(eta, _d),
                                     _p(eti, _d) if imag else None, _stream_ptr(stream)),
               "kpm_moments_local")
        return (eta, eti) if imag else eta

    def moments_plane_wave(self, M, dims, norb, q, orb, imag=False, stream=None):
        """kpm_moments_plane_wave: eta[R][M] of the Bloch waves with wave
        vectors 2 pi q[r] (q: R x 3) on orbitals orb[r] of a dims lattice."""
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 3)
        orb = np.ascontiguousarray(orb, dtype=np.int32)
        R = q.shape[0]
        if orb.size != R:
            raise ValueError("one orbital per wave vector")
        eta = np.empty((R, M))
        eti = np.empty((R, M)) if imag else None
        nx, ny, nz = (int(d) for d in dims)
        _check(lib.kpm_moments_plane_wave(self.handle, M, R, nx, ny, nz, int(norb), _p(q, _d),
                                          _p(orb, _i32), _p(eta, _d),
                                          _p(eti, _d) if imag else None, _stream_ptr(stream)),
               "kpm_moments_plane_wave")
        return (eta, eti) if imag else eta

    # -- device-buffer calls (torch tensors)
    def halo_pack(self, R, V, rows_dev, buf, stream=None):
        """kpm_halo_pack: local rows rows_dev (device int32 tensor) of block V into buf."""
        _check(lib.kpm_halo_pack(self.handle, R, ctypes.c_void_p(V.data_ptr()),
                                 ctypes.c_void_p(rows_dev.data_ptr()), int(rows_dev.numel()),
                                 ctypes.c_void_p(buf.data_ptr()), _stream_ptr(stream)),
               "kpm_halo_pack")

    def halo_unpack(self, R, V, buf, first, count, stream=None):
        """kpm_halo_unpack: count rows of buf into halo slots first.. of block V."""
        _check(lib.kpm_halo_unpack(self.handle, R, ctypes.c_void_p(V.data_ptr()),
                                   ctypes.c_void_p(buf.data_ptr()), int(first), int(count),
                                   _stream_ptr(stream)), "kpm_halo_unpack")

    def block_phases(self, R, seed, V, stream=None):
        """kpm_block_phases: random-phase start block (by global row) into V."""
        _check(lib.kpm_block_phases(self.handle, R, seed, ctypes.c_void_p(V.data_ptr()),
                                    _stream_ptr(stream)), "kpm_block_phases")

    def new_block(self, R):
        torch = _torch()
        nbytes = self.block_bytes(R)
        return torch.zeros(nbytes, dtype=torch.uint8, device="cuda")

    def block_upload(self, R, host, dev, stream=None):
        host = np.ascontiguousarray(host, dtype=np.complex128)
        _check(lib.kpm_block_upload(self.handle, R, _p(host.view(np.float64), _d),
                                    ctypes.c_void_p(dev.data_ptr()), _stream_ptr(stream)),
               "kpm_block_upload")

    def block_download(self, R, dev, stream=None):
        out = np.empty((self.n, R), dtype=np.complex128)
        _check(lib.kpm_block_download(self.handle, R, ctypes.c_void_p(dev.data_ptr()),
                                      _p(out.view(np.float64), _d), _stream_ptr(stream)),
               "kpm_block_download")
        return out

    def aug_spmmv(self, R, V, W, eta_dev, init=False, with_imag=True, stream=None):
        eta_p = ctypes.c_void_p(eta_dev.data_ptr()) if eta_dev is not None else None
        _check(lib.kpm_aug_spmmv(self.handle, R, ctypes.c_void_p(V.data_ptr()),
                                 ctypes.c_void_p(W.data_ptr()), eta_p,
                                 1 if init else 0, 1 if with_imag else 0, _stream_ptr(stream)),
               "kpm_aug_spmmv")

    def aug_spmmv_static(self, R, V, W, eta_dev, init=False, with_imag=True, stream=None):
        """kpm_aug_spmmv_static: the sweep with its scratch in the library's
        fixed device array (no allocation inside the call)."""
        eta_p = ctypes.c_void_p(eta_dev.data_ptr()) if eta_dev is not None else None
        _check(lib.kpm_aug_spmmv_static(self.handle, R, ctypes.c_void_p(V.data_ptr()),
                                        ctypes.c_void_p(W.data_ptr()), eta_p, 1 if init else 0,
                                        1 if with_imag else 0, _stream_ptr(stream)),
               "kpm_aug_spmmv_static")

    def sweep_variant(self, R, V, W, variant, stream=None):
        """kpm_sweep_variant: 0 fully augmented, 1 without dots, 2 plain SpMMV."""
        _check(lib.kpm_sweep_variant(self.handle, R, ctypes.c_void_p(V.data_ptr()),
                                     ctypes.c_void_p(W.data_ptr()), variant, _stream_ptr(stream)),
               "kpm_sweep_variant")

    def set_reduce_interval(self, sweeps):
        _check(lib.kpm_set_reduce_interval(self.handle, sweeps), "kpm_set_reduce_interval")

    def test_corrupt_record(self, chunk, word, x, y):
        """kpm_test_corrupt_record (checked builds only)."""
        _check(lib.kpm_test_corrupt_record(self.handle, chunk, word, x, y),
               "kpm_test_corrupt_record")

    def set_sweep_overlap(self, mode):
        """kpm_set_sweep_overlap: OVERLAP_NONE (one plain launch per sweep)
        or OVERLAP_PDL (programmatic dependent launches, the default)."""
        _check(lib.kpm_set_sweep_overlap(self.handle, mode), "kpm_set_sweep_overlap")

    def moments_device(self, M, R, seed, eta_dev, eta_imag_dev=None, stream=None):
        _check(lib.kpm_moments_device(
            self.handle, M, R, seed, ctypes.c_void_p(eta_dev.data_ptr()),
            ctypes.c_void_p(eta_imag_dev.data_ptr()) if eta_imag_dev is not None else None,
            _stream_ptr(stream)), "kpm_moments_device")


def autotune_layout(csr, a, b, R, precision=PREC_FP64, sweeps=5, device=0):
    """kpm_autotune_layout: the fastest SELL (C, sigma) for width R, as
    {"chunk_height", "sigma", "ms_per_sweep"}."""
    n, rp, col, val = _csr(csr)
    base = default_options()
    base.precision = precision
    base.device = device
    best = Options()
    ms = _d()
    _check(lib.kpm_autotune_layout(n, _p(rp, _i64), _p(col, _i32), _p(val, _d), a, b,
                                   ctypes.byref(base), R, sweeps, ctypes.byref(best),
                                   ctypes.byref(ms)), "kpm_autotune_layout")
    return {"chunk_height": best.chunk_height, "sigma": best.sigma, "ms_per_sweep": ms.value}


class Naive:
    """kpm_naive_create / kpm_naive_moments / kpm_naive_destroy: the library-call
    KPM-DOS of Fig. 3 (ablation baseline)."""

    def __init__(self, csr, a, b, device=0):
        n, rp, col, val = _csr(csr)
        h = ctypes.c_void_p()
        _check(lib.kpm_naive_create(n, _p(rp, _i64), _p(col, _i32), _p(val, _d), a, b, device,
                                    ctypes.byref(h)), "kpm_naive_create")
        self.handle = h

    def moments_device(self, M, R, seed, eta_dev, stream=None):
        _check(lib.kpm_naive_moments(self.handle, M, R, seed, ctypes.c_void_p(eta_dev.data_ptr()),
                                     _stream_ptr(stream)), "kpm_naive_moments")

    def moments(self, M, R, seed):
        torch = _torch()
        eta = torch.empty((R, M), dtype=torch.float64, device="cuda")
        self.moments_device(M, R, seed, eta)
        torch.cuda.synchronize()
        return eta.cpu().numpy()

    def close(self):
        if getattr(self, "handle", None):
            lib.kpm_naive_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def create(csr, a, b, **kw):
    return Context(csr, a, b, **kw)


def moments_batch(ctxs, Ms, Rs, seeds, stream=None):
    """kpm_moments_batch: returns a list of eta arrays [R_p][M_p]."""
    count = len(ctxs)
    handles = (ctypes.c_void_p * count)(*[c.handle for c in ctxs])
    Ma = np.ascontiguousarray(Ms, dtype=np.int32)
    Ra = np.ascontiguousarray(Rs, dtype=np.int32)
    Sa = np.ascontiguousarray(seeds, dtype=np.uint64)
    etas = [np.empty((int(R), int(M))) for M, R in zip(Ms, Rs)]
    ptrs = (_pd * count)(*[_p(e, _d) for e in etas])
    _check(lib.kpm_moments_batch(handles, count, _p(Ma, _i32), _p(Ra, _i32),
                                 Sa.ctypes.data_as(ctypes.POINTER(_u64)), ptrs,
                                 _stream_ptr(stream)), "kpm_moments_batch")
    return etas


class Batch:
    """kpm_batch_create / kpm_batch_launch / kpm_batch_eta / kpm_batch_destroy."""

    def __init__(self, ctxs, Ms, Rs, seeds):
        self.count = len(ctxs)
        self.ctxs = list(ctxs)  # keep the contexts alive
        self.Ms = [int(m) for m in Ms]
        self.Rs = [int(r) for r in Rs]
        handles = (ctypes.c_void_p * self.count)(*[c.handle for c in ctxs])
        Ma = np.ascontiguousarray(Ms, dtype=np.int32)
        Ra = np.ascontiguousarray(Rs, dtype=np.int32)
        Sa = np.ascontiguousarray(seeds, dtype=np.uint64)
        h = ctypes.c_void_p()
        _check(lib.kpm_batch_create(handles, self.count, _p(Ma, _i32), _p(Ra, _i32),
                                    Sa.ctypes.data_as(ctypes.POINTER(_u64)), ctypes.byref(h)),
               "kpm_batch_create")
        self.handle = h

    def launch(self, stream=None):
        _check(lib.kpm_batch_launch(self.handle, _stream_ptr(stream)), "kpm_batch_launch")

    def eta(self, p, stream=None):
        out = np.empty((self.Rs[p], self.Ms[p]))
        _check(lib.kpm_batch_eta(self.handle, p, _p(out, _d), _stream_ptr(stream)), "kpm_batch_eta")
        return out

    def info(self):
        i = BatchInfo()
        _check(lib.kpm_batch_get_info(self.handle, ctypes.byref(i)), "kpm_batch_get_info")
        return {f: getattr(i, f) for f, _ in BatchInfo._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib.kpm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
