"""Python front end of the plain-C FP64 KPM oracle (kpm_oracle.c).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module.  It never touches the GPU library.

The shared object is compiled with gcc into oracle/_build/ on first use
(or by ``build()``).  Calls go through ctypes, which releases the GIL, so
``moments`` runs one start vector per thread in a thread pool -- the
C code itself stays single-threaded and plain.
"""
import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kpm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkpm_oracle.so")
_lib = None
_lock = threading.Lock()

_d = ctypes.c_double
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_pd = ctypes.POINTER(ctypes.c_double)
_pi32 = ctypes.POINTER(ctypes.c_int32)
_pi64 = ctypes.POINTER(ctypes.c_int64)

_SIGNATURES = {
    "oracle_uniform": (_d, [_u64, _u64, _u64]),
    "oracle_random_phase_vector": (ctypes.c_int, [_u64, _i64, _i64, _pd]),
    "oracle_gershgorin": (ctypes.c_int, [_i64, _pi64, _pi32, _pd, _pd, _pd]),
    "oracle_scale_from_bounds": (ctypes.c_int, [_d, _d, _d, _pd, _pd]),
    "oracle_aug_spmv": (ctypes.c_int, [_i64, _pi64, _pi32, _pd, _d, _d, _pd, _pd, _pd]),
    "oracle_kpm_vector": (ctypes.c_int, [_i64, _pi64, _pi32, _pd, _d, _d, _i32, _pd, _pd, _pd]),
    "oracle_kpm_random_vector": (ctypes.c_int, [_i64, _pi64, _pi32, _pd, _d, _d, _i32, _u64, _i64,
                                                _pd, _pd]),
    "oracle_eta_to_mu": (ctypes.c_int, [_pd, _i32, _i32, _pd]),
    "oracle_jackson": (ctypes.c_int, [_i32, _pd]),
    "oracle_dos": (ctypes.c_int, [_pd, _i32, _i32, _d, _d, _pd, _pd]),
}


def build(force=False):
    """Compile kpm_oracle.c into oracle/_build/libkpm_oracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = ctypes.CDLL(build())
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(so, name)
                f.restype = res
                f.argtypes = args
            _lib = so
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _csr_args(csr):
    rp = np.ascontiguousarray(csr["row_ptr"], dtype=np.int64)
    col = np.ascontiguousarray(csr["col"], dtype=np.int32)
    vri = np.ascontiguousarray(csr["val"], dtype=np.complex128).view(np.float64)
    return rp, col, vri


def _check(rc, what):
    if rc != 0:
        raise ValueError("%s failed with status %d" % (what, rc))


def uniform(seed, stream, index):
    return lib().oracle_uniform(seed, stream, index)


def random_phase_vector(seed, n, r):
    out = np.empty(2 * n, dtype=np.float64)
    _check(lib().oracle_random_phase_vector(seed, n, r, _ptr(out, _d)), "random_phase_vector")
    return out.view(np.complex128)


def gershgorin(csr):
    rp, col, vri = _csr_args(csr)
    lo, hi = _d(), _d()
    _check(lib().oracle_gershgorin(csr["n"], _ptr(rp, _i64), _ptr(col, _i32), _ptr(vri, _d),
                                   ctypes.byref(lo), ctypes.byref(hi)), "gershgorin")
    return lo.value, hi.value


def scale_from_bounds(emin, emax, eps=0.01):
    a, b = _d(), _d()
    _check(lib().oracle_scale_from_bounds(emin, emax, eps, ctypes.byref(a), ctypes.byref(b)),
           "scale_from_bounds")
    return a.value, b.value


def aug_spmv(csr, a, b, v, w):
    """One fused step on single vectors: returns (w_new, [<v|v>, Re<w|v>, Im<w|v>])."""
    rp, col, vri = _csr_args(csr)
    v = np.ascontiguousarray(v, dtype=np.complex128).view(np.float64)
    w = np.array(w, dtype=np.complex128).view(np.float64)
    eta = np.empty(3, dtype=np.float64)
    _check(lib().oracle_aug_spmv(csr["n"], _ptr(rp, _i64), _ptr(col, _i32), _ptr(vri, _d), a, b,
                                 _ptr(v, _d), _ptr(w, _d), _ptr(eta, _d)), "aug_spmv")
    return w.view(np.complex128), eta


def kpm_vector(csr, a, b, M, v0):
    """eta_0..eta_{M-1} (real, imag) for one explicit start vector."""
    rp, col, vri = _csr_args(csr)
    v0 = np.ascontiguousarray(v0, dtype=np.complex128).view(np.float64)
    er = np.empty(M, dtype=np.float64)
    ei = np.empty(M, dtype=np.float64)
    _check(lib().oracle_kpm_vector(csr["n"], _ptr(rp, _i64), _ptr(col, _i32), _ptr(vri, _d), a, b,
                                   M, _ptr(v0, _d), _ptr(er, _d), _ptr(ei, _d)), "kpm_vector")
    return er, ei


def _pool_size(jobs, threads):
    if threads is None:
        threads = os.cpu_count() or 1
    return max(1, min(int(threads), jobs))


def moments(csr, a, b, M, seed, cols, threads=None):
    """eta for random-phase vectors ``cols`` drawn from ``seed``: (re[R][M], im[R][M])."""
    rp, col, vri = _csr_args(csr)
    cols = list(cols)
    er = np.empty((len(cols), M), dtype=np.float64)
    ei = np.empty((len(cols), M), dtype=np.float64)
    L = lib()

    def one(k):
        rc = L.oracle_kpm_random_vector(csr["n"], _ptr(rp, _i64), _ptr(col, _i32), _ptr(vri, _d),
                                        a, b, M, seed, cols[k], _ptr(er[k], _d), _ptr(ei[k], _d))
        _check(rc, "kpm_random_vector")

    with ThreadPoolExecutor(_pool_size(len(cols), threads)) as ex:
        list(ex.map(one, range(len(cols))))
    return er, ei


def moments_v0(csr, a, b, M, v0_block, threads=None):
    """eta for the columns of an explicit start block v0_block[n][R]."""
    v0_block = np.asarray(v0_block, dtype=np.complex128)
    R = v0_block.shape[1]
    er = np.empty((R, M), dtype=np.float64)
    ei = np.empty((R, M), dtype=np.float64)

    def one(k):
        er[k], ei[k] = kpm_vector(csr, a, b, M, np.ascontiguousarray(v0_block[:, k]))

    with ThreadPoolExecutor(_pool_size(R, threads)) as ex:
        list(ex.map(one, range(R)))
    return er, ei


def eta_to_mu(eta):
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    R, M = eta.shape
    mu = np.empty(M, dtype=np.float64)
    _check(lib().oracle_eta_to_mu(_ptr(eta, _d), M, R, _ptr(mu, _d)), "eta_to_mu")
    return mu


def jackson(M):
    g = np.empty(M, dtype=np.float64)
    _check(lib().oracle_jackson(M, _ptr(g, _d)), "jackson")
    return g


def dos(mu, K, a, b):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    e = np.empty(K, dtype=np.float64)
    rho = np.empty(K, dtype=np.float64)
    _check(lib().oracle_dos(_ptr(mu, _d), mu.size, K, a, b, _ptr(e, _d), _ptr(rho, _d)), "dos")
    return e, rho
